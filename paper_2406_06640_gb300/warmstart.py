"""Learned warm start: train the U-Net on forward-model patterns, then estimate the object and sigma.

The paper has no learned component; it reconstructs the source's partial coherence
without prior knowledge of it. This module adds a start point for that
reconstruction: a network trained only on patterns that the library's own forward
model generates on the GPU (random hexagonal crystals seen through the measured
probe, blurred by Eq. 2 with sigma drawn uniformly, Poisson counts at the
measurement's dose) predicts, from each measured pattern, the object's central
box and the blur width. The stitched boxes and the median sigma then seed the
engine in place of a flat object and an assumed sigma.

Every step (data generation, forward, backward, Adam, inference, stitch, median)
runs in libptycho.so; this module draws the per-pattern lattice parameters with
numpy and marshals device pointers.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import binding as _b


@dataclass
class LatticeSpec:
    """Training crystals: lattice constant, peak phase and width in pixels / radians."""

    a: float = 16.0
    peak: float = 0.1
    peak_sd: float = 1.5
    cutoff: float = 6.0
    vacancy: float = 0.05


@dataclass
class WarmStartConfig:
    S: int = 128                 # pattern side (the engine's M)
    C: int = 32                  # base channel count
    batch: int = 64
    dose: float = 200.0          # counts per training pattern (the measurement's dose)
    sigma_range: tuple = (0.5, 3.0)
    target_scale: float = 0.1    # network outputs are (ln|o|, arg o) / target_scale
    lam: float = 0.1             # weight of the sigma term of the loss
    lattice: LatticeSpec = field(default_factory=LatticeSpec)
    seed: int = 0


def subsample_scan(positions: np.ndarray, spacing: float) -> np.ndarray:
    """Indices of a subset of scan positions at least `spacing` px apart (greedy, in scan order)."""
    pos = np.asarray(positions, dtype=np.float64)
    keep = []
    for i, p in enumerate(pos):
        if all(np.max(np.abs(p - pos[j])) >= spacing for j in keep):
            keep.append(i)
    return np.asarray(keep, dtype=np.int64)


class WarmStart:
    """The network plus its training-data generator for one probe.

    probe: torch complex64 (S, S) tensor on the CUDA device (the nominal probe the
    engine starts from; its scale does not matter).
    """

    def __init__(self, probe, cfg: Optional[WarmStartConfig] = None, stream_ptr: int = 0):
        import torch

        self.cfg = cfg or WarmStartConfig()
        c = self.cfg
        if probe.shape != (c.S, c.S):
            raise ValueError(f"probe must be {c.S} x {c.S}")
        self._torch = torch
        self.device = probe.device
        self._probe = torch.view_as_real(probe.to(torch.complex64).contiguous()).contiguous()
        self.net = _b.UNet(c.S, c.C, c.batch, seed=c.seed, stream_ptr=stream_ptr)
        self._stream = stream_ptr
        self._rng = np.random.default_rng(np.random.SeedSequence(c.seed).spawn(2)[1])
        self._samples = 0
        B, S = c.batch, c.S
        self._x = torch.zeros(B, S, S, device=self.device)
        self._target = torch.zeros(B, S // 2, S // 2, 2, device=self.device)
        self._sigma = torch.zeros(B, device=self.device)
        self._params = torch.zeros(B, 4, device=self.device)
        self._gen = dict(S=S, noise=1, dose=c.dose, lattice_a=c.lattice.a, peak=c.lattice.peak,
                         peak_sd=c.lattice.peak_sd, cutoff=c.lattice.cutoff, vacancy=c.lattice.vacancy,
                         target_scale=c.target_scale, key=(c.seed * 0x9E3779B97F4A7C15 + 1) & ((1 << 64) - 1))

    def _draw(self):
        c, B = self.cfg, self.cfg.batch
        r = self._rng
        p = np.stack([r.uniform(0, math.pi / 3, B), r.uniform(0, c.lattice.a, B), r.uniform(0, c.lattice.a, B),
                      r.uniform(c.sigma_range[0], c.sigma_range[1], B)], axis=1).astype(np.float32)
        self._params.copy_(self._torch.from_numpy(p))

    def generate_batch(self):
        """One batch of forward-model patterns into the internal buffers."""
        self._draw()
        _b.generate(self._gen, self._probe.data_ptr(), self._params.data_ptr(), self.cfg.batch, self._samples,
                    x=self._x.data_ptr(), target=self._target.data_ptr(), sigma=self._sigma.data_ptr(),
                    stream_ptr=self._stream)
        self._samples += self.cfg.batch

    def train(self, n_patterns: int, lr: float = 1e-3, lr_final: float = 5e-5, log_every: int = 0) -> list:
        """Adam over ceil(n_patterns / batch) fresh batches, cosine learning-rate decay; returns [(step, loss)]."""
        steps = max(1, -(-n_patterns // self.cfg.batch))
        log = []
        for s in range(steps):
            cur = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * s / max(steps - 1, 1)))
            self.generate_batch()
            want = bool(log_every) and (s % log_every == 0 or s == steps - 1)
            loss = self.net.train_step(self._x.data_ptr(), self._target.data_ptr(), self._sigma.data_ptr(),
                                       self.cfg.lam, cur, want_loss=want)
            if want:
                log.append((s, loss))
        return log

    def estimate(self, intensities, positions: np.ndarray, obj_h: int, obj_w: int):
        """Object estimate (torch complex64, obj_h x obj_w) and median sigma from N measured patterns.

        intensities: torch float32 (N, S, S) on the device (counts, detector-centred);
        positions: (N, 2) int32 box corners of those patterns."""
        torch = self._torch
        pos = np.ascontiguousarray(positions, dtype=np.int32)
        O = torch.empty(obj_h, obj_w, 2, device=self.device)
        I = intensities.contiguous()
        sigma = self.net.warmstart(I.data_ptr(), pos.ctypes.data, pos.shape[0], obj_h, obj_w,
                                   self.cfg.target_scale, O.data_ptr())
        return torch.view_as_complex(O), sigma

    def close(self):
        self.net.close()


def eval_kernel_size(sigma: float) -> int:
    """Odd kernel side covering +-min(ceil(5 sigma), 15) taps (the simulator's truncation)."""
    return 2 * min(int(math.ceil(5.0 * max(sigma, 0.0))), 15) + 1


def time_to_nrmse(params: dict, intensities, clean, positions, obj, probe, sigma_eval: float,
                  target: float = 0.05, max_iter: int = 100) -> dict:
    """Iterate one engine iteration at a time until the intensity NRMSE against the noise-free
    patterns, sqrt(sum (Ihat - I_clean)^2 / sum I_clean^2) with Ihat = (sum_k |Psi_k|^2) (x) g of
    width sigma_eval (Eq. 2), reaches `target`. Evaluation runs on copies through a second plan
    and is not timed; the engine's device time per iteration is (CUDA events on its stream).
    For synthetic data whose noise-free intensities are known. obj / probe are updated in place.
    Returns dict(iterations, engine_ms, reached, curve=[(iteration, nrmse)])."""
    import torch

    from .engine import Reconstruction

    ev_params = dict(params, blur_domain="intensity", sigma1=sigma_eval, sigma2=sigma_eval,
                     kernel_size=eval_kernel_size(sigma_eval), probe_update_start=1 << 30, windows=[],
                     start_iteration=1)
    ev = Reconstruction(ev_params, clean, positions)
    rec = Reconstruction(params, intensities, positions)

    def nrmse():
        o, p = obj.clone(), probe.clone()
        ev.iterate(o, p, 1)
        return ev.error()

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    curve = [(0, nrmse())]
    ms, it = 0.0, 0
    while curve[-1][1] > target and it < max_iter:
        e0.record(rec.stream)
        rec.iterate(obj, probe, 1)
        e1.record(rec.stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        it += 1
        curve.append((it, nrmse()))
    rec.close()
    ev.close()
    return dict(iterations=it, engine_ms=ms, reached=curve[-1][1] <= target, curve=curve)


def time_to_nrmse_batch(members, target: float = 0.05, max_iter: int = 100) -> dict:
    """time_to_nrmse for several reconstructions iterated together as one batch plan (one CUDA
    graph launch per iteration, one persistent work-queue launch per shape class).

    members: sequence of dict(params, intensities, clean, positions, obj, probe, sigma_eval) as the
    arguments of time_to_nrmse. The batch iterates until every member's intensity NRMSE against its
    noise-free patterns reaches `target` (members that got there keep iterating with the others).
    The evaluation runs on copies through one plan per member and is not timed; the batch's device
    time per iteration is (CUDA events on its stream). Returns dict(iterations, engine_ms, reached,
    curves=[[(iteration, nrmse)] per member])."""
    import torch

    from .engine import Reconstruction, ReconstructionBatch

    evs = []
    for m in members:
        s = m["sigma_eval"]
        ev_params = dict(m["params"], blur_domain="intensity", sigma1=s, sigma2=s, kernel_size=eval_kernel_size(s),
                         probe_update_start=1 << 30, windows=[], start_iteration=1)
        evs.append(Reconstruction(ev_params, m["clean"], m["positions"]))
    batch = ReconstructionBatch([(m["params"], m["intensities"], m["positions"]) for m in members])
    objs, prbs = [m["obj"] for m in members], [m["probe"] for m in members]

    def nrmse():
        out = []
        for ev, o, p in zip(evs, objs, prbs):
            oc, pc = o.clone(), p.clone()
            ev.iterate(oc, pc, 1)
            out.append(ev.error())
        return out

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    curves = [[(0, e)] for e in nrmse()]
    ms, it = 0.0, 0
    while max(c[-1][1] for c in curves) > target and it < max_iter:
        e0.record(batch.stream)
        batch.iterate(objs, prbs, 1)
        e1.record(batch.stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        it += 1
        for c, e in zip(curves, nrmse()):
            c.append((it, e))
    batch.close()
    for ev in evs:
        ev.close()
    return dict(iterations=it, engine_ms=ms, reached=max(c[-1][1] for c in curves) <= target, curves=curves)
