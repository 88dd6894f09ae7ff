"""Torch-facing wrapper of the C ABI: device tensors in, device tensors updated in place.

PyTorch provides device memory and the stream; every step of the iteration
runs in libptycho.so. Inputs on the host, or a missing CUDA device, raise.
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import torch

from .binding import BatchPlan, Plan, monochromatise_raw


def _require_cuda(t: torch.Tensor, name: str, dtype: torch.dtype):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Reconstruction:
    """A plan bound to a torch stream.

    params: dict with the fields of ptycho_params (see include/ptycho.h).
    intensities: (N, M, M) float32 CUDA tensor.
    positions: (N, 2) int32 tensor (CPU or CUDA) or numpy array of (row, col) top-left corners.
    """

    def __init__(self, params: dict, intensities: torch.Tensor, positions, stream: Optional[torch.cuda.Stream] = None):
        _require_cuda(intensities, "intensities", torch.float32)
        if isinstance(positions, np.ndarray):
            positions = torch.from_numpy(np.ascontiguousarray(positions, dtype=np.int32))
        positions = positions.to(torch.int32).contiguous()
        self.params = dict(params)
        self.stream = stream if stream is not None else torch.cuda.current_stream(intensities.device)
        self._positions = positions  # keep alive across the plan call
        self._plan = Plan(self.params, intensities.data_ptr(), positions.data_ptr(), self.stream.cuda_stream)

    def iterate(self, obj: torch.Tensor, probe: torch.Tensor, n_iter: int = 1):
        _require_cuda(obj, "object", torch.complex64)
        _require_cuda(probe, "probe", torch.complex64)
        self._plan.iterate(obj.data_ptr(), probe.data_ptr(), n_iter)

    def error(self) -> float:
        return self._plan.error()

    def errors(self, n: int) -> list:
        return self._plan.error_history(n)

    def profile(self, enable: bool = True):
        self._plan.profile(enable)

    def profile_read(self) -> tuple:
        return self._plan.profile_read()

    def launches_per_iteration(self, in_window: bool) -> int:
        return self._plan.launches_per_iteration(in_window)

    def staged_chunk(self) -> int:
        """Positions per chunk of the staged M = 256 passes (0 for M <= 128)."""
        return self._plan.staged_chunk()

    def close(self):
        self._plan.close()


class ReconstructionBatch:
    """Independent reconstructions of uneven sizes, iterated together as one CUDA graph per iteration.

    problems: sequence of (params dict, intensities CUDA tensor, positions) as for Reconstruction.
    """

    def __init__(self, problems, stream: Optional[torch.cuda.Stream] = None):
        self._pos = []
        iptr, pptr, params = [], [], []
        for prm, I, pos in problems:
            _require_cuda(I, "intensities", torch.float32)
            if isinstance(pos, np.ndarray):
                pos = torch.from_numpy(np.ascontiguousarray(pos, dtype=np.int32))
            pos = pos.to(torch.int32).contiguous()
            self._pos.append(pos)
            params.append(dict(prm))
            iptr.append(I.data_ptr())
            pptr.append(pos.data_ptr())
        dev = problems[0][1].device
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self._plan = BatchPlan(params, iptr, pptr, self.stream.cuda_stream)

    def iterate(self, objects, probes, n_iter: int = 1):
        for o in objects:
            _require_cuda(o, "object", torch.complex64)
        for p in probes:
            _require_cuda(p, "probe", torch.complex64)
        self._plan.iterate([o.data_ptr() for o in objects], [p.data_ptr() for p in probes], n_iter)

    def errors(self) -> list:
        return self._plan.errors()

    def classes(self) -> list:
        """The work-queue classes of this batch (shape, members, tuned chunk length, ...)."""
        return self._plan.classes()

    def launches_per_iteration(self) -> int:
        """Kernel launches of one iteration (kernel nodes of the last replayed graph)."""
        return self._plan.launches_per_iteration()

    def close(self):
        self._plan.close()


def monochromatise(b: torch.Tensor, scales, weights, k: int, clamp: bool = False, out: Optional[torch.Tensor] = None,
                   with_residuals: bool = False, stream: Optional[torch.cuda.Stream] = None):
    """Numerical monochromatisation (Sec. 4.2, Eqs. 12-13) of broadband patterns b ((N, M, M) float32 CUDA,
    detector-centred): k CGLS steps per pattern on min ||C x - b|| with C the spectrum operator of
    relative wavelengths `scales` (a_j = lambda_j / lambda_c) and `weights`. Returns x (or out), and
    with_residuals the (N, k + 1) float64 residual norms as well. Enqueued on `stream`."""
    _require_cuda(b, "b", torch.float32)
    if b.dim() != 3 or b.shape[1] != b.shape[2]:
        raise ValueError("b must be (N, M, M)")
    x = out if out is not None else torch.empty_like(b)
    _require_cuda(x, "out", torch.float32)
    if x.shape != b.shape:
        raise ValueError("out must have the shape of b")
    N, M = b.shape[0], b.shape[1]
    res = torch.empty((N, k + 1), dtype=torch.float64, device=b.device) if with_residuals else None
    st = stream if stream is not None else torch.cuda.current_stream(b.device)
    monochromatise_raw(M, scales, weights, N, k, b.data_ptr(), x.data_ptr(), res.data_ptr() if res is not None else 0,
                       clamp, st.cuda_stream)
    return (x, res) if with_residuals else x
