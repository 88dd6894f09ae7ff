"""FP64 CPU oracle of one data-parallel pc-engine iteration.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU-baseline
leg of the benchmark may import this module. The product path never calls it.

It is written from the paper (arXiv 2406.06640, "A high-performance
reconstruction method for partially coherent ptychography"), step by step and
in the paper's order, with numpy.fft / scipy.signal as library primitives.
It shares no code with the CUDA path.

Per iteration t (1-based), with every position using the same O and P:

  for each position n (any order; the update is simultaneous):
    o_n      = O[y_n:y_n+M, x_n:x_n+M]                 Fig. 1: object box
    psi_k    = P_k o_n                                   Eq. 1, mixed-state modes k
    Psi_k    = forward propagation of psi_k              Eq. 1 (far: centred FFT;
                                                         near: Fresnel transfer function)
    amplitude mode (Eq. 6, default):
      A      = sqrt(sum_k |Psi_k|^2);  A^G = A (x) g      Eqs. 6-7
      Ihat   = (A^G)^2;  R = sqrt(I_n) / (A^G + eps)      Fig. 1 box 1
    intensity mode (Eq. 2):
      I_m    = (sum_k |Psi_k|^2) (x) g;  Ihat = I_m;  R = sqrt(I_n) / sqrt(I_m + eps^2)
    Psi'_k   = R Psi_k;  psi'_k = back-propagation;  dpsi_k = psi'_k - psi_k
    N_O[box] += sum_k conj(P_k) dpsi_k;   D_O[box] += sum_k |P_k|^2
    N_P[k]   += conj(o_n) dpsi_k;         D_P      += |o_n|^2
    errnum   += sum (Ihat - I_n)^2;       errden   += sum I_n^2
  O   += beta_O N_O / (D_O + delta_O max D_O)       (pixels with D_O = 0 unchanged)
  P_k += beta_P N_P[k] / (D_P + delta_P max D_P)     (t >= probe_update_start)
  if t lies in a complex-constraint window: Eqs. 9-11 on the new O
  E_t = sqrt(errnum / errden)                         NRMSE of Sec. 4.2 (state before the update)

Readings of passages that the paper leaves open (kept identical on the GPU):
  * blur domain: amplitude (Eq. 6) by default, intensity (Eq. 2) as a flag;
  * modulus: Psi' = Psi sqrt(I) / A^G (the formula sits in the Fig. 1 box 1 image);
  * g: Eq. 7 normalised to sum 1 over the size x size support, x = column
    (sigma_1), y = row (sigma_2), zero padding, sigma = 0 gives a delta;
  * eps = 1e-6 sqrt(mean I) unless given; amplitude floor a_min = 1e-6 and a
    floor of 1e-30 on sum |phi| in Eq. 11;
  * the simultaneous (Jacobi) update above, beta = 1, delta = 1e-3;
  * the complex constraint acts on the whole updated object: C_n of Eq. 11
    per box, clamped to [cbar_min, cbar_max] (Sec. 4.8), averaged over the
    boxes that cover a pixel, then Eqs. 9-10; uncovered pixels are unchanged;
  * phase = angle() in (-pi, pi], no unwrapping; windows are 1-based inclusive;
  * pc-DM (iteration_dm): the constraint acts between the object and the probe
    steps and moves each exit-wave state with its box.

Parity unpinned (only oracle <-> GPU agreement fixes them; no passage of the
paper does): the constants beta, delta, eps and the clamp range, the per-pixel
mean of C_n, and where pc-DM applies the complex constraint.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Sequence

import numpy as np
from scipy import signal

from . import philox

A_MIN = 1e-6
PHI_FLOOR = 1e-30


@dataclasses.dataclass
class Params:
    M: int
    K: int
    N: int
    obj_h: int
    obj_w: int
    geometry: str = "far"  # "far" | "near"
    blur_domain: str = "amplitude"  # "amplitude" (Eq. 6) | "intensity" (Eq. 2)
    fresnel_F: float = 0.0
    sigma1: float = 1.0
    sigma2: float = 1.0
    kernel_size: int = 11
    eps_mod: float = 0.0  # 0 => 1e-6 sqrt(mean I)
    beta_obj: float = 1.0
    beta_probe: float = 1.0
    delta_obj: float = 1e-3
    delta_probe: float = 1e-3
    probe_update_start: int = 1
    alpha1: float = 1.0
    alpha2: float = 0.0
    cbar_min: float = 0.01
    cbar_max: float = 10.0
    windows: Sequence = ()
    start_iteration: int = 1
    step_rule: str = "normalised"  # "normalised" | "rpie"
    rpie_alpha_obj: float = 0.0
    rpie_alpha_probe: float = 0.0
    engine: str = "pie"  # "pie": the step of reading 4 / 10b / 10c; "dm": pc-DM (reading 10d)
    minibatch: int = 0  # 0: every position in one simultaneous step; B >= 1: batches of B positions
    order_seed: int = 0  # key of the batch partition and of each iteration's visiting order

    @classmethod
    def from_dict(cls, d):
        names = {f.name for f in dataclasses.fields(cls)}
        return cls(**{k: v for k, v in d.items() if k in names})


# ----------------------------------------------------------------------------------------
# Eq. 7: the Gaussian kernel
# ----------------------------------------------------------------------------------------

def gaussian_kernel(size: int, sigma1: float, sigma2: float) -> np.ndarray:
    """g[i, j] = exp(-(j^2 / (2 s1^2) + i^2 / (2 s2^2))), i = row offset, j = column offset (Eq. 7).

    Normalised to sum 1 over the support (Sec. 2 calls g normalised). A zero
    sigma makes that axis a delta.
    """
    h = (size - 1) // 2
    off = np.arange(-h, h + 1, dtype=np.float64)
    gx = np.exp(-off ** 2 / (2.0 * sigma1 ** 2)) if sigma1 > 0 else (off == 0).astype(np.float64)
    gy = np.exp(-off ** 2 / (2.0 * sigma2 ** 2)) if sigma2 > 0 else (off == 0).astype(np.float64)
    g = gy[:, None] * gx[None, :]
    return g / g.sum()


def blur(img: np.ndarray, g: np.ndarray) -> np.ndarray:
    """A (x) g with zero padding, output the size of the input (Eqs. 2 and 6)."""
    return signal.correlate2d(img, g, mode="same", boundary="fill", fillvalue=0.0)


# ----------------------------------------------------------------------------------------
# propagation (Eq. 1; near field: Fresnel transfer function)
# ----------------------------------------------------------------------------------------

def fresnel_tf(M: int, F: float) -> np.ndarray:
    """H[u, v] = exp(-i pi (u^2 + v^2) / (M F)), u, v the signed integer frequencies."""
    u = np.fft.fftfreq(M) * M
    return np.exp(-1j * np.pi * (u[:, None] ** 2 + u[None, :] ** 2) / (M * F))


def propagate_forward(psi: np.ndarray, prm: Params) -> np.ndarray:
    if prm.geometry == "far":
        return np.fft.fftshift(np.fft.fft2(psi), axes=(-2, -1))
    H = fresnel_tf(prm.M, prm.fresnel_F)
    return np.fft.ifft2(np.fft.fft2(psi) * H)


def propagate_backward(Psi: np.ndarray, prm: Params) -> np.ndarray:
    if prm.geometry == "far":
        return np.fft.ifft2(np.fft.ifftshift(Psi, axes=(-2, -1)))
    H = fresnel_tf(prm.M, prm.fresnel_F)
    return np.fft.ifft2(np.fft.fft2(Psi) * np.conj(H))


# ----------------------------------------------------------------------------------------
# Fig. 1 box 1: partial-coherence intensity model and modulus constraint
# ----------------------------------------------------------------------------------------

def default_eps(I: np.ndarray) -> float:
    return 1e-6 * math.sqrt(math.fsum(np.asarray(I, dtype=np.float64).ravel()) / I.size)


def modulus(Psi: np.ndarray, I_n: np.ndarray, g: np.ndarray, eps: float, blur_domain: str):
    """Returns (Psi', Ihat) for one position; Psi has shape (K, M, M)."""
    S = np.sum(np.abs(Psi) ** 2, axis=0)
    if blur_domain == "amplitude":
        AG = blur(np.sqrt(S), g)
        Ihat = AG ** 2
        R = np.sqrt(I_n) / (AG + eps)
    else:
        Im = blur(S, g)
        Ihat = Im
        R = np.sqrt(I_n) / np.sqrt(Im + eps * eps)
    return R[None] * Psi, Ihat


# ----------------------------------------------------------------------------------------
# Eqs. 9-11: complex constraint on the updated object
# ----------------------------------------------------------------------------------------

def cbar_per_position(O: np.ndarray, positions: np.ndarray, M: int, cmin: float, cmax: float) -> np.ndarray:
    """C_n = sum_box |ln A| / sum_box |phi| (Eq. 11), clamped to [cmin, cmax] (Sec. 4.8)."""
    a = np.maximum(np.abs(O), A_MIN)
    lna = np.log(a)
    phi = np.angle(O)
    out = np.empty(len(positions))
    for n, (y, x) in enumerate(positions):
        num = np.sum(np.abs(lna[y:y + M, x:x + M]))
        den = max(np.sum(np.abs(phi[y:y + M, x:x + M])), PHI_FLOOR)
        out[n] = min(max(num / den, cmin), cmax)
    return out


def complex_constraint(O: np.ndarray, positions: np.ndarray, prm: Params) -> np.ndarray:
    M = prm.M
    cb = cbar_per_position(O, positions, M, prm.cbar_min, prm.cbar_max)
    csum = np.zeros(O.shape)
    cnt = np.zeros(O.shape)
    for n, (y, x) in enumerate(positions):
        csum[y:y + M, x:x + M] += cb[n]
        cnt[y:y + M, x:x + M] += 1.0
    covered = cnt > 0
    C = np.where(covered, csum / np.maximum(cnt, 1.0), 1.0)
    a = np.maximum(np.abs(O), A_MIN)
    lna = np.log(a)
    phi = np.angle(O)
    a_c = np.exp((1.0 - prm.alpha1) * lna + prm.alpha1 * C * phi)  # Eq. 9
    phi_c = (1.0 - prm.alpha2) * phi + prm.alpha2 * lna / C  # Eq. 10
    return np.where(covered, a_c * np.exp(1j * phi_c), O)


def in_window(t: int, windows) -> bool:
    return any(lo <= t <= hi for (lo, hi) in windows)


# ----------------------------------------------------------------------------------------
# one iteration and the iteration loop
# ----------------------------------------------------------------------------------------

def _normalised_step(beta, num, den, c_den, c_max):
    """beta num / (c_den den + c_max max den); pixels that no box reaches (den = 0) get no step.

    The normalised rule (reading 4) is (c_den, c_max) = (1, delta). The rPIE family (Sec. 5,
    Fig. 11c) regularises the denominator as (1 - alpha) den + alpha max den, i.e.
    (c_den, c_max) = (1 - alpha, alpha); alpha = 1 gives the ePIE-style max-normalised step."""
    out = np.zeros(num.shape, np.complex128)
    reached = den > 0
    out[reached] = beta * num[reached] / (c_den * den[reached] + c_max * den.max())
    return out


def step_coefficients(prm: "Params"):
    """(c_den, c_max) of the object step and of the probe step."""
    if prm.step_rule == "rpie":
        return (1.0 - prm.rpie_alpha_obj, prm.rpie_alpha_obj), (1.0 - prm.rpie_alpha_probe, prm.rpie_alpha_probe)
    if prm.step_rule != "normalised":
        raise ValueError(f"unknown step rule {prm.step_rule!r}")
    return (1.0, prm.delta_obj), (1.0, prm.delta_probe)


def _batch_step(I, positions, idx, O, P, prm: Params, t: int, eps: float, g):
    """The simultaneous normalised step over the positions idx (Fig. 1 boxes 1 and 2 for each,
    then one update of O and P from the old O and P). Returns (O_new, P_new, [error numerators])."""
    M, K = prm.M, prm.K
    NO = np.zeros(O.shape, np.complex128)
    DO = np.zeros(O.shape, np.float64)
    NP = np.zeros(P.shape, np.complex128)
    DP = np.zeros((M, M), np.float64)
    P2 = np.sum(np.abs(P) ** 2, axis=0)
    errnum = []
    for n in idx:
        y, x = positions[n]
        o = O[y:y + M, x:x + M]
        psi = P * o[None]
        Psi = propagate_forward(psi, prm)
        In = I[n].astype(np.float64)
        Psi_new, Ihat = modulus(Psi, In, g, eps, prm.blur_domain)
        errnum.append(math.fsum(((Ihat - In) ** 2).ravel()))
        dpsi = propagate_backward(Psi_new, prm) - psi
        NO[y:y + M, x:x + M] += np.sum(np.conj(P) * dpsi, axis=0)
        DO[y:y + M, x:x + M] += P2
        NP += np.conj(o)[None] * dpsi
        DP += np.abs(o) ** 2
    c_obj, c_probe = step_coefficients(prm)
    O_new = O + _normalised_step(prm.beta_obj, NO, DO, *c_obj)
    if t >= prm.probe_update_start:
        P_new = P + np.stack([_normalised_step(prm.beta_probe, NP[k], DP, *c_probe) for k in range(K)])
    else:
        P_new = P.copy()
    return O_new, P_new, errnum


def iteration_dm(I, positions, O, P, psi, prm: Params, t: int, eps: float, g):
    """One pc-DM iteration (reading 10d; difference map of Thibault et al. with the pc intensity model
    of Fig. 1 box 1 in its modulus projection). psi: exit-wave state, (N, K, M, M), updated in place.
    Per position: psi_ov = P o_n, chi = 2 psi_ov - psi_n, psi_n <- psi_n + Pi_F(chi) - psi_ov. Then the
    overlap projection, alternating: the object takes one normalised step with dpsi = psi_n - psi_ov,
    then the probe one from the new object, sum conj(o'_n) (psi_n - P o'_n) over sum |o'_n|^2.
    Inside a complex-constraint window the constraint (Eqs. 9-11) acts on the object between the
    two steps, and every state moves with its box, psi_n += P (o_n constrained - o_n), so that the
    difference psi_n - P o_n the map carries is the constraint's to keep.
    E_t is the estimate's error: the pc model of psi_ov against I_n."""
    M, K = prm.M, prm.K
    NO = np.zeros(O.shape, np.complex128)
    DO = np.zeros(O.shape, np.float64)
    NP = np.zeros(P.shape, np.complex128)
    DP = np.zeros((M, M), np.float64)
    P2 = np.sum(np.abs(P) ** 2, axis=0)
    errnum, errden = [], []
    for n, (y, x) in enumerate(positions):
        o = O[y:y + M, x:x + M]
        psi_ov = P * o[None]
        chi = 2.0 * psi_ov - psi[n]
        In = I[n].astype(np.float64)
        _, Ihat = modulus(propagate_forward(psi_ov, prm), In, g, eps, prm.blur_domain)
        errnum.append(math.fsum(((Ihat - In) ** 2).ravel()))
        errden.append(math.fsum((In ** 2).ravel()))
        Chi_new, _ = modulus(propagate_forward(chi, prm), In, g, eps, prm.blur_domain)
        psi[n] = psi[n] + propagate_backward(Chi_new, prm) - psi_ov
        dpsi = psi[n] - psi_ov
        NO[y:y + M, x:x + M] += np.sum(np.conj(P) * dpsi, axis=0)
        DO[y:y + M, x:x + M] += P2
    c_obj, c_probe = step_coefficients(prm)
    O_new = O + _normalised_step(prm.beta_obj, NO, DO, *c_obj)
    if in_window(t, prm.windows):
        O_con = complex_constraint(O_new, positions, prm)
        for n, (y, x) in enumerate(positions):
            psi[n] += P * (O_con[y:y + M, x:x + M] - O_new[y:y + M, x:x + M])[None]
        O_new = O_con
    if t >= prm.probe_update_start:
        for n, (y, x) in enumerate(positions):
            o = O_new[y:y + M, x:x + M]
            NP += np.conj(o)[None] * (psi[n] - P * o[None])
            DP += np.abs(o) ** 2
        P_new = P + np.stack([_normalised_step(prm.beta_probe, NP[k], DP, *c_probe) for k in range(K)])
    else:
        P_new = P.copy()
    return O_new, P_new, math.sqrt(math.fsum(errnum) / math.fsum(errden))


def batches(N: int, prm: Params):
    """Partition of the positions into batches of prm.minibatch (reading 11b): consecutive groups of
    a Philox permutation of 0..N-1 (stream 3); one batch of every position when minibatch is 0."""
    if prm.minibatch <= 0 or prm.minibatch >= N:
        return [np.arange(N)]
    perm = philox.permutation(N, prm.order_seed, 3, 0)
    return [perm[b:b + prm.minibatch] for b in range(0, N, prm.minibatch)]


def visit_order(nb: int, prm: Params, t: int):
    """Order in which iteration t visits the batches: a Philox permutation (stream 4, counter t)."""
    return philox.permutation(nb, prm.order_seed, 4, t) if nb > 1 else np.arange(nb)


def iteration(I: np.ndarray, positions: np.ndarray, O: np.ndarray, P: np.ndarray, prm: Params,
              t: int, eps: float, g: np.ndarray, parts=None):
    """One pc-engine iteration. Returns (O_new, P_new, E_t) in complex128.

    Without mini-batches: one simultaneous step over every position. With batches (the paper's
    sequential pc-ePIE of Fig. 1 for batches of one position): the batches are visited in the
    iteration's order, each step starting from the object and probe the previous one left; the
    complex constraint (inside its windows) follows the last batch, over every box; E_t sums the
    error numerators of all positions, each at the state its batch saw."""
    parts = batches(len(positions), prm) if parts is None else parts
    errnum = []
    for b in visit_order(len(parts), prm, t):
        O, P, en = _batch_step(I, positions, parts[b], O, P, prm, t, eps, g)
        errnum += en
    if in_window(t, prm.windows):
        O = complex_constraint(O, positions, prm)
    errden = [math.fsum((I[n].astype(np.float64) ** 2).ravel()) for n in range(len(positions))]
    E = math.sqrt(math.fsum(errnum) / math.fsum(errden))
    return O, P, E


def iterate(I, positions, O, P, prm: Params, n_iter: int):
    """Run n_iter iterations from iteration number prm.start_iteration.

    Returns (O, P, errors) with O, P complex128 and one E per iteration.
    """
    I = np.asarray(I)
    positions = np.asarray(positions, dtype=np.int64)
    O = np.asarray(O, dtype=np.complex128).copy()
    P = np.asarray(P, dtype=np.complex128).reshape(prm.K, prm.M, prm.M).copy()
    eps = prm.eps_mod if prm.eps_mod > 0 else default_eps(I)
    g = gaussian_kernel(prm.kernel_size, prm.sigma1, prm.sigma2)
    errors = []
    if prm.engine == "dm":
        # exit-wave state of pc-DM, started at the overlap estimate
        psi = np.stack([P * O[y:y + prm.M, x:x + prm.M][None] for (y, x) in positions])
        for i in range(n_iter):
            t = prm.start_iteration + i
            O, P, E = iteration_dm(I, positions, O, P, psi, prm, t, eps, g)
            errors.append(E)
        return O, P, np.array(errors)
    if prm.engine != "pie":
        raise ValueError(f"unknown engine {prm.engine!r}")
    parts = batches(len(positions), prm)
    for i in range(n_iter):
        t = prm.start_iteration + i
        O, P, E = iteration(I, positions, O, P, prm, t, eps, g, parts)
        errors.append(E)
    return O, P, np.array(errors)
