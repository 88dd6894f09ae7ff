"""FP64 CPU oracle of the warm-start data generator and of the warm-start assembly.

TEST INFRASTRUCTURE ONLY (see oracle/pc_engine.py): imported by tests/, by the
smoke check and by the benchmark's CPU baseline, never by the product path.

The paper has no learned component; the warm start estimates the object and the
blur width from the patterns before the iteration. What is computed here:

* Philox4x32-10, the counter-based generator of Salmon, Moraes, Dror and Shaw
  ("Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of two
  32x32->64-bit products with the published multipliers and Weyl key bumps.
  Both this oracle and the CUDA generator implement it from that definition;
  it decides the lattice vacancies (and, on the GPU only, the Poisson noise).
* The lattice phase: phi(r) = h sum_{sites p not vacant, |r - p| <= cutoff}
  exp(-|r - p|^2 / (2 s^2)), sites p_ij = origin + i a1 + j a2, a1 = a (cos t, sin t),
  a2 = a (cos(t + pi/3), sin(t + pi/3)) in (row, col); site (i, j) of sample m is
  vacant when word 0 of Philox((i, j, m, 1), key) < floor(vacancy 2^32). Brute force over
  every site near the box.
* The noise-free pattern: psi = P exp(i phi), the centred far-field DFT (Eq. 1),
  |Psi|^2 blurred by the isotropic Gaussian of Eq. 2 (taps +-min(ceil(5 sigma), 15),
  normalised, zero padding), scaled so that its sum is the dose.
* The stitch: O(r) = sum_n w(r - c_n) patch_n(r) / sum_n w(r - c_n) with a separable
  Hann window w(y, x) = sin^2(pi (y + 1/2) / Q) sin^2(pi (x + 1/2) / Q) over the
  Q x Q patch with corner c_n, and 1 where no patch covers r; patch values are
  exp(scale (out0 + i out1)).
* The median of the predicted sigma (mean of the two middle values for even N).
"""
from __future__ import annotations

import math

import numpy as np

from .pc_engine import Params, blur, propagate_forward

from .philox import key_words, philox4x32_10  # noqa: F401  (re-exported)
_MASK = 0xFFFFFFFF


def vacancy_threshold(vacancy: float) -> int:
    """Philox words below this integer mark a vacant site: min(floor(vacancy 2^32), 2^32 - 1)."""
    return int(min(math.floor(vacancy * 4294967296.0), 4294967295))


def lattice_basis(a: float, theta: float):
    a1 = a * np.array([math.cos(theta), math.sin(theta)])
    a2 = a * np.array([math.cos(theta + math.pi / 3), math.sin(theta + math.pi / 3)])
    return a1, a2


def lattice_phase(S, theta, oy, ox, sample, key64, a=16.0, peak=0.1, s_pk=1.5, cutoff=6.0, vacancy=0.05):
    """phi on the S x S box (rows y, cols x = 0..S-1), FP64, brute force over the sites near the box."""
    a1, a2 = lattice_basis(a, theta)
    origin = np.array([oy, ox], dtype=np.float64)
    # every site within `cutoff` of the box has lattice coordinates inside this range
    corners = np.array([[-cutoff, -cutoff], [-cutoff, S + cutoff], [S + cutoff, -cutoff], [S + cutoff, S + cutoff]])
    B = np.stack([a1, a2], axis=1)  # columns a1, a2
    uv = np.linalg.solve(B, (corners - origin).T).T
    i_lo, i_hi = int(math.floor(uv[:, 0].min())) - 1, int(math.ceil(uv[:, 0].max())) + 1
    j_lo, j_hi = int(math.floor(uv[:, 1].min())) - 1, int(math.ceil(uv[:, 1].max())) + 1
    ii, jj = np.meshgrid(np.arange(i_lo, i_hi + 1), np.arange(j_lo, j_hi + 1), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()
    ctr = np.stack([ii.astype(np.int64) & _MASK, jj.astype(np.int64) & _MASK,
                    np.full_like(ii, sample, dtype=np.int64), np.ones_like(ii, dtype=np.int64)], axis=-1)
    words = philox4x32_10(ctr.astype(np.uint64), key_words(key64))
    present = words[:, 0] >= np.uint64(vacancy_threshold(vacancy))
    sites = origin[None, :] + ii[:, None] * a1[None, :] + jj[:, None] * a2[None, :]
    sites = sites[present]
    y = np.arange(S, dtype=np.float64)
    phi = np.zeros((S, S))
    for py, px in sites:
        d2 = (y[:, None] - py) ** 2 + (y[None, :] - px) ** 2
        phi += np.where(d2 <= cutoff * cutoff, peak * np.exp(-d2 / (2.0 * s_pk * s_pk)), 0.0)
    return phi


def blur_taps(sigma: float) -> np.ndarray:
    """Normalised 1-D Gaussian taps, half-width min(ceil(5 sigma), 15); sigma = 0 is a delta."""
    if sigma <= 0:
        return np.ones(1)
    h = min(int(math.ceil(5.0 * sigma)), 15)
    d = np.arange(-h, h + 1, dtype=np.float64)
    g = np.exp(-d ** 2 / (2.0 * sigma * sigma))
    return g / g.sum()


def clean_pattern(probe, phi, sigma, dose):
    """Noise-free far-field pattern of psi = P exp(i phi), blurred (Eq. 2) and scaled to sum `dose`."""
    S = probe.shape[0]
    psi = probe * np.exp(1j * phi)
    Psi = propagate_forward(psi, Params(M=S, K=1, N=1, obj_h=S, obj_w=S, geometry="far"))
    g1 = blur_taps(sigma)
    I = blur(np.abs(Psi) ** 2, g1[:, None] * g1[None, :])
    return I * (dose / I.sum())


def target_patch(phi, scale):
    """(ln|o|, arg o) / scale on the central S/2 x S/2 box of a pure phase object: (Q, Q, 2)."""
    S = phi.shape[0]
    c = phi[S // 4:3 * S // 4, S // 4:3 * S // 4]
    return np.stack([np.zeros_like(c), c / scale], axis=-1)


def hann_window(Q):
    s = np.sin(np.pi * (np.arange(Q) + 0.5) / Q) ** 2
    return s[:, None] * s[None, :]


def stitch(patches, corners, obj_h, obj_w, scale):
    """patches (N, Q, Q, 2) network outputs; corners (N, 2) top-left of each Q x Q box."""
    N, Q = patches.shape[0], patches.shape[1]
    w = hann_window(Q)
    num = np.zeros((obj_h, obj_w), dtype=np.complex128)
    den = np.zeros((obj_h, obj_w))
    for n in range(N):
        r, c = int(corners[n][0]), int(corners[n][1])
        val = np.exp(scale * (patches[n, ..., 0] + 1j * patches[n, ..., 1]))
        num[r:r + Q, c:c + Q] += w * val
        den[r:r + Q, c:c + Q] += w
    out = np.ones((obj_h, obj_w), dtype=np.complex128)
    covered = den > 0
    out[covered] = num[covered] / den[covered]
    return out


def median(values):
    v = sorted(float(x) for x in values)
    n = len(v)
    return v[n // 2] if n % 2 else 0.5 * (v[n // 2 - 1] + v[n // 2])
