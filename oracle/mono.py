"""FP64 oracle of numerical monochromatisation (Sec. 4.2, Eqs. 12-13). TEST INFRASTRUCTURE ONLY:
only the tests, the smoke check and the benchmark's CPU baseline use it.

A broadband far-field pattern b is the spectrum-weighted sum of the monochromatic pattern m at a
reference wavelength lambda_c, each term magnified about the detector centre by a_j =
lambda_j / lambda_c (diffraction angles scale with the wavelength) and divided by a_j^2 so that each
term keeps the weight's share of the energy:

    b = C m,   C = sum_j w_j / a_j^2 * T_j,   (T_j m)(y, x) = m(c + (y - c) / a_j, c + (x - c) / a_j)

with c = M / 2 and T_j linear interpolation on the pixel grid, zero outside it (a sample between
the last pixel and the outside blends toward zero, so T_j is continuous in the coordinates). T_j is
separable: T_j m = S_j m S_j^T with S_j the M x M one-dimensional interpolation matrix.

Eq. 12 asks for min ||C x - b||_2 over the Krylov subspace of Eq. 13; CGLS (conjugate gradients on
the normal equations, in the form that never forms C^T C) reaches it after k steps from x_0 = 0.
Readings: the operator above (the paper defines C only as depending on the spectrum; this is the
wavelength-scaling model of its reference [17]); k is the number of CGLS steps, so x_k lies in the
k-dimensional subspace of Eq. 13.
"""
from __future__ import annotations

import math

import numpy as np


def interp_matrix(M: int, a: float) -> np.ndarray:
    """S (M x M): (S v)(i) = linear interpolation of v at t = c + (i - c) / a, c = M / 2, with v = 0
    outside 0..M-1."""
    c = M / 2.0
    S = np.zeros((M, M))
    for i in range(M):
        t = c + (i - c) / a
        i0 = math.floor(t)
        f = t - i0
        if 0 <= i0 < M:
            S[i, i0] += 1.0 - f
        if 0 <= i0 + 1 < M:
            S[i, i0 + 1] += f
    return S


def spectrum_operator(M: int, scales, weights):
    """C as the list of (w_j / a_j^2, S_j)."""
    assert len(scales) == len(weights) and len(scales) > 0
    return [(float(w) / (float(a) * float(a)), interp_matrix(M, float(a))) for a, w in zip(scales, weights)]


def apply_C(X: np.ndarray, ops) -> np.ndarray:
    """C X = sum_j w_j S_j X S_j^T."""
    return sum(w * (S @ X @ S.T) for w, S in ops)


def apply_CT(R: np.ndarray, ops) -> np.ndarray:
    """C^T R = sum_j w_j S_j^T R S_j (the adjoint of apply_C)."""
    return sum(w * (S.T @ R @ S) for w, S in ops)


def cgls(b: np.ndarray, ops, k: int):
    """k CGLS steps on min ||C x - b|| from x_0 = 0 (Eqs. 12-13). Returns x_k and the residual
    norms ||b - C x_i|| for i = 0..k (from the recurrence for r_i)."""
    x = np.zeros_like(b, dtype=np.float64)
    r = np.array(b, dtype=np.float64)
    s = apply_CT(r, ops)
    p = s.copy()
    gamma = float(np.sum(s * s))
    res = [math.sqrt(float(np.sum(r * r)))]
    for _ in range(k):
        if gamma == 0.0:  # C^T r = 0: x is the least-squares solution already
            res.append(res[-1])
            continue
        q = apply_C(p, ops)
        qq = float(np.sum(q * q))
        alpha = gamma / qq
        x = x + alpha * p
        r = r - alpha * q
        s = apply_CT(r, ops)
        gamma_new = float(np.sum(s * s))
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
        res.append(math.sqrt(float(np.sum(r * r))))
    return x, np.array(res)


def monochromatise(B: np.ndarray, scales, weights, k: int, clamp: bool = False):
    """CGLS_k of every pattern of B (N x M x M); clamp sets negative intensities to zero (the pc
    engine takes non-negative patterns). Returns (X, residual norms N x (k + 1))."""
    N, M, _ = B.shape
    ops = spectrum_operator(M, scales, weights)
    X = np.empty((N, M, M))
    R = np.empty((N, k + 1))
    for n in range(N):
        X[n], R[n] = cgls(B[n].astype(np.float64), ops, k)
    if clamp:
        X = np.maximum(X, 0.0)
    return X, R
