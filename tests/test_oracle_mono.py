"""Pins of the monochromatisation oracle (Sec. 4.2, Eqs. 12-13) against library routines, closed
forms and the least-squares problem it solves, each independent of the oracle's own code."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import mono


def _rng(seed):
    return np.random.default_rng(seed)


def _dense_C(M, scales, weights):
    """C as an M^2 x M^2 matrix, column by column, from scipy's interpolation (not the oracle's)."""
    c = M / 2.0
    y, x = np.mgrid[0:M, 0:M].astype(np.float64)
    cols = []
    for i in range(M * M):
        e = np.zeros(M * M)
        e[i] = 1.0
        E = e.reshape(M, M)
        out = np.zeros((M, M))
        for a, w in zip(scales, weights):
            coords = np.stack([(y - c) / a + c, (x - c) / a + c])
            out += w / (a * a) * ndimage.map_coordinates(E, coords, order=1, mode="grid-constant", cval=0.0)
        cols.append(out.ravel())
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("M,a", [(8, 1.0), (16, 1.3), (16, 0.8), (17, 1.75), (12, 1.05)])
def test_interpolation_is_scipy_linear_interpolation(M, a):
    """T = S v S^T samples v at c + (i - c) / a with linear interpolation and zero outside the
    grid: scipy.ndimage.map_coordinates, order 1, 'grid-constant'."""
    rng = _rng(1)
    V = rng.standard_normal((M, M))
    S = mono.interp_matrix(M, a)
    c = M / 2.0
    y, x = np.mgrid[0:M, 0:M].astype(np.float64)
    ref = ndimage.map_coordinates(V, np.stack([(y - c) / a + c, (x - c) / a + c]), order=1,
                                  mode="grid-constant", cval=0.0)
    assert np.max(np.abs(S @ V @ S.T - ref)) < 1e-12


def test_identity_and_linear_ramp():
    M = 16
    assert np.array_equal(mono.interp_matrix(M, 1.0), np.eye(M))
    # a linear function is reproduced exactly at the scaled coordinates (a >= 1: every sample inside)
    a = 1.37
    c = M / 2.0
    y, x = np.mgrid[0:M, 0:M].astype(np.float64)
    F = 0.3 * y - 1.1 * x + 2.0
    S = mono.interp_matrix(M, a)
    ref = 0.3 * ((y - c) / a + c) - 1.1 * ((x - c) / a + c) + 2.0
    assert np.max(np.abs(S @ F @ S.T - ref)) < 1e-12


def test_operator_matches_the_broadband_measurement_model():
    """For a_j >= 1 (reference = shortest wavelength) C with equal weights is the energy-keeping
    average of the magnified patterns the data generator sums (scipy, 'constant' mode)."""
    from synth.generators import _rescale_about_centre

    rng = _rng(2)
    M = 32
    m = rng.random((1, M, M))
    scales = [1.0, 1.0125, 1.025, 1.0375, 1.05]
    ops = mono.spectrum_operator(M, scales, [1.0 / len(scales)] * len(scales))
    ref = sum(_rescale_about_centre(m, s) for s in scales)[0] / len(scales)
    assert np.max(np.abs(mono.apply_C(m[0], ops) - ref)) < 1e-12


def test_adjoint():
    rng = _rng(3)
    M = 16
    ops = mono.spectrum_operator(M, [0.9, 1.0, 1.2, 1.6], [0.1, 0.4, 0.3, 0.2])
    X, Y = rng.standard_normal((2, M, M))
    lhs = np.sum(mono.apply_C(X, ops) * Y)
    rhs = np.sum(X * mono.apply_CT(Y, ops))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # and C agrees with the dense matrix built from scipy
    C = _dense_C(M, [0.9, 1.0, 1.2, 1.6], [0.1, 0.4, 0.3, 0.2])
    assert np.max(np.abs(C @ X.ravel() - mono.apply_C(X, ops).ravel())) < 1e-12


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_cgls_is_the_krylov_least_squares_solution(k):
    """x_k minimises ||C x - b|| over span{C^T b, (C^T C) C^T b, ...} (Eqs. 12-13): an explicit Krylov
    basis, orthonormalised, and a dense least-squares solve."""
    rng = _rng(4)
    M = 6
    scales, weights = [1.0, 1.15, 1.4], [0.5, 0.3, 0.2]
    C = _dense_C(M, scales, weights)
    b = rng.random(M * M)
    v = C.T @ b
    basis = []
    for _ in range(k):
        basis.append(v)
        v = C.T @ (C @ v)
    Q, _ = np.linalg.qr(np.stack(basis, axis=1))
    yk, *_ = np.linalg.lstsq(C @ Q, b, rcond=None)
    ref = Q @ yk
    x, res = mono.cgls(b.reshape(M, M), mono.spectrum_operator(M, scales, weights), k)
    assert np.linalg.norm(x.ravel() - ref) < 1e-9 * np.linalg.norm(ref)
    assert abs(res[-1] - np.linalg.norm(C @ ref - b)) < 1e-9 * np.linalg.norm(b)


def test_cgls_reaches_the_least_squares_solution():
    """With as many steps as unknowns (a well-conditioned spectrum) x_k is the least-squares
    solution of the full system."""
    rng = _rng(5)
    M = 4
    scales, weights = [1.0, 1.1], [0.7, 0.3]
    C = _dense_C(M, scales, weights)
    b = rng.random(M * M)
    ref, *_ = np.linalg.lstsq(C, b, rcond=None)
    x, _ = mono.cgls(b.reshape(M, M), mono.spectrum_operator(M, scales, weights), M * M)
    assert np.linalg.norm(x.ravel() - ref) < 1e-8 * np.linalg.norm(ref)


def test_monochromatic_light_needs_one_step():
    rng = _rng(6)
    b = rng.random((16, 16))
    x, res = mono.cgls(b, mono.spectrum_operator(16, [1.0], [1.0]), 1)
    assert np.max(np.abs(x - b)) < 1e-14 and res[-1] < 1e-12 * res[0]


def test_residual_decreases_and_solution_norm_grows():
    """CGLS: ||b - C x_i|| does not increase and ||x_i|| does not decrease with i."""
    rng = _rng(7)
    M = 24
    scales = list(np.linspace(1.0, 1.75, 12))
    ops = mono.spectrum_operator(M, scales, [1.0 / 12] * 12)
    b = mono.apply_C(rng.random((M, M)), ops) + 1e-3 * rng.standard_normal((M, M))
    norms = []
    for k in range(0, 13):
        x, res = mono.cgls(b, ops, k)
        norms.append(np.linalg.norm(x))
    assert np.all(np.diff(res) <= 1e-12 * res[0])
    assert np.all(np.diff(norms) >= -1e-12 * norms[-1])


def test_monochromatise_batch_and_clamp():
    rng = _rng(8)
    B = rng.random((3, 8, 8))
    X, R = mono.monochromatise(B, [1.0, 1.2], [0.5, 0.5], 4, clamp=True)
    assert X.shape == (3, 8, 8) and R.shape == (3, 5) and X.min() >= 0.0
    x1, r1 = mono.cgls(B[1], mono.spectrum_operator(8, [1.0, 1.2], [0.5, 0.5]), 4)
    assert np.array_equal(np.maximum(x1, 0.0), X[1]) and np.array_equal(r1, R[1])
