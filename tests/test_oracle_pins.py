"""Pins of the FP64 oracle against facts the paper or mathematics fix (CPU only).

Each test ties one step of oracle/pc_engine.py to something other than itself:
a brute-force definition, a closed form, an identity or a number printed in
the paper. A dropped term, a wrong sign or index, or a transposed operand in
the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import pc_engine as pe
from synth import electron_wavelength, far_field_object_pixel, make_problem, qpt_phase

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed=0):
    return np.random.default_rng(seed)


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _prm(M, K=1, geometry="far", **kw):
    return pe.Params(M=M, K=K, N=1, obj_h=M, obj_w=M, geometry=geometry, **kw)


# ------------------------------------------------------------------------ P1: FFT (Eq. 1)

def _brute_dft2_centred(psi):
    """Psi[u, v] = sum_{y,x} psi[y,x] exp(-2 pi i ((u - M/2) y + (v - M/2) x) / M), by loops."""
    M = psi.shape[0]
    out = np.zeros((M, M), complex)
    for u in range(M):
        for v in range(M):
            acc = 0j
            for y in range(M):
                for x in range(M):
                    acc += psi[y, x] * complex(math.cos(-2 * math.pi * ((u - M // 2) * y + (v - M // 2) * x) / M),
                                               math.sin(-2 * math.pi * ((u - M // 2) * y + (v - M // 2) * x) / M))
            out[u, v] = acc
    return out


def test_p1_brute_force_dft_8x8():
    psi = _crandn(_rng(1), 8, 8)
    got = pe.propagate_forward(psi, _prm(8))
    assert np.max(np.abs(got - _brute_dft2_centred(psi))) < 1e-12 * np.max(np.abs(got))


def test_p1_parseval_and_round_trip():
    psi = _crandn(_rng(2), 3, 32, 32)
    prm = _prm(32, 3)
    Psi = pe.propagate_forward(psi, prm)
    assert abs(np.sum(np.abs(Psi) ** 2) - 32 * 32 * np.sum(np.abs(psi) ** 2)) < 1e-10 * np.sum(np.abs(Psi) ** 2)
    assert np.max(np.abs(pe.propagate_backward(Psi, prm) - psi)) < 1e-13


def test_p1_checkerboard_equals_fftshift():
    M = 16
    psi = _crandn(_rng(3), M, M)
    y, x = np.mgrid[0:M, 0:M]
    chk = np.fft.fft2(psi * (-1.0) ** (y + x))
    assert np.max(np.abs(chk - pe.propagate_forward(psi, _prm(M)))) < 1e-12


# ------------------------------------------------------------------------ P2: blur (Eqs. 6-7)

def _brute_blur(img, s1, s2, size=11):
    """Direct zero-padded sum with Eq. 7 written out: x = column offset (sigma_1), y = row offset (sigma_2)."""
    h = size // 2
    w = {}
    for dy in range(-h, h + 1):
        for dx in range(-h, h + 1):
            ex = dx * dx / (2 * s1 * s1) if s1 > 0 else (0.0 if dx == 0 else math.inf)
            ey = dy * dy / (2 * s2 * s2) if s2 > 0 else (0.0 if dy == 0 else math.inf)
            w[dy, dx] = math.exp(-(ex + ey))
    tot = sum(w.values())
    H, W = img.shape
    out = np.zeros_like(img)
    for r in range(H):
        for c in range(W):
            acc = 0.0
            for (dy, dx), wt in w.items():
                rr, cc = r + dy, c + dx
                if 0 <= rr < H and 0 <= cc < W:
                    acc += wt * img[rr, cc]
            out[r, c] = acc / tot
    return out


def test_p2_kernel_normalised_and_anisotropy_axes():
    g = pe.gaussian_kernel(11, 0.7, 2.0)
    assert abs(g.sum() - 1.0) < 1e-15
    # sigma_1 acts along x (columns): the kernel is wider along rows (y) when sigma_2 > sigma_1
    assert g[5, 0] < g[0, 5]
    assert np.allclose(g, g[::-1, :]) and np.allclose(g, g[:, ::-1])


def test_p2_blur_matches_direct_sum_with_asymmetric_sigmas():
    img = _rng(4).random((13, 17))
    got = pe.blur(img, pe.gaussian_kernel(11, 0.8, 1.7))
    assert np.max(np.abs(got - _brute_blur(img, 0.8, 1.7))) < 1e-14


def test_p2_sigma_zero_is_identity_and_constant_field():
    img = _rng(5).random((20, 20))
    assert np.array_equal(pe.blur(img, pe.gaussian_kernel(11, 0.0, 0.0)), img)
    const = np.full((30, 30), 2.5)
    out = pe.blur(const, pe.gaussian_kernel(11, 1.3, 1.3))
    assert np.max(np.abs(out[5:-5, 5:-5] - 2.5)) < 1e-14
    assert out[0, 0] < 2.5  # zero padding at the border


def test_p2_transpose_symmetry_for_equal_sigmas():
    img = _rng(6).random((16, 16))
    g = pe.gaussian_kernel(11, 1.1, 1.1)
    assert np.max(np.abs(pe.blur(img.T, g) - pe.blur(img, g).T)) < 1e-14


# ------------------------------------------------------------------------ P3: Fresnel transfer function

def test_p3_fresnel_unitary_and_dc():
    H = pe.fresnel_tf(64, 10.0)
    assert np.max(np.abs(np.abs(H) - 1)) < 1e-15
    assert H[0, 0] == 1.0
    psi = _crandn(_rng(7), 2, 64, 64)
    prm = _prm(64, 2, "near", fresnel_F=10.0)
    Psi = pe.propagate_forward(psi, prm)
    assert abs(np.sum(np.abs(Psi) ** 2) - np.sum(np.abs(psi) ** 2)) < 1e-10 * np.sum(np.abs(psi) ** 2)
    assert np.max(np.abs(pe.propagate_backward(Psi, prm) - psi)) < 1e-13


def test_p3_gaussian_beam_closed_form():
    """A Gaussian exp(-r^2 / (2 s^2)) propagated by exp(-i pi D f^2), D = M / F px^2, stays Gaussian
    with complex parameter q = s^2 + i D / (2 pi): psi = s^2 / q exp(-r^2 / (2 q))."""
    M, F, s = 128, 4.0, 6.0
    c = M // 2
    y, x = np.mgrid[0:M, 0:M].astype(float)
    r2 = (y - c) ** 2 + (x - c) ** 2
    psi0 = np.exp(-r2 / (2 * s * s))
    D = M / F
    q = s * s + 1j * D / (2 * np.pi)
    expected = (s * s / q) * np.exp(-r2 / (2 * q))
    got = pe.propagate_forward(psi0, _prm(M, 1, "near", fresnel_F=F))
    assert np.max(np.abs(got - expected)) < 1e-9


# ------------------------------------------------------------------------ P4: modulus (Fig. 1 box 1)

def test_p4_coherent_modulus_restores_measured_intensity_and_is_idempotent():
    rng = _rng(8)
    Psi = _crandn(rng, 1, 16, 16)
    I = rng.random((16, 16)) * 5
    g = pe.gaussian_kernel(11, 0, 0)
    P1, _ = pe.modulus(Psi, I, g, 0.0, "amplitude")
    assert np.max(np.abs(np.abs(P1[0]) ** 2 - I)) < 1e-12
    assert np.max(np.abs(np.angle(P1[0] / Psi[0]))) < 1e-12
    P2, _ = pe.modulus(P1, I, g, 0.0, "amplitude")
    assert np.max(np.abs(P2 - P1)) < 1e-12


def test_p4_consistent_blurred_amplitude_leaves_psi_unchanged():
    rng = _rng(9)
    Psi = _crandn(rng, 3, 24, 24)
    g = pe.gaussian_kernel(11, 1.2, 0.9)
    AG = _brute_blur(np.sqrt(np.sum(np.abs(Psi) ** 2, 0)), 1.2, 0.9)
    out, Ihat = pe.modulus(Psi, AG ** 2, g, 0.0, "amplitude")
    assert np.max(np.abs(out - Psi)) < 1e-12
    assert np.max(np.abs(Ihat - AG ** 2)) < 1e-12
    Im = _brute_blur(np.sum(np.abs(Psi) ** 2, 0), 1.2, 0.9)
    out, Ihat = pe.modulus(Psi, Im, g, 0.0, "intensity")
    assert np.max(np.abs(out - Psi)) < 1e-12


# ------------------------------------------------------------------------ P5: fixed point

def _consistent_data(O, P, pos, prm):
    """Noise-free data from the engine's own forward model, written without the oracle."""
    M = prm.M
    out = []
    for (y, x) in pos:
        psi = P * O[y:y + M, x:x + M][None]
        if prm.geometry == "far":
            Psi = np.fft.fftshift(np.fft.fft2(psi), axes=(-2, -1))
        else:
            u = np.fft.fftfreq(M) * M
            H = np.exp(-1j * np.pi * (u[:, None] ** 2 + u[None, :] ** 2) / (M * prm.fresnel_F))
            Psi = np.fft.ifft2(np.fft.fft2(psi) * H)
        S = np.sum(np.abs(Psi) ** 2, 0)
        if prm.blur_domain == "amplitude":
            out.append(_brute_blur(np.sqrt(S), prm.sigma1, prm.sigma2) ** 2)
        else:
            out.append(_brute_blur(S, prm.sigma1, prm.sigma2))
    return np.array(out)


@pytest.mark.parametrize("geometry,blur_domain,K", [("far", "amplitude", 2), ("near", "intensity", 1),
                                                     ("far", "intensity", 1), ("near", "amplitude", 3)])
def test_p5_fixed_point_on_consistent_data(geometry, blur_domain, K):
    rng = _rng(10)
    M, side = 16, 28
    O = (0.5 + rng.random((side, side))) * np.exp(1j * rng.random((side, side)))
    P = _crandn(rng, K, M, M)
    pos = np.array([(0, 0), (0, 12), (12, 0), (12, 12), (6, 6)])
    prm = pe.Params(M=M, K=K, N=len(pos), obj_h=side, obj_w=side, geometry=geometry, blur_domain=blur_domain,
                    fresnel_F=3.0, sigma1=1.0, sigma2=0.6, eps_mod=1e-300)
    I = _consistent_data(O, P, pos, prm)
    O1, P1, E = pe.iterate(I, pos, O, P, prm, 1)
    assert np.max(np.abs(O1 - O)) < 1e-12
    assert np.max(np.abs(P1 - P)) < 1e-12
    assert E[0] < 1e-12


# ------------------------------------------------------------------------ P6: scatter-add and D_O

def test_p6_update_matches_vectorised_add_at_and_correlation():
    rng = _rng(11)
    M, side, K = 8, 30, 2
    O = np.exp(1j * rng.random((side, side)))
    P = _crandn(rng, K, M, M)
    pos = rng.integers(0, side - M + 1, size=(9, 2))
    prm = pe.Params(M=M, K=K, N=len(pos), obj_h=side, obj_w=side, sigma1=0.9, sigma2=0.9,
                    delta_obj=0.0, delta_probe=0.0, beta_obj=1.0, beta_probe=1.0, eps_mod=1e-3)
    I = rng.random((len(pos), M, M)) * 40
    O1, P1, _ = pe.iterate(I, pos, O, P, prm, 1)
    # independent accumulation with np.add.at on flat indices
    g = pe.gaussian_kernel(11, 0.9, 0.9)
    NO = np.zeros(side * side, complex)
    DO = np.zeros(side * side)
    idx_box = (np.arange(M)[:, None] * side + np.arange(M)[None, :]).ravel()
    for n, (y, x) in enumerate(pos):
        o = O[y:y + M, x:x + M]
        Psi = np.fft.fftshift(np.fft.fft2(P * o), axes=(-2, -1))
        S = np.sqrt(np.sum(np.abs(Psi) ** 2, 0))
        R = np.sqrt(I[n]) / (_brute_blur(S, 0.9, 0.9) + 1e-3)
        dpsi = np.fft.ifft2(np.fft.ifftshift(R * Psi, axes=(-2, -1))) - P * o
        np.add.at(NO, y * side + x + idx_box, np.sum(np.conj(P) * dpsi, 0).ravel())
        np.add.at(DO, y * side + x + idx_box, np.sum(np.abs(P) ** 2, 0).ravel())
    # D_O is the correlation of sum_k |P_k|^2 with the position indicator image
    ind = np.zeros((side, side))
    np.add.at(ind, (pos[:, 0], pos[:, 1]), 1.0)
    from scipy import signal
    DO_corr = signal.convolve2d(ind, np.sum(np.abs(P) ** 2, 0), mode="full")[:side, :side]
    assert np.max(np.abs(DO.reshape(side, side) - DO_corr)) < 1e-10
    cov = DO > 0
    expect = O.ravel().copy()
    expect[cov] += NO[cov] / DO[cov]
    assert np.max(np.abs(O1.ravel() - expect)) < 1e-10
    del g


def test_p6_single_position_update_is_the_projection():
    """N = 1, K = 1, delta = 0, sigma = 0: the updated object gives exactly the projected exit wave,
    P o_new = psi' (and likewise o P_new = psi'), since conj(P) dpsi / |P|^2 = dpsi / P."""
    rng = _rng(12)
    M = 16
    O = (0.5 + rng.random((M, M))) * np.exp(1j * rng.random((M, M)))
    P = _crandn(rng, 1, M, M)
    I = rng.random((1, M, M)) * 10
    prm = pe.Params(M=M, K=1, N=1, obj_h=M, obj_w=M, sigma1=0, sigma2=0, delta_obj=0.0, delta_probe=0.0,
                    eps_mod=1e-300)
    O1, P1, _ = pe.iterate(I, np.array([[0, 0]]), O, P, prm, 1)
    Psi = np.fft.fft2(P[0] * O)
    psi_proj = np.fft.ifft2(np.sqrt(np.fft.ifftshift(I[0])) * np.exp(1j * np.angle(Psi)))
    assert np.max(np.abs(P[0] * O1 - psi_proj)) < 1e-10 * np.max(np.abs(psi_proj))
    assert np.max(np.abs(O * P1[0] - psi_proj)) < 1e-10 * np.max(np.abs(psi_proj))


@pytest.mark.parametrize("alpha", [0.0, 1.0])
def test_p6b_rpie_single_position_closed_forms(alpha):
    """rPIE step (Sec. 5, Fig. 11c), N = 1, K = 1, sigma = 0, object and probe steps both rPIE.
    alpha = 0: the denominator is |P|^2 alone, so P o_new = psi' (the projection);
    alpha = 1: the ePIE step o_new = o + conj(P) (psi' - psi) / max|P|^2 (and the same for P)."""
    rng = _rng(13)
    M = 16
    O = (0.5 + rng.random((M, M))) * np.exp(1j * rng.random((M, M)))
    P = _crandn(rng, 1, M, M)
    I = rng.random((1, M, M)) * 10
    prm = pe.Params(M=M, K=1, N=1, obj_h=M, obj_w=M, sigma1=0, sigma2=0, eps_mod=1e-300, step_rule="rpie",
                    rpie_alpha_obj=alpha, rpie_alpha_probe=alpha)
    O1, P1, _ = pe.iterate(I, np.array([[0, 0]]), O, P, prm, 1)
    psi = P[0] * O
    Psi = np.fft.fft2(psi)
    psi_proj = np.fft.ifft2(np.sqrt(np.fft.ifftshift(I[0])) * np.exp(1j * np.angle(Psi)))
    tol = 1e-10 * np.max(np.abs(psi_proj))
    if alpha == 0.0:
        assert np.max(np.abs(P[0] * O1 - psi_proj)) < tol
        assert np.max(np.abs(O * P1[0] - psi_proj)) < tol
    else:
        d = psi_proj - psi
        assert np.max(np.abs(O1 - (O + np.conj(P[0]) * d / np.max(np.abs(P[0]) ** 2)))) < tol
        assert np.max(np.abs(P1[0] - (P[0] + np.conj(O) * d / np.max(np.abs(O) ** 2)))) < tol


def test_p6c_rpie_is_a_rescaled_normalised_step_and_keeps_the_fixed_point():
    """(1 - a) D + a max D = (1 - a) (D + a / (1 - a) max D): an rPIE step with weight a and step
    beta equals the normalised step with delta = a / (1 - a) and step beta / (1 - a); and any rule
    leaves consistent data fixed."""
    rng = _rng(14)
    M, side = 16, 28
    O = (0.5 + rng.random((side, side))) * np.exp(1j * rng.random((side, side)))
    P = _crandn(rng, 2, M, M)
    pos = np.array([(0, 0), (0, 12), (12, 0), (12, 12), (6, 6)])
    base = dict(M=M, K=2, N=len(pos), obj_h=side, obj_w=side, sigma1=1.0, sigma2=0.6, eps_mod=1e-300)
    I = rng.random((len(pos), M, M)) * 5
    a_o, a_p = 0.3, 0.6
    r = pe.iterate(I, pos, O, P, pe.Params(**base, step_rule="rpie", rpie_alpha_obj=a_o, rpie_alpha_probe=a_p), 1)
    n_o = pe.iterate(I, pos, O, P, pe.Params(**base, beta_obj=1 / (1 - a_o), delta_obj=a_o / (1 - a_o),
                                            beta_probe=1 / (1 - a_p), delta_probe=a_p / (1 - a_p)), 1)
    assert np.max(np.abs(r[0] - n_o[0])) < 1e-12 * np.max(np.abs(r[0]))
    assert np.max(np.abs(r[1] - n_o[1])) < 1e-12 * np.max(np.abs(r[1]))
    prm = pe.Params(**base, step_rule="rpie", rpie_alpha_obj=0.5, rpie_alpha_probe=1.0)
    Ic = _consistent_data(O, P, pos, prm)
    O1, P1, E = pe.iterate(Ic, pos, O, P, prm, 1)
    assert np.max(np.abs(O1 - O)) < 1e-12 and np.max(np.abs(P1 - P)) < 1e-12 and E[0] < 1e-12
    with pytest.raises(ValueError):
        pe.iterate(I, pos, O, P, pe.Params(**base, step_rule="sequential"), 1)


# ------------------------------------------------------------------------ mini-batch (sequential) engine

def test_philox_permutation():
    from oracle import philox

    a = philox.permutation(10, 99, 4, 1)
    assert sorted(a.tolist()) == list(range(10))
    assert np.array_equal(a, philox.permutation(10, 99, 4, 1))
    assert not np.array_equal(a, philox.permutation(10, 99, 4, 2))
    assert not np.array_equal(a, philox.permutation(10, 98, 4, 1))
    # every position lands in exactly one batch
    prm = pe.Params(M=8, K=1, N=23, obj_h=8, obj_w=8, minibatch=5, order_seed=3)
    parts = pe.batches(23, prm)
    assert [len(b) for b in parts] == [5, 5, 5, 5, 3]
    assert sorted(np.concatenate(parts).tolist()) == list(range(23))


def test_philox_permutation_is_a_uniform_shuffle():
    """A Fisher-Yates shuffle (j uniform in 0..i) reaches all n! orders equally often; over 6000
    counters the 6 orders of 3 elements each appear 1000 +- 145 times (5 binomial standard
    deviations). Drawing j from 0..i-1 instead (Sattolo's variant) gives only the two 3-cycles."""
    from collections import Counter

    from oracle import philox

    counts = Counter(tuple(philox.permutation(3, 12345, 4, t).tolist()) for t in range(6000))
    assert len(counts) == 6
    assert all(abs(c - 1000) <= 145 for c in counts.values()), counts


def test_minibatch_of_one_is_textbook_epie():
    """Batches of one position with the rPIE weight 1 on both steps are the ePIE engine (Fig. 1 with
    sigma = 0, K = 1): for each position in the iteration's order, psi' = the projection of P o,
    o += conj(P) (psi' - psi) / max|P|^2, P += conj(o_old) (psi' - psi) / max|o_old|^2."""
    rng = _rng(21)
    M, side = 16, 28
    O0 = (0.5 + rng.random((side, side))) * np.exp(1j * rng.random((side, side)))
    P0 = _crandn(rng, 1, M, M)
    pos = np.array([(0, 0), (0, 12), (12, 0), (12, 12), (6, 6)])
    I = rng.random((len(pos), M, M)) * 10
    prm = pe.Params(M=M, K=1, N=len(pos), obj_h=side, obj_w=side, sigma1=0, sigma2=0, eps_mod=1e-300,
                    step_rule="rpie", rpie_alpha_obj=1.0, rpie_alpha_probe=1.0, minibatch=1, order_seed=5)
    O1, P1, E1 = pe.iterate(I, pos, O0, P0, prm, 2)
    O, P = O0.copy(), P0[0].copy()
    parts = pe.batches(len(pos), prm)
    for t in (1, 2):
        for b in pe.visit_order(len(parts), prm, t):
            n = int(parts[b][0])
            y, x = pos[n]
            o = O[y:y + M, x:x + M].copy()
            psi = P * o
            Psi = np.fft.fftshift(np.fft.fft2(psi))
            Psi_p = np.sqrt(np.fft.fftshift(np.fft.ifftshift(I[n]))) * Psi / np.abs(Psi)
            d = np.fft.ifft2(np.fft.ifftshift(Psi_p)) - psi
            O[y:y + M, x:x + M] = o + np.conj(P) * d / np.max(np.abs(P) ** 2)
            P = P + np.conj(o) * d / np.max(np.abs(o) ** 2)
    assert np.max(np.abs(O1 - O)) < 1e-10 * np.max(np.abs(O))
    assert np.max(np.abs(P1[0] - P)) < 1e-10 * np.max(np.abs(P))


def test_minibatch_of_all_positions_is_the_simultaneous_step_and_keeps_the_fixed_point():
    rng = _rng(22)
    M, side = 16, 28
    O = (0.5 + rng.random((side, side))) * np.exp(1j * rng.random((side, side)))
    P = _crandn(rng, 2, M, M)
    pos = np.array([(0, 0), (0, 12), (12, 0), (12, 12), (6, 6)])
    base = dict(M=M, K=2, N=len(pos), obj_h=side, obj_w=side, sigma1=1.0, sigma2=0.6, eps_mod=1e-300)
    I = rng.random((len(pos), M, M)) * 5
    a = pe.iterate(I, pos, O, P, pe.Params(**base), 2)
    b = pe.iterate(I, pos, O, P, pe.Params(**base, minibatch=len(pos), order_seed=9), 2)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    c = pe.iterate(I, pos, O, P, pe.Params(**base, minibatch=2, order_seed=9), 2)
    assert np.max(np.abs(c[0] - a[0])) > 1e-6  # batches change the result
    prm = pe.Params(**base, minibatch=2, order_seed=9)
    Ic = _consistent_data(O, P, pos, prm)
    O1, P1, E = pe.iterate(Ic, pos, O, P, prm, 2)
    assert np.max(np.abs(O1 - O)) < 1e-12 and np.max(np.abs(P1 - P)) < 1e-12 and max(E) < 1e-12


# ------------------------------------------------------------------------ pc-DM engine

def test_dm_fixed_point_and_single_position_projection():
    rng = _rng(31)
    M, side = 16, 28
    O = (0.5 + rng.random((side, side))) * np.exp(1j * rng.random((side, side)))
    P = _crandn(rng, 2, M, M)
    pos = np.array([(0, 0), (0, 12), (12, 0), (12, 12), (6, 6)])
    prm = pe.Params(M=M, K=2, N=len(pos), obj_h=side, obj_w=side, sigma1=1.0, sigma2=0.6, eps_mod=1e-300,
                    engine="dm")
    Ic = _consistent_data(O, P, pos, prm)
    O1, P1, E = pe.iterate(Ic, pos, O, P, prm, 3)
    assert np.max(np.abs(O1 - O)) < 1e-12 and np.max(np.abs(P1 - P)) < 1e-12 and max(E) < 1e-12
    # one position, one mode, no blur, no floor: the first DM step is the projection (P o_new = psi')
    O = (0.5 + rng.random((M, M))) * np.exp(1j * rng.random((M, M)))
    P = _crandn(rng, 1, M, M)
    I = rng.random((1, M, M)) * 10
    prm = pe.Params(M=M, K=1, N=1, obj_h=M, obj_w=M, sigma1=0, sigma2=0, delta_obj=0.0, delta_probe=0.0,
                    eps_mod=1e-300, engine="dm", probe_update_start=10 ** 9)
    O1, _, _ = pe.iterate(I, np.array([[0, 0]]), O, P, prm, 1)
    Psi = np.fft.fft2(P[0] * O)
    proj = np.fft.ifft2(np.sqrt(np.fft.ifftshift(I[0])) * np.exp(1j * np.angle(Psi)))
    assert np.max(np.abs(P[0] * O1 - proj)) < 1e-10 * np.max(np.abs(proj))


def test_dm_probe_step_uses_the_new_object_and_error_is_the_estimates():
    """The probe step follows the object step (alternating projections): with one position, no blur
    and no floors, after one iteration o_new P_new = the projection (both factors fit psi' exactly);
    E of the first iteration is the NRMSE of P o_n itself (psi starts at P o_n)."""
    rng = _rng(33)
    M = 16
    O = (0.5 + rng.random((M, M))) * np.exp(1j * rng.random((M, M)))
    P = _crandn(rng, 1, M, M)
    I = rng.random((1, M, M)) * 10
    prm = pe.Params(M=M, K=1, N=1, obj_h=M, obj_w=M, sigma1=0, sigma2=0, delta_obj=0.0, delta_probe=0.0,
                    eps_mod=1e-300, engine="dm")
    O1, P1, E = pe.iterate(I, np.array([[0, 0]]), O, P, prm, 1)
    Psi = np.fft.fft2(P[0] * O)
    proj = np.fft.ifft2(np.sqrt(np.fft.ifftshift(I[0])) * np.exp(1j * np.angle(Psi)))
    assert np.max(np.abs(P1[0] * O1 - proj)) < 1e-10 * np.max(np.abs(proj))
    model = np.abs(np.fft.fftshift(Psi)) ** 2
    assert abs(E[0] - np.sqrt(np.sum((model - I[0]) ** 2) / np.sum(I[0] ** 2))) < 1e-12


def test_dm_with_a_fixed_probe_is_textbook_difference_map():
    """Probe fixed, no floor, sigma = 0, K = 1: the overlap projection is exact in one step, so pc-DM is
    the difference map: O = sum conj(P) psi_n / sum |P|^2 over the covering boxes, then
    psi_n <- psi_n + Pi_F(2 P o_n - psi_n) - P o_n, starting from psi_n = P o_n."""
    rng = _rng(32)
    M, side = 16, 30
    O0 = (0.5 + rng.random((side, side))) * np.exp(1j * rng.random((side, side)))
    P = _crandn(rng, 1, M, M)
    pos = np.array([(0, 0), (0, 14), (14, 0), (14, 14), (7, 7)])
    I = rng.random((len(pos), M, M)) * 10
    prm = pe.Params(M=M, K=1, N=len(pos), obj_h=side, obj_w=side, sigma1=0, sigma2=0, delta_obj=0.0,
                    eps_mod=1e-300, engine="dm", probe_update_start=10 ** 9)
    O1, _, _ = pe.iterate(I, pos, O0, P, prm, 3)

    def proj_f(chi, In):
        X = np.fft.fftshift(np.fft.fft2(chi))
        return np.fft.ifft2(np.fft.ifftshift(np.sqrt(In) * X / np.abs(X)))

    O = O0.copy()
    psi = [P[0] * O[y:y + M, x:x + M] for y, x in pos]
    for _ in range(3):
        new_psi = []
        for n, (y, x) in enumerate(pos):
            ov = P[0] * O[y:y + M, x:x + M]
            new_psi.append(psi[n] + proj_f(2 * ov - psi[n], I[n]) - ov)
        psi = new_psi
        num = np.zeros_like(O)
        den = np.zeros(O.shape)
        for n, (y, x) in enumerate(pos):
            num[y:y + M, x:x + M] += np.conj(P[0]) * psi[n]
            den[y:y + M, x:x + M] += np.abs(P[0]) ** 2
        O = np.where(den > 0, num / np.where(den > 0, den, 1), O)
    assert np.max(np.abs(O1 - O)) < 1e-10 * np.max(np.abs(O))


# ------------------------------------------------------------------------ P7 / P8: coherent reduction, modes

def _minimal_coherent_engine(I, pos, O, P, n_iter, delta):
    """Plain simultaneous projection engine: Psi' = sqrt(I) sign(Psi) (sign(0) = 0), normalised scatter-add."""
    M = P.shape[-1]
    O, P = O.copy(), P.copy()
    errs = []
    for _ in range(n_iter):
        NO = np.zeros_like(O)
        DO = np.zeros(O.shape)
        NP = np.zeros_like(P)
        DP = np.zeros(P.shape)
        num = den = 0.0
        for n, (y, x) in enumerate(pos):
            o = O[y:y + M, x:x + M]
            F = np.fft.fftshift(np.fft.fft2(P * o))
            num += np.sum((np.abs(F) ** 2 - I[n]) ** 2)
            den += np.sum(I[n] ** 2)
            d = np.fft.ifft2(np.fft.ifftshift(np.sqrt(I[n]) * np.sign(F))) - P * o
            NO[y:y + M, x:x + M] += np.conj(P) * d
            DO[y:y + M, x:x + M] += np.abs(P) ** 2
            NP += np.conj(o) * d
            DP += np.abs(o) ** 2
        O, P = O + NO / (DO + delta * DO.max()), P + NP / (DP + delta * DP.max())
        errs.append(math.sqrt(num / den))
    return O, P, np.array(errs)


def test_p7_reduces_to_coherent_engine():
    p = make_problem(0, scan_side=4, obj_side=112)
    prm = pe.Params.from_dict(dict(p.params, sigma1=0.0, sigma2=0.0, eps_mod=1e-300))
    O1, P1, E1 = pe.iterate(p.I, p.positions, p.O0, p.P0, prm, 3)
    O2, P2, E2 = _minimal_coherent_engine(p.I.astype(float), p.positions, p.O0.astype(complex),
                                          p.P0[0].astype(complex), 3, 1e-3)
    assert np.max(np.abs(O1 - O2)) < 1e-9
    assert np.max(np.abs(P1[0] - P2)) < 1e-9 * np.max(np.abs(P2))
    assert np.max(np.abs(E1 - E2)) < 1e-12


def test_p8_zero_extra_modes_equal_single_mode():
    p = make_problem(0, scan_side=3, obj_side=96)
    prm1 = pe.Params.from_dict(p.params)
    prm1.eps_mod = pe.default_eps(p.I)
    prm3 = pe.Params.from_dict(dict(p.params, K=3, eps_mod=prm1.eps_mod))
    P3 = np.concatenate([p.P0, np.zeros((2, 64, 64), np.complex64)])
    O1, P1, E1 = pe.iterate(p.I, p.positions, p.O0, p.P0, prm1, 2)
    O3, P3o, E3 = pe.iterate(p.I, p.positions, p.O0, P3, prm3, 2)
    assert np.max(np.abs(O1 - O3)) < 1e-12
    assert np.max(np.abs(P1[0] - P3o[0])) < 1e-12 * np.max(np.abs(P1))
    assert np.max(np.abs(E1 - E3)) < 1e-14


# ------------------------------------------------------------------------ P9: complex constraint (Eqs. 9-11, 19)

def _homogeneous(side, C, rng):
    """Eqs. 17-18 with beta/delta = C: ln A = C phi with phi in (0, 1] (so phi stays in (-pi, pi])."""
    phi = 0.05 + 0.9 * rng.random((side, side))
    return np.exp(C * phi) * np.exp(1j * phi)


def test_p9_identity_when_alphas_zero():
    rng = _rng(13)
    O = (0.5 + rng.random((40, 40))) * np.exp(1j * (rng.random((40, 40)) - 0.5))
    pos = np.array([(0, 0), (10, 10), (20, 5)])
    prm = pe.Params(M=16, K=1, N=3, obj_h=40, obj_w=40, alpha1=0.0, alpha2=0.0)
    out = pe.complex_constraint(O, pos, prm)
    assert np.max(np.abs(out - O)) < 1e-14


@pytest.mark.parametrize("alpha1,alpha2", [(1.0, 0.0), (0.0, 1.0), (0.5, 0.5)])
def test_p9_homogeneous_object_has_cbar_c_and_is_unchanged(alpha1, alpha2):
    rng = _rng(14)
    C = 0.25  # the QPT value of Sec. 4.7
    O = _homogeneous(40, C, rng)
    pos = np.array([(0, 0), (8, 16), (24, 24), (4, 6), (12, 12)])  # the last two overlap the others
    cb = pe.cbar_per_position(O, pos, 16, 0.01, 10.0)
    assert np.max(np.abs(cb - C)) < 1e-12
    prm = pe.Params(M=16, K=1, N=5, obj_h=40, obj_w=40, alpha1=alpha1, alpha2=alpha2)
    assert np.max(np.abs(pe.complex_constraint(O, pos, prm) - O)) < 1e-12


def test_p9_clamp_and_uncovered_pixels():
    rng = _rng(15)
    O = _homogeneous(40, 50.0, rng) / np.exp(50.0)  # |ln A| / |phi| is large
    pos = np.array([(0, 0)])
    assert pe.cbar_per_position(O, pos, 16, 0.01, 10.0)[0] == 10.0
    O2 = _homogeneous(40, 1e-4, rng)
    assert pe.cbar_per_position(O2, pos, 16, 0.01, 10.0)[0] == 0.01
    prm = pe.Params(M=16, K=1, N=1, obj_h=40, obj_w=40, alpha1=1.0, alpha2=0.0)
    out = pe.complex_constraint(O2, pos, prm)
    assert np.array_equal(out[16:, :], O2[16:, :]) and np.array_equal(out[:, 16:], O2[:, 16:])
    # covered pixels: amplitude becomes exp(C phi) with the clamped C (Eq. 9, alpha1 = 1)
    assert np.max(np.abs(np.abs(out[:16, :16]) - np.exp(0.01 * np.angle(O2[:16, :16])))) < 1e-12


def test_p9_eq19_ratio_from_refractive_index():
    """Eqs. 15-19: A = exp(-2 pi / lambda beta tau), phi = -2 pi / lambda delta tau give ln A / phi = beta / delta."""
    lam, beta, delta = 0.5e-6, 2e-3, 8e-3
    tau = np.linspace(1e-6, 8e-6, 30 * 30).reshape(30, 30)
    phi = -2 * np.pi / lam * delta * tau
    phi = phi * (3.0 / np.abs(phi).max())  # keep the phase inside (-pi, pi]; the ratio is scale free
    A = np.exp(beta / delta * phi)
    cb = pe.cbar_per_position(A * np.exp(1j * phi), np.array([(0, 0)]), 30, 0.01, 10.0)
    assert abs(cb[0] - beta / delta) < 1e-12


# ------------------------------------------------------------------------ P10: error

def test_p10_error_zero_on_consistent_data_and_nonnegative():
    rng = _rng(16)
    M, side = 16, 24
    O = np.exp(1j * rng.random((side, side)))
    P = _crandn(rng, 1, M, M)
    pos = np.array([(0, 0), (8, 8)])
    prm = pe.Params(M=M, K=1, N=2, obj_h=side, obj_w=side, sigma1=1.0, sigma2=1.0)
    I = _consistent_data(O, P, pos, prm)
    _, _, E = pe.iterate(I, pos, O, P, prm, 1)
    assert E[0] < 1e-12
    _, _, E2 = pe.iterate(I * 1.3, pos, O, P, prm, 2)
    assert np.all(E2 > 0)
    # relative error of a pure rescale: Ihat = I / 1.3 against 1.3 I ... E = |1/1.3 - 1| / 1 relative to I
    assert abs(E2[0] - abs(1 / 1.3 - 1)) < 1e-9


# ------------------------------------------------------------------------ P11: worked examples from the paper

def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


def test_p11_table1_far_field_object_pixel():
    for lam_nm, px_um in _golden("table1_far_field_pixel.txt"):
        got = far_field_object_pixel(lam_nm * 1e-9, 35e-3, 1024, 6.5e-6) * 1e6
        assert round(got, 2) == px_um


def test_p11_qpt_phase():
    for lam_nm, phase in _golden("qpt_roi_phase.txt"):
        assert round(qpt_phase(lam_nm * 1e-9, 1.52, 205e-9), 2) == phase


def test_p11_electron_wavelength():
    for kv, pm in _golden("electron_wavelength.txt"):
        assert float(f"{electron_wavelength(kv * 1e3) * 1e12:.3g}") == pm


# ------------------------------------------------------------------------ P12: the paper's qualitative claim

@pytest.mark.parametrize("blur_domain,sigma", [("amplitude", 1.0), ("intensity", 2.0)])
def test_p12_pc_engine_beats_coherent_engine_on_blurred_data(blur_domain, sigma):
    """Sec. 3.1 (Figs. 3-4) and Sec. 4.2 (Fig. 7n): on data blurred by partial coherence, the engine
    with the Gaussian model ends at a lower intensity NRMSE than the coherent engine (sigma = 0)
    after the same number of iterations."""
    p = make_problem(0, scan_side=6, obj_side=144, sigma=sigma, dose=1e7)
    prm = pe.Params.from_dict(dict(p.params, sigma1=sigma, sigma2=sigma, blur_domain=blur_domain))
    prm0 = pe.Params.from_dict(dict(p.params, sigma1=0.0, sigma2=0.0))
    _, _, E_pc = pe.iterate(p.I, p.positions, p.O0, p.P0, prm, 20)
    _, _, E_c = pe.iterate(p.I, p.positions, p.O0, p.P0, prm0, 20)
    assert E_pc[-1] < 0.9 * E_c[-1]


def test_probe_update_starts_at_the_given_iteration():
    p = make_problem(0, scan_side=3, obj_side=96)
    prm = pe.Params.from_dict(dict(p.params, probe_update_start=2))
    O1, P1, _ = pe.iterate(p.I, p.positions, p.O0, p.P0, prm, 1)
    assert np.array_equal(P1, p.P0.astype(complex)) and not np.array_equal(O1, p.O0.astype(complex))
    _, P2, _ = pe.iterate(p.I, p.positions, p.O0, p.P0, prm, 2)
    assert not np.array_equal(P2, P1)


def test_windows_are_one_based_inclusive():
    assert pe.in_window(5, [(5, 35)]) and pe.in_window(35, [(5, 35)])
    assert not pe.in_window(4, [(5, 35)]) and not pe.in_window(36, [(5, 35)])


def test_dm_constraint_sits_between_the_steps_and_keeps_the_difference():
    """Inside a window the complex constraint acts on the object after the object step and before
    the probe step, and each state moves with its box: with the probe step off, O equals the
    constraint of the no-window result and psi_n - P o_n is the same with and without the window;
    with the probe step on, the probe step sees the constrained object."""
    rng = _rng(34)
    M, side = 16, 30
    O = (0.5 + rng.random((side, side))) * np.exp(1j * (rng.random((side, side)) - 0.5))
    P = _crandn(rng, 2, M, M)
    pos = np.array([(0, 0), (0, 14), (14, 0), (14, 14), (7, 7)])
    I = rng.random((len(pos), M, M)) * 10
    base = dict(M=M, K=2, N=len(pos), obj_h=side, obj_w=side, sigma1=0.8, sigma2=0.8, engine="dm",
                alpha1=1.0, alpha2=0.3)
    eps = pe.default_eps(I)
    for start, in ((10 ** 9,), (1,)):
        prm_w = pe.Params(**base, windows=[(1, 1)], probe_update_start=start)
        prm_n = pe.Params(**base, probe_update_start=start)
        g = pe.gaussian_kernel(prm_w.kernel_size, prm_w.sigma1, prm_w.sigma2)
        psi0 = np.stack([P * O[y:y + M, x:x + M][None] for y, x in pos])
        psi_w, psi_n = psi0.copy(), psi0.copy()
        Ow, Pw, Ew = pe.iteration_dm(I, pos, O, P, psi_w, prm_w, 1, eps, g)
        On, Pn, En = pe.iteration_dm(I, pos, O, P, psi_n, prm_n, 1, eps, g)
        assert Ew == En
        assert np.max(np.abs(Ow - On)) > 1e-3  # the constraint does something here
        if start > 1:
            assert np.array_equal(Ow, pe.complex_constraint(On, pos, prm_w)) and np.array_equal(Pw, P)
            for n, (y, x) in enumerate(pos):
                dw = psi_w[n] - P * Ow[y:y + M, x:x + M][None]
                dn = psi_n[n] - P * On[y:y + M, x:x + M][None]
                assert np.max(np.abs(dw - dn)) < 1e-10 * np.max(np.abs(dn))
        else:
            Oc = pe.complex_constraint(On, pos, prm_w)
            assert np.max(np.abs(Ow - Oc)) < 1e-13
            NP = sum(np.conj(Oc[y:y + M, x:x + M])[None] * (psi_n[n] - P * On[y:y + M, x:x + M][None])
                     for n, (y, x) in enumerate(pos))
            DP = sum(np.abs(Oc[y:y + M, x:x + M]) ** 2 for y, x in pos)
            c = pe.step_coefficients(prm_w)[1]
            ref = P + np.stack([pe._normalised_step(prm_w.beta_probe, NP[k], DP, *c) for k in range(2)])
            assert np.max(np.abs(Pw - ref)) < 1e-12 * np.max(np.abs(ref))
