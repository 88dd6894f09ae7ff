"""Pins of the warm-start oracle (generator, stitch, median) against facts fixed
independently of it: the published Philox known-answer vectors, closed forms of a
single Gaussian peak, lattice symmetries, the DFT definition, Parseval and the
window algebra of the stitch."""
import math
import os

import numpy as np
import pytest

from oracle import warmstart as ws

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        w = [int(v, 16) for v in r]
        out = ws.philox4x32_10(w[:4], w[4:6])
        assert [int(v) for v in out] == w[6:10]


def test_philox_vectorised_matches_scalar():
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2 ** 32, size=(7, 4), dtype=np.uint64)
    key = (0x12345678, 0x9ABCDEF0)
    many = ws.philox4x32_10(ctr, key)
    for i in range(7):
        assert np.array_equal(many[i], ws.philox4x32_10(ctr[i], key))


def test_philox_uniformity():
    ctr = np.stack([np.arange(20000), np.zeros(20000), np.full(20000, 3), np.ones(20000)], axis=-1)
    w = ws.philox4x32_10(ctr.astype(np.uint64), (7, 0)).astype(np.float64) / 2 ** 32
    assert abs(w.mean() - 0.5) < 0.005
    assert abs(w.var() - 1 / 12) < 0.002


def test_single_peak_closed_form():
    # a lattice constant far larger than the box leaves the one site at the origin
    S, oy, ox, s_pk, cut = 32, 15.25, 16.5, 1.5, 6.0
    phi = ws.lattice_phase(S, 0.3, oy, ox, 0, 0, a=1000.0, peak=0.1, s_pk=s_pk, cutoff=cut, vacancy=0.0)
    y, x = np.mgrid[0:S, 0:S].astype(np.float64)
    d2 = (y - oy) ** 2 + (x - ox) ** 2
    ref = np.where(d2 <= cut * cut, 0.1 * np.exp(-d2 / (2 * s_pk * s_pk)), 0.0)
    assert np.allclose(phi, ref, rtol=0, atol=1e-15)
    assert phi.max() <= 0.1 and phi[(d2 > cut * cut)].max() == 0.0


def test_lattice_symmetries():
    S, a = 48, 16.0
    base = ws.lattice_phase(S, 0.2, 3.0, 5.0, 0, 0, a=a, vacancy=0.0)
    # a hexagonal lattice is unchanged by a 60-degree rotation of its basis and by a lattice translation
    rot = ws.lattice_phase(S, 0.2 + math.pi / 3, 3.0, 5.0, 0, 0, a=a, vacancy=0.0)
    a1, _ = ws.lattice_basis(a, 0.2)
    shift = ws.lattice_phase(S, 0.2, 3.0 + a1[0], 5.0 + a1[1], 0, 0, a=a, vacancy=0.0)
    assert np.allclose(base, rot, atol=1e-12)
    assert np.allclose(base, shift, atol=1e-12)
    # peaks sit on the sites: phase at a site far from the edges equals the peak height
    # (neighbours lie a = 16 px > cutoff away)
    p = np.array([3.0, 5.0]) + 2 * a1 + ws.lattice_basis(a, 0.2)[1]
    field = ws.lattice_phase(S, 0.2, 3.0 - (p[0] - round(p[0])), 5.0 - (p[1] - round(p[1])), 0, 0, a=a, vacancy=0.0)
    assert abs(field[int(round(p[0])), int(round(p[1]))] - 0.1) < 1e-12


def test_vacancies_follow_threshold():
    S = 256
    full = ws.lattice_phase(S, 0.1, 0.0, 0.0, 5, 99, a=16.0, vacancy=0.0)
    none = ws.lattice_phase(S, 0.1, 0.0, 0.0, 5, 99, a=16.0, vacancy=1.0)
    assert none.max() == 0.0 and full.max() > 0.09
    part = ws.lattice_phase(S, 0.1, 0.0, 0.0, 5, 99, a=16.0, vacancy=0.3)
    # the surviving peak mass is about 70 % of the full lattice
    frac = part.sum() / full.sum()
    assert 0.6 < frac < 0.8
    assert ws.vacancy_threshold(1.0) == 2 ** 32 - 1 and ws.vacancy_threshold(0.0) == 0


def test_blur_taps():
    for s in (0.5, 1.0, 2.0, 3.0, 4.0):
        g = ws.blur_taps(s)
        h = (len(g) - 1) // 2
        assert h == min(math.ceil(5 * s), 15)
        assert abs(g.sum() - 1) < 1e-15 and np.allclose(g, g[::-1])
    assert np.array_equal(ws.blur_taps(0.0), [1.0])


def test_clean_pattern_against_dft_definition():
    S = 8
    rng = np.random.default_rng(3)
    P = rng.standard_normal((S, S)) + 1j * rng.standard_normal((S, S))
    phi = rng.uniform(0, 0.3, (S, S))
    psi = P * np.exp(1j * phi)
    ref = np.zeros((S, S))
    for u in range(S):
        for v in range(S):
            acc = 0j
            for y in range(S):
                for x in range(S):
                    acc += psi[y, x] * np.exp(-2j * np.pi * ((u - S // 2) * y + (v - S // 2) * x) / S)
            ref[u, v] = abs(acc) ** 2
    ref *= 123.0 / ref.sum()
    assert np.allclose(ws.clean_pattern(P, phi, 0.0, 123.0), ref, rtol=1e-12, atol=1e-12)
    # blur keeps the mean inside the support; the sum is the dose
    I = ws.clean_pattern(np.ones((32, 32)), np.zeros((32, 32)), 1.0, 200.0)
    assert abs(I.sum() - 200.0) < 1e-9
    # a flat probe and object give a single bright pixel at the centre, then the blur
    g = ws.blur_taps(1.0)
    assert np.allclose(I[16 - 5:16 + 6, 16], 200.0 * g[:, None][:, 0] * g[5])


def test_stitch_algebra():
    Q, scale = 8, 0.1
    rng = np.random.default_rng(4)
    # identical constant patches reproduce the constant on covered pixels, 1 elsewhere
    val = np.array([0.3, -0.7])
    patches = np.broadcast_to(val, (5, Q, Q, 2)).copy()
    corners = rng.integers(0, 20, size=(5, 2))
    out = ws.stitch(patches, corners, 32, 32, scale)
    cov = np.zeros((32, 32), bool)
    for r, c in corners:
        cov[r:r + Q, c:c + Q] = True
    assert np.allclose(out[cov], np.exp(scale * (val[0] + 1j * val[1])))
    assert np.all(out[~cov] == 1)
    # two overlapping patches: the Hann-weighted mean, written out at one pixel
    p2 = rng.standard_normal((2, Q, Q, 2))
    c2 = np.array([[0, 0], [3, 2]])
    out = ws.stitch(p2, c2, 16, 16, scale)
    y, x = 5, 4
    w0 = math.sin(math.pi * (y + 0.5) / Q) ** 2 * math.sin(math.pi * (x + 0.5) / Q) ** 2
    w1 = math.sin(math.pi * (y - 3 + 0.5) / Q) ** 2 * math.sin(math.pi * (x - 2 + 0.5) / Q) ** 2
    v0 = np.exp(scale * (p2[0, y, x, 0] + 1j * p2[0, y, x, 1]))
    v1 = np.exp(scale * (p2[1, y - 3, x - 2, 0] + 1j * p2[1, y - 3, x - 2, 1]))
    assert abs(out[y, x] - (w0 * v0 + w1 * v1) / (w0 + w1)) < 1e-14


def test_median_small_cases():
    assert ws.median([3.0]) == 3.0
    assert ws.median([5.0, 1.0, 3.0]) == 3.0
    assert ws.median([4.0, 1.0, 3.0, 2.0]) == 2.5
    assert ws.median([2.0, 2.0, 9.0, -1.0, 7.0, 2.0]) == 2.0


def test_target_patch():
    phi = np.arange(64.0).reshape(8, 8)
    t = ws.target_patch(phi, 0.5)
    assert t.shape == (4, 4, 2) and np.all(t[..., 0] == 0)
    assert np.array_equal(t[..., 1], phi[2:6, 2:6] / 0.5)
