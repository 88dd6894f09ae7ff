"""Seeded input generators: shapes, determinism, scan geometry (CPU only)."""
import numpy as np

from synth import make_problem
from synth.generators import cfg3_members, make_cfg3_member


def test_cfg0_shapes_and_determinism():
    a = make_problem(0)
    b = make_problem(0)
    assert a.I.shape == (100, 64, 64) and a.I.dtype == np.float32
    assert a.positions.shape == (100, 2) and a.positions.dtype == np.int32
    assert a.O0.shape == (192, 192) and a.P0.shape == (1, 64, 64)
    assert np.array_equal(a.I, b.I) and np.array_equal(a.positions, b.positions)
    assert a.positions.min() >= 0 and a.positions.max() <= 192 - 64
    assert abs(a.I.sum((1, 2)).mean() - 1e5) < 2e3  # dose
    assert np.all(a.I == np.round(a.I))  # Poisson counts


def test_cfg0_jitter_is_integer_and_bounded():
    a = make_problem(0)
    grid = np.array([(10 + 12 * i, 10 + 12 * j) for i in range(10) for j in range(10)])
    assert np.max(np.abs(a.positions - grid)) <= 1


def test_small_variants_and_modes():
    p = make_problem(0, scan_side=3, obj_side=96, M=32, K=3, geometry="near")
    assert p.I.shape == (9, 32, 32) and p.P0.shape == (3, 32, 32)
    assert p.params["geometry"] == "near" and p.params["fresnel_F"] == 10.0
    # extra modes at 10 % amplitude
    assert np.allclose(np.abs(p.P0[1]), 0.1 * np.abs(p.P0[0]), atol=1e-6)


def test_cfg3_descriptors():
    d = cfg3_members()
    assert len(d) == 64
    assert {m for m, *_ in d} <= {64, 128, 256}
    assert all(100 <= n <= 1600 for _, _, n, _, _ in d)
    p = make_cfg3_member(0, N=20, M=64)
    assert p.I.shape == (20, 64, 64)
    assert p.positions.max() + 64 <= p.params["obj_h"]
