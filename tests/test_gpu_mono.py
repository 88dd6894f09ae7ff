"""GPU parity of numerical monochromatisation (Sec. 4.2, Eqs. 12-13): the CUDA CGLS (through the
C ABI) against the FP64 oracle on seeded synthetic patterns.

Tolerance: relative L2 1e-4 per pattern for x and for the residual norms. The arithmetic is FP32
with FP64 step sizes and norms; the same CGLS run in FP32 numpy stays within 2e-7 (5-line
spectrum, k = 40) and 6e-6 (32 lines over a factor 1.75, k = 40) of FP64 on the benchmark's
patterns, so 1e-4 leaves room for the different summation orders of the GPU.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mono  # noqa: E402
from synth import make_problem  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-4
LINES5 = [1.0, 1.0125, 1.025, 1.0375, 1.05]  # 5 % bandwidth about the shortest wavelength
WHITE32 = list(np.linspace(1.0, 1.75, 32))   # 400-700 nm about 400 nm


def _dev():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return torch.device("cuda:0")


def run_gpu(B, scales, weights, k, clamp=False, inplace=False):
    from paper_2406_06640_gb300.engine import monochromatise

    b = torch.from_numpy(np.ascontiguousarray(B, dtype=np.float32)).to(_dev())
    if inplace:
        x, res = monochromatise(b, scales, weights, k, clamp=clamp, out=b, with_residuals=True)
    else:
        x, res = monochromatise(b, scales, weights, k, clamp=clamp, with_residuals=True)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.float64), res.cpu().numpy()


def check(B, scales, weights, k, tol=TOL, clamp=False):
    Xg, Rg = run_gpu(B, scales, weights, k, clamp)
    Xo, Ro = mono.monochromatise(B.astype(np.float64), scales, weights, k, clamp)
    for n in range(B.shape[0]):
        den = np.linalg.norm(Xo[n])
        ex = np.linalg.norm(Xg[n] - Xo[n]) / den if den > 0 else np.linalg.norm(Xg[n])
        er = np.max(np.abs(Rg[n] - Ro[n]) / Ro[n])
        assert ex <= tol and er <= tol, (n, ex, er)
    return Xg, Rg


def _patterns(cfg, count, **kw):
    return make_problem(cfg, **kw).I[:count].astype(np.float64)


@pytest.mark.parametrize("k", [0, 1, 6, 25])
def test_benchmark_patterns_five_lines(k):
    """Patterns of the 128^2 benchmark problem (generated with this 5-line spectrum)."""
    B = _patterns(1, 4)
    check(B, LINES5, [0.2] * 5, k)


def test_white_light_32_lines():
    B = _patterns(1, 3)
    w = np.exp(-0.5 * ((np.array(WHITE32) - 1.3) / 0.2) ** 2)
    check(B, WHITE32, w, 25)


@pytest.mark.parametrize("M", [8, 16, 32, 64])
def test_probe_sizes_and_scales_below_one(M):
    """Every pattern size, a spectrum on both sides of the reference (samples outside the grid
    blend toward zero) and the widest scale accepted (2.5)."""
    rng = np.random.default_rng(M)
    B = rng.random((5, M, M)) * 100
    check(B, [0.8, 0.95, 1.0, 1.3, 2.5], [0.1, 0.3, 0.3, 0.2, 0.1], 5)


@pytest.mark.parametrize("scales,weights,k", [([1.0, 1.05, 1.1], [0.5, 0.3, 0.2], 6),
                                              ([0.8, 1.0, 1.4, 2.5], [0.2, 0.4, 0.3, 0.1], 4)])
def test_m256_cluster_of_four_bands(scales, weights, k):
    """256^2 patterns: one cluster of four CTAs per pattern (64-row bands, neighbours read across
    bands, CTA sums combined in rank order); scales on both sides of 1 and the widest accepted."""
    rng = np.random.default_rng(256)
    B = rng.random((3, 256, 256)) * 50
    check(B, scales, weights, k)


def test_monochromatic_light_is_exact_and_clamp():
    rng = np.random.default_rng(3)
    B = rng.standard_normal((3, 32, 32)).astype(np.float32).astype(np.float64)
    X, R = run_gpu(B, [1.0], [1.0], 1)
    assert np.array_equal(X, B)
    assert np.all(R[:, 1] <= 1e-6 * R[:, 0])
    Xc, _ = run_gpu(B, [1.0], [1.0], 1, clamp=True)
    assert np.array_equal(Xc, np.maximum(B, 0.0))


def test_deterministic_and_in_place():
    B = _patterns(1, 6)
    a = run_gpu(B, WHITE32[:12], [1.0] * 12, 8)
    b = run_gpu(B, WHITE32[:12], [1.0] * 12, 8)
    c = run_gpu(B, WHITE32[:12], [1.0] * 12, 8, inplace=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1])


def test_empty_batch_and_invalid_arguments():
    from paper_2406_06640_gb300.binding import PtychoError
    from paper_2406_06640_gb300.engine import monochromatise

    dev = _dev()
    b = torch.zeros((0, 64, 64), dtype=torch.float32, device=dev)
    assert monochromatise(b, [1.0], [1.0], 3).shape == (0, 64, 64)
    b = torch.zeros((1, 64, 64), dtype=torch.float32, device=dev)
    for scales, weights in (([3.0], [1.0]), ([1.0], [0.0]), ([1.0, 1.1], [1.0, -1.0]), ([0.0], [1.0])):
        with pytest.raises(PtychoError):
            monochromatise(b, scales, weights, 3)
    with pytest.raises(PtychoError):
        monochromatise(torch.zeros((1, 48, 48), dtype=torch.float32, device=dev), [1.0], [1.0], 3)
    with pytest.raises(PtychoError):
        monochromatise(torch.zeros((1, 512, 512), dtype=torch.float32, device=dev), [1.0], [1.0], 3)


def test_full_size_sampled():
    """The benchmark launch (900 patterns of 128^2, 32 lines, k = 25) against the oracle on sampled
    patterns, and the residual norms non-increasing for every pattern."""
    p = make_problem(1)
    w = [1.0 / 32] * 32
    Xg, Rg = run_gpu(p.I, WHITE32, w, 25)
    assert np.all(np.diff(Rg, axis=1) <= 1e-6 * Rg[:, :1])
    for n in (0, 451, 899):
        Xo, Ro = mono.cgls(p.I[n].astype(np.float64), mono.spectrum_operator(128, WHITE32, w), 25)
        assert np.linalg.norm(Xg[n] - Xo) <= TOL * np.linalg.norm(Xo)
        assert np.max(np.abs(Rg[n] - Ro) / Ro) <= TOL
