"""Pins of the warm-start network oracle (oracle/unet.py) on the CPU: the analytic gradients equal
central finite differences of the FP64 loss, and the bfloat16 rounding equals torch's."""
import numpy as np
import pytest

from oracle import unet as U


def _case(seed=0, S=16, C=4, n=2):
    rng = np.random.default_rng(seed)
    params = U.init_params(C, seed)
    x = rng.random((n, S, S, 1))
    target = rng.standard_normal((n, S // 2, S // 2, 2)) * 0.3
    sig = rng.uniform(0.5, 3.0, n)
    return params, x, target, sig


def test_shapes():
    params, x, target, sig = _case()
    out, sigma, _ = U.forward(params, x)
    assert out.shape == (2, 8, 8, 2) and sigma.shape == (2,)


@pytest.mark.parametrize("name", ["w0", "b0", "w1", "w2", "w3", "b3", "w4", "w5", "w6", "b6", "w7", "b7"])
def test_gradients_match_central_differences(name):
    params, x, target, sig = _case(seed=1)
    loss, g, _, _ = U.loss_and_grads(params, x, target, sig)
    rng = np.random.default_rng(7)
    flat = params[name].ravel()
    gflat = g[name].ravel()
    for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
        h = 1e-6
        old = flat[idx]
        flat[idx] = old + h
        lp, _, _, _ = U.loss_and_grads(params, x, target, sig)
        flat[idx] = old - h
        lm, _, _, _ = U.loss_and_grads(params, x, target, sig)
        flat[idx] = old
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[idx]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, (name, idx, fd, gflat[idx])


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    v = np.random.default_rng(3).standard_normal(10000) * 10
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(U.bf16_round(v), ref)
