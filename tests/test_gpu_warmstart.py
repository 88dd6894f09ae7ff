"""GPU: the learned warm start against its FP64 oracles.

* U-Net forward and every parameter gradient through the C ABI against
  oracle/unet.py with bf16 rounding at the points the GPU stores bf16. Tolerance
  2e-3 relative L2: the GPU accumulates in FP32 (about sqrt(K) 2^-24 ~ 3e-6
  relative), so a fraction ~3e-6 / 2^-8 ~ 1e-3 of the bf16 roundings land on the
  other side of a tie-free boundary (one bf16 ulp = 2^-8 relative); through
  seven layers that is a few 1e-4 relative L2.
* The forward-model generator (noise off) against oracle/warmstart.py: clean
  patterns within 1e-4 relative L2 (FP32 FFT of S^2 points), targets within 4e-4
  absolute (a site at exactly the cutoff radius may be kept on one side only:
  0.1 rad e^-8 / 0.1 = 3.4e-4).
* Poisson counts: moments of the pattern totals and of standardised residuals.
* The stitched warm start and the median sigma against the oracle's stitch of
  the oracle network's outputs.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import unet as ou  # noqa: E402
from oracle import warmstart as ows  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _pg():
    import paper_2406_06640_gb300 as pg

    return pg


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).to(DEV).contiguous()


def _flat(params, C):
    parts = []
    for i in range(7):
        parts += [params[f"w{i}"].ravel(), params[f"b{i}"].ravel()]
    parts += [params["w7"].ravel(), params["b7"].ravel()]
    return np.concatenate(parts).astype(np.float32)


def _unflat(flat, C):
    out, off = {}, 0
    for i, (ci, co) in enumerate(ou.layer_shapes(C)):
        out[f"w{i}"] = flat[off:off + co * 9 * ci].reshape(co, 9, ci)
        off += co * 9 * ci
        out[f"b{i}"] = flat[off:off + co]
        off += co
    out["w7"] = flat[off:off + 8 * C]
    out["b7"] = flat[off + 8 * C:off + 8 * C + 1]
    return out


def _params32(C, seed):
    p = ou.init_params(C, seed)
    return {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-30))


TOL = 2e-3


def test_unet_parameter_layout_roundtrip():
    pg = _pg()
    C = 16
    net = pg.UNet(32, C, 8, seed=3)
    n = net.param_count()
    p = _params32(C, 5)
    assert n == sum(v.size for v in p.values())
    flat = _flat(p, C)
    net.set_params(flat)
    back = net.get_params(np.zeros(n, np.float32))
    assert np.array_equal(back, flat)
    net.close()


@pytest.mark.parametrize("S,C,n", [(32, 16, 8), (64, 16, 2)])
def test_unet_forward_and_gradients_match_oracle(S, C, n):
    pg = _pg()
    rng = np.random.default_rng(S + n)
    params = _params32(C, 11)
    x = np.log1p(rng.poisson(1.5, (n, S, S))).astype(np.float32) / 4
    target = (0.5 * rng.standard_normal((n, S // 2, S // 2, 2))).astype(np.float32)
    sigma_t = rng.uniform(0.5, 3.0, n).astype(np.float32)
    lam = 0.1
    loss_o, g_o, out_o, sig_o = ou.loss_and_grads(params, x[..., None].astype(np.float64),
                                                  target.astype(np.float64), sigma_t.astype(np.float64), lam,
                                                  bf16=True)
    net = pg.UNet(S, C, n, seed=0)
    net.set_params(_flat(params, C))
    xd, td, sd = _dev(x), _dev(target), _dev(sigma_t)
    out = torch.zeros(n, S // 2, S // 2, 2, device=DEV)
    sig = torch.zeros(n, device=DEV)
    net.forward(xd.data_ptr(), out.data_ptr(), sig.data_ptr())
    assert _rel(out.cpu().numpy(), out_o) < TOL
    assert _rel(sig.cpu().numpy(), sig_o) < TOL
    grads = np.zeros(net.param_count(), np.float32)
    loss = net.gradients(xd.data_ptr(), td.data_ptr(), sd.data_ptr(), lam, grads)
    assert abs(loss - loss_o) / loss_o < TOL
    g = _unflat(grads, C)
    for k in g_o:
        assert _rel(g[k], g_o[k]) < TOL, (k, _rel(g[k], g_o[k]))
    net.close()


def test_train_step_is_adam_on_the_gradients():
    pg = _pg()
    S, C, n = 32, 16, 8
    rng = np.random.default_rng(7)
    params = _params32(C, 13)
    x = np.log1p(rng.poisson(1.0, (n, S, S))).astype(np.float32) / 4
    target = (0.3 * rng.standard_normal((n, S // 2, S // 2, 2))).astype(np.float32)
    sigma_t = rng.uniform(0.5, 3.0, n).astype(np.float32)
    net = pg.UNet(S, C, n, seed=0)
    flat = _flat(params, C)
    net.set_params(flat)
    xd, td, sd = _dev(x), _dev(target), _dev(sigma_t)
    grads = np.zeros(net.param_count(), np.float32)
    net.gradients(xd.data_ptr(), td.data_ptr(), sd.data_ptr(), 0.1, grads)
    lr = 1e-3
    net.train_step(xd.data_ptr(), td.data_ptr(), sd.data_ptr(), 0.1, lr)
    after = net.get_params(np.zeros_like(flat))
    # first Adam step: m / (1 - b1) = g, v / (1 - b2) = g^2, so each weight moves by lr g / (|g| + 1e-8)
    g = grads.astype(np.float64)
    expect = flat - lr * g / (np.abs(g) + 1e-8)
    assert np.allclose(after, expect, rtol=0, atol=2e-6)
    net.close()


def _probe(S, rng):
    k = np.fft.fftshift(np.fft.fftfreq(S))
    k2 = k[:, None] ** 2 + k[None, :] ** 2
    ap = (np.sqrt(k2) <= 0.25).astype(np.float64)
    P = np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(ap * np.exp(-1j * 40.0 * k2))))
    return (P / np.abs(P).max()).astype(np.complex64)


SPEC = dict(dose=200.0, lattice_a=16.0, peak=0.1, peak_sd=1.5, cutoff=6.0, vacancy=0.05, target_scale=0.1,
            key=0x0123456789ABCDEF)


@pytest.mark.parametrize("S", [64, 128])
def test_generator_matches_oracle(S):
    pg = _pg()
    rng = np.random.default_rng(S)
    n, first = 5, 1000
    P = _probe(S, rng)
    prm = np.stack([rng.uniform(0, np.pi / 3, n), rng.uniform(0, 16, n), rng.uniform(0, 16, n),
                    np.array([0.0, 0.5, 1.3, 2.0, 3.0])], axis=1).astype(np.float32)
    spec = dict(SPEC, S=S, noise=0)
    Pd = _dev(P.view(np.float32).reshape(S, S, 2))
    prmd = _dev(prm)
    clean = torch.zeros(n, S, S, device=DEV)
    counts = torch.zeros(n, S, S, device=DEV)
    x = torch.zeros(n, S, S, device=DEV)
    target = torch.zeros(n, S // 2, S // 2, 2, device=DEV)
    sig = torch.zeros(n, device=DEV)
    pg.generate(spec, Pd.data_ptr(), prmd.data_ptr(), n, first, x.data_ptr(), counts.data_ptr(), clean.data_ptr(),
                target.data_ptr(), sig.data_ptr())
    torch.cuda.synchronize()
    clean, counts, x, target, sig = (t.cpu().numpy() for t in (clean, counts, x, target, sig))
    assert np.array_equal(sig, prm[:, 3])
    assert np.array_equal(counts, clean)
    assert np.allclose(x, 0.25 * np.log1p(clean.astype(np.float64)), rtol=1e-6, atol=1e-7)
    for i in range(n):
        th, oy, ox, s = (float(v) for v in prm[i])
        phi = ows.lattice_phase(S, th, oy, ox, first + i, SPEC["key"], a=16.0, peak=0.1, s_pk=1.5, cutoff=6.0,
                                vacancy=0.05)
        ref = ows.clean_pattern(P.astype(np.complex128), phi, s, 200.0)
        assert _rel(clean[i], ref) < 1e-4, (i, _rel(clean[i], ref))
        tref = ows.target_patch(phi, 0.1)
        assert np.abs(target[i] - tref).max() < 4e-4


def test_generator_poisson_statistics_and_determinism():
    pg = _pg()
    S, n = 64, 512
    rng = np.random.default_rng(9)
    P = _probe(S, rng)
    prm = np.stack([rng.uniform(0, np.pi / 3, n), rng.uniform(0, 16, n), rng.uniform(0, 16, n),
                    rng.uniform(0.5, 3.0, n)], axis=1).astype(np.float32)
    Pd, prmd = _dev(P.view(np.float32).reshape(S, S, 2)), _dev(prm)
    counts = torch.zeros(n, S, S, device=DEV)
    clean = torch.zeros(n, S, S, device=DEV)
    pg.generate(dict(SPEC, S=S, noise=1), Pd.data_ptr(), prmd.data_ptr(), n, 0, counts=counts.data_ptr(),
                clean=clean.data_ptr())
    again = torch.zeros_like(counts)
    pg.generate(dict(SPEC, S=S, noise=1), Pd.data_ptr(), prmd.data_ptr(), n, 0, counts=again.data_ptr())
    other = torch.zeros_like(counts)
    pg.generate(dict(SPEC, S=S, noise=1), Pd.data_ptr(), prmd.data_ptr(), n, 7, counts=other.data_ptr())
    torch.cuda.synchronize()
    c = counts.cpu().numpy().astype(np.float64)
    assert torch.equal(counts, again) and not torch.equal(counts, other)
    assert np.all(c >= 0) and np.array_equal(c, np.round(c))
    tot = c.reshape(n, -1).sum(axis=1)  # Poisson(200) per pattern
    assert abs(tot.mean() - 200.0) < 5 * np.sqrt(200.0 / n)
    assert 0.75 < tot.var() / 200.0 < 1.25
    # high dose: the transformed-rejection branch, standardised residuals ~ (0, 1)
    hi = torch.zeros(64, S, S, device=DEV)
    hic = torch.zeros(64, S, S, device=DEV)
    pg.generate(dict(SPEC, S=S, noise=1, dose=2e6), Pd.data_ptr(), prmd.data_ptr(), 64, 0, counts=hi.data_ptr(),
                clean=hic.data_ptr())
    torch.cuda.synchronize()
    lam = hic.cpu().numpy().astype(np.float64)
    k = hi.cpu().numpy().astype(np.float64)
    m = lam >= 10
    assert m.sum() > 10000
    z = (k[m] - lam[m]) / np.sqrt(lam[m])
    assert abs(z.mean()) < 0.05 and 0.9 < z.var() < 1.1
    # mid dose: the inversion branch (means below 10)
    pg.generate(dict(SPEC, S=S, noise=1, dose=5e3), Pd.data_ptr(), prmd.data_ptr(), 64, 0, counts=hi.data_ptr(),
                clean=hic.data_ptr())
    torch.cuda.synchronize()
    lam = hic.cpu().numpy().astype(np.float64)
    k = hi.cpu().numpy().astype(np.float64)
    ms = (lam > 0.5) & (lam < 10)
    zs = (k[ms] - lam[ms]) / np.sqrt(lam[ms])
    assert ms.sum() > 10000 and abs(zs.mean()) < 0.05 and 0.9 < zs.var() < 1.1


def test_warmstart_matches_oracle_stitch():
    pg = _pg()
    S, C, batch, N = 32, 16, 8, 21  # a ragged last batch
    obj_h, obj_w = 80, 72
    rng = np.random.default_rng(21)
    params = _params32(C, 17)
    I = rng.poisson(2.0, (N, S, S)).astype(np.float32)
    pos = np.stack([rng.integers(0, obj_h - S + 1, N), rng.integers(0, obj_w - S + 1, N)], axis=1).astype(np.int32)
    net = pg.UNet(S, C, batch, seed=0)
    net.set_params(_flat(params, C))
    Id = _dev(I)
    O = torch.zeros(obj_h, obj_w, 2, device=DEV)
    sigma_est = net.warmstart(Id.data_ptr(), pos.ctypes.data, N, obj_h, obj_w, 0.1, O.data_ptr())
    x = np.log1p(I.astype(np.float64)) / 4
    out_o, sig_o, _ = ou.forward(params, x[..., None], bf16=True)
    ref = ows.stitch(out_o, pos + S // 4, obj_h, obj_w, 0.1)
    got = O.cpu().numpy().astype(np.float64)
    got = got[..., 0] + 1j * got[..., 1]
    assert _rel(got, ref) < TOL
    covered = np.zeros((obj_h, obj_w), bool)
    for r, c in pos:
        covered[r + S // 4:r + 3 * S // 4, c + S // 4:c + 3 * S // 4] = True
    assert np.all(got[~covered] == 1)
    assert abs(sigma_est - ows.median(sig_o)) < TOL * abs(ows.median(sig_o))
    net.close()


def test_training_reduces_loss_on_generated_data():
    pg = _pg()
    S, C, n = 64, 16, 32
    rng = np.random.default_rng(5)
    P = _probe(S, rng)
    Pd = _dev(P.view(np.float32).reshape(S, S, 2))
    net = pg.UNet(S, C, n, seed=1)
    x = torch.zeros(n, S, S, device=DEV)
    target = torch.zeros(n, S // 2, S // 2, 2, device=DEV)
    sig = torch.zeros(n, device=DEV)
    losses = []
    # a dose high enough that the patterns carry the lattice clearly (the loss reaches its floor
    # in about 100 steps of Adam at 1e-3)
    for step in range(120):
        prm = np.stack([rng.uniform(0, np.pi / 3, n), rng.uniform(0, 16, n), rng.uniform(0, 16, n),
                        rng.uniform(0.5, 3.0, n)], axis=1).astype(np.float32)
        pg.generate(dict(SPEC, S=S, noise=1, dose=2e4), Pd.data_ptr(), _dev(prm).data_ptr(), n, step * n,
                    x=x.data_ptr(), target=target.data_ptr(), sigma=sig.data_ptr())
        losses.append(net.train_step(x.data_ptr(), target.data_ptr(), sig.data_ptr(), 0.1, 1e-3, want_loss=True))
    assert np.all(np.isfinite(losses))
    assert np.mean(losses[-20:]) < 0.5 * np.mean(losses[:10]), (losses[:10], losses[-20:])
    net.close()
