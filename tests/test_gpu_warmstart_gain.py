"""GPU: what the trained warm start gains over the method without it.

The network is trained on the GPU (200k patterns from the library's own forward
model, its own forward / backward / Adam kernels) and then seeds the engine.

* Crystal with 1.0 rad phase peaks at 2e4 counts per pattern, engine with the
  intensity-blur model of Eq. 2: the warm start (network over 64 sampled patterns,
  stitched, median sigma) reaches an intensity NRMSE of 0.05 against the
  noise-free patterns in less GPU time than the flat start given the true sigma.
* The stated electron workload (0.1 rad peaks, 200 counts per pattern): the
  network recovers sigma (the quantity the paper's method otherwise needs as
  prior knowledge) within 10 % from the data alone. (There a flat start already
  sits at NRMSE 0.017, so a time-to-target comparison is empty.)
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _setup(dose, peak):
    from paper_2406_06640_gb300.warmstart import LatticeSpec, WarmStart, WarmStartConfig, subsample_scan
    from synth import make_problem

    dev = torch.device("cuda:0")
    pb = make_problem(4, dose=dose, peak=peak)
    prm = dict(pb.params)
    prm.pop("n_iter", None)
    M = prm["M"]
    I = torch.from_numpy(pb.I).to(dev)
    Ic = torch.from_numpy(pb.I_clean.astype(np.float32)).to(dev)
    pos = pb.positions.astype(np.int32)
    P0 = torch.from_numpy(pb.P0.reshape(1, M, M)).to(dev)
    net = WarmStart(P0[0], WarmStartConfig(S=M, C=32, batch=64, dose=dose, target_scale=peak,
                                           lattice=LatticeSpec(peak=peak), seed=1))
    net.train(200_000)
    idx = subsample_scan(pos, 16.0)
    return pb, prm, I, Ic, pos, P0, net, idx


def test_warm_start_reaches_target_sooner():
    from paper_2406_06640_gb300.warmstart import eval_kernel_size, time_to_nrmse

    pb, prm, I, Ic, pos, P0, net, idx = _setup(2e4, 1.0)
    s_true = pb.sim_sigma

    def engine(sig):
        return dict(prm, blur_domain="intensity", sigma1=sig, sigma2=sig, kernel_size=eval_kernel_size(sig))

    Isub = I[torch.from_numpy(idx).to(I.device)].contiguous()
    net.estimate(Isub, pos[idx], prm["obj_h"], prm["obj_w"])  # warm-up
    plain, warm = [], []
    for _ in range(3):
        O = torch.ones(prm["obj_h"], prm["obj_w"], dtype=torch.complex64, device=I.device)
        plain.append(time_to_nrmse(engine(s_true), I, Ic, pos, O, P0.clone(), s_true))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        Ow, sig = net.estimate(Isub, pos[idx], prm["obj_h"], prm["obj_w"])
        e1.record()
        e1.synchronize()
        r = time_to_nrmse(engine(sig), I, Ic, pos, Ow.clone(), P0.clone(), s_true)
        r["total_ms"] = e0.elapsed_time(e1) + r["engine_ms"]
        warm.append(r)
    net.close()
    assert all(r["reached"] for r in plain + warm)
    assert warm[0]["curve"][0][1] < plain[0]["curve"][0][1]  # a better start
    t_plain = np.median([r["engine_ms"] for r in plain])
    t_warm = np.median([r["total_ms"] for r in warm])
    assert t_warm < t_plain, (t_warm, t_plain, [r["curve"] for r in warm[:1]], [r["curve"] for r in plain[:1]])


def test_sigma_estimate_on_the_stated_electron_workload():
    pb, prm, I, Ic, pos, P0, net, idx = _setup(200.0, 0.1)
    Isub = I[torch.from_numpy(idx).to(I.device)].contiguous()
    _, sig = net.estimate(Isub, pos[idx], prm["obj_h"], prm["obj_w"])
    net.close()
    assert abs(sig - pb.sim_sigma) < 0.1 * pb.sim_sigma, sig
