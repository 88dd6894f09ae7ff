"""GPU: batched reconstructions of uneven sizes (ptycho_plan_batch / ptycho_iterate_batch).

Each problem in a batch is an independent reconstruction; replaying the
batch's CUDA graph must give exactly the result of running every problem
through its own plan (same kernels, fixed reduction orders), across graph
re-use and call splits, and therefore the oracle's result within 1e-4.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from synth import make_problem  # noqa: E402

pytestmark = pytest.mark.gpu


def _problems():
    out = []
    p = make_problem(0, scan_side=3, obj_side=96, M=32, K=2, sigma=1.0)
    out.append((p, dict(p.params, windows=[(2, 3)])))
    p = make_problem(0, scan_side=4, obj_side=160, M=64, K=1, geometry="near", sigma=1.5)
    out.append((p, dict(p.params, sigma1=1.5, sigma2=1.5)))
    p = make_problem(0, scan_side=3, obj_side=224, M=128, K=4, sigma=1.5)
    out.append((p, dict(p.params, sigma1=1.5, sigma2=1.5)))
    p = make_problem(0, scan_side=2, obj_side=320, M=256, K=2, geometry="near", sigma=2.0)
    out.append((p, dict(p.params, sigma1=2.0, sigma2=2.0)))
    p = make_problem(0, scan_side=3, obj_side=128, M=64, K=3, sigma=1.2)
    out.append((p, dict(p.params, blur_domain="intensity", probe_update_start=2, windows=[(1, 1)])))
    return out


def _tensors(dev, prob):
    return (torch.from_numpy(prob.I).to(dev), torch.from_numpy(prob.O0.astype(np.complex64)).to(dev),
            torch.from_numpy(prob.P0.astype(np.complex64)).to(dev))


def test_batch_matches_individual_plans_and_oracle():
    from paper_2406_06640_gb300.engine import Reconstruction, ReconstructionBatch

    dev = torch.device("cuda:0")
    probs = _problems()
    n_iter = 4
    # individual plans
    single = []
    for prob, prm in probs:
        I, O, P = _tensors(dev, prob)
        rec = Reconstruction(prm, I, prob.positions)
        rec.iterate(O, P, n_iter)
        single.append((O.cpu().numpy(), P.cpu().numpy(), rec.errors(n_iter)[-1]))
        rec.close()
    # batch, run as 1 + 3 iterations (the graph is captured once per window / probe-update pattern)
    tens = [_tensors(dev, prob) for prob, _ in probs]
    batch = ReconstructionBatch([(prm, t[0], prob.positions) for (prob, prm), t in zip(probs, tens)])
    objs, prbs = [t[1] for t in tens], [t[2] for t in tens]
    batch.iterate(objs, prbs, 1)
    batch.iterate(objs, prbs, n_iter - 1)
    E = batch.errors()
    for b, (O1, P1, E1) in enumerate(single):
        assert np.array_equal(objs[b].cpu().numpy(), O1), b
        assert np.array_equal(prbs[b].cpu().numpy(), P1), b
        assert E[b] == E1, b
    batch.close()
    # oracle on two members
    for b in (0, 4):
        prob, prm = probs[b]
        Oo, Po, Eo = oracle.iterate(prob.I, prob.positions, prob.O0, prob.P0, oracle.Params.from_dict(prm), n_iter)
        rel = lambda a, c: np.linalg.norm(a - c) / np.linalg.norm(c)  # noqa: E731
        assert rel(single[b][0], Oo) < 1e-4 and rel(single[b][1], Po) < 1e-4
        assert abs(single[b][2] - Eo[-1]) / Eo[-1] < 1e-4


def test_batch_rejects_single_plan_calls():
    from paper_2406_06640_gb300 import PtychoError
    from paper_2406_06640_gb300.engine import ReconstructionBatch

    dev = torch.device("cuda:0")
    prob, prm = _problems()[0]
    I, O, P = _tensors(dev, prob)
    batch = ReconstructionBatch([(prm, I, prob.positions)])
    with pytest.raises(PtychoError):
        batch._plan.errors()  # nothing has run yet
    batch.iterate([O], [P], 1)
    assert len(batch.errors()) == 1
    batch.close()
