"""GPU: batched reconstructions of uneven sizes (ptycho_plan_batch / ptycho_iterate_batch).

Members with M in {32, 64, 128} are drained by one persistent work-queue launch per
shape class (M, K, geometry, kernel width): chunks of 16 positions from every
problem of the class, each chunk with its own probe / error partials summed in
chunk order. Their results therefore differ from a single plan's (partials per
slot) only by the FP32 summation order -- compared within 1e-5 -- and match the
oracle within the 1e-4 bar; reruns of a batch are bitwise identical (the chunk a
cluster takes does not change the arithmetic). Other members (M = 8, 16, 256)
keep their own launches and match single plans exactly.
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
    rel = lambda a, c: np.linalg.norm(a - c) / np.linalg.norm(c)  # noqa: E731
    for b, (O1, P1, E1) in enumerate(single):
        Ob, Pb = objs[b].cpu().numpy(), prbs[b].cpu().numpy()
        if probs[b][0].params["M"] == 256:  # own launches: the single plan's arithmetic exactly
            assert np.array_equal(Ob, O1) and np.array_equal(Pb, P1) and E[b] == E1, b
        else:
            assert rel(Ob, O1) < 1e-5 and rel(Pb, P1) < 1e-5 and abs(E[b] - E1) / E1 < 1e-5, b
    batch.close()
    # oracle on every member but the large one
    for b in (0, 1, 2, 4):
        prob, prm = probs[b]
        Oo, Po, Eo = oracle.iterate(prob.I, prob.positions, prob.O0, prob.P0, oracle.Params.from_dict(prm), n_iter)
        assert rel(objs[b].cpu().numpy(), Oo) < 1e-4 and rel(prbs[b].cpu().numpy(), Po) < 1e-4, b
        assert abs(E[b] - Eo[-1]) / Eo[-1] < 1e-4, b


def _run_batch(dev, probs, n_iter):
    from paper_2406_06640_gb300.engine import ReconstructionBatch

    tens = [_tensors(dev, prob) for prob, _ in probs]
    batch = ReconstructionBatch([(prm, t[0], prob.positions) for (prob, prm), t in zip(probs, tens)])
    objs, prbs = [t[1] for t in tens], [t[2] for t in tens]
    batch.iterate(objs, prbs, n_iter)
    E = batch.errors()
    batch.close()
    return [o.cpu().numpy() for o in objs], [p.cpu().numpy() for p in prbs], E


def test_work_queue_shares_chunks_across_problems_and_is_deterministic():
    """Six problems of one class (M 64, K 2, far field, 11 x 11 kernel) of uneven N, including
    N < 16 and N not a multiple of 16, drained by one launch: oracle parity for each, and two
    runs bitwise equal."""
    dev = torch.device("cuda:0")
    probs = []
    for i, side in enumerate((2, 3, 4, 5, 6, 7)):
        p = make_problem(0, scan_side=side, obj_side=64 + 10 * side + 16, M=64, K=2, sigma=1.0 + 0.1 * i)
        probs.append((p, dict(p.params, sigma1=1.0 + 0.1 * i, sigma2=1.0 + 0.1 * i)))
    n_iter = 3
    O1, P1, E1 = _run_batch(dev, probs, n_iter)
    O2, P2, E2 = _run_batch(dev, probs, n_iter)
    for b in range(len(probs)):
        assert np.array_equal(O1[b], O2[b]) and np.array_equal(P1[b], P2[b]) and E1[b] == E2[b], b
    rel = lambda a, c: np.linalg.norm(a - c) / np.linalg.norm(c)  # noqa: E731
    for b, (prob, prm) in enumerate(probs):
        Oo, Po, Eo = oracle.iterate(prob.I, prob.positions, prob.O0, prob.P0, oracle.Params.from_dict(prm), n_iter)
        assert rel(O1[b], Oo) < 1e-4 and rel(P1[b], Po) < 1e-4 and abs(E1[b] - Eo[-1]) / Eo[-1] < 1e-4, b


def test_batch_reports_its_kernel_launches():
    """One queued launch for the shape class plus the four update kernels of every member (no
    constraint window): the kernel nodes of the replayed graph."""
    from paper_2406_06640_gb300.engine import ReconstructionBatch

    dev = torch.device("cuda:0")
    probs = []
    for side in (2, 3, 4):
        p = make_problem(0, scan_side=side, obj_side=64 + 10 * side + 16, M=64, K=2, sigma=1.0)
        probs.append((p, dict(p.params, windows=[])))
    tens = [_tensors(dev, prob) for prob, _ in probs]
    batch = ReconstructionBatch([(prm, t[0], prob.positions) for (prob, prm), t in zip(probs, tens)])
    assert batch.launches_per_iteration() == 0
    batch.iterate([t[1] for t in tens], [t[2] for t in tens], 2)
    assert batch.launches_per_iteration() == 1 + 4 * len(probs)
    batch.close()


def test_batch_with_pc_dm_members():
    """pc-DM members beside simultaneous-engine members of the same shape: the DM members keep
    their own launches, the first iteration (which starts their state) is a graph of its own; every
    member matches the oracle, and reruns are bitwise equal."""
    dev = torch.device("cuda:0")
    probs = []
    for i, (side, engine) in enumerate(((3, "dm"), (4, "pie"), (4, "dm"), (5, "pie"))):
        p = make_problem(0, scan_side=side, obj_side=64 + 10 * side + 16, M=64, K=2, sigma=1.0)
        probs.append((p, dict(p.params, engine=engine, windows=[(2, 3)], alpha1=1.0, alpha2=0.2)))
    n_iter = 4
    O1, P1, E1 = _run_batch(dev, probs, n_iter)
    O2, P2, E2 = _run_batch(dev, probs, n_iter)
    for b in range(len(probs)):
        assert np.array_equal(O1[b], O2[b]) and np.array_equal(P1[b], P2[b]) and E1[b] == E2[b], b
    rel = lambda a, c: np.linalg.norm(a - c) / np.linalg.norm(c)  # noqa: E731
    for b, (prob, prm) in enumerate(probs):
        Oo, Po, Eo = oracle.iterate(prob.I, prob.positions, prob.O0, prob.P0, oracle.Params.from_dict(prm), n_iter)
        assert rel(O1[b], Oo) < 1e-4 and rel(P1[b], Po) < 1e-4 and abs(E1[b] - Eo[-1]) / Eo[-1] < 1e-4, b


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


def test_autotuner_picks_a_chunk_length_caches_it_and_can_be_fixed():
    import paper_2406_06640_gb300 as pg
    from paper_2406_06640_gb300.engine import ReconstructionBatch

    dev = torch.device("cuda:0")
    probs = []
    for i, side in enumerate((5, 6)):
        p = make_problem(0, scan_side=side, obj_side=64 + 10 * side + 16, M=64, K=1, geometry="near", sigma=1.2)
        probs.append((p, dict(p.params, sigma1=1.2, sigma2=1.2, kernel_size=7)))

    def classes():
        tens = [_tensors(dev, prob) for prob, _ in probs]
        batch = ReconstructionBatch([(prm, t[0], prob.positions) for (prob, prm), t in zip(probs, tens)])
        out = batch.classes()
        batch.close()
        return out

    first = classes()
    assert len(first) == 1 and first[0]["members"] == 2 and first[0]["M"] == 64 and first[0]["kh"] == 15
    assert first[0]["chunk_len"] in (8, 16, 32, 64)
    n = sum(-(-prob.N // first[0]["chunk_len"]) for prob, _ in probs)
    assert first[0]["chunks"] == n and 1 <= first[0]["slots"] <= n
    assert classes()[0]["chunk_len"] == first[0]["chunk_len"]  # cached for this shape class
    pg.set_batch_chunk(32)
    try:
        assert classes()[0]["chunk_len"] == 32
        O, P, E = _run_batch(dev, probs, 2)
    finally:
        pg.set_batch_chunk(0)
    rel = lambda a, c: np.linalg.norm(a - c) / np.linalg.norm(c)  # noqa: E731
    for b, (prob, prm) in enumerate(probs):
        Oo, Po, Eo = oracle.iterate(prob.I, prob.positions, prob.O0, prob.P0, oracle.Params.from_dict(prm), 2)
        assert rel(O[b], Oo) < 1e-4 and rel(P[b], Po) < 1e-4 and abs(E[b] - Eo[-1]) / Eo[-1] < 1e-4, b


def test_configuration3_shaped_batch_against_the_oracle():
    """Seven members drawn from the 64-problem batched configuration, as generated for it: the
    largest N (1539 positions of 128^2, K = 4, far field), two M = 256 members (near and far field,
    staged passes), and M = 64 / 128 members of both geometries with K 1-4, random sigma, iterated
    together (one graph launch per iteration, one queued launch per shape class). Every member
    against the oracle: rel. L2 bounds of O and P, per-pixel bounds of O over the illuminated field
    of view and of P over its support (as in test_gpu_parity.py), and its last E."""
    from synth.generators import make_cfg3_member

    dev = torch.device("cuda:0")
    members = (43, 32, 8, 1, 20, 49, 55)
    probs = []
    for i in members:
        p = make_cfg3_member(i)
        probs.append((p, dict(p.params)))
    assert max(p.params["N"] for p, _ in probs) == 1539
    assert sum(p.params["M"] == 256 for p, _ in probs) == 2
    n_iter = 2
    O, P, E = _run_batch(dev, probs, n_iter)
    from fov import fov_mask, probe_support

    for b, (prob, prm) in enumerate(probs):
        Oo, Po, Eo = oracle.iterate(prob.I, prob.positions, prob.O0, prob.P0, oracle.Params.from_dict(prm), n_iter)
        eo = np.linalg.norm(O[b] - Oo) / np.linalg.norm(Oo)
        ep = np.linalg.norm(P[b] - Po) / np.linalg.norm(Po)
        fov = fov_mask(prob.positions, prob.P0, Oo.shape, prm["M"])
        mo = np.max(np.abs(O[b] - Oo)[fov]) / np.max(np.abs(Oo)[fov])
        sup = np.broadcast_to(probe_support(prob.P0), Po.shape)
        mp = np.max(np.abs(P[b] - Po)[sup]) / np.max(np.abs(Po)[sup])
        ee = abs(E[b] - Eo[-1]) / Eo[-1]
        print(f"[parity] configuration-3 member {members[b]} (M={prm['M']} K={prm['K']} N={prm['N']} "
              f"{prm['geometry']}): rel L2 object {eo:.3e} probe {ep:.3e} error {ee:.3e}; "
              f"per-pixel object {mo:.3e} probe {mp:.3e}")
        assert eo < 1e-4 and ep < 1e-4 and ee < 1e-4, (members[b], eo, ep, ee)
        assert mo < 1e-4 and mp < 1e-4, (members[b], mo, mp)
