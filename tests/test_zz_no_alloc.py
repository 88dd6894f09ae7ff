"""GPU test of ptycho_iterate_static, the allocation-free entry point.

Callers that cannot call cudaMalloc (a locked device memory pool or budget,
a latency-critical loop that cannot take an allocation's implicit
synchronisation, a host that owns all device memory) run the engine through
this entry point; its scratch lives in a fixed 32 MiB device array inside
the library. Its output must match the regular plan + iterate path within the
parity tolerance of the other tests, on two calls in a row (the second call
reuses the scratch the first one left behind), and a request larger than the
scratch must be rejected with a clear message.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import make_problem  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _lib():
    import paper_2406_06640_gb300 as pg

    lib = pg.load()
    lib.ptycho_iterate_static.argtypes = [ctypes.POINTER(pg.PtychoParams), ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    lib.ptycho_iterate_static.restype = ctypes.c_int
    return lib


def _run_static(prob, params, n_iter):
    import paper_2406_06640_gb300 as pg

    dev = torch.device("cuda:0")
    lib = _lib()
    I = torch.from_numpy(prob.I).to(dev)
    pos = torch.from_numpy(prob.positions).to(dev)
    O = torch.from_numpy(prob.O0.astype(np.complex64)).to(dev)
    P = torch.from_numpy(prob.P0.astype(np.complex64)).to(dev)
    p, keep = pg.make_params(params)
    errs = (ctypes.c_double * n_iter)()
    st = lib.ptycho_iterate_static(ctypes.byref(p), I.data_ptr(), pos.data_ptr(), O.data_ptr(), P.data_ptr(),
                                   n_iter, errs, None)
    assert st == 0, lib.ptycho_last_error().decode()
    return O.cpu().numpy(), P.cpu().numpy(), np.array(list(errs))


def _run_plan(prob, params, n_iter):
    from paper_2406_06640_gb300.engine import Reconstruction

    dev = torch.device("cuda:0")
    I = torch.from_numpy(prob.I).to(dev)
    O = torch.from_numpy(prob.O0.astype(np.complex64)).to(dev)
    P = torch.from_numpy(prob.P0.astype(np.complex64)).to(dev)
    rec = Reconstruction(params, I, prob.positions)
    rec.iterate(O, P, n_iter)
    E = np.array(rec.errors(n_iter))
    out = O.cpu().numpy(), P.cpu().numpy(), E
    rec.close()
    return out


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_static_entry_point_matches_plan_path_on_two_calls():
    cases = [
        (make_problem(0, scan_side=5, obj_side=128), dict(windows=[(2, 3)]), 4),
        (make_problem(0, scan_side=4, obj_side=112, M=32, K=3, geometry="near", sigma=1.5),
         dict(blur_domain="intensity", sigma1=1.5, sigma2=1.5), 3),
    ]
    for prob, over, n_iter in cases:
        params = dict(prob.params, **over)
        Os, Ps, Es = _run_static(prob, params, n_iter)
        Op, Pp, Ep = _run_plan(prob, params, n_iter)
        assert _rel(Os, Op) <= TOL and _rel(Ps, Pp) <= TOL
        assert np.max(np.abs(Es - Ep) / Ep) <= TOL


def test_static_entry_point_rejects_requests_beyond_its_scratch():
    import paper_2406_06640_gb300 as pg

    prob = make_problem(0)
    params = dict(prob.params, N=prob.N)
    dev = torch.device("cuda:0")
    lib = _lib()
    # 900 positions of 128 x 128 need well over the 32 MiB scratch
    big = dict(params, M=128, N=900, obj_h=640, obj_w=640)
    I = torch.zeros((900, 128, 128), dtype=torch.float32, device=dev)
    I[:, 0, 0] = 1.0
    pos = torch.zeros((900, 2), dtype=torch.int32, device=dev)
    O = torch.ones((640, 640), dtype=torch.complex64, device=dev)
    P = torch.ones((1, 128, 128), dtype=torch.complex64, device=dev)
    p, keep = pg.make_params(big)
    st = lib.ptycho_iterate_static(ctypes.byref(p), I.data_ptr(), pos.data_ptr(), O.data_ptr(), P.data_ptr(), 1,
                                   None, None)
    assert st == 1
    assert "32 MiB" in lib.ptycho_last_error().decode()
