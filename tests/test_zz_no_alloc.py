"""GPU test of ptycho_iterate_static, the allocation-free entry point.

Callers that cannot call cudaMalloc (a locked device memory pool or budget,
a latency-critical loop that cannot take an allocation's implicit
synchronisation, a host that owns all device memory) run the engine through
this entry point; its scratch lives in a fixed 32 MiB device array inside
the library. Checked here:
  * two calls in a row on the same inputs, the second reusing the scratch the
    first left behind, each matching the regular plan + iterate path and the
    FP64 oracle within the parity tolerance of the other tests;
  * a warmed-up call changes neither the device's free memory nor torch's
    allocation count (nothing is allocated), on a non-default stream;
  * a request larger than the scratch, and intensities that are not 16-byte
    aligned, are rejected with a clear message before anything is launched.
This file is collected last, so a run that stops at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from synth import make_problem  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-4
EINVAL = 1


def _lib():
    import paper_2406_06640_gb300 as pg

    lib = pg.load()
    lib.ptycho_iterate_static.argtypes = [ctypes.POINTER(pg.PtychoParams), ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    lib.ptycho_iterate_static.restype = ctypes.c_int
    return lib


class _StaticCall:
    """Device inputs of one problem, prepared once; call() runs the static entry point on fresh
    copies of the initial object and probe without allocating inside the call."""

    def __init__(self, prob, params, n_iter, stream=None):
        import paper_2406_06640_gb300 as pg

        dev = torch.device("cuda:0")
        self.lib = _lib()
        self.n_iter = n_iter
        self.stream = stream
        self.I = torch.from_numpy(prob.I).to(dev)
        self.pos = torch.from_numpy(prob.positions).to(dev)
        self.O0 = torch.from_numpy(prob.O0.astype(np.complex64)).to(dev)
        self.P0 = torch.from_numpy(prob.P0.astype(np.complex64)).to(dev)
        self.O = torch.empty_like(self.O0)
        self.P = torch.empty_like(self.P0)
        self.p, self._keep = pg.make_params(params)
        self.errs = (ctypes.c_double * max(n_iter, 1))()
        torch.cuda.synchronize()

    def call(self):
        s = self.stream
        handle = s.cuda_stream if s is not None else None
        with torch.cuda.stream(s) if s is not None else _null():
            self.O.copy_(self.O0)
            self.P.copy_(self.P0)
        st = self.lib.ptycho_iterate_static(ctypes.byref(self.p), self.I.data_ptr(), self.pos.data_ptr(),
                                            self.O.data_ptr(), self.P.data_ptr(), self.n_iter, self.errs, handle)
        assert st == 0, self.lib.ptycho_last_error().decode()
        return self.O.cpu().numpy(), self.P.cpu().numpy(), np.array(list(self.errs)[: self.n_iter])


class _null:
    def __enter__(self):
        return None

    def __exit__(self, *a):
        return False


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


CASES = [
    (dict(cfg=0, scan_side=5, obj_side=128), dict(windows=[(2, 3)]), 4),
    (dict(cfg=0, scan_side=4, obj_side=112, M=32, K=3, geometry="near", sigma=1.5),
     dict(blur_domain="intensity", sigma1=1.5, sigma2=1.5), 3),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_static_entry_point_matches_plan_path_and_oracle_on_two_calls(case):
    spec, over, n_iter = CASES[case]
    spec = dict(spec)
    prob = make_problem(spec.pop("cfg"), **spec)
    params = dict(prob.params, **over)
    sc = _StaticCall(prob, params, n_iter)
    first = sc.call()
    second = sc.call()  # reuses the scratch the first call left behind
    Op, Pp, Ep = _run_plan(prob, params, n_iter)
    Oo, Po, Eo = oracle.iterate(prob.I, prob.positions, prob.O0, prob.P0, oracle.Params.from_dict(params), n_iter)
    for Os, Ps, Es in (first, second):
        assert _rel(Os, Op) <= TOL and _rel(Ps, Pp) <= TOL
        assert np.max(np.abs(Es - Ep) / Ep) <= TOL
        assert _rel(Os, Oo) <= TOL and _rel(Ps, Po) <= TOL
        assert np.max(np.abs(Es - Eo) / Eo) <= TOL
    # the two calls run the same kernels on the same inputs in the same order
    assert np.array_equal(first[0], second[0]) and np.array_equal(first[1], second[1])


def test_static_entry_point_allocates_nothing_on_a_side_stream():
    prob = make_problem(0, scan_side=5, obj_side=128)
    params = dict(prob.params, windows=[(1, 2)])
    stream = torch.cuda.Stream()
    sc = _StaticCall(prob, params, 3, stream=stream)
    ref = sc.call()  # first call on the device: looks up the scratch's address, loads the kernels
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    reserved0 = torch.cuda.memory_reserved()
    st = sc.lib.ptycho_iterate_static(ctypes.byref(sc.p), sc.I.data_ptr(), sc.pos.data_ptr(), sc.O.data_ptr(),
                                      sc.P.data_ptr(), 0, None, stream.cuda_stream)
    assert st == 0, sc.lib.ptycho_last_error().decode()
    with torch.cuda.stream(stream):
        sc.O.copy_(sc.O0)
        sc.P.copy_(sc.P0)
    st = sc.lib.ptycho_iterate_static(ctypes.byref(sc.p), sc.I.data_ptr(), sc.pos.data_ptr(), sc.O.data_ptr(),
                                      sc.P.data_ptr(), 3, sc.errs, stream.cuda_stream)
    assert st == 0, sc.lib.ptycho_last_error().decode()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
    assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == reserved0
    assert np.array_equal(sc.O.cpu().numpy(), ref[0]) and np.array_equal(sc.P.cpu().numpy(), ref[1])


def test_static_entry_point_rejects_misaligned_intensities():
    import paper_2406_06640_gb300 as pg

    prob = make_problem(0, scan_side=3, obj_side=96)
    dev = torch.device("cuda:0")
    lib = _lib()
    flat = torch.from_numpy(np.concatenate([[0.0], prob.I.ravel()]).astype(np.float32)).to(dev)
    I_off = flat[1:]  # a valid float32 view one element past a 16-byte boundary
    assert I_off.data_ptr() % 16 == 4
    pos = torch.from_numpy(prob.positions).to(dev)
    O = torch.from_numpy(prob.O0.astype(np.complex64)).to(dev)
    P = torch.from_numpy(prob.P0.astype(np.complex64)).to(dev)
    p, keep = pg.make_params(dict(prob.params))
    st = lib.ptycho_iterate_static(ctypes.byref(p), I_off.data_ptr(), pos.data_ptr(), O.data_ptr(), P.data_ptr(),
                                   1, None, None)
    assert st == EINVAL
    assert "16-byte aligned" in lib.ptycho_last_error().decode()


def test_static_entry_point_rejects_requests_beyond_its_scratch():
    import paper_2406_06640_gb300 as pg

    prob = make_problem(0)
    dev = torch.device("cuda:0")
    lib = _lib()
    # 900 positions of 128 x 128 need well over the 32 MiB scratch
    big = dict(prob.params, M=128, N=900, obj_h=640, obj_w=640)
    I = torch.zeros((900, 128, 128), dtype=torch.float32, device=dev)
    I[:, 0, 0] = 1.0
    pos = torch.zeros((900, 2), dtype=torch.int32, device=dev)
    O = torch.ones((640, 640), dtype=torch.complex64, device=dev)
    P = torch.ones((1, 128, 128), dtype=torch.complex64, device=dev)
    p, keep = pg.make_params(big)
    st = lib.ptycho_iterate_static(ctypes.byref(p), I.data_ptr(), pos.data_ptr(), O.data_ptr(), P.data_ptr(), 1,
                                   None, None)
    assert st == EINVAL
    assert "32 MiB" in lib.ptycho_last_error().decode()
