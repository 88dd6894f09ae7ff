"""C-ABI boundary on the CPU: the library builds, loads, exports every declared
symbol, the ctypes mirror of ptycho_params matches the C layout, and host-side
validation rejects bad requests before any device work."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2406_06640_gb300 as pg
from paper_2406_06640_gb300.binding import PtychoParams, make_params

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def _declared_functions():
    names = set()
    for h in os.listdir(INCLUDE):
        if h.endswith(".h"):
            text = open(os.path.join(INCLUDE, h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(ptycho_\w+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    lib = pg.load()
    declared = _declared_functions()
    assert {"ptycho_plan", "ptycho_iterate", "ptycho_error", "ptycho_destroy"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(pg.EXPORTED) <= declared


def test_ctypes_params_layout_matches_c(tmp_path):
    fields = [f for f, _ in PtychoParams._fields_]
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "ptycho.h"', "int main(void) {",
           '  printf("%zu\\n", sizeof(ptycho_params));']
    src += [f'  printf("%zu\\n", offsetof(ptycho_params, {f}));' for f in fields]
    src += ["  return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", f"-I{INCLUDE}", str(c), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(PtychoParams)
    for f, off in zip(fields, out[1:]):
        assert getattr(PtychoParams, f).offset == off, f


def _plan_status(**over):
    base = dict(M=64, K=1, N=4, obj_h=128, obj_w=128, geometry="far", sigma1=1.0, sigma2=1.0)
    base.update(over)
    p, keep = make_params(base)
    h = ctypes.c_void_p()
    lib = pg.load()
    # valid-looking non-NULL host buffers: validation runs before any device call
    I = np.zeros(4, np.float32)
    pos = np.zeros(8, np.int32)
    st = lib.ptycho_plan(ctypes.byref(p), I.ctypes.data, pos.ctypes.data, None, ctypes.byref(h))
    return st, lib.ptycho_last_error().decode()


@pytest.mark.parametrize("over,expect", [
    (dict(M=7), 1), (dict(M=1024), 1), (dict(K=0), 1), (dict(K=9), 4), (dict(N=0), 1),
    (dict(obj_h=32), 1), (dict(geometry=5), 1), (dict(blur_domain=3), 1), (dict(geometry="near", fresnel_F=0.0), 1),
    (dict(sigma1=-1.0), 1), (dict(kernel_size=10), 1), (dict(kernel_size=33), 1), (dict(alpha1=1.5), 1),
    (dict(cbar_min=0.0), 1), (dict(cbar_min=2.0, cbar_max=1.0), 1), (dict(windows=[(0, 3)]), 1),
    (dict(windows=[(5, 4)]), 1), (dict(start_iteration=0), 1), (dict(delta_obj=-1.0), 1),
    (dict(eps_mod=float("nan")), 1), (dict(step_rule=2), 1), (dict(step_rule="rpie", rpie_alpha_obj=1.5), 1),
    (dict(step_rule="rpie", rpie_alpha_probe=-0.1), 1), (dict(minibatch=-1), 1),
    (dict(engine=2), 1), (dict(engine="dm", minibatch=2), 4),
])
def test_validation_rejects_bad_requests(over, expect):
    st, msg = _plan_status(**over)
    assert st == expect, msg
    assert msg


def test_null_arguments():
    lib = pg.load()
    p, keep = make_params(dict(M=64, K=1, N=4, obj_h=128, obj_w=128))
    assert lib.ptycho_plan(ctypes.byref(p), None, None, None, None) == 1
    h = ctypes.c_void_p()
    assert lib.ptycho_plan(None, None, None, None, ctypes.byref(h)) == 1
    assert lib.ptycho_iterate(None, None, None, 1) == 1
    e = ctypes.c_double()
    assert lib.ptycho_error(None, ctypes.byref(e)) == 1
    assert lib.ptycho_destroy(None) == 0


def test_wait_selftest_budget_is_validated_before_device_work():
    lib = pg.load()
    for bad in (-1, 2_000_000_001):
        assert lib.ptycho_wait_selftest(ctypes.c_int64(bad), 0, None) == 1
        assert "budget_ns" in lib.ptycho_last_error().decode()


def test_version_string():
    assert "sm_103a" in pg.version()


def test_batch_validation_names_the_problem():
    lib = pg.load()
    good, k1 = make_params(dict(M=64, K=1, N=4, obj_h=128, obj_w=128))
    bad, k2 = make_params(dict(M=64, K=0, N=4, obj_h=128, obj_w=128))
    arr = (ctypes.POINTER(pg.PtychoParams) * 2)(ctypes.pointer(good), ctypes.pointer(bad))
    ip = (ctypes.c_void_p * 2)(1, 1)
    pp = (ctypes.c_void_p * 2)(1, 1)
    h = ctypes.c_void_p()
    assert lib.ptycho_plan_batch(2, arr, ip, pp, None, ctypes.byref(h)) == 1
    assert lib.ptycho_last_error().decode().startswith("problem 1:")
    assert lib.ptycho_plan_batch(0, arr, ip, pp, None, ctypes.byref(h)) == 1


def test_batch_chunk_setting_is_validated():
    lib = pg.load()
    assert lib.ptycho_set_batch_chunk(7) == 1
    assert lib.ptycho_set_batch_chunk(-8) == 1
    assert lib.ptycho_set_batch_chunk(0) == 0
    assert lib.ptycho_set_staged_chunk(12) == 1
    assert lib.ptycho_set_staged_chunk(0) == 0


@pytest.mark.parametrize("n,seed,stream,t", [(1, 0, 3, 0), (2, 5, 3, 0), (37, 123456789012345, 4, 7),
                                             (100, 2 ** 64 - 1, 3, 0), (9, 42, 4, 4096)])
def test_host_permutation_matches_the_oracle(n, seed, stream, t):
    from oracle import philox

    assert pg.permutation(n, seed, stream, t) == philox.permutation(n, seed, stream, t).tolist()


@pytest.mark.parametrize("M,scales,weights,N,k,clamp,expect", [
    (48, [1.0], [1.0], 1, 3, 0, 4), (512, [1.0], [1.0], 1, 3, 0, 4), (0, [1.0], [1.0], 1, 3, 0, 1),
    (64, [], [], 1, 3, 0, 1), (64, [1.0] * 65, [1.0] * 65, 1, 3, 0, 4), (64, [1.0], [1.0], 1, -1, 0, 1),
    (64, [1.0], [1.0], -1, 3, 0, 1), (64, [2.6], [1.0], 1, 3, 0, 1), (64, [0.0], [1.0], 1, 3, 0, 1),
    (64, [1.0], [float("nan")], 1, 3, 0, 1), (64, [1.0, 1.2], [0.0, 0.0], 1, 3, 0, 1),
    (64, [1.0], [1.0], 1, 3, 2, 1),
])
def test_monochromatisation_validation(M, scales, weights, N, k, clamp, expect):
    """Rejected before any device work (non-NULL dummy pointers stand in for the device buffers)."""
    lib = pg.load()
    J = len(scales)
    sc = (ctypes.c_double * max(J, 1))(*scales)
    wt = (ctypes.c_double * max(J, 1))(*weights)
    dummy = ctypes.c_void_p(16)
    st = lib.ptycho_monochromatise(M, J, sc, wt, N, k, dummy, dummy, None, clamp, None)
    assert st == expect, lib.ptycho_last_error().decode()
    assert lib.ptycho_last_error().decode()


def test_monochromatisation_null_buffers_and_empty_batch():
    lib = pg.load()
    one = (ctypes.c_double * 1)(1.0)
    assert lib.ptycho_monochromatise(64, 1, one, one, 2, 3, None, None, None, 0, None) == 1
    assert lib.ptycho_monochromatise(64, 1, None, one, 2, 3, ctypes.c_void_p(16), ctypes.c_void_p(16), None, 0,
                                     None) == 1
    # no patterns: nothing to launch, no device needed
    assert lib.ptycho_monochromatise(64, 1, one, one, 0, 3, None, None, None, 0, None) == 0


def test_batch_launch_count_arguments():
    lib = pg.load()
    n = ctypes.c_int32(-1)
    assert lib.ptycho_batch_launches(None, ctypes.byref(n)) == 1
    assert lib.ptycho_launches_per_iteration(None, 1) == 0


def test_ctypes_gen_spec_layout_matches_c(tmp_path):
    from paper_2406_06640_gb300.binding import GenSpec

    fields = [f for f, _ in GenSpec._fields_]
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "ptycho.h"', "int main(void) {",
           '  printf("%zu\\n", sizeof(ptycho_gen_spec));']
    src += [f'  printf("%zu\\n", offsetof(ptycho_gen_spec, {f}));' for f in fields]
    src += ["  return 0;", "}"]
    c = tmp_path / "gen_layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "gen_layout"
    subprocess.run(["gcc", "-std=c99", f"-I{INCLUDE}", str(c), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(GenSpec)
    for f, off in zip(fields, out[1:]):
        assert getattr(GenSpec, f).offset == off, f


@pytest.mark.parametrize("S,C,batch", [(20, 32, 64), (16, 8, 64), (128, 80, 64), (128, 32, 0), (128, 32, 1025),
                                       (16, 32, 1), (528, 32, 64)])
def test_unet_create_validation(S, C, batch):
    lib = pg.load()
    h = ctypes.c_void_p()
    assert lib.ptycho_unet_create(S, C, batch, 0, None, ctypes.byref(h)) == 1
    assert h.value is None
    assert lib.ptycho_unet_create(128, 32, 64, 0, None, None) == 1


def test_warmstart_and_network_null_handles():
    lib = pg.load()
    x = np.zeros(16, np.float32)
    sig = ctypes.c_double()
    assert lib.ptycho_unet_param_count(None) == 0
    assert lib.ptycho_unet_set_params(None, x.ctypes.data, 16) == 1
    assert lib.ptycho_unet_destroy(None) == 0
    assert lib.ptycho_warmstart(None, x.ctypes.data, x.ctypes.data, 1, 8, 8, 1.0, x.ctypes.data, ctypes.byref(sig)) == 1


def test_generator_validation_before_device_work():
    from paper_2406_06640_gb300.binding import GenSpec

    lib = pg.load()
    buf = np.zeros(64, np.float32)  # 16-byte aligned by numpy's allocator
    ok = dict(S=128, noise=1, dose=2e4, lattice_a=16.0, peak=0.1, peak_sd=1.5, cutoff=6.0, vacancy=0.05,
              target_scale=1.0, key=7)

    def status(n=1, params=None, **over):
        spec = GenSpec(**dict(ok, **over))
        p = buf.ctypes.data if params is None else params
        return lib.ptycho_generate(ctypes.byref(spec), buf.ctypes.data, p, n, 0, None, None, None, None, None, None)

    assert lib.ptycho_generate(None, buf.ctypes.data, buf.ctypes.data, 1, 0, None, None, None, None, None, None) == 1
    assert status(S=32) == 4
    assert status(n=-1) == 1
    for bad in (dict(dose=0.0), dict(lattice_a=-1.0), dict(peak_sd=0.0), dict(cutoff=-1.0), dict(cutoff=40.0),
                dict(vacancy=1.5), dict(target_scale=0.0), dict(peak=float("nan"))):
        assert status(**bad) == 1, bad
    assert status(params=buf.ctypes.data + 4) == 1  # params not 16-byte aligned
    assert "aligned" in lib.ptycho_last_error().decode()


def test_entry_points_reject_null_handles_before_device_work():
    """Every plan, batch, network and utility call given a NULL handle or output returns PTYCHO_EINVAL
    (or its documented default) from the host, without touching a device."""
    lib = pg.load()
    P = ctypes.c_void_p
    d, i32 = ctypes.c_double(), ctypes.c_int32()
    buf = (ctypes.c_double * 4)()
    f = np.zeros(64, np.float32)
    assert lib.ptycho_error_history(None, buf, 4, ctypes.byref(i32)) == 1
    assert lib.ptycho_profile(None, 1) == 1
    assert lib.ptycho_profile_read(None, ctypes.byref(d), ctypes.byref(i32)) == 1
    assert lib.ptycho_launches_per_iteration(None, 1) == 0
    assert lib.ptycho_staged_chunk(None) == 0
    assert lib.ptycho_iterate_batch(None, None, None, 1) == 1
    assert lib.ptycho_error_batch(None, ctypes.byref(d)) == 1
    assert lib.ptycho_batch_classes(None, 0, None, ctypes.byref(i32)) == 1
    assert lib.ptycho_batch_launches(None, ctypes.byref(i32)) == 1
    assert lib.ptycho_measure_fp32_peak(None, None, None) == 1
    assert lib.ptycho_unet_forward(None, f.ctypes.data, None, None) == 1
    assert lib.ptycho_unet_get_params(None, f.ctypes.data, 64) == 1
    assert lib.ptycho_unet_gradients(None, f.ctypes.data, f.ctypes.data, f.ctypes.data, 0.1, ctypes.byref(d), None) == 1
    assert lib.ptycho_unet_train_step(None, f.ctypes.data, f.ctypes.data, f.ctypes.data, 0.1, 1e-3, ctypes.byref(d)) == 1
    lib.ptycho_iterate_static.argtypes = [P, P, P, P, P, ctypes.c_int32, P, P]
    lib.ptycho_iterate_static.restype = ctypes.c_int
    assert lib.ptycho_iterate_static(None, None, None, None, None, 1, None, None) == 1
    assert "params is NULL" in lib.ptycho_last_error().decode()
    lib.ptycho_gemm_bf16.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
    lib.ptycho_gemm_bf16.restype = ctypes.c_int
    assert lib.ptycho_gemm_bf16(None, None, None, 128, 16, 64, 0, None) == 1
    assert lib.ptycho_set_staged_chunk(3) == 1
