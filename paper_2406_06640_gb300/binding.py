"""ctypes binding of the C ABI in include/ptycho.h (argument marshalling only).

Tensors are passed as raw device pointers; every step of the engine runs in
libptycho.so. PyTorch provides device memory and streams only. If the shared
library is missing or fails to load, importing this module raises: there is
no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

from . import build as _build

PTYCHO_OK = 0
STATUS_NAMES = {0: "PTYCHO_OK", 1: "PTYCHO_EINVAL", 2: "PTYCHO_ENOMEM", 3: "PTYCHO_ECUDA",
                4: "PTYCHO_EUNSUPPORTED", 5: "PTYCHO_ENUMERIC", 6: "PTYCHO_ETIMEOUT"}
FARFIELD, NEARFIELD = 0, 1
BLUR_AMPLITUDE, BLUR_INTENSITY = 0, 1
STEP_NORMALISED, STEP_RPIE = 0, 1
ENGINE_PIE, ENGINE_DM = 0, 1

EXPORTED = ("ptycho_plan", "ptycho_iterate", "ptycho_error", "ptycho_error_history", "ptycho_destroy",
            "ptycho_plan_batch", "ptycho_iterate_batch", "ptycho_error_batch",
            "ptycho_profile", "ptycho_profile_read", "ptycho_launches_per_iteration", "ptycho_last_error",
            "ptycho_version", "ptycho_set_batch_chunk", "ptycho_batch_classes", "ptycho_batch_launches", "ptycho_set_staged_chunk", "ptycho_staged_chunk", "ptycho_permutation", "ptycho_unet_create", "ptycho_unet_param_count", "ptycho_unet_set_params",
            "ptycho_unet_get_params", "ptycho_unet_forward", "ptycho_unet_gradients", "ptycho_unet_train_step",
            "ptycho_unet_destroy", "ptycho_generate", "ptycho_warmstart", "ptycho_monochromatise",
            "ptycho_measure_fp32_peak", "ptycho_wait_selftest")


class PtychoError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class PtychoParams(ctypes.Structure):
    """Mirror of ptycho_params (field order and types must match include/ptycho.h)."""

    _fields_ = [
        ("M", ctypes.c_int32), ("K", ctypes.c_int32), ("N", ctypes.c_int32),
        ("obj_h", ctypes.c_int32), ("obj_w", ctypes.c_int32),
        ("geometry", ctypes.c_int32), ("blur_domain", ctypes.c_int32),
        ("fresnel_F", ctypes.c_double), ("sigma1", ctypes.c_double), ("sigma2", ctypes.c_double),
        ("kernel_size", ctypes.c_int32), ("eps_mod", ctypes.c_double),
        ("beta_obj", ctypes.c_double), ("beta_probe", ctypes.c_double),
        ("delta_obj", ctypes.c_double), ("delta_probe", ctypes.c_double),
        ("probe_update_start", ctypes.c_int32),
        ("alpha1", ctypes.c_double), ("alpha2", ctypes.c_double),
        ("cbar_min", ctypes.c_double), ("cbar_max", ctypes.c_double),
        ("n_windows", ctypes.c_int32), ("windows", ctypes.POINTER(ctypes.c_int32)),
        ("start_iteration", ctypes.c_int32),
        ("step_rule", ctypes.c_int32), ("rpie_alpha_obj", ctypes.c_double), ("rpie_alpha_probe", ctypes.c_double),
        ("minibatch", ctypes.c_int32), ("order_seed", ctypes.c_uint64), ("engine", ctypes.c_int32),
    ]


class GenSpec(ctypes.Structure):
    """Mirror of ptycho_gen_spec."""

    _fields_ = [
        ("S", ctypes.c_int32), ("noise", ctypes.c_int32), ("dose", ctypes.c_double),
        ("lattice_a", ctypes.c_double), ("peak", ctypes.c_double), ("peak_sd", ctypes.c_double),
        ("cutoff", ctypes.c_double), ("vacancy", ctypes.c_double), ("target_scale", ctypes.c_double),
        ("key", ctypes.c_uint64),
    ]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libptycho.so (building it first if it is missing or stale and nvcc exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libptycho.so not found at {_build.LIB}; run paper_2406_06640_gb300/build.py")
    lib = ctypes.CDLL(_build.LIB)
    P = ctypes.c_void_p
    st = ctypes.c_int
    lib.ptycho_plan.argtypes = [ctypes.POINTER(PtychoParams), P, P, P, ctypes.POINTER(P)]
    lib.ptycho_plan.restype = st
    lib.ptycho_iterate.argtypes = [P, P, P, ctypes.c_int32]
    lib.ptycho_iterate.restype = st
    lib.ptycho_error.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
    lib.ptycho_error.restype = st
    lib.ptycho_error_history.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_int32)]
    lib.ptycho_error_history.restype = st
    lib.ptycho_destroy.argtypes = [P]
    lib.ptycho_destroy.restype = st
    lib.ptycho_profile.argtypes = [P, ctypes.c_int32]
    lib.ptycho_profile.restype = st
    lib.ptycho_profile_read.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]
    lib.ptycho_profile_read.restype = st
    lib.ptycho_launches_per_iteration.argtypes = [P, ctypes.c_int32]
    lib.ptycho_launches_per_iteration.restype = ctypes.c_int32
    PP = ctypes.POINTER(ctypes.c_void_p)
    lib.ptycho_plan_batch.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.POINTER(PtychoParams)), PP, PP, P,
                                      ctypes.POINTER(P)]
    lib.ptycho_plan_batch.restype = st
    lib.ptycho_iterate_batch.argtypes = [P, PP, PP, ctypes.c_int32]
    lib.ptycho_iterate_batch.restype = st
    lib.ptycho_error_batch.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
    lib.ptycho_error_batch.restype = st
    lib.ptycho_set_batch_chunk.argtypes = [ctypes.c_int32]
    lib.ptycho_set_batch_chunk.restype = st
    lib.ptycho_permutation.argtypes = [ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_int32)]
    lib.ptycho_permutation.restype = st
    D = ctypes.POINTER(ctypes.c_double)
    lib.ptycho_monochromatise.argtypes = [ctypes.c_int32, ctypes.c_int32, D, D, ctypes.c_int32, ctypes.c_int32,
                                          P, P, P, ctypes.c_int32, P]
    lib.ptycho_monochromatise.restype = st
    lib.ptycho_set_staged_chunk.argtypes = [ctypes.c_int32]
    lib.ptycho_set_staged_chunk.restype = st
    lib.ptycho_staged_chunk.argtypes = [P]
    lib.ptycho_staged_chunk.restype = ctypes.c_int32
    lib.ptycho_batch_classes.argtypes = [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int32)]
    lib.ptycho_batch_classes.restype = st
    lib.ptycho_batch_launches.argtypes = [P, ctypes.POINTER(ctypes.c_int32)]
    lib.ptycho_batch_launches.restype = st
    lib.ptycho_last_error.argtypes = []
    lib.ptycho_last_error.restype = ctypes.c_char_p
    lib.ptycho_version.argtypes = []
    lib.ptycho_version.restype = ctypes.c_char_p
    lib.ptycho_measure_fp32_peak.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), P]
    lib.ptycho_measure_fp32_peak.restype = st
    lib.ptycho_wait_selftest.argtypes = [ctypes.c_int64, ctypes.c_int32, P]
    lib.ptycho_wait_selftest.restype = st
    F32 = ctypes.c_float
    lib.ptycho_unet_create.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, P,
                                       ctypes.POINTER(P)]
    lib.ptycho_unet_create.restype = st
    lib.ptycho_unet_param_count.argtypes = [P]
    lib.ptycho_unet_param_count.restype = ctypes.c_int64
    lib.ptycho_unet_set_params.argtypes = [P, P, ctypes.c_int64]
    lib.ptycho_unet_set_params.restype = st
    lib.ptycho_unet_get_params.argtypes = [P, P, ctypes.c_int64]
    lib.ptycho_unet_get_params.restype = st
    lib.ptycho_unet_forward.argtypes = [P, P, P, P]
    lib.ptycho_unet_forward.restype = st
    lib.ptycho_unet_gradients.argtypes = [P, P, P, P, F32, ctypes.POINTER(ctypes.c_double), P]
    lib.ptycho_unet_gradients.restype = st
    lib.ptycho_unet_train_step.argtypes = [P, P, P, P, F32, F32, ctypes.POINTER(ctypes.c_double)]
    lib.ptycho_unet_train_step.restype = st
    lib.ptycho_unet_destroy.argtypes = [P]
    lib.ptycho_unet_destroy.restype = st
    lib.ptycho_generate.argtypes = [ctypes.POINTER(GenSpec), P, P, ctypes.c_int32, ctypes.c_uint32, P, P, P, P, P, P]
    lib.ptycho_generate.restype = st
    lib.ptycho_warmstart.argtypes = [P, P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, P,
                                     ctypes.POINTER(ctypes.c_double)]
    lib.ptycho_warmstart.restype = st
    _lib = lib
    return lib


def _check(status: int):
    if status != PTYCHO_OK:
        raise PtychoError(status, load().ptycho_last_error().decode())


def make_params(d: dict) -> tuple:
    """Build a PtychoParams from a dict with the field names of ptycho_params.

    `geometry` may be "far"/"near", `blur_domain` "amplitude"/"intensity",
    `windows` a sequence of (first, last). Returns (params, keepalive).
    """
    p = PtychoParams()
    geo = d.get("geometry", FARFIELD)
    blur = d.get("blur_domain", BLUR_AMPLITUDE)
    p.M, p.K, p.N = int(d["M"]), int(d["K"]), int(d["N"])
    p.obj_h, p.obj_w = int(d["obj_h"]), int(d["obj_w"])
    p.geometry = {"far": FARFIELD, "near": NEARFIELD}.get(geo, geo)
    p.blur_domain = {"amplitude": BLUR_AMPLITUDE, "intensity": BLUR_INTENSITY}.get(blur, blur)
    p.fresnel_F = float(d.get("fresnel_F", 0.0))
    p.sigma1, p.sigma2 = float(d.get("sigma1", 1.0)), float(d.get("sigma2", 1.0))
    p.kernel_size = int(d.get("kernel_size", 11))
    p.eps_mod = float(d.get("eps_mod", 0.0))
    p.beta_obj, p.beta_probe = float(d.get("beta_obj", 1.0)), float(d.get("beta_probe", 1.0))
    p.delta_obj, p.delta_probe = float(d.get("delta_obj", 1e-3)), float(d.get("delta_probe", 1e-3))
    p.probe_update_start = int(d.get("probe_update_start", 1))
    p.alpha1, p.alpha2 = float(d.get("alpha1", 1.0)), float(d.get("alpha2", 0.0))
    p.cbar_min, p.cbar_max = float(d.get("cbar_min", 0.01)), float(d.get("cbar_max", 10.0))
    wins = [int(v) for w in d.get("windows", ()) for v in w]
    arr = (ctypes.c_int32 * max(len(wins), 1))(*wins)
    p.n_windows = len(wins) // 2
    p.windows = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int32)) if wins else None
    p.start_iteration = int(d.get("start_iteration", 1))
    rule = d.get("step_rule", STEP_NORMALISED)
    if isinstance(rule, str):
        rule = {"normalised": STEP_NORMALISED, "rpie": STEP_RPIE}[rule]
    p.step_rule = int(rule)
    p.rpie_alpha_obj = float(d.get("rpie_alpha_obj", 0.0))
    p.rpie_alpha_probe = float(d.get("rpie_alpha_probe", 0.0))
    p.minibatch = int(d.get("minibatch", 0))
    p.order_seed = int(d.get("order_seed", 0)) & ((1 << 64) - 1)
    eng = d.get("engine", ENGINE_PIE)
    if isinstance(eng, str):
        eng = {"pie": ENGINE_PIE, "dm": ENGINE_DM}[eng]
    p.engine = int(eng)
    return p, arr


class Plan:
    """One reconstruction plan: wraps ptycho_plan / ptycho_iterate / ptycho_error / ptycho_destroy."""

    def __init__(self, params: dict, intensities_ptr: int, positions_ptr: int, stream_ptr: int = 0):
        lib = load()
        self._p, self._keep = make_params(params)
        h = ctypes.c_void_p()
        _check(lib.ptycho_plan(ctypes.byref(self._p), ctypes.c_void_p(intensities_ptr),
                               ctypes.c_void_p(positions_ptr), ctypes.c_void_p(stream_ptr), ctypes.byref(h)))
        self._h = h

    def iterate(self, object_ptr: int, probe_ptr: int, n_iter: int):
        _check(load().ptycho_iterate(self._h, ctypes.c_void_p(object_ptr), ctypes.c_void_p(probe_ptr), int(n_iter)))

    def error(self) -> float:
        e = ctypes.c_double()
        _check(load().ptycho_error(self._h, ctypes.byref(e)))
        return e.value

    def error_history(self, n: int) -> list:
        buf = (ctypes.c_double * max(n, 1))()
        c = ctypes.c_int32()
        _check(load().ptycho_error_history(self._h, buf, int(n), ctypes.byref(c)))
        return [buf[i] for i in range(c.value)]

    def profile(self, enable: bool):
        _check(load().ptycho_profile(self._h, 1 if enable else 0))

    def profile_read(self) -> tuple:
        """(summed fused-kernel milliseconds, launches) since the last read."""
        ms = ctypes.c_double()
        c = ctypes.c_int32()
        _check(load().ptycho_profile_read(self._h, ctypes.byref(ms), ctypes.byref(c)))
        return ms.value, c.value

    def staged_chunk(self) -> int:
        return int(load().ptycho_staged_chunk(self._h))

    def launches_per_iteration(self, in_window: bool) -> int:
        return int(load().ptycho_launches_per_iteration(self._h, 1 if in_window else 0))

    def close(self):
        if getattr(self, "_h", None):
            load().ptycho_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class BatchPlan:
    """Several independent reconstructions iterated together (ptycho_plan_batch / ptycho_iterate_batch)."""

    def __init__(self, params: Sequence[dict], intensities_ptrs: Sequence[int], positions_ptrs: Sequence[int],
                 stream_ptr: int = 0):
        lib = load()
        self.B = len(params)
        made = [make_params(p) for p in params]
        self._keep = made
        arr = (ctypes.POINTER(PtychoParams) * self.B)(*[ctypes.pointer(m[0]) for m in made])
        ip = (ctypes.c_void_p * self.B)(*intensities_ptrs)
        pp = (ctypes.c_void_p * self.B)(*positions_ptrs)
        h = ctypes.c_void_p()
        _check(lib.ptycho_plan_batch(self.B, arr, ip, pp, ctypes.c_void_p(stream_ptr), ctypes.byref(h)))
        self._h = h

    def iterate(self, object_ptrs: Sequence[int], probe_ptrs: Sequence[int], n_iter: int):
        op = (ctypes.c_void_p * self.B)(*object_ptrs)
        pp = (ctypes.c_void_p * self.B)(*probe_ptrs)
        _check(load().ptycho_iterate_batch(self._h, op, pp, int(n_iter)))

    def classes(self) -> list:
        """Work-queue classes: dicts with M, K, near, kh, members, chunk_len, chunks, slots."""
        n = ctypes.c_int32()
        _check(load().ptycho_batch_classes(self._h, 0, None, ctypes.byref(n)))
        buf = (ctypes.c_int32 * (8 * max(n.value, 1)))()
        _check(load().ptycho_batch_classes(self._h, n.value, buf, ctypes.byref(n)))
        keys = ("M", "K", "near", "kh", "members", "chunk_len", "chunks", "slots")
        return [dict(zip(keys, buf[8 * c:8 * c + 8])) for c in range(n.value)]

    def launches_per_iteration(self) -> int:
        """Kernel nodes of the graph the last iterate replayed per iteration."""
        n = ctypes.c_int32()
        _check(load().ptycho_batch_launches(self._h, ctypes.byref(n)))
        return n.value

    def errors(self) -> list:
        out = (ctypes.c_double * self.B)()
        _check(load().ptycho_error_batch(self._h, out))
        return list(out)

    def close(self):
        if getattr(self, "_h", None):
            load().ptycho_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def version() -> str:
    return load().ptycho_version().decode()


class UNet:
    """The warm-start network (ptycho_unet_*): device pointers in, status checked."""

    def __init__(self, S: int, C: int, batch: int, seed: int = 0, stream_ptr: int = 0):
        self._lib = load()
        self._h = ctypes.c_void_p()
        _check(self._lib.ptycho_unet_create(S, C, batch, seed, stream_ptr, ctypes.byref(self._h)))
        self.S, self.C, self.batch = S, C, batch

    def param_count(self) -> int:
        return int(self._lib.ptycho_unet_param_count(self._h))

    def set_params(self, flat):
        """flat: contiguous float32 host array (numpy) of param_count() values."""
        _check(self._lib.ptycho_unet_set_params(self._h, flat.ctypes.data, flat.size))

    def get_params(self, out):
        _check(self._lib.ptycho_unet_get_params(self._h, out.ctypes.data, out.size))
        return out

    def forward(self, x_ptr: int, out2_ptr: int = 0, sigma_ptr: int = 0):
        _check(self._lib.ptycho_unet_forward(self._h, x_ptr, out2_ptr or None, sigma_ptr or None))

    def gradients(self, x_ptr: int, target_ptr: int, sigma_t_ptr: int, lam: float, grads=None) -> float:
        loss = ctypes.c_double()
        _check(self._lib.ptycho_unet_gradients(self._h, x_ptr, target_ptr, sigma_t_ptr, lam, ctypes.byref(loss),
                                               grads.ctypes.data if grads is not None else None))
        return loss.value

    def train_step(self, x_ptr: int, target_ptr: int, sigma_t_ptr: int, lam: float, lr: float,
                   want_loss: bool = False):
        loss = ctypes.c_double()
        _check(self._lib.ptycho_unet_train_step(self._h, x_ptr, target_ptr, sigma_t_ptr, lam, lr,
                                                ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def warmstart(self, intensities_ptr: int, positions_ptr: int, N: int, obj_h: int, obj_w: int,
                  target_scale: float, object_ptr: int) -> float:
        sigma = ctypes.c_double()
        _check(self._lib.ptycho_warmstart(self._h, intensities_ptr, positions_ptr, N, obj_h, obj_w, target_scale,
                                          object_ptr, ctypes.byref(sigma)))
        return sigma.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _check(self._lib.ptycho_unet_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_gen_spec(d: dict) -> GenSpec:
    g = GenSpec()
    g.S = int(d.get("S", 128))
    g.noise = int(d.get("noise", 1))
    g.dose = float(d.get("dose", 200.0))
    g.lattice_a = float(d.get("lattice_a", 16.0))
    g.peak = float(d.get("peak", 0.1))
    g.peak_sd = float(d.get("peak_sd", 1.5))
    g.cutoff = float(d.get("cutoff", 6.0))
    g.vacancy = float(d.get("vacancy", 0.05))
    g.target_scale = float(d.get("target_scale", 0.1))
    g.key = int(d.get("key", 0)) & ((1 << 64) - 1)
    return g


def generate(spec: dict, probe_ptr: int, params_ptr: int, n: int, first: int = 0, x: int = 0, counts: int = 0,
             clean: int = 0, target: int = 0, sigma: int = 0, stream_ptr: int = 0):
    """ptycho_generate: forward-model training patterns into the given device buffers (0 = not wanted)."""
    g = make_gen_spec(spec)
    _check(load().ptycho_generate(ctypes.byref(g), probe_ptr, params_ptr, n, first, x or None, counts or None,
                                  clean or None, target or None, sigma or None, stream_ptr or None))


def set_batch_chunk(chunk_len: int):
    """Fix the positions per work-queue chunk of later batch plans (8, 16, 32, 64; 0 = autotune)."""
    _check(load().ptycho_set_batch_chunk(chunk_len))


def set_staged_chunk(chunk: int):
    """Fix the positions per chunk of the staged M = 256 passes of later plans (4, 8, 16, 32; 0 = autotune)."""
    _check(load().ptycho_set_staged_chunk(chunk))


def monochromatise_raw(M: int, scales, weights, N: int, k: int, b_ptr: int, x_ptr: int, resid_ptr: int = 0,
                       clamp: bool = False, stream: int = 0):
    """ptycho_monochromatise on device pointers: x = k CGLS steps of min ||C x - b|| per pattern."""
    J = len(scales)
    if len(weights) != J:
        raise ValueError("scales and weights differ in length")
    sc = (ctypes.c_double * max(J, 1))(*[float(v) for v in scales])
    wt = (ctypes.c_double * max(J, 1))(*[float(v) for v in weights])
    _check(load().ptycho_monochromatise(M, J, sc, wt, N, k, ctypes.c_void_p(b_ptr or None),
                                        ctypes.c_void_p(x_ptr or None), ctypes.c_void_p(resid_ptr or None),
                                        1 if clamp else 0, ctypes.c_void_p(stream or None)))


def permutation(n: int, seed: int, stream: int, t: int) -> list:
    """ptycho_permutation: the Philox permutation of 0..n-1 that mini-batch plans use."""
    out = (ctypes.c_int32 * max(n, 1))()
    _check(load().ptycho_permutation(n, seed & ((1 << 64) - 1), stream, t, out))
    return list(out[:n])


def measure_fp32_peak(stream_ptr: int = 0) -> tuple:
    """Measured FP32 FMA throughput of the current device: (TFLOP/s, duration of the timed launch in ms)."""
    lib = load()
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib.ptycho_measure_fp32_peak(ctypes.byref(tf), ctypes.byref(ms), stream_ptr))
    return tf.value, ms.value
