"""Thin Python binding of the C ABI in include/pft.h (argument marshalling only).

Every function here has the name of the C entry point it calls and forwards to it
through ctypes; all computation happens in ``libpft.so``.  Arrays may be numpy arrays
(host memory) or torch CUDA tensors (device memory); outputs are written into caller
buffers exactly as in C.  If the library has not been built, loading raises: there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpft.so")

# enums (include/pft.h)
PFT_OK, PFT_ERR_ARG, PFT_ERR_SHAPE, PFT_ERR_OOM, PFT_ERR_CUDA = 0, 1, 2, 3, 4
PFT_ERR_TIMEOUT, PFT_ERR_NONFINITE, PFT_ERR_STATE, PFT_ERR_IO, PFT_ERR_UNSUPPORTED = 5, 6, 7, 8, 9
PFT_SCFT_REAL, PFT_CL_COMPLEX = 0, 1
PFT_FP64, PFT_FP32_MIXED = 0, 1
PFT_HOST, PFT_DEVICE = 0, 1
PFT_STEP_SCFT_EULER, PFT_STEP_CL_EULER_MARUYAMA = 0, 1
PFT_MARCH_AUTO, PFT_MARCH_PASSES = 0, 1
PFT_BATCH_GRAPHED, PFT_BATCH_PER_INSTANCE = 0, 1
PFT_SCHEME_SPLIT2, PFT_SCHEME_RQM4 = 0, 1
PFT_STEP_SCFT_SIS, PFT_STEP_CL_SIS = 2, 3
PFT_ARCH_DIBLOCK, PFT_ARCH_EDWARDS = 0, 1
PFT_BATCH_PLANS = 7  # batch plans 0, 1, 2, 3, 19, 35, 51 (the order of tuned_ms)


class pft_grid(ct.Structure):
    _fields_ = [("n", ct.c_int * 3), ("L", ct.c_double * 3)]


class pft_chain(ct.Structure):
    _fields_ = [("Ns", ct.c_int), ("fA", ct.c_double)]


class pft_model(ct.Structure):
    _fields_ = [("chiN", ct.c_double), ("C", ct.c_double), ("kind", ct.c_int), ("arch", ct.c_int),
                ("B", ct.c_double)]


class pft_opts(ct.Structure):
    _fields_ = [("precision", ct.c_int), ("use_graph", ct.c_int), ("stream", ct.c_void_p),
                ("seed", ct.c_ulonglong), ("instance", ct.c_ulonglong), ("march", ct.c_int), ("scheme", ct.c_int),
                ("checkpoint", ct.c_int), ("autotune", ct.c_int)]


class pft_obs(ct.Structure):
    _fields_ = [("Q", ct.c_double * 2), ("lnQ", ct.c_double * 2), ("H", ct.c_double * 2), ("h", ct.c_double * 2),
                ("phiA_mean", ct.c_double * 2), ("phiB_mean", ct.c_double * 2), ("force_p_rms", ct.c_double),
                ("force_m_rms", ct.c_double), ("fA_eff", ct.c_double), ("NsA", ct.c_int), ("step", ct.c_longlong)]

    def as_dict(self):
        def z(a):
            return complex(a[0], a[1])
        return {"Q": z(self.Q), "lnQ": z(self.lnQ), "H": z(self.H), "h": z(self.h),
                "phiA_mean": z(self.phiA_mean), "phiB_mean": z(self.phiB_mean),
                "force_p_rms": self.force_p_rms, "force_m_rms": self.force_m_rms,
                "fA_eff": self.fA_eff, "NsA": self.NsA, "step": self.step}


class pft_instance_desc(ct.Structure):
    _fields_ = [("grid", pft_grid), ("chain", pft_chain), ("model", pft_model), ("seed", ct.c_ulonglong)]


class pft_profile(ct.Structure):
    _fields_ = [("nkinds", ct.c_int), ("name", (ct.c_char * 24) * 16), ("launches", ct.c_longlong * 16),
                ("ms", ct.c_double * 16), ("bytes_per_launch", ct.c_double * 16), ("step_fwd_ms", ct.c_double),
                ("step_bwd_ms", ct.c_double), ("total_ms", ct.c_double)]

    def as_dict(self):
        kinds = {}
        for k in range(self.nkinds):
            kinds[self.name[k].value.decode()] = {"launches": self.launches[k], "ms": self.ms[k],
                                                   "bytes_per_launch": self.bytes_per_launch[k]}
        return {"kinds": kinds, "step_fwd_ms": self.step_fwd_ms, "step_bwd_ms": self.step_bwd_ms,
                "total_ms": self.total_ms}


class PftError(RuntimeError):
    def __init__(self, status, where):
        lib = _lib()
        msg = lib.pft_status_string(status).decode()
        detail = lib.pft_last_error().decode()
        super().__init__(f"{where}: {msg}" + (f" ({detail})" if detail else ""))
        self.status = status


_L = None

# Every entry point declared in include/pft.h, with its ctypes signature.
_P = ct.c_void_p
_SIGS = {
    "pft_status_string": (ct.c_char_p, [ct.c_int]),
    "pft_last_error": (ct.c_char_p, []),
    "pft_create": (ct.c_int, [ct.POINTER(ct.c_void_p), ct.POINTER(pft_grid), ct.POINTER(pft_chain),
                              ct.POINTER(pft_model), ct.POINTER(pft_opts)]),
    "pft_destroy": (ct.c_int, [_P]),
    "pft_memory_bytes": (ct.c_int, [_P, ct.POINTER(ct.c_size_t)]),
    "pft_get_stream": (ct.c_int, [_P, ct.POINTER(ct.c_void_p)]),
    "pft_synchronize": (ct.c_int, [_P]),
    "pft_set_fields": (ct.c_int, [_P, _P, _P, ct.c_int]),
    "pft_get_fields": (ct.c_int, [_P, _P, _P, ct.c_int]),
    "pft_set_box": (ct.c_int, [_P, ct.POINTER(ct.c_double)]),
    "pft_save": (ct.c_int, [_P, ct.c_char_p]),
    "pft_load": (ct.c_int, [_P, ct.c_char_p]),
    "pft_get_box": (ct.c_int, [_P, ct.POINTER(ct.c_double)]),
    "pft_solve": (ct.c_int, [_P]),
    "pft_get_observables": (ct.c_int, [_P, ct.POINTER(pft_obs)]),
    "pft_get_densities": (ct.c_int, [_P, _P, _P, ct.c_int]),
    "pft_field_step": (ct.c_int, [_P, ct.c_int, ct.c_double, _P, _P, ct.c_int]),
    "pft_gradients": (ct.c_int, [_P, _P, _P, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double), ct.c_int]),
    "pft_batch_create": (ct.c_int, [ct.POINTER(ct.c_void_p), ct.c_int, ct.POINTER(pft_instance_desc), ct.c_int,
                                     _P]),
    "pft_batch_destroy": (ct.c_int, [_P]),
    "pft_batch_set_fields": (ct.c_int, [_P, ct.c_int, _P, _P, ct.c_int]),
    "pft_batch_get_fields": (ct.c_int, [_P, ct.c_int, _P, _P, ct.c_int]),
    "pft_batch_run": (ct.c_int, [_P, ct.c_int, ct.c_double, ct.c_double, ct.c_int]),
    "pft_batch_get_observables": (ct.c_int, [_P, ct.c_int, ct.POINTER(pft_obs)]),
    "pft_batch_get_densities": (ct.c_int, [_P, ct.c_int, _P, _P, ct.c_int]),
    "pft_batch_synchronize": (ct.c_int, [_P]),
    "pft_batch_info": (ct.c_int, [_P, ct.POINTER(ct.c_double), ct.POINTER(ct.c_int), ct.POINTER(ct.c_longlong)]),
    "pft_batch_get_stream": (ct.c_int, [_P, ct.POINTER(ct.c_void_p)]),
    "pft_profile_step": (ct.c_int, [_P, ct.c_int, ct.c_double, ct.POINTER(pft_profile)]),
    "pft_contour_step_static": (ct.c_int, [ct.POINTER(ct.c_int), ct.POINTER(ct.c_double), ct.c_int, _P, _P, _P,
                                            _P]),
    "pft_fft3d": (ct.c_int, [_P, _P, _P, ct.c_int, ct.c_int]),
    "pft_get_propagator": (ct.c_int, [_P, ct.c_int, ct.c_int, _P, ct.c_int]),
    "pft_debug_set_q0": (ct.c_int, [_P, _P, ct.c_int]),
    "pft_launch_counts": (ct.c_int, [_P, ct.POINTER(ct.c_longlong), ct.POINTER(ct.c_longlong)]),
    "pft_get_checkpoint": (ct.c_int, [_P, ct.POINTER(ct.c_int)]),
    "pft_get_plan": (ct.c_int, [_P, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]),
    "pft_fma_throughput": (ct.c_int, [ct.c_int, ct.POINTER(ct.c_double), _P]),
    "pft_set_plan": (ct.c_int, [_P, ct.c_int, ct.c_int]),
    "pft_adjoint": (ct.c_int, [_P, _P, _P, _P, _P, ct.c_int]),
    "pft_batch_autotune": (ct.c_int, [_P]),
    "pft_batch_set_plan": (ct.c_int, [_P, ct.c_int, ct.c_int]),
    "pft_batch_class_info": (ct.c_int, [_P, ct.c_int, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int),
                                        ct.POINTER(ct.c_int), ct.POINTER(ct.c_int), ct.POINTER(ct.c_float)]),
    "pft_philox_normals": (ct.c_int, [ct.c_ulonglong, ct.c_ulonglong, ct.c_ulonglong, ct.c_int, ct.c_longlong,
                                      _P, _P]),
    "pft_philox_raw": (ct.c_int, [ct.POINTER(ct.c_uint), ct.POINTER(ct.c_uint), ct.c_longlong, _P, _P]),
    "pft_debug_narrow_rn": (ct.c_int, [_P, _P, ct.c_longlong, _P]),
}


def _lib():
    global _L
    if _L is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1204_5434_gb300.build.build() "
                               "(there is no fallback implementation)")
        lib = ct.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _L = lib
    return _L


def exported_symbols():
    return list(_SIGS)


def _check(status, where):
    if status != PFT_OK:
        raise PftError(status, where)


def _ptr(a, writable=False):
    """(pointer, where) of a numpy array (host) or a torch CUDA tensor (device)."""
    if a is None:
        return None, PFT_HOST
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        if writable and not a.flags["WRITEABLE"]:
            raise ValueError("output array is read-only")
        return a.ctypes.data, PFT_HOST
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr(), (PFT_DEVICE if a.is_cuda else PFT_HOST)
    raise TypeError(f"unsupported array type {type(a)}")


def _where(*arrays):
    ws = {w for (_, w) in (_ptr(a) for a in arrays if a is not None)}
    if len(ws) > 1:
        raise ValueError("mix of host and device arrays in one call")
    return ws.pop() if ws else PFT_HOST


# ---------------------------------------------------------------- entry points
def pft_status_string(status: int) -> str:
    return _lib().pft_status_string(status).decode()


def pft_last_error() -> str:
    return _lib().pft_last_error().decode()


def pft_create(n, L, Ns, fA, chiN, C, kind=PFT_SCFT_REAL, precision=PFT_FP64, use_graph=True, stream=None,
               seed=0, instance=0, march=PFT_MARCH_AUTO, scheme=PFT_SCHEME_SPLIT2, checkpoint=0,
               arch=PFT_ARCH_DIBLOCK, B=0.0, autotune=0):
    g = pft_grid((ct.c_int * 3)(*[int(v) for v in n]), (ct.c_double * 3)(*[float(v) for v in L]))
    ch = pft_chain(int(Ns), float(fA))
    m = pft_model(float(chiN), float(C), int(kind), int(arch), float(B))
    o = pft_opts(int(precision), 1 if use_graph else 0, ct.c_void_p(stream or 0), int(seed), int(instance),
                 int(march), int(scheme), int(checkpoint), int(autotune))
    h = ct.c_void_p()
    _check(_lib().pft_create(ct.byref(h), ct.byref(g), ct.byref(ch), ct.byref(m), ct.byref(o)), "pft_create")
    return h


def pft_destroy(h):
    _check(_lib().pft_destroy(h), "pft_destroy")


def pft_memory_bytes(h) -> int:
    b = ct.c_size_t()
    _check(_lib().pft_memory_bytes(h, ct.byref(b)), "pft_memory_bytes")
    return b.value


def pft_get_stream(h) -> int:
    s = ct.c_void_p()
    _check(_lib().pft_get_stream(h, ct.byref(s)), "pft_get_stream")
    return s.value or 0


def pft_synchronize(h):
    _check(_lib().pft_synchronize(h), "pft_synchronize")


def pft_set_fields(h, wp, wm):
    w = _where(wp, wm)
    _check(_lib().pft_set_fields(h, _ptr(wp)[0], _ptr(wm)[0], w), "pft_set_fields")


def pft_get_fields(h, wp, wm):
    w = _where(wp, wm)
    _check(_lib().pft_get_fields(h, _ptr(wp, True)[0], _ptr(wm, True)[0], w), "pft_get_fields")


def pft_set_box(h, L):
    _check(_lib().pft_set_box(h, (ct.c_double * 3)(*[float(v) for v in L])), "pft_set_box")


def pft_save(h, path):
    _check(_lib().pft_save(h, os.fsencode(path)), "pft_save")


def pft_load(h, path):
    _check(_lib().pft_load(h, os.fsencode(path)), "pft_load")


def pft_get_box(h):
    L = (ct.c_double * 3)()
    _check(_lib().pft_get_box(h, L), "pft_get_box")
    return tuple(L)


def pft_solve(h):
    _check(_lib().pft_solve(h), "pft_solve")


def pft_get_observables(h) -> dict:
    o = pft_obs()
    _check(_lib().pft_get_observables(h, ct.byref(o)), "pft_get_observables")
    return o.as_dict()


def pft_get_densities(h, phiA, phiB):
    w = _where(phiA, phiB)
    _check(_lib().pft_get_densities(h, _ptr(phiA, True)[0], _ptr(phiB, True)[0], w), "pft_get_densities")


def pft_field_step(h, kind, lam_or_dt, eta_p=None, eta_m=None):
    w = _where(eta_p, eta_m)
    _check(_lib().pft_field_step(h, int(kind), float(lam_or_dt), _ptr(eta_p)[0], _ptr(eta_m)[0], w),
           "pft_field_step")


def pft_adjoint(h, dL_dphiA, dL_dphiB, dL_dwp, dL_dwm):
    """Reverse-mode adjoint of the last solve: fills dL_dwp, dL_dwm from dL/dphiA, dL/dphiB."""
    w = _where(dL_dphiA, dL_dphiB, dL_dwp, dL_dwm)
    _check(_lib().pft_adjoint(h, _ptr(dL_dphiA)[0], _ptr(dL_dphiB)[0], _ptr(dL_dwp, True)[0], _ptr(dL_dwm, True)[0],
                              w), "pft_adjoint")


def pft_gradients(h, dH_dwp=None, dH_dwm=None):
    """Returns (dH_dL, dlnQ_dL) as 3-tuples; fills dH_dwp / dH_dwm if given."""
    w = _where(dH_dwp, dH_dwm)
    dL = (ct.c_double * 3)()
    dq = (ct.c_double * 3)()
    _check(_lib().pft_gradients(h, _ptr(dH_dwp, True)[0], _ptr(dH_dwm, True)[0], dL, dq, w), "pft_gradients")
    return tuple(dL), tuple(dq)


def pft_batch_create(instances, precision=PFT_FP32_MIXED, stream=None):
    """instances: list of dicts with n, L, Ns, fA, chiN, C, kind, seed."""
    arr = (pft_instance_desc * len(instances))()
    for i, d in enumerate(instances):
        arr[i].grid = pft_grid((ct.c_int * 3)(*[int(v) for v in d["n"]]), (ct.c_double * 3)(*[float(v) for v in d["L"]]))
        arr[i].chain = pft_chain(int(d["Ns"]), float(d["fA"]))
        arr[i].model = pft_model(float(d["chiN"]), float(d["C"]), int(d["kind"]))
        arr[i].seed = int(d.get("seed", 0))
    h = ct.c_void_p()
    _check(_lib().pft_batch_create(ct.byref(h), len(instances), arr, int(precision), stream), "pft_batch_create")
    return h


def pft_batch_destroy(b):
    _check(_lib().pft_batch_destroy(b), "pft_batch_destroy")


def pft_batch_set_fields(b, i, wp, wm):
    w = _where(wp, wm)
    _check(_lib().pft_batch_set_fields(b, int(i), _ptr(wp)[0], _ptr(wm)[0], w), "pft_batch_set_fields")


def pft_batch_get_fields(b, i, wp, wm):
    w = _where(wp, wm)
    _check(_lib().pft_batch_get_fields(b, int(i), _ptr(wp, True)[0], _ptr(wm, True)[0], w), "pft_batch_get_fields")


def pft_batch_run(b, updates, lam, dt, mode=PFT_BATCH_GRAPHED):
    _check(_lib().pft_batch_run(b, int(updates), float(lam), float(dt), int(mode)), "pft_batch_run")


def pft_batch_get_observables(b, i) -> dict:
    o = pft_obs()
    _check(_lib().pft_batch_get_observables(b, int(i), ct.byref(o)), "pft_batch_get_observables")
    return o.as_dict()


def pft_batch_get_densities(b, i, phiA, phiB):
    w = _where(phiA, phiB)
    _check(_lib().pft_batch_get_densities(b, int(i), _ptr(phiA, True)[0], _ptr(phiB, True)[0], w),
           "pft_batch_get_densities")


def pft_batch_autotune(b):
    _check(_lib().pft_batch_autotune(b), "pft_batch_autotune")


def pft_batch_set_plan(b, cls, plan):
    _check(_lib().pft_batch_set_plan(b, int(cls), int(plan)), "pft_batch_set_plan")


def pft_batch_class_info(b, cls):
    n = (ct.c_int * 3)()
    kind = ct.c_int()
    members = ct.c_int()
    plan = ct.c_int()
    ms = (ct.c_float * PFT_BATCH_PLANS)()
    _check(_lib().pft_batch_class_info(b, int(cls), n, ct.byref(kind), ct.byref(members), ct.byref(plan), ms),
           "pft_batch_class_info")
    return {"n": tuple(n), "kind": kind.value, "members": members.value, "plan": plan.value,
            "tuned_ms": tuple(ms[k] for k in range(PFT_BATCH_PLANS))}


def pft_batch_synchronize(b):
    _check(_lib().pft_batch_synchronize(b), "pft_batch_synchronize")


def pft_batch_info(b):
    u = ct.c_double()
    c = ct.c_int()
    n = ct.c_longlong()
    _check(_lib().pft_batch_info(b, ct.byref(u), ct.byref(c), ct.byref(n)), "pft_batch_info")
    return {"units_per_update": u.value, "classes": c.value, "launches": n.value}


def pft_batch_get_stream(b) -> int:
    s = ct.c_void_p()
    _check(_lib().pft_batch_get_stream(b, ct.byref(s)), "pft_batch_get_stream")
    return s.value or 0


def pft_profile_step(h, step_kind=-1, lam_or_dt=0.0) -> dict:
    p = pft_profile()
    _check(_lib().pft_profile_step(h, int(step_kind), float(lam_or_dt), ct.byref(p)), "pft_profile_step")
    return p.as_dict()


def pft_contour_step_static(n, L, Ns, w, q_in, q_out, stream=None):
    """Device arrays only (torch CUDA tensors of float64)."""
    ptrs = [_ptr(a) for a in (w, q_in, q_out)]
    if any(wh != PFT_DEVICE for _, wh in ptrs):
        raise ValueError("pft_contour_step_static takes device arrays")
    _check(_lib().pft_contour_step_static((ct.c_int * 3)(*[int(v) for v in n]),
                                          (ct.c_double * 3)(*[float(v) for v in L]), int(Ns),
                                          ptrs[0][0], ptrs[1][0], ptrs[2][0], stream), "pft_contour_step_static")


def pft_fft3d(h, x, out, inverse=False):
    w = _where(x, out)
    _check(_lib().pft_fft3d(h, _ptr(x)[0], _ptr(out, True)[0], 1 if inverse else 0, w), "pft_fft3d")


def pft_get_propagator(h, which, s, out):
    _check(_lib().pft_get_propagator(h, int(which), int(s), *(_ptr(out, True))), "pft_get_propagator")


def pft_debug_set_q0(h, q0=None):
    p, w = _ptr(q0)
    _check(_lib().pft_debug_set_q0(h, p, w), "pft_debug_set_q0")


def pft_fma_throughput(precision=PFT_FP64, stream=None) -> float:
    """Fused multiply-add throughput of the current device in TFLOP/s (FP64 or FP32)."""
    t = ct.c_double()
    _check(_lib().pft_fma_throughput(int(precision), ct.byref(t), stream), "pft_fma_throughput")
    return t.value


def pft_set_plan(h, plane, streams=1):
    """Fix the march plan: 0 pencil passes, 1 plane kernel + x pass, 2 separable march on the
    plane kernel, 3 separable march on pencils, 4 the same in double-float arithmetic (FP64
    contexts), 18 plan 2 with the alternative x kernel, 19 plan 3 with register lines (FP32,
    x and y lengths of at most 48 points), 35 plan 3 with 32-line tiles (FP32), 51 plan 3 with
    twice the elements a thread in 32-line tiles (FP32, x and y lengths of 32, 48 or 64)."""
    _check(_lib().pft_set_plan(h, int(plane), int(streams)), "pft_set_plan")


def pft_get_plan(h):
    """(plane kernel in use, two chains on two streams) of the pass march."""
    a = ct.c_int()
    b = ct.c_int()
    _check(_lib().pft_get_plan(h, ct.byref(a), ct.byref(b)), "pft_get_plan")
    return a.value, b.value


def pft_get_checkpoint(h) -> int:
    """History interval in use: 1 = every slice, K >= 2 = every K-th slice."""
    k = ct.c_int()
    _check(_lib().pft_get_checkpoint(h, ct.byref(k)), "pft_get_checkpoint")
    return k.value


def pft_launch_counts(h):
    """(kernels per graphed pft_solve or -1, kernels per pft_field_step)."""
    a = ct.c_longlong()
    b = ct.c_longlong()
    _check(_lib().pft_launch_counts(h, ct.byref(a), ct.byref(b)), "pft_launch_counts")
    return a.value, b.value


def pft_philox_normals(seed, instance, step, field, M, out_device, stream=None):
    p, w = _ptr(out_device, True)
    if w != PFT_DEVICE:
        raise ValueError("pft_philox_normals writes device memory")
    _check(_lib().pft_philox_normals(int(seed), int(instance), int(step), int(field), int(M), p, stream),
           "pft_philox_normals")


def pft_philox_raw(ctr, key, count, out_device, stream=None):
    p, w = _ptr(out_device, True)
    if w != PFT_DEVICE:
        raise ValueError("pft_philox_raw writes device memory")
    c = (ct.c_uint * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ct.c_uint * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    _check(_lib().pft_philox_raw(c, k, int(count), p, stream), "pft_philox_raw")


# ------------------------------------------------------------- convenience
class System:
    """Owning wrapper of one context (pft_create / pft_destroy) with host-array helpers."""

    def __init__(self, n, L, Ns, fA, chiN, C=1.0, kind=PFT_SCFT_REAL, precision=PFT_FP64, use_graph=True,
                 stream=None, seed=0, instance=0, march=PFT_MARCH_AUTO, scheme=PFT_SCHEME_SPLIT2, checkpoint=0,
                 arch=PFT_ARCH_DIBLOCK, B=0.0, autotune=0):
        self.n = tuple(int(v) for v in n)
        self.kind = kind
        self.M = self.n[0] * self.n[1] * self.n[2]
        self.h = None
        self.arch = arch
        self.h = pft_create(n, L, Ns, fA, chiN, C, kind, precision, use_graph, stream, seed, instance, march,
                            scheme, checkpoint, arch, B, autotune)

    @property
    def dtype(self):
        return np.float64 if self.kind == PFT_SCFT_REAL else np.complex128

    def close(self):
        if self.h:
            pft_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_fields(self, wp, wm=None):
        """wm may be None for the one-field Edwards model."""
        if isinstance(wp, np.ndarray):
            wp = np.ascontiguousarray(wp, dtype=self.dtype)
            if wm is not None:
                wm = np.ascontiguousarray(wm, dtype=self.dtype)
        pft_set_fields(self.h, wp, wm)

    def get_fields(self):
        a = np.empty(self.n, self.dtype)
        b = np.empty(self.n, self.dtype)
        pft_get_fields(self.h, a, b)
        return a, b

    def solve(self):
        pft_solve(self.h)

    def observables(self):
        return pft_get_observables(self.h)

    def densities(self):
        a = np.empty(self.n, self.dtype)
        b = np.empty(self.n, self.dtype)
        pft_get_densities(self.h, a, b)
        return a, b

    def field_step(self, lam_or_dt, eta_p=None, eta_m=None, semi_implicit=False):
        if self.kind == PFT_SCFT_REAL:
            kind = PFT_STEP_SCFT_SIS if semi_implicit else PFT_STEP_SCFT_EULER
        else:
            kind = PFT_STEP_CL_SIS if semi_implicit else PFT_STEP_CL_EULER_MARUYAMA
        if isinstance(eta_p, np.ndarray):
            eta_p = np.ascontiguousarray(eta_p, dtype=np.float64)
            eta_m = np.ascontiguousarray(eta_m, dtype=np.float64)
        pft_field_step(self.h, kind, lam_or_dt, eta_p, eta_m)

    def adjoint(self, dL_dphiA, dL_dphiB):
        """dL/dW+, dL/dW- of a loss on the densities of the last solve (host arrays)."""
        gp = np.empty(self.n)
        gm = np.empty(self.n)
        pft_adjoint(self.h, np.ascontiguousarray(dL_dphiA, dtype=np.float64),
                    np.ascontiguousarray(dL_dphiB, dtype=np.float64), gp, gm)
        return gp, gm

    def propagator(self, which, s):
        out = np.empty(self.n, self.dtype)
        pft_get_propagator(self.h, which, s, out)
        return out

    def fft3d(self, x, inverse=False):
        x = np.ascontiguousarray(x, dtype=np.complex128)
        out = np.empty_like(x)
        pft_fft3d(self.h, x, out, inverse)
        return out

    def set_box(self, L):
        pft_set_box(self.h, L)

    def save(self, path):
        pft_save(self.h, path)

    def load(self, path):
        pft_load(self.h, path)

    def gradients(self, want_fields=True):
        if want_fields:
            a = np.empty(self.n, np.float64)
            b = np.empty(self.n, np.float64)
            dL, dq = pft_gradients(self.h, a, b)
            return a, b, dL, dq
        dL, dq = pft_gradients(self.h)
        return None, None, dL, dq


def pft_debug_narrow_rn(x_device, y_device, stream=None):
    """torch CUDA tensors: x float64, y float32 of the same size."""
    (px, wx), (py, wy) = _ptr(x_device), _ptr(y_device, True)
    if wx != PFT_DEVICE or wy != PFT_DEVICE:
        raise ValueError("pft_debug_narrow_rn takes device arrays")
    _check(_lib().pft_debug_narrow_rn(px, py, int(x_device.numel()), stream), "pft_debug_narrow_rn")
