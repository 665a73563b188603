"""ctypes binding of libsfw (include/sfw.h): the C entry points under the same names.

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Loading fails loudly if the library has not been built.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsfw.so")

SFW_OK = 0
STATUS_NAMES = {0: "SFW_OK", 1: "SFW_ERR_ARG", 2: "SFW_ERR_SHAPE", 3: "SFW_ERR_CUDA",
                4: "SFW_ERR_NAN", 5: "SFW_ERR_TIMEOUT", 6: "SFW_ERR_ALLOC",
                7: "SFW_ERR_UNSUPPORTED"}
SFW_PREC_FP32 = 0
SFW_PREC_BF16 = 1
SFW_ROUTE_AUTO = 0
SFW_ROUTE_FFT = 1
SFW_ROUTE_DIRECT = 2

# every symbol declared in include/sfw.h
EXPORTS = ("sfw_plan_create", "sfw_plan_destroy", "sfw_plan_query", "sfw_plan_check", "sfw_autotune",
           "sfw_forward",
           "sfw_certificate_grid", "sfw_certificate_topk", "sfw_eta_points", "sfw_argmax", "sfw_argmax_noalloc",
           "sfw_slide_loss_grad", "sfw_step", "sfw_step_topk", "sfw_gram", "sfw_batch_create", "sfw_batch_destroy",
           "sfw_batch_query", "sfw_batch_step", "sfw_batch_autotune", "sfw_profile_start", "sfw_profile_collect", "sfw_profile_stop", "sfw_last_error",
           "sfw_launch_count",
           "sfw_version")


class SfwError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class PlanDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("R", ctypes.c_int * 3),
                ("psf", ctypes.POINTER(ctypes.c_float)), ("n_sigma", ctypes.c_int),
                ("n_d", ctypes.c_int), ("sigmas", ctypes.POINTER(ctypes.c_float)),
                ("ds", ctypes.POINTER(ctypes.c_float)), ("precision", ctypes.c_int),
                ("eps", ctypes.c_float), ("route", ctypes.c_int)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("E", ctypes.c_int * 3), ("P_conv", ctypes.c_int * 3), ("P_cert", ctypes.c_int * 3),
                ("K", ctypes.c_int), ("real_table", ctypes.c_int), ("table_bytes", ctypes.c_size_t),
                ("workspace_bytes", ctypes.c_size_t), ("route_blur", ctypes.c_int),
                ("route_cert", ctypes.c_int), ("tensor_cores", ctypes.c_int)]


class Atoms(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("m", ctypes.c_void_p), ("sigma", ctypes.c_void_p),
                ("d", ctypes.c_void_p), ("w", ctypes.c_void_p)]


class BatchVolume(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("y", ctypes.c_void_p), ("m", ctypes.c_void_p),
                ("sigma", ctypes.c_void_p), ("d", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("residual", ctypes.c_void_p), ("grad", ctypes.c_void_p), ("loss", ctypes.c_void_p),
                ("best_val", ctypes.c_void_p), ("best_idx", ctypes.c_void_p)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libsfw.so (built in-tree by ``build.py``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libsfw.so not found at {LIB_PATH}: run paper_2009_05473_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    L.sfw_plan_create.argtypes = [ctypes.POINTER(PlanDesc), ctypes.POINTER(vp)]
    L.sfw_plan_destroy.argtypes = [vp]
    L.sfw_plan_query.argtypes = [vp, ctypes.POINTER(PlanInfo)]
    L.sfw_autotune.argtypes = [vp, ctypes.c_char_p, vp]
    L.sfw_forward.argtypes = [vp, ctypes.POINTER(Atoms), vp, vp]
    L.sfw_certificate_grid.argtypes = [vp, vp, dbl, vp, vp, vp, vp, vp, vp]
    L.sfw_eta_points.argtypes = [vp, vp, dbl, i32, vp, vp, vp, vp]
    L.sfw_certificate_topk.argtypes = [vp, vp, dbl, i32, vp, vp, vp, vp, vp, vp]
    L.sfw_argmax.argtypes = [vp, i64, i32, vp, vp, vp]
    L.sfw_argmax_noalloc.argtypes = [vp, i64, i32, vp, vp, vp]
    L.sfw_slide_loss_grad.argtypes = [vp, vp, ctypes.POINTER(Atoms), dbl, vp, vp, vp, vp]
    L.sfw_step.argtypes = [vp, vp, ctypes.POINTER(Atoms), dbl, vp, vp, vp, vp, vp, vp, vp]
    L.sfw_step_topk.argtypes = [vp, vp, ctypes.POINTER(Atoms), dbl, vp, vp, vp, i32, vp, vp, vp, vp, vp, vp, vp]
    L.sfw_plan_check.argtypes = [vp]
    L.sfw_profile_start.argtypes = [i32, ctypes.c_char_p]
    L.sfw_gram.argtypes = [vp, ctypes.POINTER(Atoms), vp, vp, vp, vp]
    L.sfw_batch_create.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(BatchVolume),
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(vp)]
    L.sfw_batch_destroy.argtypes = [vp]
    L.sfw_batch_query.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.sfw_batch_step.argtypes = [vp, vp]
    L.sfw_batch_autotune.argtypes = [vp, ctypes.c_char_p, vp]
    L.sfw_profile_stop.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    L.sfw_profile_collect.argtypes = []
    for name in ("sfw_plan_create", "sfw_plan_destroy", "sfw_plan_query", "sfw_plan_check", "sfw_autotune",
                 "sfw_forward",
                 "sfw_certificate_grid", "sfw_certificate_topk", "sfw_eta_points", "sfw_argmax", "sfw_argmax_noalloc",
                 "sfw_slide_loss_grad", "sfw_step", "sfw_step_topk", "sfw_gram", "sfw_batch_create", "sfw_batch_destroy",
           "sfw_batch_query", "sfw_batch_step", "sfw_batch_autotune", "sfw_profile_start", "sfw_profile_collect",
                 "sfw_profile_stop"):
        getattr(L, name).restype = ctypes.c_int
    L.sfw_last_error.restype = ctypes.c_char_p
    L.sfw_last_error.argtypes = []
    L.sfw_launch_count.restype = ctypes.c_int64
    L.sfw_launch_count.argtypes = []
    L.sfw_version.restype = ctypes.c_char_p
    L.sfw_version.argtypes = []
    _lib = L
    return L


def check(status: int, where: str) -> None:
    if status != SFW_OK:
        raise SfwError(status, where, lib().sfw_last_error().decode())


# ---- the entry points, same names as the C ABI ------------------------------------------

def sfw_plan_create(desc: PlanDesc) -> int:
    h = ctypes.c_void_p()
    check(lib().sfw_plan_create(ctypes.byref(desc), ctypes.byref(h)), "sfw_plan_create")
    return h.value


def sfw_plan_destroy(plan: int) -> None:
    check(lib().sfw_plan_destroy(plan), "sfw_plan_destroy")


def sfw_plan_query(plan: int) -> PlanInfo:
    info = PlanInfo()
    check(lib().sfw_plan_query(plan, ctypes.byref(info)), "sfw_plan_query")
    return info


def sfw_autotune(plan: int, cache_path, stream: int) -> None:
    check(lib().sfw_autotune(plan, cache_path.encode() if cache_path else None, stream), "sfw_autotune")


def sfw_forward(plan: int, atoms: Atoms, y_out: int, stream: int) -> None:
    check(lib().sfw_forward(plan, ctypes.byref(atoms), y_out, stream), "sfw_forward")


def sfw_certificate_grid(plan: int, residual: int, lam: float, eta_out: int, max_out: int,
                         argk_out: int, best_val: int, best_idx: int, stream: int) -> None:
    check(lib().sfw_certificate_grid(plan, residual, float(lam), eta_out, max_out, argk_out,
                                     best_val, best_idx, stream), "sfw_certificate_grid")


def sfw_certificate_topk(plan: int, residual: int, lam: float, topk: int, cand_theta: int,
                         cand_grid: int, cand_eta: int, best_theta: int, best_eta: int,
                         stream: int) -> None:
    check(lib().sfw_certificate_topk(plan, residual, float(lam), int(topk), cand_theta, cand_grid,
                                     cand_eta, best_theta, best_eta, stream), "sfw_certificate_topk")


def sfw_eta_points(plan: int, residual: int, lam: float, P: int, theta: int, eta_out: int,
                   grad_out: int, stream: int) -> None:
    check(lib().sfw_eta_points(plan, residual, float(lam), int(P), theta, eta_out, grad_out, stream),
          "sfw_eta_points")


def sfw_argmax(values: int, count: int, topk: int, val_out: int, idx_out: int, stream: int) -> None:
    check(lib().sfw_argmax(values, int(count), int(topk), val_out, idx_out, stream), "sfw_argmax")


def sfw_argmax_noalloc(values: int, count: int, topk: int, val_out: int, idx_out: int,
                       stream: int) -> None:
    """sfw_argmax for callers that cannot allocate device memory: its scratch is a static
    2 MiB device array of the library (see include/sfw.h for the size limit and the
    sharing rules)."""
    check(lib().sfw_argmax_noalloc(values, int(count), int(topk), val_out, idx_out, stream),
          "sfw_argmax_noalloc")


def sfw_slide_loss_grad(plan: int, y: int, atoms: Atoms, lam: float, loss_out: int, grad_out: int,
                        residual_out: int, stream: int) -> None:
    check(lib().sfw_slide_loss_grad(plan, y, ctypes.byref(atoms), float(lam), loss_out, grad_out,
                                    residual_out, stream), "sfw_slide_loss_grad")


def sfw_plan_check(plan: int) -> None:
    check(lib().sfw_plan_check(plan), "sfw_plan_check")


def sfw_step(plan: int, y: int, atoms: Atoms, lam: float, loss_out: int, grad_out: int,
             residual_out: int, best_val: int, best_idx: int, stream: int, aux_stream: int) -> None:
    check(lib().sfw_step(plan, y, ctypes.byref(atoms), float(lam), loss_out, grad_out, residual_out,
                         best_val, best_idx, stream, aux_stream), "sfw_step")


def sfw_step_topk(plan: int, y: int, atoms: Atoms, lam: float, loss_out: int, grad_out: int,
                  residual_out: int, topk: int, cand_theta: int, cand_grid: int, cand_eta: int,
                  best_theta: int, best_eta: int, stream: int, aux_stream: int) -> None:
    check(lib().sfw_step_topk(plan, y, ctypes.byref(atoms), float(lam), loss_out, grad_out, residual_out,
                              int(topk), cand_theta, cand_grid, cand_eta, best_theta, best_eta, stream,
                              aux_stream), "sfw_step_topk")


def sfw_gram(plan: int, atoms: Atoms, y: int, G_out: int, c_out: int, stream: int) -> None:
    check(lib().sfw_gram(plan, ctypes.byref(atoms), y, G_out, c_out, stream), "sfw_gram")


def sfw_batch_create(plans, vols, lambdas) -> int:
    n = len(plans)
    arr = (ctypes.c_void_p * n)(*plans)
    va = (BatchVolume * n)(*vols)
    la = (ctypes.c_double * n)(*[float(x) for x in lambdas])
    h = ctypes.c_void_p()
    check(lib().sfw_batch_create(n, arr, va, la, ctypes.byref(h)), "sfw_batch_create")
    return h.value


def sfw_batch_destroy(batch: int) -> None:
    check(lib().sfw_batch_destroy(batch), "sfw_batch_destroy")


def sfw_batch_query(batch: int) -> int:
    n = ctypes.c_int()
    check(lib().sfw_batch_query(batch, ctypes.byref(n)), "sfw_batch_query")
    return n.value


def sfw_batch_step(batch: int, stream: int) -> None:
    check(lib().sfw_batch_step(batch, stream), "sfw_batch_step")


def sfw_batch_autotune(batch: int, cache_path, stream: int) -> None:
    check(lib().sfw_batch_autotune(batch, cache_path.encode() if cache_path else None, stream),
          "sfw_batch_autotune")


def sfw_profile_start(max_launches: int, only_tag: str = None) -> None:
    check(lib().sfw_profile_start(int(max_launches), only_tag.encode() if only_tag else None),
          "sfw_profile_start")


def sfw_profile_collect() -> None:
    check(lib().sfw_profile_collect(), "sfw_profile_collect")


def sfw_profile_stop() -> dict:
    import json
    buf = ctypes.create_string_buffer(1 << 16)
    check(lib().sfw_profile_stop(buf, len(buf)), "sfw_profile_stop")
    return {k: {"launches": v[0], "ms": v[1]} for k, v in json.loads(buf.value.decode()).items()}


def sfw_launch_count() -> int:
    return int(lib().sfw_launch_count())


def sfw_version() -> str:
    return lib().sfw_version().decode()
