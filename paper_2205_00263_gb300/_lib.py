"""ctypes declarations of the libmnbab C ABI (include/mnbab.h)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmnbab.so")

status = C.c_int32
node_id = C.c_int64

OK = 0
E_INVALID_ARG = -1
E_BUDGET = -2
E_DEVICE = -3
E_TIMEOUT = -4
E_UNSUPPORTED = -5
UNKNOWN, VERIFIED, FALSIFIED = 0, 1, -1
FC, CONV2D, RELU, ADD = 1, 2, 3, 4


class Options(C.Structure):
    _fields_ = [("device", C.c_int32), ("hbm_budget_bytes", C.c_uint64), ("stream", C.c_void_p),
                ("node_capacity", C.c_int32), ("max_mnc_rows", C.c_int32),
                ("row_chunk", C.c_int32), ("gemm_path", C.c_int32),
                ("use_graphs", C.c_int32)]


class LayerDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("in_c", C.c_int32), ("in_h", C.c_int32),
                ("in_w", C.c_int32), ("out_c", C.c_int32), ("out_h", C.c_int32),
                ("out_w", C.c_int32), ("k", C.c_int32), ("stride", C.c_int32),
                ("pad", C.c_int32), ("W", C.POINTER(C.c_float)), ("b", C.POINTER(C.c_float)),
                ("src_a", C.c_int32), ("src_b", C.c_int32)]


class Adam(C.Structure):
    _fields_ = [("steps", C.c_int32), ("lr_alpha", C.c_float), ("lr_beta", C.c_float),
                ("lr_gamma", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("grad_floor", C.c_float), ("eps_rel", C.c_float)]


class StepStats(C.Structure):
    _fields_ = [("nodes_bounded", C.c_int32), ("nodes_verified", C.c_int32),
                ("nodes_falsified", C.c_int32), ("nodes_branched", C.c_int32),
                ("nodes_leaf", C.c_int32), ("props_done", C.c_int32),
                ("rows_rebounded", C.c_int64), ("h2d_bytes", C.c_int64),
                ("d2h_bytes", C.c_int64)]


class ServeStats(C.Structure):
    _fields_ = [("admitted", C.c_int32), ("finished", C.c_int32), ("active", C.c_int32),
                ("queued", C.c_int32), ("step", StepStats), ("reserved_bytes", C.c_int64)]


class TuneRec(C.Structure):
    _fields_ = [("node", C.c_int32), ("edge", C.c_int32), ("dir", C.c_int32),
                ("rows", C.c_int32), ("variant", C.c_int32), ("ms", C.c_float * 8)]


class KernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("ms", C.c_double),
                ("flops", C.c_double), ("bytes", C.c_double)]


class TraceRec(C.Structure):
    _fields_ = [("seq", C.c_int64), ("row", C.c_int32), ("depth", C.c_int32), ("lb", C.c_float),
                ("lb_deeppoly", C.c_float), ("f_xstar", C.c_float), ("verdict", C.c_int32),
                ("split_layer", C.c_int32), ("split_neuron", C.c_int32),
                ("fallback", C.c_int32), ("leaf", C.c_int32)]


FP = C.POINTER(C.c_float)
IP = C.POINTER(C.c_int32)
VP = C.c_void_p

# name -> (restype, argtypes); every entry point of include/mnbab.h
SIGNATURES = {
    "mnbab_create": (status, [C.POINTER(Options), C.POINTER(VP)]),
    "mnbab_destroy": (None, [VP]),
    "mnbab_last_error": (C.c_char_p, [VP]),
    "mnbab_load_network": (status, [VP, C.POINTER(LayerDesc), C.c_int32, C.POINTER(VP)]),
    "mnbab_set_property": (status, [VP, VP, FP, FP, FP, FP, C.c_int32, C.POINTER(VP)]),
    "mnbab_get_root_bounds": (status, [VP, VP, C.c_int32, FP, FP]),
    "mnbab_set_mnc": (status, [VP, VP, C.c_int32, C.c_int32, C.c_int32, IP, FP, FP, FP]),
    "mnbab_generate_mnc": (status, [VP, VP, C.c_int32, C.POINTER(C.c_int64)]),
    "mnbab_get_mnc": (status, [VP, VP, C.c_int32, C.c_int32, IP, FP, FP, FP, IP]),
    "mnbab_mnc_group": (status, [C.POINTER(C.c_double), C.c_int32, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), C.POINTER(C.c_double), IP]),
    "mnbab_node_root": (status, [VP, VP, C.c_int32, C.POINTER(node_id)]),
    "mnbab_node_free": (status, [VP, node_id]),
    "mnbab_export_params": (status, [VP, node_id, VP, C.POINTER(C.c_size_t)]),
    "mnbab_import_params": (status, [VP, node_id, VP, C.c_size_t]),
    "mnbab_bound_batch": (status, [VP, C.POINTER(node_id), C.c_int32, FP, FP]),
    "mnbab_deeppoly_batch": (status, [VP, C.POINTER(node_id), C.c_int32, FP]),
    "mnbab_bound_grad": (status, [VP, C.POINTER(node_id), C.c_int32, FP, FP]),
    "mnbab_set_params": (status, [VP, C.POINTER(node_id), C.c_int32, FP]),
    "mnbab_optimize": (status, [VP, C.POINTER(node_id), C.c_int32, C.POINTER(Adam), FP]),
    "mnbab_optimize_intermediate": (status, [VP, C.POINTER(node_id), C.c_int32, C.c_int32,
                                             C.POINTER(Adam), C.POINTER(C.c_int64)]),
    "mnbab_score_branches": (status, [VP, C.POINTER(node_id), C.c_int32, IP, IP, FP]),
    "mnbab_bab_step": (status, [VP, C.POINTER(VP), C.c_int32, C.c_int32, C.POINTER(Adam),
                                C.POINTER(StepStats)]),
    "mnbab_set_budget": (status, [VP, VP, C.c_int32]),
    "mnbab_set_timeout": (status, [VP, VP, C.c_double]),
    "mnbab_get_status": (status, [VP, VP, IP, IP, C.POINTER(C.c_double)]),
    "mnbab_set_leaf_steps": (status, [VP, VP, C.c_int32]),
    "mnbab_set_branching": (status, [VP, VP, C.c_int32]),
    "mnbab_set_intermediate_steps": (status, [VP, VP, C.c_int32]),
    "mnbab_get_verdict": (status, [VP, VP, C.c_int32, IP, FP, FP]),
    "mnbab_get_trace": (status, [VP, VP, C.POINTER(TraceRec), C.c_int32, IP]),
    "mnbab_queue_size": (status, [VP, VP, IP]),
    "mnbab_attack": (status, [VP, VP, C.c_int32, C.c_int32, FP, FP, FP]),
    "mnbab_set_attack": (status, [VP, VP, C.c_int32, C.c_int32, C.c_uint64]),
    "mnbab_profile": (status, [VP, C.c_int32]),
    "mnbab_profile_mask": (status, [VP, C.c_uint64]),
    "mnbab_submit": (status, [VP, VP, C.c_double, C.POINTER(C.c_uint64)]),
    "mnbab_serve_step": (status, [VP, C.c_int32, C.POINTER(Adam), C.POINTER(ServeStats)]),
    "mnbab_set_serving_budget": (status, [VP, C.c_uint64]),
    "mnbab_set_attack_path": (status, [VP, C.c_int32]),
    "mnbab_autotune": (status, [VP, VP, C.c_int32, C.POINTER(TuneRec), C.c_int32, IP]),
    "mnbab_set_variant": (status, [VP, VP, C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    "mnbab_poll": (status, [VP, C.c_uint64, IP]),
    "mnbab_request_result": (status, [VP, C.c_uint64, IP, C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), IP]),
    "mnbab_deeppoly_fc_noalloc": (status, [C.c_int32, IP, C.POINTER(VP), C.POINTER(VP), VP, VP,
                                           VP, VP, VP, VP, C.c_int32, VP, VP, C.c_char_p,
                                           C.c_size_t]),
    "mnbab_profile_read": (status, [VP, C.POINTER(KernelStat), C.c_int32, IP,
                                    C.POINTER(C.c_int64)]),
}

_lib = None


def load(path: str | None = None):
    """Loads libmnbab.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libmnbab.so not built at {p}; run paper_2205_00263_gb300.build.build()")
    lib = C.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib
