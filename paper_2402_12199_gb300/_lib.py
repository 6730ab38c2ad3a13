"""ctypes loader for the in-tree CUDA library (librb.so) and its C ABI.

Argument marshalling only.  The library must have been built (see
``build_lib.build``); there is no fallback: a missing library raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "_build", "librb.so")

STATUS = {0: "RB_OK", 1: "RB_EINVAL", 2: "RB_ENOMEM", 3: "RB_ECUDA", 4: "RB_EOVERFLOW",
          5: "RB_ENOT_READY", 6: "RB_ETIMEOUT", 7: "RB_EFAULT", 8: "RB_EBUSY", 9: "RB_ENOTSUP"}
RB_OK, RB_EINVAL, RB_ENOMEM, RB_ECUDA, RB_EOVERFLOW = 0, 1, 2, 3, 4
RB_ENOT_READY, RB_ETIMEOUT, RB_EFAULT, RB_EBUSY, RB_ENOTSUP = 5, 6, 7, 8, 9
RB_SHAPE_CUBE, RB_SHAPE_CYLINDER, RB_SHAPE_CUSTOM = 0, 1, 2
RB_POT_LJ, RB_POT_HPHC, RB_POT_HPHC_PRINTED = 0, 1, 2
RB_PATH_BEADS, RB_PATH_NN, RB_PATH_FNET = 0, 1, 2
RB_FP32, RB_BF16, RB_F16X3 = 0, 1, 2
RB_DESC_FEATURES10, RB_DESC_PAPER6 = 0, 1


class RBError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class rb_body_type(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int32), ("n_beads", ctypes.c_int32),
                ("bead_xyz_host", ctypes.POINTER(ctypes.c_float)), ("bead_mass", ctypes.c_float)]


class rb_bead_potential(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("eps", ctypes.c_float), ("sigma", ctypes.c_float),
                ("rcut", ctypes.c_float), ("A", ctypes.c_float), ("b", ctypes.c_float),
                ("c", ctypes.c_float), ("p", ctypes.c_float)]


class rb_system_desc(ctypes.Structure):
    _fields_ = [("body", rb_body_type), ("pot", rb_bead_potential), ("box", ctypes.c_float * 3),
                ("n_bodies", ctypes.c_int64), ("max_neighbors", ctypes.c_int32),
                ("skin", ctypes.c_float)]


class rb_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("fell_back", ctypes.c_int32),
                ("n_bodies", ctypes.c_int64), ("steps_done", ctypes.c_int64),
                ("pairs", ctypes.c_int64), ("e_start", ctypes.c_double),
                ("e_end", ctypes.c_double), ("step_ms_p50", ctypes.c_double),
                ("step_ms_p99", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double)]


class rb_server_stats_t(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int64), ("resident", ctypes.c_int64),
                ("peak_resident", ctypes.c_int64), ("bytes_in_use", ctypes.c_int64),
                ("steps", ctypes.c_int64), ("pair_evals", ctypes.c_double),
                ("step_ms_p50", ctypes.c_double), ("step_ms_p99", ctypes.c_double)]


P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
F32 = ctypes.c_float
DP = ctypes.POINTER(ctypes.c_double)
FP = ctypes.POINTER(ctypes.c_float)
I32P = ctypes.POINTER(ctypes.c_int32)
I64P = ctypes.POINTER(ctypes.c_int64)

# name -> (restype, argtypes)
SIGNATURES = {
    "rb_last_error": (ctypes.c_char_p, []),
    "rb_abi_version": (I32, []),
    "rb_create_system": (I32, [ctypes.POINTER(rb_system_desc), P, ctypes.POINTER(P)]),
    "rb_destroy_system": (I32, [P]),
    "rb_body_info": (I32, [P, FP, FP, FP, FP, I32P]),
    "rb_body_template": (I32, [P, FP]),
    "rb_set_state": (I32, [P, P, P, P, P, I32]),
    "rb_get_state": (I32, [P, P, P, P, P, I32]),
    "rb_get_forces": (I32, [P, P, P, I32]),
    "rb_set_forces": (I32, [P, I32, P, I32, P, P, I32]),
    "rb_step_host_state": (I32, [P, I32, P, I32, I64, F32, P, I32]),
    "rb_build_pairs": (I32, [P, I64P]),
    "rb_get_pairs": (I32, [P, I32P, I64, I64P]),
    "rb_forces_beads": (I32, [P, P, P, DP, DP]),
    "rb_step": (I32, [P, I32, P, I32, I64, F32]),
    "rb_eval_pairs": (I32, [P, I32, P, I32]),
    "rb_energy": (I32, [P, DP, DP, DP]),
    "rb_sync": (I32, [P]),
    "rb_checkpoint": (I32, [P, ctypes.c_char_p]),
    "rb_restore": (I32, [P, ctypes.c_char_p]),
    "rb_get_step": (I32, [P, I64P]),
    "rb_fnet_n_params": (I64, [I32, I32]),
    "rb_fnet_create": (I32, [I32, I32, P, ctypes.POINTER(P)]),
    "rb_fnet_destroy": (I32, [P]),
    "rb_fnet_set_params": (I32, [P, P, I64, I32]),
    "rb_fnet_get_params": (I32, [P, P, I64, I32]),
    "rb_fnet_pairs": (I32, [P, I64, P, P]),
    "rb_forces_fnet": (I32, [P, P, P, P, DP]),
    "rb_step_fnet": (I32, [P, P, I64, F32]),
    "rb_fnet_trainer_create": (I32, [P, I64, F32, F32, F32, F32, ctypes.POINTER(P)]),
    "rb_fnet_trainer_destroy": (I32, [P]),
    "rb_fnet_trainer_set_lr": (I32, [P, F32]),
    "rb_fnet_trainer_set_cap": (I32, [P, F32, F32]),
    "rb_fnet_train_grad": (I32, [P, I64, P, P, P, DP]),
    "rb_fnet_train_step": (I32, [P, I64, P, P, DP]),
    "rb_set_thermostat": (I32, [P, F32, F32]),
    "rb_get_thermostat": (I32, [P, DP]),
    "rb_set_reference": (I32, [P]),
    "rb_msd_msr": (I32, [P, DP, DP]),
    "rb_get_images": (I32, [P, I32P]),
    "rb_gr_counts": (I32, [P, F32, I32, P]),
    "rb_gr_normalise": (I32, [P, ctypes.POINTER(ctypes.c_uint32), I32, F32, I64, DP]),
    "rb_mlp_n_params": (I64, [I32, I32]),
    "rb_mlp_create": (I32, [I32, I32, P, ctypes.POINTER(P)]),
    "rb_mlp_destroy": (I32, [P]),
    "rb_mlp_set_params": (I32, [P, P, I64, I32]),
    "rb_mlp_get_params": (I32, [P, P, I64, I32]),
    "rb_forces_nn": (I32, [P, P, I32, P, P, DP, DP]),
    "rb_nn_pairs": (I32, [P, I32, I64, P, P, P]),
    "rb_mlp_sync": (I32, [P]),
    "rb_template_symmetry": (I32, [P, I32, P, P, P]),
    "rb_mlp_set_symmetry": (I32, [P, P, I32, I32]),
    "rb_mlp_set_cutoff": (I32, [P, F32, F32]),
    "rb_mlp_set_pair_symmetrised": (I32, [P, I32]),
    "rb_pairs_swap_reference": (I32, [I64, P, P, P]),
    "rb_nn_canonical": (I32, [P, I64, P, P]),
    "rb_mlp_set_descriptor": (I32, [P, I32]),
    "rb_nn_features": (I32, [P, I64, P, P]),
    "rb_set_nn_fallback": (I32, [P, F32]),
    "rb_set_skin": (I32, [P, F32]),
    "rb_nn_fallback_count": (I32, [P, I64P]),
    "rb_system_footprint": (I64, [ctypes.POINTER(rb_system_desc)]),
    "rb_server_create": (I32, [ctypes.c_size_t, I32, P, I32, ctypes.POINTER(P)]),
    "rb_server_destroy": (I32, [P]),
    "rb_server_set_lanes": (I32, [P, I32]),
    "rb_server_set_network": (I32, [P, I32, P, ctypes.c_float]),
    "rb_submit": (I32, [P, ctypes.POINTER(rb_system_desc), P, P, P, P, I32, I32, I64, F32,
                        ctypes.POINTER(ctypes.c_uint64)]),
    "rb_poll": (I32, [P, ctypes.c_uint64, ctypes.POINTER(rb_result)]),
    "rb_wait": (I32, [P, ctypes.c_uint64, I32, ctypes.POINTER(rb_result)]),
    "rb_fetch_state": (I32, [P, ctypes.c_uint64, P, P, P, P]),
    "rb_server_stats": (I32, [P, ctypes.POINTER(rb_server_stats_t)]),
    "rb_sample_pairs": (I32, [P, I64, P, P, P, P]),
    "rb_sample_pairs_at": (I32, [P, I64, P, F32, P, P, P]),
    "rb_trainer_create": (I32, [P, I64, F32, F32, F32, F32, ctypes.POINTER(P)]),
    "rb_trainer_destroy": (I32, [P]),
    "rb_trainer_set_lr": (I32, [P, F32]),
    "rb_train_grad": (I32, [P, I64, P, P, F32, F32, F32, F32, P, DP]),
    "rb_train_step": (I32, [P, I64, P, P, F32, F32, F32, F32, DP]),
    "rb_nn_weight_vjp": (I32, [P, I64, P, P, P, P]),
    "rb_tc_gemm_check": (I32, [I32, I32, P, P, P, P]),
    "rb_gemm_f32": (I32, [I64, I64, I64, P, I64, I64, P, I64, I64, P, I64, F32, F32, P, I64, P]),
    "rb_peak_probe": (I32, [I32, I32, I64, P, P]),
}

_lock = threading.Lock()
_lib = None


def load() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(SO):
                raise RuntimeError(f"CUDA library not built ({SO} missing): run "
                                   "paper_2402_12199_gb300.build_lib.build() first")
            L = ctypes.CDLL(SO)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def check(status: int) -> None:
    if status != RB_OK:
        raise RBError(status, load().rb_last_error().decode(errors="replace"))
