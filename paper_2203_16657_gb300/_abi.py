"""ctypes declarations of the libcia C ABI (include/cia.h).

Argument marshalling only: every computation happens inside libcia.so.
Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libcia.so")

CIA_MAX_HARMONICS = 4
CIA_MAX_POLY = 4

STATUS = {
    0: "CIA_OK", 1: "CIA_ERR_INVALID_ARG", 2: "CIA_ERR_INVALID_GRAPH", 3: "CIA_ERR_UNSUPPORTED",
    4: "CIA_ERR_CUDA", 5: "CIA_ERR_TIMEOUT", 6: "CIA_ERR_FALLBACK", 7: "CIA_ERR_NUMERIC",
    8: "CIA_ERR_OOM",
}
PRECISION = {"fp64": 0, "fp32": 1}
METHOD = {"cia": 0, "direct": 1}
STAGING = {"auto": 0, "plain": 1, "window": 2, "pipeline": 3, "stream": 4}
MODEL = {"kuramoto": 0, "kuramoto_ho": 1, "cucker_smale": 2, "polynomial": 3, "polynomial_general": 4,
         "fourier_general": 5}


class CiaError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        self.status_name = STATUS.get(status, "CIA_ERR_UNKNOWN")
        super().__init__("%s: %s" % (self.status_name, message))


class Graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p)]


class Coupling(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("p", ctypes.c_int),
                ("d_sin", ctypes.c_double * CIA_MAX_HARMONICS),
                ("d_cos", ctypes.c_double * CIA_MAX_HARMONICS),
                ("K", ctypes.c_double), ("K2", ctypes.c_double),
                ("sigma", ctypes.c_double), ("beta", ctypes.c_double),
                ("poly_c", ctypes.c_double * (CIA_MAX_POLY + 1)),
                ("dV", ctypes.c_double * (CIA_MAX_POLY + 1)),
                ("poly_g", ctypes.c_double * ((CIA_MAX_POLY + 1) * (CIA_MAX_POLY + 1))),
                ("fourier_L", ctypes.c_double),
                ("fourier_c", (ctypes.c_double * ((CIA_MAX_HARMONICS + 1) * (CIA_MAX_HARMONICS + 1))) * 4)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("build_direct", ctypes.c_int),
                ("tile_nodes", ctypes.c_int), ("group_size", ctypes.c_int),
                ("tile_index_bytes", ctypes.c_int), ("staging", ctypes.c_int),
                ("use_graphs", ctypes.c_int)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("M", ctypes.c_int64), ("n_free", ctypes.c_int64),
                ("max_community", ctypes.c_int64), ("nnz_graph", ctypes.c_int64),
                ("nnz_missing", ctypes.c_int64), ("nnz_inter", ctypes.c_int64),
                ("n_tiles", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("precision", ctypes.c_int), ("group_size", ctypes.c_int),
                ("tile_nodes", ctypes.c_int), ("missing_index_bytes", ctypes.c_int),
                ("staging", ctypes.c_int), ("group_size_direct", ctypes.c_int),
                ("max_tile_index_bytes", ctypes.c_int64), ("model", ctypes.c_int),
                ("state_dim", ctypes.c_int), ("instances", ctypes.c_int64), ("ring_slots", ctypes.c_int)]


class DetectOptions(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("community_cost", ctypes.c_double),
                ("min_size", ctypes.c_int), ("max_levels", ctypes.c_int), ("seed", ctypes.c_uint64)]


class DetectReport(ctypes.Structure):
    _fields_ = [("communities", ctypes.c_int64), ("unlabelled", ctypes.c_int64),
                ("nnz_missing", ctypes.c_int64), ("nnz_inter", ctypes.c_int64),
                ("hamiltonian", ctypes.c_double), ("levels", ctypes.c_int), ("moves", ctypes.c_int64)]


class TuneReport(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_int), ("tile_nodes", ctypes.c_int),
                ("tile_index_bytes", ctypes.c_int), ("staging", ctypes.c_int),
                ("best_ms_per_step", ctypes.c_double), ("worst_ms_per_step", ctypes.c_double)]


class PartitionReport(ctypes.Structure):
    _fields_ = [("communities", ctypes.c_int64 * 3), ("tiles", ctypes.c_int64 * 3), ("nnz_s", ctypes.c_int64 * 3),
                ("ms_per_step", ctypes.c_double * 3), ("per_tile_us", ctypes.c_double),
                ("per_byte_ps", ctypes.c_double), ("gamma", ctypes.c_double), ("community_cost", ctypes.c_double),
                ("probe_community_cost", ctypes.c_double), ("chosen", ctypes.c_int)]


class Profile(ctypes.Structure):
    _fields_ = [("stage_launches", ctypes.c_int64), ("stage_ms", ctypes.c_double),
                ("other_launches", ctypes.c_int64)]


CIA_BASIS_IN, CIA_BASIS_HIDDEN, CIA_BASIS_RANK = 2, 128, 64
CIA_BASIS_PARAMS = (CIA_BASIS_HIDDEN * CIA_BASIS_IN + CIA_BASIS_HIDDEN
                    + CIA_BASIS_RANK * CIA_BASIS_HIDDEN + CIA_BASIS_RANK)


class AdamOptions(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double)]


class FitOptions(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int64), ("epochs", ctypes.c_int64), ("adam", AdamOptions),
                ("lr_final", ctypes.c_double)]


class FitReport(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("first_loss", ctypes.c_double),
                ("last_epoch_loss", ctypes.c_double)]


class CheckReport(ctypes.Structure):
    _fields_ = [("checks", ctypes.c_int64), ("last_error", ctypes.c_double),
                ("max_error", ctypes.c_double), ("fell_back", ctypes.c_int),
                ("fallback_step", ctypes.c_int64)]


class LearnOptions(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("steps", ctypes.c_int64), ("snapshots", ctypes.c_int64),
                ("pairs", ctypes.c_int64), ("seed", ctypes.c_uint64), ("fit", FitOptions)]


class LearnReport(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_int64), ("fit", FitReport)]


# exported symbol -> (restype, argtypes)
_P = ctypes.c_void_p
SIGNATURES = {
    "cia_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "cia_last_error": (ctypes.c_char_p, []),
    "cia_plan_create": (ctypes.c_int, [ctypes.POINTER(Graph), _P, _P, ctypes.POINTER(Coupling),
                                       ctypes.POINTER(Options), ctypes.POINTER(_P)]),
    "cia_plan_destroy": (ctypes.c_int, [_P]),
    "cia_plan_create_batch": (ctypes.c_int, [ctypes.c_int64, _P, _P, _P, ctypes.POINTER(Coupling),
                                             ctypes.POINTER(Options), ctypes.POINTER(_P)]),
    "cia_plan_batch_begin": (ctypes.c_int, [ctypes.POINTER(Coupling), ctypes.POINTER(Options), ctypes.POINTER(_P)]),
    "cia_plan_batch_add": (ctypes.c_int, [_P, ctypes.POINTER(Graph), _P, _P]),
    "cia_plan_batch_finish": (ctypes.c_int, [_P]),
    "cia_plan_retile": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "cia_choose_partition": (ctypes.c_int, [ctypes.POINTER(Graph), _P, ctypes.POINTER(Coupling),
                                            ctypes.POINTER(Options), _P, ctypes.c_double, ctypes.c_int64, _P,
                                            ctypes.POINTER(PartitionReport)]),
    "cia_detect_options_default": (None, [_P]),
    "cia_detect_communities": (ctypes.c_int, [_P, _P, _P, _P]),
    "cia_plan_set_weights": (ctypes.c_int, [_P, _P, _P]),
    "cia_plan_autotune": (ctypes.c_int, [_P, _P, ctypes.c_double, ctypes.c_int64,
                                         ctypes.POINTER(TuneReport), _P]),
    "cia_plan_get_info": (ctypes.c_int, [_P, ctypes.POINTER(PlanInfo)]),
    "cia_plan_get_permutation": (ctypes.c_int, [_P, _P, _P]),
    "cia_plan_get_split": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "cia_rhs": (ctypes.c_int, [_P, _P, _P, _P]),
    "cia_rhs_direct": (ctypes.c_int, [_P, _P, _P, _P]),
    "cia_integrate": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_double, ctypes.c_int64, _P, _P]),
    "cia_integrate_host": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_double, ctypes.c_int64,
                                          _P, _P]),
    "cia_sync": (ctypes.c_int, [_P, _P]),
    "cia_selftest_bounded_wait": (ctypes.c_int, [_P, ctypes.c_int64, _P]),
    "cia_state_load": (ctypes.c_int, [_P, _P, _P]),
    "cia_state_store": (ctypes.c_int, [_P, _P, _P]),
    "cia_advance": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_int64, _P, _P]),
    "cia_profile_begin": (ctypes.c_int, [_P, ctypes.c_int64]),
    "cia_profile_end": (ctypes.c_int, [_P, ctypes.POINTER(Profile)]),
    "cia_rhs_kuramoto_static": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, _P, _P, _P, _P, _P,
                                               _P, _P, ctypes.POINTER(Coupling), _P, _P]),
    # include/cia_basis.h
    "cia_basis_create": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
    "cia_basis_params_fourier": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_uint64, _P]),
    "cia_basis_destroy": (ctypes.c_int, [_P]),
    "cia_basis_get_params": (ctypes.c_int, [_P, _P]),
    "cia_basis_features": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P]),
    "cia_basis_pair_grad": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P]),
    "cia_basis_adam_step": (ctypes.c_int, [_P, _P, ctypes.POINTER(AdamOptions), _P]),
    "cia_basis_fit": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.POINTER(FitOptions),
                                     ctypes.POINTER(FitReport), _P]),
    "cia_basis_sync": (ctypes.c_int, [_P, _P]),
    "cia_plan_set_basis": (ctypes.c_int, [_P, _P]),
    "cia_plan_sample_pairs": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_uint64, _P, _P]),
    "cia_plan_set_check": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double]),
    "cia_plan_get_check": (ctypes.c_int, [_P, ctypes.POINTER(CheckReport)]),
    "cia_learn_fit": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(LearnOptions),
                                     ctypes.POINTER(LearnReport), _P]),
}

_lib = None


def load() -> ctypes.CDLL:
    """Load libcia.so (built by paper_2203_16657_gb300.build); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libcia.so is not built (%s); run `python -m "
                              "paper_2203_16657_gb300.build` -- there is no fallback" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(status: int) -> None:
    if status != 0:
        msg = load().cia_last_error().decode(errors="replace")
        raise CiaError(status, msg)
