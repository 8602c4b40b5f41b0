"""ctypes declarations of the C ABI in include/satsampler.h.

Argument marshalling only.  The shared library must have been built
(``paper_2502_08673_b300.build``); there is no fallback when it is missing.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

LIB_PATH = Path(__file__).resolve().parent / "libsatsampler.so"

SAT_OK, SAT_PARTIAL = 0, 1
STATUS_NAMES = {0: "SAT_OK", 1: "SAT_PARTIAL", -1: "SAT_ERR_PARSE", -2: "SAT_ERR_ARG", -3: "SAT_ERR_OOM",
                -4: "SAT_ERR_CUDA", -5: "SAT_ERR_TABLE_FULL", -6: "SAT_ERR_UNSAT_TRIVIAL"}
ACT_DTYPES = {"f32": 0, "bf16": 1, "f16": 2}
TILE = 128  # SAT_TILE
OPTIMIZERS = {"adam": 0, "gd": 1}


class SatError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class BuildOpts(C.Structure):
    _fields_ = [("max_support", C.c_uint32), ("max_window", C.c_uint32), ("direct", C.c_uint32),
                ("reorder", C.c_uint32)]


class BuildStats(C.Structure):
    _fields_ = [("n_vars", C.c_uint32), ("n_pi", C.c_uint32), ("n_iv", C.c_uint32), ("n_outputs", C.c_uint32),
                ("n_const", C.c_uint32), ("n_gates", C.c_uint64), ("n_cone_pi", C.c_uint32),
                ("n_cone_gates", C.c_uint64), ("n_levels", C.c_uint32), ("n_cone_levels", C.c_uint32),
                ("max_span", C.c_uint32), ("ops_cnf", C.c_uint64), ("ops_circuit", C.c_uint64),
                ("transform_ms", C.c_double), ("plan_ms", C.c_double)]


class PlanInfo(C.Structure):
    _fields_ = [("n_vars", C.c_uint32), ("n_pi", C.c_uint32), ("n_cone_pi", C.c_uint32), ("n_outputs", C.c_uint32),
                ("n_cone_levels", C.c_uint32), ("n_levels", C.c_uint32), ("key_words", C.c_uint32),
                ("max_span", C.c_uint32), ("n_cone", C.c_uint64), ("n_nodes", C.c_uint64),
                ("n_cone_gates", C.c_uint64), ("n_gates", C.c_uint64), ("n_clauses", C.c_uint64),
                ("n_fanout_edges", C.c_uint64), ("upload_bytes", C.c_uint64)]


class OptParams(C.Structure):
    _fields_ = [("optimizer", C.c_int32), ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float)]


class SampleOpts(C.Structure):
    _fields_ = [("batch", C.c_int64), ("steps", C.c_int32), ("max_rounds", C.c_int32), ("opt", OptParams),
                ("seed", C.c_uint64), ("first_round", C.c_uint32), ("init_scale", C.c_float),
                ("act_dtype", C.c_int32), ("steps_per_launch", C.c_int32), ("init_logits", C.c_void_p),
                ("init_ld", C.c_int64), ("stream", C.c_void_p), ("proposal", C.c_void_p),
                ("proposal_tau", C.c_float), ("check_every", C.c_int32), ("max_age", C.c_int32),
                ("recompute_segment", C.c_int32), ("step_kernel", C.c_int32)]


class SampleStats(C.Structure):
    _fields_ = [("rounds", C.c_uint32), ("samples", C.c_uint64), ("valid", C.c_uint64), ("unique", C.c_uint64),
                ("ms_init", C.c_double), ("ms_steps", C.c_double), ("ms_verify", C.c_double),
                ("ms_dedup", C.c_double), ("ms_total", C.c_double), ("ms_upload", C.c_double),
                ("ms_download", C.c_double)]


class RoundInfo(C.Structure):
    _fields_ = [("available", C.c_int32), ("compiled", C.c_int32), ("registers", C.c_int32),
                ("spill_bytes", C.c_int32), ("min_blocks", C.c_int32), ("compile_ms", C.c_double)]


P, I32, I64, U32, U64, F32, SZ = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_float, C.c_size_t
PP = C.POINTER(C.c_void_p)

# name -> (restype, argtypes); restype int32 = sat_status
PROTOTYPES = {
    "sat_version": (C.c_char_p, []),
    "sat_last_error": (C.c_char_p, []),
    "sat_cnf_from_dimacs": (I32, [C.c_char_p, SZ, PP]),
    "sat_cnf_from_file": (I32, [C.c_char_p, PP]),
    "sat_cnf_info": (I32, [P, C.POINTER(U32), C.POINTER(U64), C.POINTER(U64)]),
    "sat_cnf_free": (None, [P]),
    "sat_circuit_build": (I32, [P, C.POINTER(BuildOpts), PP, C.POINTER(BuildStats)]),
    "sat_circuit_dump": (I32, [P, C.c_char_p, SZ, C.POINTER(SZ)]),
    "sat_circuit_free": (None, [P]),
    "sat_plan_create": (I32, [P, P, PP]),
    "sat_plan_get_info": (I32, [P, C.POINTER(PlanInfo)]),
    "sat_plan_pi_vars": (I32, [P, P]),
    "sat_plan_var_nodes": (I32, [P, P, P, P]),
    "sat_plan_scratch_elems": (I32, [P, I64, C.POINTER(U64)]),
    "sat_plan_layout_elems": (I32, [P, I32, I64, C.POINTER(U64), C.POINTER(U64)]),
    "sat_diag_bounded_wait": (I32, [U32, C.POINTER(U32), P]),
    "sat_diag_angle_signs": (I32, [C.POINTER(U32), P]),
    "sat_cached_memory": (I32, [C.POINTER(U64), C.POINTER(U64)]),
    "sat_release_cached_memory": (I32, []),
    "sat_plan_status": (I32, [P, C.POINTER(U32), I32, P]),
    "sat_plan_set_step_kernel": (I32, [P, I32]),
    "sat_plan_step_kernel": (I32, [P, I32, C.POINTER(I32)]),
    "sat_plan_free": (None, [P]),
    "sat_init_normal": (I32, [P, U64, U32, F32, P, I64, I64, P]),
    "sat_forward": (I32, [P, I32, P, I64, P, P, I64, P]),
    "sat_backward": (I32, [P, I32, P, I64, P, P, P, P, I64, P]),
    "sat_opt_update": (I32, [P, C.POINTER(OptParams), P, P, P, P, I64, I32, I64, P]),
    "sat_steps": (I32, [P, I32, C.POINTER(OptParams), P, P, P, I64, P, P, P, I32, I32, I64, P]),
    "sat_steps_noalloc": (I32, [P, I32, C.POINTER(OptParams), P, P, P, I64, P, I32, I32, I64, P]),
    "sat_steps_aged": (I32, [P, I32, C.POINTER(OptParams), P, P, P, I64, P, P, P, P, I32, I32, I64, P]),
    "sat_steps_recompute": (I32, [P, I32, C.POINTER(OptParams), P, P, P, I64, P, P, P, P, I32, I32, I64, I32, P]),
    "sat_retire": (I32, [P, P, P, I32, I32, I64, P]),
    "sat_restart": (I32, [P, P, U64, U32, F32, P, I64, P, P, P, I64, I64, P]),
    "sat_threshold": (I32, [P, P, I64, P, I64, P, I64, P]),
    "sat_hard_eval": (I32, [P, P, I64, I64, P]),
    "sat_cnf_check": (I32, [P, P, I64, P, I64, P]),
    "sat_circuit_round_program": (I32, [P, I32, C.c_char_p, SZ, C.POINTER(SZ)]),
    "sat_plan_round_info": (I32, [P, I32, C.POINTER(RoundInfo)]),
    "sat_round_gd": (I32, [P, F32, I32, U64, U32, F32, P, I64, P, P, I64, P]),
    "sat_dedup_create": (I32, [P, U64, I64, PP]),
    "sat_dedup_insert": (I32, [P, P, P, I64, P, P, P]),
    "sat_dedup_insert_async": (I32, [P, P, P, I64, P]),
    "sat_dedup_check": (I32, [P, P]),
    "sat_dedup_count": (I32, [P, C.POINTER(U64), P]),
    "sat_dedup_copy_keys": (I32, [P, U64, U64, P, P]),
    "sat_dedup_clear": (I32, [P, P]),
    "sat_dedup_free": (None, [P]),
    "sat_gemm_bf16": (I32, [I32, I32, I32, P, I64, P, I64, P, I32, P, I64, F32, P, P, I64, P, P, I64, P, P]),
    "sat_mlp_create": (I32, [U32, U32, U32, I64, U64, PP]),
    "sat_mlp_num_params": (I32, [P, C.POINTER(U64)]),
    "sat_mlp_get_params": (I32, [P, P]),
    "sat_mlp_set_params": (I32, [P, P]),
    "sat_mlp_draw_noise": (I32, [P, U64, U32, P, I64, P]),
    "sat_mlp_forward": (I32, [P, P, I64, F32, P, I64, P]),
    "sat_mlp_propose": (I32, [P, U64, U32, F32, P, I64, I64, P]),
    "sat_mlp_imle_select": (I32, [P, P, P, I32, I64, I32, P, P, P]),
    "sat_mlp_loss_grad": (I32, [P, P, P, I32, I64, P, P, P]),
    "sat_mlp_apply_grad": (I32, [P, P, F32, P]),
    "sat_mlp_train_step": (I32, [P, P, I32, I64, I32, F32, U64, U32, P, P]),
    "sat_mlp_train": (I32, [P, P, P, U64, I32, I64, I32, F32, U64, P, P]),
    "sat_mlp_status": (I32, [P, C.POINTER(U32)]),
    "sat_mlp_free": (None, [P]),
    "sat_sample_opts_default": (None, [C.POINTER(SampleOpts)]),
    "sat_sample": (I32, [P, P, C.POINTER(SampleOpts), U64, PP, C.POINTER(SampleStats)]),
    "sat_sample_plan": (I32, [P, P, C.POINTER(SampleOpts), U64, C.POINTER(SampleStats)]),
    "sat_solutions_count": (U64, [P]),
    "sat_solutions_nvars": (U32, [P]),
    "sat_solutions_copy": (I32, [P, U64, U64, P]),
    "sat_solutions_free": (None, [P]),
}

_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise ImportError(f"{LIB_PATH.name} is not built: run `python -m paper_2502_08673_b300.build`")
        L = C.CDLL(str(LIB_PATH))
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int, allow_partial: bool = False) -> int:
    if status == SAT_OK or (allow_partial and status == SAT_PARTIAL):
        return status
    raise SatError(status, lib().sat_last_error().decode(errors="replace"))
