"""Argument checking of the C entry points (no GPU needed: every check below runs
before any device work).  Each invalid call returns SAT_ERR_ARG and leaves a
message in sat_last_error; no exception crosses the ABI."""
import ctypes as C

import pytest

from paper_2502_08673_b300 import _native as N

ERR_ARG = -2
L = N.lib()


def _err(status):
    assert status == ERR_ARG, status
    msg = L.sat_last_error().decode()
    assert msg
    return msg


def test_null_objects_are_rejected():
    out = C.c_void_p()
    _err(L.sat_circuit_build(None, None, C.byref(out), None))
    _err(L.sat_plan_create(None, None, C.byref(out)))
    _err(L.sat_dedup_create(None, 16, 16, C.byref(out)))
    opts = N.SampleOpts()
    L.sat_sample_opts_default(C.byref(opts))
    st = N.SampleStats()
    _err(L.sat_sample(None, None, C.byref(opts), 1, C.byref(out), C.byref(st)))
    _err(L.sat_sample_plan(None, None, C.byref(opts), 1, C.byref(st)))
    opt = N.OptParams(0, 0.1, 0.9, 0.999, 1e-8)
    _err(L.sat_steps(None, 0, C.byref(opt), None, None, None, 0, None, None, None, 1, 1, 0, None))
    _err(L.sat_steps_aged(None, 0, C.byref(opt), None, None, None, 0, None, None, None, None, 1, 1, 0, None))
    _err(L.sat_steps_recompute(None, 0, C.byref(opt), None, None, None, 0, None, None, None, None, 1, 1, 0, 8,
                               None))
    a, g = C.c_uint64(), C.c_uint64()
    _err(L.sat_plan_layout_elems(None, 8, 128, C.byref(a), C.byref(g)))
    _err(L.sat_threshold(None, None, 0, None, 0, None, 0, None))
    k = C.c_int32()
    _err(L.sat_plan_set_step_kernel(None, 0))
    _err(L.sat_plan_step_kernel(None, 0, C.byref(k)))
    _err(L.sat_cached_memory(None, None))
    assert L.sat_solutions_count(None) == 0
    # the allocation-free steps and the proposal's optimiser step
    _err(L.sat_steps_noalloc(None, 0, C.byref(opt), None, None, None, 0, None, 1, 1, 0, None))
    _err(L.sat_mlp_apply_grad(None, None, 1e-3, None))
    _err(L.sat_mlp_train_step(None, None, 1, 1, 1, 1e-3, 0, 0, None, None))


def test_bad_sizes_and_options():
    # early exit: negative step count, non-positive age
    _err(L.sat_retire(None, None, None, -1, 10, 8, None))
    _err(L.sat_retire(None, None, None, 5, 0, 8, None))
    # GEMM: leading dimensions must be >= K and multiples of 8; aligned operands; a status word
    a = (C.c_uint16 * 64)()
    st = C.c_uint32()
    _err(L.sat_gemm_bf16(8, 8, 8, a, 4, a, 8, None, 0, None, 0, 1.0, None, None, 0, None, None, 0, C.byref(st), None))
    _err(L.sat_gemm_bf16(8, 8, 8, a, 12, a, 8, None, 0, None, 0, 1.0, None, None, 0, None, None, 0, C.byref(st), None))
    _err(L.sat_gemm_bf16(8, 8, 8, a, 8, a, 8, None, 3, None, 0, 1.0, None, None, 0, None, None, 0, C.byref(st), None))
    _err(L.sat_gemm_bf16(8, 8, 8, a, 8, a, 8, None, 0, None, 0, 1.0, None, None, 0, None, None, 0, None, None))
    _err(L.sat_gemm_bf16(-1, 8, 8, a, 8, a, 8, None, 0, None, 0, 1.0, None, None, 0, None, None, 0, C.byref(st), None))
    # an empty product is a no-op
    assert L.sat_gemm_bf16(0, 8, 8, a, 8, a, 8, None, 0, None, 0, 1.0, None, None, 0, None, None, 0,
                           C.byref(st), None) == 0


def test_build_options_are_checked():
    cnf = C.c_void_p()
    text = b"p cnf 3 2\n1 -2 0\n2 3 0\n"
    assert L.sat_cnf_from_dimacs(text, len(text), C.byref(cnf)) == 0
    try:
        out = C.c_void_p()
        for bad in (N.BuildOpts(0, 16, 0, 0), N.BuildOpts(9, 16, 0, 0), N.BuildOpts(8, 0, 0, 0)):
            _err(L.sat_circuit_build(cnf, C.byref(bad), C.byref(out), None))
            assert not out.value
    finally:
        L.sat_cnf_free(cnf)
