"""sat_steps_noalloc, the allocation-free variant of sat_steps, checked against it.

Some callers cannot allocate device memory at the moment they run the
optimiser: a process whose device budget has been handed to another allocator
(a framework's caching pool, a serving loop with a fixed footprint), or a
latency-critical loop that must not wait for the device synchronisation that
cudaMalloc implies.  They call sat_steps_noalloc, which takes the activation and
adjoint scratch from a fixed array inside the library instead of from buffers
the caller would have to allocate.

This file is named so that pytest collects it last: a failure here leaves every
other test already run.  It calls the C ABI directly, through ctypes.
"""
import ctypes

import numpy as np
import pytest

from workloads import planted_3sat, normal_logits

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _plan():
    import paper_2502_08673_b300 as P
    cnf = P.Cnf.from_dimacs(planted_3sat(50, 200, 1).dimacs())
    circ = P.Circuit.build(cnf)
    return P, P.Plan.create(circ, cnf)


def _p(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def test_noalloc_matches_sat_steps_on_two_calls(gpu):
    """Two consecutive calls (steps 1-10, then 11-20) give what sat_steps gives."""
    P, plan = _plan()
    from paper_2502_08673_b300 import _native as N
    B = 1000  # not a multiple of the 128-sample tile: the last tile is ragged
    opt = P.opt_params("adam", lr=0.1)
    V0 = torch.tensor(normal_logits(plan.n_pi, B, seed=21), device=gpu)
    # existing entry point, caller-provided scratch
    Va, ma, va = V0.clone(), torch.zeros_like(V0), torch.zeros_like(V0)
    act, adj = P.new_act(plan, B), P.new_adj(plan, B)
    la = torch.zeros(B, device=gpu)
    # allocation-free entry point
    Vb, mb, vb = V0.clone(), torch.zeros_like(V0), torch.zeros_like(V0)
    lb = torch.zeros(B, device=gpu)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for t0 in (1, 11):
        P.sat_steps(plan, opt, Va, ma, va, act, adj, t0, 10, loss=la)
        status = N.lib().sat_steps_noalloc(plan.handle, N.ACT_DTYPES["f32"], ctypes.byref(opt), _p(Vb), _p(mb),
                                           _p(vb), Vb.stride(0), _p(lb), t0, 10, B, stream)
        assert status == 0, N.lib().sat_last_error()
        torch.cuda.synchronize()
        for got, want in ((Vb, Va), (mb, ma), (vb, va), (lb, la)):
            torch.testing.assert_close(got, want, rtol=0, atol=1e-6)
    assert plan.status() == 0


def test_noalloc_rejects_scratch_beyond_its_array(gpu):
    """A batch whose scratch exceeds the fixed array is refused with SAT_ERR_ARG, before any launch."""
    P, plan = _plan()
    from paper_2502_08673_b300 import _native as N
    B = 65536
    assert plan.scratch_elems(B) * 8 > (64 << 20)
    V = torch.zeros(plan.n_pi, B, device=gpu)
    m, v = torch.zeros_like(V), torch.zeros_like(V)
    opt = P.opt_params("adam")
    status = N.lib().sat_steps_noalloc(plan.handle, 0, ctypes.byref(opt), _p(V), _p(m), _p(v), B, None, 1, 1, B,
                                       None)
    assert status == -2
    msg = N.lib().sat_last_error().decode()
    assert "sat_steps_noalloc needs" in msg and str(64 << 20) in msg
    assert torch.count_nonzero(V).item() == 0
