"""sat_steps_noalloc, the allocation-free variant of sat_steps, checked against it.

Some callers cannot allocate device memory at the moment they run the
optimiser: a process whose device budget has been handed to another allocator
(a framework's caching pool, a serving loop with a fixed footprint), or a
latency-critical loop that must not wait for the device synchronisation that
cudaMalloc implies.  They call sat_steps_noalloc, which takes the activation and
adjoint scratch from a fixed array inside the library instead of from buffers
the caller would have to allocate.

The same kernel on the same inputs is deterministic, so the allocation-free call
must give what sat_steps gives bit for bit.  The tiled cases force the tiled step
kernel, so the fixed array and its act/adj split are what the kernel reads and
writes; the resident case runs the shared-memory kernel, which needs no scratch.
The caller-provided scratch of the sat_steps side is filled with NaN first, so a
row read before it is written would show up as a difference.

This file is named so that pytest collects it last: a failure here leaves every
other test already run.  It calls the C ABI directly, through ctypes.
"""
import ctypes

import pytest

from workloads import planted_3sat, tseitin_random_circuit, normal_logits

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NOALLOC_BYTES = 64 << 20

CASES = {
    # name: (instance, step kernel, act dtype, optimiser, batch)
    "planted3sat_tiled_f32_adam": (lambda: planted_3sat(50, 200, 1).dimacs(), "tiled", "f32", "adam", 1000),
    "tseitin2k_tiled_f32_adam": (lambda: tseitin_random_circuit(200, 2000, 10, 8, seed=5).dimacs(),
                                 "tiled", "f32", "adam", 700),
    "tseitin2k_tiled_bf16_gd": (lambda: tseitin_random_circuit(200, 2000, 10, 8, seed=5).dimacs(),
                                "tiled", "bf16", "gd", 333),
    "planted3sat_resident_f32_adam": (lambda: planted_3sat(50, 200, 1).dimacs(), "auto", "f32", "adam", 1000),
}


def _plan(text):
    import paper_2502_08673_b300 as P
    cnf = P.Cnf.from_dimacs(text)
    circ = P.Circuit.build(cnf)
    return P, P.Plan.create(circ, cnf)


def _p(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _noalloc_bytes(plan, B, act_dtype):
    """The fixed array's share a tiled call takes: act and adj blocks, each rounded up to 256 bytes."""
    tiles = -(-B // 128)
    act_rows, adj_rows = plan.layout_rows(0)
    act = tiles * act_rows * 128 * (4 if act_dtype == "f32" else 2)
    adj = tiles * adj_rows * 128 * 4
    return -(-act // 256) * 256 + -(-adj // 256) * 256


@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_matches_sat_steps_on_two_calls(gpu, case):
    """Two consecutive calls (steps 1-10, then 11-20) give exactly what sat_steps gives."""
    make, kind, act_dtype, optname, B = CASES[case]
    P, plan = _plan(make())
    from paper_2502_08673_b300 import _native as N
    plan.set_step_kernel(kind)
    expect = "resident" if kind == "auto" else "tiled"
    assert plan.step_kernel(act_dtype) == expect
    if expect == "tiled":
        assert _noalloc_bytes(plan, B, act_dtype) <= NOALLOC_BYTES
    opt = P.opt_params(optname, lr=0.1 if optname == "adam" else 1.0)
    V0 = torch.tensor(normal_logits(plan.n_pi, B, seed=21), device=gpu)
    # existing entry point, caller-provided scratch (NaN until written)
    Va, ma, va = V0.clone(), torch.zeros_like(V0), torch.zeros_like(V0)
    act, adj = P.new_act(plan, B, act_dtype), P.new_adj(plan, B)
    act.fill_(float("nan"))
    adj.fill_(float("nan"))
    la = torch.zeros(B, device=gpu)
    # allocation-free entry point
    Vb, mb, vb = V0.clone(), torch.zeros_like(V0), torch.zeros_like(V0)
    lb = torch.zeros(B, device=gpu)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for t0 in (1, 11):
        P.sat_steps(plan, opt, Va, ma, va, act, adj, t0, 10, loss=la, act_dtype=act_dtype)
        status = N.lib().sat_steps_noalloc(plan.handle, N.ACT_DTYPES[act_dtype], ctypes.byref(opt), _p(Vb), _p(mb),
                                           _p(vb), Vb.stride(0), _p(lb), t0, 10, B, stream)
        assert status == 0, N.lib().sat_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(la).all()
        for got, want, what in ((Vb, Va, "V"), (mb, ma, "m"), (vb, va, "v"), (lb, la, "loss")):
            assert torch.equal(got, want), (case, t0, what, (got - want).abs().max().item())
    assert plan.status() == 0
    plan.set_step_kernel("auto")


def test_noalloc_rejects_scratch_beyond_its_array(gpu):
    """A tiled call whose scratch exceeds the fixed array is refused with SAT_ERR_ARG, before any launch."""
    P, plan = _plan(planted_3sat(50, 200, 1).dimacs())
    from paper_2502_08673_b300 import _native as N
    plan.set_step_kernel("tiled")
    B = 65536
    assert _noalloc_bytes(plan, B, "f32") > NOALLOC_BYTES
    V = torch.zeros(plan.n_pi, B, device=gpu)
    m, v = torch.zeros_like(V), torch.zeros_like(V)
    opt = P.opt_params("adam")
    status = N.lib().sat_steps_noalloc(plan.handle, 0, ctypes.byref(opt), _p(V), _p(m), _p(v), B, None, 1, 1, B,
                                       None)
    assert status == -2
    msg = N.lib().sat_last_error().decode()
    assert "sat_steps_noalloc needs" in msg and str(NOALLOC_BYTES) in msg
    assert torch.count_nonzero(V).item() == 0
    # the same batch on the resident kernel needs no scratch and is accepted
    plan.set_step_kernel("auto")
    assert plan.step_kernel("f32") == "resident"
    status = N.lib().sat_steps_noalloc(plan.handle, 0, ctypes.byref(opt), _p(V), _p(m), _p(v), B, None, 1, 1, B,
                                       None)
    assert status == 0, N.lib().sat_last_error()
    torch.cuda.synchronize()


def test_noalloc_rejects_bad_optimiser_parameters(gpu):
    """beta1 = 1 is refused as sat_steps refuses it (no NaN run)."""
    P, plan = _plan(planted_3sat(50, 200, 1).dimacs())
    from paper_2502_08673_b300 import _native as N
    B = 64
    V = torch.zeros(plan.n_pi, B, device=gpu)
    m, v = torch.zeros_like(V), torch.zeros_like(V)
    opt = P.opt_params("adam")
    opt.beta1 = 1.0
    status = N.lib().sat_steps_noalloc(plan.handle, 0, ctypes.byref(opt), _p(V), _p(m), _p(v), B, None, 1, 1, B,
                                       None)
    assert status == -2
    assert torch.count_nonzero(V).item() == 0
