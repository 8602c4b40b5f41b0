"""Failure detection without a GPU fault.

Each failure is made on the host or by a wait that nothing completes: an expired
bounded wait (the diagnostic kernel polls an mbarrier whose phase no copy
completes), a dedup table too small for the batch, a workspace larger than the
device, a zero step budget and a corrupt CNF.  Each call returns its error code, and
the device stays usable: a normal call right after it gives the right answer.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from workloads import planted_3sat, normal_logits

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SAT_ERR_PARSE, SAT_ERR_OOM, SAT_ERR_TABLE_FULL = -1, -3, -5
STATUS_WAIT_TIMEOUT = 4


def _device_still_works(P, gpu):
    """A Philox init after the failure equals the oracle's draw (the context is healthy)."""
    text = planted_3sat(20, 60, 3).dimacs()
    cnf = P.Cnf.from_dimacs(text)
    plan = P.Plan.create(P.Circuit.build(cnf), cnf)
    V = torch.empty(plan.n_pi, 33, device=gpu)
    P.sat_init_normal(plan, V, seed=5, round_=2, scale=1.0)
    torch.cuda.synchronize()
    np.testing.assert_allclose(V.cpu().numpy().T, oracle.init_normal(33, plan.n_pi, 5, 2, 1.0), rtol=1e-5, atol=1e-5)


def test_expired_wait_is_reported_and_context_survives(gpu):
    import paper_2502_08673_b300 as P
    from paper_2502_08673_b300 import _native as N
    st = C.c_uint32(0)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    N.check(N.lib().sat_diag_bounded_wait(20000, C.byref(st), None))
    t1.record()
    torch.cuda.synchronize()
    assert st.value == STATUS_WAIT_TIMEOUT
    ms = t0.elapsed_time(t1)
    print(f"a 20 ms bounded wait expired after {ms:.3f} ms")
    assert 19.0 <= ms < 1000.0
    _device_still_works(P, gpu)


def test_dedup_table_too_small(gpu):
    import paper_2502_08673_b300 as P
    text = planted_3sat(50, 200, 1).dimacs()
    cnf = P.Cnf.from_dimacs(text)
    circ = P.Circuit.build(cnf)
    plan = P.Plan.create(circ, cnf)
    ws = P.new_workspace(plan, 256)
    dd = P.Dedup.create(plan, max_keys=100, max_batch=256)
    P.sat_init_normal(plan, ws.V, seed=0, round_=0)
    P.sat_threshold(plan, ws.V, ws.bits, ws.keys)
    P.sat_cnf_check(plan, ws.bits, ws.valid, 256)
    with pytest.raises(P.SatError) as e:
        dd.insert(ws.keys, ws.valid, 256)
    assert e.value.status == SAT_ERR_TABLE_FULL
    assert dd.count() == 0
    # the asynchronous insert finds the overflow on the device (here every one of 256 random
    # assignments of a clause-free CNF is valid and distinct); check() reports it
    cnf0 = P.Cnf.from_dimacs("p cnf 20 0\n")
    plan0 = P.Plan.create(P.Circuit.build(cnf0), cnf0)
    ws0 = P.new_workspace(plan0, 256)
    P.sat_init_normal(plan0, ws0.V, seed=0, round_=0)
    P.sat_threshold(plan0, ws0.V, ws0.bits, ws0.keys)
    P.sat_hard_eval(plan0, ws0.bits, 256)
    P.sat_cnf_check(plan0, ws0.bits, ws0.valid, 256)
    assert P.valid_mask(ws0.valid, 256).all()
    dd2 = P.Dedup.create(plan0, max_keys=100, max_batch=256)
    dd2.insert(ws0.keys, ws0.valid, 256, sync=False)
    with pytest.raises(P.SatError) as e2:
        dd2.check()
    assert e2.value.status == SAT_ERR_TABLE_FULL
    assert dd2.count() <= 100
    # the end-to-end loop on the plan reports the same code
    from paper_2502_08673_b300 import _native as N
    o = N.SampleOpts()
    N.lib().sat_sample_opts_default(C.byref(o))
    o.batch, o.steps, o.max_rounds = 256, 50, 3
    st = N.SampleStats()
    assert N.lib().sat_sample_plan(plan.handle, dd.handle, C.byref(o), 10 ** 9, C.byref(st)) == SAT_ERR_TABLE_FULL
    assert N.lib().sat_last_error()
    _device_still_works(P, gpu)


def test_workspace_beyond_device_memory(gpu):
    import paper_2502_08673_b300 as P
    text = planted_3sat(50, 200, 1).dimacs()
    cnf = P.Cnf.from_dimacs(text)
    circ = P.Circuit.build(cnf)
    # 2^31 - 1 samples: V, m, v alone would need 3 x 50 x 8 GB
    with pytest.raises(P.SatError) as e:
        P.sample(circ, cnf, n_wanted=1, batch=(1 << 31) - 1, steps=1)
    assert e.value.status in (SAT_ERR_OOM, -2)
    _device_still_works(P, gpu)


def test_zero_step_budget_and_corrupt_cnf(gpu):
    import paper_2502_08673_b300 as P
    inst = planted_3sat(50, 200, 1)
    cnf = P.Cnf.from_dimacs(inst.dimacs())
    circ = P.Circuit.build(cnf)
    # zero descent steps: the random starts are verified as they are; every result is valid
    sols = P.sample(circ, cnf, n_wanted=10 ** 9, batch=512, steps=0, max_rounds=1, seed=3)
    A = sols.assignments()
    n, cl = oracle.parse_dimacs(inst.dimacs())
    if len(A):
        assign = np.zeros((len(A), n + 1), np.uint8)
        assign[:, 1:] = A
        assert oracle.cnf_check(n, cl, assign).all()
    for bad in ("p cnf 3 2\n1 -2 0\n", "p cnf 2 1\n1 3 0\n", "p cnf x 1\n1 0\n", "1 2 0\n"):
        with pytest.raises(P.SatError) as e:
            P.Cnf.from_dimacs(bad)
        assert e.value.status == SAT_ERR_PARSE
    _device_still_works(P, gpu)


def test_degenerate_instances_end_to_end(gpu):
    """No variables at all; and free variables without clauses, where every assignment is a
    solution and the sampler returns each of the 2^3 exactly once, in canonical order."""
    import paper_2502_08673_b300 as P
    cnf = P.Cnf.from_dimacs("p cnf 0 0\n")
    sols = P.sample(P.Circuit.build(cnf), cnf, n_wanted=5, batch=64, steps=3, max_rounds=2)
    assert len(sols) <= 1
    cnf = P.Cnf.from_dimacs("p cnf 3 0\n")
    sols = P.sample(P.Circuit.build(cnf), cnf, n_wanted=8, batch=1024, steps=3, max_rounds=3, seed=5)
    A = sols.assignments()
    assert len(A) == 8
    key = A.astype(np.int64) @ (1 << np.arange(3))
    assert key.tolist() == list(range(8))


def test_async_insert_equals_sync(gpu):
    """sat_dedup_insert_async stores the same distinct keys as sat_dedup_insert."""
    import paper_2502_08673_b300 as P
    text = planted_3sat(50, 200, 1).dimacs()
    cnf = P.Cnf.from_dimacs(text)
    plan = P.Plan.create(P.Circuit.build(cnf), cnf)
    ws = P.new_workspace(plan, 4096)
    a = P.Dedup.create(plan, max_keys=40000, max_batch=4096)
    b = P.Dedup.create(plan, max_keys=40000, max_batch=4096)
    for r in range(6):
        P.run_round(plan, ws, P.opt_params("adam", lr=0.1), steps=60, seed=1, round_=r)
        a.insert(ws.keys, ws.valid, 4096)
        b.insert(ws.keys, ws.valid, 4096, sync=False)
    b.check()
    ka, kb = a.keys(), b.keys()
    assert len(ka) > 0
    assert sorted(map(bytes, ka)) == sorted(map(bytes, kb))
