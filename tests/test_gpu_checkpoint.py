"""Checkpoint and resume of a sampling run (the state between epochs: V, m, v, the
early-exit ages and the distinct keys).  The kernels are deterministic, so a run that
is stopped, saved, restored into fresh buffers and continued ends in exactly the
state of the uninterrupted run."""
import numpy as np
import pytest

from workloads import planted_3sat

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_resume_equals_uninterrupted(gpu, tmp_path):
    import paper_2502_08673_b300 as P
    text = planted_3sat(50, 200, 2).dimacs()
    cnf = P.Cnf.from_dimacs(text)
    plan = P.Plan.create(P.Circuit.build(cnf), cnf)
    B, k, max_age = 512, 10, 30
    opt = P.opt_params("adam", lr=0.1)

    def fresh():
        return P.new_workspace(plan, B), P.Dedup.create(plan, max_keys=B * 16, max_batch=B)

    wa, da = fresh()
    P.run_epochs(plan, wa, opt, 40, k, max_age, seed=4, round_=0, dedup=da)
    P.run_epochs(plan, wa, opt, 40, k, max_age, seed=4, round_=4096, dedup=da, fresh=False)
    torch.cuda.synchronize()

    wb, db = fresh()
    P.run_epochs(plan, wb, opt, 40, k, max_age, seed=4, round_=0, dedup=db)
    path = tmp_path / "run.npz"
    P.save_checkpoint(path, wb, db, next_round=4096)
    del wb, db
    wc, dc = fresh()
    meta = P.load_checkpoint(path, wc, dc)
    assert meta == {"next_round": 4096}
    P.run_epochs(plan, wc, opt, 40, k, max_age, seed=4, round_=meta["next_round"], dedup=dc, fresh=False)
    torch.cuda.synchronize()

    assert len(da.keys()) > 0
    assert {r.tobytes() for r in da.keys()} == {r.tobytes() for r in dc.keys()}
    for name in ("V", "m", "v", "age"):
        assert torch.equal(getattr(wa, name), getattr(wc, name)), name
