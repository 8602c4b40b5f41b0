"""B300-native SAT sampler (gradient descent over a relaxed multi-level circuit).

Every call goes to the CUDA library built in-tree by
``python -m paper_2502_08673_b300.build``; the library is loaded on first use
and a missing library raises ImportError.  There is no CPU fallback.
"""
from ._native import SatError, lib  # noqa: F401
from .api import (  # noqa: F401
    Cnf, Circuit, Plan, Dedup, Solutions, Workspace, Mlp, opt_params, new_workspace, new_act, new_adj, run_round,
    run_epochs, sample, valid_mask, round32, untile, sat_retire, sat_restart, save_checkpoint, load_checkpoint,
    sat_init_normal, sat_forward, sat_backward, sat_opt_update, sat_steps, sat_steps_noalloc, sat_threshold,
    sat_hard_eval, sat_gemm_bf16,
    sat_cnf_check, sat_round_gd, cached_memory, release_cached_memory,
)
