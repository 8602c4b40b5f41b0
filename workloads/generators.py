"""Synthetic instance generators.

Two families are drawn, both with a planted satisfying assignment so that every
instance is satisfiable:

* ``planted_3sat``: random 3-SAT.  Each clause picks 3 distinct variables
  uniformly and uniform polarities and is redrawn until the hidden assignment
  satisfies it.
* ``tseitin_random_circuit``: a levelled random circuit of 2-input AND/OR/XOR
  gates (each input negated with probability 1/2), Tseitin-encoded.  A gate on
  level l takes its first input uniformly from level l-1 (so the depth is exact)
  and its second input uniformly from levels max(0, l-4) .. l-1, distinct from
  the first.  ``n_out`` distinct gates of the last level are constrained by unit
  clauses to their values under a uniform random planted input.

The CNF signatures used for the encoding are those of Section III-A, Eqs. 1-4
(output literal first in every clause, each gate's clauses contiguous, gates in
topological order, output unit clauses last).  Variable ids: primary inputs are
1..n_pi, gate outputs follow in creation order.

Random streams come from numpy's PCG64 (``numpy.random.default_rng(seed)``).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

AND, OR, XOR = 0, 1, 2
OP_NAMES = {AND: "AND", OR: "OR", XOR: "XOR"}


@dataclass
class TseitinInstance:
    n_pi: int
    depth: int
    gates_per_level: int
    in0: np.ndarray          # int64 [G], 0-based node ids (PIs are 0..n_pi-1)
    in1: np.ndarray
    op: np.ndarray           # uint8 [G] AND/OR/XOR
    neg0: np.ndarray         # uint8 [G]
    neg1: np.ndarray
    out_nodes: np.ndarray    # int64 [m] node ids of the constrained gates
    targets: np.ndarray      # uint8 [m]
    planted: np.ndarray      # uint8 [n_pi]
    clauses: list = field(default_factory=list, repr=False)

    @property
    def n_gates(self) -> int:
        return int(self.op.shape[0])

    @property
    def n_vars(self) -> int:
        return self.n_pi + self.n_gates

    def dimacs(self) -> str:
        return dimacs_text(self.n_vars, self.clauses)

    def ground_truth_values(self, pi_bits: np.ndarray) -> np.ndarray:
        """Boolean values of every node for PI rows ``pi_bits`` [S, n_pi] (0/1).

        Used to plant targets and as ground truth for tests of the circuit
        recovered from the CNF.
        """
        S = pi_bits.shape[0]
        vals = np.zeros((S, self.n_vars), dtype=np.uint8)
        vals[:, : self.n_pi] = pi_bits
        for g in range(self.n_gates):
            a = vals[:, self.in0[g]] ^ self.neg0[g]
            b = vals[:, self.in1[g]] ^ self.neg1[g]
            o = self.op[g]
            vals[:, self.n_pi + g] = (a & b) if o == AND else ((a | b) if o == OR else (a ^ b))
        return vals


def _tseitin_clauses(y: int, a: int, b: int, op: int) -> list:
    """CNF signature of y = op(a, b) for DIMACS literals a, b (Eqs. 1-4)."""
    if op == AND:
        return [[-y, a], [-y, b], [y, -a, -b]]
    if op == OR:
        return [[y, -a], [y, -b], [-y, a, b]]
    return [[-y, a, b], [-y, -a, -b], [y, -a, b], [y, a, -b]]


def tseitin_random_circuit(n_pi: int, n_gates: int, depth: int, n_out: int,
                           seed: int, fanin_window: int = 4,
                           planted_seed: int | None = None) -> TseitinInstance:
    """Random levelled circuit + Tseitin CNF with planted output targets.

    ``planted_seed`` (default: ``seed``) draws the planted input separately, so
    instances that share a topology seed can differ only in their targets.
    """
    if n_gates % depth:
        raise ValueError("n_gates must be a multiple of depth")
    gpl = n_gates // depth
    rng = np.random.default_rng(seed)
    level_start = [0, n_pi]
    in0 = np.empty(n_gates, np.int64)
    in1 = np.empty(n_gates, np.int64)
    for l in range(1, depth + 1):
        lo_prev, hi_prev = level_start[l - 1], level_start[l]
        lo_win = level_start[max(0, l - fanin_window)]
        a = rng.integers(lo_prev, hi_prev, gpl)
        b = rng.integers(lo_win, hi_prev, gpl)
        clash = a == b
        while clash.any():
            b[clash] = rng.integers(lo_win, hi_prev, int(clash.sum()))
            clash = a == b
        s = (l - 1) * gpl
        in0[s:s + gpl] = a
        in1[s:s + gpl] = b
        level_start.append(hi_prev + gpl)
    op = rng.integers(0, 3, n_gates).astype(np.uint8)
    neg0 = rng.integers(0, 2, n_gates).astype(np.uint8)
    neg1 = rng.integers(0, 2, n_gates).astype(np.uint8)
    last_lo = n_pi + (depth - 1) * gpl
    out_nodes = np.sort(rng.choice(np.arange(last_lo, n_pi + n_gates), n_out, replace=False))
    prng = np.random.default_rng(seed if planted_seed is None else planted_seed + 0x5EED)
    planted = prng.integers(0, 2, n_pi).astype(np.uint8)
    inst = TseitinInstance(n_pi, depth, gpl, in0, in1, op, neg0, neg1,
                           out_nodes, np.zeros(n_out, np.uint8), planted)
    vals = _planted_values(inst)
    inst.targets = vals[out_nodes].astype(np.uint8)
    clauses = []
    for g in range(n_gates):
        y = n_pi + g + 1
        a = int(in0[g]) + 1
        b = int(in1[g]) + 1
        la = -a if neg0[g] else a
        lb = -b if neg1[g] else b
        clauses.extend(_tseitin_clauses(y, la, lb, int(op[g])))
    for node, t in zip(out_nodes, inst.targets):
        v = int(node) + 1
        clauses.append([v if t else -v])
    inst.clauses = clauses
    return inst


def _planted_values(inst: TseitinInstance) -> np.ndarray:
    """Node values under the planted input, evaluated level by level."""
    vals = np.zeros(inst.n_vars, np.uint8)
    vals[: inst.n_pi] = inst.planted
    gpl = inst.gates_per_level
    for l in range(inst.depth):
        s, e = l * gpl, (l + 1) * gpl
        a = vals[inst.in0[s:e]] ^ inst.neg0[s:e]
        b = vals[inst.in1[s:e]] ^ inst.neg1[s:e]
        o = inst.op[s:e]
        vals[inst.n_pi + s: inst.n_pi + e] = np.where(o == AND, a & b, np.where(o == OR, a | b, a ^ b))
    return vals


@dataclass
class PlantedSATInstance:
    n_vars: int
    clauses: list
    hidden: np.ndarray  # uint8 [n_vars]

    def dimacs(self) -> str:
        return dimacs_text(self.n_vars, self.clauses)


def planted_3sat(n_vars: int, n_clauses: int, seed: int, k: int = 3) -> PlantedSATInstance:
    rng = np.random.default_rng(seed)
    hidden = rng.integers(0, 2, n_vars).astype(np.uint8)
    clauses = []
    while len(clauses) < n_clauses:
        vs = rng.choice(n_vars, k, replace=False)
        pol = rng.integers(0, 2, k)
        if any(hidden[v] == p for v, p in zip(vs, pol)):
            clauses.append([int(v) + 1 if p else -(int(v) + 1) for v, p in zip(vs, pol)])
    return PlantedSATInstance(n_vars, clauses, hidden)


def dimacs_text(n_vars: int, clauses: list, comments: list | None = None) -> str:
    parts = [f"c {c}" for c in (comments or [])]
    parts.append(f"p cnf {n_vars} {len(clauses)}")
    parts.extend(" ".join(map(str, c)) + " 0" for c in clauses)
    return "\n".join(parts) + "\n"


def fig1_example_dimacs() -> str:
    """The worked CNF of Fig. 1(a) (14 variables, 21 clauses), as text."""
    from pathlib import Path
    return (Path(__file__).resolve().parent.parent / "tests" / "golden" / "fig1_example.cnf").read_text()


def normal_logits(n_rows: int, n_cols: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded N(0, scale^2) float32 matrix, used as initial logits V0 [n_rows, n_cols]."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n_rows, n_cols)) * scale).astype(np.float32)


def mlp_params(n_in: int, n_hidden: int, n_out: int, seed: int) -> np.ndarray:
    """Seeded float32 parameter vector of the proposal network n_in -> n_hidden ->
    n_hidden -> n_out (order W1, b1, W2, b2, W3, b3), every entry of a layer uniform in
    +-1/sqrt(fan_in) (the usual dense-layer initialisation)."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((n_hidden, n_in), (n_hidden, n_hidden), (n_out, n_hidden)):
        k = 1.0 / np.sqrt(fan_in)
        parts.append(rng.uniform(-k, k, fan_out * fan_in))
        parts.append(rng.uniform(-k, k, fan_out))
    return np.concatenate(parts).astype(np.float32)


def normal_vector(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded N(0, scale^2) float32 vector (e.g. a gradient fed to an optimiser)."""
    return (np.random.default_rng(seed).standard_normal(n) * scale).astype(np.float32)
