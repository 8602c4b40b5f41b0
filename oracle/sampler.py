"""Oracle orchestration (test infrastructure): one sampling round as the paper states it.

Section III-A: the primary inputs V (b x n) are embedded as P = sigmoid(V)
(Eq. 5), the relaxed circuit gives Y = F(P) (Eq. 6), the l2 loss of Eq. 7 is
minimised by gradient steps (Eqs. 8-9; Adam is the optional optimiser), then V
is thresholded, and only satisfiable, non-redundant rows are kept.

Readings: threshold bit = [V > 0] (sigmoid(V) > 1/2, ties to 0); a row is kept
when the full assignment it induces satisfies every ORIGINAL clause; rows are
redundant when their full assignments are equal.  Solution hashes fold the
packed primary-input bits with the SplitMix64 finaliser (Steele, Lea, Flood,
OOPSLA 2014).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import lib, ptr, OrcCircuit
from .transform import Circuit, LIT, AND, OR, XOR, SOP

OPC = {LIT: 0, AND: 1, OR: 2, XOR: 3}
MASK64 = (1 << 64) - 1


@dataclass
class FlatCircuit:
    """Instruction form of a Circuit: var v is node v-1; SOP terms and outputs get extra nodes."""
    n_vars: int
    n_nodes: int
    ins_out: np.ndarray
    ins_op: np.ndarray
    ins_neg: np.ndarray
    ins_off: np.ndarray
    ins_cnt: np.ndarray
    lit_node: np.ndarray
    lit_neg: np.ndarray
    pi_node: np.ndarray      # V column j -> node (ascending var id)
    out_node: np.ndarray
    target: np.ndarray
    circuit: Circuit

    def cstruct(self):
        s = OrcCircuit()
        s.n_nodes, s.n_instr = self.n_nodes, len(self.ins_out)
        s.ins_out, s.ins_op, s.ins_neg = self.ins_out.ctypes.data, self.ins_op.ctypes.data, self.ins_neg.ctypes.data
        s.ins_off, s.ins_cnt = self.ins_off.ctypes.data, self.ins_cnt.ctypes.data
        s.lit_node, s.lit_neg = self.lit_node.ctypes.data, self.lit_neg.ctypes.data
        s.n_pi, s.pi_node = len(self.pi_node), self.pi_node.ctypes.data
        s.n_out, s.out_node, s.target = len(self.out_node), self.out_node.ctypes.data, self.target.ctypes.data
        return s


def flatten(circ: Circuit) -> FlatCircuit:
    ins = []   # (out_node, op, neg, [(node, neg)])
    nxt = circ.n_vars

    def L(l):
        return (abs(l) - 1, 1 if l < 0 else 0)

    for d in circ.defs:
        if d.kind == SOP:
            term_nodes = []
            for t in d.lits:
                ins.append((nxt, OPC[AND], 0, [L(l) for l in t]))
                term_nodes.append((nxt, 0))
                nxt += 1
            ins.append((d.var - 1, OPC[OR], int(d.out_neg), term_nodes))
        else:
            ins.append((d.var - 1, OPC[d.kind], int(d.out_neg), [L(l) for l in d.lits]))
    out_node = []
    for c in circ.outputs:
        ins.append((nxt, OPC[OR], 0, [L(l) for l in c]))
        out_node.append(nxt)
        nxt += 1
    lit_node, lit_neg, off, cnt = [], [], [], []
    for _, _, _, lits in ins:
        off.append(len(lit_node))
        cnt.append(len(lits))
        for n, g in lits:
            lit_node.append(n)
            lit_neg.append(g)
    i32 = lambda x: np.ascontiguousarray(np.array(x, dtype=np.int32))
    return FlatCircuit(
        circ.n_vars, nxt,
        i32([x[0] for x in ins]), i32([x[1] for x in ins]), i32([x[2] for x in ins]),
        i32(off), i32(cnt), i32(lit_node), i32(lit_neg),
        i32([v - 1 for v in circ.pis]), i32(out_node),
        np.ones(len(out_node), dtype=np.float64), circ)


def forward(fc: FlatCircuit, V: np.ndarray):
    """P = sigmoid(V) (Eq. 5), Y = F(P) (Eq. 6), per-sample loss (Eq. 7).  V: [S, n_pi]."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    S = V.shape[0]
    vals = np.empty((S, fc.n_nodes), np.float64)
    loss = np.empty(S, np.float64)
    cs = fc.cstruct()
    lib().orc_forward(ctypes_ref(cs), S, ptr(V), ptr(vals), ptr(loss))
    return vals, loss


def backward(fc: FlatCircuit, vals: np.ndarray):
    """dL/dV by the chain rule (Eq. 8) with Table 1 derivatives; also node adjoints."""
    S = vals.shape[0]
    adj = np.empty_like(vals)
    gV = np.empty((S, len(fc.pi_node)), np.float64)
    cs = fc.cstruct()
    lib().orc_backward(ctypes_ref(cs), S, ptr(vals), ptr(adj), ptr(gV))
    return gV, adj


def backward_magnitude(fc: FlatCircuit, vals: np.ndarray):
    """Sum of the absolute chain-rule terms behind each dL/dV (Eq. 8 with every fan-out
    term taken in absolute value, seeded with |2(Y - T)|): an upper bound of |dL/dV| and
    the scale of the rounding error of any floating-point evaluation of it."""
    S = vals.shape[0]
    amag = np.empty_like(vals)
    gmag = np.empty((S, len(fc.pi_node)), np.float64)
    cs = fc.cstruct()
    lib().orc_backward_mag(ctypes_ref(cs), S, ptr(vals), ptr(amag), ptr(gmag))
    return gmag


def ctypes_ref(s):
    import ctypes
    return ctypes.byref(s)


def gd_step(V, g, lr):
    """Eq. 9: V <- V - lr * dL/dV (in place on float64 arrays)."""
    lib().orc_gd(V.size, ptr(V), ptr(g), lr)


def adam_step(V, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    lib().orc_adam(V.size, ptr(V), ptr(m), ptr(v), ptr(g), t, lr, b1, b2, eps)


def hard_eval(fc: FlatCircuit, pi_bits: np.ndarray) -> np.ndarray:
    """Boolean value of every node; pi_bits [S, n_pi] of 0/1."""
    pi_bits = np.ascontiguousarray(pi_bits, dtype=np.uint8)
    S = pi_bits.shape[0]
    bits = np.zeros((S, fc.n_nodes), np.uint8)
    cs = fc.cstruct()
    lib().orc_hard(ctypes_ref(cs), S, ptr(pi_bits), ptr(bits))
    return bits


def full_assignment(fc: FlatCircuit, bits: np.ndarray) -> np.ndarray:
    """[S, n_vars+1] assignment (column 0 unused) from node bits."""
    S = bits.shape[0]
    out = np.zeros((S, fc.n_vars + 1), np.uint8)
    out[:, 1:] = bits[:, : fc.n_vars]
    return out


def cnf_check(n_vars: int, clauses, assign: np.ndarray) -> np.ndarray:
    """1 where every original clause has a true literal (Section II-A)."""
    off = np.zeros(len(clauses) + 1, np.int64)
    off[1:] = np.cumsum([len(c) for c in clauses])
    lits = np.ascontiguousarray(np.array([l for c in clauses for l in c], dtype=np.int32))
    assign = np.ascontiguousarray(assign, dtype=np.uint8)
    ok = np.zeros(assign.shape[0], np.uint8)
    lib().orc_cnf_check(len(clauses), ptr(off), ptr(lits), n_vars, assign.shape[0], ptr(assign), ptr(ok))
    return ok


def _mix64(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def pack_pi_words(pi_bits_row) -> list:
    """64-bit words: bit j of word w = primary input 64w+j (ascending var id)."""
    n = len(pi_bits_row)
    words = []
    for w in range((n + 63) // 64):
        x = 0
        for j in range(64):
            i = 64 * w + j
            if i < n and pi_bits_row[i]:
                x |= 1 << j
        words.append(x)
    return words


def solution_hash(pi_bits_row) -> int:
    """h = golden gamma; h = mix64(h + word) per word; h = mix64(h ^ n_words)."""
    words = pack_pi_words(pi_bits_row)
    h = 0x9E3779B97F4A7C15
    for x in words:
        h = _mix64((h + x) & MASK64)
    return _mix64(h ^ len(words))


def philox4x32_10(ctr, key):
    c = np.array(ctr, dtype=np.uint32)
    k = np.array(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(ptr(c), ptr(k), ptr(o))
    return [int(x) for x in o]


def init_normal(S, n_pi, seed, rnd, scale=1.0):
    V = np.empty((S, n_pi), np.float64)
    lib().orc_init_normal(S, n_pi, seed, rnd, scale, ptr(V))
    return V


def sample_round(fc: FlatCircuit, n_vars, clauses, V0, steps, lr, opt="adam",
                 betas=(0.9, 0.999), eps=1e-8, trace=None):
    """One round from logits V0 [S, n_pi]; returns dict with final V, bits, validity, keys."""
    V = np.array(V0, dtype=np.float64, copy=True)
    m = np.zeros_like(V)
    v = np.zeros_like(V)
    for t in range(1, steps + 1):
        vals, loss = forward(fc, V)
        gV, _ = backward(fc, vals)
        if trace is not None:
            trace.append((V.copy(), loss, gV))
        if opt == "adam":
            adam_step(V, m, v, gV, t, lr, betas[0], betas[1], eps)
        else:
            gd_step(V, gV, lr)
    return verify(fc, n_vars, clauses, V) | {"V": V, "m": m, "v": v}


def verify(fc: FlatCircuit, n_vars, clauses, V):
    """Threshold, Boolean evaluation, CNF check and deduplication of rows of V."""
    pi_bits = (np.asarray(V) > 0).astype(np.uint8)
    bits = hard_eval(fc, pi_bits)
    assign = full_assignment(fc, bits)
    ok = cnf_check(n_vars, clauses, assign)
    uniq = {}
    for s in np.nonzero(ok)[0]:
        key = assign[s, 1:].tobytes()
        uniq.setdefault(key, int(s))
    return {"pi_bits": pi_bits, "assign": assign, "valid": ok, "unique": uniq}


class Oracle:
    """Convenience bundle: DIMACS text -> oracle circuit -> rounds."""

    def __init__(self, dimacs_text: str, direct: bool = False, reorder: bool = False):
        from .dimacs import parse_dimacs
        from .transform import factorize, direct_circuit
        self.n_vars, self.clauses = parse_dimacs(dimacs_text)
        self.circuit = (direct_circuit(self.n_vars, self.clauses) if direct
                        else factorize(self.n_vars, self.clauses, reorder=reorder))
        self.flat = flatten(self.circuit)

    @property
    def n_pi(self):
        return len(self.flat.pi_node)
