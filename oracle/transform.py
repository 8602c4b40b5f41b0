"""Oracle transformation of a CNF into a multi-level, multi-output circuit.

Test infrastructure: a plain restatement of Algorithm 1 (Section III-A) plus the
under-specified-clause fallback described after it.  Boolean functions are truth
tables held in Python ints over a sorted list of support variables (bit i of a
minterm index = value of support[i]).

Readings of the paper taken here (each is listed with its reason in the design
notes):

* Candidates v of the sub-clause window SC are tried in descending variable id.
  Fig. 1 defines, in every gate group, the variable with the largest id.
* FindBooleanExpression(v, SC) conjoins, over the clauses of SC that hold the
  literal -v (resp. v), the clause with that literal removed; the definition
  v = f is accepted when f is the complement of the expression found for -v.
  Clauses of SC that do not mention v are not part of the definition; on
  acceptance they become constraint outputs instead of being dropped.
* An accepted constant function makes v a primary output: the unit constraint
  (v) or (-v).  v stays definable by later clauses.
* Every other variable of the defining clauses that is not yet an intermediate
  variable becomes a primary input (as in Algorithm 1).
* Fallback: when no definition is found and no variable of SC occurs in a later
  clause, every clause of SC becomes its own OR output constrained to 1.  SC is
  also kept within ``max_window`` clauses and ``max_support`` variables by
  emitting its oldest clause the same way.  Clauses left at the end are emitted
  likewise.
* Simplification of an accepted f: constants and single literals are aliases;
  AND, OR and XOR/XNOR of literals (any arity) are recognised; any other f is
  written as a sum of products over a minimum cover of its prime implicants
  (fewest terms, then fewest literals, then first in the sorted prime order;
  with more than 20 primes all primes are used).
* Variables that are never defined are primary inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from itertools import combinations

LIT, AND, OR, XOR, SOP = "LIT", "AND", "OR", "XOR", "SOP"


@dataclass
class Definition:
    var: int
    kind: str               # LIT / AND / OR / XOR / SOP
    lits: list              # LIT/AND/OR/XOR: signed var ids; SOP: list of terms (lists of signed ids)
    out_neg: bool = False   # XNOR = XOR with out_neg; NAND/NOR are AND/OR with out_neg
    support: list = field(default_factory=list)
    table: int = 0          # truth table of v over ``support`` (for structural comparisons)


@dataclass
class Circuit:
    n_vars: int
    pis: list               # ascending var ids
    defs: list              # Definitions, in acceptance (= topological) order
    outputs: list           # list of clauses (signed ids): each OR output is constrained to 1
    n_accept_const: int = 0

    def iv_vars(self):
        return [d.var for d in self.defs]


def _var_mask(i: int, k: int) -> int:
    """Truth table of support variable i over k variables."""
    m = 0
    for x in range(1 << k):
        if (x >> i) & 1:
            m |= 1 << x
    return m


def _clause_table(lits, pos, k):
    full = (1 << (1 << k)) - 1
    t = 0
    for l in lits:
        m = _var_mask(pos[abs(l)], k)
        t |= m if l > 0 else (full & ~m)
    return t


def find_boolean_expression(lit: int, clauses, support):
    """Conjunction over clauses holding ``-lit`` of the rest of the clause.

    With lit = v this is the expression of v (the clauses with -v must hold when
    v = 1); with lit = -v it is the expression of -v.
    """
    k = len(support)
    pos = {v: i for i, v in enumerate(support)}
    full = (1 << (1 << k)) - 1
    f = full
    for c in clauses:
        if -lit in c:
            f &= _clause_table([l for l in c if l != -lit], pos, k)
    return f


def _depends(table: int, i: int, k: int) -> bool:
    for x in range(1 << k):
        if not (x >> i) & 1:
            if ((table >> x) & 1) != ((table >> (x | (1 << i))) & 1):
                return True
    return False


def _restrict_support(table, support):
    """Drop support variables that the function does not depend on."""
    k = len(support)
    keep = [i for i in range(k) if _depends(table, i, k)]
    if len(keep) == k:
        return table, list(support)
    nk = len(keep)
    nt = 0
    for y in range(1 << nk):
        x = 0
        for j, i in enumerate(keep):
            if (y >> j) & 1:
                x |= 1 << i
        if (table >> x) & 1:
            nt |= 1 << y
    return nt, [support[i] for i in keep]


def _prime_implicants(table, k):
    """Prime implicants as (care_mask, value) cubes, by Quine-McCluskey merging."""
    cur = {((1 << k) - 1, x) for x in range(1 << k) if (table >> x) & 1}
    primes = set()
    while cur:
        nxt = set()
        merged = set()
        cl = sorted(cur)
        for a in cl:
            for b in cl:
                if a[0] == b[0] and a < b:
                    d = a[1] ^ b[1]
                    if d and not (d & (d - 1)):
                        nxt.add((a[0] & ~d, a[1] & ~d))
                        merged.add(a)
                        merged.add(b)
        primes |= cur - merged
        cur = nxt
    return primes


def _cube_minterms(cube, k):
    care, val = cube
    return {x for x in range(1 << k) if (x & care) == val}


def minimum_sop(table, k):
    """Cover of the true minterms by prime implicants (reading of Simplify)."""
    primes = sorted(_prime_implicants(table, k), key=lambda c: (bin(c[0]).count("1"), c[0], c[1]))
    ones = {x for x in range(1 << k) if (table >> x) & 1}
    if len(primes) > 20:
        return primes
    cov = [_cube_minterms(p, k) for p in primes]
    for size in range(1, len(primes) + 1):
        best = None
        for comb in combinations(range(len(primes)), size):
            s = set()
            for i in comb:
                s |= cov[i]
            if s >= ones:
                nlit = sum(bin(primes[i][0]).count("1") for i in comb)
                if best is None or nlit < best[0]:
                    best = (nlit, comb)
        if best is not None:
            return [primes[i] for i in best[1]]
    return primes


def classify(var, table, support):
    """Simplified Definition (or None for a constant) of var = table over support."""
    table, support = _restrict_support(table, support)
    k = len(support)
    full = (1 << (1 << k)) - 1
    if k == 0:
        return None
    if k == 1:
        lit = support[0] if table == 0b10 else -support[0]
        return Definition(var, LIT, [lit], False, support, table)
    ones = [x for x in range(1 << k) if (table >> x) & 1]
    zeros = [x for x in range(1 << k) if not (table >> x) & 1]
    if len(ones) == 1:
        x = ones[0]
        lits = [support[i] if (x >> i) & 1 else -support[i] for i in range(k)]
        return Definition(var, AND, lits, False, support, table)
    if len(zeros) == 1:
        x = zeros[0]
        lits = [-support[i] if (x >> i) & 1 else support[i] for i in range(k)]
        return Definition(var, OR, lits, False, support, table)
    parity = 0
    for x in range(1 << k):
        if bin(x).count("1") & 1:
            parity |= 1 << x
    if table == parity or table == (full & ~parity):
        return Definition(var, XOR, list(support), table != parity, support, table)
    terms = []
    for care, val in minimum_sop(table, k):
        terms.append([support[i] if (val >> i) & 1 else -support[i] for i in range(k) if (care >> i) & 1])
    return Definition(var, SOP, terms, False, support, table)


def _clean(clauses):
    out = []
    for c in clauses:
        seen = []
        for l in c:
            if l not in seen:
                seen.append(l)
        if any(-l in seen for l in seen):
            continue  # tautology: always satisfied, carries no constraint
        if not seen:
            raise ValueError("empty clause: the CNF is unsatisfiable")
        out.append(seen)
    return out


def direct_circuit(n_vars: int, clauses) -> Circuit:
    """No factorization: every clause is an OR output constrained to 1 and every
    variable a primary input -- the CNF itself relaxed clause by clause (the
    'CNF' side of the operation counts of Fig. 5), used for the ablation against
    Algorithm 1."""
    return Circuit(n_vars, list(range(1, n_vars + 1)), [], _clean(clauses), 0)


def factorize(n_vars: int, clauses, max_support: int = 8, max_window: int = 16, reorder: bool = False) -> Circuit:
    """Algorithm 1 with the readings listed in the module docstring.  reorder: first
    sort the (cleaned) clauses by their largest variable, then longer clauses first,
    then position, so that a variable's defining clauses are adjacent (and ahead of
    unit clauses on it) in files that interleave them."""
    clauses = _clean(clauses)
    if reorder:
        keyed = sorted((max(abs(l) for l in c), -len(c), i) for i, c in enumerate(clauses))
        clauses = [clauses[i] for _, _, i in keyed]
    last = {}
    for i, c in enumerate(clauses):
        for l in c:
            last[abs(l)] = i
    PI, IV = set(), set()
    defs, outputs = [], []
    n_const = 0
    SC = []

    def sc_vars(sc):
        return {abs(l) for c in sc for l in c}

    for i, c in enumerate(clauses):
        SC.append(c)
        accepted = False
        for v in sorted(sc_vars(SC), reverse=True):
            if v in PI or v in IV:
                continue
            with_v = [cl for cl in SC if v in cl or -v in cl]
            support = sorted(sc_vars(with_v) - {v})
            if len(support) > max_support:
                continue
            f = find_boolean_expression(v, with_v, support)
            g = find_boolean_expression(-v, with_v, support)
            full = (1 << (1 << len(support))) - 1
            if f != (full & ~g):
                continue
            outputs.extend(cl for cl in SC if not (v in cl or -v in cl))
            d = classify(v, f, support)
            if d is None:
                outputs.append([v] if f == full else [-v])
                n_const += 1
            else:
                defs.append(d)
                IV.add(v)
            for w in support:
                if w not in IV:
                    PI.add(w)
            SC = []
            accepted = True
            break
        if accepted:
            continue
        if all(last[w] <= i for w in sc_vars(SC)):
            outputs.extend(SC)
            SC = []
            continue
        while SC and (len(SC) > max_window or len(sc_vars(SC)) > max_support):
            outputs.append(SC.pop(0))
    outputs.extend(SC)
    pis = [v for v in range(1, n_vars + 1) if v not in IV]
    return Circuit(n_vars, pis, defs, outputs, n_const)


def circuit_assignment(circ: Circuit, pi_bits: dict) -> dict:
    """Boolean value of every variable given PI values (dict var -> 0/1)."""
    val = dict(pi_bits)

    def lit(l):
        return val[abs(l)] if l > 0 else 1 - val[abs(l)]

    for d in circ.defs:
        if d.kind == LIT:
            y = lit(d.lits[0])
        elif d.kind == AND:
            y = int(all(lit(l) for l in d.lits))
        elif d.kind == OR:
            y = int(any(lit(l) for l in d.lits))
        elif d.kind == XOR:
            y = sum(lit(l) for l in d.lits) & 1
        else:
            y = int(any(all(lit(l) for l in t) for t in d.lits))
        val[d.var] = y ^ int(d.out_neg)
    return val


def outputs_satisfied(circ: Circuit, val: dict) -> bool:
    return all(any((val[abs(l)] == 1) == (l > 0) for l in c) for c in circ.outputs)
