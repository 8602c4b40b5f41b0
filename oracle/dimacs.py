"""Oracle DIMACS reader (test infrastructure).

Reads the ``p cnf V C`` format of the CNF example in Fig. 1(a) (Section III-A):
``c`` lines are comments, each clause is a list of non-zero integers ended by 0
and may span lines.  A clause count different from the header's is an error,
as is a literal outside 1..V.  A ``%`` token ends the input.
"""
from __future__ import annotations


class DimacsError(ValueError):
    pass


def parse_dimacs(text: str):
    """Return (n_vars, clauses) with clauses as lists of int literals."""
    n_vars = n_clauses = None
    clauses, cur = [], []
    for line in text.splitlines():
        s = line.strip()
        if not s or s[0] == "c":
            continue
        if s[0] == "p":
            parts = s.split()
            if len(parts) != 4 or parts[1] != "cnf" or n_vars is not None:
                raise DimacsError(f"bad header: {s!r}")
            try:
                n_vars, n_clauses = int(parts[2]), int(parts[3])
            except ValueError as e:
                raise DimacsError(f"bad header: {s!r}") from e
            if n_vars < 0 or n_clauses < 0:
                raise DimacsError("negative header field")
            continue
        if s[0] == "%":
            break
        if n_vars is None:
            raise DimacsError("clause before header")
        for tok in s.split():
            try:
                lit = int(tok)
            except ValueError as e:
                raise DimacsError(f"bad token {tok!r}") from e
            if lit == 0:
                clauses.append(cur)
                cur = []
            else:
                if abs(lit) > n_vars:
                    raise DimacsError(f"literal {lit} outside 1..{n_vars}")
                cur.append(lit)
    if n_vars is None:
        raise DimacsError("missing header")
    if cur:
        raise DimacsError("last clause not terminated by 0")
    if len(clauses) != n_clauses:
        raise DimacsError(f"header says {n_clauses} clauses, found {len(clauses)}")
    return n_vars, clauses


def cnf_satisfied(clauses, assignment) -> bool:
    """True iff every clause has a true literal; ``assignment[v]`` is var v's bit (index 0 unused)."""
    for c in clauses:
        if not any((assignment[abs(l)] == 1) == (l > 0) for l in c):
            return False
    return True
