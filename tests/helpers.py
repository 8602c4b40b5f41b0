"""Shared test helpers (no sampler arithmetic here)."""
from __future__ import annotations

import re
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent


def oracle_dump(circ) -> str:
    """The oracle circuit in the library's canonical dump format."""
    lines = [f"vars {circ.n_vars}", "pi" + "".join(f" {v}" for v in circ.pis)]
    for d in circ.defs:
        if d.kind == "SOP":
            body = " |".join("".join(f" {l}" for l in t) for t in d.lits)
        else:
            body = "".join(f" {l}" for l in d.lits)
        lines.append(f"def {d.var} {d.kind} {int(d.out_neg)} :{body}")
    for o in circ.outputs:
        lines.append("out" + "".join(f" {l}" for l in o))
    return "\n".join(lines) + "\n"


def header_functions() -> list:
    """Names of the functions declared in include/satsampler.h."""
    text = (ROOT / "include" / "satsampler.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(sat_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))
