"""Readers for the text fixtures under tests/golden/ (tables typed in from the paper)."""
import os

import numpy as np
import sympy as sp

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def sections(name):
    """Parse ``[section]`` blocks of a fixture into {section: [lines]} (comments dropped)."""
    out, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as fh:
        for raw in fh:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("[") and line.endswith("]"):
                cur = line[1:-1]
                out[cur] = []
            else:
                out[cur].append(line)
    return out


def matrix(sec):
    return np.array([[float(v) for v in ln.split()] for ln in sec])


def paper_tables():
    s = sections("paper_tables.txt")
    return {
        "cx": matrix(s["c_x"])[0].astype(int),
        "cy": matrix(s["c_y"])[0].astype(int),
        "T": matrix(s["T"]),
        "Tm": matrix(s["T_m"]),
        "T_rows": [sp.sympify(e) for e in s["T_rows"]],
        "Tm_rows": [sp.sympify(e) for e in s["T_m_rows"]],
    }


def equilibrium_exprs():
    s = sections("equilibrium_moments.txt")
    return [sp.sympify(e) for e in s["M_eq"]], [sp.sympify(e) for e in s["N_eq"]]
