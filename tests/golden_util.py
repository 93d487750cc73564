"""Loader for the hand-derived fixtures under tests/golden (exact expressions as strings)."""
import json
import math
import os

import numpy as np

_ENV = {"__builtins__": {}, "sqrt": math.sqrt}


def _num(v):
    return float(eval(v, _ENV, {})) if isinstance(v, str) else float(v)


def load(name):
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    with open(path) as f:
        d = json.load(f)
    cols = [[_num(v) for v in col] for col in d["A_columns"]]
    d["A"] = np.array(cols, dtype=np.float64).T            # (M, N)
    d["y"] = np.array([_num(v) for v in d["y"]])
    for key in ("coef", "resid_trace", "margin"):
        if key in d:
            d[key] = np.array([_num(v) for v in d[key]])
    return d


FIXTURES = ["worked_example_3x4.json", "dependent_atom_3x3.json", "tie_duplicate_2x3.json"]


def load_candidates(name):
    """A candidate-restricted fixture: the common fields as load(), and each case's numbers."""
    d = load(name)
    d["cand"] = np.array(d["cand"], dtype=np.int64)
    for c in d["cases"]:
        c["tau"] = np.array([_num(v) for v in c["tau"]])
        for key in ("coef", "resid_trace", "margin", "drops"):
            if key in c:
                c[key] = np.array([_num(v) for v in c[key]])
    return d


CANDIDATE_FIXTURES = ["candidates_fallback_3x4.json", "candidates_unequal_norms_3x3.json"]
