"""Loader for tests/golden/hand_cases.ini (hand-derived scores)."""
import configparser
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
PATH = os.path.join(HERE, "golden", "hand_cases.ini")


def _expand(text, alphabet):
    out = []
    for tok in text.split():
        if "*" in tok:
            ch, k = tok.split("*")
            out.extend([alphabet.index(ch)] * int(k))
        else:
            out.extend(alphabet.index(ch) for ch in tok)
    return np.array(out, dtype=np.uint8)


def _matrix(spec, A):
    parts = spec.split()
    if parts[0] == "diag":
        d, x = int(parts[1]), int(parts[3])
        M = np.full((A, A), x, dtype=np.int8)
        M[np.arange(A), np.arange(A)] = d
        return M
    if parts[0] == "rows":
        rows = " ".join(parts[1:]).split(";")
        M = np.array([[int(v) for v in r.split(",")] for r in rows], dtype=np.int8)
        assert M.shape == (A, A)
        return M
    raise ValueError(spec)


def load():
    cp = configparser.ConfigParser(interpolation=None)
    cp.read(PATH)
    cases = []
    for name in cp.sections():
        s = cp[name]
        alpha = s["alphabet"]
        cases.append(dict(
            name=name,
            cite=s["cite"],
            M=_matrix(s["matrix"], len(alpha)),
            o=int(s["gap_open"]),
            e=int(s["gap_extend"]),
            q=_expand(s["query"], alpha),
            r=_expand(s["ref"], alpha),
            score=int(s["score"]),
            end=tuple(int(x) for x in s["end"].split()) if "end" in s else None,
        ))
    return cases
