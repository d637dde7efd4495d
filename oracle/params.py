"""Reader of the plain-text energy parameter file for the Python checkers.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The format is the one the
seeded input generator writes: ``SDENERGY 1``, then named integer tables in
row-major order, ``lxc <float>``, then the special hairpin lists
(triloops 5 nt, tetraloops 6 nt, hexaloops 8 nt, each with a total energy).
"""
from __future__ import annotations

import numpy as np

SHAPES = (
    ("stack", (6, 6)),
    ("mismatch_hairpin", (6, 4, 4)),
    ("mismatch_interior", (6, 4, 4)),
    ("mismatch_interior_1n", (6, 4, 4)),
    ("mismatch_interior_23", (6, 4, 4)),
    ("int11", (6, 6, 4, 4)),
    ("int21", (6, 6, 4, 4, 4)),
    ("int22", (6, 6, 4, 4, 4, 4)),
    ("hairpin", (31,)),
    ("bulge", (31,)),
    ("interior", (31,)),
    ("terminal_au", (6,)),
    ("ninio", (1,)),
    ("max_ninio", (1,)),
    ("ml_closing", (1,)),
    ("ml_intern", (1,)),
    ("ml_base", (1,)),
)


def read_params(path: str) -> dict:
    toks = open(path).read().split()
    pos = 0

    def take():
        nonlocal pos
        pos += 1
        return toks[pos - 1]

    assert take() == "SDENERGY" and take() == "1"
    P = {}
    for name, shape in SHAPES:
        assert take() == name, name
        cnt = int(take())
        assert cnt == int(np.prod(shape))
        P[name] = np.array([int(take()) for _ in range(cnt)], dtype=np.int64).reshape(shape)
    assert take() == "lxc"
    P["lxc"] = float(take())
    for name in ("triloop", "tetraloop", "hexaloop"):
        assert take() == name
        cnt = int(take())
        P[name] = {}
        for _ in range(cnt):
            s = take()
            P[name][s] = int(take())
    for k in ("ninio", "max_ninio", "ml_closing", "ml_intern", "ml_base"):
        P[k] = int(P[k][0])
    return P
