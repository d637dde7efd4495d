"""Independent structure-energy evaluator (loop decomposition), in Python.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Written separately from
the C oracle so that the DP value of an emitted design can be re-evaluated
from its (mRNA, dot-bracket) pair (Sec. 5: every design is checked against a
separately recomputed structure-energy-plus-path-penalty objective).

Energy model: Turner-2004-style dangle-0 decomposition (Sec. 3), in integer
dcal/mol, read as the ViennaRNA d0 loop decomposition:
  exterior loop: terminal AU/GU penalty per exterior branch;
  hairpin: special tri/tetra/hexaloop totals, else hairpin[L] (+ terminal AU
    for L = 3, + mismatchH for L >= 4; lxc*ln(L/30) extrapolation beyond 30);
  two-loops: stack, bulge, int11/int21/int22, 1xn, 2x3, generic; loops with
    more than 30 unpaired nucleotides are scored with the lxc extrapolation
    (the 30-nt cap restricts the optimisation domain, not the evaluator);
  multiloop: ML_closing + ML_intern*(branches+1) + ML_base*unpaired + AU terms.
"""
from __future__ import annotations

import math

NUC = "ACGU"
PAIRS = ("AU", "CG", "GC", "UA", "GU", "UG")


def ptype(x: str, y: str) -> int:
    try:
        return PAIRS.index(x + y)
    except ValueError:
        return -1


def parse_structure(structure: str) -> list[int]:
    """Partner table (-1 unpaired) of a pseudoknot-free dot-bracket string."""
    stack, pt = [], [-1] * len(structure)
    for k, ch in enumerate(structure):
        if ch == "(":
            stack.append(k)
        elif ch == ")":
            if not stack:
                raise ValueError("unbalanced")
            i = stack.pop()
            pt[i], pt[k] = k, i
        elif ch != ".":
            raise ValueError("bad character")
    if stack:
        raise ValueError("unbalanced")
    return pt


def _loop_len_energy(table, lxc: float, L: int) -> int:
    if L <= 30:
        return int(table[L])
    return int(table[30]) + int(lxc * math.log(L / 30.0))


def hairpin_energy(P: dict, seq: str, i: int, j: int) -> int:
    L = j - i - 1
    if L < 3:
        raise ValueError("hairpin shorter than 3")
    t = ptype(seq[i], seq[j])
    sub = seq[i:j + 1]
    for name, size in (("triloop", 3), ("tetraloop", 4), ("hexaloop", 6)):
        if L == size and sub in P[name]:
            return P[name][sub]
    if L == 3:
        return int(P["hairpin"][3]) + int(P["terminal_au"][t])
    e = _loop_len_energy(P["hairpin"], P["lxc"], L)
    return e + int(P["mismatch_hairpin"][t][NUC.index(seq[i + 1])][NUC.index(seq[j - 1])])


def interior_energy(P: dict, seq: str, i: int, j: int, p: int, q: int) -> int:
    """Two-loop closed by (i,j) with inner pair (p,q), i < p < q < j."""
    t = ptype(seq[i], seq[j])
    s = ptype(seq[q], seq[p])          # inner pair as seen from inside the loop
    l1, l2 = p - i - 1, j - q - 1
    nt = lambda k: NUC.index(seq[k])
    au = P["terminal_au"]
    if l1 == 0 and l2 == 0:
        return int(P["stack"][t][s])
    if l1 == 0 or l2 == 0:
        L = l1 + l2
        if L == 1:
            return int(P["bulge"][1]) + int(P["stack"][t][s])
        return _loop_len_energy(P["bulge"], P["lxc"], L) + int(au[t]) + int(au[s])
    if l1 == 1 and l2 == 1:
        return int(P["int11"][t][s][nt(i + 1)][nt(j - 1)])
    if l1 == 1 and l2 == 2:
        return int(P["int21"][t][s][nt(i + 1)][nt(q + 1)][nt(j - 1)])
    if l1 == 2 and l2 == 1:
        # the same loop read from the inner pair's side
        return int(P["int21"][s][t][nt(q + 1)][nt(i + 1)][nt(p - 1)])
    if l1 == 2 and l2 == 2:
        return int(P["int22"][t][s][nt(i + 1)][nt(p - 1)][nt(q + 1)][nt(j - 1)])
    L = l1 + l2
    asym = min(P["max_ninio"], P["ninio"] * abs(l1 - l2))
    if l1 == 1 or l2 == 1:
        mm = P["mismatch_interior_1n"]
        return (_loop_len_energy(P["interior"], P["lxc"], L) + asym
                + int(mm[t][nt(i + 1)][nt(j - 1)]) + int(mm[s][nt(q + 1)][nt(p - 1)]))
    if (l1, l2) in ((2, 3), (3, 2)):
        mm = P["mismatch_interior_23"]
        return (int(P["interior"][5]) + P["ninio"]
                + int(mm[t][nt(i + 1)][nt(j - 1)]) + int(mm[s][nt(q + 1)][nt(p - 1)]))
    mm = P["mismatch_interior"]
    return (_loop_len_energy(P["interior"], P["lxc"], L) + asym
            + int(mm[t][nt(i + 1)][nt(j - 1)]) + int(mm[s][nt(q + 1)][nt(p - 1)]))


def energy(P: dict, seq: str, structure: str) -> int:
    """Dangle-0 free energy (dcal/mol) of a structure on a sequence."""
    if len(seq) != len(structure):
        raise ValueError("length mismatch")
    pt = parse_structure(structure)
    n = len(seq)
    for i in range(n):
        j = pt[i]
        if j > i and ptype(seq[i], seq[j]) < 0:
            raise ValueError(f"non-canonical pair {i},{j}")
    au = P["terminal_au"]
    E = 0
    # exterior loop
    k = 0
    while k < n:
        if pt[k] > k:
            E += int(au[ptype(seq[k], seq[pt[k]])])
            k = pt[k] + 1
        else:
            k += 1
    # loops closed by each pair
    for i in range(n):
        j = pt[i]
        if j <= i:
            continue
        inner = []
        k = i + 1
        unpaired = 0
        while k < j:
            if pt[k] > k:
                inner.append((k, pt[k]))
                k = pt[k] + 1
            else:
                unpaired += 1
                k += 1
        t = ptype(seq[i], seq[j])
        if not inner:
            E += hairpin_energy(P, seq, i, j)
        elif len(inner) == 1:
            p, q = inner[0]
            E += interior_energy(P, seq, i, j, p, q)
        else:
            E += P["ml_closing"] + P["ml_intern"] + int(au[t])
            for p, q in inner:
                E += P["ml_intern"] + int(au[ptype(seq[p], seq[q])])
            E += P["ml_base"] * unpaired
    return E


def max_two_loop_unpaired(structure: str) -> int:
    """Largest l1 + l2 over the two-loops of a structure (0 if none)."""
    pt = parse_structure(structure)
    best = 0
    for i, j in enumerate(pt):
        if j <= i:
            continue
        inner, k = [], i + 1
        while k < j:
            if pt[k] > k:
                inner.append((k, pt[k]))
                k = pt[k] + 1
            else:
                k += 1
        if len(inner) == 1:
            p, q = inner[0]
            best = max(best, (p - i - 1) + (j - q - 1))
    return best
