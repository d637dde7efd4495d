"""Independent fixed-sequence Zuker MFE fold (dangle-0), in Python.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  A textbook O(n^3) fold
with the bulge/internal-loop cap of Sec. 3 (at most 30 unpaired nucleotides),
written independently of the lattice DP: its multiloop uses the usual
fML / fM1 decomposition rather than the right-normal D1/D2 recurrences of
Sec. 4.1, and its exterior loop is a prefix recursion rather than the
final-state suffix recursion of Sec. 5.  On a width-1 lattice (one fixed
sequence) the lattice DP must give the same minimum free energy.

Loop energies come from oracle.evaluate (the independent evaluator).
"""
from __future__ import annotations

from .evaluate import hairpin_energy, interior_energy, ptype

INF = 10 ** 12


def mfe(P: dict, seq: str) -> int:
    """Minimum free energy (dcal/mol) of seq over pseudoknot-free structures
    with canonical pairs, hairpins >= 3 and two-loops with <= 30 unpaired."""
    n = len(seq)
    if n == 0:
        return 0
    au = P["terminal_au"]
    mlc, mli, mlb = P["ml_closing"], P["ml_intern"], P["ml_base"]
    V = [[INF] * n for _ in range(n)]
    fML = [[INF] * n for _ in range(n)]
    fM1 = [[INF] * n for _ in range(n)]
    typ = [[ptype(seq[i], seq[j]) for j in range(n)] for i in range(n)]
    for span in range(4, n):
        for i in range(0, n - span):
            j = i + span
            t = typ[i][j]
            best = INF
            if t >= 0:
                best = hairpin_energy(P, seq, i, j)
                # two-loops (stack, bulge, internal), at most 30 unpaired
                for p in range(i + 1, min(i + 32, j - 4)):
                    l1 = p - i - 1
                    for q in range(j - 1, p + 3, -1):
                        l2 = j - q - 1
                        if l1 + l2 > 30:
                            break
                        if typ[p][q] < 0 or V[p][q] >= INF:
                            continue
                        e = interior_energy(P, seq, i, j, p, q) + V[p][q]
                        if e < best:
                            best = e
                # multiloop: closing pair + at least two branches inside
                for k in range(i + 2, j):
                    a = fML[i + 1][k - 1] if k - 1 >= i + 1 else INF
                    b = fM1[k][j - 1]
                    if a < INF and b < INF:
                        e = mlc + mli + int(au[t]) + a + b
                        if e < best:
                            best = e
            V[i][j] = best
            # fM1: branch starting exactly at i, followed by unpaired bases
            m1 = INF
            if V[i][j] < INF:
                m1 = V[i][j] + mli + int(au[t])
            if j - 1 > i and fM1[i][j - 1] < INF:
                m1 = min(m1, fM1[i][j - 1] + mlb)
            fM1[i][j] = m1
            # fML: at least one branch in [i, j]
            m = m1
            if fML[i + 1][j] < INF:
                m = min(m, fML[i + 1][j] + mlb)
            for k in range(i + 1, j + 1):
                if fML[i][k - 1] < INF and fM1[k][j] < INF:
                    m = min(m, fML[i][k - 1] + fM1[k][j])
            fML[i][j] = m
    # exterior loop prefix recursion
    f5 = [0] * (n + 1)            # f5[k]: best for seq[0:k]
    for k in range(1, n + 1):
        best = f5[k - 1]
        j = k - 1
        for i in range(0, j - 3):
            if V[i][j] < INF:
                best = min(best, f5[i] + V[i][j] + int(au[typ[i][j]]))
        f5[k] = best
    return f5[n]


def all_structures(n: int):
    """Every pseudoknot-free dot-bracket of length n with hairpins >= 3
    (pairing compatibility is checked by the caller). Small n only."""
    memo = {}

    def rec(i, j):
        if i > j:
            return [""]
        key = (i, j)
        if key in memo:
            return memo[key]
        out = ["." + s for s in rec(i + 1, j)]
        for k in range(i + 4, j + 1):
            for inner in rec(i + 1, k - 1):
                for rest in rec(k + 1, j):
                    out.append("(" + inner + ")" + rest)
        memo[key] = out
        return out

    return rec(0, n - 1)
