"""Brute-force exact design by enumeration of synonymous mRNAs.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Follows Eq. (1) of
Sec. 3 literally: for every synonymous mRNA r of the protein, fold r with the
independent Zuker MFE (oracle.zuker), add lambda' C(r) and take the minimum.
The codon penalty is the fixed-point quantity the DP uses,
round_half_even(100*lambda * (-ln w) * 2^32) per codon, so the brute-force
minimum must equal the DP value exactly.  Small synonymous spaces only.
"""
from __future__ import annotations

import itertools
import math

from .zuker import mfe

NUC = "ACGU"
_CODE = ("KNKNTTTTRSRSIIMIQHQHPPPPRRRRLLLLEDEDAAAAGGGGVVVV*Y*YSSSS*CWCLFLF")


def codons_of(aa: str) -> list[str]:
    out = []
    for x in range(4):
        for y in range(4):
            for z in range(4):
                if _CODE[16 * x + 4 * y + z] == aa:
                    out.append(NUC[x] + NUC[y] + NUC[z])
    return out


def qfx(lam: float, w: float) -> int:
    x = (100.0 * lam) * (-math.log(w))
    return round(math.ldexp(x, 32))


def synonymous_space(protein: str) -> int:
    k = 1
    for aa in protein:
        k *= len(codons_of(aa))
    return k


def brute_force(P: dict, protein: str, weights, lam: float, motifs=()):
    """Returns (best objective in fixed point, list of optimal mRNAs); with
    motifs, only the mRNAs containing none of them (None, [] if none is
    left)."""
    choices = [codons_of(aa) for aa in protein]
    best, arg = None, []
    cache = {}
    for combo in itertools.product(*choices):
        r = "".join(combo)
        if any(m in r for m in motifs):
            continue
        if r not in cache:
            cache[r] = mfe(P, r)
        cost = sum(qfx(lam, weights[16 * NUC.index(c[0]) + 4 * NUC.index(c[1]) + NUC.index(c[2])])
                   for c in combo)
        v = cache[r] * (1 << 32) + cost
        if best is None or v < best:
            best, arg = v, [r]
        elif v == best:
            arg.append(r)
    return best, arg
