"""Many values of lambda for one protein (Sec. 10 supported-envelope and
inverse-lambda tools), marked gpu.

The envelope is pinned by brute force: for tiny proteins every synonymous
mRNA is folded by the independent Zuker code (its line is E(r) + 100 lambda
C(r)), and the lower envelope of those lines on [lo, hi] is computed exactly
here; the library's supported lines and breakpoints must be the same.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import zuker
from oracle.brute import codons_of
from oracle.params import read_params
from paper_2609_32308_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2609_32308_b300 as sd
    sd.lib()
    return sd


@pytest.fixture(scope="module")
def E1(sd, par1):
    return sd.sd_load_energy(par1)


def test_sweep_equals_separate_designs(sd, E1):
    prot = inputs.random_protein(60, 41)
    w = inputs.random_codon_weights(41)
    lams = [0.0, 0.5, 1.0, 2.0, 4.0, 8.0]
    sweep = sd.sd_design_sweep(E1, prot, w, lams)
    for lam, r in zip(lams, sweep):
        one = sd.sd_design(E1, prot, w, lam)
        for key in ("mrna", "structure", "energy", "objective_fx", "codon_cost", "objective", "Z"):
            assert r[key] == one[key], (lam, key)


def brute_envelope(P, prot, w, lo, hi):
    """Exact lower envelope of the lines (E(r), C(r)) of every synonymous r."""
    nt = "ACGU"
    lines = set()
    for combo in itertools.product(*[codons_of(a) for a in prot]):
        r = "".join(combo)
        C = 0.0
        for c in combo:
            C += -math.log(w[16 * nt.index(c[0]) + 4 * nt.index(c[1]) + nt.index(c[2])])
        lines.add((zuker.mfe(P, r), C))
    lines = sorted(lines)
    val = lambda l, x: l[0] + 100.0 * x * l[1]
    # the line minimal just right of lo (ties: smallest C stays minimal longest)
    cur = min(lines, key=lambda l: (val(l, lo), l[1]))
    out, breaks, x = [cur], [], lo
    while True:
        nxt, xb = None, None
        for l in lines:
            if l[1] >= cur[1]:
                continue
            xi = (l[0] - cur[0]) / (100.0 * (cur[1] - l[1]))
            if xi <= x + 1e-12:
                continue
            if xb is None or xi < xb - 1e-12 or (abs(xi - xb) <= 1e-12 and l[1] < nxt[1]):
                nxt, xb = l, xi
        if nxt is None or xb >= hi:
            return out, breaks
        out.append(nxt)
        breaks.append(xb)
        cur, x = nxt, xb


@pytest.mark.parametrize("prot,seed", [("MKLFS", 3), ("LSRWM", 15), ("LSRLS", 21), ("GLSRA", 22), ("LRSLR", 23)])
def test_envelope_matches_brute_force(sd, E1, par1, prot, seed):
    P = read_params(par1)
    w = inputs.random_codon_weights(seed)
    lo, hi = 0.05, 20.0
    exp_lines, exp_breaks = brute_envelope(P, prot, w, lo, hi)
    lines, breaks = sd.sd_envelope(E1, prot, w, lo, hi)
    got = [(r["energy"], r["codon_cost"]) for r in lines]
    assert len(got) == len(exp_lines), (got, exp_lines)
    for (e, c), (e2, c2) in zip(got, exp_lines):
        assert e == e2 and abs(c - c2) <= 1e-12
    assert np.allclose(breaks, exp_breaks, rtol=0, atol=1e-6)
    # every line's design is exact at a lambda inside its segment
    edges = [lo] + breaks + [hi]
    for q, r in enumerate(lines):
        mid = 0.5 * (edges[q] + edges[q + 1])
        d = sd.sd_design(E1, prot, w, mid)
        assert abs(d["objective"] - (r["energy"] + 100.0 * mid * r["codon_cost"])) <= 1e-6


def test_envelope_of_a_longer_protein_is_consistent(sd, E1):
    """40 aa: lines ordered by decreasing codon cost and increasing energy, the
    breakpoints increase, and the design at each breakpoint ties both lines."""
    prot = inputs.random_protein(40, 52)
    w = inputs.random_codon_weights(52)
    lines, breaks = sd.sd_envelope(E1, prot, w, 0.0, 8.0)
    assert len(lines) >= 2
    for a, b in zip(lines, lines[1:]):
        assert b["codon_cost"] < a["codon_cost"] and b["energy"] > a["energy"]
    assert all(x < y for x, y in zip(breaks, breaks[1:]))
    for q, x in enumerate(breaks):
        d = sd.sd_design(E1, prot, w, x)
        la = lines[q]["energy"] + 100.0 * x * lines[q]["codon_cost"]
        lb = lines[q + 1]["energy"] + 100.0 * x * lines[q + 1]["codon_cost"]
        assert abs(la - lb) <= 1e-6 and abs(d["objective"] - la) <= 1e-6


def test_inverse_lambda(sd, E1):
    prot = inputs.random_protein(40, 52)
    w = inputs.random_codon_weights(52)
    lines, breaks = sd.sd_envelope(E1, prot, w, 0.0, 8.0)
    q = len(lines) // 2
    target = 0.5 * (lines[q - 1]["codon_cost"] + lines[q]["codon_cost"])
    lam, r = sd.sd_inverse_lambda(E1, prot, w, target, 8.0)
    assert lam == breaks[q - 1]
    assert r["codon_cost"] <= target and r["codon_cost"] == lines[q]["codon_cost"]
    below = sd.sd_design(E1, prot, w, lam * (1 - 1e-6))
    assert below["codon_cost"] > target
    with pytest.raises(sd.SdError) as ei:
        sd.sd_inverse_lambda(E1, prot, w, -1.0, 8.0)
    assert ei.value.code == sd.SD_EINFEASIBLE
