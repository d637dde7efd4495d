"""Pins of the CPU oracle against facts independent of its own code.

Chain of pins (no value here is produced by the CUDA path):
  * the Python evaluator against hand-derived loop decompositions (each
    expected energy lists the table entries a loop must read, Sec. 3 model);
  * the Python Zuker fold against exhaustive structure enumeration scored by
    the evaluator (tiny sequences);
  * the C oracle on a width-1 lattice (one fixed sequence) against Zuker --
    the textbook special case of the lattice DP;
  * the C oracle on codon lattices against brute-force enumeration of every
    synonymous mRNA (Eq. 1), exact in fixed point, at lambda = 0 (heavily
    tied) and lambda > 0, with zero and nonzero multiloop unpaired penalty;
  * invariants of Sec. 4-5: translation, re-evaluated objective equals the DP
    value, Z <= B_finite, candidates only among finite direct intervals,
    D1 = min(B, P_D); the 30 / 31 unpaired two-loop boundary; lambda limits.
"""
import itertools
import math
import random

import numpy as np
import pytest

import oracle
from oracle import brute, evaluate, zuker
from oracle.params import read_params
from paper_2609_32308_b300 import inputs

NUC = "ACGU"
PT = {p: k for k, p in enumerate(("AU", "CG", "GC", "UA", "GU", "UG"))}


def nt(c):
    return NUC.index(c)


@pytest.fixture(scope="module")
def P1(par1):
    return read_params(par1)


# ----------------------------------------------------------------------
# evaluator against hand-derived loop decompositions
# ----------------------------------------------------------------------

def test_eval_stacked_hairpin(P1):
    seq, st = "GGGAAACCC", "(((...)))"
    hp = P1["triloop"].get("GAAAC", int(P1["hairpin"][3]) + int(P1["terminal_au"][PT["GC"]]))
    # outer G0-C8 (GC) over G1-C7 seen from the loop as C7-G1 (CG), twice
    exp = 2 * int(P1["stack"][PT["GC"]][PT["CG"]]) + hp + int(P1["terminal_au"][PT["GC"]])
    assert evaluate.energy(P1, seq, st) == exp


def test_eval_special_tetraloop(P1):
    tl, tot = sorted(P1["tetraloop"].items())[0]
    seq = "G" + tl + "C"
    st = "((....))"
    inner = PT[tl[-1] + tl[0]]            # inner pair read 3'->5' from the loop
    exp = int(P1["stack"][PT["GC"]][inner]) + tot + int(P1["terminal_au"][PT["GC"]])
    assert evaluate.energy(P1, seq, st) == exp


def test_eval_generic_hairpin_and_long_hairpin(P1):
    seq = "CAAAAAG"        # L = 5 generic hairpin: hairpin[5] + mismatchH[CG][A][A]
    exp = int(P1["hairpin"][5]) + int(P1["mismatch_hairpin"][PT["CG"]][0][0])
    assert evaluate.energy(P1, seq, "(.....)") == exp + int(P1["terminal_au"][PT["CG"]])
    L = 40
    seq = "U" + "C" * L + "A"
    exp = (int(P1["hairpin"][30]) + int(P1["lxc"] * math.log(L / 30.0))
           + int(P1["mismatch_hairpin"][PT["UA"]][1][1]) + int(P1["terminal_au"][PT["UA"]]))
    assert evaluate.energy(P1, seq, "(" + "." * L + ")") == exp


def _two_loop_case(P1, left, right, inner_seq="GAAAAC"):
    # outer pair C...G around: left unpaired, inner pair G...C with hairpin AAAA
    seq = "C" + left + inner_seq + right + "G"
    st = "(" + "." * len(left) + "(....)" + "." * len(right) + ")"
    hp_seq = inner_seq
    hp = P1["tetraloop"].get(hp_seq, int(P1["hairpin"][4]) +
                             int(P1["mismatch_hairpin"][PT["GC"]][0][0]))
    base = hp + int(P1["terminal_au"][PT["CG"]])
    return seq, st, base


def test_eval_two_loop_classes(P1):
    t, s = PT["CG"], PT["CG"]        # outer C-G; inner G-C seen from loop as C-G
    ninio, mx = P1["ninio"], P1["max_ninio"]
    au = P1["terminal_au"]
    cases = []
    # stack
    cases.append(("", "", int(P1["stack"][t][s])))
    # bulge 1 (left) and bulge 3 (right)
    cases.append(("U", "", int(P1["bulge"][1]) + int(P1["stack"][t][s])))
    cases.append(("", "UUU", int(P1["bulge"][3]) + int(au[t]) + int(au[s])))
    # 1x1: int11[t][s][x_{i+1}][x_{j-1}]
    cases.append(("A", "U", int(P1["int11"][t][s][nt("A")][nt("U")])))
    # 1x2: int21[t][s][x_{i+1}][x_{q+1}][x_{j-1}]
    cases.append(("A", "CU", int(P1["int21"][t][s][nt("A")][nt("C")][nt("U")])))
    # 2x1: read from the inner pair's side: int21[s][t][x_{q+1}][x_{i+1}][x_{p-1}]
    cases.append(("AC", "U", int(P1["int21"][s][t][nt("U")][nt("A")][nt("C")])))
    # 2x2: int22[t][s][x_{i+1}][x_{p-1}][x_{q+1}][x_{j-1}]
    cases.append(("AC", "UA", int(P1["int22"][t][s][0][1][3][0])))
    # 1x4: interior[5] + min(MAXNINIO, 3 ninio) + mm1n both pairs
    m1 = P1["mismatch_interior_1n"]
    cases.append(("A", "CCUU", int(P1["interior"][5]) + min(mx, 3 * ninio)
                  + int(m1[t][nt("A")][nt("U")]) + int(m1[s][nt("C")][nt("A")])))
    # 2x3: interior[5] + ninio + mm23 both pairs
    m23 = P1["mismatch_interior_23"]
    cases.append(("AC", "UAU", int(P1["interior"][5]) + ninio
                  + int(m23[t][nt("A")][nt("U")]) + int(m23[s][nt("U")][nt("C")])))
    # generic 3x5
    mi = P1["mismatch_interior"]
    cases.append(("ACU", "UAUCA", int(P1["interior"][8]) + min(mx, 2 * ninio)
                  + int(mi[t][nt("A")][nt("A")]) + int(mi[s][nt("U")][nt("U")])))
    for left, right, loop in cases:
        seq, st, base = _two_loop_case(P1, left, right)
        assert evaluate.energy(P1, seq, st) == loop + base, (left, right)


def test_eval_multiloop(P1):
    # closing pair G0-C20, branches (1..8) and (10..17), unpaired 9, 18, 19
    seq = "G" + "GAAAAAAC" + "A" + "CAAAAAAG" + "AA" + "C"
    st = "(" + "(......)" + "." + "(......)" + ".." + ")"
    au = P1["terminal_au"]
    hp1 = int(P1["hairpin"][6]) + int(P1["mismatch_hairpin"][PT["GC"]][0][0])
    hp2 = int(P1["hairpin"][6]) + int(P1["mismatch_hairpin"][PT["CG"]][0][0])
    hp1 = P1["hexaloop"].get("GAAAAAAC", hp1)
    hp2 = P1["hexaloop"].get("CAAAAAAG", hp2)
    ml = (P1["ml_closing"] + P1["ml_intern"] + int(au[PT["GC"]])
          + 2 * P1["ml_intern"] + int(au[PT["GC"]]) + int(au[PT["CG"]]) + 3 * P1["ml_base"])
    assert evaluate.energy(P1, seq, st) == hp1 + hp2 + ml + int(au[PT["GC"]])


def test_eval_rejects_bad_structures(P1):
    with pytest.raises(ValueError):
        evaluate.energy(P1, "GAAAA", "(...)")      # G-A cannot pair
    with pytest.raises(ValueError):
        evaluate.energy(P1, "GAAC", "(..)")        # hairpin shorter than 3
    with pytest.raises(ValueError):
        evaluate.energy(P1, "GGAAACC", "((...)")


def test_oracle_hairpin_energy_matches_evaluator(par1, P1):
    # the C oracle's loop function and the Python evaluator, special and generic
    for seqs in (list(P1["triloop"]) + list(P1["tetraloop"]) + list(P1["hexaloop"])):
        assert oracle.hairpin_energy(par1, seqs) == evaluate.hairpin_energy(P1, seqs, 0, len(seqs) - 1)
    rng = random.Random(5)
    for _ in range(200):
        L = rng.randint(3, 40)
        pr = rng.choice(["AU", "CG", "GC", "UA", "GU", "UG"])
        s = pr[0] + "".join(rng.choice(NUC) for _ in range(L)) + pr[1]
        assert oracle.hairpin_energy(par1, s) == evaluate.hairpin_energy(P1, s, 0, len(s) - 1)


def _two_loop_classes():
    """(l1, l2) of every two-loop class of the Sec. 3 model (l1 + l2 <= 30)."""
    yield "stack", [(0, 0)]
    yield "bulge1", [(1, 0), (0, 1)]
    yield "bulge", [(0, l) for l in range(2, 31)] + [(l, 0) for l in range(2, 31)]
    yield "1x1", [(1, 1)]
    yield "1x2", [(1, 2)]
    yield "2x1", [(2, 1)]
    yield "2x2", [(2, 2)]
    yield "1xn", [(1, l) for l in range(3, 30)] + [(l, 1) for l in range(3, 30)]
    yield "2x3", [(2, 3), (3, 2)]
    yield "generic", [(a, b) for a in range(2, 29) for b in range(2, 29)
                      if a + b <= 30 and (a, b) not in ((2, 2), (2, 3), (3, 2))]


@pytest.mark.parametrize("cls,shapes", list(_two_loop_classes()))
def test_oracle_two_loop_energy_matches_evaluator(par1, P1, cls, shapes):
    """The C oracle's two-loop function against the independent evaluator,
    class by class, with random outer and inner pair types and loop
    nucleotides (a swapped mismatch argument or a wrong int21 rotation in
    any class fails here, whether or not that class is ever optimal)."""
    rng = random.Random(sum(map(ord, cls)))
    pairs = ["AU", "CG", "GC", "UA", "GU", "UG"]
    for k in range(max(300, 4 * len(shapes))):
        l1, l2 = shapes[k % len(shapes)]
        outer, inner = rng.choice(pairs), rng.choice(pairs)
        left = outer[0] + "".join(rng.choice(NUC) for _ in range(l1)) + inner[0]
        right = inner[1] + "".join(rng.choice(NUC) for _ in range(l2)) + outer[1]
        seq = left + right
        i, p, q, j = 0, len(left) - 1, len(left), len(seq) - 1
        exp = evaluate.interior_energy(P1, seq, i, j, p, q)
        assert oracle.twoloop_energy(par1, left, right) == exp, (cls, left, right)


# ----------------------------------------------------------------------
# Zuker against exhaustive enumeration
# ----------------------------------------------------------------------

def test_zuker_equals_exhaustive_enumeration(P1):
    rng = random.Random(11)
    for _ in range(40):
        n = rng.randint(5, 14)
        s = "".join(rng.choice("ACGU" if rng.random() < 0.5 else "GCCG") for _ in range(n))
        best = 0
        for st in zuker.all_structures(n):
            try:
                best = min(best, evaluate.energy(P1, s, st))
            except ValueError:
                pass
        assert zuker.mfe(P1, s) == best, s


# ----------------------------------------------------------------------
# oracle on a single fixed sequence == Zuker
# ----------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(12))
def test_oracle_width1_equals_zuker(par1, P1, seed):
    rng = random.Random(100 + seed)
    n = rng.randint(12, 48)
    s = "".join(rng.choice(NUC) for _ in range(n))
    o = oracle.run_rna(par1, s)
    assert o.status == 0
    assert o.mrna == s
    z = zuker.mfe(P1, s)
    assert o.obj_fx == z << 32
    assert o.energy == z
    assert evaluate.energy(P1, o.mrna, o.structure) == z


def test_oracle_width1_nonzero_ml_base(par_mlbase):
    P = read_params(par_mlbase)
    rng = random.Random(7)
    for _ in range(6):
        n = rng.randint(30, 50)
        s = "".join(rng.choice("GGCCAU") for _ in range(n))
        o = oracle.run_rna(par_mlbase, s)
        assert o.status == 0
        assert o.energy == zuker.mfe(P, s)
        assert evaluate.energy(P, o.mrna, o.structure) == o.energy


def _golden(name):
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    with open(path) as f:
        return [l.split() for l in f if l.strip() and not l.startswith("#")]


def test_internal_loop_cap_30_vs_31(par1, P1):
    """Sec. 3 / Sec. 6.1 fixture (tests/golden/loop_cap_30_31.txt): a two-loop
    with 30 unpaired nucleotides is inside the optimisation domain, one with
    31 is not (the evaluator still scores it)."""
    rows = _golden("loop_cap_30_31.txt")
    assert [(int(r[0]), int(r[1])) for r in rows] == [(30, 1), (31, 0)]
    for unp, inside, seq, st in rows:
        unp, inside = int(unp), int(inside)
        e_struct = evaluate.energy(P1, seq, st)
        assert evaluate.max_two_loop_unpaired(st) == unp
        o = oracle.run_rna(par1, seq)
        assert o.status == 0
        assert evaluate.max_two_loop_unpaired(o.structure) <= 30
        assert o.energy == zuker.mfe(P1, seq)
        if inside:
            assert o.energy <= e_struct
        else:
            # the 31-unpaired structure scores strictly below the oracle's
            # optimum: only the cap keeps it out of the domain
            assert e_struct < o.energy
        assert o.energy == evaluate.energy(P1, o.mrna, o.structure)


# ----------------------------------------------------------------------
# oracle on codon lattices == brute force over synonymous mRNAs (Eq. 1)
# ----------------------------------------------------------------------

def _small_cases():
    rng = random.Random(2024)
    out = []
    while len(out) < 10:
        A = rng.randint(3, 6)
        prot = "".join(rng.choice("LSRAGVKMWFYC") for _ in range(A))
        if brute.synonymous_space(prot) <= 1500:
            out.append((prot, rng.randint(1, 10**6)))
    out.append(("MLS*", 5))
    out.append(("WMW", 6))
    return out


@pytest.mark.parametrize("prot,wseed", _small_cases())
def test_oracle_equals_brute_force(par1, P1, prot, wseed):
    w = inputs.random_codon_weights(wseed)
    for lam in (0.0, 0.25, 4.0):
        o = oracle.run(par1, prot, w, lam)
        assert o.status == 0
        best, arg = brute.brute_force(P1, prot, w, lam)
        assert o.obj_fx == best
        assert o.mrna in arg
        assert evaluate.energy(P1, o.mrna, o.structure) == o.energy


def test_oracle_brute_force_nonzero_ml_base(par_mlbase):
    P = read_params(par_mlbase)
    w = inputs.random_codon_weights(3)
    for prot in ("LLRS", "GSLRA"):
        for lam in (0.0, 2.0):
            o = oracle.run(par_mlbase, prot, w, lam)
            best, arg = brute.brute_force(P, prot, w, lam)
            assert o.obj_fx == best and o.mrna in arg


# ----------------------------------------------------------------------
# invariants on larger designs
# ----------------------------------------------------------------------

def translate(mrna):
    return "".join(inputs.GENETIC_CODE[mrna[k:k + 3]] for k in range(0, len(mrna), 3))


@pytest.mark.parametrize("A,seed,lam", [(40, 1, 0.0), (40, 2, 4.0), (60, 3, 4.0), (25, 4, 1.5)])
def test_oracle_design_invariants(par1, P1, A, seed, lam):
    prot = inputs.random_protein(A, seed)
    w = inputs.random_codon_weights(seed)
    o = oracle.run(par1, prot, w, lam)
    assert o.status == 0
    assert translate(o.mrna) == prot
    assert evaluate.energy(P1, o.mrna, o.structure) == o.energy
    assert evaluate.max_two_loop_unpaired(o.structure) <= 30
    codons = [o.mrna[k:k + 3] for k in range(0, len(o.mrna), 3)]
    qsum = sum(brute.qfx(lam, w[inputs.codon_index(c)]) for c in codons)
    assert o.obj_fx == (o.energy << 32) + qsum
    cc = 0.0
    for c in codons:
        cc += -math.log(w[inputs.codon_index(c)])
    assert o.codon_cost == cc
    assert o.objective == float(o.energy) + (100.0 * lam) * cc
    # Sec. 4.1: D1 = min(B, P_D); C_b only among finite direct intervals; Z <= B_finite
    fin = o.B < oracle.INF
    assert np.array_equal(o.D1, np.minimum(o.B, o.PD))
    assert not np.any(o.cand.astype(bool) & ~fin)
    assert np.array_equal(o.cand.astype(bool), fin & (o.B < o.PD))
    assert o.Z == int(o.cand.sum()) <= o.finite_direct == int(fin.sum())
    # the DP value is the exterior value at the source
    assert o.obj_fx == o.Ext[0]


def test_oracle_lattice_and_codon_costs(par1):
    prot = "LSR*"
    w = inputs.random_codon_weights(9)
    o = oracle.run(par1, prot, w, 4.0)
    # layers 0..12; boundary layers single states; Leu/Ser/Arg/stop split
    counts = np.bincount(o.layer, minlength=o.n + 1)
    assert list(counts) == [1, 2, 2, 1, 2, 2, 1, 2, 2, 1, 1, 2, 1]
    # third-codon-position edges carry the fixed-point -ln w, the rest 0
    for f, t, lab, c in zip(o.edge_from, o.edge_to, o.edge_label, o.edge_cost):
        if o.layer[t] % 3 != 0:
            assert c == 0
    stop_costs = sorted(int(c) for f, t, lab, c in zip(o.edge_from, o.edge_to, o.edge_label,
                                                        o.edge_cost) if o.layer[t] == 12)
    exp = sorted(brute.qfx(4.0, w[inputs.codon_index(c)]) for c in ("UAA", "UAG", "UGA"))
    assert stop_costs == exp
    assert oracle.codon_cost_fx(4.0, 0.5) == round(math.ldexp(400.0 * math.log(2.0), 32))


def test_lambda_limits(par1, P1):
    """lambda = 0 gives a pure-MFE design; a lambda large enough that any
    codon change costs more than any energy gain forces the w = 1 codons."""
    prot = "MKLFSRG"
    w = np.full(64, 0.5)
    for aa in set(prot):
        w[inputs.codon_index(inputs.synonymous_codons(aa)[-1])] = 1.0
    best_seq = "".join(inputs.synonymous_codons(aa)[-1] for aa in prot)
    o = oracle.run(par1, prot, w, 100.0)
    assert o.mrna == best_seq
    assert o.energy == zuker.mfe(P1, best_seq)
    o0 = oracle.run(par1, prot, w, 0.0)
    assert o0.obj_fx == o0.energy << 32
    assert o0.energy <= o.energy


def test_empty_and_tiny_proteins(par1):
    w = inputs.random_codon_weights(1)
    o = oracle.run(par1, "", w, 4.0)
    assert o.mrna == "" and o.structure == "" and o.energy == 0 and o.obj_fx == 0
    o = oracle.run(par1, "M", w, 4.0)
    assert o.mrna == "AUG" and o.structure == "..." and o.energy == 0
    with pytest.raises(ValueError):
        oracle.run(par1, "M*M", w, 1.0)          # stop only at the end
    with pytest.raises(ValueError):
        oracle.run(par1, "MBX", w, 1.0)          # unknown amino acids
    bad = w.copy()
    bad[inputs.codon_index("AUG")] = 0.9         # max over Met's codons is not 1
    with pytest.raises(ValueError):
        oracle.run(par1, "M", bad, 1.0)


def test_oracle_reproduces_its_golden_designs(par1):
    """tests/golden/oracle_designs.txt was written by the oracle alone
    (tests/golden/make_oracle_designs.py); a change to the oracle's arithmetic
    or tie-break shows up here."""
    for A, seed, lam, mrna, st, e, ofx, Z in _golden("oracle_designs.txt"):
        prot = inputs.random_protein(int(A), int(seed))
        w = inputs.random_codon_weights(int(seed))
        o = oracle.run(par1, prot, w, float(lam))
        assert (o.mrna, o.structure, o.energy, o.obj_fx, o.Z) == (mrna, st, int(e), int(ofx), int(Z))


def test_oracle_threads_do_not_change_tables(par1):
    """Filling each span's layer pairs on several threads (the paper's scheme,
    Algorithm 1) gives the same tables and design as one thread."""
    prot = inputs.random_protein(40, 77)
    w = inputs.random_codon_weights(77)
    a = oracle.run(par1, prot, w, 4.0)
    old = oracle.set_threads(4)
    try:
        b = oracle.run(par1, prot, w, 4.0)
    finally:
        oracle.set_threads(old)
    assert (a.mrna, a.structure, a.obj_fx) == (b.mrna, b.structure, b.obj_fx)
    for name in ("H", "V", "B", "D1", "D2", "PD", "Ext", "cand"):
        assert np.array_equal(getattr(a, name), getattr(b, name)), name


# ----------------------------------------------------------------------
# forbidden motifs (Sec. 3: codon DFA x Aho-Corasick automaton)
# ----------------------------------------------------------------------

MOTIF_CASES = [("MKLFS", ["CUG", "AAA"], 3), ("LSRWM", ["UCG", "CGA", "AGC"], 15),
               ("GLSRA", ["CUG", "UCU", "GCA"], 22), ("RLS", ["AGA", "CUU", "UUA"], 5),
               ("MLS*", ["UAA", "UAG"], 9), ("LRSLR", ["CG", "UUA"], 23)]


@pytest.mark.parametrize("prot,motifs,wseed", MOTIF_CASES)
def test_oracle_motifs_equal_brute_force(par1, P1, prot, motifs, wseed):
    """The motif-constrained optimum is the brute-force minimum over the
    synonymous mRNAs that contain no motif (Eq. 1 restricted to the motif-free
    language), at lambda 0 and > 0."""
    w = inputs.random_codon_weights(wseed)
    for lam in (0.0, 4.0):
        o = oracle.run_motifs(par1, prot, w, lam, motifs)
        best, arg = brute.brute_force(P1, prot, w, lam, motifs)
        assert best is not None, "every test case has a motif-free design"
        assert o is not None and o.status == 0
        assert o.obj_fx == best and o.mrna in arg
        assert not any(m in o.mrna for m in motifs)
        assert evaluate.energy(P1, o.mrna, o.structure) == o.energy
        plain = oracle.run(par1, prot, w, lam)
        assert o.obj_fx >= plain.obj_fx


def _walk_states(prot, motifs):
    """States (layer, codon-trie state, matcher prefix) visited by every
    motif-free synonymous mRNA, the last layer merged: the trimmed product."""
    seen = set()
    prefixes = {""} | {m[:l] for m in motifs for l in range(1, len(m) + 1)}
    for combo in itertools.product(*[brute.codons_of(a) for a in prot]):
        r = "".join(combo)
        if any(m in r for m in motifs):
            continue
        cur = ""
        for k in range(len(r) + 1):
            # codon-trie state: the prefix of the current codon
            q = r[3 * (k // 3):k] if k % 3 else ""
            seen.add((k, k // 3, q, cur if k < len(r) else ""))
            if k < len(r):
                t = cur + r[k]
                while t not in prefixes:
                    t = t[1:]
                cur = t
    return seen


@pytest.mark.parametrize("prot,motifs,wseed", MOTIF_CASES)
def test_oracle_motif_product_states(par1, prot, motifs, wseed):
    o = oracle.run_motifs(par1, prot, inputs.random_codon_weights(wseed), 1.0, motifs)
    counts = np.bincount(o.layer, minlength=o.n + 1)
    exp = np.zeros(o.n + 1, dtype=int)
    for (k, _, _, _) in _walk_states(prot, motifs):
        exp[k] += 1
    assert counts.tolist() == exp.tolist()


def test_oracle_motifs_empty_inventory_and_infeasible(par1):
    prot = inputs.random_protein(30, 44)
    w = inputs.random_codon_weights(44)
    a = oracle.run(par1, prot, w, 4.0)
    b = oracle.run_motifs(par1, prot, w, 4.0, [])
    assert (a.mrna, a.obj_fx, a.N) == (b.mrna, b.obj_fx, b.N)
    assert np.array_equal(a.V, b.V) and np.array_equal(a.D2, b.D2)
    # unavoidable motifs: the brute force finds no motif-free mRNA either
    for p, m in (("M", ["AUG"]), ("KK", ["A"]), ("MW", ["GU"]), ("LSRWM", ["UCG", "CGA", "GAU"]),
                 ("GLSRA", ["GG", "UCU"])):
        assert oracle.run_motifs(par1, p, w, 1.0, m) is None
        assert brute.brute_force(read_params(par1), p, w, 1.0, m) == (None, [])


def test_branch_interface_is_the_best_type_plus_ml_intern(par1, P1):
    """Eq. (branch): B(a, b) = min over pair types t of V_t(a, b) + ML_intern +
    AU(t), so B - ML_intern is the exterior branch cost min_t V_t + AU(t) (the
    identity the device exterior pass and traceback read B through), on the
    oracle's tables of two designs; cells that no type closes stay +inf."""
    scale = 1 << 32
    au = np.array([int(x) for x in P1["terminal_au"]], dtype=np.int64)
    mli = int(P1["ml_intern"])
    for A, seed, lam in ((14, 41, 4.0), (20, 42, 0.0)):
        prot = inputs.random_protein(A, seed)
        w = inputs.random_codon_weights(seed)
        o = oracle.run(par1, prot, w, lam)
        fin = o.V < oracle.INF
        closed = o.B < oracle.INF
        assert closed.any() and not closed.all()
        best = np.where(fin, o.V + (mli + au)[None, None, :] * scale, oracle.INF).min(axis=2)
        assert np.array_equal(np.where(closed, o.B, 0), np.where(closed, best, 0))
        assert (best[~closed] >= oracle.INF).all()
        ext = np.where(fin, o.V + au[None, None, :] * scale, oracle.INF).min(axis=2)
        assert np.array_equal(ext[closed], o.B[closed] - mli * scale)
