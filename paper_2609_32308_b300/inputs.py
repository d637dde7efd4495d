"""Seeded synthetic inputs for the exact codon-lattice design problem.

This module is shared by the CUDA path's tests/benchmarks and by the CPU
oracle's tests.  It only draws random inputs and writes them out; it holds
none of the design method's arithmetic (no loop energies, no lattice, no DP).

Inputs follow the problem statement of Sec. 3 (Eq. 1):
  * a protein of A codon positions (one-letter amino acids, optional final
    ``*`` stop; no stop is appended implicitly),
  * relative adaptiveness weights w(c) in (0, 1] for the 64 codons, indexed
    16*x + 4*y + z with A=0, C=1, G=2, U=3, the maximum over the synonymous
    codons of every amino acid being exactly 1,
  * lambda >= 0 in kcal/mol,
  * integer nearest-neighbour parameters in dcal/mol (0.01 kcal/mol).

The paper's Turner-2004 tables, Swiss-Prot proteins and codon tables are not
available here, so everything is synthetic and seeded: Turner-shaped integer
tables with realistic signs, magnitudes and the rotation symmetries of the
two-loop tables; amino acids i.i.d. from a published composition vector;
per-amino-acid weights u ~ U(0.05, 1] normalised by their maximum.
"""
from __future__ import annotations

import io
import itertools
import math
import os

import numpy as np

NUC = "ACGU"
# Oriented pair types (5' nucleotide, 3' nucleotide), fixed order.
PAIRS = ("AU", "CG", "GC", "UA", "GU", "UG")
PAIR_INDEX = {p: k for k, p in enumerate(PAIRS)}

# Standard genetic code, codon -> one-letter amino acid ('*' = stop).
_BASES = "UCAG"
_AA_STRING = ("FFLLSSSSYY**CC*W"
              "LLLLPPPPHHQQRRRR"
              "IIIMTTTTNNKKSSRR"
              "VVVVAAAADDEEGGGG")
GENETIC_CODE = {}
for _i, _x in enumerate(_BASES):
    for _j, _y in enumerate(_BASES):
        for _k, _z in enumerate(_BASES):
            GENETIC_CODE[_x + _y + _z] = _AA_STRING[16 * _i + 4 * _j + _k]

AMINO_ACIDS = "ACDEFGHIKLMNPQRSTVWY"

# Amino-acid composition (%) of UniProtKB/Swiss-Prot (release statistics,
# rounded to two decimals); used only as the i.i.d. sampling vector.
AA_COMPOSITION = {
    "A": 8.25, "R": 5.53, "N": 4.06, "D": 5.45, "C": 1.37, "Q": 3.93,
    "E": 6.75, "G": 7.07, "H": 2.27, "I": 5.96, "L": 9.66, "K": 5.84,
    "M": 2.42, "F": 3.86, "P": 4.70, "S": 6.56, "T": 5.34, "W": 1.08,
    "Y": 2.92, "V": 6.87,
}


def codon_index(codon: str) -> int:
    """Index of a codon in the 64-entry weight vector (A=0, C=1, G=2, U=3)."""
    return 16 * NUC.index(codon[0]) + 4 * NUC.index(codon[1]) + NUC.index(codon[2])


def synonymous_codons(aa: str) -> list[str]:
    """Codons of one amino acid (or '*'), in ACGU lexicographic order."""
    out = [c for c, a in GENETIC_CODE.items() if a == aa]
    return sorted(out, key=codon_index)


# --------------------------------------------------------------------------
# proteins and codon weights
# --------------------------------------------------------------------------

def random_protein(length: int, seed: int, stop: bool = False) -> str:
    """Amino acids i.i.d. from AA_COMPOSITION; optional explicit final stop."""
    rng = np.random.default_rng(np.random.SeedSequence([0x5D, 1, int(seed)]))
    aas = list(AA_COMPOSITION)
    p = np.array([AA_COMPOSITION[a] for a in aas], dtype=np.float64)
    p /= p.sum()
    idx = rng.choice(len(aas), size=int(length), p=p)
    s = "".join(aas[k] for k in idx)
    return s + ("*" if stop else "")


def random_codon_weights(seed: int, floor: float = 1e-3) -> np.ndarray:
    """w(c) = u(c)/max_syn u, u ~ U(0.05, 1], w >= floor, max exactly 1 per aa."""
    rng = np.random.default_rng(np.random.SeedSequence([0x5D, 2, int(seed)]))
    w = np.zeros(64, dtype=np.float64)
    for aa in AMINO_ACIDS + "*":
        cods = synonymous_codons(aa)
        u = 1.0 - 0.95 * rng.random(len(cods))      # in (0.05, 1]
        m = float(u.max())
        for c, v in zip(cods, u):
            x = v / m
            w[codon_index(c)] = max(x, floor)
        # the maximiser is exactly v/v == 1.0
    return w


def uniform_codon_weights() -> np.ndarray:
    """All weights 1 (every synonymous codon equally adapted)."""
    return np.ones(64, dtype=np.float64)


def lengths_log_uniform(count: int, lo: int, hi: int, seed: int) -> list[int]:
    """Protein lengths round(exp(U(ln lo, ln hi)))."""
    rng = np.random.default_rng(np.random.SeedSequence([0x5D, 3, int(seed)]))
    x = np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))
    return [int(min(hi, max(lo, round(v)))) for v in x]


def lengths_log_normal(count: int, mu: float, sigma: float, lo: int, hi: int,
                       seed: int) -> list[int]:
    """Protein lengths from a log-normal, clipped to [lo, hi]."""
    rng = np.random.default_rng(np.random.SeedSequence([0x5D, 4, int(seed)]))
    x = rng.lognormal(mu, sigma, size=count)
    return [int(min(hi, max(lo, round(v)))) for v in x]


def protein_batch(lengths, seed: int, lambdas=(0.0, 4.0)):
    """A batch of (protein, weights, lambda) triples with per-protein seeds."""
    rng = np.random.default_rng(np.random.SeedSequence([0x5D, 5, int(seed)]))
    out = []
    for k, L in enumerate(lengths):
        s = int(rng.integers(1, 2**31 - 1))
        lam = float(lambdas[int(rng.integers(0, len(lambdas)))])
        out.append((random_protein(L, s), random_codon_weights(s), lam))
    return out


# --------------------------------------------------------------------------
# energy parameters
# --------------------------------------------------------------------------

# Order and shapes of the integer tables in the parameter file.
TABLE_SHAPES = (
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
SPECIAL_LISTS = (("triloop", 5), ("tetraloop", 6), ("hexaloop", 8))
INF_ENTRY = 99999   # marks loop sizes outside the model (never read)


def _strength(t: int) -> int:
    return {0: 2, 1: 3, 2: 3, 3: 2, 4: 1, 5: 1}[t]


def _rev(t: int) -> int:
    p = PAIRS[t]
    return PAIR_INDEX[p[1] + p[0]]


def make_energy_params(seed: int, ml_base: int | None = None) -> dict:
    """Seeded Turner-shaped synthetic integer tables (dcal/mol).

    Two-loop tables are indexed [outer pair][inner pair seen from the loop]
    and carry the 180-degree rotation symmetry of a two-loop:
      stack[t][s] == stack[s][t], int11[t][s][x][y] == int11[s][t][y][x],
      int22[t][s][a][b][c][d] == int22[s][t][c][d][a][b].
    """
    rng = np.random.default_rng(np.random.SeedSequence([0x5D, 6, int(seed)]))
    P: dict = {}
    st = np.zeros((6, 6), dtype=np.int64)
    for t in range(6):
        for s in range(t, 6):
            if _strength(t) == 1 and _strength(s) == 1:
                v = int(rng.integers(-150, 51))
            else:
                v = -(50 * (_strength(t) + _strength(s)) - 50) - int(rng.integers(0, 101))
            st[t, s] = st[s, t] = v
    P["stack"] = st
    for name in ("mismatch_hairpin", "mismatch_interior", "mismatch_interior_1n",
                 "mismatch_interior_23"):
        P[name] = rng.integers(-150, 1, size=(6, 4, 4)).astype(np.int64)
    i11 = np.zeros((6, 6, 4, 4), dtype=np.int64)
    for t in range(6):
        for s in range(6):
            for x in range(4):
                for y in range(4):
                    if (s, t, y, x) < (t, s, x, y):
                        i11[t, s, x, y] = i11[s, t, y, x]
                    else:
                        i11[t, s, x, y] = int(rng.integers(-100, 351))
    P["int11"] = i11
    P["int21"] = rng.integers(-100, 351, size=(6, 6, 4, 4, 4)).astype(np.int64)
    i22 = np.zeros((6, 6, 4, 4, 4, 4), dtype=np.int64)
    for t in range(6):
        for s in range(6):
            for a in range(4):
                for b in range(4):
                    for c in range(4):
                        for d in range(4):
                            if (s, t, c, d, a, b) < (t, s, a, b, c, d):
                                i22[t, s, a, b, c, d] = i22[s, t, c, d, a, b]
                            else:
                                i22[t, s, a, b, c, d] = int(rng.integers(-100, 351))
    P["int22"] = i22

    def increasing(lo, hi, first):
        v = np.full(31, INF_ENTRY, dtype=np.int64)
        xs = np.sort(rng.integers(lo, hi + 1, size=31 - first))
        v[first:] = xs
        return v

    P["hairpin"] = increasing(350, 650, 3)
    P["bulge"] = increasing(280, 600, 1)
    P["interior"] = increasing(100, 500, 2)
    P["terminal_au"] = np.array([50 if _strength(t) != 3 else 0 for t in range(6)],
                                dtype=np.int64)
    P["ninio"] = np.array([60], dtype=np.int64)
    P["max_ninio"] = np.array([300], dtype=np.int64)
    P["ml_closing"] = np.array([int(rng.integers(300, 401))], dtype=np.int64)
    P["ml_intern"] = np.array([int(rng.integers(-100, 51))], dtype=np.int64)
    P["ml_base"] = np.array([0 if ml_base is None else int(ml_base)], dtype=np.int64)
    P["lxc"] = 107.856
    counts = {"triloop": 20, "tetraloop": 30, "hexaloop": 4}
    for name, L in SPECIAL_LISTS:
        seen = {}
        while len(seen) < counts[name]:
            t = int(rng.integers(0, 6))
            mid = "".join(NUC[int(k)] for k in rng.integers(0, 4, size=L - 2))
            seq = PAIRS[t][0] + mid + PAIRS[t][1]
            if seq not in seen:
                seen[seq] = int(rng.integers(150, 501))
        P[name] = sorted(seen.items())
    return P


class SplitMix64:
    """SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): a 64-bit counter
    advanced by 0x9E3779B97F4A7C15, mixed by two xor-shift-multiply rounds.
    The library's seeded parameter sets (sd_load_energy with no file) draw
    from the same generator, so both sides produce identical tables."""
    MASK = (1 << 64) - 1

    def __init__(self, seed: int):
        self.x = (int(seed) ^ 0x5D5D5D5D5D5D5D5D) & self.MASK

    def next(self) -> int:
        self.x = (self.x + 0x9E3779B97F4A7C15) & self.MASK
        z = self.x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self, lo: int, hi: int) -> int:
        """Integer in [lo, hi]."""
        return lo + self.next() % (hi - lo + 1)


def synthetic_energy_params(seed: int) -> dict:
    """The seeded Turner-shaped tables of the library's sd_load_energy(NULL,
    seed): the recipe of make_energy_params (same ranges, shapes and
    rotation symmetries) drawn from SplitMix64 in a fixed order."""
    R = SplitMix64(seed)
    P: dict = {}
    st = np.zeros((6, 6), dtype=np.int64)
    for t in range(6):
        for s in range(t, 6):
            if _strength(t) == 1 and _strength(s) == 1:
                v = R.uniform(-150, 50)
            else:
                v = -(50 * (_strength(t) + _strength(s)) - 50) - R.uniform(0, 100)
            st[t, s] = st[s, t] = v
    P["stack"] = st
    for name in ("mismatch_hairpin", "mismatch_interior", "mismatch_interior_1n",
                 "mismatch_interior_23"):
        P[name] = np.array([R.uniform(-150, 0) for _ in range(96)], dtype=np.int64).reshape(6, 4, 4)
    i11 = np.zeros((6, 6, 4, 4), dtype=np.int64)
    for t, s_, x, y in itertools.product(range(6), range(6), range(4), range(4)):
        i11[t, s_, x, y] = (i11[s_, t, y, x] if (s_, t, y, x) < (t, s_, x, y)
                            else R.uniform(-100, 350))
    P["int11"] = i11
    P["int21"] = np.array([R.uniform(-100, 350) for _ in range(2304)],
                          dtype=np.int64).reshape(6, 6, 4, 4, 4)
    i22 = np.zeros((6, 6, 4, 4, 4, 4), dtype=np.int64)
    for t, s_, a, b, c, d in itertools.product(range(6), range(6), range(4), range(4), range(4),
                                               range(4)):
        i22[t, s_, a, b, c, d] = (i22[s_, t, c, d, a, b] if (s_, t, c, d, a, b) < (t, s_, a, b, c, d)
                                  else R.uniform(-100, 350))
    P["int22"] = i22

    def increasing(lo, hi, first):
        v = np.full(31, INF_ENTRY, dtype=np.int64)
        v[first:] = sorted(R.uniform(lo, hi) for _ in range(31 - first))
        return v

    P["hairpin"] = increasing(350, 650, 3)
    P["bulge"] = increasing(280, 600, 1)
    P["interior"] = increasing(100, 500, 2)
    P["terminal_au"] = np.array([50 if _strength(t) != 3 else 0 for t in range(6)],
                                dtype=np.int64)
    P["ninio"] = np.array([60], dtype=np.int64)
    P["max_ninio"] = np.array([300], dtype=np.int64)
    P["ml_closing"] = np.array([R.uniform(300, 400)], dtype=np.int64)
    P["ml_intern"] = np.array([R.uniform(-100, 50)], dtype=np.int64)
    P["ml_base"] = np.array([0], dtype=np.int64)
    P["lxc"] = 107.856
    for (name, L), count in zip(SPECIAL_LISTS, (20, 30, 4)):
        seen = {}
        while len(seen) < count:
            t = R.uniform(0, 5)
            seq = PAIRS[t][0] + "".join(NUC[R.uniform(0, 3)] for _ in range(L - 2)) + PAIRS[t][1]
            if seq not in seen:
                seen[seq] = R.uniform(150, 500)
        P[name] = sorted(seen.items())
    return P


def synthetic_energy_file(seed: int, directory: str) -> str:
    """Write (once) the file of synthetic_energy_params(seed) and return its path."""
    os.makedirs(directory, exist_ok=True)
    path = os.path.join(directory, f"sd_synth_{seed}.par")
    if not os.path.exists(path):
        tmp = path + f".tmp{os.getpid()}"
        write_energy_file(synthetic_energy_params(seed), tmp)
        os.replace(tmp, path)
    return path


def energy_text(P: dict) -> str:
    """Serialise a parameter dict to the plain-text parameter format.

    Format: a header line ``SDENERGY 1``; then for each table in
    TABLE_SHAPES a line ``<name> <count>`` followed by <count> integers in
    C (row-major) order; then ``lxc <float>``; then for each special hairpin
    list ``<name> <count>`` followed by <count> lines ``<sequence> <total>``.
    """
    out = io.StringIO()
    out.write("SDENERGY 1\n")
    for name, shape in TABLE_SHAPES:
        a = np.asarray(P[name], dtype=np.int64).reshape(-1)
        assert a.size == int(np.prod(shape)), name
        out.write(f"{name} {a.size}\n")
        for k in range(0, a.size, 16):
            out.write(" ".join(str(int(v)) for v in a[k:k + 16]) + "\n")
    out.write(f"lxc {float(P['lxc'])!r}\n")
    for name, _L in SPECIAL_LISTS:
        items = P[name]
        out.write(f"{name} {len(items)}\n")
        for seq, e in items:
            out.write(f"{seq} {int(e)}\n")
    return out.getvalue()


def write_energy_file(P: dict, path: str) -> str:
    with open(path, "w") as f:
        f.write(energy_text(P))
    return path


def energy_file_for_seed(seed: int, directory: str, ml_base: int | None = None) -> str:
    """Write (once) the synthetic parameter file for a seed and return its path."""
    os.makedirs(directory, exist_ok=True)
    tag = "" if ml_base is None else f"_mlb{ml_base}"
    path = os.path.join(directory, f"sd_energy_{seed}{tag}.par")
    if not os.path.exists(path):
        tmp = path + f".tmp{os.getpid()}"
        write_energy_file(make_energy_params(seed, ml_base), tmp)
        os.replace(tmp, path)
    return path
