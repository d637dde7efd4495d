"""CPU oracle for exact codon-lattice design -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline /
reference leg may import this package.  The product path (the CUDA library
and its Python binding) never imports, links or executes anything here.

Contents
  * ``sd_oracle.c`` -- the dense square-table DP of Sec. 4.1 (Eqs. dense2,
    partitionable, dense1; typed closed values; final-column exterior of
    Sec. 5) over the codon DFA of Sec. 3, plus its canonical traceback.
    Built into ``liboracle.so`` by :func:`build` (plain ``gcc``).
  * ``params.py``  -- a parameter-file reader for the Python checkers.
  * ``evaluate.py`` -- an independent structure-energy evaluator.
  * ``zuker.py``   -- an independent fixed-sequence Zuker MFE fold.
  * ``brute.py``   -- brute-force enumeration of synonymous mRNAs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

FX_ONE = 1 << 32          # one energy unit (0.01 kcal/mol) in fixed point
INF = 1 << 62


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (plain gcc, no GPU)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-Wall", "-fopenmp",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        lib.orc_run.argtypes = [ctypes.c_char_p, ctypes.c_char_p,
                                ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                ctypes.POINTER(P)]
        lib.orc_run.restype = ctypes.c_int
        lib.orc_run_rna.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(P)]
        lib.orc_run_rna.restype = ctypes.c_int
        lib.orc_free.argtypes = [P]
        for f in ("orc_n", "orc_num_states", "orc_num_edges"):
            getattr(lib, f).argtypes = [P]
            getattr(lib, f).restype = ctypes.c_int
        lib.orc_layers.argtypes = [P, P]
        lib.orc_edges.argtypes = [P, P, P, P, P]
        lib.orc_tables.argtypes = [P] * 9
        lib.orc_result.argtypes = [P] * 8
        lib.orc_counts.argtypes = [P] * 4
        lib.orc_codon_cost_fx.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.orc_codon_cost_fx.restype = ctypes.c_int64
        lib.orc_hairpin_energy.argtypes = [ctypes.c_char_p, ctypes.c_char_p]
        lib.orc_hairpin_energy.restype = ctypes.c_int
        lib.orc_twoloop_energy.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p]
        lib.orc_twoloop_energy.restype = ctypes.c_int
        lib.orc_run_motifs.argtypes = [ctypes.c_char_p, ctypes.c_char_p,
                                       ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                       ctypes.c_char_p, ctypes.POINTER(P)]
        lib.orc_run_motifs.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleDesign:
    """Result and dense tables of one oracle run (square N x N layout)."""

    def __init__(self, handle, status):
        lib = _load()
        self.status = status
        self.n = lib.orc_n(handle)
        self.N = lib.orc_num_states(handle)
        E = lib.orc_num_edges(handle)
        self.layer = np.zeros(self.N, dtype=np.int32)
        lib.orc_layers(handle, _ptr(self.layer))
        self.edge_from = np.zeros(E, dtype=np.int32)
        self.edge_to = np.zeros(E, dtype=np.int32)
        self.edge_label = np.zeros(E, dtype=np.int32)
        self.edge_cost = np.zeros(E, dtype=np.int64)
        lib.orc_edges(handle, _ptr(self.edge_from), _ptr(self.edge_to), _ptr(self.edge_label),
                      _ptr(self.edge_cost))
        N = self.N
        self.H = np.zeros((N, N), dtype=np.int64)
        self.V = np.zeros((N, N, 6), dtype=np.int64)
        self.B = np.zeros((N, N), dtype=np.int64)
        self.D1 = np.zeros((N, N), dtype=np.int64)
        self.D2 = np.zeros((N, N), dtype=np.int64)
        self.PD = np.zeros((N, N), dtype=np.int64)
        self.Ext = np.zeros(N, dtype=np.int64)
        self.cand = np.zeros((N, N), dtype=np.uint8)
        lib.orc_tables(handle, _ptr(self.H), _ptr(self.V), _ptr(self.B), _ptr(self.D1),
                       _ptr(self.D2), _ptr(self.PD), _ptr(self.Ext), _ptr(self.cand))
        mrna = ctypes.create_string_buffer(self.n + 1)
        st = ctypes.create_string_buffer(self.n + 1)
        e = ctypes.c_int32()
        cc = ctypes.c_double()
        obj = ctypes.c_double()
        ofx = ctypes.c_int64()
        pfx = ctypes.c_int64()
        lib.orc_result(handle, mrna, st, ctypes.byref(e), ctypes.byref(cc), ctypes.byref(obj),
                       ctypes.byref(ofx), ctypes.byref(pfx))
        self.mrna = mrna.value.decode()
        self.structure = st.value.decode()
        self.energy = int(e.value)
        self.codon_cost = float(cc.value)
        self.objective = float(obj.value)
        self.obj_fx = int(ofx.value)
        self.path_cost_fx = int(pfx.value)
        Z = ctypes.c_int64()
        fd = ctypes.c_int64()
        rc = ctypes.c_int64()
        lib.orc_counts(handle, ctypes.byref(Z), ctypes.byref(fd), ctypes.byref(rc))
        self.Z = int(Z.value)
        self.finite_direct = int(fd.value)
        self.retained_cells = int(rc.value)


def run(param_path: str, protein: str, weights, lam: float) -> OracleDesign:
    """Exact design of one protein by the dense oracle."""
    lib = _load()
    w = np.ascontiguousarray(weights, dtype=np.float64)
    assert w.shape == (64,)
    h = ctypes.c_void_p()
    st = lib.orc_run(param_path.encode(), protein.encode(),
                     w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(lam), ctypes.byref(h))
    if not h.value:
        raise ValueError(f"oracle rejected input (code {st})")
    try:
        return OracleDesign(h, st)
    finally:
        lib.orc_free(h)


def run_motifs(param_path: str, protein: str, weights, lam: float, motifs):
    """Exact design whose mRNA contains none of the motifs (the codon DFA
    intersected with the motifs' Aho-Corasick automaton, Sec. 3); None when no
    motif-free synonymous mRNA exists."""
    lib = _load()
    w = np.ascontiguousarray(weights, dtype=np.float64)
    assert w.shape == (64,)
    h = ctypes.c_void_p()
    st = lib.orc_run_motifs(param_path.encode(), protein.encode(),
                            w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(lam),
                            ",".join(motifs).encode(), ctypes.byref(h))
    if st == -3:
        return None
    if not h.value:
        raise ValueError(f"oracle rejected input (code {st})")
    try:
        return OracleDesign(h, st)
    finally:
        lib.orc_free(h)


def run_rna(param_path: str, rna: str) -> OracleDesign:
    """MFE of a fixed RNA sequence by the same DP on a width-1 lattice."""
    lib = _load()
    h = ctypes.c_void_p()
    st = lib.orc_run_rna(param_path.encode(), rna.encode(), ctypes.byref(h))
    if not h.value:
        raise ValueError(f"oracle rejected input (code {st})")
    try:
        return OracleDesign(h, st)
    finally:
        lib.orc_free(h)


def set_threads(n: int) -> int:
    """Threads filling the layer pairs of one span (the paper's scheme of
    parallelising each span over its layer pairs); 1 by default.  Returns the
    previous setting.  Results do not depend on it."""
    return int(_load().orc_set_threads(int(n)))


def codon_cost_fx(lam: float, w: float) -> int:
    return int(_load().orc_codon_cost_fx(float(lam), float(w)))


def hairpin_energy(param_path: str, seq: str) -> int:
    return int(_load().orc_hairpin_energy(param_path.encode(), seq.encode()))


def twoloop_energy(param_path: str, left: str, right: str) -> int:
    """Two-loop energy of the oracle's loop function: left = outer 5' nt,
    l1 unpaired, inner 5' nt; right = inner 3' nt, l2 unpaired, outer 3' nt."""
    return int(_load().orc_twoloop_energy(param_path.encode(), left.encode(), right.encode()))
