"""B300-native exact codon-lattice design (SparseDesign, arXiv 2609.32308).

Thin ctypes binding of libsd_b300.so (C ABI in include/sd.h): argument
marshalling only.  Every step of the design -- the span wavefront fill, the
exterior pass and the traceback -- runs in the library's CUDA kernels; there
is no CPU fallback.  If the shared library is missing or cannot be loaded the
calls raise, they never compute anything on the host.

Names follow the C ABI: sd_load_energy, sd_design, sd_design_batch,
sd_plan_create / sd_plan_run / sd_plan_results / sd_plan_dump / sd_plan_free.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsd_b300.so")
_lib = None

SD_OK, SD_EINVAL, SD_ERANGE, SD_EINFEASIBLE = 0, -1, -2, -3
SD_ENOMEM, SD_ECUDA, SD_ETIMEOUT, SD_EINTERNAL, SD_ESIZE = -4, -5, -6, -7, -8
SD_LAYOUT_SPAN, SD_LAYOUT_SQUARE, SD_LAYOUT_PACKED = 0, 1, 2
SD_GROUP_BY_SPAN = 0  # fill group chosen per span (sd_plan_set_group)
INF = 1 << 62          # +infinity in table dumps
FX_ONE = 1 << 32       # one dcal/mol in the fixed-point unit


class SdError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {sd_strerror(code)} ({code})" if what else sd_strerror(code))


class sd_result(ctypes.Structure):
    _fields_ = [
        ("mrna", ctypes.c_void_p), ("structure", ctypes.c_void_p),
        ("energy", ctypes.c_int32), ("n", ctypes.c_int32),
        ("codon_cost", ctypes.c_double), ("objective", ctypes.c_double),
        ("objective_fx", ctypes.c_int64), ("Z", ctypes.c_int64),
        ("finite_direct", ctypes.c_int64), ("retained_cells", ctypes.c_int64),
        ("states", ctypes.c_int64), ("edges", ctypes.c_int64),
        ("regrows", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


def lib():
    """Load libsd_b300.so (raises if it is absent: no host fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing; build it with "
                              "`python -m paper_2609_32308_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.sd_load_energy.argtypes = [ctypes.c_char_p, ctypes.c_uint64, ctypes.POINTER(P)]
        L.sd_energy_save.argtypes = [P, ctypes.c_char_p]
        L.sd_energy_save.restype = I
        L.sd_energy_free.argtypes = [P]
        L.sd_energy_free.restype = None
        L.sd_design.argtypes = [P, ctypes.c_char_p, P, D, ctypes.POINTER(sd_result)]
        L.sd_design_batch.argtypes = [P, I, P, P, I, P, P, P]
        L.sd_design_noalloc.argtypes = [P, ctypes.c_char_p, P, D, ctypes.POINTER(sd_result)]
        L.sd_result_free.argtypes = [ctypes.POINTER(sd_result)]
        L.sd_result_free.restype = None
        L.sd_strerror.argtypes = [I]
        L.sd_strerror.restype = ctypes.c_char_p
        L.sd_plan_create.argtypes = [P, I, P, P, I, P, ctypes.POINTER(P), P]
        L.sd_plan_create_layout.argtypes = [P, I, P, P, I, P, I, ctypes.POINTER(P), P]
        L.sd_plan_create_motifs.argtypes = [P, I, P, P, I, P, P, I, ctypes.POINTER(P), P]
        L.sd_design_motifs.argtypes = [P, ctypes.c_char_p, P, D, P, I, ctypes.POINTER(sd_result)]
        L.sd_plan_run.argtypes = [P, P]
        L.sd_plan_launches.argtypes = [P]
        L.sd_plan_launches.restype = ctypes.c_int64
        L.sd_plan_device_bytes.argtypes = [P]
        L.sd_plan_device_bytes.restype = ctypes.c_int64
        L.sd_plan_results.argtypes = [P, P, P]
        L.sd_plan_item_size.argtypes = [P, I, P, P, P]
        L.sd_plan_dump.argtypes = [P, I] + [P] * 8
        L.sd_plan_edges.argtypes = [P, I, P, P, P, P]
        L.sd_plan_set_timing.argtypes = [P, I]
        L.sd_plan_count_ops.argtypes = [P, P]
        L.sd_plan_set_group.argtypes = [P, I]
        L.sd_plan_set_graph.argtypes = [P, I]
        L.sd_plan_set_streams.argtypes = [P, I]
        L.sd_design_sweep.argtypes = [P, ctypes.c_char_p, P, I, P, P, P]
        L.sd_envelope.argtypes = [P, ctypes.c_char_p, P, D, D, I, P, P, ctypes.POINTER(I)]
        L.sd_inverse_lambda.argtypes = [P, ctypes.c_char_p, P, D, D, ctypes.POINTER(D),
                                        ctypes.POINTER(sd_result)]
        L.sd_plan_get_streams.argtypes = [P]
        L.sd_peak_addmin.argtypes = [I, I, ctypes.POINTER(D)]
        L.sd_plan_retention.argtypes = [P, I, P]
        L.sd_plan_candidate_room.argtypes = [P]
        L.sd_plan_candidate_room.restype = ctypes.c_int64
        L.sd_plan_set_dense.argtypes = [P, I]
        L.sd_plan_candidate_room_worst.argtypes = [P]
        L.sd_plan_candidate_room_worst.restype = ctypes.c_int64
        L.sd_plan_create_predicted.argtypes = [P, P, D, I, P, P, I, P, ctypes.POINTER(P), P]
        L.sd_pred_create.argtypes = [ctypes.c_uint64, ctypes.POINTER(P)]
        L.sd_pred_free.argtypes = [P]
        L.sd_pred_free.restype = None
        L.sd_pred_num_params.argtypes = []
        L.sd_pred_num_params.restype = ctypes.c_int64
        L.sd_pred_get_params.argtypes = [P, P]
        L.sd_pred_set_params.argtypes = [P, P]
        L.sd_pred_features.argtypes = [ctypes.c_char_p, P, D, P]
        L.sd_pred_forward.argtypes = [P, I, I, P, P, P]
        L.sd_pred_gradients.argtypes = [P, I, I, P, P, P, P, P]
        L.sd_pred_train_step.argtypes = [P, I, I, P, P, P, ctypes.c_float, P]
        L.sd_plan_get_group.argtypes = [P]
        L.sd_plan_autotune.argtypes = [P, P]
        L.sd_plan_phase_times.argtypes = [P, P]
        L.sd_plan_free.argtypes = [P]
        L.sd_plan_free.restype = None
        for f in ("sd_load_energy", "sd_design", "sd_design_batch", "sd_design_noalloc",
                  "sd_plan_create",
                  "sd_plan_run", "sd_plan_results", "sd_plan_item_size", "sd_plan_dump",
                  "sd_plan_edges", "sd_plan_set_timing", "sd_plan_phase_times",
                  "sd_plan_count_ops", "sd_plan_set_group", "sd_plan_get_group",
                  "sd_plan_autotune", "sd_plan_set_graph", "sd_plan_retention", "sd_plan_set_dense",
                  "sd_plan_set_streams", "sd_plan_get_streams", "sd_peak_addmin",
                  "sd_design_sweep", "sd_envelope", "sd_inverse_lambda", "sd_plan_create_layout",
                  "sd_plan_create_motifs", "sd_design_motifs",
                  "sd_plan_create_predicted", "sd_pred_create", "sd_pred_get_params",
                  "sd_pred_set_params", "sd_pred_features", "sd_pred_forward",
                  "sd_pred_gradients", "sd_pred_train_step"):
            getattr(L, f).restype = I
        _lib = L
    return _lib


def sd_strerror(code: int) -> str:
    try:
        return lib().sd_strerror(int(code)).decode()
    except ImportError:
        return f"error {code}"


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


class Energy:
    """Loaded parameter set (host + device copy); frees itself.  path: a
    parameter file, or None for the library's seeded synthetic set `seed`."""

    def __init__(self, path: str | None = None, seed: int = 0):
        h = ctypes.c_void_p()
        rc = lib().sd_load_energy(None if path is None else str(path).encode(), int(seed),
                                  ctypes.byref(h))
        if rc != SD_OK:
            raise SdError(rc, f"sd_load_energy({path}, {seed})")
        self.handle = h

    def save(self, path: str) -> None:
        """Write the parameter set in the text format (sd_energy_save)."""
        rc = lib().sd_energy_save(self.handle, str(path).encode())
        if rc != SD_OK:
            raise SdError(rc, "sd_energy_save")

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.sd_energy_free(self.handle)
            self.handle = None


def sd_load_energy(path: str | None = None, seed: int = 0) -> Energy:
    """A parameter file, or (path None) the library's seeded synthetic set."""
    return Energy(path, seed)


def _result_dict(r: sd_result, status: int) -> dict:
    out = {"status": int(status)}
    if status == SD_OK:
        out.update(
            mrna=ctypes.string_at(r.mrna).decode(),
            structure=ctypes.string_at(r.structure).decode(),
            energy=int(r.energy), n=int(r.n), codon_cost=float(r.codon_cost),
            objective=float(r.objective), objective_fx=int(r.objective_fx), Z=int(r.Z),
            finite_direct=int(r.finite_direct), retained_cells=int(r.retained_cells),
            states=int(r.states), edges=int(r.edges), regrows=int(r.regrows))
    return out


def _weights(weights, count):
    w = np.ascontiguousarray(weights, dtype=np.float64)
    if w.shape == (64,):
        return w, 1
    w = w.reshape(count, 64)
    return np.ascontiguousarray(w), 0


def sd_design(energy: Energy, protein: str, weights, lam: float) -> dict:
    """One exact design; raises SdError on failure."""
    w = np.ascontiguousarray(weights, dtype=np.float64).reshape(64)
    r = sd_result()
    rc = lib().sd_design(energy.handle, protein.encode(), _ptr(w), float(lam), ctypes.byref(r))
    try:
        if rc != SD_OK:
            raise SdError(rc, "sd_design")
        return _result_dict(r, rc)
    finally:
        lib().sd_result_free(ctypes.byref(r))


def sd_design_noalloc(energy: Energy, protein: str, weights, lam: float) -> dict:
    """One exact design through the entry point that allocates no device
    memory (for callers that may not call cudaMalloc; see include/sd.h).
    The output strings live in buffers made here, on the host."""
    w = np.ascontiguousarray(weights, dtype=np.float64).reshape(64)
    n = 3 * len(protein)
    mbuf = ctypes.create_string_buffer(n + 1)
    sbuf = ctypes.create_string_buffer(n + 1)
    r = sd_result()
    r.mrna = ctypes.cast(mbuf, ctypes.c_void_p)
    r.structure = ctypes.cast(sbuf, ctypes.c_void_p)
    rc = lib().sd_design_noalloc(energy.handle, protein.encode(), _ptr(w), float(lam),
                                 ctypes.byref(r))
    if rc != SD_OK:
        raise SdError(rc, "sd_design_noalloc")
    return _result_dict(r, rc)


def sd_design_batch(energy: Energy, proteins, weights, lambdas) -> list:
    """Designs of many proteins; per-item dicts carry their own status."""
    count = len(proteins)
    w, shared = _weights(weights, count)
    lam = np.ascontiguousarray(lambdas, dtype=np.float64).reshape(count)
    enc = [p.encode() for p in proteins]
    arr = (ctypes.c_char_p * count)(*enc)
    outs = (sd_result * count)()
    st = np.zeros(count, dtype=np.int32)
    rc = lib().sd_design_batch(energy.handle, count, arr, _ptr(w), shared, _ptr(lam), outs,
                               _ptr(st))
    try:
        if rc != SD_OK:
            raise SdError(rc, "sd_design_batch")
        return [_result_dict(outs[k], int(st[k])) for k in range(count)]
    finally:
        for k in range(count):
            lib().sd_result_free(ctypes.byref(outs[k]))


def sd_design_motifs(energy: Energy, protein: str, weights, lam: float, motifs) -> dict:
    """One exact design whose mRNA contains none of the motifs."""
    w = np.ascontiguousarray(weights, dtype=np.float64).reshape(64)
    enc = [m.encode() for m in motifs]
    marr = (ctypes.c_char_p * max(1, len(enc)))(*enc)
    r = sd_result()
    rc = lib().sd_design_motifs(energy.handle, protein.encode(), _ptr(w), float(lam), marr,
                                len(enc), ctypes.byref(r))
    try:
        if rc != SD_OK:
            raise SdError(rc, "sd_design_motifs")
        return _result_dict(r, rc)
    finally:
        lib().sd_result_free(ctypes.byref(r))


def sd_design_sweep(energy: Energy, protein: str, weights, lambdas) -> list:
    """Designs of one protein at several lambdas, one batched launch sequence."""
    k = len(lambdas)
    w = np.ascontiguousarray(weights, dtype=np.float64).reshape(64)
    lam = np.ascontiguousarray(lambdas, dtype=np.float64).reshape(k)
    outs = (sd_result * max(k, 1))()
    st = np.zeros(max(k, 1), dtype=np.int32)
    rc = lib().sd_design_sweep(energy.handle, protein.encode(), _ptr(w), k, _ptr(lam), outs,
                               _ptr(st))
    try:
        if rc != SD_OK:
            raise SdError(rc, "sd_design_sweep")
        return [_result_dict(outs[q], int(st[q])) for q in range(k)]
    finally:
        for q in range(k):
            lib().sd_result_free(ctypes.byref(outs[q]))


def sd_envelope(energy: Energy, protein: str, weights, lam_lo: float, lam_hi: float,
                max_lines: int = 256):
    """Supported lines of the lower envelope of F*(lambda) on [lam_lo, lam_hi]:
    (list of design dicts in increasing lambda, list of breakpoints)."""
    w = np.ascontiguousarray(weights, dtype=np.float64).reshape(64)
    lines = (sd_result * max_lines)()
    brk = np.zeros(max_lines, dtype=np.float64)
    cnt = ctypes.c_int()
    rc = lib().sd_envelope(energy.handle, protein.encode(), _ptr(w), float(lam_lo),
                           float(lam_hi), int(max_lines), lines, _ptr(brk), ctypes.byref(cnt))
    try:
        if rc != SD_OK:
            raise SdError(rc, "sd_envelope")
        n = int(cnt.value)
        return [_result_dict(lines[q], SD_OK) for q in range(n)], [float(x) for x in brk[:n - 1]]
    finally:
        for q in range(int(cnt.value)):
            lib().sd_result_free(ctypes.byref(lines[q]))


def sd_inverse_lambda(energy: Energy, protein: str, weights, target_codon_cost: float,
                      lam_hi: float):
    """Smallest lambda in [0, lam_hi] whose design has C(r) <= target; (lambda, design)."""
    w = np.ascontiguousarray(weights, dtype=np.float64).reshape(64)
    lam = ctypes.c_double()
    r = sd_result()
    rc = lib().sd_inverse_lambda(energy.handle, protein.encode(), _ptr(w),
                                 float(target_codon_cost), float(lam_hi), ctypes.byref(lam),
                                 ctypes.byref(r))
    try:
        if rc != SD_OK:
            raise SdError(rc, "sd_inverse_lambda")
        return float(lam.value), _result_dict(r, SD_OK)
    finally:
        lib().sd_result_free(ctypes.byref(r))


class Plan:
    """A batch of designs resident on the GPU (sd_plan_* calls)."""

    def __init__(self, energy: Energy, proteins, weights, lambdas, predictor=None,
                 margin: float = 2.0, layout: int = SD_LAYOUT_SPAN, motifs=None):
        """predictor: a Predictor to presize the candidate lists
        (sd_plan_create_predicted), or None for worst-case room.  layout: the
        layout of the full tables (sd_plan_create_layout; worst-case room)."""
        self.energy = energy
        self.count = len(proteins)
        w, shared = _weights(weights, self.count)
        lam = np.ascontiguousarray(lambdas, dtype=np.float64).reshape(self.count)
        self._keep = [p.encode() for p in proteins]
        arr = (ctypes.c_char_p * self.count)(*self._keep)
        self.item_status = np.zeros(self.count, dtype=np.int32)
        h = ctypes.c_void_p()
        if motifs is not None:
            if predictor is not None or layout != SD_LAYOUT_SPAN:
                raise ValueError("motif plans take worst-case room and their own layout")
            self._motifs = [m.encode() for m in motifs]
            marr = (ctypes.c_char_p * max(1, len(motifs)))(*self._motifs)
            rc = lib().sd_plan_create_motifs(energy.handle, self.count, arr, _ptr(w), shared,
                                             _ptr(lam), marr, len(motifs), ctypes.byref(h),
                                             _ptr(self.item_status))
        elif layout != SD_LAYOUT_SPAN:
            if predictor is not None:
                raise ValueError("a layout other than the default takes worst-case room")
            rc = lib().sd_plan_create_layout(energy.handle, self.count, arr, _ptr(w), shared,
                                             _ptr(lam), int(layout), ctypes.byref(h),
                                             _ptr(self.item_status))
        elif predictor is None:
            rc = lib().sd_plan_create(energy.handle, self.count, arr, _ptr(w), shared, _ptr(lam),
                                      ctypes.byref(h), _ptr(self.item_status))
        else:
            rc = lib().sd_plan_create_predicted(energy.handle, predictor.handle, float(margin),
                                                self.count, arr, _ptr(w), shared, _ptr(lam),
                                                ctypes.byref(h), _ptr(self.item_status))
        if rc != SD_OK:
            raise SdError(rc, "sd_plan_create")
        self.handle = h

    def run(self, stream=None):
        """Enqueue the whole design on `stream` (an int cudaStream_t, a torch
        stream, or None for the legacy default stream)."""
        s = getattr(stream, "cuda_stream", stream)
        rc = lib().sd_plan_run(self.handle, ctypes.c_void_p(s) if s else None)
        if rc != SD_OK:
            raise SdError(rc, "sd_plan_run")

    def set_timing(self, enable: bool = True):
        rc = lib().sd_plan_set_timing(self.handle, int(bool(enable)))
        if rc != SD_OK:
            raise SdError(rc, "sd_plan_set_timing")

    @property
    def group(self) -> int:
        return int(lib().sd_plan_get_group(self.handle))

    @group.setter
    def group(self, g: int):
        rc = lib().sd_plan_set_group(self.handle, int(g))
        if rc != SD_OK:
            raise SdError(rc, "sd_plan_set_group")

    def set_graph(self, enable: bool = True):
        """Replay the whole run as one CUDA graph (captured on the next run)."""
        rc = lib().sd_plan_set_graph(self.handle, int(bool(enable)))
        if rc != SD_OK:
            raise SdError(rc, "sd_plan_set_graph")

    @property
    def streams(self) -> int:
        return int(lib().sd_plan_get_streams(self.handle))

    @streams.setter
    def streams(self, k: int):
        """Split the designs over k concurrent streams, LPT by predicted work."""
        rc = lib().sd_plan_set_streams(self.handle, int(k))
        if rc != SD_OK:
            raise SdError(rc, "sd_plan_set_streams")

    def autotune(self):
        """Pick the fastest group choice (SD_GROUP_BY_SPAN, 8, 16 or 32 threads
        per layer pair); returns {group: fill ms}."""
        ms = np.zeros(4, dtype=np.float32)
        rc = lib().sd_plan_autotune(self.handle, _ptr(ms))
        if rc != SD_OK:
            raise SdError(rc, "sd_plan_autotune")
        return dict(zip((SD_GROUP_BY_SPAN, 8, 16, 32), (float(x) for x in ms)))

    def count_ops(self):
        """Algorithmic INT32 slots of the fill, per item (counting variant)."""
        ops = np.zeros(self.count, dtype=np.int64)
        rc = lib().sd_plan_count_ops(self.handle, _ptr(ops))
        if rc != SD_OK:
            raise SdError(rc, "sd_plan_count_ops")
        return ops

    def phase_times(self):
        """(fill, exterior, traceback) milliseconds of the last timed run."""
        ms = np.zeros(3, dtype=np.float32)
        rc = lib().sd_plan_phase_times(self.handle, _ptr(ms))
        if rc != SD_OK:
            raise SdError(rc, "sd_plan_phase_times")
        return tuple(float(x) for x in ms)

    @property
    def launches(self) -> int:
        return int(lib().sd_plan_launches(self.handle))

    @property
    def device_bytes(self) -> int:
        return int(lib().sd_plan_device_bytes(self.handle))

    def results(self) -> list:
        outs = (sd_result * self.count)()
        st = np.zeros(self.count, dtype=np.int32)
        rc = lib().sd_plan_results(self.handle, outs, _ptr(st))
        try:
            if rc != SD_OK:
                raise SdError(rc, "sd_plan_results")
            return [_result_dict(outs[k], int(st[k])) for k in range(self.count)]
        finally:
            for k in range(self.count):
                lib().sd_result_free(ctypes.byref(outs[k]))

    def retention(self, item: int) -> np.ndarray:
        """Retained candidates of one item by (codon, span band), shape (A, 8)."""
        A = len(self._keep[item]) if item < len(self._keep) else 0
        out = np.zeros((max(A, 1), 8), dtype=np.int32)
        rc = lib().sd_plan_retention(self.handle, item, _ptr(out))
        if rc != SD_OK:
            raise SdError(rc, "sd_plan_retention")
        return out[:A]

    @property
    def candidate_room(self) -> int:
        return int(lib().sd_plan_candidate_room(self.handle))

    def set_dense(self, enable: bool) -> None:
        """Scalar-dense control: retain every finite direct interval."""
        rc = lib().sd_plan_set_dense(self.handle, int(bool(enable)))
        if rc != SD_OK:
            raise SdError(rc, "sd_plan_set_dense")

    @property
    def candidate_room_worst(self) -> int:
        return int(lib().sd_plan_candidate_room_worst(self.handle))

    def size(self, item: int):
        n, N, E = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        rc = lib().sd_plan_item_size(self.handle, item, ctypes.byref(n), ctypes.byref(N),
                                     ctypes.byref(E))
        return int(n.value), int(N.value), int(E.value), rc

    def edges(self, item: int) -> dict:
        _, _, E, _ = self.size(item)
        f, t, l = (np.zeros(E, dtype=np.int32) for _ in range(3))
        c = np.zeros(E, dtype=np.int64)
        rc = lib().sd_plan_edges(self.handle, item, _ptr(f), _ptr(t), _ptr(l), _ptr(c))
        if rc != SD_OK:
            raise SdError(rc, "sd_plan_edges")
        return {"from": f, "to": t, "label": l, "cost": c}

    def dump(self, item: int) -> dict:
        """Dense square-layout copies of one item's tables (tests only)."""
        n, N, E, st = self.size(item)
        if st != SD_OK:
            raise SdError(st, "sd_plan_dump")
        out = {"layer": np.zeros(N, dtype=np.int32),
               "H": np.zeros((N, N), dtype=np.int64), "V": np.zeros((N, N, 6), dtype=np.int64),
               "B": np.zeros((N, N), dtype=np.int64), "S1": np.zeros((N, N), dtype=np.int64),
               "S2": np.zeros((N, N), dtype=np.int64), "Ext": np.zeros(N, dtype=np.int64),
               "cand": np.zeros((N, N), dtype=np.uint8)}
        rc = lib().sd_plan_dump(self.handle, item, *[_ptr(out[k]) for k in
                                                     ("layer", "H", "V", "B", "S1", "S2", "Ext",
                                                      "cand")])
        if rc != SD_OK:
            raise SdError(rc, "sd_plan_dump")
        return out

    def free(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.sd_plan_free(self.handle)
            self.handle = None

    def __del__(self):
        self.free()


def sd_plan_create(energy, proteins, weights, lambdas) -> Plan:
    return Plan(energy, proteins, weights, lambdas)


class Predictor:
    """Retention-count predictor (sd_pred_*): a 1-D conv net whose forward,
    backward and Adam steps run in the library's BF16/FP32 kernels."""

    def __init__(self, seed: int = 0):
        h = ctypes.c_void_p()
        rc = lib().sd_pred_create(int(seed), ctypes.byref(h))
        if rc != SD_OK:
            raise SdError(rc, "sd_pred_create")
        self.handle = h
        self.nparams = int(lib().sd_pred_num_params())

    def params(self) -> np.ndarray:
        out = np.zeros(self.nparams, dtype=np.float32)
        rc = lib().sd_pred_get_params(self.handle, _ptr(out))
        if rc != SD_OK:
            raise SdError(rc, "sd_pred_get_params")
        return out

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(p, dtype=np.float32).reshape(self.nparams)
        rc = lib().sd_pred_set_params(self.handle, _ptr(p))
        if rc != SD_OK:
            raise SdError(rc, "sd_pred_set_params")

    @staticmethod
    def features(protein: str, weights, lam: float) -> np.ndarray:
        w = np.ascontiguousarray(weights, dtype=np.float64).reshape(64)
        out = np.zeros((max(len(protein), 1), 32), dtype=np.float32)
        rc = lib().sd_pred_features(protein.encode(), _ptr(w), float(lam), _ptr(out))
        if rc != SD_OK:
            raise SdError(rc, "sd_pred_features")
        return out[:len(protein)]

    def forward(self, feats: np.ndarray, lengths) -> np.ndarray:
        f = np.ascontiguousarray(feats, dtype=np.float32)
        B, L, _ = f.shape
        ln = np.ascontiguousarray(lengths, dtype=np.int32)
        out = np.zeros((B, L, 8), dtype=np.float32)
        rc = lib().sd_pred_forward(self.handle, B, L, _ptr(f), _ptr(ln), _ptr(out))
        if rc != SD_OK:
            raise SdError(rc, "sd_pred_forward")
        return out

    def gradients(self, feats, targets, lengths):
        f = np.ascontiguousarray(feats, dtype=np.float32)
        t = np.ascontiguousarray(targets, dtype=np.float32)
        B, L, _ = f.shape
        ln = np.ascontiguousarray(lengths, dtype=np.int32)
        g = np.zeros(self.nparams, dtype=np.float32)
        loss = ctypes.c_float()
        rc = lib().sd_pred_gradients(self.handle, B, L, _ptr(f), _ptr(t), _ptr(ln), _ptr(g),
                                     ctypes.byref(loss))
        if rc != SD_OK:
            raise SdError(rc, "sd_pred_gradients")
        return float(loss.value), g

    def train_step(self, feats, targets, lengths, lr: float) -> float:
        f = np.ascontiguousarray(feats, dtype=np.float32)
        t = np.ascontiguousarray(targets, dtype=np.float32)
        B, L, _ = f.shape
        ln = np.ascontiguousarray(lengths, dtype=np.int32)
        loss = ctypes.c_float()
        rc = lib().sd_pred_train_step(self.handle, B, L, _ptr(f), _ptr(t), _ptr(ln),
                                      float(lr), ctypes.byref(loss))
        if rc != SD_OK:
            raise SdError(rc, "sd_pred_train_step")
        return float(loss.value)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.sd_pred_free(self.handle)
            self.handle = None

