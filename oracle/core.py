"""ctypes front of the C oracle (trk_oracle.c).  Test infrastructure only."""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(_build.build())
        lib.orc_run.restype = C.c_int
        lib.orc_run.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.c_void_p,
                                C.c_int32, C.c_void_p]
        lib.orc_result_free.argtypes = [C.c_void_p]
        lib.orc_fit.restype = C.c_int
        lib.orc_fit.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]
        lib.orc_fit_list.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int32,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        lib.orc_max_threads.restype = C.c_int32
        lib.orc_fit_track.restype = C.c_int
        lib.orc_fit_track.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_double,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        lib.orc_fit_tracks.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_double,
                                       C.c_double, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p]
        lib.orc_run_blocks.restype = C.c_int
        lib.orc_run_blocks.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.c_void_p,
                                       C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p]
        lib.orc_block_result_free.argtypes = [C.c_void_p]
        lib.orc_block_peaks.restype = C.c_int64
        lib.orc_block_peaks.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                        C.c_void_p, C.c_void_p, C.c_int64]
        _lib = lib
    return _lib


class _Setup(C.Structure):
    _fields_ = [("b_tesla", C.c_double), ("n_layers", C.c_int32), ("n_triples", C.c_int32),
                ("triples", C.c_void_p), ("lo", C.c_double * 5), ("hi", C.c_double * 5),
                ("n", C.c_int32 * 5), ("periodic", C.c_int32), ("eps_rel", C.c_double)]


class _Result(C.Structure):
    _fields_ = [("n_acc", C.c_int64), ("acc_event", C.c_void_p), ("acc_ijk", C.c_void_p),
                ("acc_bin", C.c_void_p), ("acc_amb", C.c_void_p), ("acc_par", C.c_void_p),
                ("n_near", C.c_int64), ("near_event", C.c_void_p), ("near_ijk", C.c_void_p),
                ("n_triplets", C.c_int64), ("n_degenerate", C.c_int64)]


class _BlockResult(C.Structure):
    _fields_ = [("n_keep", C.c_int64), ("keep_ijk", C.c_void_p), ("keep_bin", C.c_void_p),
                ("n_flip", C.c_int64), ("flip_ijk", C.c_void_p), ("flip_bin", C.c_void_p),
                ("flip_acc", C.c_void_p), ("n_triplets", C.c_int64), ("n_degenerate", C.c_int64)]


def _arr(ptr, dtype, count):
    if count == 0:
        return np.zeros(0, dtype=dtype)
    buf = (C.c_char * (count * np.dtype(dtype).itemsize)).from_address(ptr)
    return np.frombuffer(buf, dtype=dtype).copy()


@dataclass
class OracleSetup:
    """Geometry and binning as the oracle reads them (from a workload description)."""
    b_tesla: float
    n_layers: int
    triples: np.ndarray          # (T, 3) int32
    lo: np.ndarray               # (5,) float64
    hi: np.ndarray
    n: np.ndarray                # (5,) int64
    periodic: np.ndarray         # (5,) bool
    threshold: int
    eps_rel: float = 1e-5

    @classmethod
    def from_workload(cls, cfg: dict, **over) -> "OracleSetup":
        g, b = cfg["geometry"], cfg["binning"]
        kw = dict(b_tesla=float(g["b_tesla"]), n_layers=len(g["radius"]),
                  triples=np.asarray(g["triples"], dtype=np.int32).reshape(-1, 3),
                  lo=np.asarray(b["lo"], dtype=np.float64), hi=np.asarray(b["hi"], dtype=np.float64),
                  n=np.asarray(b["n"], dtype=np.int64), periodic=np.asarray(b["periodic"], dtype=bool),
                  threshold=int(b["threshold"]))
        kw.update(over)
        return cls(**kw)

    @property
    def n_bins(self) -> int:
        return int(np.prod(self.n))

    def _c(self):
        tri = np.ascontiguousarray(self.triples, dtype=np.int32)
        s = _Setup()
        s.b_tesla = self.b_tesla
        s.n_layers = self.n_layers
        s.n_triples = len(tri)
        s.triples = tri.ctypes.data
        for k in range(5):
            s.lo[k] = float(self.lo[k])
            s.hi[k] = float(self.hi[k])
            s.n[k] = int(self.n[k])
        s.periodic = int(sum(1 << k for k in range(5) if self.periodic[k]))
        s.eps_rel = self.eps_rel
        return s, tri


def _hits_struct(xyz: np.ndarray, layer: np.ndarray) -> np.ndarray:
    h = np.empty((len(xyz), 4), dtype=np.float32)
    h[:, :3] = np.asarray(xyz, dtype=np.float32)
    h[:, 3] = np.asarray(layer, dtype=np.int32).view(np.float32)
    return np.ascontiguousarray(h)


def max_threads() -> int:
    return int(_load().orc_max_threads())


def enumerate_batch(xyz, layer, offsets, setup: OracleSetup, n_threads: int = 0) -> dict:
    """Every triplet of the definition; accepted ones with bins, ambiguity, parameters."""
    lib = _load()
    hits = _hits_struct(xyz, layer)
    offs = np.ascontiguousarray(offsets, dtype=np.int64)
    s, tri = setup._c()
    res = _Result()
    rc = lib.orc_run(hits.ctypes.data, C.c_int64(len(hits)), offs.ctypes.data,
                     C.c_int32(len(offs) - 1), C.byref(s), C.c_int32(n_threads), C.byref(res))
    if rc != 0:
        raise ValueError("oracle: invalid input (layer id out of range or bad offsets)")
    try:
        na, nn = res.n_acc, res.n_near

        def arr(ptr, dtype, count):
            if count == 0:
                return np.zeros(0, dtype=dtype)
            buf = (C.c_char * (count * np.dtype(dtype).itemsize)).from_address(ptr)
            return np.frombuffer(buf, dtype=dtype).copy()
        out = dict(
            event=arr(res.acc_event, np.int32, na),
            ijk=arr(res.acc_ijk, np.int32, 3 * na).reshape(-1, 3),
            bin=arr(res.acc_bin, np.uint64, na).astype(np.int64),
            amb=arr(res.acc_amb, np.uint8, na).astype(bool),
            amb_bits=arr(res.acc_amb, np.uint8, na),
            par=arr(res.acc_par, np.float64, 5 * na).reshape(-1, 5),
            near_event=arr(res.near_event, np.int32, nn),
            near_ijk=arr(res.near_ijk, np.int32, 3 * nn).reshape(-1, 3),
            n_triplets=int(res.n_triplets),
            n_degenerate=int(res.n_degenerate),
            n_events=len(offs) - 1,
        )
    finally:
        lib.orc_result_free(C.byref(res))
    return out


def fit_list(xyz, layer, ijk, setup: OracleSetup, n_threads: int = 0) -> dict:
    """Fit and bin explicit triplets (global input hit indices)."""
    lib = _load()
    hits = _hits_struct(xyz, layer)
    ijk = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
    n = len(ijk)
    par = np.zeros((n, 5), dtype=np.float64)
    binv = np.zeros(n, dtype=np.uint64)
    status = np.zeros(n, dtype=np.int32)
    amb = np.zeros(n, dtype=np.uint8)
    s, tri = setup._c()
    lib.orc_fit_list(hits.ctypes.data, ijk.ctypes.data, C.c_int64(n), C.byref(s),
                     C.c_int32(n_threads), par.ctypes.data, binv.ctypes.data,
                     status.ctypes.data, amb.ctypes.data)
    return dict(par=par, bin=binv.astype(np.int64), status=status, amb=amb.astype(bool),
                amb_bits=amb)


def fit_one(p1, p2, p3, b_tesla: float):
    """Helix parameters of one triplet (FP64), or None if degenerate."""
    lib = _load()
    a = np.ascontiguousarray(p1, dtype=np.float64)
    b = np.ascontiguousarray(p2, dtype=np.float64)
    c = np.ascontiguousarray(p3, dtype=np.float64)
    par = np.zeros(5, dtype=np.float64)
    rc = lib.orc_fit(a.ctypes.data, b.ctypes.data, c.ctypes.data, C.c_double(b_tesla),
                     par.ctypes.data)
    return None if rc != 0 else par


def fit_tracks(xyz, layer, hit_lists, b_tesla: float, eps_rel: float = 1e-5,
               n_threads: int = 0) -> dict:
    """Candidate fits (trk_oracle.c, orc_fit_track) of the given hit lists (each a sequence
    of global input hit indices, in the order the fit reads them)."""
    lib = _load()
    hits = _hits_struct(xyz, layer)
    off = np.zeros(len(hit_lists) + 1, dtype=np.int64)
    for t, h in enumerate(hit_lists):
        off[t + 1] = off[t] + len(h)
    ids = (np.concatenate([np.asarray(h, dtype=np.int64) for h in hit_lists])
           if len(hit_lists) and off[-1] else np.zeros(0, dtype=np.int64))
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    n = len(hit_lists)
    use = np.zeros(max(int(off[-1]), 1), dtype=np.uint8)
    par = np.zeros((n, 5), dtype=np.float64)
    chi2 = np.zeros((n, 2), dtype=np.float64)
    status = np.zeros(n, dtype=np.int32)
    amb = np.zeros(n, dtype=np.int32)
    lib.orc_fit_tracks(hits.ctypes.data, ids.ctypes.data, off.ctypes.data, C.c_int64(n),
                       C.c_double(b_tesla), C.c_double(eps_rel), C.c_int32(n_threads),
                       use.ctypes.data, par.ctypes.data, chi2.ctypes.data, status.ctypes.data,
                       amb.ctypes.data)
    return dict(par=par, chi2=chi2, status=status, amb=amb,
                use=[use[off[t]:off[t + 1]].astype(bool) for t in range(n)])


def fit_track_points(xyz, layer, b_tesla: float, eps_rel: float = 1e-5) -> dict:
    """The candidate fit of one hit list given as double-precision points (pins)."""
    lib = _load()
    pts = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    lay = np.ascontiguousarray(layer, dtype=np.int32)
    n = len(pts)
    use = np.zeros(max(n, 1), dtype=np.uint8)
    par = np.zeros(5, dtype=np.float64)
    chi2 = np.zeros(2, dtype=np.float64)
    amb = np.zeros(1, dtype=np.int32)
    st = lib.orc_fit_track(pts.ctypes.data, lay.ctypes.data, n, C.c_double(b_tesla),
                           C.c_double(eps_rel), use.ctypes.data, par.ctypes.data,
                           chi2.ctypes.data, amb.ctypes.data)
    return dict(status=int(st), par=par, chi2=chi2, amb=int(amb[0]), use=use[:n].astype(bool))


def enumerate_blocks(xyz, layer, setup: OracleSetup, count_blocks, keep_blocks, flip_blocks,
                     n_threads: int = 0) -> dict:
    """The definition over every triplet of ONE event, keeping only part of the output
    (trk_oracle.c, orc_run_blocks).  A block is a (phi0 row, q/pT row) pair of bin indices.
    count_blocks: list of (i0, i1) whose bins are counted (dense); keep_blocks: blocks whose
    accepted triplets are listed; flip_blocks: blocks whose edge-ambiguous accepted triplets
    are listed (near-accepted and antipode-ambiguous triplets are listed wherever they fall).
    """
    lib = _load()
    hits = _hits_struct(xyz, layer)
    n0, n1 = int(setup.n[0]), int(setup.n[1])
    inner = int(setup.n[2] * setup.n[3] * setup.n[4])
    slot = -np.ones(n0 * n1, dtype=np.int32)
    for q, (i0, i1) in enumerate(count_blocks):
        slot[i0 * n1 + i1] = q
    keep = np.zeros(n0 * n1, dtype=np.uint8)
    for i0, i1 in keep_blocks:
        keep[i0 * n1 + i1] = 1
    flip = np.zeros(n0 * n1, dtype=np.uint8)
    for i0, i1 in flip_blocks:
        flip[i0 * n1 + i1] = 1
    counts = np.zeros(max(len(count_blocks), 1) * inner, dtype=np.int32)
    offs = np.array([0, len(hits)], dtype=np.int64)
    s, tri = setup._c()
    res = _BlockResult()
    rc = lib.orc_run_blocks(hits.ctypes.data, C.c_int64(len(hits)), offs.ctypes.data, 1,
                            C.byref(s), C.c_int32(n_threads), slot.ctypes.data, keep.ctypes.data,
                            flip.ctypes.data, counts.ctypes.data, C.byref(res))
    if rc != 0:
        raise ValueError("oracle: invalid input")
    try:
        out = dict(slot=slot, counts=counts.reshape(max(len(count_blocks), 1), inner),
                   keep_ijk=_arr(res.keep_ijk, np.int32, 3 * res.n_keep).reshape(-1, 3),
                   keep_bin=_arr(res.keep_bin, np.uint64, res.n_keep).astype(np.int64),
                   flip_ijk=_arr(res.flip_ijk, np.int32, 3 * res.n_flip).reshape(-1, 3),
                   flip_bin=_arr(res.flip_bin, np.uint64, res.n_flip).astype(np.int64),
                   flip_acc=_arr(res.flip_acc, np.uint8, res.n_flip).astype(bool),
                   n_triplets=int(res.n_triplets), n_degenerate=int(res.n_degenerate))
    finally:
        lib.orc_block_result_free(C.byref(res))
    return out


def block_peaks(blocks: dict, setup: OracleSetup, keep_blocks) -> tuple:
    """Candidates (bins, votes) of the keep blocks from enumerate_blocks' counts, by the peak
    rule in plain C (trk_oracle.c, orc_block_peaks)."""
    lib = _load()
    n0, n1 = int(setup.n[0]), int(setup.n[1])
    keep = np.zeros(n0 * n1, dtype=np.uint8)
    for i0, i1 in keep_blocks:
        keep[i0 * n1 + i1] = 1
    counts = np.ascontiguousarray(blocks["counts"], dtype=np.int32)
    cap = int(len(keep_blocks) * counts.shape[1])
    bins = np.zeros(max(cap, 1), dtype=np.uint64)
    votes = np.zeros(max(cap, 1), dtype=np.int32)
    s, tri = setup._c()
    n = lib.orc_block_peaks(C.byref(s), blocks["slot"].ctypes.data, counts.ctypes.data,
                            keep.ctypes.data, C.c_int32(setup.threshold), bins.ctypes.data,
                            votes.ctypes.data, C.c_int64(cap))
    if n < 0:
        raise ValueError("oracle: a neighbour block of a keep block is not counted")
    return bins[:n].astype(np.int64), votes[:n].astype(np.int64)
