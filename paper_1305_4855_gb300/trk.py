"""Python binding of libtrk (include/trk.h): argument marshalling only.

Every step of the reconstruction runs in the library's CUDA kernels; this module mirrors
the C structs with ctypes, passes torch tensors by pointer and wraps the library-owned
device outputs as zero-copy torch tensors.  There is no CPU fallback: if the compiled
library is missing, importing the binding fails with an error.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libtrk.so")

TRK_MAX_LAYERS = 64
TRK_MAX_TRIPLES = 512
TRK_OK, TRK_ERR_INVALID, TRK_ERR_CAPACITY, TRK_ERR_CUDA, TRK_ERR_NOMEM = 0, -1, -2, -3, -4
TRK_PENDING = -5
TRK_EV_BAD_HIT, TRK_EV_TOO_MANY_HITS, TRK_EV_VOTE_OVERFLOW = 1, 2, 4
TRK_EV_CAND_OVERFLOW, TRK_EV_BAD_OFFSETS = 8, 16

EXPORTED = ["trk_options_default", "trk_create", "trk_reconstruct", "trk_reconstruct_host",
            "trk_destroy", "trk_get_stats", "trk_get_histogram", "trk_histogram_size",
            "trk_get_votes", "trk_fit_triplets", "trk_profile_stages", "trk_last_error", "trk_version",
            "trk_autotune",
            "trk_find_peaks_noalloc", "trk_server_create", "trk_server_submit", "trk_server_wait",
            "trk_server_take", "trk_server_counts", "trk_server_destroy",
            "trk2d_create", "trk2d_reconstruct", "trk2d_get_histogram", "trk2d_last_ms",
            "trk2d_last_error", "trk2d_destroy", "trk2d_find_vertices"]
TRK2D_STRAIGHT, TRK2D_CURVED_IP = 0, 1


class trk_geometry(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("n_triples", C.c_int32), ("b_tesla", C.c_double),
                ("radius", C.c_double * TRK_MAX_LAYERS), ("z_half", C.c_double * TRK_MAX_LAYERS),
                ("triples", (C.c_int32 * 3) * TRK_MAX_TRIPLES)]


class trk_binning(C.Structure):
    _fields_ = [("lo", C.c_double * 5), ("hi", C.c_double * 5), ("n", C.c_int32 * 5),
                ("periodic", C.c_int32), ("threshold", C.c_int32), ("sagitta_fp64_cm", C.c_float)]


class trk_options(C.Structure):
    _fields_ = [("device", C.c_int32), ("max_events", C.c_int32), ("max_hits", C.c_int64),
                ("max_hits_per_event", C.c_int32), ("vote_capacity", C.c_int64),
                ("cand_capacity", C.c_int64), ("assign_capacity", C.c_int64),
                ("peak_scratch_bytes", C.c_int64), ("tile_i", C.c_int32), ("tile_j", C.c_int32),
                ("k_chunk", C.c_int32), ("blocks_per_sm", C.c_int32), ("use_graph", C.c_int32),
                ("vote_level", C.c_int32), ("fit_candidates", C.c_int32)]


class trk_candidate(C.Structure):
    _fields_ = [("bin", C.c_uint32), ("event", C.c_int32), ("votes", C.c_int32),
                ("n_hits", C.c_int32), ("hit_off", C.c_int64), ("params", C.c_float * 5),
                ("reserved", C.c_int32)]


class trk_candidates(C.Structure):
    _fields_ = [("n_events", C.c_int32), ("n_candidates", C.c_int64), ("n_hit_ids", C.c_int64),
                ("cand_off", C.POINTER(C.c_int64)), ("status", C.POINTER(C.c_int32)),
                ("d_cand", C.c_void_p), ("d_hit_ids", C.c_void_p), ("h_cand", C.c_void_p),
                ("h_hit_ids", C.c_void_p), ("d_tracks", C.c_void_p), ("d_hit_used", C.c_void_p),
                ("h_tracks", C.c_void_p), ("h_hit_used", C.c_void_p)]


class trk_track(C.Structure):
    _fields_ = [("params", C.c_float * 5), ("chi2_rphi", C.c_float), ("chi2_rz", C.c_float),
                ("n_used", C.c_int32), ("status", C.c_int32), ("event", C.c_int32),
                ("layers", C.c_uint64)]


class trk2d_config(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_cols", C.c_int32), ("n_rows", C.c_int32),
                ("threshold", C.c_int32), ("lo", C.c_double), ("hi", C.c_double),
                ("b_tesla", C.c_double), ("max_events", C.c_int32), ("reserved", C.c_int32),
                ("max_hits", C.c_int64), ("cand_capacity", C.c_int64), ("hit_capacity", C.c_int64),
                ("vertex_bins", C.c_int32), ("vertex_threshold", C.c_int32),
                ("vertex_min_votes", C.c_int32), ("max_vertices", C.c_int32),
                ("vertex_range", C.c_double)]


class trk2d_candidate(C.Structure):
    _fields_ = [("bin", C.c_uint32), ("event", C.c_int32), ("votes", C.c_int32),
                ("reserved", C.c_int32), ("hit_off", C.c_int64), ("params", C.c_float * 2)]


class trk2d_result(C.Structure):
    _fields_ = [("n_events", C.c_int32), ("n_candidates", C.c_int64), ("n_hit_ids", C.c_int64),
                ("cand_off", C.POINTER(C.c_int64)), ("d_cand", C.c_void_p),
                ("d_hit_ids", C.c_void_p), ("n_vertices", C.c_int64),
                ("vertex_off", C.POINTER(C.c_int64)), ("d_vertices", C.c_void_p),
                ("d_vertex_tracks", C.c_void_p), ("vertex_overflow", C.c_int32)]


class trk2d_vertex(C.Structure):
    _fields_ = [("cell", C.c_uint32), ("event", C.c_int32), ("votes", C.c_int32),
                ("n_tracks", C.c_int32), ("xy", C.c_float * 2), ("track_off", C.c_int64)]


CAND2D_DTYPE = np.dtype([("bin", "<u4"), ("event", "<i4"), ("votes", "<i4"), ("reserved", "<i4"),
                         ("hit_off", "<i8"), ("params", "<f4", (2,))])
VERTEX_DTYPE = np.dtype([("cell", "<u4"), ("event", "<i4"), ("votes", "<i4"), ("n_tracks", "<i4"),
                         ("xy", "<f4", (2,)), ("track_off", "<i8")])
TRK2D_VERTEX_MAX_TRACKS = 64


class trk_tuning(C.Structure):
    _fields_ = [("tile_i", C.c_int32), ("tile_j", C.c_int32), ("vote_level", C.c_int32),
                ("vote_ms", C.c_float)]


class trk_served_event(C.Structure):
    _fields_ = [("status", C.c_int32), ("rc", C.c_int32), ("latency_s", C.c_double),
                ("batch_events", C.c_int32), ("n_candidates", C.c_int64), ("n_hit_ids", C.c_int64)]


class trk_stats(C.Structure):
    _fields_ = [("n_triplets", C.c_int64), ("n_fit", C.c_int64), ("n_exact", C.c_int64),
                ("n_votes", C.c_int64),
                ("n_fp64", C.c_int64), ("n_candidates", C.c_int64), ("n_hit_ids", C.c_int64),
                ("n_work_items", C.c_int64), ("ms_total", C.c_double),
                ("n_plateau", C.c_int64), ("n_cand_votes", C.c_int64)]


# numpy view of trk_candidate (48 bytes)
CAND_DTYPE = np.dtype([("bin", "<u4"), ("event", "<i4"), ("votes", "<i4"), ("n_hits", "<i4"),
                       ("hit_off", "<i8"), ("params", "<f4", (5,)), ("reserved", "<i4")])
assert CAND_DTYPE.itemsize == C.sizeof(trk_candidate) == 48
# numpy view of trk_track (48 bytes)
TRACK_DTYPE = np.dtype({"names": ["params", "chi2_rphi", "chi2_rz", "n_used", "status", "event",
                                  "layers"],
                        "formats": [("<f4", (5,)), "<f4", "<f4", "<i4", "<i4", "<i4", "<u8"],
                        "offsets": [0, 20, 24, 28, 32, 36, 40], "itemsize": 48})
TRK_FIT_OK, TRK_FIT_FEW_LAYERS, TRK_FIT_DEGENERATE = 0, 1, 2

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libtrk.so (must have been built; see paper_1305_4855_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libtrk.so not built ({path}); run paper_1305_4855_gb300.build.build()")
    lib = C.CDLL(path)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    lib.trk_options_default.argtypes = [C.POINTER(trk_options), i32, i64]
    lib.trk_options_default.restype = None
    lib.trk_create.argtypes = [C.POINTER(vp), C.POINTER(trk_geometry), C.POINTER(trk_binning),
                               C.POINTER(trk_options)]
    lib.trk_create.restype = C.c_int
    for name in ("trk_reconstruct", "trk_reconstruct_host"):
        f = getattr(lib, name)
        f.argtypes = [vp, vp, i64, vp, i32, C.POINTER(trk_candidates), vp]
        f.restype = C.c_int
    lib.trk_destroy.argtypes = [vp]
    lib.trk_destroy.restype = C.c_int
    lib.trk_get_stats.argtypes = [vp, C.POINTER(trk_stats)]
    lib.trk_get_stats.restype = C.c_int
    lib.trk_get_histogram.argtypes = [vp, i32, vp, vp]
    lib.trk_get_histogram.restype = C.c_int
    lib.trk_histogram_size.argtypes = [vp]
    lib.trk_histogram_size.restype = i64
    lib.trk_get_votes.argtypes = [vp, vp, vp, i64, C.POINTER(i64), vp]
    lib.trk_get_votes.restype = C.c_int
    lib.trk_fit_triplets.argtypes = [vp, vp, i64, vp, i64, vp, vp, vp, vp]
    lib.trk_fit_triplets.restype = C.c_int
    lib.trk_profile_stages.argtypes = [vp, vp, vp]
    lib.trk_profile_stages.restype = C.c_int
    lib.trk_last_error.argtypes = [vp]
    lib.trk_last_error.restype = C.c_char_p
    lib.trk_find_peaks_noalloc.argtypes = [vp, i32, C.POINTER(trk_binning), vp, vp]
    lib.trk_find_peaks_noalloc.restype = C.c_int
    lib.trk_autotune.argtypes = [vp, vp, i64, vp, i32, i32, C.POINTER(trk_tuning), vp]
    lib.trk_autotune.restype = C.c_int
    lib.trk_server_create.argtypes = [C.POINTER(vp), C.POINTER(trk_geometry), C.POINTER(trk_binning),
                                      C.POINTER(trk_options), i32]
    lib.trk_server_create.restype = C.c_int
    lib.trk_server_submit.argtypes = [vp, vp, i64, C.POINTER(C.c_uint64)]
    lib.trk_server_submit.restype = C.c_int
    lib.trk_server_wait.argtypes = [vp, C.c_uint64, C.c_double, C.POINTER(trk_served_event)]
    lib.trk_server_wait.restype = C.c_int
    lib.trk_server_take.argtypes = [vp, C.c_uint64, vp, i64, vp, i64]
    lib.trk_server_take.restype = C.c_int
    lib.trk_server_counts.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
    lib.trk_server_counts.restype = C.c_int
    lib.trk_server_destroy.argtypes = [vp]
    lib.trk_server_destroy.restype = C.c_int
    lib.trk_version.argtypes = []
    lib.trk_version.restype = C.c_char_p
    lib.trk2d_create.argtypes = [C.POINTER(vp), vp, i32]
    lib.trk2d_create.restype = C.c_int
    lib.trk2d_reconstruct.argtypes = [vp, vp, i64, vp, i32, vp, vp]
    lib.trk2d_reconstruct.restype = C.c_int
    lib.trk2d_get_histogram.argtypes = [vp, i32, vp, vp]
    lib.trk2d_get_histogram.restype = C.c_int
    lib.trk2d_last_ms.argtypes = [vp, C.POINTER(C.c_float), C.POINTER(C.c_float)]
    lib.trk2d_last_ms.restype = C.c_int
    lib.trk2d_last_error.argtypes = [vp]
    lib.trk2d_last_error.restype = C.c_char_p
    lib.trk2d_destroy.argtypes = [vp]
    lib.trk2d_destroy.restype = C.c_int
    lib.trk2d_find_vertices.argtypes = [vp, vp, vp, i32, vp, vp]
    lib.trk2d_find_vertices.restype = C.c_int
    _lib = lib
    return lib


class TrkError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"trk error {code}: {msg}")
        self.code = code


class _DevArray:
    """__cuda_array_interface__ view of a library-owned device array."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


# ---------------------------------------------------------------------------------------
# structs from a workload description
# ---------------------------------------------------------------------------------------

def geometry_from_workload(cfg: dict) -> trk_geometry:
    g = cfg["geometry"]
    geo = trk_geometry()
    geo.n_layers = len(g["radius"])
    geo.b_tesla = float(g["b_tesla"])
    for i, (r, z) in enumerate(zip(g["radius"], g["z_half"])):
        geo.radius[i] = r
        geo.z_half[i] = z
    geo.n_triples = len(g["triples"])
    for t, tri in enumerate(g["triples"]):
        for k in range(3):
            geo.triples[t][k] = int(tri[k])
    return geo


def binning_from_workload(cfg: dict, sagitta_fp64_cm: float = 1e-4) -> trk_binning:
    b = cfg["binning"]
    out = trk_binning()
    for k in range(5):
        out.lo[k] = float(b["lo"][k])
        out.hi[k] = float(b["hi"][k])
        out.n[k] = int(b["n"][k])
    out.periodic = int(sum(1 << k for k in range(5) if b["periodic"][k]))
    out.threshold = int(b["threshold"])
    out.sagitta_fp64_cm = float(b.get("sagitta_fp64_cm", sagitta_fp64_cm))
    return out


def default_options(max_events: int, max_hits: int, **over) -> trk_options:
    lib = load_library()
    o = trk_options()
    lib.trk_options_default(C.byref(o), int(max_events), int(max_hits))
    for k, v in over.items():
        setattr(o, k, v)
    return o


@dataclass
class Result:
    """Candidates of one call, as torch tensors on the device (cloned out of the library's
    buffers) and per-event host arrays."""
    cand: np.ndarray          # structured CAND_DTYPE (host copy)
    hit_ids: np.ndarray       # int32 (host copy)
    cand_off: np.ndarray      # int64 [n_events + 1]
    status: np.ndarray        # int32 [n_events]
    rc: int
    tracks: np.ndarray = None     # structured TRACK_DTYPE, parallel to cand (fit_candidates)
    hit_used: np.ndarray = None   # bool, parallel to hit_ids (fit_candidates)

    def event(self, e: int):
        a, b = int(self.cand_off[e]), int(self.cand_off[e + 1])
        c = self.cand[a:b]
        hits = [self.hit_ids[int(r["hit_off"]):int(r["hit_off"]) + int(r["n_hits"])] for r in c]
        return c, hits

    def event_fits(self, e: int):
        """(tracks of event e's candidates, per candidate the bool mask of kept hits)."""
        a, b = int(self.cand_off[e]), int(self.cand_off[e + 1])
        c = self.cand[a:b]
        used = [self.hit_used[int(r["hit_off"]):int(r["hit_off"]) + int(r["n_hits"])] for r in c]
        return self.tracks[a:b], used


class Reconstructor:
    """One trk handle.  Calls map one to one onto the C ABI."""

    def __init__(self, cfg: dict, max_events: int, max_hits: int, device: int = 0,
                 sagitta_fp64_cm: float = 1e-4, **opts):
        self.lib = load_library()
        self.cfg = cfg
        self.geo = geometry_from_workload(cfg)
        self.bin = binning_from_workload(cfg, sagitta_fp64_cm)
        self.opt = default_options(max_events, max_hits, device=device, **opts)
        h = C.c_void_p()
        rc = self.lib.trk_create(C.byref(h), C.byref(self.geo), C.byref(self.bin),
                                 C.byref(self.opt))
        if rc != TRK_OK:
            raise TrkError(rc, self.lib.trk_last_error(None).decode())
        self.h = h
        self.out = trk_candidates()

    def close(self):
        if getattr(self, "h", None):
            self.lib.trk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def error(self) -> str:
        return self.lib.trk_last_error(self.h).decode()

    # -- calls --------------------------------------------------------------------------
    def reconstruct_device(self, hits, offsets, stream=None) -> int:
        """hits: cuda float32 tensor (N, 4) (x, y, z, layer id bits); offsets: cuda int64
        tensor (n_events + 1).  Returns the C return code; outputs stay in the library."""
        n_events = offsets.numel() - 1
        rc = self.lib.trk_reconstruct(self.h, C.c_void_p(hits.data_ptr()), hits.shape[0],
                                      C.c_void_p(offsets.data_ptr()), n_events,
                                      C.byref(self.out), C.c_void_p(_stream_handle(stream)))
        if rc not in (TRK_OK, TRK_ERR_CAPACITY):
            raise TrkError(rc, self.error())
        return rc

    def reconstruct_host(self, hits: np.ndarray, offsets: np.ndarray, stream=None) -> int:
        """Host (ideally pinned) arrays in, host results in library-owned pinned memory."""
        n_events = len(offsets) - 1
        hp = hits.ctypes.data if isinstance(hits, np.ndarray) else hits.data_ptr()
        op = offsets.ctypes.data if isinstance(offsets, np.ndarray) else offsets.data_ptr()
        rc = self.lib.trk_reconstruct_host(self.h, C.c_void_p(hp), int(hits.shape[0]),
                                           C.c_void_p(op), n_events, C.byref(self.out),
                                           C.c_void_p(_stream_handle(stream)))
        if rc not in (TRK_OK, TRK_ERR_CAPACITY):
            raise TrkError(rc, self.error())
        return rc

    def device_outputs(self):
        """Zero-copy torch views of the library-owned device candidates and hit ids."""
        import torch
        o = self.out
        cand = torch.as_tensor(_DevArray(o.d_cand, (o.n_candidates * 48,), "|u1"), device="cuda") \
            if o.n_candidates else torch.zeros(0, dtype=torch.uint8, device="cuda")
        hits = torch.as_tensor(_DevArray(o.d_hit_ids, (o.n_hit_ids,), "<i4"), device="cuda") \
            if o.n_hit_ids else torch.zeros(0, dtype=torch.int32, device="cuda")
        return cand, hits

    def result(self, rc: int = TRK_OK, from_host: bool = False) -> Result:
        o = self.out
        n_ev = o.n_events
        cand_off = np.ctypeslib.as_array(o.cand_off, shape=(n_ev + 1,)).copy()
        status = np.ctypeslib.as_array(o.status, shape=(n_ev,)).copy()
        tracks = hit_used = None
        if from_host:
            nb = o.n_candidates * 48
            cand = np.frombuffer((C.c_char * nb).from_address(o.h_cand), dtype=CAND_DTYPE).copy() \
                if nb else np.zeros(0, CAND_DTYPE)
            hit_ids = np.frombuffer((C.c_char * (4 * o.n_hit_ids)).from_address(o.h_hit_ids),
                                    dtype=np.int32).copy() if o.n_hit_ids else np.zeros(0, np.int32)
            if o.h_tracks:
                tracks = np.frombuffer((C.c_char * nb).from_address(o.h_tracks),
                                       dtype=TRACK_DTYPE).copy() if nb else np.zeros(0, TRACK_DTYPE)
                hit_used = np.frombuffer((C.c_char * o.n_hit_ids).from_address(o.h_hit_used),
                                         dtype=np.uint8).astype(bool) if o.n_hit_ids \
                    else np.zeros(0, bool)
        else:
            cd, hd = self.device_outputs()
            cand = cd.cpu().numpy().view(CAND_DTYPE)
            hit_ids = hd.cpu().numpy()
            if o.d_tracks:
                tracks, used = self.device_fits()
                tracks = tracks.cpu().numpy().view(TRACK_DTYPE).reshape(-1)
                hit_used = used.cpu().numpy().astype(bool)
        return Result(cand, hit_ids, cand_off, status, rc, tracks, hit_used)

    def device_fits(self):
        """(tracks uint8 (n, 48), hit_used uint8 (n_hit_ids,)) as torch tensors on the device,
        cloned out of the library's buffers (needs fit_candidates)."""
        import torch
        o = self.out
        if not o.d_tracks:
            raise TrkError(TRK_ERR_INVALID, "handle created without fit_candidates")
        tr = torch.as_tensor(_DevArray(o.d_tracks, (o.n_candidates, 48), "|u1"), device="cuda").clone() \
            if o.n_candidates else torch.zeros((0, 48), dtype=torch.uint8, device="cuda")
        used = torch.as_tensor(_DevArray(o.d_hit_used, (o.n_hit_ids,), "|u1"), device="cuda").clone() \
            if o.n_hit_ids else torch.zeros(0, dtype=torch.uint8, device="cuda")
        return tr, used

    def stats(self) -> dict:
        s = trk_stats()
        self.lib.trk_get_stats(self.h, C.byref(s))
        return {k: getattr(s, k) for k, _ in trk_stats._fields_}

    def autotune(self, hits, offsets, reps: int = 2, stream=None) -> dict:
        """Pick the fastest vote-kernel tile and occupancy on these events."""
        best = trk_tuning()
        rc = self.lib.trk_autotune(self.h, C.c_void_p(hits.data_ptr()), hits.shape[0],
                                   C.c_void_p(offsets.data_ptr()), offsets.numel() - 1, reps,
                                   C.byref(best), C.c_void_p(_stream_handle(stream)))
        if rc != TRK_OK:
            raise TrkError(rc, self.error())
        return {k: getattr(best, k) for k, _ in trk_tuning._fields_}

    def stage_ms(self, stream=None) -> dict:
        """Device time of the stages of the last call (ms)."""
        ms = (C.c_float * 8)()
        rc = self.lib.trk_profile_stages(self.h, ms, C.c_void_p(_stream_handle(stream)))
        if rc != TRK_OK:
            raise TrkError(rc, self.error())
        return dict(vote=ms[0], setup=ms[1], peaks=ms[2], candidates=ms[3], assign=ms[4],
                    fit=ms[5])

    def histogram(self, event: int = 0):
        import torch
        n = self.lib.trk_histogram_size(self.h)
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        rc = self.lib.trk_get_histogram(self.h, event, C.c_void_p(out.data_ptr()),
                                        C.c_void_p(_stream_handle(None)))
        if rc != TRK_OK:
            raise TrkError(rc, self.error())
        torch.cuda.synchronize()
        return out

    def votes(self):
        """(event, i, j, k) input indices and bins of every accepted triplet of the last call."""
        import torch
        n = C.c_int64(0)
        rc = self.lib.trk_get_votes(self.h, None, None, 0, C.byref(n), C.c_void_p(_stream_handle(None)))
        if rc != TRK_OK:
            raise TrkError(rc, self.error())
        cap = n.value
        dst = torch.empty((max(cap, 1), 4), dtype=torch.int32, device="cuda")
        bins = torch.empty(max(cap, 1), dtype=torch.int32, device="cuda")
        rc = self.lib.trk_get_votes(self.h, C.c_void_p(dst.data_ptr()), C.c_void_p(bins.data_ptr()),
                                    cap, C.byref(n), C.c_void_p(_stream_handle(None)))
        if rc != TRK_OK:
            raise TrkError(rc, self.error())
        return dst[:n.value], bins[:n.value].view(torch.int32)

    def fit_triplets(self, hits, ijk, stream=None):
        """FP32 (FP64 where needed) parameters, bins and flags of explicit triplets."""
        import torch
        n = ijk.shape[0]
        params = torch.empty((max(n, 1), 5), dtype=torch.float32, device="cuda")
        bins = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
        flags = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
        rc = self.lib.trk_fit_triplets(self.h, C.c_void_p(hits.data_ptr()), hits.shape[0],
                                       C.c_void_p(ijk.data_ptr()), n, C.c_void_p(params.data_ptr()), C.c_void_p(bins.data_ptr()),
                                       C.c_void_p(flags.data_ptr()), C.c_void_p(_stream_handle(stream)))
        if rc != TRK_OK:
            raise TrkError(rc, self.error())
        return params[:n], bins[:n], flags[:n]


class Server:
    """A trk server (continuous batching over n_lanes resident handles)."""

    def __init__(self, cfg: dict, lane_events: int, lane_hits: int, n_lanes: int = 2,
                 device: int = 0, sagitta_fp64_cm: float = 1e-4, **opts):
        self.lib = load_library()
        self.geo = geometry_from_workload(cfg)
        self.bin = binning_from_workload(cfg, sagitta_fp64_cm)
        self.opt = default_options(lane_events, lane_hits, device=device, **opts)
        s = C.c_void_p()
        rc = self.lib.trk_server_create(C.byref(s), C.byref(self.geo), C.byref(self.bin),
                                        C.byref(self.opt), n_lanes)
        if rc != TRK_OK:
            raise TrkError(rc, self.lib.trk_last_error(None).decode())
        self.s = s

    def submit(self, hits: np.ndarray) -> int:
        """hits: host float32 (N, 4) array (x, y, z, layer id bits)."""
        hits = np.ascontiguousarray(hits, dtype=np.float32)
        t = C.c_uint64(0)
        rc = self.lib.trk_server_submit(self.s, C.c_void_p(hits.ctypes.data), hits.shape[0], C.byref(t))
        if rc != TRK_OK:
            raise TrkError(rc, "submit failed")
        return t.value

    def wait(self, ticket: int, timeout_s: float = 60.0):
        ev = trk_served_event()
        rc = self.lib.trk_server_wait(self.s, ticket, timeout_s, C.byref(ev))
        if rc == TRK_PENDING:
            return None
        if rc != TRK_OK:
            raise TrkError(rc, "wait failed")
        return {k: getattr(ev, k) for k, _ in trk_served_event._fields_}

    def take(self, ticket: int, info: dict):
        """The event's candidates (CAND_DTYPE) and per-candidate hit lists (event-local)."""
        nc, nh = int(info["n_candidates"]), int(info["n_hit_ids"])
        cand = np.zeros(max(nc, 1), dtype=CAND_DTYPE)
        hits = np.zeros(max(nh, 1), dtype=np.int32)
        rc = self.lib.trk_server_take(self.s, ticket, C.c_void_p(cand.ctypes.data), nc,
                                      C.c_void_p(hits.ctypes.data), nh)
        if rc != TRK_OK:
            raise TrkError(rc, "take failed")
        cand = cand[:nc]
        return cand, [hits[int(c["hit_off"]):int(c["hit_off"]) + int(c["n_hits"])] for c in cand]

    def counts(self) -> dict:
        v = [C.c_int64(0) for _ in range(4)]
        self.lib.trk_server_counts(self.s, *[C.byref(x) for x in v])
        return dict(batches=v[0].value, events=v[1].value, failed=v[2].value, queued=v[3].value)

    def close(self):
        if getattr(self, "s", None):
            self.lib.trk_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hough2d_config(cfg: dict, max_events: int, max_hits: int, **over) -> trk2d_config:
    """trk2d_config from a workload's "hough2d" block."""
    h = cfg["hough2d"]
    c = trk2d_config()
    c.kind = TRK2D_STRAIGHT if h["kind"] == "straight" else TRK2D_CURVED_IP
    c.n_cols, c.n_rows, c.threshold = int(h["n_cols"]), int(h["n_rows"]), int(h["threshold"])
    c.lo, c.hi = float(h["lo"]), float(h["hi"])
    c.b_tesla = float(cfg["geometry"].get("b_tesla", 0.0))
    c.max_events, c.max_hits = int(max_events), int(max_hits)
    c.cand_capacity = int(over.pop("cand_capacity", 4096 * max_events + 4096))
    c.hit_capacity = int(over.pop("hit_capacity", 64 * max_hits + 4096))
    v = h.get("vertex")
    if v:
        c.vertex_bins, c.vertex_threshold = int(v["n_bins"]), int(v["threshold"])
        c.vertex_min_votes = int(v.get("min_track_votes", 0))
        c.vertex_range = float(v["range"])
        c.max_vertices = int(over.pop("max_vertices", v.get("max_vertices", 1024)))
    for k, v in over.items():
        setattr(c, k, v)
    return c


class Hough2D:
    """One trk2d handle (per-hit straight-line or interaction-point curved Hough)."""

    def __init__(self, cfg: dict, max_events: int, max_hits: int, device: int = 0, **over):
        self.lib = load_library()
        self.cfg = hough2d_config(cfg, max_events, max_hits, **over)
        h = C.c_void_p()
        rc = self.lib.trk2d_create(C.byref(h), C.byref(self.cfg), device)
        if rc != TRK_OK:
            raise TrkError(rc, self.lib.trk2d_last_error(None).decode())
        self.h = h
        self.out = trk2d_result()

    def reconstruct_device(self, hits, offsets, stream=None) -> int:
        """hits: cuda float32 (N, 4); offsets: cuda int64 (n_events + 1).  Synchronises."""
        return self.lib.trk2d_reconstruct(self.h, C.c_void_p(hits.data_ptr()), hits.shape[0],
                                          C.c_void_p(offsets.data_ptr()), offsets.numel() - 1,
                                          C.byref(self.out), C.c_void_p(_stream_handle(stream)))

    def result(self, rc: int = TRK_OK):
        """(candidates CAND2D_DTYPE, hit ids int32, cand_off int64) copied to the host."""
        import torch
        o = self.out
        cand_off = np.ctypeslib.as_array(o.cand_off, shape=(o.n_events + 1,)).copy()
        cand = torch.as_tensor(_DevArray(o.d_cand, (o.n_candidates * 32,), "|u1"), device="cuda") \
            .cpu().numpy().view(CAND2D_DTYPE) if o.n_candidates else np.zeros(0, CAND2D_DTYPE)
        hit_ids = torch.as_tensor(_DevArray(o.d_hit_ids, (o.n_hit_ids,), "<i4"), device="cuda") \
            .cpu().numpy() if o.n_hit_ids else np.zeros(0, np.int32)
        return cand, hit_ids, cand_off

    def vertices(self):
        """(vertices VERTEX_DTYPE, vertex_off int64, per vertex its candidate indices, overflow)
        of the last call (vertex transform enabled)."""
        import torch
        o = self.out
        if not o.vertex_off:
            raise TrkError(TRK_ERR_INVALID, "the handle has no vertex transform")
        voff = np.ctypeslib.as_array(o.vertex_off, shape=(o.n_events + 1,)).copy()
        n = int(o.n_vertices)
        v = torch.as_tensor(_DevArray(o.d_vertices, (n * 32,), "|u1"), device="cuda").cpu().numpy() \
            .view(VERTEX_DTYPE) if n else np.zeros(0, VERTEX_DTYPE)
        tracks = []
        if n:
            hi = int(v["track_off"].max()) + TRK2D_VERTEX_MAX_TRACKS
            t = torch.as_tensor(_DevArray(o.d_vertex_tracks, (hi,), "<i4"), device="cuda").cpu().numpy()
            tracks = [t[int(r["track_off"]):int(r["track_off"]) + int(r["n_tracks"])] for r in v]
        return v, voff, tracks, int(o.vertex_overflow)

    def find_vertices(self, cand: np.ndarray, cand_off: np.ndarray, stream=None) -> int:
        """The vertex transform over given candidates (CAND2D_DTYPE host array sorted by
        event, int64 offsets); results through vertices()."""
        import torch
        c = torch.from_numpy(np.ascontiguousarray(cand).view(np.uint8).copy()).cuda()
        o = torch.from_numpy(np.ascontiguousarray(cand_off, dtype=np.int64)).cuda()
        self._keep = (c, o)
        return self.lib.trk2d_find_vertices(self.h, C.c_void_p(c.data_ptr()), C.c_void_p(o.data_ptr()),
                                            len(cand_off) - 1, C.byref(self.out),
                                            C.c_void_p(_stream_handle(stream)))

    def histogram(self, event: int = 0):
        import torch
        out = torch.empty(self.cfg.n_cols * self.cfg.n_rows, dtype=torch.int32, device="cuda")
        rc = self.lib.trk2d_get_histogram(self.h, event, C.c_void_p(out.data_ptr()), None)
        if rc != TRK_OK:
            raise TrkError(rc, self.error())
        return out

    def last_ms(self) -> dict:
        a, b = C.c_float(0), C.c_float(0)
        rc = self.lib.trk2d_last_ms(self.h, C.byref(a), C.byref(b))
        if rc != TRK_OK:
            raise TrkError(rc, self.error())
        return {"vote_peak": a.value, "total": b.value}

    def error(self) -> str:
        return self.lib.trk2d_last_error(self.h).decode()

    def close(self):
        if getattr(self, "h", None):
            self.lib.trk2d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
