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
            "trk_server_take", "trk_server_counts", "trk_server_destroy"]


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
                ("vote_level", C.c_int32)]


class trk_candidate(C.Structure):
    _fields_ = [("bin", C.c_uint32), ("event", C.c_int32), ("votes", C.c_int32),
                ("n_hits", C.c_int32), ("hit_off", C.c_int64), ("params", C.c_float * 5),
                ("reserved", C.c_int32)]


class trk_candidates(C.Structure):
    _fields_ = [("n_events", C.c_int32), ("n_candidates", C.c_int64), ("n_hit_ids", C.c_int64),
                ("cand_off", C.POINTER(C.c_int64)), ("status", C.POINTER(C.c_int32)),
                ("d_cand", C.c_void_p), ("d_hit_ids", C.c_void_p), ("h_cand", C.c_void_p),
                ("h_hit_ids", C.c_void_p)]


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
                ("n_work_items", C.c_int64), ("ms_total", C.c_double)]


# numpy view of trk_candidate (48 bytes)
CAND_DTYPE = np.dtype([("bin", "<u4"), ("event", "<i4"), ("votes", "<i4"), ("n_hits", "<i4"),
                       ("hit_off", "<i8"), ("params", "<f4", (5,)), ("reserved", "<i4")])
assert CAND_DTYPE.itemsize == C.sizeof(trk_candidate) == 48

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

    def event(self, e: int):
        a, b = int(self.cand_off[e]), int(self.cand_off[e + 1])
        c = self.cand[a:b]
        hits = [self.hit_ids[int(r["hit_off"]):int(r["hit_off"]) + int(r["n_hits"])] for r in c]
        return c, hits


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
        if from_host:
            nb = o.n_candidates * 48
            cand = np.frombuffer((C.c_char * nb).from_address(o.h_cand), dtype=CAND_DTYPE).copy() \
                if nb else np.zeros(0, CAND_DTYPE)
            hit_ids = np.frombuffer((C.c_char * (4 * o.n_hit_ids)).from_address(o.h_hit_ids),
                                    dtype=np.int32).copy() if o.n_hit_ids else np.zeros(0, np.int32)
        else:
            cd, hd = self.device_outputs()
            cand = cd.cpu().numpy().view(CAND_DTYPE)
            hit_ids = hd.cpu().numpy()
        return Result(cand, hit_ids, cand_off, status, rc)

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
        return dict(vote=ms[0], setup=ms[1], peaks=ms[2], candidates=ms[3], assign=ms[4])

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
