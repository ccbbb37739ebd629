"""The C-ABI library builds, loads and exports every symbol include/trk.h declares, and
the Python mirrors of its structs have the C layout (CPU only: no compute call)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "trk.h")


@pytest.fixture(scope="module")
def lib_path():
    from paper_1305_4855_gb300 import build
    try:
        return build.build()
    except RuntimeError as e:  # pragma: no cover - nvcc missing
        pytest.skip(str(e))


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|int64_t|const char \*)\s*\*?\s*(trk(?:2d)?_\w+)\s*\(",
                                 text, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("trk_create", "trk_reconstruct", "trk_destroy", "trk_reconstruct_host",
              "trk_fit_triplets", "trk_get_histogram", "trk_get_votes"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\b(trk(?:2d)?_\w+)\b", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = C.CDLL(lib_path)
    for n in declared_functions():
        getattr(lib, n)


def test_binding_names_match_header():
    from paper_1305_4855_gb300 import trk
    assert sorted(trk.EXPORTED) == declared_functions()


def test_struct_layouts_match_c(tmp_path, lib_path):
    from paper_1305_4855_gb300 import trk
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "trk.h"
#define S(t) printf(#t " %zu\n", sizeof(t));
#define O(t, f) printf(#t "." #f " %zu\n", offsetof(t, f));
int main(void) {
  S(trk_hit) S(trk_geometry) S(trk_binning) S(trk_options) S(trk_candidate) S(trk_candidates) S(trk_stats)
  S(trk_track)
  O(trk_geometry, b_tesla) O(trk_geometry, triples) O(trk_binning, n) O(trk_binning, sagitta_fp64_cm)
  O(trk_options, vote_capacity) O(trk_options, tile_i) O(trk_options, use_graph)
  O(trk_candidate, hit_off) O(trk_candidate, params) O(trk_candidates, cand_off) O(trk_candidates, h_hit_ids)
  O(trk_stats, ms_total) O(trk_options, fit_candidates) O(trk_candidates, d_tracks)
  O(trk_candidates, h_hit_used) O(trk_track, chi2_rphi) O(trk_track, event) O(trk_track, layers)
  return 0; }
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    py = {"trk_hit": 16, "trk_geometry": C.sizeof(trk.trk_geometry),
          "trk_binning": C.sizeof(trk.trk_binning), "trk_options": C.sizeof(trk.trk_options),
          "trk_candidate": C.sizeof(trk.trk_candidate),
          "trk_candidates": C.sizeof(trk.trk_candidates), "trk_stats": C.sizeof(trk.trk_stats),
          "trk_track": C.sizeof(trk.trk_track)}
    for k, v in py.items():
        assert int(got[k]) == v, k
    for key, val in got.items():
        if "." in key:
            t, f = key.split(".")
            assert getattr(getattr(trk, t), f).offset == int(val), key


def test_create_rejects_bad_setups(lib_path):
    # validation happens before any device call, but trk_create needs a CUDA device for the
    # rest; only the argument checks are exercised here
    from paper_1305_4855_gb300 import events, trk
    lib = trk.load_library()
    cfg = events.load_workload("barrel4_20trk")
    geo = trk.geometry_from_workload(cfg)
    binning = trk.binning_from_workload(cfg)
    opt = trk.trk_options()
    lib.trk_options_default(C.byref(opt), 1, 1000)
    h = C.c_void_p()
    bad = trk.trk_binning.from_buffer_copy(binning)
    bad.periodic = 2
    assert lib.trk_create(C.byref(h), C.byref(geo), C.byref(bad), C.byref(opt)) == trk.TRK_ERR_INVALID
    assert b"periodic" in lib.trk_last_error(None)
    g2 = trk.trk_geometry.from_buffer_copy(geo)
    g2.triples[0][1] = g2.triples[0][0]
    assert lib.trk_create(C.byref(h), C.byref(g2), C.byref(binning), C.byref(opt)) == trk.TRK_ERR_INVALID
    o2 = trk.trk_options.from_buffer_copy(opt)
    o2.tile_i = 3
    assert lib.trk_create(C.byref(h), C.byref(geo), C.byref(binning), C.byref(o2)) == trk.TRK_ERR_INVALID
    assert lib.trk_create(None, C.byref(geo), C.byref(binning), C.byref(opt)) == trk.TRK_ERR_INVALID


def test_hough2d_create_rejects_bad_configs(lib_path):
    # the 2-D transforms validate their configuration before any device call
    from paper_1305_4855_gb300 import events, trk
    lib = trk.load_library()
    cfg = events.load_workload("sht_jets")
    h = C.c_void_p()

    def bad(**kw):
        c = trk.hough2d_config(cfg, 4, 1000)
        for k, v in kw.items():
            setattr(c, k, v)
        return lib.trk2d_create(C.byref(h), C.byref(c), 0)

    assert bad(lo=-10.0) == trk.TRK_ERR_INVALID                  # straight needs lo = -hi
    assert b"symmetric" in lib.trk2d_last_error(None)
    assert bad(n_cols=2) == trk.TRK_ERR_INVALID
    assert bad(kind=7) == trk.TRK_ERR_INVALID
    assert bad(threshold=0) == trk.TRK_ERR_INVALID
    assert bad(vertex_bins=200) == trk.TRK_ERR_INVALID
    assert bad(kind=trk.TRK2D_CURVED_IP, b_tesla=0.0, lo=-1.0, hi=1.0,
               vertex_bins=0) == trk.TRK_ERR_INVALID                 # curved needs a field
    assert lib.trk2d_create(None, None, 0) == trk.TRK_ERR_INVALID
