"""trk_find_peaks_noalloc -- the peak step for callers that may not allocate device memory
-- must give exactly the candidates trk_reconstruct gives for the same histograms (GPU).

The entry point keeps its scratch in a static device array shared by all calls, so it is
called twice in a row on different histograms: stale contents from the first call must
not leak into the second.  This file sorts last so that a stop-at-first-failure run has
run every other test before it; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1305_4855_gb300 import events as ev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trk():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1305_4855_gb300 import build
    build.build()
    from paper_1305_4855_gb300 import trk as t
    t.load_library()
    return t


def _bits_to_bins(words: np.ndarray, nbins: int) -> np.ndarray:
    bits = np.unpackbits(words.view(np.uint8), bitorder="little")[:nbins]
    return np.nonzero(bits)[0].astype(np.int64)


def _check_against_reconstruct(trk, cfg, batches, pad_ints=0):
    for batch in batches:
        rec = trk.Reconstructor(cfg, max_events=batch.n_events, max_hits=batch.n_hits,
                                vote_capacity=1 << 20, cand_capacity=1 << 16,
                                assign_capacity=1 << 20)
        hits = torch.from_numpy(batch.packed()).cuda()
        offs = torch.from_numpy(batch.offsets).cuda()
        res = rec.result(rec.reconstruct_device(hits, offs))
        assert res.rc == 0
        nbins = int(rec.lib.trk_histogram_size(rec.h))
        words = (nbins + 31) // 32
        # pad_ints int32 in front: the histograms start 4 * pad_ints bytes past an aligned
        # allocation (any int32 pointer is valid input)
        hist = torch.cat([torch.zeros(pad_ints, dtype=torch.int32, device="cuda")] +
                         [rec.histogram(e) for e in range(batch.n_events)])
        bits = torch.full((batch.n_events * words,), -1, dtype=torch.int32, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        rc = rec.lib.trk_find_peaks_noalloc(C.c_void_p(hist.data_ptr() + 4 * pad_ints),
                                            batch.n_events,
                                            C.byref(rec.bin), C.c_void_p(bits.data_ptr()),
                                            C.c_void_p(stream))
        assert rc == trk.TRK_OK, rec.lib.trk_last_error(None)
        torch.cuda.synchronize()
        got = bits.cpu().numpy().view(np.uint32).reshape(batch.n_events, words)
        for e in range(batch.n_events):
            cand, _ = res.event(e)
            expect = np.sort(cand["bin"].astype(np.int64))
            assert len(expect) > 3
            assert np.array_equal(_bits_to_bins(got[e], nbins), expect)
        rec.close()


def test_noalloc_peaks_equal_reconstruct_candidates(trk):
    cfg = ev.load_workload("barrel4_20trk")
    # two different batches (2 events, then 1 event), one call each, in a row
    batches = [ev.concat([ev.make_batch(cfg, seed=41), ev.make_batch(cfg, seed=42)]),
               ev.make_batch(cfg, seed=43)]
    _check_against_reconstruct(trk, cfg, batches)


def test_noalloc_unaligned_and_non_periodic(trk):
    # histograms 4 bytes past a 16-byte boundary (narrower loads), then a binning whose
    # phi0 does not wrap, with a d0 axis shorter than the filter's slab
    cfg = ev.load_workload("barrel4_20trk")
    _check_against_reconstruct(trk, cfg, [ev.make_batch(cfg, seed=44)], pad_ints=1)
    _check_against_reconstruct(trk, cfg, [ev.make_batch(cfg, seed=45)], pad_ints=3)
    flat = dict(cfg, binning=dict(cfg["binning"], periodic=[False] * 5,
                                  n=[16, 16, 2, 16, 16]))
    _check_against_reconstruct(trk, flat, [ev.concat([ev.make_batch(flat, seed=46),
                                                      ev.make_batch(flat, seed=47)])])


def test_noalloc_rejects_misaligned_pointers(trk):
    cfg = ev.load_workload("barrel4_20trk")
    binning = trk.binning_from_workload(cfg)
    lib = trk.load_library()
    buf = torch.zeros(1 << 20, dtype=torch.int32, device="cuda")
    words = torch.zeros(1 << 16, dtype=torch.int32, device="cuda")
    rc = lib.trk_find_peaks_noalloc(C.c_void_p(buf.data_ptr() + 2), 1, C.byref(binning),
                                    C.c_void_p(words.data_ptr()), None)
    assert rc == trk.TRK_ERR_INVALID
    assert b"aligned" in lib.trk_last_error(None)
    rc = lib.trk_find_peaks_noalloc(C.c_void_p(buf.data_ptr()), 1, C.byref(binning),
                                    C.c_void_p(words.data_ptr() + 1), None)
    assert rc == trk.TRK_ERR_INVALID


def test_noalloc_rejects_oversized_histograms(trk):
    cfg = ev.load_workload("barrel10_500trk")        # 64x64x32x32x16 bins > 2^21
    binning = trk.binning_from_workload(cfg)
    lib = trk.load_library()
    dummy = torch.zeros(8, dtype=torch.int32, device="cuda")
    rc = lib.trk_find_peaks_noalloc(C.c_void_p(dummy.data_ptr()), 1, C.byref(binning),
                                    C.c_void_p(dummy.data_ptr()), None)
    assert rc == trk.TRK_ERR_INVALID
    assert b"TRK_NOALLOC_MAX_BINS" in lib.trk_last_error(None)
