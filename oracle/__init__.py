"""FP64 CPU oracle of the displaced-track Hough transform -- TEST INFRASTRUCTURE ONLY.

Only the tests, the entry point's smoke check and the benchmark's CPU-baseline leg may
import this package.  It shares no code with the CUDA library and never reads anything
the CUDA path produced as an input.

  enumerate_batch  -- the C definition (trk_oracle.c): every triplet of every listed
                      layer triple, FP64 helix fit, binning, edge-ambiguity flags;
  reconstruct      -- votes, peak rule and hit assignment (reconstruct.py, numpy);
  enumerate_blocks -- the same definition over one event, keeping only the counts and
                      triplets of chosen (phi0, q/pT) blocks (events too large to list);
  block_peaks      -- the peak rule over those counts (trk_oracle.c);
  fit_tracks       -- the candidate fit (trk_oracle.c): algebraic circle fit, one hit per
                      layer, signed arcs and the least-squares line;
  hough2d          -- the per-hit 2-D transforms (straight lines, curved tracks through the
                      interaction point) and the vertex transform over straight-line peaks
                      (numpy, FP64).
"""
from .core import (OracleSetup, block_peaks, enumerate_batch, enumerate_blocks,  # noqa: F401
                   fit_list, fit_tracks, max_threads)
from .reconstruct import (histogram, neighbour_offsets, peaks, assign_hits, bin_centres,  # noqa: F401
                          reconstruct)
