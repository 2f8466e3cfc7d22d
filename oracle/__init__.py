"""FP64 CPU oracle of the GES rasterizer.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline use it; the CUDA library and its Python binding never import it.

  oracle.oracle   per-pixel brute-force forward and analytic backward (C, FP64)
  oracle.binning  the integer stage (tile overlap, keys, order) in float32
  oracle.drt      the cosine dynamic-resolution schedule, Eq. 15
"""
