"""GB300-native GES (generalized-exponential splatting) rasterizer.

The compute path is the CUDA library libges.so (csrc/, C-ABI in include/ges.h);
this package holds its thin ctypes binding (`api`), the autograd wrapper
(`autograd`), the batched dynamic-resolution driver (`batch`, `drt`) and the
seeded synthetic scenes (`scenes`). Submodules load lazily, so importing the
package never touches CUDA.
"""
__all__ = ["api", "autograd", "batch", "drt", "scenes", "build"]
