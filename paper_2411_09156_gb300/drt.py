"""Dynamic Resolution Training schedule (Eq. 15, Sec. 3.4) as the view-size generator
of a batched dynamic-resolution step.

scale(it) = end + 1/2 (start - end) (1 + cos(pi it / total)). A batch of V views
samples it / total = k / (V - 1); view k is round(W s_k) x round(H s_k) (rounding
half to even; the paper does not state its rounding).
"""
from __future__ import annotations

import math
from typing import List, Tuple


def drt_scale(it: float, total: float, start: float, end: float) -> float:
    return end + 0.5 * (start - end) * (1.0 + math.cos(math.pi * it / total))


def drt_sizes(width: int, height: int, n_views: int, start: float = 0.25, end: float = 1.0) -> List[Tuple[int, int]]:
    if n_views == 1:
        return [(width, height)]
    return [(int(round(width * drt_scale(k, n_views - 1, start, end))),
             int(round(height * drt_scale(k, n_views - 1, start, end)))) for k in range(n_views)]
