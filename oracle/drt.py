"""Dynamic Resolution Training schedule, Eq. 15 (Sec. 3.4) -- oracle side.

TEST INFRASTRUCTURE ONLY.

value(it) = end + 1/2 (start - end) (1 + cos(pi * it / total))

A batch of V views samples the schedule at it / total = k / (V - 1), k = 0..V-1,
and scales a full-resolution W x H frame to round(W s_k) x round(H s_k), with
rounding half to even (the paper does not say how sizes are rounded).
"""
import math


def scale(it: float, total: float, start: float, end: float) -> float:
    return end + 0.5 * (start - end) * (1.0 + math.cos(math.pi * it / total))


def batch_sizes(width: int, height: int, n_views: int, start: float = 0.25, end: float = 1.0):
    out = []
    for k in range(n_views):
        s = scale(k, max(n_views - 1, 1), start, end) if n_views > 1 else end
        out.append((int(round(width * s)), int(round(height * s))))
    return out
