"""EXP2Q, the 256-entry table of the integer softmax: EXP2Q[f] = round(2^(23 - f/256)).

Part of the CPU oracle (test infrastructure only).  The integer softmax that turns the
context model's logits into a 16-bit CDF (the learned CDF of Sec. 3.4, "Autoregressive
Prediction Coding") needs 2^(-x) at 1/256 steps; a table keeps both coder sides on the same
integers, with no libm in the loop.

Derived here with exact integer arithmetic: e = round(y) with y^256 = 2^(5888 - f), i.e. the
largest e with (2e - 1)^256 <= 2^(6144 - f).  No floating point is involved.
"""
from __future__ import annotations

from functools import lru_cache


def _entry(f: int) -> int:
    target = 1 << (6144 - f)
    lo, hi = 1 << 21, 1 << 24
    while lo < hi:  # largest e with (2e-1)^256 <= target
        mid = (lo + hi + 1) // 2
        if (2 * mid - 1) ** 256 <= target:
            lo = mid
        else:
            hi = mid - 1
    return lo


@lru_cache(maxsize=1)
def exp2q_table() -> tuple[int, ...]:
    return tuple(_entry(f) for f in range(256))
