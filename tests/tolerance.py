"""Element-wise tolerance of the fp32 training kernels against the fp64 oracle.

Every element must satisfy |x32 - x64| <= RTOL |x64| + ATOL_FRAC max|x64| (per tensor).
RTOL = 1e-4 is the relative bound the learned part is held to.  A pure relative bound cannot
hold for elements that are sums of terms of both signs: a gradient element that cancels to
1e-7 of its tensor's largest still carries the fp32 rounding of its summands (about 2^-24 of
each, accumulated over the batch), so its own relative error can reach 1e-2.  The absolute
term, 1e-5 of the tensor's largest magnitude, is that floor: 4096 fp32 summands of the
tensor's scale give a rounding error near 2^-24 sqrt(4096) = 4e-6 of it.  One wrong element
(a dropped term, a wrong row) is off by a fraction of its own value and fails."""
import numpy as np

RTOL = 1e-4
ATOL_FRAC = 1e-5


def assert_close(x32, x64, name: str, rtol: float = RTOL, atol_frac: float = ATOL_FRAC) -> None:
    a = np.asarray(x32, np.float64)
    b = np.asarray(x64, np.float64)
    assert a.shape == b.shape, (name, a.shape, b.shape)
    atol = atol_frac * float(np.abs(b).max()) if b.size else 0.0
    err = np.abs(a - b)
    bound = rtol * np.abs(b) + atol
    bad = err > bound
    if bad.any():
        i = np.unravel_index(int(np.argmax(err - bound)), b.shape)
        raise AssertionError("%s: %d of %d elements outside |d| <= %.0e |x| + %.3e; worst at %s: %r vs %r"
                             % (name, int(bad.sum()), b.size, rtol, atol, i, a[i], b[i]))
