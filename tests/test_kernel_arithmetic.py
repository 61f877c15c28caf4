"""Integer results that the kernels take from FP32 arithmetic, checked on the
host against their exact definitions (numpy reproduces the FP32 operations:
one correctly rounded multiply, a truncating conversion, integer fixes).

The diagnostics push bins an O- particle of cell c into the x bin
floor(c X / N) of the f-(E, x) histogram (X bins over N cells) without an
integer division: an estimate (int)(fl(c X) * fl(1/N)) in FP32, corrected by
one step up or down.  The host accepts N <= 4096 and X N <= 16384 N, so
c X < 2^26, and the estimate is within one of the exact quotient."""
import numpy as np


def _xbin_kernel(c, X, N):
    pr = (c * X).astype(np.int64)
    rN = np.float32(1.0) / np.float32(N)
    est = (pr.astype(np.float32) * rN).astype(np.float32)
    xb = np.trunc(est).astype(np.int64)
    xb = xb + ((xb + 1) * N <= pr)
    xb = xb - (xb * N > pr)
    return xb, np.trunc(est).astype(np.int64)


def test_fm_x_bin_equals_the_integer_quotient():
    rng = np.random.default_rng(5)
    Ns = [2, 3, 7, 64, 127, 128, 129, 500, 512, 1000, 2047, 4095, 4096]
    Xs = [1, 2, 3, 7, 10, 64, 100, 128, 1000, 4096, 16384]
    for N in Ns:
        c = np.arange(N, dtype=np.int64)
        for X in Xs:
            xb, est = _xbin_kernel(c, X, N)
            exact = (c * X) // N
            assert np.array_equal(xb, exact), (N, X)
            # the estimate alone is never off by more than one
            assert np.max(np.abs(est - exact)) <= 1, (N, X)
    # random (N, X) pairs within the host's limits
    for _ in range(200):
        N = int(rng.integers(2, 4097))
        X = int(rng.integers(1, 16385))
        c = np.arange(N, dtype=np.int64)
        xb, est = _xbin_kernel(c, X, N)
        assert np.array_equal(xb, (c * X) // N), (N, X)
        assert np.max(np.abs(est - (c * X) // N)) <= 1, (N, X)
