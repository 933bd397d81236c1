"""NumPy model of the stacked layout of the grouped I x I products (one
tensor-core launch for every problem of a batched eigensolve; documentation
of the layout, the GPU kernel itself is checked against the oracle in
tests/test_gpu_eigen.py): problem b's operand rows sit at row offsets ra[b]
(A, n rows) and rb[b] = 2 ra[b] (B, 2n rows) of two stacked buffers with one
common row stride ld = round_up(2 n_max, 8), zeros from K = 2n on; the work
list is the output tiles of every problem in order (prefix sums tile0); a
tile that runs past its problem's rows reads the next problem's rows, whose
outputs are not stored (so a gated-off neighbour's unwritten rows never reach a
stored value); the partials of problem b start at po[b] with rows of 2n.  The layout's sizes stay within what the batch reserve provides for nb
problems of up to I_max states."""
import numpy as np
import pytest

BM, BN, BK = 128, 80, 32


def round_up(x, m):
    return (x + m - 1) // m * m


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_stacked_tiles_reproduce_every_product(seed):
    rng = np.random.default_rng(seed)
    n = [int(v) for v in rng.integers(1, 300, size=int(rng.integers(9, 40)))]
    imax = max(n) + int(rng.integers(0, 20))
    nb = len(n)
    ld = round_up(2 * imax, 8)
    rows = sum(n)
    assert rows <= nb * imax                                   # the reserve's row bound
    A = np.full((rows, ld), np.nan)                            # unwritten memory
    B = np.full((2 * rows, ld), np.nan)
    gated = int(rng.integers(0, nb))     # a problem the device gate switches off: its
    ra, rb, po, tile0, Ab, Bb = [], [], [], [0], [], []   # rows are never written
    r = p = 0
    for b, k in enumerate(n):
        a = rng.integers(-128, 129, size=(k, 2 * k)).astype(float)   # digit values
        bm = rng.integers(-128, 129, size=(2 * k, 2 * k)).astype(float)
        ra.append(r); rb.append(2 * r); po.append(p)
        Ab.append(a); Bb.append(bm)
        tile0.append(tile0[-1] + round_up(k, BM) // BM * (round_up(2 * k, BN) // BN))
        if b == gated:
            r += k
            p += 2 * k * k
            continue
        A[r:r + k, :] = 0.0
        A[r:r + k, :2 * k] = a                                 # zeros from K = 2n on
        B[2 * r:2 * r + 2 * k, :] = 0.0
        B[2 * r:2 * r + 2 * k, :2 * k] = bm
        r += k
        p += 2 * k * k
    assert p <= nb * 2 * imax * imax                           # the reserve's partial bound
    P = np.full(p, np.nan)
    for t in range(tile0[-1]):
        b = int(np.searchsorted(tile0, t, side="right") - 1)
        if b == gated:
            continue
        k = n[b]
        mt = round_up(k, BM) // BM
        mi, nj = (t - tile0[b]) % mt, (t - tile0[b]) // mt
        m0, n0 = ra[b] + mi * BM, rb[b] + nj * BN
        kk = round_up(2 * k, BK)                               # the K blocks of the item
        def rows_of(X, r0, cnt):                               # out-of-range rows / columns: zeros
            out = np.zeros((cnt, kk))
            hi = min(r0 + cnt, X.shape[0])
            cols = min(kk, X.shape[1])
            out[:hi - r0, :cols] = X[r0:hi, :cols]
            return out
        with np.errstate(invalid="ignore"):
            D = rows_of(A, m0, BM) @ rows_of(B, n0, BN).T
        for i in range(BM):
            row = mi * BM + i
            if row >= k:
                continue
            for j in range(BN):
                col = nj * BN + j
                if col < 2 * k:
                    P[po[b] + row * 2 * k + col] = D[i, j]
    for b, k in enumerate(n):
        if b == gated:
            continue
        got = P[po[b]:po[b] + 2 * k * k].reshape(k, 2 * k)
        assert not np.isnan(got).any()                         # written, and untouched by the
                                                               # neighbours' unwritten rows
        assert np.array_equal(got, Ab[b] @ Bb[b].T)
