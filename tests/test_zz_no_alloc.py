"""sky_overlap_noalloc: the overlap matrix for callers that may not allocate
device memory (their host application's allocator owns the device budget),
so they cannot create a context.  Checked against sky_overlap, the existing
entry point, on two calls in a row (its fixed scratch array is reused)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1610_07522_gb300 import binding as B
from paper_1610_07522_gb300 import inputs as IN

pytestmark = pytest.mark.gpu


def _ref_overlap(ctx, a, b, I):
    X = torch.zeros((I, I), dtype=torch.complex128, device="cuda:0")
    B.sky_overlap(ctx, a, b, I, X)
    B.sky_sync(ctx)
    return X.cpu().numpy()


@pytest.mark.parametrize("prec", [B.SKY_F64, B.SKY_F32])
def test_noalloc_overlap_matches_context_overlap_twice(prec):
    from paper_1610_07522_gb300 import build
    build.build()
    grid, I = (16, 16, 16), 150
    V = 2 * 16 ** 3
    ctype = torch.complex128 if prec == B.SKY_F64 else torch.complex64
    stream = torch.cuda.current_stream().cuda_stream
    ctx = B.sky_init(grid, (1.0, 1.0, 1.0), IN.SLY4, False, (0.0, 0.0, 0.0), prec, I, stream)
    try:
        rng = np.random.default_rng(77)
        for call in range(2):
            a = torch.from_numpy(IN.random_spinors(grid, I, rng)).to(ctype).cuda()
            b = torch.from_numpy(IN.random_spinors(grid, I, rng)).to(ctype).cuda()
            want = _ref_overlap(ctx, a, b, I)
            X = torch.zeros((I, I), dtype=torch.complex128, device="cuda:0")
            B.sky_overlap_noalloc(a, b, I, V, 1.0, prec, X, stream)
            torch.cuda.synchronize()
            got = X.cpu().numpy()
            assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want)), call
    finally:
        B.sky_destroy(ctx)


def test_noalloc_overlap_rejects_oversize():
    X = torch.zeros(4, dtype=torch.complex128, device="cuda:0")
    with pytest.raises(B.SkyError) as ei:
        B.sky_overlap_noalloc(X, X, 1025, 8, 1.0, B.SKY_F64, X)
    assert ei.value.status == B.SKY_EINVAL
