"""sky_overlap_noalloc: the overlap matrix for callers that may not allocate
device memory (their host application's allocator owns the device budget),
so they cannot create a context.  Checked against the FP64 oracle on two
calls in a row (its fixed scratch array is reused), at the largest state
count the array admits (I = 1024: one K split) and at counts where the
array, not the SM count, limits the K splits; and checked to allocate
nothing (free device memory unchanged across a call)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_1610_07522_gb300 import binding as B
from paper_1610_07522_gb300 import inputs as IN

pytestmark = pytest.mark.gpu


def _rel(got, want):
    return float(np.max(np.abs(got - want)) / np.max(np.abs(want)))


# (grid, I): 16^3 with the SM count limiting the splits; 8^3 (V = 1024) with
# I = 1024 (array fits one split) and I = 600 (array fits two, fewer than the
# SMs ask for)
CASES = [((16, 16, 16), 150), ((8, 8, 8), 1024), ((8, 8, 8), 600)]


@pytest.mark.parametrize("prec", [B.SKY_F64, B.SKY_F32])
@pytest.mark.parametrize("grid,I", CASES)
def test_noalloc_overlap_matches_oracle_twice(prec, grid, I):
    from paper_1610_07522_gb300 import build
    build.build()
    g = O.Grid(grid, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    V = 2 * g.G
    ctype = torch.complex128 if prec == B.SKY_F64 else torch.complex64
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(77 + I)
    for call in range(2):
        a = IN.random_spinors(grid, I, rng)
        b = IN.random_spinors(grid, I, rng)
        if prec == B.SKY_F32:
            a = a.astype(np.complex64).astype(np.complex128)
            b = b.astype(np.complex64).astype(np.complex128)
        da = torch.from_numpy(a).to(ctype).cuda()
        db = torch.from_numpy(b).to(ctype).cuda()
        X = torch.zeros((I, I), dtype=torch.complex128, device="cuda:0")
        B.sky_overlap_noalloc(da, db, I, V, g.dV, prec, X, stream)
        torch.cuda.synchronize()
        # FP64 accumulation in both precisions (FP32 inputs widened exactly)
        assert _rel(X.cpu().numpy(), O.overlap(a, b, g)) <= 1e-12, call


def test_noalloc_overlap_allocates_nothing():
    grid, I = (16, 16, 16), 200
    V = 2 * 16 ** 3
    rng = np.random.default_rng(5)
    a = torch.from_numpy(IN.random_spinors(grid, I, rng)).cuda()
    X = torch.zeros((I, I), dtype=torch.complex128, device="cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    B.sky_overlap_noalloc(a, a, I, V, 1.0, B.SKY_F64, X, stream)   # first call: loads the code
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        B.sky_overlap_noalloc(a, a, I, V, 1.0, B.SKY_F64, X, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_overlap_rejects_oversize():
    X = torch.zeros(4, dtype=torch.complex128, device="cuda:0")
    with pytest.raises(B.SkyError) as ei:
        B.sky_overlap_noalloc(X, X, 1025, 8, 1.0, B.SKY_F64, X)
    assert ei.value.status == B.SKY_EINVAL
