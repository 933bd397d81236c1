"""The exact-integer split GEMMs of the FP64 and FP32 forms (tensor cores)
against the FP64 oracle: the overlap / Hamiltonian matrices (Eqs.
normmatrix, hammatrix) and the recombination (Sec. 3.3.3).

Each operand row is scaled by a power of two and cut into signed 8-bit
digits; digit products are summed exactly in FP32 over segments of 128
values of K.  Cases: ragged state counts around the 128-row and 80/96-column
tiles, K and row chunks forced by a small digit buffer (SKY_OZ_MB), the
FP64 FMA kernels selected by SKY_KNOB_SPLIT_GEMM = 0, and an exactness pin:
operands whose digits all fit in the kept digit products give the exact
integer result.  Tolerances: FP64 form 1e-12 of the largest element (as for
every FP64 call), FP32 form 1e-8 for the matrices (the FP32-rounded inputs,
digits to 2^-32) and 2^-23 for the recombined states, which are stored in FP32.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_1610_07522_gb300 import binding as B
from paper_1610_07522_gb300 import inputs as IN

pytestmark = pytest.mark.gpu

P = dict(IN.SLY4)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def relerr(got, want):
    return float(np.max(np.abs(got - want)) / max(np.max(np.abs(want)), 1e-300))


def make_ctx(grid, prec, I, twist=(0.0, 0.0, 0.0)):
    return B.sky_init(grid, (1.0, 1.0, 1.0), P, False, twist, prec, I,
                      torch.cuda.current_stream().cuda_stream)


def _states(grid, I, rng, prec):
    a = IN.random_spinors(grid, I, rng)
    if prec == B.SKY_F32:
        a = a.astype(np.complex64).astype(np.complex128)
    return a


def _dt(prec):
    return torch.complex128 if prec == B.SKY_F64 else torch.complex64


TOL = {B.SKY_F64: 1e-12, B.SKY_F32: 1e-8}
# the FP32 form stores the recombined states in FP32: half an ulp, 2^-24 relative
TOL_OUT = {B.SKY_F64: 1e-12, B.SKY_F32: 2.0 ** -23}


@pytest.mark.parametrize("prec", [B.SKY_F64, B.SKY_F32])
@pytest.mark.parametrize("grid,I", [((8, 8, 8), 1), ((16, 16, 16), 2), ((16, 16, 16), 37),
                                    ((12, 16, 20), 129), ((16, 16, 16), 300)])
def test_overlap_matches_oracle(prec, grid, I):
    rng = np.random.default_rng(100 + I)
    g = O.Grid(grid, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    a, b = _states(grid, I, rng, prec), _states(grid, I, rng, prec)
    c = make_ctx(grid, prec, I)
    try:
        assert B.sky_tune_get(c, B.SKY_KNOB_SPLIT_GEMM) == 1
        X = torch.zeros((I, I), dtype=torch.complex128, device="cuda:0")
        da, db = dev(a).to(_dt(prec)), dev(b).to(_dt(prec))
        B.sky_overlap(c, da, db, I, X)
        B.sky_sync(c)
        assert relerr(host(X), O.overlap(a, b, g)) < TOL[prec]
        B.sky_overlap(c, da, da, I, X)
        B.sky_sync(c)
        Xh = host(X)
        assert relerr(Xh, O.overlap(a, a, g)) < TOL[prec]
        assert np.array_equal(Xh, Xh.conj().T)      # mirrored lower triangle
    finally:
        B.sky_destroy(c)


@pytest.mark.parametrize("prec", [B.SKY_F64, B.SKY_F32])
@pytest.mark.parametrize("I", [1, 3, 40, 129, 300])
def test_rotate_matches_oracle(prec, I):
    rng = np.random.default_rng(200 + I)
    grid = (16, 16, 16)
    phi = _states(grid, I, rng, prec)
    M = rng.standard_normal((I, I)) + 1j * rng.standard_normal((I, I))
    c = make_ctx(grid, prec, I)
    try:
        out = torch.zeros(phi.shape, dtype=_dt(prec), device="cuda:0")
        B.sky_rotate(c, dev(phi).to(_dt(prec)), dev(M), I, out)
        B.sky_sync(c)
        assert relerr(host(out).astype(np.complex128), O.rotate(phi, M)) < TOL_OUT[prec]
    finally:
        B.sky_destroy(c)


def test_chunked_buffers_give_the_same_result(monkeypatch):
    """A 2 MiB digit buffer: the overlap runs in K chunks accumulated into X,
    the recombination in chunks of grid points."""
    rng = np.random.default_rng(7)
    grid, I = (24, 24, 24), 61
    g = O.Grid(grid, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    a, b = IN.random_spinors(grid, I, rng), IN.random_spinors(grid, I, rng)
    M = rng.standard_normal((I, I)) + 1j * rng.standard_normal((I, I))
    monkeypatch.setenv("SKY_OZ_MB", "2")
    c = make_ctx(grid, B.SKY_F64, I)
    try:
        X = torch.zeros((I, I), dtype=torch.complex128, device="cuda:0")
        B.sky_overlap(c, dev(a), dev(b), I, X)
        B.sky_sync(c)
        assert relerr(host(X), O.overlap(a, b, g)) < 1e-12
        out = torch.zeros(a.shape, dtype=torch.complex128, device="cuda:0")
        B.sky_rotate(c, dev(a), dev(M), I, out)
        B.sky_sync(c)
        assert relerr(host(out), O.rotate(a, M)) < 1e-12
    finally:
        B.sky_destroy(c)


def test_fma_kernels_by_knob_agree():
    rng = np.random.default_rng(8)
    grid, I = (16, 16, 16), 50
    g = O.Grid(grid, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    a, b = IN.random_spinors(grid, I, rng), IN.random_spinors(grid, I, rng)
    c = make_ctx(grid, B.SKY_F64, I)
    try:
        got = {}
        for knob in (0, 1):
            B.sky_tune_set(c, B.SKY_KNOB_SPLIT_GEMM, knob)
            assert B.sky_tune_get(c, B.SKY_KNOB_SPLIT_GEMM) == knob
            X = torch.zeros((I, I), dtype=torch.complex128, device="cuda:0")
            B.sky_overlap(c, dev(a), dev(b), I, X)
            B.sky_sync(c)
            got[knob] = host(X)
        want = O.overlap(a, b, g)
        assert relerr(got[0], want) < 1e-12 and relerr(got[1], want) < 1e-12
        with pytest.raises(B.SkyError):
            B.sky_tune_set(c, B.SKY_KNOB_SPLIT_GEMM, 2)
    finally:
        B.sky_destroy(c)


@pytest.mark.parametrize("grid,bits", [((24, 24, 24), 8), ((16, 16, 16), 15)])
def test_integer_operands_are_exact(grid, bits):
    """Entries k 2^-(bits+1) with integers |k| < 2^bits, every row holding the
    largest k: each entry is one (bits = 8) or two (bits = 15) digits of its
    row, all their digit products are kept and every segment sum is an exact
    FP32 integer, so the result equals the exact integer product bit for bit
    (K = 4G = 55296 values on 24^3, 16384 on 16^3)."""
    rng = np.random.default_rng(9 + bits)
    I = 45
    shape = (I, 2) + tuple(reversed(grid))
    km = 2 ** bits - 1
    ka = rng.integers(-km, km + 1, size=shape) + 1j * rng.integers(-km, km + 1, size=shape)
    kb = rng.integers(-km, km + 1, size=shape) + 1j * rng.integers(-km, km + 1, size=shape)
    ka[:, 0, 0, 0, 0] = km   # the same row maximum in every row
    kb[:, 0, 0, 0, 0] = km
    sc = 2.0 ** -(bits + 1)
    a, b = ka * sc, kb * sc
    A = ka.reshape(I, -1)
    Bm = kb.reshape(I, -1)
    Ar, Ai = A.real.astype(np.int64), A.imag.astype(np.int64)
    Br, Bi = Bm.real.astype(np.int64), Bm.imag.astype(np.int64)
    re = Ar @ Br.T + Ai @ Bi.T          # exact: |sum| < 2 K 2^(2 bits) < 2^53
    im = Ar @ Bi.T - Ai @ Br.T
    want = (re.astype(np.float64) + 1j * im.astype(np.float64)) * sc * sc
    want = np.tril(want) + np.conj(np.tril(want, -1)).T
    c = make_ctx(grid, B.SKY_F64, I)
    try:
        X = torch.zeros((I, I), dtype=torch.complex128, device="cuda:0")
        B.sky_overlap(c, dev(a), dev(b), I, X)
        B.sky_sync(c)
        assert np.array_equal(host(X), want)
    finally:
        B.sky_destroy(c)


@pytest.mark.parametrize("I", [200, 413, 800])
@pytest.mark.parametrize("near_identity", [True, False])
def test_large_loewdin_and_ritz_products_on_the_tensor_cores(I, near_identity):
    """From 192 states on, the I x I complex products of the Rayleigh-Ritz
    step, and from 768 on also the device-gated ones of the Loewdin factor
    (Newton-Schulz when S is near the identity, else the eigendecomposition
    route, the Newton-Schulz products then gated off on the device), run as
    digit-split tensor-core products; against the oracle's
    eigendecomposition-based Loewdin and Ritz."""
    rng = np.random.default_rng(300 + I + near_identity)
    A = rng.standard_normal((I, I)) + 1j * rng.standard_normal((I, I))
    Hm = A + A.conj().T
    if near_identity:
        S = np.eye(I) + 0.02 * Hm / np.sqrt(I)
    else:
        X = rng.standard_normal((I, I)) + 1j * rng.standard_normal((I, I))
        S = X @ X.conj().T / I + 0.05 * np.eye(I)
    H = 30.0 * Hm / np.sqrt(I)
    H = S @ H @ S          # a Hamiltonian matrix in the non-orthonormal basis
    H = 0.5 * (H + H.conj().T)
    C_w = O.loewdin(S)
    M_w, lam_w = O.rayleigh_ritz(S, H)
    c = make_ctx((8, 8, 8), B.SKY_F64, I)
    try:
        dS, dH = dev(S), dev(H)
        C = torch.zeros_like(dS)
        M = torch.zeros_like(dS)
        lam = torch.zeros(I, dtype=torch.float64, device="cuda:0")
        B.sky_orthonormalize(c, dS, I, C)
        B.sky_subspace_diag(c, dH, C, I, M, lam)
        B.sky_sync(c)
        Cg, Mg, lg = host(C), host(M), host(lam)
        assert relerr(Cg, C_w) < 1e-10
        nrm = max(1.0, float(np.max(np.abs(lam_w))))
        assert np.max(np.abs(lg - lam_w)) < 1e-10 * nrm
        assert np.max(np.abs(Mg.conj().T @ S @ Mg - np.eye(I))) < 1e-10
    finally:
        B.sky_destroy(c)
