"""NumPy models of the tridiagonal eigensolver's algorithmic choices (CPU).

These check the design of the GPU route on small matrices, independently of
the CUDA code: the one-barrier-per-step distribution of the Householder
reduction (blocks own columns cyclically, owners publish p = A v and the next
column, every block rebuilds the column and reflector itself), the
division-free Sturm count (leading-minor recurrence with power-of-two
rescaling) against the LDL^T pivot count, and inverse iteration followed by
windowed first-order Loewdin steps.  The reference values are numpy's
eigenvalues of the same matrices."""
import numpy as np
import pytest


def _herm(rng, n, kind="random"):
    if kind == "random":
        a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        return (a + a.conj().T) / 2
    q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    c = np.sort(rng.uniform(-60.0, 40.0, (n + 1) // 2))
    sp = 10.0 ** rng.uniform(-12.0, -3.0, c.size)
    ev = np.concatenate([c - sp / 2, c + sp / 2])[:n]
    h = (q * ev) @ q.conj().T
    return (h + h.conj().T) / 2


def _reflector(col, t, n):
    """Reflector t from column t (rows t+1..n-1): beta, tau, v (v[t+1] = 1)."""
    alpha = col[t + 1]
    sigma = float(np.sum(np.abs(col[t + 2:]) ** 2))
    v = np.zeros(n, complex)
    v[t + 1] = 1.0
    if sigma == 0.0 and alpha.imag == 0.0:
        return alpha.real, 0j, v
    nr = np.sqrt(abs(alpha) ** 2 + sigma)
    beta = -nr if alpha.real >= 0 else nr
    tau = complex((beta - alpha.real) / beta, -alpha.imag / beta)
    v[t + 2:] = col[t + 2:] / (alpha - beta)
    return beta, tau, v


def distributed_tridiag(A, G):
    """Householder reduction with G 'blocks' and one exchange per step."""
    n = A.shape[0]
    own = {j: np.conj(A[j, :]).copy() for j in range(n)}          # column j, owner j % G
    d, e = np.zeros(n), np.zeros(max(n - 1, 0))
    V, taus = np.zeros((n, n), complex), np.zeros(n, complex)
    P, Cb = np.zeros(n, complex), np.zeros(n, complex)              # published last step
    v_old = w = None
    tau_old = 0j
    for t in range(n):
        # head (every block alike)
        if t == 0:
            col = np.conj(A[0, :]).copy()
        else:
            s = float(np.real(np.vdot(v_old[t:], P[t:])))
            w = np.zeros(n, complex)
            w[t:] = tau_old * P[t:] - 0.5 * abs(tau_old) ** 2 * s * v_old[t:]
            col = np.zeros(n, complex)
            col[t:] = Cb[t:] - v_old[t:] * np.conj(w[t]) - w[t:]
        d[t] = col[t].real
        if t <= n - 2:
            e[t], tau_new, v_new = _reflector(col, t, n)
            V[t], taus[t] = v_new, tau_new
        # body (owners of columns j >= t+1), results published after the exchange
        newP, newCb = np.zeros(n, complex), np.zeros(n, complex)
        for g in range(G):
            for j in range(g, n, G):
                if j < t + 1 or t > n - 2:
                    continue
                a = own[j]
                if t >= 1:
                    a[t + 1:] -= v_old[t + 1:] * np.conj(w[j]) + w[t + 1:] * np.conj(v_old[j])
                newP[j] = np.vdot(a[t + 1:], v_new[t + 1:])
                if j == t + 1:
                    newCb[t + 1:] = a[t + 1:]
        if t <= n - 2:
            P, Cb, v_old, tau_old = newP, newCb, v_new, tau_new
    return d, e, V, taus


def q_from_reflectors(V, taus):
    n = V.shape[0]
    Q = np.eye(n, dtype=complex)
    for k in range(n - 2, -1, -1):
        v = V[k]
        Q = Q - taus[k] * np.outer(v, np.conj(v) @ Q)
    return Q


@pytest.mark.parametrize("n,G", [(1, 2), (2, 2), (3, 3), (17, 5), (40, 7), (64, 152)])
def test_distributed_householder_reduction(n, G):
    rng = np.random.default_rng(n * 10 + G)
    A = _herm(rng, n)
    d, e, V, taus = distributed_tridiag(A, G)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    Q = q_from_reflectors(V, taus)
    assert np.max(np.abs(Q.conj().T @ Q - np.eye(n))) < 1e-13
    assert np.max(np.abs(Q @ T @ Q.conj().T - A)) < 1e-13 * max(1.0, np.max(np.abs(A)))


def sturm_pivots(d, e2, x, pivmin):
    q = d[0] - x
    q = -pivmin if abs(q) < pivmin else q
    c = int(q < 0)
    for i in range(1, len(d)):
        q = (d[i] - x) - e2[i - 1] / q
        q = -pivmin if abs(q) < pivmin else q
        c += q < 0
    return c


def sturm_minors(d, e2, x):
    """Sign changes of p_0 = 1, p_k = (d_k - x) p_{k-1} - e2_{k-1} p_{k-2}."""
    p2, p1 = 1.0, d[0] - x
    if p1 == 0.0:
        p1 = -2.0 ** -600
    c = int(np.signbit(p1))
    for i in range(1, len(d)):
        p = (d[i] - x) * p1 - e2[i - 1] * p2
        if p == 0.0:
            p = -np.copysign(2.0 ** -600 * abs(p1), p1)
        c += int(np.signbit(p) != np.signbit(p1))
        p2, p1 = p1, p
        ex = max(np.frexp(p1)[1], np.frexp(p2)[1])
        if ex > 500 or ex < -500:
            p1, p2 = np.ldexp(p1, -ex), np.ldexp(p2, -ex)
    return c


@pytest.mark.parametrize("kind", ["random", "pairs"])
def test_division_free_sturm_count(kind):
    rng = np.random.default_rng(3 if kind == "random" else 4)
    n = 120
    A = _herm(rng, n, kind) * (1.0 if kind == "pairs" else 25.0)
    d, e, _, _ = distributed_tridiag(A, 8)
    e2 = e * e
    lam = np.linalg.eigvalsh(A)
    nrm = np.max(np.abs(lam))
    xs = np.concatenate([rng.uniform(lam[0] - 5, lam[-1] + 5, 150), lam + 1e-9 * nrm,
                         lam - 1e-9 * nrm])
    for x in xs:
        c = sturm_minors(d, e2, x)
        assert c == sturm_pivots(d, e2, x, 1e-30 * nrm)
        assert c == int(np.sum(lam < x))                       # away from eigenvalues
    # growth far beyond the double range is absorbed by the rescaling
    big = sturm_minors(d * 1e3, e2 * 1e6, 0.0)
    assert big == int(np.sum(lam * 1e3 < 0.0))


def inverse_iteration(d, e, lam, tight_rel=1e-9, iters=3):
    n = len(d)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    nrm = max(abs(lam[0]), abs(lam[-1]))
    rng = np.random.default_rng(0)
    Y = np.zeros((n, n))
    j = 0
    while j < n:
        end = j + 1
        while end < n and lam[end] - lam[end - 1] <= tight_rel * nrm:
            end += 1
        for k in range(j, end):
            y = rng.uniform(-1, 1, n)
            M = T - lam[k] * np.eye(n)
            for it in range(iters):
                try:
                    y = np.linalg.solve(M, y)
                except np.linalg.LinAlgError:      # an exactly singular shift
                    y = np.linalg.solve(M + 2.2e-16 * nrm * np.eye(n), y)
                for c in range(j, k):
                    y -= (Y[:, c] @ y) * Y[:, c]
                y /= np.max(np.abs(y)) if it + 1 < iters else np.linalg.norm(y)
            Y[:, k] = y
        j = end
    return Y


def window_loewdin(Y, lam, rel=0.05, kmax=128, passes=2):
    n = len(lam)
    gw = rel * max(abs(lam[0]), abs(lam[-1]))
    for _ in range(passes):
        Yn = np.empty_like(Y)
        for j in range(n):
            lo, hi = j, j
            while lo > 0 and j - lo < kmax and lam[j] - lam[lo - 1] <= gw:
                lo -= 1
            while hi < n - 1 and hi - j < kmax and lam[hi + 1] - lam[j] <= gw:
                hi += 1
            idx = np.arange(lo, hi + 1)
            g = Y[:, idx].T @ Y[:, j]
            coef = -0.5 * g
            coef[idx == j] = 1.5 - 0.5 * g[idx == j]
            Yn[:, j] = Y[:, idx] @ coef
        Y = Yn
    return Y


@pytest.mark.parametrize("kind", ["random", "pairs"])
def test_inverse_iteration_and_windowed_loewdin(kind):
    rng = np.random.default_rng(7 if kind == "random" else 8)
    n = 90
    A = _herm(rng, n, kind)
    d, e, V, taus = distributed_tridiag(A, 6)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    lam = np.linalg.eigvalsh(T)
    nrm = np.max(np.abs(lam))
    Y = window_loewdin(inverse_iteration(d, e, lam), lam)
    assert np.max(np.abs(Y.T @ Y - np.eye(n))) < 1e-13
    assert np.max(np.abs(T @ Y - Y * lam)) < 1e-12 * nrm
    Z = q_from_reflectors(V, taus) @ Y
    assert np.max(np.abs(A @ Z - Z * lam)) < 1e-12 * nrm
