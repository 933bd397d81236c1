"""Thin ctypes binding of libsky (include/sky.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Array
arguments may be torch tensors (their ``data_ptr()`` is passed), raw integer
device addresses, or None for nullable pointers.  A non-OK status raises
``SkyError``.  There is no fallback: if the library is missing, ``lib()``
raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

SKY_OK, SKY_EINVAL, SKY_ENOMEM, SKY_ECUDA, SKY_ENOTPD, SKY_ENOCONV, SKY_ETIMEOUT, SKY_ENAN, SKY_EUNSUPPORTED = range(9)
STATUS_NAMES = ["SKY_OK", "SKY_EINVAL", "SKY_ENOMEM", "SKY_ECUDA", "SKY_ENOTPD",
                "SKY_ENOCONV", "SKY_ETIMEOUT", "SKY_ENAN", "SKY_EUNSUPPORTED"]
SKY_F64, SKY_F32, SKY_F32_BF16X3, SKY_F32_BF16X6 = 0, 1, 2, 3
(SKY_KNOB_LINE_YZ, SKY_KNOB_LINE_X, SKY_KNOB_OVERLAP_WAVES, SKY_KNOB_TC_WAVES,
 SKY_KNOB_JACOBI_BLOCKS, SKY_KNOB_JACOBI_BLOCKS_MAX, SKY_KNOB_WAIT_SPINS,
 SKY_KNOB_JACOBI_MAX_SWEEPS, SKY_KNOB_EIGEN_METHOD, SKY_KNOB_SPLIT_GEMM,
 SKY_KNOB_LINE_ARITH, SKY_KNOB_TC_TILE_N, SKY_KNOB_FUSED_H) = range(13)
SKY_EIG_AUTO, SKY_EIG_JACOBI, SKY_EIG_TRIDIAGONAL = range(3)

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double


class SkySkyrme(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("t0", "t1", "t2", "t3", "x0", "x1", "x2", "x3", "alpha", "W0",
                 "hb2m_n", "hb2m_p", "e2")] + [("coulomb", ctypes.c_int)]


class SkyError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


_SIGNATURES = {
    "sky_init": (_I, [ctypes.POINTER(_P), ctypes.POINTER(_I), ctypes.POINTER(_D),
                      ctypes.POINTER(SkySkyrme), ctypes.POINTER(_D), _I, _I, _P]),
    "sky_destroy": (_I, [_P]),
    "sky_set_stream": (_I, [_P, _P]),
    "sky_sync": (_I, [_P]),
    "sky_last_error": (ctypes.c_char_p, [_P]),
    "sky_supported_size": (_I, [_I, _I]),
    "sky_kernel_launches": (ctypes.c_ulonglong, []),
    "sky_tri_team_plan": (_I, [_I, ctypes.POINTER(_I), _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                               ctypes.POINTER(_I)]),
    "sky_stats": (_I, [_P, ctypes.POINTER(ctypes.c_longlong), _I]),
    "sky_apply_h": (_I, [_P, _P, _P, _P, _P, _P, _I, _P, _P]),
    "sky_derivative": (_I, [_P, _I, _P, _P, _I]),
    "sky_damped_step": (_I, [_P, _I, _P, _P, _P, _P, _I, _D, _D, _P]),
    "sky_overlap": (_I, [_P, _P, _P, _I, _P]),
    "sky_orthonormalize": (_I, [_P, _P, _I, _P]),
    "sky_subspace_diag": (_I, [_P, _P, _P, _I, _P, _P]),
    "sky_rotate": (_I, [_P, _P, _P, _I, _P]),
    "sky_densities": (_I, [_P, _P, _I, _P, _P, _P, _P]),
    "sky_mean_fields": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "sky_energy": (_I, [_P, _P, _P, _P, _P]),
    "sky_sp_spread": (_I, [_P, _P, _P, _I, _P]),
    "sky_overlap_noalloc": (_I, [_P, _P, _I, ctypes.c_longlong, _D, _I, _P, _P]),
    "sky_orthonormalize_batched": (_I, [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_I), ctypes.POINTER(_P)]),
    "sky_subspace_diag_batched": (_I, [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_I),
                                       ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "sky_reserve_batch": (_I, [_P, _I]),
    "sky_subspace_diag_literal_batched": (_I, [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                               ctypes.POINTER(_I), ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "sky_set_prec": (_I, [_P, _I]),
    "sky_tune_set": (_I, [_P, _I, _I]),
    "sky_tune_get": (_I, [_P, _I]),
    "sky_net_forward": (_I, [_P, _I, _P, _P, _P, _P, _D, _P, _P]),
    "sky_net_backward": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "sky_net_adam": (_I, [_P, _P, _P, _P, _P, _I, _D, _D, _D, _D]),
    "sky_cross_overlap": (_I, [_P, _P, _P, _I, _P]),
    "sky_precond_stats": (_I, [_P, _P, _P, _P, _I, _P, _P]),
    "sky_fma_probe": (_I, [_I, _I, _I, _P, ctypes.POINTER(_D)]),
    "sky_td_taylor": (_I, [_P, _P, _P, _P, _P, _P, _P, _I, _D, _I]),
    "sky_memcpy_h2d": (_I, [_P, _P, _P, ctypes.c_size_t]),
    "sky_memcpy_d2h": (_I, [_P, _P, _P, ctypes.c_size_t]),
}

# Constants of the damping network (the #defines of include/sky.h).
SKY_NET_HIDDEN = 16
SKY_NET_NPARAM = 8673
SKY_NET_WS_PER_POINT = 69
SKY_NET_WMAX = 4.0
SKY_NET_USCALE = 50.0
SKY_NET_WSCALE = 5.0

_LIB = None


def lib_path():
    return _build.LIB


def lib():
    """Load libsky.so (built in-tree by ``build.build()``); raise if absent."""
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libsky is not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _check(ctx, st):
    if st != SKY_OK:
        msg = lib().sky_last_error(ctx).decode() if ctx else ""
        raise SkyError(st, msg)


def skyrme_struct(params, coulomb):
    s = SkySkyrme()
    for k in ("t0", "t1", "t2", "t3", "x0", "x1", "x2", "x3", "alpha", "W0", "hb2m_n", "hb2m_p", "e2"):
        setattr(s, k, float(params[k]))
    s.coulomb = 1 if coulomb else 0
    return s


def sky_init(grid, dx, params, coulomb, twist=(0.0, 0.0, 0.0), prec=SKY_F64, max_states=1, stream=0):
    ctx = _P()
    g = (_I * 3)(*[int(v) for v in grid])
    d = (_D * 3)(*[float(v) for v in dx])
    t = (_D * 3)(*[float(v) for v in twist])
    s = skyrme_struct(params, coulomb)
    st = lib().sky_init(ctypes.byref(ctx), g, d, ctypes.byref(s), t, int(prec), int(max_states),
                        _P(stream) if stream else None)
    if st != SKY_OK:
        raise SkyError(st, "sky_init failed")
    return ctx


def sky_destroy(ctx):
    _check(None, lib().sky_destroy(ctx))


def sky_set_stream(ctx, stream):
    _check(ctx, lib().sky_set_stream(ctx, _P(stream) if stream else None))


def sky_sync(ctx):
    _check(ctx, lib().sky_sync(ctx))


def sky_supported_size(n, prec):
    return bool(lib().sky_supported_size(int(n), int(prec)))


def sky_stats(ctx, reset=False):
    """Solver counters: dict of Jacobi solves / sweeps, Loewdin routes and
    tridiagonal-route eigensolves."""
    buf = (ctypes.c_longlong * 8)()
    _check(ctx, lib().sky_stats(ctx, buf, 1 if reset else 0))
    keys = ("jacobi_solves", "jacobi_sweeps", "jacobi_last_sweeps", "loewdin_calls",
            "loewdin_newton_schulz", "newton_schulz_iters", "tridiagonal_solves")
    return {k: int(buf[i]) for i, k in enumerate(keys)}


def sky_kernel_launches():
    return int(lib().sky_kernel_launches())


def sky_tri_team_plan(n, blocks):
    """The batched eigensolver's team split for problems of sizes n on
    ``blocks`` blocks (host only): (team of each problem, [(first block,
    block count) per team]), or None when the batch cannot be split."""
    np_ = len(n)
    arr = (_I * max(np_, 1))
    team, first, count = arr(), arr(), arr()
    k = lib().sky_tri_team_plan(np_, arr(*[int(x) for x in n]), int(blocks), team, first, count)
    if k <= 0:
        return None
    return [int(team[b]) for b in range(np_)], [(int(first[t]), int(count[t])) for t in range(k)]


def sky_apply_h(ctx, U, B, W, psi, hpsi, I, eps=None, hnorm2=None):
    _check(ctx, lib().sky_apply_h(ctx, _ptr(U), _ptr(B), _ptr(W), _ptr(psi), _ptr(hpsi), int(I),
                                  _ptr(eps), _ptr(hnorm2)))


def sky_derivative(ctx, axis, src, dst, n):
    _check(ctx, lib().sky_derivative(ctx, int(axis), _ptr(src), _ptr(dst), int(n)))


def sky_damped_step(ctx, q, psi, hpsi, eps, phi, I, x0, E0, w=None):
    _check(ctx, lib().sky_damped_step(ctx, int(q), _ptr(psi), _ptr(hpsi), _ptr(eps), _ptr(phi),
                                      int(I), float(x0), float(E0), _ptr(w)))


def sky_td_taylor(ctx, U, B, W, psi, out, work, I, tau, order=6):
    _check(ctx, lib().sky_td_taylor(ctx, _ptr(U), _ptr(B), _ptr(W), _ptr(psi), _ptr(out),
                                    _ptr(work), int(I), float(tau), int(order)))


def sky_overlap(ctx, a, b, I, X):
    _check(ctx, lib().sky_overlap(ctx, _ptr(a), _ptr(b), int(I), _ptr(X)))


def sky_orthonormalize(ctx, S, I, C):
    _check(ctx, lib().sky_orthonormalize(ctx, _ptr(S), int(I), _ptr(C)))


def sky_subspace_diag(ctx, H, C, I, M, eps):
    _check(ctx, lib().sky_subspace_diag(ctx, _ptr(H), _ptr(C), int(I), _ptr(M), _ptr(eps)))


def _ptrs(xs):
    return (_P * len(xs))(*[_ptr(x) for x in xs])


def sky_orthonormalize_batched(ctx, S, I, C):
    n = len(I)
    _check(ctx, lib().sky_orthonormalize_batched(ctx, n, _ptrs(S), (_I * n)(*I), _ptrs(C)))


def sky_subspace_diag_batched(ctx, H, C, I, M, eps):
    n = len(I)
    _check(ctx, lib().sky_subspace_diag_batched(ctx, n, _ptrs(H), _ptrs(C), (_I * n)(*I), _ptrs(M),
                                                _ptrs(eps)))


def sky_set_prec(ctx, prec):
    _check(ctx, lib().sky_set_prec(ctx, int(prec)))


def sky_tune_set(ctx, knob, value):
    _check(ctx, lib().sky_tune_set(ctx, int(knob), int(value)))


def sky_tune_get(ctx, knob):
    return int(lib().sky_tune_get(ctx, int(knob)))


def sky_reserve_batch(ctx, nb):
    _check(ctx, lib().sky_reserve_batch(ctx, int(nb)))


def sky_subspace_diag_literal_batched(ctx, H, C, I, M, eps):
    n = len(I)
    _check(ctx, lib().sky_subspace_diag_literal_batched(ctx, n, _ptrs(H), _ptrs(C), (_I * n)(*I),
                                                        _ptrs(M), _ptrs(eps)))


def sky_rotate(ctx, phi, M, I, psi_out):
    _check(ctx, lib().sky_rotate(ctx, _ptr(phi), _ptr(M), int(I), _ptr(psi_out)))


def sky_densities(ctx, psi, I, rho, tau, J, divJ):
    _check(ctx, lib().sky_densities(ctx, _ptr(psi), int(I), _ptr(rho), _ptr(tau), _ptr(J), _ptr(divJ)))


def sky_mean_fields(ctx, rho, tau, divJ, U, B, W):
    _check(ctx, lib().sky_mean_fields(ctx, _ptr(rho), _ptr(tau), _ptr(divJ), _ptr(U), _ptr(B), _ptr(W)))


def sky_energy(ctx, rho, tau, divJ, out):
    _check(ctx, lib().sky_energy(ctx, _ptr(rho), _ptr(tau), _ptr(divJ), _ptr(out)))


def sky_sp_spread(ctx, eps, hnorm2, A, out):
    _check(ctx, lib().sky_sp_spread(ctx, _ptr(eps), _ptr(hnorm2), int(A), _ptr(out)))


def sky_overlap_noalloc(a, b, I, V, dV, prec, X, stream=0):
    """Overlap matrix with no context and no device allocation (include/sky.h)."""
    st = lib().sky_overlap_noalloc(_ptr(a), _ptr(b), int(I), int(V), float(dV), int(prec), _ptr(X),
                                   _P(stream) if stream else None)
    if st != SKY_OK:
        raise SkyError(st, "sky_overlap_noalloc failed")


def sky_net_forward(ctx, q, theta, U, B, W, ws, w, scale=1.0):
    _check(ctx, lib().sky_net_forward(ctx, int(q), _ptr(theta), _ptr(U), _ptr(B), _ptr(W),
                                      float(scale), _ptr(ws), _ptr(w)))


def sky_net_backward(ctx, theta, ws, abc, norm, grad, loss):
    _check(ctx, lib().sky_net_backward(ctx, _ptr(theta), _ptr(ws), _ptr(abc), _ptr(norm),
                                       _ptr(grad), _ptr(loss)))


def sky_net_adam(ctx, theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    _check(ctx, lib().sky_net_adam(ctx, _ptr(theta), _ptr(grad), _ptr(m), _ptr(v), int(step),
                                   float(lr), float(beta1), float(beta2), float(eps)))


def sky_cross_overlap(ctx, a, b, I, X):
    _check(ctx, lib().sky_cross_overlap(ctx, _ptr(a), _ptr(b), int(I), _ptr(X)))


def sky_precond_stats(ctx, psi, phi, ppsi, I, abc, norm):
    _check(ctx, lib().sky_precond_stats(ctx, _ptr(psi), _ptr(phi), _ptr(ppsi), int(I), _ptr(abc),
                                        _ptr(norm)))


def sky_fma_probe(fp64, blocks_per_sm, iters, stream=0):
    """Enqueue the FMA-chain probe kernel; returns the flops it executes."""
    f = _D(0.0)
    st = lib().sky_fma_probe(int(bool(fp64)), int(blocks_per_sm), int(iters),
                             _P(stream) if stream else None, ctypes.byref(f))
    if st != SKY_OK:
        raise SkyError(st, "sky_fma_probe failed")
    return f.value


def _nbytes(t):
    return t.numel() * t.element_size()


def sky_memcpy_h2d(ctx, dst, src):
    """Copy the host tensor src into the device tensor dst on the context stream."""
    n = _nbytes(src)
    if _nbytes(dst) != n:
        raise ValueError("sky_memcpy_h2d: size mismatch")
    _check(ctx, lib().sky_memcpy_h2d(ctx, _ptr(dst), _ptr(src), n))


def sky_memcpy_d2h(ctx, dst, src):
    """Copy the device tensor src into the host tensor dst on the context stream."""
    n = _nbytes(src)
    if _nbytes(dst) != n:
        raise ValueError("sky_memcpy_d2h: size mismatch")
    _check(ctx, lib().sky_memcpy_d2h(ctx, _ptr(dst), _ptr(src), n))
