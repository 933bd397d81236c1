"""Plain FP64 CPU oracle of the learned damping weight: the per-voxel
correction w_q(r) of the damped gradient step (Sec. 2.2, Eq. dampstep) made
by a small periodic 3D convolutional network from the local mean field.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or call this module.  It imports
nothing from the product package and shares no code with the CUDA path.

The paper has no learned part; this is an extension of its step.  With w
the damped step reads

    phi_a(r) = psi_a(r) - w_q(r) x0 [ (E0 + T)^{-1} (h - eps_a) psi_a ](r),

so w = 1 is the paper's step and any w leaves the fixed point unchanged
(where (h - eps_a) psi_a = 0 the update vanishes for every w).

Network (all convolutions 3x3x3, periodic, cross-correlation):
    x   = features(U_q, B_q, |W_q|)            3 channels
    h1  = tanh(conv(x;  W1, b1))               16 channels
    h2  = tanh(conv(h1; W2, b2))               16 channels
    z   = conv(h2; W3, b3)                      1 channel
    w   = WMAX * sigmoid(z)
conv(x; W, b)_o(r) = b_o + sum_i sum_d W[o, i, d] x_i(r + d), d in {-1,0,1}^3,
tap index t = 9 (dz+1) + 3 (dy+1) + (dx+1).

Training objective (one-step error, separable form): with g_a = psi_a - phi_a
the plain step (w = 1) and d_a = (1 - P*) psi_a the part of psi_a outside
the converged occupied space (P* its projector), the step with w leaves
e_a = d_a - w g_a.  Summed over states and spin:
    sum_a |e_a(r)|^2 = a(r) w(r)^2 - 2 b(r) w(r) + c(r),
    a = sum |g|^2,  b = sum Re(conj(g) d),  c = sum |d|^2,
and the loss of one sample is L = sum_r (a w^2 - 2 b w + c) / sum_r c, so
L = 1 at w = 0 and L is minimal at w = b/a voxel by voxel.

Parameter vector order: W1 [16,3,27], b1 [16], W2 [16,16,27], b2 [16],
W3 [1,16,27], b3 [1]  (8673 numbers).

Pins (tests/test_oracle_precond.py): the convolution against a brute-force
loop with modular indices; translation equivariance; a one-hot kernel is a
lattice shift; every gradient against central finite differences; the loss
at w = 0 and its voxel-wise minimum; the first Adam step (-lr sign(g)); the
weighted step against the unweighted one (w = 1) and its linearity in w;
the statistics a, b, c in the cases P* psi = psi and P* psi = 0.
"""
from __future__ import annotations

import numpy as np

HIDDEN = 16
CIN = 3
WMAX = 4.0
U_SCALE = 50.0     # MeV
W_SCALE = 5.0      # MeV fm
SHAPES = [("W1", (HIDDEN, CIN, 27)), ("b1", (HIDDEN,)),
          ("W2", (HIDDEN, HIDDEN, 27)), ("b2", (HIDDEN,)),
          ("W3", (1, HIDDEN, 27)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def taps():
    """(t, dz, dy, dx) for the 27 taps, t = 9 (dz+1) + 3 (dy+1) + (dx+1)."""
    out = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                out.append((9 * (dz + 1) + 3 * (dy + 1) + (dx + 1), dz, dy, dx))
    return out


def unpack(theta):
    """Flat parameter vector -> dict of arrays (views, float64)."""
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = theta[o:o + n].reshape(shape)
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).reshape(-1)
                           for name, _ in SHAPES])


def features(U, B, W, hb2m):
    """Input channels from the mean field of one species: U/50 MeV,
    B/(hbar^2/2m) - 1 and |W|/(5 MeV fm).  U, B [nz,ny,nx]; W [3,nz,ny,nx]."""
    return np.stack([U / U_SCALE, B / hb2m - 1.0, np.sqrt(np.sum(W * W, axis=0)) / W_SCALE])


def shifted(x, dz, dy, dx):
    """y(r) = x(r + d) on the periodic grid (x has [..., nz, ny, nx])."""
    return np.roll(x, shift=(-dz, -dy, -dx), axis=(-3, -2, -1))


def conv(x, Wt, b):
    """Periodic 3x3x3 cross-correlation: out_o(r) = b_o + sum_{i,d} W[o,i,t(d)] x_i(r+d)."""
    out = np.zeros((Wt.shape[0],) + x.shape[1:])
    out += np.asarray(b)[:, None, None, None]
    for t, dz, dy, dx in taps():
        xs = shifted(x, dz, dy, dx)
        out += np.einsum("oi,izyx->ozyx", Wt[:, :, t], xs)
    return out


def conv_input_grad(dout, Wt):
    """d/dx_i of sum_o <dout_o, conv(x)_o>: sum_{o,d} W[o,i,t(d)] dout_o(r - d)."""
    din = np.zeros((Wt.shape[1],) + dout.shape[1:])
    for t, dz, dy, dx in taps():
        ds = shifted(dout, -dz, -dy, -dx)
        din += np.einsum("oi,ozyx->izyx", Wt[:, :, t], ds)
    return din


def conv_weight_grad(dout, x):
    """d/dW[o,i,t] = sum_r dout_o(r) x_i(r+d);  d/db_o = sum_r dout_o(r)."""
    dW = np.zeros((dout.shape[0], x.shape[0], 27))
    for t, dz, dy, dx in taps():
        xs = shifted(x, dz, dy, dx)
        dW[:, :, t] = np.einsum("ozyx,izyx->oi", dout, xs)
    return dW, dout.sum(axis=(1, 2, 3))


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(theta, x):
    """Weight w [nz,ny,nx] and the activations needed by ``backward``."""
    P = unpack(theta)
    h1 = np.tanh(conv(x, P["W1"], P["b1"]))
    h2 = np.tanh(conv(h1, P["W2"], P["b2"]))
    z = conv(h2, P["W3"], P["b3"])[0]
    w = WMAX * sigmoid(z)
    return w, {"x": x, "h1": h1, "h2": h2, "z": z}


def loss(w, abc):
    """L = sum_r (a w^2 - 2 b w + c) / sum_r c for one sample."""
    a, b, c = abc
    return float(np.sum(a * w * w - 2.0 * b * w + c) / np.sum(c))


def backward(theta, w, cache, abc):
    """Gradient of ``loss(forward(theta, x), abc)`` with respect to theta
    (flat, the order of ``SHAPES``) by the chain rule through each layer."""
    P = unpack(theta)
    a, b, c = abc
    dw = 2.0 * (a * w - b) / np.sum(c)
    dz = (dw * w * (1.0 - w / WMAX))[None]               # d sigmoid
    dW3, db3 = conv_weight_grad(dz, cache["h2"])
    dh2 = conv_input_grad(dz, P["W3"]) * (1.0 - cache["h2"] ** 2)
    dW2, db2 = conv_weight_grad(dh2, cache["h1"])
    dh1 = conv_input_grad(dh2, P["W2"]) * (1.0 - cache["h1"] ** 2)
    dW1, db1 = conv_weight_grad(dh1, cache["x"])
    return pack({"W1": dW1, "b1": db1, "W2": dW2, "b2": db2, "W3": dW3, "b3": db3})


def adam(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015, Algorithm 1) with bias correction;
    ``step`` counts from 1.  Returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def weighted_damped_step(psi, phi_plain, w):
    """phi_w = psi - w (psi - phi_plain): the damped step of Eq. dampstep with
    its update scaled voxel by voxel (same w for both spin components)."""
    return psi - w[None, None] * (psi - phi_plain)


def stats(psi, phi_plain, psi_star, dV):
    """Per-voxel a, b, c of the training objective for one species.
    psi, phi_plain, psi_star: [I, 2, nz, ny, nx]; psi_star orthonormal.
    P* psi_a = sum_b psi*_b <psi*_b | psi_a>."""
    I = psi.shape[0]
    Ps = psi_star.reshape(psi_star.shape[0], -1)
    Pm = psi.reshape(I, -1)
    O = dV * (np.conj(Ps) @ Pm.T)                      # O[b, a] = <psi*_b | psi_a>
    proj = (Ps.T @ O).T.reshape(psi.shape)             # sum_b psi*_b O[b, a]
    g = psi - phi_plain
    d = psi - proj
    a = np.sum(np.abs(g) ** 2, axis=(0, 1))
    b = np.sum((np.conj(g) * d).real, axis=(0, 1))
    c = np.sum(np.abs(d) ** 2, axis=(0, 1))
    return np.stack([a, b, c])
