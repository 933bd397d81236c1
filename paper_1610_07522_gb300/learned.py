"""Learned per-voxel damping weight for the damped gradient step (an
extension of Sec. 2.2, Eq. dampstep; the paper has no learned part).

The network, its training kernels and the weighted step are libsky calls
(include/sky.h, "Learned damping weight"); this module holds the parameter
vector, collects training samples from trajectories the solver itself
generates, and runs the Adam loop.  PyTorch only allocates device memory.

Training sample (one species at one iteration n of a plain run):
  the mean field U, B, W of iteration n, and the per-voxel statistics a, b, c
  of the one-step loss, from psi_n, the plain damped step phi_n of psi_n and
  the projection P* psi_n on a target occupied space psi* (sky_cross_overlap
  + sky_rotate): the plain iterate k steps later, psi_{n+k}, or a converged
  iterate.
The loss of a sample is sum_r (a w^2 - 2 b w + c) / sum_r c: the squared
distance of the weighted step from the target space, relative to the
distance at w = 0 (the separable form of the one-step error).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import binding as B

NPARAM = B.SKY_NET_NPARAM
H = B.SKY_NET_HIDDEN


def init_params(seed=0):
    """Flat FP32 parameter vector: uniform He initialisation of W1 and W2,
    zero biases, and a zero last layer with b3 = -log(WMAX - 1), so that the
    untrained network gives w = 1 everywhere (the paper's step)."""
    rng = np.random.default_rng(seed)
    parts = []
    for cin, cout in ((3, H), (H, H)):
        lim = math.sqrt(6.0 / (cin * 27))
        parts += [rng.uniform(-lim, lim, cout * cin * 27), np.zeros(cout)]
    parts += [np.zeros(H * 27), np.array([-math.log(B.SKY_NET_WMAX - 1.0)])]
    theta = np.concatenate(parts).astype(np.float32)
    assert theta.size == NPARAM
    return theta


class DampingNet:
    """Parameters and Adam state of the damping network on one device."""

    def __init__(self, device="cuda:0", theta=None, seed=0):
        self.device = torch.device(device)
        th = init_params(seed) if theta is None else np.asarray(theta, dtype=np.float32)
        self.theta = torch.from_numpy(th.copy()).to(self.device)
        f64 = dict(dtype=torch.float64, device=self.device)
        self.grad = torch.zeros(NPARAM, **f64)
        self.m = torch.zeros(NPARAM, **f64)
        self.v = torch.zeros(NPARAM, **f64)
        self.loss = torch.zeros(1, **f64)
        self.step_count = 0
        self._ws = {}

    def workspace(self, G):
        """(ws, w) buffers for a grid of G points, allocated once per size."""
        if G not in self._ws:
            self._ws[G] = (torch.zeros(B.SKY_NET_WS_PER_POINT * G, dtype=torch.float32, device=self.device),
                           torch.zeros(G, dtype=torch.float32, device=self.device))
        return self._ws[G]

    def view(self):
        """A handle on the same parameters with workspaces of its own, for
        solvers that run the network concurrently on different streams."""
        v = object.__new__(DampingNet)
        v.__dict__.update(self.__dict__)
        v._ws = {}
        return v

    def weights(self, ctx, G, q, U, Bf, W, out, scale=1.0):
        """w_q(r) = 1 + scale (w_net - 1) into ``out`` [G] float from the mean
        field of species q."""
        ws, _ = self.workspace(G)
        B.sky_net_forward(ctx, q, self.theta, U, Bf, W, ws, out, scale)

    def state_dict(self):
        return {"theta": self.theta.cpu().numpy(), "step": self.step_count}

    @classmethod
    def from_state(cls, state, device="cuda:0"):
        net = cls(device, theta=state["theta"])
        net.step_count = int(state.get("step", 0))
        return net


class Sample:
    """One species' mean field and loss statistics at one iteration."""

    def __init__(self, ctx, G, q, U, Bf, W, abc, norm, it):
        self.ctx, self.G, self.q, self.it = ctx, G, q, it
        self.U, self.Bf, self.W = U, Bf, W
        self.abc, self.norm = abc, norm


def collect(solver, iterations, psi_star=None, ahead=None):
    """Re-run ``solver`` (freshly loaded, same initial state as the plain run
    that produced the target) and record a Sample per species at each
    iteration n in ``iterations``.  The target space is either ``psi_star``
    (a converged iterate of that run) or, with ``ahead = k``, the plain
    iterate psi_{n+k} of this same run: one weighted step is then trained to
    reach where k plain steps go, which carries the self-consistent
    (mean-field) dynamics of the trajectory into the target.  Returns the
    samples; ``solver`` is left after the last iteration it needed."""
    if (psi_star is None) == (ahead is None):
        raise ValueError("give exactly one of psi_star and ahead")
    its = sorted(set(int(i) for i in iterations))
    k = 0 if ahead is None else int(ahead)
    dev, G = solver.device, solver.G
    ppsi = [torch.empty_like(p) for p in solver.psi]
    X = [torch.empty((I, I), dtype=torch.complex128, device=dev) for I in solver.I]
    pending = {}
    out = []
    last = its[-1] + k
    for it in range(last + 1):
        if it in its:
            rec = {}
            for q in solver._species():
                I, o = solver.I[q], solver.off[q]
                ctx = solver.ctx
                B.sky_apply_h(ctx, solver.U[q], solver.Bf[q], solver.W[q], solver.psi[q], solver.h[q], I,
                              solver.eps[o:o + I])
                B.sky_damped_step(ctx, q, solver.psi[q], solver.h[q], solver.eps[o:o + I], solver.phi[q], I,
                                  solver.w.x0, solver.w.E0)
                rec[q] = (solver.psi[q].clone(), solver.phi[q].clone(), solver.U[q].clone(),
                          solver.Bf[q].clone(), solver.W[q].clone())
            pending.setdefault(it + k, []).append((it, rec))
        for n, rec in pending.pop(it, []):
            for q, (psi_n, phi_n, U, Bf, W) in rec.items():
                I = solver.I[q]
                ctx = solver.ctx
                star = solver.psi[q] if psi_star is None else psi_star[q]
                B.sky_cross_overlap(ctx, star, psi_n, I, X[q])
                B.sky_rotate(ctx, star, X[q], I, ppsi[q])
                abc = torch.empty((3, G), dtype=torch.float64, device=dev)
                norm = torch.empty(1, dtype=torch.float64, device=dev)
                B.sky_precond_stats(ctx, psi_n, phi_n, ppsi[q], I, abc, norm)
                out.append(Sample(ctx, G, q, U, Bf, W, abc, norm, n))
        if it < last:
            solver.step()
    solver.sync()
    return out


def sample_loss(net, samples, weight_one=False):
    """Mean loss over ``samples`` with the current network (or with w = 1)."""
    total = torch.zeros(1, dtype=torch.float64, device=net.device)
    scratch = torch.zeros(NPARAM, dtype=torch.float64, device=net.device)
    theta = net.theta
    if weight_one:
        theta = torch.from_numpy(init_params(0)).to(net.device)
    for s in samples:
        ws, w = net.workspace(s.G)
        B.sky_net_forward(s.ctx, s.q, theta, s.U, s.Bf, s.W, ws, w)
        B.sky_net_backward(s.ctx, theta, ws, s.abc, s.norm, scratch, total)
    torch.cuda.synchronize(net.device)
    return float(total.item()) / max(1, len(samples))


def train(net, samples, steps, lr=3e-3, beta1=0.9, beta2=0.999, eps=1e-8, log_every=0):
    """Adam on the summed loss of ``samples``; returns the mean-loss history
    (one entry per logged step)."""
    hist = []
    ctx0 = samples[0].ctx
    for k in range(steps):
        net.loss.zero_()
        for s in samples:
            ws, w = net.workspace(s.G)
            B.sky_net_forward(s.ctx, s.q, net.theta, s.U, s.Bf, s.W, ws, w)
            B.sky_net_backward(s.ctx, net.theta, ws, s.abc, s.norm, net.grad, net.loss)
        net.step_count += 1
        B.sky_net_adam(ctx0, net.theta, net.grad, net.m, net.v, net.step_count, lr, beta1, beta2, eps)
        if log_every and (k % log_every == 0 or k == steps - 1):
            hist.append((k, float(net.loss.item()) / len(samples)))
    torch.cuda.synchronize(net.device)
    return hist
