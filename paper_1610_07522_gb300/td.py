"""Time-dependent stepping of a Solver's states through the libsky C ABI
(Sky3D's time-dependent mode, Sec. 1; Sec. 2.2: the time-evolution operator
is unitary, so the states stay orthonormal with no orthonormalisation, and
the nucleons couple only through the mean field).

One ``step(dt)`` (dt in fm/c) is a predictor-corrector pair of Taylor
propagations (``sky_td_taylor``): the states are carried half a step with
h(t) to give the densities and mean field at t + dt/2, then the full step
from psi(t) uses that midpoint h; densities, mean field and energy at
t + dt follow.  PyTorch provides the buffers; every arithmetic step is a
library call.
"""
from __future__ import annotations

import torch

from . import binding as B

HBARC = 197.3269804   # MeV fm


class TimeStepper:
    def __init__(self, solver, order=6):
        self.s = solver
        self.order = order
        # Taylor-term scratch per species: two state arrays
        self.work = [torch.zeros((2,) + tuple(p.shape), dtype=p.dtype, device=p.device)
                     for p in solver.psi]
        self.t = 0.0

    def _fields(self, states):
        """Densities of ``states`` (both species) and the mean field they give."""
        s = self.s
        s._fork()
        for q in range(2):
            B.sky_densities(s.ctxq[q], states[q], s.I[q], s.rho[q], s.tau[q], s.J[q], s.divJ[q])
        s._join()
        B.sky_mean_fields(s.ctx, s.rho, s.tau, s.divJ, s.U, s.Bf, s.W)

    def init_fields(self):
        """Mean field and energy of the current states (the start of an evolution)."""
        self._fields(self.s.psi)
        s = self.s
        B.sky_energy(s.ctx, s.rho, s.tau, s.divJ, s.eout)

    def step(self, dt):
        """Advance the states of both species by dt (fm/c); enqueued."""
        s = self.s
        tau = dt / HBARC
        qs = s._species()
        s._fork()
        for q in qs:
            B.sky_td_taylor(s.ctxq[q], s.U[q], s.Bf[q], s.W[q], s.psi[q], s.phi[q], self.work[q],
                            s.I[q], 0.5 * tau, self.order)
        s._join()
        self._fields(s.phi)            # midpoint mean field (h(t) is no longer needed)
        s._fork()
        for q in qs:
            B.sky_td_taylor(s.ctxq[q], s.U[q], s.Bf[q], s.W[q], s.psi[q], s.h[q], self.work[q],
                            s.I[q], tau, self.order)
        s._join()
        for q in qs:
            s.psi[q], s.h[q] = s.h[q], s.psi[q]
        self._fields(s.psi)
        B.sky_energy(s.ctx, s.rho, s.tau, s.divJ, s.eout)
        self.t += dt

    def energy(self):
        return self.s.energy()[0]
