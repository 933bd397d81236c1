"""Plain FP64 CPU oracle of time-dependent stepping (the time-dependent mode of
Sky3D that the paper sets beside the static solver, Sec. 1 and Sec. 2.2).

TEST INFRASTRUCTURE.  Only ``tests/`` (and, like the rest of ``oracle/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``) may
import or call this module.  It imports nothing from the product package.

What the paper fixes (Sec. 2.2, the paragraph after Fig. 1): the time
evolution operator is unitary, so the states stay orthonormal without any
orthonormalisation step, every nucleon evolves independently of the others,
and the nucleons interact only through the mean field built from the
densities.  It gives no propagator.  Readings (also in the design notes):
  * propagator exp(-i h dt / hbar) as its Taylor polynomial of order m
    (default 6), sum_{k<=m} (-i dt h / hbar c)^k / k! psi, time in fm/c;
  * the mean field of a step is taken at its midpoint: a predictor half step
    with h(t) gives the densities and mean field at t + dt/2, then the full
    step from psi(t) uses that h (second order in dt);
  * the functional is the static solver's time-even one (rho, tau, div J);
    h is its derivative with respect to psi^*, so the exact evolution
    conserves the energy; the time-odd terms are dropped as in the static
    part.
"""
from __future__ import annotations

import math

import numpy as np

from .sky_oracle import apply_h, densities, energy, mean_fields

HBARC = 197.3269804   # MeV fm


def taylor_step(psi, U, B, W, grid, dt, order=6):
    """psi(t + dt) = sum_{k=0}^{order} (-i dt h / hbar c)^k / k! psi, h with the
    fixed mean field (U, B, W) of one species; dt in fm/c."""
    out = psi.astype(np.complex128).copy()
    term = out.copy()
    for k in range(1, order + 1):
        term = (-1j * dt / (HBARC * k)) * apply_h(term, U, B, W, grid)
        out = out + term
    return out


def field_of(psi, grid, p, coulomb):
    """Densities of both species and the mean field they give (Eq. Skyrme)."""
    d = [densities(psi[q], grid) for q in range(2)]
    rho = np.stack([d[q][0] for q in range(2)])
    tau = np.stack([d[q][1] for q in range(2)])
    divJ = np.stack([d[q][3] for q in range(2)])
    U, B, W = mean_fields(rho, tau, divJ, p, grid, coulomb)
    return U, B, W, rho, tau, divJ


def td_step(st, grid, p, coulomb, dt, order=6):
    """One time step of both species (mutates ``st``: psi and the mean field
    at t + dt).  Predictor: psi(t + dt/2) with h(t); corrector: psi(t + dt)
    from psi(t) with h(t + dt/2).  Returns the energy at t + dt."""
    half = [taylor_step(st.psi[q], st.U[q], st.B[q], st.W[q], grid, 0.5 * dt, order)
            for q in range(2)]
    Uh, Bh, Wh = field_of(half, grid, p, coulomb)[:3]
    st.psi = [taylor_step(st.psi[q], Uh[q], Bh[q], Wh[q], grid, dt, order) for q in range(2)]
    st.U, st.B, st.W, rho, tau, divJ = field_of(st.psi, grid, p, coulomb)
    E = energy(rho, tau, divJ, p, grid, coulomb)
    return {"E": E["total"], "rho": rho, "tau": tau, "divJ": divJ}


def scalar_taylor(z, order=6):
    """sum_{k<=order} z^k / k! (the propagator on an eigenvector of h, z = -i eps dt / hbar c)."""
    return sum(z ** k / math.factorial(k) for k in range(order + 1))
