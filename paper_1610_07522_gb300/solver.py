"""Driver of the damped-gradient iteration (Fig. 1) through the libsky C ABI.

PyTorch provides device memory and the stream; every arithmetic step is a
libsky call.  One ``step()`` is one full iteration for both species:
steps 2-3 per species (h psi, damped step, h phi, matrices, Loewdin and
Rayleigh-Ritz, recombination), then the densities of both species, the new
mean field and the energy (steps 4-5).

Buffers per species q: ``psi`` (orthonormal states), ``phi`` (damped
states), ``h`` (h psi, then h phi); matrices S, H, C, M; the mean field
U, B, W and densities rho, tau, J, divJ of both species.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class Solver:
    def __init__(self, workload, prec=B.SKY_F64, device="cuda:0", max_states=None, stream=None,
                 variant="exact", concurrent_species=False, split_eigensolve=False):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (there is no CPU path)")
        if variant not in ("exact", "paper_literal"):
            raise ValueError(variant)
        self.variant = variant      # steps 3b-3e: exact Rayleigh-Ritz or the paper's combined form
        self.w = workload
        self.device = torch.device(device)
        self.prec = prec
        self.cdtype = torch.complex128 if prec == B.SKY_F64 else torch.complex64   # FP32 forms
        nx, ny, nz = workload.grid
        self.shape = (nz, ny, nx)
        self.G = nx * ny * nz
        self.I = (workload.N, workload.Z)
        self.A = workload.N + workload.Z
        Imax = max_states or max(self.I)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.ctx = B.sky_init(workload.grid, workload.dx, workload.params, workload.coulomb,
                                  workload.twist, prec, Imax, self.stream.cuda_stream)
            # species contexts: the same one, or (concurrent_species) the protons
            # on a second context and stream, so that the work of the two species
            # overlaps; both join for the batched eigensolve and the mean field
            self.ctxq = [self.ctx, self.ctx]
            self.streamq = [self.stream, self.stream]
            if concurrent_species and workload.Z > 0:
                self.streamq[1] = torch.cuda.Stream(device=self.device)
                self.ctxq[1] = B.sky_init(workload.grid, workload.dx, workload.params,
                                          workload.coulomb, workload.twist, prec, workload.Z,
                                          self.streamq[1].cuda_stream)
        self.concurrent = self.ctxq[1] is not self.ctx
        # with concurrent species: each species' Loewdin and Rayleigh-Ritz solve on its
        # own context and stream right after its matrices (the species couple only
        # through the mean field), instead of one batched solve of both
        self.split_eig = bool(split_eigensolve and self.concurrent)
        dev, G = self.device, self.G
        f64 = dict(dtype=torch.float64, device=dev)
        self.psi = [torch.zeros((I, 2) + self.shape, dtype=self.cdtype, device=dev) for I in self.I]
        self.phi = [torch.zeros_like(p) for p in self.psi]
        self.h = [torch.zeros_like(p) for p in self.psi]
        self.U = torch.zeros((2, G), **f64)
        self.Bf = torch.zeros((2, G), **f64)
        self.W = torch.zeros((2, 3, G), **f64)
        self.rho = torch.zeros((2, G), **f64)
        self.tau = torch.zeros((2, G), **f64)
        self.J = torch.zeros((2, 3, G), **f64)
        self.divJ = torch.zeros((2, G), **f64)
        mat = lambda I: torch.zeros((I, I), dtype=torch.complex128, device=dev)
        self.S = [mat(I) for I in self.I]
        self.H = [mat(I) for I in self.I]
        self.C = [mat(I) for I in self.I]
        self.M = [mat(I) for I in self.I]
        self.eps = torch.zeros(self.A, **f64)
        self.hn2 = torch.zeros(self.A, **f64)
        self.lam = torch.zeros(self.A, **f64)
        self.eout = torch.zeros(8, **f64)
        self.spread = torch.zeros(2, **f64)
        self.off = (0, workload.N)
        self.overlap_events = None   # list to collect (I, start, end, a is b) per overlap call, or None
        # dict to collect (I, start, end) per call of sky_apply_h / sky_overlap / sky_rotate
        # (keys "apply_h", "overlap", "rotate"), events on the species' stream, or None
        self.call_events = None
        self.graph = None            # CUDA graph of one step (capture()), replayed by step()
        self.damping = None          # learned.DampingNet giving the per-voxel step weight, or None
        self.damping_on = False
        self.damping_fallbacks = 0
        self.wq = None
        self.const_w = None          # [2, G] constant damping weight, or None

    def set_damping(self, net, rise_tol=1e-5, min_scale=1.0 / 16.0):
        """Use the learned per-voxel weight in the damped step,
        w_q(r) = 1 + s (net(U_q, B_q, |W_q|) - 1) with s = 1 at the start.
        The plain step is the fallback: each time E/A rises by more than
        ``rise_tol`` MeV in one iteration (the damped gradient step lowers the
        energy) ``run`` halves s, and below ``min_scale`` it returns to the
        plain step for good."""
        self.graph = None
        self.damping = net
        self.damping_on = net is not None
        self.damping_scale = 1.0
        self.rise_tol = rise_tol
        self.min_scale = min_scale
        if net is not None and self.wq is None:
            self.wq = torch.zeros((2, self.G), dtype=torch.float32, device=self.device)
        # with concurrent species the proton stream runs the network on its own workspace
        self.dampq = [net, net]
        if net is not None and self.concurrent:
            self.dampq[1] = net.view()
            self.dampq[1].workspace(self.G)
        if net is not None:
            net.workspace(self.G)

    def set_constant_weight(self, c):
        """Scale the damped update of every voxel by the constant ``c``
        (phi = psi - c (psi - phi_plain); c = 1 is the plain step, None turns it
        off): the uniform step size a learned per-voxel weight has to beat.
        Ignored while a learned weight is on."""
        self.graph = None
        self.const_w = None if c is None else torch.full((2, self.G), float(c), dtype=torch.float32,
                                                         device=self.device)

    # ------------------------------------------------------------ set-up
    def _species(self):
        return [q for q in range(2) if self.I[q] > 0]

    def load(self, psi0, rho0=None, tau0=None):
        """Fig. 1 step 1 from host arrays (or device tensors): orthonormalise the trial states
        (psi = Loewdin(phi), Eqs. Loewedin, orthmatvec); the mean field from
        their densities or from given initial densities."""
        qs = self._species()
        for q in qs:
            src = psi0[q]
            if torch.is_tensor(src):      # already on the device (large workloads)
                self.phi[q].copy_(src.reshape(self.phi[q].shape))
            else:
                self.phi[q].copy_(torch.from_numpy(np.ascontiguousarray(src)).to(self.cdtype))
            B.sky_overlap(self.ctx, self.phi[q], self.phi[q], self.I[q], self.S[q])
        B.sky_orthonormalize_batched(self.ctx, [self.S[q] for q in qs], [self.I[q] for q in qs],
                                     [self.C[q] for q in qs])
        for q in qs:
            B.sky_rotate(self.ctx, self.phi[q], self.C[q], self.I[q], self.psi[q])
        if rho0 is None:
            self._fork()
            self.densities()
            self._join()
        else:
            self.rho.copy_(torch.from_numpy(np.asarray(rho0).reshape(2, -1)))
            self.tau.copy_(torch.from_numpy(np.asarray(tau0).reshape(2, -1)))
            self.divJ.zero_()
        B.sky_mean_fields(self.ctx, self.rho, self.tau, self.divJ, self.U, self.Bf, self.W)
        B.sky_sync(self.ctx)

    # ------------------------------------------------------------ iteration
    def densities(self):
        for q in range(2):   # I = 0 gives zero densities
            self._timed("densities", q, lambda: B.sky_densities(
                self.ctxq[q], self.psi[q], self.I[q], self.rho[q], self.tau[q], self.J[q],
                self.divJ[q]))

    def _timed(self, kind, q, fn):
        """Run fn(); with call_events set, bracket it with CUDA events on the
        stream species q's calls are enqueued on."""
        if self.call_events is None:
            return fn()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(self.streamq[q])
        fn()
        e1.record(self.streamq[q])
        self.call_events.setdefault(kind, []).append((self.I[q], e0, e1))

    def species_step(self, q):
        """Step 2 and 3a for species q: h psi, damped step, h phi, S and H."""
        I, o = self.I[q], self.off[q]
        ctx = self.ctxq[q]
        self._timed("apply_h", q, lambda: B.sky_apply_h(
            ctx, self.U[q], self.Bf[q], self.W[q], self.psi[q], self.h[q], I,
            self.eps[o:o + I], self.hn2[o:o + I]))
        w = None
        if self.damping_on:
            self.dampq[q].weights(ctx, self.G, q, self.U[q], self.Bf[q], self.W[q], self.wq[q],
                                 self.damping_scale)
            w = self.wq[q]
        elif self.const_w is not None:
            w = self.const_w[q]
        self._timed("damped_step", q, lambda: B.sky_damped_step(
            ctx, q, self.psi[q], self.h[q], self.eps[o:o + I], self.phi[q], I,
            self.w.x0, self.w.E0, w))
        self._timed("apply_h", q, lambda: B.sky_apply_h(
            ctx, self.U[q], self.Bf[q], self.W[q], self.phi[q], self.h[q], I))
        for X, rhs in ((self.S[q], self.phi[q]), (self.H[q], self.h[q])):
            if self.overlap_events is None:
                self._timed("overlap", q, lambda: B.sky_overlap(ctx, self.phi[q], rhs, I, X))
            else:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(self.streamq[q])
                B.sky_overlap(ctx, self.phi[q], rhs, I, X)
                e1.record(self.streamq[q])
                self.overlap_events.append((I, e0, e1, rhs is self.phi[q]))

    def ritz_step(self):
        """Steps 3b-3e for both species: Loewdin factors and Rayleigh-Ritz in one
        batched solve (the species couple only through the mean field), then
        the recombination psi = phi M."""
        qs = self._species()
        I = [self.I[q] for q in qs]
        self._timed("loewdin", 0, lambda: B.sky_orthonormalize_batched(
            self.ctx, [self.S[q] for q in qs], I, [self.C[q] for q in qs]))
        diag = (B.sky_subspace_diag_batched if self.variant == "exact"
                else B.sky_subspace_diag_literal_batched)
        self._timed("ritz", 0, lambda: diag(
            self.ctx, [self.H[q] for q in qs], [self.C[q] for q in qs], I, [self.M[q] for q in qs],
            [self.lam[self.off[q]:self.off[q] + self.I[q]] for q in qs]))
        self._fork()
        for q in qs:
            self._timed("rotate", q, lambda: B.sky_rotate(self.ctxq[q], self.phi[q], self.M[q],
                                                          self.I[q], self.psi[q]))

    def _fork(self):
        """Let the proton stream start after the work enqueued so far."""
        if self.concurrent:
            ev = torch.cuda.Event()
            ev.record(self.stream)
            self.streamq[1].wait_event(ev)

    def _join(self):
        """Let the main stream continue after the proton stream's work."""
        if self.concurrent:
            ev = torch.cuda.Event()
            ev.record(self.streamq[1])
            self.stream.wait_event(ev)

    def species_ritz(self, q):
        """Steps 3b-3e of species q alone on its own context and stream."""
        I = self.I[q]
        ctx = self.ctxq[q]
        B.sky_orthonormalize_batched(ctx, [self.S[q]], [I], [self.C[q]])
        diag = (B.sky_subspace_diag_batched if self.variant == "exact"
                else B.sky_subspace_diag_literal_batched)
        diag(ctx, [self.H[q]], [self.C[q]], [I], [self.M[q]],
             [self.lam[self.off[q]:self.off[q] + I]])
        self._timed("rotate", q, lambda: B.sky_rotate(ctx, self.phi[q], self.M[q], I, self.psi[q]))

    def _set_main_stream(self, st):
        self.stream = st
        self.streamq[0] = st
        if not self.concurrent:
            self.streamq[1] = st
        B.sky_set_stream(self.ctx, st.cuda_stream)

    def capture(self, frozen=False):
        """Record one iteration into a CUDA graph; ``step()`` then replays it
        (the ~300 launches of an iteration as one graph launch).  Call after at
        least one eager iteration (first-use allocations and attributes happen
        there) and again after anything that changes the launch sequence
        (precision, damping, eigensolver route)."""
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        old = self.stream
        cap = torch.cuda.Stream(device=self.device)
        n0 = B.sky_kernel_launches()
        try:
            with torch.cuda.graph(g, stream=cap):
                self._set_main_stream(cap)
                self.step_eager(frozen)
        finally:
            self._set_main_stream(old)
        self.launches_per_step = B.sky_kernel_launches() - n0
        self.graph = g
        self.graph_frozen = frozen
        torch.cuda.synchronize(self.device)

    def release_graph(self):
        self.graph = None

    def step(self, frozen=False):
        """One full iteration (Fig. 1 steps 2-5); enqueued, not synchronised:
        the captured graph when there is one, else the calls one by one."""
        if self.graph is not None and frozen == self.graph_frozen and self.call_events is None:
            with torch.cuda.stream(self.stream):
                self.graph.replay()
            return
        self.step_eager(frozen)

    def step_eager(self, frozen=False):
        """One full iteration enqueued call by call."""
        self._fork()
        if self.split_eig:
            # two independent chains (neutrons on the main stream, protons on the
            # second) up to the densities; joined for the mean field
            for q in self._species():
                self.species_step(q)
                self.species_ritz(q)
            self.densities()
            self._join()
            B.sky_sp_spread(self.ctx, self.eps, self.hn2, self.A, self.spread)
            if not frozen:
                B.sky_mean_fields(self.ctx, self.rho, self.tau, self.divJ, self.U, self.Bf, self.W)
            B.sky_energy(self.ctx, self.rho, self.tau, self.divJ, self.eout)
            return
        for q in self._species():
            self.species_step(q)
        self._join()
        self.ritz_step()          # batched eigensolve on the main stream; rotations forked
        B.sky_sp_spread(self.ctx, self.eps, self.hn2, self.A, self.spread)
        self.densities()
        self._join()

        def fields():
            if not frozen:
                B.sky_mean_fields(self.ctx, self.rho, self.tau, self.divJ, self.U, self.Bf, self.W)
            B.sky_energy(self.ctx, self.rho, self.tau, self.divJ, self.eout)
        self._timed("fields", 0, fields)

    def step_host(self, host, eout_host):
        """One iteration from host state: copy psi and the mean field in from
        pinned host tensors through the library's copy calls (on the context
        stream), iterate, copy the energies back (end to end)."""
        for q in range(2):
            if self.I[q] > 0:
                B.sky_memcpy_h2d(self.ctx, self.psi[q], host["psi"][q])
        B.sky_memcpy_h2d(self.ctx, self.U, host["U"])
        B.sky_memcpy_h2d(self.ctx, self.Bf, host["B"])
        B.sky_memcpy_h2d(self.ctx, self.W, host["W"])
        self.step()
        B.sky_memcpy_d2h(self.ctx, eout_host, self.eout)
        self.sync()
        return eout_host

    def sync(self):
        B.sky_sync(self.ctx)
        if self.concurrent:
            B.sky_sync(self.ctxq[1])

    def energy(self):
        """Host copy of (E, delta_eps) after synchronising."""
        self.sync()
        e = self.eout.cpu().numpy()
        return float(e[0]), float(self.spread[0].item()), e

    def set_prec(self, prec):
        """Switch the GEMM form of an FP32-spinor solver (sky_set_prec)."""
        self.graph = None
        B.sky_set_prec(self.ctx, prec)
        if self.concurrent:
            B.sky_set_prec(self.ctxq[1], prec)
        self.prec = prec

    def set_eigen_method(self, method):
        """Choose the FP64 eigensolver of the diagonalisations
        (B.SKY_EIG_AUTO, B.SKY_EIG_JACOBI or B.SKY_EIG_TRIDIAGONAL)."""
        self.graph = None
        for c in {id(x): x for x in self.ctxq}.values():
            B.sky_tune_set(c, B.SKY_KNOB_EIGEN_METHOD, method)

    def run(self, maxit=None, tol=None, callback=None, window=1, escalate=None):
        """Iterate until |E_n/A - E_{n-1}/A| < tol for ``window`` consecutive
        iterations (1: the plain rule) or maxit; returns (history, converged).
        A window > 1 keeps a single small change, e.g. rounding noise of an
        FP32 form on a flat stretch of the path, from ending the run.
        ``escalate = (tol_switch, prec)`` switches the GEMM form to ``prec``
        once the change has stayed below tol_switch for ``window`` iterations
        (e.g. split-BF16 far from convergence, then FP32).  ``callback(it, record)``
        returning True ends the run there (not converged)."""
        maxit = self.w.maxit if maxit is None else maxit
        tol = self.w.tol if tol is None else tol
        hist, E_prev, below, below_sw = [], None, 0, 0
        for it in range(maxit):
            self.step()
            E, de, _ = self.energy()
            hist.append({"it": it, "E": E, "delta_eps": de})
            if callback and callback(it, hist[-1]) is True:
                return hist, False          # the caller asked to stop here
            dE = abs(E - E_prev) / self.A if E_prev is not None else None
            if escalate is not None and dE is not None:
                below_sw = below_sw + 1 if dE < escalate[0] else 0
                if below_sw >= window:
                    self.set_prec(escalate[1])
                    hist[-1]["escalated"] = escalate[1]
                    escalate, below = None, 0
            if dE is not None and dE < tol and escalate is None:
                below += 1
                if below >= window:
                    return hist, True
            else:
                below = 0
            if self.damping_on and E_prev is not None and (E - E_prev) / self.A > self.rise_tol:
                self.graph = None            # the scale is a launch argument
                self.damping_scale *= 0.5
                self.damping_fallbacks += 1
                hist[-1]["fallback"] = self.damping_scale
                if self.damping_scale < self.min_scale:
                    self.damping_on = False
            E_prev = E
        return hist, False

    def close(self):
        if self.ctx:
            if getattr(self, "concurrent", False) and self.ctxq[1]:
                B.sky_destroy(self.ctxq[1])
                self.ctxq[1] = None
            B.sky_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
