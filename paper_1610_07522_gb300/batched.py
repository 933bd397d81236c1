"""Many independent boxes iterated together (twist-averaged boundary
conditions and uneven box sizes, each box its own damped-gradient solve of
Fig. 1).

Each box has its own libsky context (its grid, particle numbers and Bloch
twist) and its own CUDA stream, on which its h psi, damped step, matrices,
recombination, densities, mean field and energy run.  The Loewdin factors
and Rayleigh-Ritz problems of every species of every box go to one shared
context in one batched solve (one cooperative eigensolver launch serves all
of them), so the latency-bound FP64 eigen work of small boxes is paid once
per iteration instead of once per box.  ``capture()`` records the whole
iteration (fork to the box streams, join, batched eigensolve, fork, join)
into one CUDA graph, replayed by ``step()``.
"""
from __future__ import annotations

import torch

from . import binding as B
from . import inputs as IN
from .solver import Solver


class BatchSolver:
    def __init__(self, workloads, prec=B.SKY_F32, device="cuda:0"):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (there is no CPU path)")
        self.device = torch.device(device)
        self.workloads = list(workloads)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in self.workloads]
        self.boxes = [Solver(w, prec=prec, device=self.device, stream=st)
                      for w, st in zip(self.workloads, self.streams)]
        self.problems = [(i, q) for i, s in enumerate(self.boxes) for q in s._species()]
        imax = max(self.boxes[i].I[q] for i, q in self.problems)
        w0 = self.workloads[0]
        main = torch.cuda.current_stream(self.device)
        self.eig = B.sky_init((8, 8, 8), (1.0, 1.0, 1.0), w0.params, False, (0.0, 0.0, 0.0),
                              B.SKY_F64, imax, main.cuda_stream)
        B.sky_reserve_batch(self.eig, len(self.problems))
        self.graph = None
        self.graph_stale = False
        self.launches_per_step = None
        self.units = sum(2 * (w.N + w.Z) for w in self.workloads)

    # ------------------------------------------------------------ set-up
    def load(self):
        """Fig. 1 step 1 for every box from its seeded synthetic inputs."""
        for s, w, st in zip(self.boxes, self.workloads, self.streams):
            inp = IN.make_inputs(w)
            with torch.cuda.stream(st):     # the copies in load() go to the box's stream too
                s.load(inp["psi0"], inp.get("rho0"), inp.get("tau0"))
        torch.cuda.synchronize(self.device)

    # ------------------------------------------------------------ iteration
    def _fork(self, main):
        ev = torch.cuda.Event()
        ev.record(main)
        for st in self.streams:
            st.wait_event(ev)

    def _join(self, main):
        for st in self.streams:
            ev = torch.cuda.Event()
            ev.record(st)
            main.wait_event(ev)

    def _enqueue(self, main):
        B.sky_set_stream(self.eig, main.cuda_stream)
        self._fork(main)
        for s in self.boxes:
            for q in s._species():
                s.species_step(q)
        self._join(main)
        self.eigensolve()
        self._fork(main)
        for s in self.boxes:
            for q in s._species():
                B.sky_rotate(s.ctx, s.phi[q], s.M[q], s.I[q], s.psi[q])
            B.sky_sp_spread(s.ctx, s.eps, s.hn2, s.A, s.spread)
            s.densities()
            B.sky_mean_fields(s.ctx, s.rho, s.tau, s.divJ, s.U, s.Bf, s.W)
            B.sky_energy(s.ctx, s.rho, s.tau, s.divJ, s.eout)
        self._join(main)

    def set_damping(self, net, rise_tol=1e-5):
        """Learned damping weight in every box (each with its own network
        workspace, as the boxes run concurrently); the per-box fallback of
        Solver.set_damping applies, and a fallback re-captures the graph."""
        for s in self.boxes:
            with torch.cuda.stream(s.stream):
                v = net.view()
                v.workspace(s.G)            # allocated now, not inside a capture
                s.set_damping(v, rise_tol=rise_tol)
        self.graph_stale = self.graph is not None

    def eigensolve(self):
        """Loewdin factors and Rayleigh-Ritz of every species of every box in
        one batched solve on the shared context (its stream)."""
        S = [self.boxes[i].S[q] for i, q in self.problems]
        H = [self.boxes[i].H[q] for i, q in self.problems]
        C = [self.boxes[i].C[q] for i, q in self.problems]
        M = [self.boxes[i].M[q] for i, q in self.problems]
        I = [self.boxes[i].I[q] for i, q in self.problems]
        lam = [self.boxes[i].lam[self.boxes[i].off[q]:self.boxes[i].off[q] + self.boxes[i].I[q]]
               for i, q in self.problems]
        B.sky_orthonormalize_batched(self.eig, S, I, C)
        B.sky_subspace_diag_batched(self.eig, H, C, I, M, lam)

    def tune(self, reps=5, cache=None):
        """Autotune the launch shapes (one box per distinct shape, then the
        shared eigensolver); call after at least one iteration and before
        ``capture()``."""
        from . import autotune
        torch.cuda.synchronize(self.device)
        res = autotune.tune_batch(self, reps, cache)
        torch.cuda.synchronize(self.device)
        return res

    def step_eager(self):
        """One iteration of every box, enqueued without a graph."""
        self._enqueue(torch.cuda.current_stream(self.device))

    def capture(self):
        """Record one iteration of every box into a CUDA graph."""
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        n0 = B.sky_kernel_launches()
        cap = torch.cuda.Stream(device=self.device)
        with torch.cuda.graph(g, stream=cap):
            self._enqueue(torch.cuda.current_stream(self.device))
        self.launches_per_step = B.sky_kernel_launches() - n0
        B.sky_set_stream(self.eig, torch.cuda.current_stream(self.device).cuda_stream)
        self.graph = g
        torch.cuda.synchronize(self.device)

    def step(self):
        """One iteration of every box: the captured graph if there is one
        (re-captured first if a box's launch sequence changed)."""
        if self.graph is None:
            self.step_eager()
            return
        if self.graph_stale:
            self.capture()
            self.graph_stale = False
        self.graph.replay()

    def sync(self):
        torch.cuda.synchronize(self.device)
        for s in self.boxes:
            B.sky_sync(s.ctx)
        B.sky_sync(self.eig)

    def energies(self, check_status=True):
        """Per-box (E, delta_eps) after synchronising, read in one copy; with
        check_status every box's device status word is checked too."""
        if check_status:
            self.sync()
        else:
            torch.cuda.synchronize(self.device)
        v = torch.stack([torch.stack([s.eout[0], s.spread[0]]) for s in self.boxes]).cpu().numpy()
        return [(float(e), float(d)) for e, d in v]

    def run(self, maxit, tol=1e-6, window=5):
        """Iterate every box until each has held |E_n/A - E_{n-1}/A| < tol for
        ``window`` consecutive iterations (boxes that are done keep iterating
        inside the batch) or maxit.  Returns per-box iterations to convergence
        (None if not reached) and the energy per nucleon of each box at the
        iteration it converged (its last one otherwise)."""
        prev = [None] * len(self.boxes)
        below = [0] * len(self.boxes)
        done = [None] * len(self.boxes)
        E_done = [None] * len(self.boxes)
        for it in range(maxit):
            self.step()
            en = self.energies(check_status=(it % 64 == 63))
            for b, (E, _) in enumerate(en):
                s = self.boxes[b]
                A = s.A
                if prev[b] is not None and abs(E - prev[b]) / A < tol:
                    below[b] += 1
                    if below[b] >= window and done[b] is None:
                        done[b] = it + 1
                        E_done[b] = E / A
                else:
                    below[b] = 0
                if s.damping_on and prev[b] is not None and (E - prev[b]) / A > s.rise_tol:
                    s.damping_scale *= 0.5          # the fallback of Solver.run
                    s.damping_fallbacks += 1
                    if s.damping_scale < s.min_scale:
                        s.damping_on = False
                    self.graph_stale = self.graph is not None
                prev[b] = E
            if all(d is not None for d in done):
                break
        last = [E / s.A for (E, _), s in zip(self.energies(check_status=True), self.boxes)]
        return done, [e if e is not None else l for e, l in zip(E_done, last)]

    def close(self):
        self.graph = None
        for s in self.boxes:
            s.close()
        if self.eig:
            B.sky_destroy(self.eig)
            self.eig = None
