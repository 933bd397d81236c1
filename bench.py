"""Benchmark of the damped-gradient Skyrme-DFT iteration on GB300.

One step = one full iteration (Fig. 1 steps 2-5, both species, neutrons and
protons on separate contexts and streams) of the 24^3 periodic box with 280
neutrons + 120 protons, FP64 complex spinors, SLy4, FFT-Poisson Coulomb, seeded
synthetic inputs (blob densities and random plane-wave superpositions).  Metric: h.psi spinor-applies per second, i.e.
2 (N + Z) applies per iteration divided by the iteration time, summed over
ranks.  With --gpus N each rank runs an independent replica (the path is
not sharded across GPUs); the timing is the max over ranks.

--impl reference times the CPU oracle (the plain FP64 NumPy restatement of
the method) on the host cores instead; each of its steps is a bounded
sample: one full oracle iteration of the same box and Coulomb physics with a
tenth of the states (28 n + 12 p).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "sly4_24cubed_280n120p_coulomb_fp64"
FORMS = {"fp64": 0, "f32": 1, "bf16x3": 2, "bf16x6": 3}     # sky_prec values
EIGEN = {"auto": 0, "jacobi": 1, "tridiagonal": 2}        # SKY_KNOB_EIGEN_METHOD values
DTYPES = {"fp64": "f64", "f32": "f32", "bf16x3": "f32+bf16x3", "bf16x6": "f32+bf16x6"}


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _maybe_init_pg(ws, backend):
    if ws > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend=backend)
        return dist
    return None


def _max_over_ranks(x, dist, device=None):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(dist):
    if dist is not None:
        dist.barrier()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); smax.append(float(f[2])); power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _gpu_smi_id(device_index):
    import torch
    try:
        u = str(torch.cuda.get_device_properties(device_index).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return device_index


# ---------------------------------------------------------------- CPU baseline
def cpu_baseline_sample(w, inp, scale_states=1.0):
    """Time the oracle on one full iteration (or a state-scaled sample)."""
    import numpy as np
    import oracle as O
    from paper_1610_07522_gb300 import inputs as IN
    if scale_states != 1.0:
        N = max(1, int(round(w.N * scale_states)))
        Z = max(1, int(round(w.Z * scale_states)))
        w = IN.Workload(**{**w.as_dict(), "N": N, "Z": Z})
        inp = IN.make_inputs(w)
    g = O.Grid(w.grid, w.dx, w.twist)
    st = O.initial_state(inp["psi0"], g, w.params, w.coulomb, inp.get("rho0"), inp.get("tau0"))
    t = time.perf_counter()
    O.iterate(st, g, w.params, w.coulomb, w.x0, w.E0)
    dt = time.perf_counter() - t
    return 2 * (w.N + w.Z) / dt, dt, w


def _cpu_threads():
    n = os.cpu_count() or 1
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        blas = [d.get("num_threads", 1) for d in info if d.get("user_api") == "blas"]
        if blas:
            return max(blas)
    except Exception:
        pass
    return int(os.environ.get("OMP_NUM_THREADS", n))


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_1610_07522_gb300 import inputs as IN
    w = IN.WORKLOADS[WORKLOAD]
    inp = IN.make_inputs(w)
    rates = []
    for k in range(args.warmup + args.steps):
        r, dt, ws_ = cpu_baseline_sample(w, inp, 0.1)
        if k >= args.warmup:
            rates.append((r, dt))
    tot_units = sum(2 * (ws_.N + ws_.Z) for _ in rates)
    tot_t = sum(dt for _, dt in rates)
    value = tot_units / tot_t
    line = {
        "impl": "reference", "metric": "h.psi spinor-applies/s (full iteration)", "value": value,
        "unit": "spinor-applies/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / len(rates),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD + " (reference step: 28 n + 12 p state sample)",
                   "grid": list(w.grid), "N": ws_.N, "Z": ws_.Z, "coulomb": True},
        "cpu_baseline": {"value": value, "unit": "spinor-applies/s", "cores": _cpu_threads(),
                         "kind": "oracle",
                         "sample": "one oracle iteration per step on 24^3 with 28 n + 12 p"},
        "e2e": {"value": value, "unit": "spinor-applies/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- convergence
CONV_WORKLOAD = "sly4_16cubed_16n16p_fp64"
CONV_SNAPS = [0, 2, 5, 12, 25, 60, 120, 180, 240, 360, 480, 600, 720, 840, 960]


CONV_WINDOW = 5


def convergence_leg(dev, maxit=4000, nets_out=None):
    """Seconds and iterations to |E_n/A - E_{n-1}/A| < 1e-6 MeV (held for
    CONV_WINDOW consecutive iterations, the same rule for every form) on the
    16^3, 16n+16p workload for each form: plain FP64, FP32, split-BF16 (x3),
    the paper's combined recombination, and the learned damping weight
    (trained here, on the GPU, by the library's kernels from plain
    trajectories; its training time is reported apart).  The reference is the
    plain method's fixed point (FP64 iterated to |dE/A| < 1e-8): a form
    reaches it when its stop point is as close as the plain FP64 stop point,
    within 1e-4 MeV per nucleon."""
    import torch
    from paper_1610_07522_gb300 import binding as B
    from paper_1610_07522_gb300 import inputs as IN
    from paper_1610_07522_gb300 import learned
    from paper_1610_07522_gb300.solver import Solver

    w = IN.WORKLOADS[CONV_WORKLOAD]
    inp = IN.make_inputs(w)

    def solve(prec, net=None, escalate=None, variant="exact", wl=None, const=None, plain_after=0):
        wl = w if wl is None else wl
        s = Solver(wl, prec=prec, device=dev, variant=variant, concurrent_species=True)
        if net is not None:
            s.set_damping(net)
        if const is not None:
            s.set_constant_weight(const)
        i_ = inp if wl is w else IN.make_inputs(wl)
        s.load(i_["psi0"], i_.get("rho0"), i_.get("tau0"))
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        try:
            hist, conv = s.run(maxit=maxit, window=CONV_WINDOW, escalate=escalate)
        except B.SkyError as err:      # a form that breaks down is reported, not fatal
            s.close()
            return {"converged": False, "iterations": None, "seconds": None, "E_per_A": None,
                    "error": str(err)}
        dt = time.perf_counter() - t
        r = {"converged": conv, "iterations": len(hist), "seconds": round(dt, 4),
             "E_per_A": hist[-1]["E"] / s.A}
        if net is not None:
            r["fallbacks"] = s.damping_fallbacks
        if plain_after and conv:
            # is the stop point a fixed point of the plain method?  continue
            # from it with the plain step and record the largest |dE/A|
            s.set_damping(None)
            s.set_constant_weight(None)
            E0_ = hist[-1]["E"]
            d = 0.0
            for _ in range(plain_after):
                s.step()
                E1_ = s.energy()[0]
                d = max(d, abs(E1_ - E0_) / s.A)
                E0_ = E1_
            r["plain_continuation"] = {"iterations": plain_after, "max_dE_per_A": d,
                                       "E_per_A_end": E0_ / s.A}
        s.close()
        return r

    out = {"workload": CONV_WORKLOAD, "tol_MeV_per_A": w.tol, "window": CONV_WINDOW, "maxit": maxit}
    # the fixed point itself: plain FP64 iterated to |dE/A| < 1e-8
    ref = Solver(w, prec=B.SKY_F64, device=dev, concurrent_species=True)
    ref.load(inp["psi0"], inp.get("rho0"), inp.get("tau0"))
    hist_ref, conv_ref = ref.run(maxit=3 * maxit, tol=1e-8, window=CONV_WINDOW)
    E_star = hist_ref[-1]["E"] / ref.A
    ref.close()
    out["fixed_point"] = {"E_per_A": E_star, "tol_MeV_per_A": 1e-8, "iterations": len(hist_ref),
                          "converged": conv_ref}
    for name, prec in (("fp64", B.SKY_F64), ("fp32", B.SKY_F32), ("bf16x3", B.SKY_F32_BF16X3)):
        out[name] = solve(prec)
    # the paper's combined form of steps 3b-3e (Sec. 3.3.3) instead of exact Ritz:
    # on this start (time-reversal symmetric: every level of H twofold
    # degenerate) and on a twisted copy of it (no degeneracy), against the
    # exact form on the same twisted box
    import numpy as np
    tw = tuple(float(v) for v in np.random.default_rng(1005).uniform(-np.pi, np.pi, 3))
    wt = IN.Workload(**{**w.as_dict(), "name": CONV_WORKLOAD + "_twisted", "twist": tw})
    out["fp64_paper_literal"] = solve(B.SKY_F64, variant="paper_literal")
    out["twisted_fp64_exact"] = solve(B.SKY_F64, wl=wt)
    out["twisted_fp64_paper_literal"] = solve(B.SKY_F64, variant="paper_literal", wl=wt)
    # split-BF16 far from convergence, FP32 GEMMs once |dE/A| < 2e-5
    out["bf16x3_to_fp32"] = solve(B.SKY_F32_BF16X3, escalate=(2e-5, B.SKY_F32))
    t = time.perf_counter()
    s = Solver(w, prec=B.SKY_F64, device=dev)
    s.load(inp["psi0"], inp.get("rho0"), inp.get("tau0"))
    samples = learned.collect(s, CONV_SNAPS, ahead=4)
    net = learned.DampingNet(dev, seed=0)
    learned.train(net, samples, 300, lr=3e-3)
    train_s = time.perf_counter() - t
    s.close()
    out["learned_train_seconds"] = round(train_s, 3)
    out["learned_fp64"] = solve(B.SKY_F64, net, plain_after=CONV_PLAIN_AFTER)
    out["learned_fp32"] = solve(B.SKY_F32, net, plain_after=CONV_PLAIN_AFTER)
    out["learned_bf16x3_to_fp32"] = solve(B.SKY_F32_BF16X3, net, escalate=(2e-5, B.SKY_F32),
                                          plain_after=CONV_PLAIN_AFTER)
    # the uniform step sizes a per-voxel weight has to beat (FP64 form)
    for c in CONV_CONST_WEIGHTS:
        out[f"const_w{c:g}_fp64"] = solve(B.SKY_F64, const=c, plain_after=CONV_PLAIN_AFTER)
    # the same network trained on trajectories of the 16^3 (FP64), 24^3 (FP64)
    # and 32^3 (split-BF16) workloads together
    t = time.perf_counter()
    keep, samples = [], []
    for name, prec, snaps in ((CONV_WORKLOAD, B.SKY_F64, CONV_SNAPS),
                              ("sly4_24cubed_280n120p_coulomb_fp64", B.SKY_F64, [0, 6, 12, 18, 24, 30, 36]),
                              ("sly4_32cubed_700n300p", B.SKY_F32_BF16X3, [0, 8, 16, 24, 32])):
        wl = IN.WORKLOADS[name]
        i_ = IN.make_inputs(wl)
        s = Solver(wl, prec=prec, device=dev)
        s.load(i_["psi0"], i_.get("rho0"), i_.get("tau0"))
        samples += learned.collect(s, snaps, ahead=4)
        keep.append(s)
    net3 = learned.DampingNet(dev, seed=0)
    learned.train(net3, samples, 300, lr=3e-3)
    for s in keep:
        s.close()
    out["learned_configs123_train_seconds"] = round(time.perf_counter() - t, 3)
    out["learned_configs123_fp32"] = solve(B.SKY_F32, net3, plain_after=CONV_PLAIN_AFTER)
    if nets_out is not None:
        nets_out["net_configs123"] = net3
    out["batched"] = batched_convergence(dev, net, maxit)
    base = out["fp64"]["seconds"]
    forms = ("fp64_paper_literal", "fp32", "bf16x3", "bf16x3_to_fp32", "learned_fp64", "learned_fp32",
             "learned_bf16x3_to_fp32", "learned_configs123_fp32") + tuple(
                 f"const_w{c:g}_fp64" for c in CONV_CONST_WEIGHTS)
    # a form reaches the fixed point when its stop point is as close to it as
    # the plain FP64 method's own stop point, within 1e-4 MeV per nucleon
    gap = abs(out["fp64"]["E_per_A"] - E_star)
    out["fixed_point"]["fp64_stop_gap_MeV_per_A"] = gap
    for k in forms:
        out[k]["same_fixed_point"] = bool(out[k]["converged"] and
                                          abs(out[k]["E_per_A"] - E_star) <= gap + 1e-4)
    t_ex, t_lit = out["twisted_fp64_exact"], out["twisted_fp64_paper_literal"]
    t_lit["same_fixed_point"] = bool(t_lit["converged"] and t_ex["converged"] and
                                     abs(t_lit["E_per_A"] - t_ex["E_per_A"]) < 1e-4)
    out["speedup_vs_fp64"] = {k: (round(base / out[k]["seconds"], 3) if out[k]["seconds"] else None)
                              for k in forms}
    consts = [k for k in forms if k.startswith("const_w") and out[k]["converged"]]
    if consts:
        best = min(consts, key=lambda k: out[k]["seconds"])
        out["best_constant_weight"] = {"form": best, "seconds": out[best]["seconds"],
                                       "iterations": out[best]["iterations"],
                                       "same_fixed_point": out[best]["same_fixed_point"]}
    return out


CONV_BOXES = 8
CONV_CONST_WEIGHTS = (1.25, 1.5, 1.75, 2.0)
CONV_PLAIN_AFTER = 20


def batched_convergence(dev, net, maxit):
    """Eight 16^3, 16n+16p boxes with seeded Bloch twists: seconds until every
    box meets the stop rule, plain FP64 one box at a time (the method without
    batching) against the FP32 batch replayed as one CUDA graph, with and
    without the learned weight."""
    import numpy as np
    import torch
    from paper_1610_07522_gb300 import binding as B
    from paper_1610_07522_gb300 import inputs as IN
    from paper_1610_07522_gb300.batched import BatchSolver
    from paper_1610_07522_gb300.solver import Solver

    base = IN.WORKLOADS[CONV_WORKLOAD]
    rng = np.random.default_rng(1005)
    ws = [IN.Workload(**{**base.as_dict(), "name": f"conv_box_{i}", "seed": 1005 * 1000 + i,
                         "twist": tuple(float(v) for v in rng.uniform(-np.pi, np.pi, 3))})
          for i in range(CONV_BOXES)]
    out = {"boxes": CONV_BOXES, "workload": f"{CONV_WORKLOAD} with seeded twists"}
    t_all, its, E = 0.0, [], []
    for w in ws:
        inp = IN.make_inputs(w)
        s = Solver(w, prec=B.SKY_F64, device=dev)
        s.load(inp["psi0"], inp.get("rho0"), inp.get("tau0"))
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        hist, conv = s.run(maxit=maxit, window=CONV_WINDOW)
        t_all += time.perf_counter() - t
        its.append(len(hist) if conv else None)
        E.append(hist[-1]["E"] / s.A)
        s.close()
    out["fp64_one_at_a_time"] = {"seconds": round(t_all, 3), "iterations": its,
                                 "boxes_converged": sum(i is not None for i in its)}
    for name, use_net in (("fp32_graph", False), ("learned_fp32_graph", True)):
        bs = BatchSolver(ws, prec=B.SKY_F32, device=dev)
        bs.load()
        if use_net:
            bs.set_damping(net)
        bs.step_eager()
        bs.capture()
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        done, EA = bs.run(maxit, window=CONV_WINDOW)
        dt = time.perf_counter() - t
        # both are stop points of the same rule, each short of the fixed point
        # by its slowest mode's remaining drop (up to a few 1e-4 MeV here)
        both = [b for b in range(len(ws)) if done[b] is not None and its[b] is not None]
        out[name] = {"seconds": round(dt, 3), "iterations": done,
                     "boxes_converged": sum(d is not None for d in done),
                     "max_stop_point_difference_MeV_per_A": (
                         max(abs(EA[b] - E[b]) for b in both) if both else None),
                     "same_fixed_point_where_both_converged": bool(
                         both and max(abs(EA[b] - E[b]) for b in both) < 5e-4)}
        bs.close()
    out["speedup_vs_fp64_one_at_a_time"] = {k: round(t_all / out[k]["seconds"], 3)
                                            for k in ("fp32_graph", "learned_fp32_graph")}
    return out


# ---------------------------------------------------------------- production shapes
# The paper's production shapes (Sec. 5.1, Tables 2-3): A = 6000, 3000 n + 3000 p,
# in 32^3 and 48^3 boxes (dx = 1 fm), blob starts; seconds per iteration on one
# GB300 in the paper's FP64 form and the FP32-spinor form (context only: the
# paper's figures are Cray XC40 seconds per iteration).
PRODUCTION = [("sly4_32cubed_3000n3000p", "fp64"), ("sly4_32cubed_3000n3000p", "f32"),
              ("sly4_48cubed_3000n3000p", "f32")]


def production_leg(dev, iters=2):
    """Seconds per full iteration (both species on two streams) of the A = 6000
    shapes after one untimed iteration from the start; input generation (host,
    NumPy) and the load are timed apart."""
    import torch
    from paper_1610_07522_gb300 import inputs as IN
    from paper_1610_07522_gb300.solver import Solver
    out = {"paper_context_s_per_iteration": {"32^3, 32 Haswell cores": 59.8,
                                             "32^3, 1536 Haswell cores": 3.5}}
    for name, form in PRODUCTION:
        w = IN.WORKLOADS[name]
        t = time.perf_counter()
        inp = IN.make_inputs(w)
        gen_s = time.perf_counter() - t
        s = Solver(w, prec=FORMS[form], device=dev, concurrent_species=True)
        t = time.perf_counter()
        s.load(inp["psi0"], inp.get("rho0"), inp.get("tau0"))
        del inp
        s.step()
        s.sync()
        load_s = time.perf_counter() - t
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        for _ in range(iters):
            s.step()
        e1.record(s.stream)
        torch.cuda.synchronize(dev)
        E, de, _ = s.energy()
        from paper_1610_07522_gb300 import binding as B
        B_stats = B.sky_stats(s.ctx)
        out[f"{name}_{form}"] = {"grid": list(w.grid), "N": w.N, "Z": w.Z, "form": form,
                                 "s_per_iteration": e0.elapsed_time(e1) / 1e3 / iters,
                                 "iterations_timed": iters, "input_generation_s": round(gen_s, 2),
                                 "load_and_first_iteration_s": round(load_s, 2),
                                 "E_per_A": E / (w.N + w.Z), "delta_eps": de,
                                 "solver_stats": B_stats}
        s.close()
        del s
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- forms at the precision config
CONV3_WORKLOAD = "sly4_32cubed_700n300p"


def convergence_config3_leg(dev, net, cap=300):
    """The forms where they are defined: 32^3, 700 n + 300 p, Coulomb, blob start.
    The stop rule (|dE/A| < 1e-6 MeV for 5 iterations) takes thousands of
    iterations here, so the comparison is capped (labelled): the plain FP64
    method runs ``cap`` iterations and reaches E_cap/A; every form then runs
    until its E/A is at or below E_cap/A (or the stop rule holds, or 2 cap
    iterations pass), and its wall time for that is compared with FP64's
    (each form stops once it gets there).
    Forms: FP32 spinors with the 4-digit tensor-core contractions,
    split-BF16 x3 escalated to them once |dE/A| < 2e-5, and the learned
    weight (FP32)."""
    import torch
    from paper_1610_07522_gb300 import binding as B
    from paper_1610_07522_gb300 import inputs as IN
    from paper_1610_07522_gb300.solver import Solver
    w = IN.WORKLOADS[CONV3_WORKLOAD]
    inp = IN.make_inputs(w)
    A = w.N + w.Z
    out = {"workload": CONV3_WORKLOAD, "cap_iterations": cap,
           "rule": "time to E/A <= the plain FP64 method's E/A after the cap (or the stop rule)"}

    def run(prec, target=None, net_=None, escalate=None, maxit=cap):
        s = Solver(w, prec=prec, device=dev, concurrent_species=True)
        if net_ is not None:
            s.set_damping(net_)
        s.load(inp["psi0"], inp.get("rho0"), inp.get("tau0"))
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        reached = {}

        def cb(it, rec):
            if target is not None and "t" not in reached and rec["E"] / A <= target:
                reached["t"] = time.perf_counter() - t
                reached["it"] = it + 1
                return True             # the comparison needs no more
        try:
            hist, conv = s.run(maxit=maxit, window=CONV_WINDOW, callback=cb, escalate=escalate)
        except B.SkyError as err:
            s.close()
            return {"error": str(err)}
        dt = time.perf_counter() - t
        r = {"iterations": len(hist), "seconds": round(dt, 3), "converged": conv,
             "E_per_A": hist[-1]["E"] / A, "s_per_iteration": dt / len(hist)}
        if target is not None:
            r["reached_target"] = "t" in reached
            r["seconds_to_target"] = round(reached["t"], 3) if "t" in reached else None
            r["iterations_to_target"] = reached.get("it")
        if net_ is not None:
            r["fallbacks"] = s.damping_fallbacks
        s.close()
        torch.cuda.empty_cache()
        return r

    base = run(B.SKY_F64)
    out["fp64"] = base
    target = base["E_per_A"]
    out["target_E_per_A"] = target
    out["fp32"] = run(B.SKY_F32, target, maxit=2 * cap)
    out["bf16x3_to_fp32"] = run(B.SKY_F32_BF16X3, target, escalate=(2e-5, B.SKY_F32), maxit=2 * cap)
    if net is not None:
        out["learned_fp32"] = run(B.SKY_F32, target, net_=net, maxit=2 * cap)
    out["speedup_vs_fp64_to_target"] = {
        k: (round(base["seconds"] / out[k]["seconds_to_target"], 3)
            if out.get(k, {}).get("seconds_to_target") else None)
        for k in ("fp32", "bf16x3_to_fp32", "learned_fp32") if k in out}
    return out


# ---------------------------------------------------------------- learned form at scale
CONFIG5 = "sly4_64cubed_5600n2400p"


def config5_leg(dev, net, iters=3):
    """The learned-weight form at scale: 64^3, 5600 n + 2400 p, FP32 spinors
    (the FP64 form has no 64-point FFT lines), blob densities and seeded noisy
    plane-wave states made on the device; ``iters`` iterations (a labelled
    cap: convergence at this size takes thousands) of the plain damped step
    and of the learned per-voxel weight (the network trained on the 16^3,
    24^3 and 32^3 trajectories), from the same start, with wall time per
    iteration (each ends with the host reading the energy)."""
    import numpy as np
    import torch
    from paper_1610_07522_gb300 import binding as B
    from paper_1610_07522_gb300 import inputs as IN
    from paper_1610_07522_gb300.solver import Solver
    w = IN.WORKLOADS[CONFIG5]
    rng = np.random.default_rng(w.seed)
    rho0, tau0 = IN.blob_densities(w.grid, w.dx, w.N, w.Z, w.nblob, w.blob_sigma, rng)
    out = {"workload": CONFIG5, "grid": list(w.grid), "N": w.N, "Z": w.Z, "form": "f32",
           "iterations_capped": iters,
           "start": "blob densities, noisy plane waves (noise 0.1) generated on the device"}
    for name, use_net in (("plain", False), ("learned", True)):
        if use_net and net is None:
            continue
        s = Solver(w, prec=B.SKY_F32, device=dev, concurrent_species=True)
        t = time.perf_counter()
        psi0 = [IN.noisy_plane_waves_device(w.grid, w.dx, I, w.noise, w.seed * 10 + q, dev,
                                            torch.complex64) for q, I in enumerate((w.N, w.Z))]
        s.load(psi0, rho0, tau0)
        del psi0
        torch.cuda.empty_cache()
        s.sync()
        load_s = time.perf_counter() - t
        if use_net:
            s.set_damping(net)
        stamps = [time.perf_counter()]
        hist, _ = s.run(maxit=iters, tol=-1.0, callback=lambda it, rec: stamps.append(time.perf_counter()))
        dts = [b - a for a, b in zip(stamps, stamps[1:])]
        out[name] = {"load_s": round(load_s, 2), "s_per_iteration": dts,
                     "E_per_A": [h["E"] / (w.N + w.Z) for h in hist],
                     "delta_eps": [h["delta_eps"] for h in hist],
                     "fallbacks": s.damping_fallbacks if use_net else None}
        s.close()
        del s
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- batched form
def batched_leg(dev, form="bf16x3", count=64, steps=10):
    """The 64 uneven, twisted boxes of inputs.batched_workloads() (grids 16^3,
    20^3, 24^3; 0.03 fm^-3, proton fraction 0.3) iterated together: every
    box's FFT and GEMM work on its own stream, one batched eigensolve for all
    128 species problems, autotuned launch shapes, the whole iteration
    replayed as one CUDA graph.  Compared with the same boxes stepped one at a
    time (each box's own solver) and with the eager (not captured) batch."""
    import torch
    from paper_1610_07522_gb300 import binding as B
    from paper_1610_07522_gb300 import inputs as IN
    from paper_1610_07522_gb300.batched import BatchSolver

    ws = IN.batched_workloads(count)
    bs = BatchSolver(ws, prec=FORMS[form], device=dev)
    bs.load()
    main = torch.cuda.current_stream(dev)

    def timed(fn, k):
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(main)
        for _ in range(k):
            fn()
        e1.record(main)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / k

    bs.step_eager()
    tuned = bs.tune(reps=3)
    bs.step_eager()
    eager_ms = timed(bs.step_eager, 3)
    bs.capture()
    for _ in range(3):
        bs.step()
    graph_ms = timed(bs.step, steps)
    try:
        bs.sync()
        status = "ok"
    except B.SkyError as e:
        status = str(e)

    # last: the same boxes one at a time (each its own two-problem eigensolve),
    # timed after the batch numbers so that those never start from the boxes'
    # solo state
    def one_at_a_time():
        for s in bs.boxes:
            s.step()
            torch.cuda.synchronize(dev)
    seq_ms = timed(one_at_a_time, 2)
    sizes = [bs.boxes[i].I[q] for i, q in bs.problems]
    plan = B.sky_tri_team_plan(sizes, torch.cuda.get_device_properties(dev).multi_processor_count)
    teams = None
    if plan is not None:
        team, tb = plan
        teams = {"problems": len(sizes), "teams": len(tb), "blocks": sum(c for _, c in tb),
                 "blocks_of_the_largest_problem": tb[team[sizes.index(max(sizes))]][1],
                 "one_block_teams": sum(1 for _, c in tb if c == 1)}
    out = {"instances": count, "form": form, "grids": sorted({w.grid[0] for w in ws}),
           "units_per_step": bs.units, "graph_ms_per_step": graph_ms, "eager_ms_per_step": eager_ms,
           "status_after_graph_steps": status, "eigensolver_teams": teams,
           "one_box_at_a_time_ms_per_step": seq_ms,
           "value": bs.units / (graph_ms / 1e3), "unit": "spinor-applies/s",
           "launches_per_step": bs.launches_per_step,
           "tuned": {k: (v[0] if isinstance(v, tuple) else {n: x[0] for n, x in v.items()})
                     for k, v in tuned.items()}}
    bs.close()
    return out


# ---------------------------------------------------------------- rooflines
# digit (or bf16 piece) products of each form's tensor-core contractions
NPROD = {0: 21, 1: 10, 2: 3, 3: 6}
# DRAM bytes per spinor of one sky_apply_h call: ncu dram__bytes_read.sum +
# dram__bytes_write.sum summed over the call's kernels (bench.py --probe-call
# apply_h; profiles/), divided by its I.  Keyed by (workload, form); absent
# until captured for the current kernels.
HPSI_TRAFFIC_PER_SPINOR = {
    # 2.784 GB over the 8 kernels of one I = 280 call (profiles/sky_apply_h_sly4_24cubed_280n_fp64.md)
    ("sly4_24cubed_280n120p_coulomb_fp64", "fp64"): 2784466176.0 / 280,
}
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_oz_deriv launch
# along y over the 560 neutron spin components of the 24^3 workload
# (profiles/k_oz_deriv_sly4_24cubed_280n_fp64.md): 124.2 + 71.5 MB
DERIV_TRAFFIC = {("sly4_24cubed_280n120p_coulomb_fp64", "fp64"): 195.7e6}


def derivative_roofline(dev, w, prec, peaks, form, reps=20):
    """The dominant kernel of the step, live: one spectral derivative pass
    (sky_derivative along y, the digit-split operator product on the tensor
    cores in the FP64 form) over the 2N spin components of the workload's
    neutrons, CUDA events on the context stream around reps launches.
    Algorithmic bytes per launch: every complex point read once and written
    once; bound: HBM (the operator work, 21 digit products of a 2n x 2n
    operator per line, runs on the tensor cores)."""
    import torch
    from paper_1610_07522_gb300 import binding as B
    st = torch.cuda.current_stream(dev)
    ctx = B.sky_init(w.grid, w.dx, w.params, w.coulomb, w.twist, prec, w.N, st.cuda_stream)
    nx, ny, nz = w.grid
    G = nx * ny * nz
    nb = 2 * w.N
    cd = torch.complex128 if prec == 0 else torch.complex64
    gen = torch.Generator(device=dev).manual_seed(3)
    src = torch.randn((nb, G), dtype=cd, device=dev, generator=gen)
    dst = torch.zeros_like(src)
    for _ in range(3):
        B.sky_derivative(ctx, 1, src, dst, nb)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        B.sky_derivative(ctx, 1, src, dst, nb)
    e1.record(st)
    torch.cuda.synchronize(dev)
    B.sky_destroy(ctx)
    ms = e0.elapsed_time(e1) / reps
    byt = 2.0 * nb * G * src.element_size()
    ach = byt / (ms / 1e3) / 1e9
    tr = DERIV_TRAFFIC.get((w.name, form))
    return {"kernel": "k_oz_deriv (sky_derivative along y: the spectral derivative as a "
                      "digit-split operator product on the tensor cores)" if prec == 0 else
                      "k_line_yz (sky_derivative along y: FFT line pass)",
            "bound": "hbm", "unit": "GB/s", "achieved": ach, "peak": peaks["hbm_gbs"],
            "frac": ach / peaks["hbm_gbs"], "avg_launch_ms": ms, "launches_timed": reps,
            "arrays": nb, "algorithmic_bytes_per_launch": byt,
            "work": "per launch: read and write every complex point of the 2N arrays once",
            "traffic": tr,
            "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of "
                               "the same shapes (writes still dirty in L2 at the kernel's end are "
                               "written back later)") if tr else "not captured for this workload "
                                                                 "and form",
            "peak_source": "measured HBM copy bandwidth (MEASURED_PEAKS.json, burst)"}


def fma_peaks(dev):
    """FP64 and FP32 FMA rates of this GPU (TFLOP/s), measured with the
    library's FMA-chain probe kernel (best of 5 launches after 2 warm-ups,
    CUDA events on the launching stream)."""
    import torch
    from paper_1610_07522_gb300 import binding as B
    st = torch.cuda.current_stream(dev)
    out = {}
    for name, fp64, iters in (("fp64", 1, 4000), ("fp32", 0, 100000)):
        for _ in range(2):
            B.sky_fma_probe(fp64, 4, iters, st.cuda_stream)
        best = 0.0
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fl = B.sky_fma_probe(fp64, 4, iters, st.cuda_stream)
            e1.record(st)
            torch.cuda.synchronize(dev)
            best = max(best, fl / (e0.elapsed_time(e1) / 1e3) / 1e12)
        out[name] = best
    return out


def hpsi_work(grid, csize):
    """Algorithmic work of one spinor h.psi (sky_apply_h): per spatial axis j a
    gradient and a divergence sweep over both spin components (2G points),
    each a forward and an inverse 1D FFT along j at 5 n log2 n flops per
    transform of n points, plus about 150 G pointwise flops; bytes: read psi
    and write h psi once (2 x 2G complex values)."""
    import math
    G = grid[0] * grid[1] * grid[2]
    flops = sum(2 * 2 * G * 2 * 5 * math.log2(n) for n in grid) + 150 * G
    return flops, 2 * 2 * G * csize


def call_rooflines(events, grid, prec, peaks, csize):
    """Per-call rooflines from CUDA-event durations of the single-stream step:
    sky_apply_h against the FP64 (FP32) FMA pipe and HBM, the overlap and the
    recombination against the tensor pipe (their digit or piece products)."""
    G = grid[0] * grid[1] * grid[2]
    V = 2 * G
    out = {}

    def mean_ms(kind):
        ev = events.get(kind, [])
        return sum(e0.elapsed_time(e1) for _, e0, e1 in ev) / max(1, len(ev)), ev

    ms, ev = mean_ms("apply_h")
    if ev:
        f1, b1 = hpsi_work(grid, csize)
        fl = sum(I for I, _, _ in ev) * f1 / len(ev)
        by = sum(I for I, _, _ in ev) * b1 / len(ev)
        pk = peaks["fp64" if prec == 0 else "fp32"]
        out["apply_h"] = {
            "kernel": "sky_apply_h (line-pass FFTs, k_h_local, k_h_sum)",
            "bound": "alu", "unit": "TFLOP/s", "avg_call_ms": ms,
            "mean_I": sum(I for I, _, _ in ev) / len(ev),
            "achieved": fl / (ms / 1e3) / 1e12, "peak": pk,
            "frac": fl / (ms / 1e3) / 1e12 / pk,
            "peak_source": (f"measured {'FP64' if prec == 0 else 'FP32'} FMA rate (sky_fma_probe, this run)"
                            + ("; in the FP64 form the derivative passes are tensor-core operator "
                               "products and the pointwise terms double-float FP32 work, so this "
                               "is an FP64-equivalent rate, not a pipe fraction" if prec == 0 else "")),
            "hbm_algorithmic_GBps": by / (ms / 1e3) / 1e9,
            "hbm_frac": by / (ms / 1e3) / 1e9 / peaks["hbm_gbs"],
            "work": "per spinor: 40 G sum_j log2 n_j + 150 G flops, 2 x 2G complex values moved"}
    for kind, tri in (("overlap", True), ("rotate", False)):
        ms, ev = mean_ms(kind)
        if not ev:
            continue
        n = NPROD[prec]
        full = prec in (2, 3)   # the split-BF16 forms compute the whole product
        f64eq = sum((8.0 * V * I * (I + 1) / 2) if (tri and not full) else 8.0 * V * I * I
                    for I, _, _ in ev) / len(ev)
        ach = n * f64eq / (ms / 1e3) / 1e12
        out[kind] = {
            "kernel": f"sky_{kind} (digit split + k_oz_gemm tcgen05 + reduce)" if prec in (0, 1)
                      else f"sky_{kind} (bf16 split + k_gemm_bf16 tcgen05)",
            "bound": "tensor", "unit": "TFLOP/s", "avg_call_ms": ms,
            "achieved": ach, "peak": peaks["bf16_tflops"], "frac": ach / peaks["bf16_tflops"],
            "peak_source": "measured dense BF16 burst (MEASURED_PEAKS.json)",
            "products": n,
            "fp64_equivalent_tflops": f64eq / (ms / 1e3) / 1e12,
            "work": ("products x 8 V I(I+1)/2 (lower triangle)" if (tri and not full)
                     else "products x 8 V I^2")}
    return out


def probe_batched(args):
    """One eager iteration of the 64-box batched form (after loading, two
    iterations and the batch autotuner), inside the NVTX range "probe", for
    an ncu launch list of exactly that iteration (ncu --nvtx --nvtx-include
    "probe/")."""
    import torch
    from paper_1610_07522_gb300 import binding as B
    from paper_1610_07522_gb300 import inputs as IN
    from paper_1610_07522_gb300.batched import BatchSolver
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    bs = BatchSolver(IN.batched_workloads(64), prec=FORMS[args.form], device=dev)
    bs.load()
    bs.step_eager()
    bs.step_eager()
    bs.tune(reps=2)
    bs.step_eager()
    torch.cuda.synchronize(dev)
    n0 = B.sky_kernel_launches()
    torch.cuda.nvtx.range_push("probe")
    bs.step_eager()
    torch.cuda.synchronize(dev)
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"probe_call": "batched", "form": args.form, "instances": len(bs.boxes),
                      "launches": B.sky_kernel_launches() - n0}))
    bs.close()
    return 0


def probe_call(args):
    """One library call on the workload's shapes (random states), for an ncu
    capture of exactly that call's kernels; prints the number of library
    launches the call made (the last ones of the capture)."""
    import torch
    from paper_1610_07522_gb300 import binding as B
    from paper_1610_07522_gb300 import inputs as IN
    if args.probe_call == "batched":
        return probe_batched(args)
    w = IN.WORKLOADS[args.workload]
    prec = FORMS[args.form]
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream(dev)
    I = w.N
    ctx = B.sky_init(w.grid, w.dx, w.params, w.coulomb, w.twist, prec, I, st.cuda_stream)
    if args.line_arith is not None:
        B.sky_tune_set(ctx, B.SKY_KNOB_LINE_ARITH, args.line_arith)
    nx, ny, nz = w.grid
    G = nx * ny * nz
    cd = torch.complex128 if prec == 0 else torch.complex64
    gen = torch.Generator(device=dev).manual_seed(1)
    psi = torch.randn((I, 2, nz, ny, nx), dtype=cd, device=dev, generator=gen) / G ** 0.5
    out = torch.zeros_like(psi)
    f64 = dict(dtype=torch.float64, device=dev)
    U = torch.full((G,), -40.0, **f64)
    Bf = torch.full((G,), 20.0, **f64)
    W = torch.zeros((3, G), **f64)
    X = torch.zeros((I, I), dtype=torch.complex128, device=dev)
    M = torch.eye(I, dtype=torch.complex128, device=dev)
    torch.cuda.synchronize(dev)
    n0 = B.sky_kernel_launches()
    if args.probe_call == "apply_h":
        B.sky_apply_h(ctx, U, Bf, W, psi, out, I)
    elif args.probe_call == "overlap":
        B.sky_overlap(ctx, psi, psi, I, X)
    elif args.probe_call == "rotate":
        B.sky_rotate(ctx, psi, M, I, out)
    elif args.probe_call == "ritz":
        # the batched Rayleigh-Ritz solve of both species (I = N and Z):
        # Hermitian H with a spread spectrum, C = identity
        Is = [w.N, w.Z]
        Hs, Cs, Ms, ls = [], [], [], []
        for n in Is:
            h = torch.randn((n, n), dtype=torch.complex128, device=dev, generator=gen) * 0.1
            h = h + h.conj().T + torch.diag(torch.linspace(-60.0, 20.0, n, dtype=torch.float64,
                                                           device=dev)).to(torch.complex128)
            Hs.append(torch.view_as_real(h.contiguous()))
            Cs.append(torch.view_as_real(torch.eye(n, dtype=torch.complex128, device=dev)))
            Ms.append(torch.zeros((n, n, 2), dtype=torch.float64, device=dev))
            ls.append(torch.zeros(n, dtype=torch.float64, device=dev))
        torch.cuda.synchronize(dev)
        n0 = B.sky_kernel_launches()
        B.sky_subspace_diag_batched(ctx, Hs, Cs, Is, Ms, ls)
    B.sky_sync(ctx)
    print(json.dumps({"probe_call": args.probe_call, "workload": args.workload, "form": args.form,
                      "I": I, "launches": B.sky_kernel_launches() - n0}))
    B.sky_destroy(ctx)
    return 0


# ---------------------------------------------------------------- GPU arm
def run_gpu(args):
    import numpy as np
    import torch
    from paper_1610_07522_gb300 import binding as B
    from paper_1610_07522_gb300 import inputs as IN
    from paper_1610_07522_gb300.solver import Solver

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = _maybe_init_pg(ws, "nccl")
    dev = torch.device("cuda", local)
    w = IN.WORKLOADS[args.workload]
    inp = IN.make_inputs(w)
    prec = FORMS[args.form]
    # neutrons and protons on separate contexts and streams (bit-identical to one
    # stream; the single-stream step is reported beside it)
    s = Solver(w, prec=prec, device=dev, concurrent_species=True)
    s.set_eigen_method(EIGEN[args.eigen])
    s.load(inp["psi0"], inp.get("rho0"), inp.get("tau0"))
    units = 2 * (w.N + w.Z)

    for _ in range(args.warmup):
        s.step()
    s.sync()
    eager_ms = None
    if args.graph:
        # the same steps enqueued call by call, for the record; then the
        # iteration captured once as a CUDA graph and replayed
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        for _ in range(args.steps):
            s.step()
        e1.record(s.stream)
        torch.cuda.synchronize()
        eager_ms = e0.elapsed_time(e1) / args.steps
        s.capture()
        for _ in range(args.warmup):
            s.step()
        s.sync()
    sampler = ClockSampler(_gpu_smi_id(local))
    B.sky_stats(s.ctx, reset=True)
    _barrier(dist)
    torch.cuda.synchronize()
    sampler.start()
    launches0 = B.sky_kernel_launches()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(s.stream)
    for _ in range(args.steps):
        s.step()
    t1.record(s.stream)
    torch.cuda.synchronize()
    launches = B.sky_kernel_launches() - launches0
    graphed = s.graph is not None
    if graphed:                  # replays launch no kernels from the host
        launches = s.launches_per_step * args.steps
    solver_stats = B.sky_stats(s.ctx)
    _barrier(dist)
    clocks = sampler.stop()
    s.sync()
    ms = t0.elapsed_time(t1) / args.steps
    ms_max = _max_over_ranks(ms, dist, dev)
    value = ws * units / (ms_max / 1e3)

    V = 2 * s.G
    csize = s.psi[0].element_size()
    peaks, peak_src = _measured_peaks()
    peaks = dict(peaks)
    probe = fma_peaks(dev)
    peaks.update(probe)

    # the same step with both species on one context and stream; then the same
    # steps again with CUDA events around every sky_apply_h, sky_overlap and
    # sky_rotate call (per-call rooflines; the events sit between the calls)
    sc = Solver(w, prec=prec, device=dev)
    sc.set_eigen_method(EIGEN[args.eigen])
    sc.load(inp["psi0"], inp.get("rho0"), inp.get("tau0"))
    for _ in range(args.warmup):
        sc.step()
    sc.sync()
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record(sc.stream)
    for _ in range(args.steps):
        sc.step()
    c1.record(sc.stream)
    torch.cuda.synchronize()
    conc_ms = c0.elapsed_time(c1) / args.steps
    # each species' eigensolve on its own stream (two independent chains up to
    # the densities) instead of the batched solve of both
    sp = Solver(w, prec=prec, device=dev, concurrent_species=True, split_eigensolve=True)
    sp.set_eigen_method(EIGEN[args.eigen])
    sp.load(inp["psi0"], inp.get("rho0"), inp.get("tau0"))
    for _ in range(args.warmup):
        sp.step()
    sp.sync()
    c0.record(sp.stream)
    for _ in range(args.steps):
        sp.step()
    c1.record(sp.stream)
    torch.cuda.synchronize()
    split_ms = c0.elapsed_time(c1) / args.steps
    sp.close()
    sc.call_events = {}
    for _ in range(args.steps):
        sc.step()
    sc.sync()
    torch.cuda.synchronize()
    calls = call_rooflines(sc.call_events, w.grid, prec, peaks, csize)
    # where a single-stream step spends its time: CUDA events around every call
    breakdown = {k: sum(e0.elapsed_time(e1) for _, e0, e1 in ev) / args.steps
                 for k, ev in sc.call_events.items()}
    sc.call_events = None
    sc.close()
    # the h.psi call beside the contractions (call-level), and the line's
    # roofline: the dominant kernel of the step, timed live on its own
    ah = dict(calls.get("apply_h", {}))
    tps = HPSI_TRAFFIC_PER_SPINOR.get((args.workload, args.form))
    if ah:
        ah["traffic"] = tps * ah["mean_I"] if tps else None
        ah["traffic_source"] = (
            "ncu dram__bytes_read.sum + dram__bytes_write.sum over the kernels of one sky_apply_h "
            "call (bench.py --probe-call apply_h) per spinor, times this run's mean I per call"
            if ah["traffic"] is not None else "not captured for this workload and form")
        ah["fma_peaks_tflops"] = probe
        calls["apply_h"] = ah
    roof = derivative_roofline(dev, w, prec, peaks, args.form)

    # end to end through the public API with pinned host buffers
    host = {
        "psi": [inp_t.pin_memory() for inp_t in (s.psi[0].cpu(), s.psi[1].cpu())],
        "U": s.U.cpu().pin_memory(), "B": s.Bf.cpu().pin_memory(), "W": s.W.cpu().pin_memory(),
    }
    eout_host = torch.zeros(8, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in host["psi"]) + sum(
        host[k].numel() * host[k].element_size() for k in ("U", "B", "W"))
    d2h = eout_host.numel() * eout_host.element_size()
    e2e_steps = max(3, min(args.steps, 10))
    s.step_host(host, eout_host)
    torch.cuda.synchronize()
    _barrier(dist)
    ta = time.perf_counter()
    for _ in range(e2e_steps):
        s.step_host(host, eout_host)
    e2e_dt = (time.perf_counter() - ta) / e2e_steps
    e2e_dt = _max_over_ranks(e2e_dt, dist, dev)
    e2e_value = ws * units / e2e_dt

    # time-dependent stepping (predictor-corrector pairs of order-6 Taylor
    # propagations) of the same states, FP64 or the chosen form
    td = None
    if not args.no_td:
        from paper_1610_07522_gb300.td import TimeStepper
        ts = TimeStepper(s, order=6)
        ts.init_fields()
        E0 = ts.energy()
        for _ in range(2):
            ts.step(0.1)
        s.sync()
        k = 5
        d0 = torch.cuda.Event(enable_timing=True)
        d1 = torch.cuda.Event(enable_timing=True)
        d0.record(s.stream)
        for _ in range(k):
            ts.step(0.1)
        d1.record(s.stream)
        torch.cuda.synchronize()
        td_ms = d0.elapsed_time(d1) / k
        E1 = ts.energy()
        td = {"dt_fm_per_c": 0.1, "taylor_order": 6, "steps_timed": k, "ms_per_step": td_ms,
              "spinor_applies_per_s": 2 * 6 * units / 2 / (td_ms / 1e3),
              "energy_drift_rel_over_7_steps": abs(E1 - E0) / abs(E0),
              "note": "each step: half step with h(t), midpoint mean field, full step with it "
                      "(12 h.psi per state), densities, mean field, energy"}
        del ts

    conv = None
    nets = {}
    if rank == 0 and not args.no_convergence:
        conv = convergence_leg(dev, nets_out=nets)
    batched = None
    if rank == 0 and not args.no_batched:
        batched = batched_leg(dev)
    production = None
    if rank == 0 and not args.no_production:
        production = production_leg(dev)
    conv3 = None
    if rank == 0 and not args.no_convergence:
        conv3 = convergence_config3_leg(dev, nets.get("net_configs123"))
    config5 = None
    if rank == 0 and not args.no_config5:
        config5 = config5_leg(dev, nets.get("net_configs123"))

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        r, dt, _ = cpu_baseline_sample(w, inp, 1.0)
        cpu = {"value": r, "unit": "spinor-applies/s", "cores": _cpu_threads(), "kind": "oracle",
               "sample": f"one full oracle iteration of the same workload ({dt:.1f} s)"}

    line = {
        "metric": "h.psi spinor-applies/s (full iteration)", "value": value,
        "unit": "spinor-applies/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[args.form], "data": "synthetic",
        "config": {"workload": args.workload, "grid": list(w.grid), "dx_fm": list(w.dx),
                   "N": w.N, "Z": w.Z, "coulomb": w.coulomb, "precision": args.form,
                   "eigensolver": args.eigen,
                   "parallelism": f"replicas x{ws}",
                   "l2": f"working set (psi, phi, h psi: {3 * s.psi[0].element_size() * V * (w.N + w.Z) / 1e9:.2f} GB) exceeds L2 (129 MB), no flush"},
        "roofline": roof,
        "roofline_calls": calls,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "spinor-applies/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "solver_stats_timed_steps": solver_stats,
        "graph": {"captured": graphed,
                  "eager_ms_per_step": eager_ms,
                  "note": "the timed steps replay one CUDA graph of the iteration (captured "
                          "after the warm-up); eager_ms_per_step: the same steps enqueued call "
                          "by call"},
        "single_stream": {"ms_per_step": conc_ms, "value": ws * units / (conc_ms / 1e3),
                          "calls_ms_per_step": breakdown,
                          "note": "both species on one context and stream (the main number "
                                  "runs them on two); calls_ms_per_step: CUDA events around "
                                  "each library call of a separate single-stream run"},
        "split_eigensolve": {"ms_per_step": split_ms, "value": ws * units / (split_ms / 1e3),
                             "note": "two streams, each species' Loewdin and Rayleigh-Ritz solve "
                                     "on its own stream (the main number: one batched solve)"},
        "clocks": clocks,
        "time_dependent": td,
        "convergence": conv,
        "batched": batched,
        "production_A6000": production,
        "convergence_32cubed_700n300p": conv3,
        "learned_at_scale_64cubed": config5,
    }
    s.close()
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--form", default="fp64", choices=sorted(FORMS),
                    help="spinor precision form (fp64: the paper's FP64 method)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", dest="graph", action="store_false",
                    help="time the steps enqueued call by call instead of as a CUDA graph")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 64-box batched (CUDA graph) form")
    ap.add_argument("--no-config5", action="store_true",
                    help="skip the 64^3, 5600 n + 2400 p learned-form leg")
    ap.add_argument("--no-production", action="store_true",
                    help="skip the A = 6000 production shapes (32^3, 48^3)")
    ap.add_argument("--no-td", action="store_true",
                    help="skip the time-dependent stepping leg")
    ap.add_argument("--no-convergence", action="store_true",
                    help="skip the time-to-convergence comparison of the forms")
    ap.add_argument("--probe-call", default=None, choices=["apply_h", "overlap", "rotate", "ritz", "batched"],
                    help="run one library call on the workload's shapes and exit (for ncu)")
    ap.add_argument("--line-arith", type=int, default=None, choices=[0, 1],
                    help="--probe-call only: FP64 form's derivative line passes in FP64 (0) "
                         "or double-float (1, the default)")
    ap.add_argument("--eigen", default="auto", choices=sorted(EIGEN),
                    help="FP64 eigensolver of the timed steps (auto: tridiagonal route for "
                         "large species, batched Jacobi for many small problems)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.probe_call:
        return probe_call(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
