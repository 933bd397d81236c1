"""Autotuner of the launch-shape knobs of libsky (include/sky.h, "Tunable
launch shapes"): FFT line-pass block shapes, the K-split counts of the
overlap contractions and the block count of the batched eigensolver.

Each knob's candidate values are timed with CUDA events on the caller's own
workload (the solver's buffers and matrices, the call the knob affects), and
the fastest is kept.  Results can be cached in a JSON file keyed by GPU,
grid, particle numbers and precision form.
"""
from __future__ import annotations

import json
import os
import statistics

import torch

from . import binding as B

CANDIDATES = {
    B.SKY_KNOB_LINE_YZ: (32, 64, 128),
    B.SKY_KNOB_LINE_X: (16, 32, 64),
    B.SKY_KNOB_OVERLAP_WAVES: (1, 2),
    B.SKY_KNOB_TC_WAVES: (1, 2, 4),
    B.SKY_KNOB_TC_TILE_N: (128, 256),
}
# boxes that share the GPU (a batch) may also take the fewest K splits
BATCH_CANDIDATES = dict(CANDIDATES)
BATCH_CANDIDATES[B.SKY_KNOB_TC_WAVES] = (0, 1, 2, 4)
NAMES = {B.SKY_KNOB_LINE_YZ: "line_yz", B.SKY_KNOB_LINE_X: "line_x",
         B.SKY_KNOB_OVERLAP_WAVES: "overlap_waves", B.SKY_KNOB_TC_WAVES: "tc_waves",
         B.SKY_KNOB_TC_TILE_N: "tc_tile_n", B.SKY_KNOB_FUSED_H: "fused_h",
         B.SKY_KNOB_JACOBI_BLOCKS: "jacobi_blocks"}
TC_FORMS = (B.SKY_F32_BF16X3, B.SKY_F32_BF16X6)


def _time(fn, stream, reps):
    """Median CUDA-event time (ms) of fn() on ``stream`` after one warm call."""
    fn()
    out = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return statistics.median(out)


def _pick(ctx, knob, values, fn, stream, reps):
    times = {}
    for v in values:
        B.sky_tune_set(ctx, knob, v)
        times[v] = _time(fn, stream, reps)
    best = min(times, key=times.get)
    B.sky_tune_set(ctx, knob, best)
    return best, times


def _key(solver):
    name = torch.cuda.get_device_name(solver.device)
    return f"{name}|{'x'.join(map(str, solver.w.grid))}|{solver.I[0]}n{solver.I[1]}p|prec{solver.prec}"


def tune_box(solver, reps=5, cache=None):
    """Tune the line-pass and overlap knobs of ``solver`` on its species with
    the most states (its psi must hold loaded states).  Returns
    {knob name: (chosen value, {value: ms})}."""
    key = _key(solver)
    if cache and os.path.exists(cache):
        with open(cache) as f:
            got = json.load(f).get(key)
        if got:
            apply(solver.ctx, got)
            return {k: (v, None) for k, v in got.items()}
    q = 0 if solver.I[0] >= solver.I[1] else 1
    I, ctx, st = solver.I[q], solver.ctx, solver.stream
    h = lambda: B.sky_apply_h(ctx, solver.U[q], solver.Bf[q], solver.W[q], solver.psi[q], solver.h[q], I)
    ov = lambda: B.sky_overlap(ctx, solver.psi[q], solver.h[q], I, solver.H[q])
    res = {}
    for knob in (B.SKY_KNOB_LINE_YZ, B.SKY_KNOB_LINE_X):
        res[NAMES[knob]] = _pick(ctx, knob, CANDIDATES[knob], h, st, reps)
    if solver.prec in TC_FORMS:
        rot = lambda: B.sky_rotate(ctx, solver.phi[q], solver.M[q], I, solver.h[q])
        res[NAMES[B.SKY_KNOB_TC_TILE_N]] = _pick(ctx, B.SKY_KNOB_TC_TILE_N,
                                                 CANDIDATES[B.SKY_KNOB_TC_TILE_N],
                                                 lambda: (ov(), rot()), st, reps)
        res[NAMES[B.SKY_KNOB_TC_WAVES]] = _pick(ctx, B.SKY_KNOB_TC_WAVES,
                                                CANDIDATES[B.SKY_KNOB_TC_WAVES], ov, st, reps)
    else:
        knob = B.SKY_KNOB_OVERLAP_WAVES
        res[NAMES[knob]] = _pick(ctx, knob, CANDIDATES[knob], ov, st, reps)
    torch.cuda.synchronize(solver.device)
    if cache:
        data = {}
        if os.path.exists(cache):
            with open(cache) as f:
                data = json.load(f)
        data[key] = {k: v[0] for k, v in res.items()}
        with open(cache, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
    return res


def apply(ctx, settings):
    """Set knob values from {knob name: value}."""
    by_name = {v: k for k, v in NAMES.items()}
    for name, value in settings.items():
        B.sky_tune_set(ctx, by_name[name], value)


def tune_eigensolver(eig_ctx, run_solve, stream, reps=3):
    """Tune the block count of the cooperative eigensolver of ``eig_ctx`` by
    timing ``run_solve()`` (a batched solve on that context)."""
    top = B.sky_tune_get(eig_ctx, B.SKY_KNOB_JACOBI_BLOCKS_MAX)
    values = sorted({max(1, top // 4), max(1, top // 2), top})
    return _pick(eig_ctx, B.SKY_KNOB_JACOBI_BLOCKS, values, run_solve, stream, reps)


def _settable(ctx, knob, value):
    """Whether the context accepts the value (leaving the knob as it was)."""
    old = B.sky_tune_get(ctx, knob)
    try:
        B.sky_tune_set(ctx, knob, value)
    except B.SkyError:
        return False
    B.sky_tune_set(ctx, knob, old)
    return True


def _concurrent(boxes, main, fn):
    """fn(box) for every box on its own stream, forked from and joined to
    ``main`` (how the boxes of a batch run)."""
    ev = torch.cuda.Event()
    ev.record(main)
    for s in boxes:
        s.stream.wait_event(ev)
        fn(s)
    for s in boxes:
        e = torch.cuda.Event()
        e.record(s.stream)
        main.wait_event(e)


def _pick_batch(boxes, knob, values, fn, main, reps):
    """Like _pick, with the knob set on every box of ``boxes`` and fn run on
    all of them at once (each box on its own stream), timed on ``main``."""
    times = {}
    for v in values:
        for s in boxes:
            B.sky_tune_set(s.ctx, knob, v)
        times[v] = _time(lambda: _concurrent(boxes, main, fn), main, reps)
    best = min(times, key=times.get)
    for s in boxes:
        B.sky_tune_set(s.ctx, knob, best)
    return best, times


def tune_batch(bs, reps=5, cache=None):
    """Tune a BatchSolver.  The boxes of one shape (grid, particle numbers,
    precision) share their knobs, and each candidate is timed on all boxes of
    that shape running together, each on its own stream, since that is how
    they run in the batch: FFT line-pass block shapes on h psi, the FP32 h psi
    as fused per-axis passes or general passes (where both exist), then for
    the split-BF16 forms the GEMM tile width (128 x 128 or 128 x 256, on the
    overlap and the recombination) and the overlap's K splits (down to the
    fewest the accumulation bound allows), else the FMA overlap's splits.
    The shared eigensolver's Jacobi block count is tuned only when the batch
    takes the Jacobi route (needs one iteration done).  Returns the choices."""
    shapes = {}
    for s in bs.boxes:
        shapes.setdefault((tuple(s.w.grid), s.I, s.prec), []).append(s)
    main = torch.cuda.current_stream(bs.device)
    out = {}
    for shape, boxes in shapes.items():
        def q_of(s):
            return 0 if s.I[0] >= s.I[1] else 1

        def h(s):
            q = q_of(s)
            B.sky_apply_h(s.ctx, s.U[q], s.Bf[q], s.W[q], s.psi[q], s.h[q], s.I[q])

        def ov(s):
            q = q_of(s)
            B.sky_overlap(s.ctx, s.psi[q], s.h[q], s.I[q], s.H[q])

        def ovrot(s):
            q = q_of(s)
            B.sky_overlap(s.ctx, s.psi[q], s.h[q], s.I[q], s.H[q])
            B.sky_rotate(s.ctx, s.phi[q], s.M[q], s.I[q], s.h[q])

        res = {}
        fusable = _settable(boxes[0].ctx, B.SKY_KNOB_FUSED_H, 1)
        if fusable:
            # line-pass shapes on the general h psi passes, which use them
            for s in boxes:
                B.sky_tune_set(s.ctx, B.SKY_KNOB_FUSED_H, 0)
        for knob in (B.SKY_KNOB_LINE_YZ, B.SKY_KNOB_LINE_X):
            res[NAMES[knob]] = _pick_batch(boxes, knob, BATCH_CANDIDATES[knob], h, main, reps)
        if fusable:
            # the FP32 h psi as fused per-axis passes or as the general passes
            res[NAMES[B.SKY_KNOB_FUSED_H]] = _pick_batch(boxes, B.SKY_KNOB_FUSED_H, (0, 1), h,
                                                         main, reps)
        if boxes[0].prec in TC_FORMS:
            res[NAMES[B.SKY_KNOB_TC_TILE_N]] = _pick_batch(
                boxes, B.SKY_KNOB_TC_TILE_N, BATCH_CANDIDATES[B.SKY_KNOB_TC_TILE_N], ovrot, main, reps)
            res[NAMES[B.SKY_KNOB_TC_WAVES]] = _pick_batch(
                boxes, B.SKY_KNOB_TC_WAVES, BATCH_CANDIDATES[B.SKY_KNOB_TC_WAVES], ov, main, reps)
        else:
            knob = B.SKY_KNOB_OVERLAP_WAVES
            res[NAMES[knob]] = _pick_batch(boxes, knob, BATCH_CANDIDATES[knob], ov, main, reps)
        out[str(shape)] = res
    torch.cuda.synchronize(bs.device)
    B.sky_stats(bs.eig, reset=True)
    bs.eigensolve()
    torch.cuda.synchronize(bs.device)
    if B.sky_stats(bs.eig)["jacobi_solves"] > 0:
        out["jacobi_blocks"] = tune_eigensolver(bs.eig, bs.eigensolve, main, reps=max(1, reps // 2))
    else:
        out["eigensolver"] = ("tridiagonal, teams", None)
    return out
