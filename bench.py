"""Benchmark of the RIS field hot path on the room workload (127-element hexagonal RIS on one wall of
a 6x4x3 m room with 40 boxes, 256x256 receivers at 1.2 m, specular order <= 2 on both legs, 28 GHz).

One step = trace_paths (candidates, BVH occlusion, direct-leg visibility, path records, c_m, E0)
+ eval_field for the workload's configurations, with the scene, RIS and receivers resident in HBM.
Metric: RIS field evaluations per second, one unit = (receiver, RIS element, Rx-leg path, config).

Prints one JSON line (rank 0). `--impl reference` times the FP64 CPU oracle on the same workload and
metric (bounded receiver samples per step) instead.
"""
from __future__ import annotations

import argparse
import copy
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2402_13034_gb300 import scenarios as S  # noqa: E402
from paper_2402_13034_gb300.replicas import combine_over_ranks, rank_receivers  # noqa: E402

METRIC = "RIS field evals/s (rx*elem*path*config)"
UNIT = "evals/s"


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------------------------------------------
# algorithmic work per kernel (counted from the formulas, not from the binary)
# ------------------------------------------------------------------------------------------------
# FP32 lane operations of one field unit (one Rx-leg term b_mq times Gamma c_m, order-0 isotropic):
# 2 sub + 3 FMA for L^2, rsqrt, L, cos, sqrt, 2 mul amplitude, 3 FMA + add + div for dL, FMA + round
# + sub for the phase, sincos (2), complex scale (2 mul), complex c_m product (4) and accumulate (4).
EVAL_OPS_PER_UNIT = 32
# Per field unit, counted from the formula (not from the binary): FP32 lane operations and
# special-function (MUFU) operations of an order-0 term, and what each bounce adds. MUFU: reciprocal
# square root of L^2, square root of cos(theta_out), reciprocal of (L + D0), sine and cosine of the
# phase; per bounce a square root and a reciprocal (Fresnel). FP32 per bounce: incidence cosine
# (3 FMA, 1 mul), eps - sin^2 (2), a - s, a + s, the quotient (1 mul), the amplitude product (1 mul).
EVAL_FP32_PER_UNIT, EVAL_FP32_PER_BOUNCE = 14, 9
EVAL_MUFU_PER_UNIT, EVAL_MUFU_PER_BOUNCE = 5, 2
# One image-method candidate test (Rx x face sequence): same-side test (3 FMA, sub, 2 compares),
# and for the ~half that pass it the reflection point (sub, div, 3 sub, 3 FMA) and the in-face test
# of a two-triangle face (6 x (3 FMA + sub) + 2 min + 2 compares): counted as 8 + 0.5 * 40.
CAND_OPS_PER_TEST = 28
# BVH traversal: a visit of a four-wide node is four slab tests of 12 lane ops each (6 sub/mul and
# 6 min/max) = 48 lane ops; a triangle test is a plane distance, hit point and three edge functions
# = 20 lane ops.
VISIT_OPS, TRI_OPS = 48, 20
PRECISIONS = {0: "fp32_simt", 1: "bf16", 2: "bf16x2", 3: "fp16"}

# DRAM bytes of all launches of one step (dram__bytes_read.sum + dram__bytes_write.sum) of a dominant
# kernel from one ncu capture of the bench workload, valid only for the kernel sources it was taken
# with: a changed source reports null traffic until the capture is repeated.
DOMINANT = "k_validate"      # the kernel whose launches the timed region brackets with events
MEASURED_TRAFFIC = {
    "k_validate": {"bytes_per_step": 194.19e6, "sha256_16": "a5748581a548a124",
                   "sources": [("trace.cu", "k_validate("), ("geom.cuh", None), ("scene.cu", None)],
                   "profile": "profiles/k_validate_room_256x256_dram.md"},
}


def kernel_source_hash(sources):
    """SHA-256 (16 hex digits) of the kernel's own source: the text of the named function (from its
    name to the first line that closes it at column 0) or the whole file when no name is given."""
    import hashlib
    h = hashlib.sha256()
    for f, fn in sources:
        with open(os.path.join(ROOT, "paper_2402_13034_gb300", "csrc", f)) as fh:
            text = fh.read()
        if fn:
            a = text.index(fn)
            text = text[a:text.index("\n}\n", a) + 3]
        h.update(text.encode())
    return h.hexdigest()[:16]


def measured_traffic(kernel):
    t = MEASURED_TRAFFIC.get(kernel)
    if not t:
        return None, None
    if kernel_source_hash(t["sources"]) != t["sha256_16"]:
        return None, "kernel sources changed since the ncu capture"
    return t["bytes_per_step"], t["profile"]


def measure_peaks(ctx, R):
    """Issue rates of the FP32 FMA, special-function and FP64 FMA pipes (lane operations per second),
    from the library's microbenchmarks (best of three launches, full occupancy)."""
    kinds = {"ffma": R.MB_FFMA, "mufu_sin": R.MB_MUFU_SIN, "mufu_cos": R.MB_MUFU_COS, "mufu_rsq": R.MB_MUFU_RSQ,
             "mufu_rcp": R.MB_MUFU_RCP, "mufu_sqrt": R.MB_MUFU_SQRT, "mufu_ex2": R.MB_MUFU_EX2, "dfma": R.MB_DFMA}
    out = {}
    for name, k in kinds.items():
        ops, ms = ctx.microbench(k, 2048 if k != R.MB_DFMA else 256)
        out[name] = ops
    out["mufu"] = min(out[k] for k in ("mufu_sin", "mufu_cos", "mufu_rsq", "mufu_rcp", "mufu_sqrt"))   # the ones the field term uses
    return out


def unit_bounce_counts(ps):
    """Field units of a path set split by the bounce count of their Rx-leg path: (order 0, 1, 2)."""
    ex = ps.export()
    st = ex["stats"]
    F, M = st.n_faces, st.M
    n1 = sum(int(np.sum(s < F)) for s in ex["seqs"])
    n2 = sum(len(s) for s in ex["seqs"]) - n1
    return st.n_rx * M, n1 * M, n2 * M


def bench_free_space(ctx, R, dev, steps=20):
    """The free-space case (37-element hexagonal RIS, 32x32 receivers, LOS + order 0, 9 configurations):
    trace + eval per step as device time, the launch-latency-bound end of the workload range."""
    import torch
    w = S.free_space()
    scene, ris, rx = R.upload_workload(ctx, w)
    g = torch.from_numpy(w.gammas).to(dev)
    E = torch.empty((g.shape[0], w.n_rx), dtype=torch.complex64, device=dev)
    P = torch.empty((g.shape[0], w.n_rx), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ps = None
    for _ in range(3):
        ps = ctx.trace_paths(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, R.flags_of(w), reuse=ps)
        ctx.eval_field(ps, g, E, P)
    torch.cuda.synchronize()
    ts, te = [], []
    for _ in range(steps):
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        ps = ctx.trace_paths(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, R.flags_of(w), reuse=ps)
        b.record(stream)
        ctx.eval_field(ps, g, E, P)
        c.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(c))
        te.append(b.elapsed_time(c))
    units = ps.stats().units * g.shape[0]
    ms = float(np.median(ts))
    out = {"workload": w.name, "n_rx": w.n_rx, "elements": w.n_elem, "n_cfg": int(g.shape[0]),
           "units_per_step": units, "step_us": ms * 1e3, "eval_us": float(np.median(te)) * 1e3,
           "evals_per_s": units / (ms / 1e3), "note": "median of %d steps; trace includes its host round trips" % steps}
    E_ref = E.clone()
    for h in (ps, rx, ris, scene):
        h.close()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    gr = bench_graph(R, dev, w, E_ref, flush, steps=steps)
    out["graph"] = gr
    out["graph_step_us"] = gr["ms_per_step"] * 1e3
    return out


def bench_graph(R, dev, w, E_ref, flush, steps=20):
    """Trace + field evaluation as one CUDA graph: the asynchronous trace (no host round trip, every
    array in a workspace) and eval_field captured on a stream of their own, replayed `steps` times
    with the L2 flushed before each; device time per replay (events on the graph's stream), the
    regular step's result compared bitwise, and the workspace size."""
    import torch
    gs = torch.cuda.Stream(dev)
    ctx = R.Context(dev.index, gs.cuda_stream)
    out = {}
    with torch.cuda.stream(gs):
        scene, ris, rx = R.upload_workload(ctx, w)
        flags = R.flags_of(w)
        ws, lim = ctx.trace_workspace(scene, ris, rx, w.max_order_tx, w.max_order_rx, flags, cand_cap=512,
                                      max_paths=64, max_env=64)
        g = torch.from_numpy(np.ascontiguousarray(w.gammas, np.complex64)).to(dev)
        E = torch.empty((g.shape[0], w.n_rx), dtype=torch.complex64, device=dev)
        P = torch.empty((g.shape[0], w.n_rx), dtype=torch.float32, device=dev)
        ps = ctx.trace_paths_async(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, flags, ws, lim)
        ctx.trace_check(ps)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        graph.capture_begin(capture_error_mode="thread_local")
        try:
            ctx.trace_paths_async(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, flags, ws, lim, reuse=ps)
            ctx.eval_field(ps, g, E, P)
        finally:
            graph.capture_end()
        for _ in range(3):
            graph.replay()
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(gs)
            graph.replay()
            b.record(gs)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        ctx.trace_check(ps)
        units = ps.stats().units * g.shape[0]
        ms = float(np.median(ts))
        out = {"ms_per_step": ms, "evals_per_s": units / (ms / 1e3), "units_per_step": units,
               "workspace_bytes": int(ws.numel()), "equals_regular_step": bool(torch.equal(E, E_ref)),
               "note": "median of %d replays of one graph holding the asynchronous trace and eval_field" % steps}
        del graph
        for h in (ps, rx, ris, scene):
            h.close()
    torch.cuda.synchronize()
    return out


def bench_plain_fp32(ctx, R, dev, w, ps, gam, E, P, flush, reps=5, oracle_rx=97):
    """The field evaluation against its plain FP32 baseline (one thread per receiver, absolute FP32
    phase with sincosf, IEEE square roots and divisions) on the same path set: device time of each and
    their errors against the FP64 oracle on a deterministic receiver sample."""
    import torch
    from oracle import oracle as O
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    ctx.eval_field(ps, gam, E, P)
    t_eval = timed(lambda: ctx.eval_field(ps, gam, E, P))
    E_fast = E.cpu().numpy().T.copy()
    ctx.eval_field_plain(ps, gam, E, P)
    t_plain = timed(lambda: ctx.eval_field_plain(ps, gam, E, P))
    E_plain = E.cpu().numpy().T.copy()
    idx = np.unique(np.linspace(0, w.n_rx - 1, oracle_rx).astype(int))
    rx = w.rx_xyz[idx]
    o = O.Oracle(w)
    fld = o.field(rx)
    E_ref, _, S_ref = O.Oracle.evaluate(fld, w.gammas)
    ok = ~fld["amb"][:, None] & (S_ref > 0)
    strong = ok & (np.abs(E_ref) >= 0.05 * S_ref)
    Sd = np.where(S_ref > 0, S_ref, 1.0)

    def err(Eg):
        Eg = Eg[idx]
        return {"max_field_err_over_S": float((np.abs(Eg - E_ref) / Sd)[ok].max()),
                "max_phase_err_rad": float(np.abs(np.angle(Eg * np.conj(E_ref)))[strong].max()),
                "max_power_rel_err": float((np.abs(np.abs(Eg) ** 2 / np.abs(E_ref) ** 2 - 1))[strong].max())}

    units = ps.stats().units * gam.shape[0]
    return {"eval_ms": t_eval, "plain_fp32_eval_ms": t_plain, "eval_evals_per_s": units / (t_eval / 1e3),
            "plain_fp32_evals_per_s": units / (t_plain / 1e3), "eval_speedup": t_plain / t_eval,
            "error_eval": err(E_fast), "error_plain_fp32": err(E_plain), "oracle_receivers": int(len(idx))}


def bench_direct_legs(R, dev, grid=1000, side=64, reps=3):
    """Element -> receiver visibility of a 4,096-element square RIS (64 x 64, lambda/2) in the room,
    1M receivers: the trace with the direct legs over spatial tiles (pyramids per tile of 32
    elements, rays for undecided tiles) against one ray per element of every undecided receiver
    (RISRT_TILES=0); median trace time, kernel times of the direct legs from a profiled trace, and
    equality of the visibility bits."""
    import torch
    w = S.room(grid=grid, square_side=side)
    stream = torch.cuda.Stream(device=dev)
    ctx = R.Context(dev.index or 0, stream.cuda_stream)
    scene, ris, rx = R.upload_workload(ctx, w)
    out, bits = {"workload": f"room_{side * side}el_{grid}x{grid}_order2", "n_rx": w.n_rx, "elements": w.n_elem}, {}
    kern = ("k_tile_geom", "k_rx_aperture", "k_vis_decided", "k_super_aperture", "k_tile_aperture", "k_vis_tiles",
            "k_direct_tiles", "k_direct_settle", "k_direct_vis")
    for mode in ("tiled", "per_element"):
        if mode == "per_element":
            os.environ["RISRT_TILES"] = "0"
        try:
            ts = []
            for _ in range(reps + 1):
                torch.cuda.synchronize()
                t = time.perf_counter()
                ps = ctx.trace_paths(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, R.flags_of(w))
                stream.synchronize()
                ts.append((time.perf_counter() - t) * 1e3)
                ps.close()
            ctx.profile_enable(True)
            ctx.profile_reset()
            ps = ctx.trace_paths(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, R.flags_of(w))
            prof = ctx.profile()
            ctx.profile_enable(False)
            bits[mode] = ps.export()["vis"]
            ps.close()
        finally:
            os.environ.pop("RISRT_TILES", None)
        out[mode] = {"trace_ms": float(np.median(ts[1:])),
                     "direct_legs_ms": float(sum(prof[k][0] for k in kern if k in prof)),
                     "kernels_ms": {k: round(prof[k][0], 3) for k in kern if k in prof}}
    out["vis_equal"] = bool(np.array_equal(bits["tiled"], bits["per_element"]))
    out["speedup_direct_legs"] = out["per_element"]["direct_legs_ms"] / max(out["tiled"]["direct_legs_ms"], 1e-9)
    for h in (rx, ris, scene):
        h.close()
    ctx.close()
    return out


def bench_vector(ctx, R, dev, w, scene, rxs, ps, gam, flush, reps=5, oracle_rx=33):
    """The vector field with polarisation (vertical Tx and Rx axes) on the same path set: device time
    of one call (Tx-leg vectors, E0 and the field kernel) with received values only and with the field
    vectors too, its units/s, and its errors against the oracle's vector mode on a receiver sample."""
    import torch
    from oracle import oracle as O
    stream = torch.cuda.current_stream(dev)
    axis = np.array([0.0, 0.0, 1.0], np.float32)
    ctx.antenna_set_polarization(R.TX, axis)
    ctx.antenna_set_polarization(R.RX, axis)
    C = gam.shape[0]
    Ev = torch.empty((C, w.n_rx), dtype=torch.complex64, device=dev)
    E3 = torch.empty((C, w.n_rx, 3), dtype=torch.complex64, device=dev)

    def timed(fn):
        fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    t_rx = timed(lambda: ctx.eval_field_vec(scene, rxs, ps, gam, Ev))
    t_3 = timed(lambda: ctx.eval_field_vec(scene, rxs, ps, gam, Ev, E3))
    Eg, E3g = Ev.cpu().numpy().T, E3.cpu().numpy().transpose(1, 0, 2)
    idx = np.unique(np.linspace(0, w.n_rx - 1, oracle_rx).astype(int))
    wv = copy.copy(w)
    wv.tx = copy.copy(w.tx)
    wv.rx = copy.copy(w.rx)
    wv.tx.pol, wv.rx.pol = axis, axis
    fld = O.Oracle(wv, vector=True).field_vec(w.rx_xyz[idx])
    E_ref, _, S_ref, E3_ref, S3_ref = O.Oracle.evaluate_vec(fld, w.gammas)
    ok = ~fld["amb"]
    Sd = np.where(S_ref > 0, S_ref, 1.0)
    S3d = np.where(S3_ref > 0, S3_ref, 1.0)[..., None]
    units = ps.stats().units * C
    return {"ms_received": t_rx, "ms_with_vectors": t_3, "evals_per_s_received": units / (t_rx / 1e3),
            "evals_per_s_with_vectors": units / (t_3 / 1e3), "axes": "Tx z, Rx z",
            "max_err_received_over_S": float((np.abs(Eg[idx] - E_ref) / Sd)[ok].max()),
            "max_err_vectors_over_S3": float((np.abs(E3g[idx] - E3_ref) / S3d)[ok].max()),
            "oracle_receivers": int(ok.sum())}


def bench_gradient(ctx, R, dev, steps=200, reps=5):
    """Adjoint phase gradient on the office workload (20k triangles, 64x64 RIS, 16,384 target
    receivers, 64 starting configurations): trace, A, time of one forward+adjoint step, and a
    200-step Adam ascent."""
    import torch
    from paper_2402_13034_gb300.autograd import PhaseObjective, ascend
    w = S.office()
    scene, ris, rx = R.upload_workload(ctx, w)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ps = ctx.trace_paths(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, R.flags_of(w))
    torch.cuda.synchronize()
    t_trace = time.perf_counter() - t0
    n, M = w.n_rx, w.n_elem
    A = torch.empty((n, M), dtype=torch.complex64, device=dev)
    E0 = torch.empty(n, dtype=torch.complex64, device=dev)
    ctx.build_A(ps, A, E0)
    phases = torch.from_numpy(w.extra["phases"]).to(dev)
    Bn = phases.shape[0]
    J = torch.empty(Bn, device=dev)
    g = torch.empty((Bn, M), device=dev)
    stream = torch.cuda.current_stream(dev)
    per_prec = {}
    # FP32 CUDA cores; split-BF16 tensor cores packing A on every call; the same with A kept packed
    # (the ascent's steady state: only the phase-dependent operands are rebuilt)
    for key, prec, keep in (("fp32", 0, False), ("bf16x2_cold", 2, False), ("bf16x2", 2, True)):
        o = PhaseObjective(ctx, A, E0, precision=prec)
        ws = o.workspace(Bn)
        ctx.grad_phases(A, E0, None, phases, None, J, g, ws, prec)
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.grad_phases(A, E0, None, phases, None, J, g, ws, prec, keep_a=keep)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        per_prec[key] = float(np.median(ts))
        del ws, o
    ms = per_prec["bf16x2"]
    # steady state of an ascent loop: steps enqueued back to back without synchronising (A kept packed,
    # timeout flag checked once afterwards)
    ws = PhaseObjective(ctx, A, E0, precision=2).workspace(Bn)
    ctx.grad_phases(A, E0, None, phases, None, J, g, ws, 2)
    n_def = 20
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(n_def):
        ctx.grad_phases(A, E0, None, phases, None, J, g, ws, 2, keep_a=True, defer_check=True)
    b.record(stream)
    ctx.grad_check(ws)
    ms_deferred = a.elapsed_time(b) / n_def
    del ws
    obj = PhaseObjective(ctx, A, E0, precision=2)
    ascend(obj, phases, steps=2, lr=0.05)        # first use of autograd and Adam (one-time set-up)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, hist = ascend(obj, phases, steps=steps, lr=0.05)
    torch.cuda.synchronize()
    t_asc = time.perf_counter() - t0
    h = hist.cpu().numpy()
    st = ps.stats()
    flop = 2 * 8.0 * n * M * Bn
    out = {"workload": w.name, "triangles": int(len(w.scene.tris)), "elements": M, "targets": n, "configs": Bn,
           "trace_s": t_trace, "rx_paths": st.n_rx_paths, "ms_per_grad_step": ms,
           "ms_per_grad_step_deferred": ms_deferred,
           "precision": "bf16x2 (split BF16, tensor cores, A kept packed)",
           "ms_per_grad_step_packing_A": per_prec["bf16x2_cold"], "ms_per_grad_step_fp32": per_prec["fp32"],
           "tflops": flop / (ms / 1e3) / 1e12, "A_bytes_read_per_step": 2 * n * M * 8,
           "hbm_GBps_equiv": 2 * n * M * 8 / (ms / 1e3) / 1e9, "ascent_steps": steps,
           "ascent_s": t_asc, "ascent_ms_per_step": t_asc / steps * 1e3, "J_mean_start": float(h[0].mean()), "J_mean_end": float(h[-1].mean()),
           "J_gain_db_per_rx": float((h[-1].mean() - h[0].mean()) / n * 10 / np.log(10))}
    for hh in (ps, rx, ris, scene):
        hh.close()
    return out


def bench_serving_load(dev_index, rates=(5.0, 10.0, 20.0, 30.0), n_req=24, slots=4):
    """Latency against offered load below saturation: the serving mix (same scenes and generator as
    bench_serving) at each rate, requests submitted at their arrival times."""
    from paper_2402_13034_gb300 import serve
    scenes = {}
    for w, name in ((S.room(grid=8), "room_492tri"), (S.office(), "office_20ktri"), (S.hall(target_grid=8), "hall_200ktri")):
        w.name = name
        scenes[name] = w
    srv = serve.Server(device=dev_index, slots=slots)
    for name, w in scenes.items():
        srv.add_scene(name, w.scene)
    table = []
    try:
        warm = [serve.Request("coverage", name, w.ris, w.tx, w.rx, w.rx_xyz[:64], w.gammas[:1], w.freq_hz, 1, 1, True)
                for name, w in scenes.items() for _ in range(slots)]
        srv.drain([srv.submit(r) for r in warm])
        for k, rate in enumerate(rates):
            reqs = serve.mixed_requests(S.SEED_BASE + 40 + k, n_req, rate, scenes)
            t0 = time.perf_counter()
            futs = []
            for t_arr, r in reqs:
                dt = t0 + t_arr - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                futs.append(srv.submit(r))
            for f in futs:
                f.exception(timeout=600)
            wall = time.perf_counter() - t0
            res = [f.result() for f in futs if f.exception() is None]
            st = serve.latency_stats(res)
            table.append({"offered_req_s": rate, "served_req_s": len(res) / wall, "p50_ms": st["p50_ms"],
                          "p99_ms": st["p99_ms"], "service_p50_ms": st["service_p50_ms"],
                          "service_p99_ms": st["service_p99_ms"], "requests": n_req, "rejected": n_req - len(res)})
    finally:
        srv.close()
    return table


def bench_serving_sustained(dev_index, rate_hz: float, seconds: float, slots=4, max_wait_s=None):
    """A sustained run of the serving mix: requests arriving as a seeded Poisson stream at rate_hz for
    `seconds`, generated as they are submitted (shared-input mode: grids and configuration pools
    reused so that generation keeps up with thousands of requests per second); per request only its
    latency and queueing time are kept (outputs are dropped on completion); GPU utilisation sampled
    by nvidia-smi during the run. max_wait_s: requests not admitted within it are shed."""
    from paper_2402_13034_gb300 import serve
    scenes = {}
    for w, name in ((S.room(grid=8), "room_492tri"), (S.office(), "office_20ktri"), (S.hall(target_grid=8), "hall_200ktri")):
        w.name = name
        scenes[name] = w
    srv = serve.Server(device=dev_index, slots=slots, max_wait_s=max_wait_s)
    for name, w in scenes.items():
        srv.add_scene(name, w.scene)
    lock = threading.Lock()
    lat, que = [], []
    state = {"pending": 0, "failed": 0}
    failures = {}                                  # exception type -> [count, first message]
    all_done = threading.Event()

    def on_done(f):
        with lock:
            e = f.exception()
            if e is None:
                r = f.result()
                lat.append(r.latency_s)
                que.append(r.queue_s)
            else:
                state["failed"] += 1
                rec = failures.setdefault(type(e).__name__, [0, str(e)[:160]])
                rec[0] += 1
            state["pending"] -= 1
            if state["pending"] == 0 and state.get("submitted_all"):
                all_done.set()

    util_path = os.path.join(os.environ.get("RISRT_CLOCKS_DIR", "/tmp"), ".util.csv")
    sampler = None
    n_sub = 0
    try:
        warm = [serve.Request("coverage", name, w.ris, w.tx, w.rx, w.rx_xyz[:64], w.gammas[:1], w.freq_hz, 1, 1, True)
                for name, w in scenes.items() for _ in range(slots)]
        srv.drain([srv.submit(r) for r in warm])
        try:
            sampler = subprocess.Popen(["nvidia-smi", "-i", str(dev_index), "--query-gpu=utilization.gpu",
                                        "--format=csv,noheader,nounits", "-lms", "500"],
                                       stdout=open(util_path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            sampler = None
        t0 = time.perf_counter()
        late_max = 0.0
        for t_arr, r in serve.iter_mixed_requests(S.SEED_BASE + 60, rate_hz, scenes, shared_inputs=True):
            if t_arr > seconds:
                break
            dt = t0 + t_arr - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            else:
                late_max = max(late_max, -dt)
            with lock:
                state["pending"] += 1
            srv.submit(r).add_done_callback(on_done)
            n_sub += 1
        with lock:
            state["submitted_all"] = True
            if state["pending"] == 0:
                all_done.set()
        t_sub = time.perf_counter() - t0
        all_done.wait(timeout=1800)
        wall = time.perf_counter() - t0
    finally:
        if sampler:
            sampler.terminate()
        srv.close()
    util = []
    try:
        util = [float(x) for x in open(util_path).read().split() if x.strip()]
    except Exception:
        pass
    l_ms, q_ms = np.array(lat) * 1e3, np.array(que) * 1e3
    return {"offered_req_s": rate_hz, "seconds_of_arrivals": seconds, "requests": n_sub, "served": len(lat),
            "submitted_req_s": n_sub / t_sub, "submission_late_max_s": late_max, "max_wait_s": max_wait_s,
            "shed_queue_full": srv.shed_full, "shed_not_admitted_in_time": srv.shed_late,
            "rejected_or_failed": state["failed"],
            "failures": {k: {"count": v[0], "first": v[1]} for k, v in failures.items()},
            "served_req_s": len(lat) / wall, "wall_s": wall,
            "p50_ms": float(np.percentile(l_ms, 50)) if len(l_ms) else None,
            "p99_ms": float(np.percentile(l_ms, 99)) if len(l_ms) else None,
            "service_p50_ms": float(np.percentile(l_ms - q_ms, 50)) if len(l_ms) else None,
            "service_p99_ms": float(np.percentile(l_ms - q_ms, 99)) if len(l_ms) else None,
            "gpu_util_mean_pct": float(np.mean(util)) if util else None, "gpu_util_samples": len(util),
            "channel_hits": srv.channel_hits, "graph_replays": srv.graph_replays,
            "phase_s": {k: round(v, 3) for k, v in srv.phase_s.items()},
            "oom_retries": srv.oom_retries, "idle_trims": srv.idle_trims}


def bench_serving(dev_index, n_req=64, rate_hz=2000.0, slots=4):
    """Seeded Poisson stream (mean rate_hz) of the serving mix: scenes of 492 (room), ~20k (office)
    and ~200k (hall) triangles, RIS of 37 / 127 / 1,024 / 4,096 elements, receiver grids of 1k-1M
    points, 1-512 configurations, coverage or sweep; half the sweeps query one of four resident
    channels. Requests are submitted at their arrival times."""
    from paper_2402_13034_gb300 import serve
    scenes = {}
    for w, name in ((S.room(grid=8), "room_492tri"), (S.office(), "office_20ktri"), (S.hall(target_grid=8), "hall_200ktri")):
        w.name = name
        scenes[name] = w
    reqs = serve.mixed_requests(S.SEED_BASE + 4, n_req, rate_hz, scenes)
    srv = serve.Server(device=dev_index, slots=slots)
    for name, w in scenes.items():
        srv.add_scene(name, w.scene)
    # warm the slot contexts and scene caches (one small coverage request per scene and slot)
    warm = []
    for name, w in scenes.items():
        for _ in range(slots):
            warm.append(serve.Request("coverage", name, w.ris, w.tx, w.rx, w.rx_xyz[:64], w.gammas[:1], w.freq_hz,
                                      1, 1, True))
    try:
        srv.drain([srv.submit(r) for r in warm])
        t0 = time.perf_counter()
        futs = []
        for t_arr, r in reqs:
            dt = t0 + t_arr - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            futs.append(srv.submit(r))
        for f in futs:                       # wait for all; requests above the budget are rejected
            f.exception(timeout=600)
        wall = time.perf_counter() - t0
    finally:
        srv.close()
    done = [(f.result(), r) for f, (_, r) in zip(futs, reqs) if f.exception() is None]
    res = [d for d, _ in done]
    out = serve.latency_stats(res)
    work = sum(len(r.rx_xyz) * r.gammas.shape[1] * r.gammas.shape[0] for _, r in done)
    out.update({"requests": n_req, "rejected": n_req - len(res), "offered_rate_hz": rate_hz,
                "throughput_req_s": len(res) / wall, "slots": slots,
                "peak_admitted_bytes": srv.admission.peak, "budget_bytes": srv.admission.budget,
                "channel_budget_bytes": srv.channel_budget, "channel_hits": srv.channel_hits,
                "graph_replays": srv.graph_replays,
                "rx_elem_cfg_per_s": work / wall,
                "mix": {name: len(w.scene.tris) for name, w in scenes.items()}})
    del res, done
    return out


def st_units(ps):
    return ps.stats().units


def bench_sweep(ctx, R, dev, n_cfg=4096, reps=3, oracle_rows=48):
    """E = E0 + A Gamma for every receiver and configuration on the sweep workload (room with a
    32x32 RIS, 65,536 receivers, 4,096 two-bit configurations), per precision."""
    import torch
    from oracle import oracle as O
    w = S.sweep(n_cfg=n_cfg)
    scene, ris, rx = R.upload_workload(ctx, w)
    ps = ctx.trace_paths(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, R.flags_of(w))
    n, M = w.n_rx, w.n_elem
    A = torch.empty((n, M), dtype=torch.complex64, device=dev)
    E0 = torch.empty(n, dtype=torch.complex64, device=dev)
    G = torch.from_numpy(w.gammas).to(dev)
    P = torch.empty((n, n_cfg), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, k):
        ts = []
        for _ in range(k):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    ctx.profile_enable(True)
    ctx.build_A(ps, A, E0)
    t_A = timed(lambda: ctx.build_A(ps, A, E0), reps)
    rows = np.unique(np.linspace(0, n - 1, oracle_rows).astype(int))
    wo = S.sweep(n_cfg=n_cfg)
    wo.rx_xyz = w.rx_xyz[rows]
    fld = O.Oracle(wo).field(wo.rx_xyz)
    E_ref, P_ref, S_ref = O.Oracle.evaluate(fld, w.gammas)
    ok = ~fld["amb"]
    strong = ok[:, None] & (P_ref >= 1e-3 * P_ref.max(0, keepdims=True))
    flop = 8.0 * n * M * n_cfg
    out = {"workload": w.name, "n_rx": n, "elements": M, "configs": n_cfg, "algorithmic_flop": flop,
           "build_A_ms": t_A, "build_A_GBps": n * M * 8 / (t_A / 1e3) / 1e9}
    for prec, name in PRECISIONS.items():
        ws = ctx.sweep_workspace(n, M, n_cfg, prec)
        ctx.sweep_configs(A, E0, G, P, prec, ws)
        ctx.profile_reset()
        ms = timed(lambda: ctx.sweep_configs(A, E0, G, P, prec, ws), reps if prec else 1)
        prof = ctx.profile()
        Pg = P[torch.from_numpy(rows).to(dev)].cpu().numpy().astype(np.float64)
        db = np.abs(10 * np.log10(np.maximum(Pg[strong], 1e-300) / P_ref[strong]))
        dE = np.abs(np.sqrt(Pg * 2 * 120 * np.pi) - np.abs(E_ref)) / np.where(S_ref > 0, S_ref, 1)
        ent = {"ms": ms, "tflops": flop / (ms / 1e3) / 1e12,
               "db_err": {"median": float(np.median(db)), "p99": float(np.percentile(db, 99)),
                          "max": float(db.max()), "frac_above_0.01dB": float(np.mean(db > 0.01))},
               "max_field_err_over_S": float(dE[ok].max())}
        kname = next((k for k in ("k_sweep_tc_pair", "k_sweep_tc") if k in prof), None)
        if kname:
            kms = prof[kname][0] / prof[kname][1]
            Kp = ((4 if prec == 2 else 2) * M + 63) // 64 * 64
            Np = (2 * n_cfg + 255) // 256 * 256
            bm = 256 if kname == "k_sweep_tc_pair" else 128
            Mp = (n + bm - 1) // bm * bm
            ent["kernel"] = kname
            ent["kernel_ms"] = kms
            ent["tensor_flop_per_launch"] = 2.0 * Mp * Np * Kp
            ent["kernel_tflops_executed"] = 2.0 * Mp * Np * Kp / (kms / 1e3) / 1e12
        out[name] = ent
    ctx.profile_enable(False)
    # the fused channel tile -> tensor-core sweep (A never materialised) against build_A + the BF16 sweep,
    # at the 128 configurations one fused call takes
    C1 = 128
    G1 = G[:C1].contiguous()
    P1 = torch.empty((n, C1), dtype=torch.float32, device=dev)
    P2 = torch.empty((n, C1), dtype=torch.float32, device=dev)
    ws1 = ctx.sweep_workspace(n, M, C1, R.PREC_BF16)

    def unfused():
        ctx.build_A(ps, A, E0)
        ctx.sweep_configs(A, E0, G1, P2, R.PREC_BF16, ws1)

    unfused()
    ctx.sweep_fused(ps, G1, P1)
    t_unf = timed(unfused, reps)
    t_fus = timed(lambda: ctx.sweep_fused(ps, G1, P1), reps)
    Pf, Pu = P1.cpu().numpy().astype(np.float64), P2.cpu().numpy().astype(np.float64)
    sel = Pu > 1e-3 * Pu.max()
    out["fused_128cfg"] = {"ms_fused": t_fus, "ms_build_A_plus_bf16_sweep": t_unf, "speedup": t_unf / t_fus,
                           "evals_per_s_fused": st_units(ps) * C1 / (t_fus / 1e3),
                           "max_db_fused_vs_unfused": float(np.max(np.abs(10 * np.log10(Pf[sel] / Pu[sel])))),
                           "A_bytes_not_written": n * M * 8}
    out["speedup_bf16_vs_fp32"] = out["fp32_simt"]["ms"] / out["bf16"]["ms"]
    out["speedup_bf16x2_vs_fp32"] = out["fp32_simt"]["ms"] / out["bf16x2"]["ms"]
    peaks = _peaks()
    pk = peaks.get("bf16_tflops", 1876.6)
    b = out["bf16"]
    out["roofline"] = {"kernel": b.get("kernel", "k_sweep_tc"), "bound": "tensor", "achieved": b.get("kernel_tflops_executed"),
                       "peak": pk, "unit": "TFLOP/s",
                       "frac": (b.get("kernel_tflops_executed") or 0) / pk, "traffic": None,
                       "peak_note": "measured bf16 burst peak (cuBLAS) of this pool" if "bf16_tflops" in peaks
                       else "fallback 1900 TF/s"}
    for h in (ps, rx, ris, scene):
        h.close()
    return out


def clocks_sampler(path):
    try:
        return subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
             "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except Exception:
        return None


def clocks_summary(path, device_index):
    try:
        rows = [r.split(",") for r in open(path).read().strip().splitlines()]
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 9 and r[0].strip() == str(device_index)]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        mx = float(rows[0][2])
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, name in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(rows)}
    except Exception:
        return None


def cpu_oracle_rate(w, n_cfg, budget_s=15.0, steps=1):
    """Time the FP64 oracle on deterministic receiver samples of the workload; returns
    (evals/s, threads, sample description, ms per sample step)."""
    from oracle import oracle as O
    o = O.Oracle(w)
    rng_idx = np.arange(w.n_rx)

    def sample(n, k):
        idx = rng_idx[(np.arange(n) * 7919 + k * 104729) % w.n_rx]
        return np.unique(idx)

    # calibrate on a few receivers
    t0 = time.perf_counter()
    o.field(w.rx_xyz[sample(32, 0)])
    per_rx = (time.perf_counter() - t0) / 32
    n = int(max(32, min(w.n_rx, budget_s / max(per_rx, 1e-6))))
    total_units, total_t = 0, 0.0
    for k in range(steps):
        idx = sample(n, k + 1)
        rx = w.rx_xyz[idx]
        paths = o.rx_paths(rx)
        units = sum(w.n_elem * (1 + len(s)) for s in paths["seqs"]) * n_cfg
        t0 = time.perf_counter()
        fld = o.field(rx)
        O.Oracle.evaluate(fld, w.gammas)
        total_t += time.perf_counter() - t0
        total_units += units
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return (total_units / total_t, threads, f"{len(idx)} of {w.n_rx} receivers per step (stride sample), {steps} step(s)",
            total_t / steps * 1e3, len(idx))


def run_reference(args, w, n_cfg):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    val, cores, samp, ms, n_sample = cpu_oracle_rate(w, n_cfg, budget_s=args.ref_budget, steps=max(1, args.steps))
    # a step of this arm is one bounded receiver sample of the workload (see cpu_baseline.sample); the
    # full grid would take about n_rx / n_sample times as long
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "ms_per_step_note": f"one step is a sample of {n_sample} of {w.n_rx} receivers, not the full grid",
            "ms_full_grid_extrapolated": ms * w.n_rx / n_sample,
            "config": {"workload": w.name, "n_rx": w.n_rx, "elements": w.n_elem, "n_cfg": n_cfg,
                       "receivers_per_step": n_sample},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": samp},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_case(args):
    """Small fixed cases for profilers: 'trace' (room workload at --grid, two traces and an eval),
    'vector' (the same with the vector field, vertical Tx and Rx axes, field vectors on), 'grad' (the
    office's 16,384 targets x 4,096 elements x 64 configurations, split-BF16 adjoint: one call packing
    A, three keeping it) and 'sweep' (16,384 receivers x 1,024 elements x 1,024 configurations,
    --precision)."""
    import torch
    from paper_2402_13034_gb300 import build as B
    from paper_2402_13034_gb300 import risrt as R
    B.build()
    ctx = R.Context(0, torch.cuda.current_stream().cuda_stream)
    if args.case in ("trace", "vector"):
        w = S.room(grid=args.grid, square_side=args.side)
        scene, ris, rx = R.upload_workload(ctx, w)
        g = torch.from_numpy(w.gammas).cuda()
        E = torch.empty((g.shape[0], w.n_rx), dtype=torch.complex64, device="cuda")
        P = torch.empty((g.shape[0], w.n_rx), dtype=torch.float32, device="cuda")
        E3 = torch.empty((g.shape[0], w.n_rx, 3), dtype=torch.complex64, device="cuda")
        axis = np.array([0.0, 0.0, 1.0], np.float32)
        ctx.antenna_set_polarization(R.TX, axis)
        ctx.antenna_set_polarization(R.RX, axis)
        ps = None
        for _ in range(2):
            ps = ctx.trace_paths(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, R.flags_of(w), reuse=ps)
            if args.case == "trace":
                ctx.eval_field(ps, g, E, P)
            else:
                ctx.eval_field_vec(scene, rx, ps, g, E, E3, P)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "grid": args.grid, "units": ps.stats().units}))
    elif args.case == "grad":
        w = S.office()
        scene, ris, rx = R.upload_workload(ctx, w)
        ps = ctx.trace_paths(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, R.flags_of(w))
        A = torch.empty((w.n_rx, w.n_elem), dtype=torch.complex64, device="cuda")
        E0 = torch.empty(w.n_rx, dtype=torch.complex64, device="cuda")
        ctx.build_A(ps, A, E0)
        phases = torch.from_numpy(w.extra["phases"]).cuda()
        J = torch.empty(phases.shape[0], device="cuda")
        g = torch.empty_like(phases)
        ws = ctx.grad_workspace(w.n_rx, phases.shape[0], w.n_elem, R.PREC_BF16X2)
        ctx.grad_phases(A, E0, None, phases, None, J, g, ws, R.PREC_BF16X2)
        for _ in range(3):
            ctx.grad_phases(A, E0, None, phases, None, J, g, ws, R.PREC_BF16X2, keep_a=True)
        torch.cuda.synchronize()
        print(json.dumps({"case": "grad", "targets": w.n_rx, "elements": w.n_elem, "configs": int(phases.shape[0])}))
    else:
        n, M, C = 16384, 1024, 1024
        rng = np.random.default_rng(0)
        A = torch.from_numpy(((rng.standard_normal((n, M)) + 1j * rng.standard_normal((n, M))) * 1e-3)
                             .astype(np.complex64)).cuda()
        G = torch.from_numpy(np.array([1, 1j, -1, -1j], np.complex64)[rng.integers(0, 4, (C, M))]).cuda()
        P = torch.empty((n, C), dtype=torch.float32, device="cuda")
        ws = ctx.sweep_workspace(n, M, C, args.precision)
        for _ in range(3):
            ctx.sweep_configs(A, None, G, P, args.precision, ws)
        torch.cuda.synchronize()
        print(json.dumps({"case": "sweep", "n": n, "M": M, "C": C, "precision": args.precision}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="risrt", choices=["risrt", "reference"])
    ap.add_argument("--grid", type=int, default=256)
    ap.add_argument("--side", type=int, default=0,
                    help="--case trace/vector: a square RIS of side x side elements instead of the 127-element hex")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-budget", type=float, default=20.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-grad", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=0.0,
                    help="also run the serving mix for this many seconds of arrivals at --serve-rate")
    ap.add_argument("--serve-slots", type=str, default="4",
                    help="stream slots of the sustained run, comma-separated for one run per count and rate")
    ap.add_argument("--serve-max-wait", type=float, default=0.0,
                    help="sustained run: shed requests not admitted within this many seconds (0: never)")
    ap.add_argument("--serve-rate", type=str, default="40",
                    help="offered rate(s) in requests/s of the sustained run, comma-separated for one run each")
    ap.add_argument("--case", choices=["trace", "vector", "grad", "sweep"], default=None,
                    help="run a small fixed case for a profiler instead of the benchmark")
    ap.add_argument("--precision", type=int, default=1)
    args = ap.parse_args()
    if args.case:
        run_case(args)
        return

    w = S.room(grid=args.grid)
    n_cfg = w.gammas.shape[0]
    if args.impl == "reference":
        run_reference(args, w, n_cfg)
        return

    import torch
    import torch.distributed as dist
    from paper_2402_13034_gb300 import build as B
    from paper_2402_13034_gb300 import risrt as R

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        dist.barrier()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ctx = R.Context(local, stream.cuda_stream)

    # each rank processes its own receiver batch (weak scaling): the grid shifted by a rank offset
    rx_host = rank_receivers(w.rx_xyz, rank)
    rx_dev = torch.from_numpy(rx_host).to(dev)
    scene, ris, _ = R.upload_workload(ctx, w)
    rxs = ctx.rx_bind(rx_dev)
    gam = torch.from_numpy(w.gammas).to(dev)
    E = torch.empty((n_cfg, w.n_rx), dtype=torch.complex64, device=dev)
    P = torch.empty((n_cfg, w.n_rx), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2
    flags = R.flags_of(w)

    ps = None

    def step():
        nonlocal ps
        ps = ctx.trace_paths(scene, ris, rxs, w.freq_hz, w.max_order_tx, w.max_order_rx, flags, reuse=ps)
        ctx.eval_field(ps, gam, E, P)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    units = ps.stats().units * n_cfg

    # timed region: per-step CUDA events on the launching stream, L2 flushed between steps
    import tempfile
    clk_path = os.path.join(os.environ.get("RISRT_CLOCKS_DIR", tempfile.gettempdir()), f".clocks_{rank}.csv")
    sampler = clocks_sampler(clk_path) if rank == 0 else None
    # inside the timed region only the dominant kernel (k_validate) is bracketed by CUDA events, for
    # its live launch duration; the per-kernel breakdown comes from profiled steps after it
    ctx.profile_only(DOMINANT)
    ctx.profile_enable(True)
    ctx.profile_reset()
    launches0 = R.launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = R.launch_count() - launches0
    prof_timed = ctx.profile()
    ctx.profile_only(None)
    ctx.profile_reset()
    n_prof_steps = min(args.steps, 5)
    for _ in range(n_prof_steps):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    prof = ctx.profile()
    ctx.profile_enable(False)
    if sampler:
        time.sleep(0.3)
        sampler.terminate()
    total_ms, units_all = combine_over_ranks(float(np.sum(times)), float(units), dev)
    ms_per_step = total_ms / args.steps
    value = units_all * args.steps / (total_ms / 1e3)

    # per-kernel shares (profiled steps after the timed region) and the dominant kernel's roofline
    # (its launches timed live, with CUDA events on its stream, inside the timed region)
    k_total = sum(v[0] for v in prof.values())
    stages = {k: {"ms_per_step": v[0] / n_prof_steps, "launches_per_step": v[1] / n_prof_steps,
                  "share": v[0] / k_total if k_total else None} for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])}
    dom = max(prof.items(), key=lambda kv: kv[1][0])[0] if prof else None
    peaks = _peaks()
    st = ps.stats()
    roof = None
    if dom:
        live = dom in prof_timed
        ms_step = (prof_timed[dom][0] / args.steps) if live else prof[dom][0] / n_prof_steps
        launches_step = (prof_timed[dom][1] / args.steps) if live else prof[dom][1] / n_prof_steps
        sm_mhz = (peaks.get("sm_max_mhz") or 2070.0)
        alu_peak = 152 * 128 * sm_mhz * 1e6 / 1e12      # T lane-ops/s: 152 SMs x 128 FP32 lanes x clock
        # work of one step; per launch it is this / launches_step, over an average launch duration of
        # ms_step / launches_step, so the ratio is the same
        if dom == "k_eval":
            work = st.units * n_cfg * EVAL_OPS_PER_UNIT
        elif dom == "k_validate":
            work = st.node_visits * VISIT_OPS + st.tri_tests * TRI_OPS
        else:
            work = None
        if work is not None:
            achieved = work / (ms_step / 1e3) / 1e12
            tstep, tnote = measured_traffic(dom)
            roof = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                    "frac": achieved / alu_peak, "traffic": tstep / launches_step if tstep else None,
                    "traffic_note": tnote, "launches_per_step": launches_step, "timed_live": live,
                    "peak_note": f"FP32 lane-op issue peak at {sm_mhz:.0f} MHz (152 SMs x 128 lanes), derived"}
            if live and dom in prof:
                # the Rx-leg and environment validations run at the same time on two streams, so the live
                # launch durations overlap; the profiled steps run every kernel alone
                ser_ms = prof[dom][0] / n_prof_steps
                roof["live_ms_per_step"] = ms_step
                roof["serialized_ms_per_step"] = ser_ms
                roof["achieved_serialized"] = work / (ser_ms / 1e3) / 1e12
                roof["frac_serialized"] = roof["achieved_serialized"] / alu_peak
        else:
            roof = {"kernel": dom, "bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
                    "traffic": None}

    # measured pipe peaks; the field kernel against the special-function and FP32 pipes (its op counts
    # per unit from the formula, split by the bounce count of each unit's path)
    mpeaks = measure_peaks(ctx, R)
    if roof is not None and dom == "k_validate":
        secs = ms_step / 1e3
        roof["node_visits_per_s"] = st.node_visits / secs
        roof["segments_per_s"] = st.n_segments / secs
        roof["candidates_per_s"] = st.n_candidates / secs
    u0, u1, u2 = unit_bounce_counts(ps)
    roof_field = None
    if "k_eval" in prof:
        ev_ms = prof["k_eval"][0] / n_prof_steps
        # the term b_mq of a (receiver, element, path) is computed once and shared by every configuration;
        # each configuration adds one complex multiply-accumulate per (receiver, element)
        mufu_ops = (u0 * EVAL_MUFU_PER_UNIT + u1 * (EVAL_MUFU_PER_UNIT + EVAL_MUFU_PER_BOUNCE)
                    + u2 * (EVAL_MUFU_PER_UNIT + 2 * EVAL_MUFU_PER_BOUNCE))
        fp32_ops = (u0 * EVAL_FP32_PER_UNIT + u1 * (EVAL_FP32_PER_UNIT + EVAL_FP32_PER_BOUNCE)
                    + u2 * (EVAL_FP32_PER_UNIT + 2 * EVAL_FP32_PER_BOUNCE)) + n_cfg * st.n_rx * st.M * 4
        units_eval = (u0 + u1 + u2) * n_cfg
        t_mufu = mufu_ops / mpeaks["mufu"]
        t_fp32 = fp32_ops / mpeaks["ffma"]
        bound = "mufu" if t_mufu >= t_fp32 else "fp32"
        roof_units = units_eval / max(t_mufu, t_fp32)
        achieved = units_eval / (ev_ms / 1e3)
        roof_field = {"kernel": "k_eval", "bound": "alu", "pipe": bound, "achieved": achieved,
                      "peak": roof_units, "unit": "units/s", "frac": achieved / roof_units, "traffic": None,
                      "ms_per_step": ev_ms, "units": units_eval, "units_by_bounces": [u0, u1, u2],
                      "mufu_ops_per_step": mufu_ops, "fp32_ops_per_step": fp32_ops,
                      "mufu_frac": (mufu_ops / (ev_ms / 1e3)) / mpeaks["mufu"],
                      "fp32_frac": (fp32_ops / (ev_ms / 1e3)) / mpeaks["ffma"],
                      "peak_note": "min over the measured MUFU and FP32 FMA issue rates of peak / ops per unit"}

    # end to end through the C ABI with host buffers (scene, RIS, receivers, configs up; P down)
    e2e = None
    if not args.no_e2e:
        rx_pin = torch.from_numpy(rx_host).pin_memory()
        g_pin = torch.from_numpy(w.gammas).pin_memory()
        P_host = torch.empty((n_cfg, w.n_rx), dtype=torch.float32).pin_memory()
        sc_ = w.scene
        h2d = (sc_.verts.nbytes + sc_.tris.nbytes + sc_.face_id.nbytes + sc_.mat_id.nbytes + sc_.mats.nbytes
               + w.ris.elem_uv.nbytes + rx_host.nbytes + w.gammas.nbytes)
        d2h = P_host.numel() * 4

        def e2e_step():
            scene2, ris2, _ = R.upload_workload(ctx, w, rx_device=rx_dev)
            rx2 = ctx.rx_upload(rx_pin.numpy())
            g2 = g_pin.to(dev, non_blocking=True)
            ps2 = ctx.trace_paths(scene2, ris2, rx2, w.freq_hz, w.max_order_tx, w.max_order_rx, flags)
            ctx.eval_field(ps2, g2, E, P)
            P_host.copy_(P, non_blocking=True)
            torch.cuda.synchronize()
            n_units = ps2.stats().units * n_cfg
            for h in (ps2, rx2, ris2, scene2):
                h.close()
            return n_units

        e2e_step()
        t_e2e, u_e2e = 0.0, 0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            u_e2e += e2e_step()
            t_e2e += time.perf_counter() - t0
        t_e2e, u_e2e = combine_over_ranks(t_e2e, u_e2e, dev)
        e2e = {"value": u_e2e / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    plain = None
    vs_baseline = None
    free = None
    vector = None
    graph = None
    if rank == 0:
        plain = bench_plain_fp32(ctx, R, dev, w, ps, gam, E, P, flush)
        # the same step with the plain FP32 field evaluation in place of eval_field
        plain_step_ms = ms_per_step - plain["eval_ms"] + plain["plain_fp32_eval_ms"]
        plain["step_ms_with_plain_eval"] = plain_step_ms
        plain["step_evals_per_s_with_plain_eval"] = units / (plain_step_ms / 1e3)
        vs_baseline = plain_step_ms / ms_per_step
        # the timed step's field (its path set carries the room's antennas; the free-space case below
        # sets the context's own)
        E_step = torch.empty_like(E)
        ctx.eval_field(ps, gam, E_step, P)
        graph = bench_graph(R, dev, w.__class__(**{**w.__dict__, "rx_xyz": rx_host}), E_step, flush, steps=10)
        free = bench_free_space(ctx, R, dev)
        vector = bench_vector(ctx, R, dev, w, scene, rxs, ps, gam, flush)
        direct = bench_direct_legs(R, dev)
        vector["vs_scalar_eval_ms"] = vector["ms_received"] / plain["eval_ms"]
    sweep = None
    if rank == 0 and not args.no_sweep:
        sweep = bench_sweep(ctx, R, dev)
    grad = None
    if rank == 0 and not args.no_grad:
        grad = bench_gradient(ctx, R, dev)
    serving = None
    if rank == 0 and not args.no_serve:
        serving = bench_serving(local)
        serving["latency_vs_load"] = bench_serving_load(local)
        if args.serve_seconds > 0:
            mw = args.serve_max_wait if args.serve_max_wait > 0 else None
            serving["sustained"] = [dict(bench_serving_sustained(local, float(r), args.serve_seconds, int(k), mw),
                                         slots=int(k))
                                    for k in args.serve_slots.split(",") for r in args.serve_rate.split(",")]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, samp, _, _ = cpu_oracle_rate(w, n_cfg, budget_s=args.cpu_budget)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": samp}

    if rank == 0:
        clk = clocks_summary(clk_path, local)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": vs_baseline,
                "vs_baseline_note": "against the same step with the plain FP32 field evaluation (one thread per "
                                    "receiver, absolute FP32 phase, sincosf) measured in this run; the paper "
                                    "prints no number",
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": w.name, "n_rx": w.n_rx, "elements": w.n_elem, "faces": st.n_faces,
                           "triangles": int(len(w.scene.tris)), "order_tx": w.max_order_tx,
                           "order_rx": w.max_order_rx, "env_paths": bool(w.env_paths), "n_cfg": n_cfg,
                           "units_per_step": units, "rx_paths": st.n_rx_paths, "env_paths_found": st.n_env_paths,
                           "tx_paths": st.n_tx_paths, "fp64_refines": st.fp64_refines,
                           "candidates": st.n_candidates, "segments": st.n_segments,
                           "bvh_node_visits": st.node_visits, "tri_tests": st.tri_tests,
                           "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"},
                "clocks": clk, "e2e": e2e, "gpu_launches": int(launches), "roofline": roof,
                "roofline_field": roof_field, "measured_peaks": mpeaks, "cpu_baseline": cpu,
                "vs_plain_fp32": plain, "free_space": free, "vector_field": vector, "graph_step": graph,
                "direct_legs_4096el": direct,
                "stages": stages, "sweep": sweep, "gradient": grad, "serving": serving}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
