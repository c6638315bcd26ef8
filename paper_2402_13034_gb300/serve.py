"""Continuous-batching request server for RIS field queries on one GPU.

Requests (coverage maps and configuration sweeps over scenes of uneven size) are admitted while a
stream slot is free and their estimated device-memory footprint fits the budget; every admitted
request runs on its own CUDA stream through its own library context, so the work of requests that
arrived at different times overlaps on the device. Scene BVHs stay resident in a cache shared by
all slots. A request's arithmetic does not depend on what else runs (per-request buffers, fixed
reduction orders), so its result is bitwise the same alone or in a mix.

The admission policy (AdmissionController) is plain host logic and is tested without a GPU.
"""
from __future__ import annotations

import math
import queue
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np


# ------------------------------------------------------------------------------------------------
# requests
# ------------------------------------------------------------------------------------------------
@dataclass
class Request:
    """kind 'coverage': P for every receiver and configuration (trace + eval_field).
    kind 'sweep': P for every receiver and configuration through the channel matrix
    (trace + build_A + tensor-core sweep)."""
    kind: str
    scene_id: str
    ris: object                  # scenarios.RIS
    tx: object                   # scenarios.Antenna
    rx: object                   # scenarios.Antenna
    rx_xyz: np.ndarray           # float32 [n, 3]
    gammas: np.ndarray           # complex64 [C, M]
    freq_hz: float = 28e9
    max_order_tx: int = 1
    max_order_rx: int = 1
    env_paths: bool = True
    precision: int = 2           # sweep precision (RISRT_PREC_*)
    arrival: float = 0.0
    rid: int = -1
    meta: dict = field(default_factory=dict)


@dataclass
class Result:
    rid: int
    P: np.ndarray                # float32 [n_rx, C] (receiver-major)
    latency_s: float
    queue_s: float
    footprint: int


def estimate_footprint(req: Request, n_faces: int) -> int:
    """Upper estimate of the device bytes one request holds while it runs."""
    n, M, C = len(req.rx_xyz), req.gammas.shape[1], req.gammas.shape[0]
    paths = n * (1 + (n_faces if req.max_order_rx >= 1 else 0) // 8 + 8)
    cap = 512
    n_ids = n_faces + (n_faces * n_faces if max(req.max_order_rx, req.max_order_tx) >= 2 else 0)
    b = paths * 96 + n * ((M + 31) // 32) * 4 + n * 64
    b += 3 * n_ids * 160 + 2 * n * cap * 4 * 6 + (64 << 10)
    b += n * C * 4 * 2 + C * M * 8 + n * 12
    if req.kind == "sweep":
        Kp = (4 * M + 63) // 64 * 64
        b += n * M * 8 + ((n + 127) // 128 * 128) * Kp * 2 + ((2 * C + 255) // 256 * 256) * Kp * 2
    return int(b)


# ------------------------------------------------------------------------------------------------
# admission (host logic only)
# ------------------------------------------------------------------------------------------------
class AdmissionController:
    """FIFO admission by stream slots and a device-memory budget. A request larger than the whole
    budget is rejected; otherwise it waits until enough in-flight requests have finished."""

    def __init__(self, budget_bytes: int, slots: int):
        self.budget = int(budget_bytes)
        self.slots = int(slots)
        self.in_use = 0
        self.running = 0
        self.peak = 0
        self._lock = threading.Lock()

    def fits_ever(self, footprint: int) -> bool:
        return footprint <= self.budget

    def try_admit(self, footprint: int) -> bool:
        with self._lock:
            if self.running < self.slots and self.in_use + footprint <= self.budget:
                self.in_use += footprint
                self.running += 1
                self.peak = max(self.peak, self.in_use)
                return True
            return False

    def release(self, footprint: int) -> None:
        with self._lock:
            self.in_use -= footprint
            self.running -= 1


# ------------------------------------------------------------------------------------------------
# server
# ------------------------------------------------------------------------------------------------
class Server:
    def __init__(self, device: int = 0, slots: int = 4, budget_bytes: int | None = None, executor=None):
        """executor(slot_index, request) -> np.ndarray replaces the GPU path (used by host tests)."""
        self.device = device
        self._executor = executor
        if budget_bytes is None:
            import torch
            free, _ = torch.cuda.mem_get_info(device)
            budget_bytes = int(free * 0.8)
        self.admission = AdmissionController(budget_bytes, slots)
        self._pending: "queue.Queue[tuple]" = queue.Queue()
        self._next_id = 0
        self._id_lock = threading.Lock()
        self._scenes = {}            # scene_id -> (host Scene, {slot: risrt scene handle})
        self._scene_lock = threading.Lock()
        self._slot_free = queue.Queue()
        self._threads = []
        self._stop = threading.Event()
        self._contexts = [None] * slots
        for s in range(slots):
            self._slot_free.put(s)
        self._dispatcher = threading.Thread(target=self._dispatch, daemon=True)
        self._dispatcher.start()

    # -- scenes --------------------------------------------------------------------------------
    def add_scene(self, scene_id: str, scene) -> None:
        """Register a scene (scenarios.Scene); its BVH is built once per slot context on first use."""
        with self._scene_lock:
            self._scenes[scene_id] = (scene, {})

    def _scene_handle(self, slot: int, ctx, scene_id: str):
        with self._scene_lock:
            if scene_id not in self._scenes:
                raise KeyError(f"unknown scene {scene_id!r}")
            sc, handles = self._scenes[scene_id]
        if slot not in handles:
            handles[slot] = ctx.scene_upload(sc.verts, sc.tris, sc.face_id, sc.mat_id, sc.mats)
        return handles[slot]

    # -- submission ------------------------------------------------------------------------------
    def submit(self, req: Request) -> Future:
        fut: Future = Future()
        with self._id_lock:
            req.rid = self._next_id
            self._next_id += 1
        req.arrival = time.perf_counter()
        problem = self._validate(req)
        if problem:
            fut.set_exception(ValueError(problem))
            return fut
        faces = self._scenes[req.scene_id][0].n_faces
        fp = estimate_footprint(req, faces)
        if not self.admission.fits_ever(fp):
            fut.set_exception(MemoryError(f"request needs ~{fp} bytes, above the budget {self.admission.budget}"))
            return fut
        self._pending.put((req, fut, fp))
        return fut

    def _validate(self, req: Request) -> str | None:
        if req.kind not in ("coverage", "sweep"):
            return f"unknown request kind {req.kind!r}"
        if req.scene_id not in self._scenes:
            return f"unknown scene {req.scene_id!r}"
        if req.rx_xyz.ndim != 2 or req.rx_xyz.shape[1] != 3 or len(req.rx_xyz) == 0:
            return "rx_xyz must be a non-empty [n, 3] array"
        if req.gammas.ndim != 2 or req.gammas.shape[1] != req.ris.elem_uv.shape[0] or req.gammas.shape[0] == 0:
            return "gammas must be [C, M] with M the RIS element count"
        if not np.all(np.isfinite(req.rx_xyz)):
            return "non-finite receiver position"
        return None

    # -- dispatch ---------------------------------------------------------------------------------
    def _dispatch(self):
        waiting = []
        while not self._stop.is_set():
            try:
                while True:
                    waiting.append(self._pending.get(timeout=0.0005 if waiting else 0.05))
            except queue.Empty:
                pass
            i = 0
            while i < len(waiting):                    # FIFO, skipping requests that do not fit yet
                req, fut, fp = waiting[i]
                if fut.cancelled():
                    waiting.pop(i)
                    continue
                if self.admission.try_admit(fp):
                    waiting.pop(i)
                    slot = self._slot_free.get()
                    t = threading.Thread(target=self._run, args=(slot, req, fut, fp), daemon=True)
                    t.start()
                    self._threads.append(t)
                else:
                    break

    def _run(self, slot: int, req: Request, fut: Future, fp: int):
        t_start = time.perf_counter()
        try:
            if not fut.set_running_or_notify_cancel():
                return
            if self._executor is not None:
                P = self._executor(slot, req)
            else:
                P = self._gpu_execute(slot, req)
            t_end = time.perf_counter()
            fut.set_result(Result(req.rid, P, t_end - req.arrival, t_start - req.arrival, fp))
        except BaseException as e:                    # noqa: BLE001 - reported through the future
            if not fut.done():
                fut.set_exception(e)
        finally:
            self.admission.release(fp)
            self._slot_free.put(slot)

    def _context(self, slot: int):
        if self._contexts[slot] is None:
            import torch
            from . import risrt as R
            stream = torch.cuda.Stream(device=self.device)
            self._contexts[slot] = (R.Context(self.device, stream.cuda_stream), stream)
        return self._contexts[slot]

    def _gpu_execute(self, slot: int, req: Request) -> np.ndarray:
        import torch
        from . import risrt as R
        ctx, stream = self._context(slot)
        with torch.cuda.stream(stream):
            scene = self._scene_handle(slot, ctx, req.scene_id)
            ris = ctx.ris_upload(req.ris.elem_uv, req.ris.center, req.ris.t1, req.ris.t2, req.ris.dy, req.ris.dz,
                                 req.ris.elem_gain, req.ris.host_face)
            ctx.antenna_set(R.TX, req.tx.pos, req.tx.orient, req.tx.power_w, req.tx.gain_lin, req.tx.pattern)
            ctx.antenna_set(R.RX, None, req.rx.orient, req.rx.power_w, req.rx.gain_lin, req.rx.pattern)
            rx = ctx.rx_upload(req.rx_xyz)
            flags = R.FLAG_ENV_PATHS if req.env_paths else 0
            ps = ctx.trace_paths(scene, ris, rx, req.freq_hz, req.max_order_tx, req.max_order_rx, flags)
            n, C, M = len(req.rx_xyz), req.gammas.shape[0], req.gammas.shape[1]
            G = torch.from_numpy(np.ascontiguousarray(req.gammas, np.complex64)).to(f"cuda:{self.device}",
                                                                                      non_blocking=False)
            if req.kind == "coverage":
                E = torch.empty((C, n), dtype=torch.complex64, device=G.device)
                P = torch.empty((C, n), dtype=torch.float32, device=G.device)
                ctx.eval_field(ps, G, E, P)
                out = P.t().contiguous()
            else:
                A = torch.empty((n, M), dtype=torch.complex64, device=G.device)
                E0 = torch.empty(n, dtype=torch.complex64, device=G.device)
                ctx.build_A(ps, A, E0)
                out = torch.empty((n, C), dtype=torch.float32, device=G.device)
                ctx.sweep_configs(A, E0, G, out, req.precision, ctx.sweep_workspace(n, M, C, req.precision))
            host = out.cpu().numpy()
            stream.synchronize()
            for h in (ps, rx, ris):
                h.close()
            return host

    # -- lifecycle ----------------------------------------------------------------------------------
    def drain(self, futures, timeout: float = 600.0):
        return [f.result(timeout=timeout) for f in futures]

    def close(self):
        self._stop.set()
        self._dispatcher.join(timeout=5)
        for t in self._threads:
            t.join(timeout=60)
        with self._scene_lock:
            for _, handles in self._scenes.values():
                for h in handles.values():
                    h.close()
        for c in self._contexts:
            if c is not None:
                c[0].close()


def latency_stats(results) -> dict:
    lat = np.array([r.latency_s for r in results]) * 1e3
    q = np.array([r.queue_s for r in results]) * 1e3
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "queue_p50_ms": float(np.percentile(q, 50)),
            "queue_p99_ms": float(np.percentile(q, 99)), "n": int(len(lat))}


def poisson_requests(seed: int, n: int, rate_hz: float, scenes: dict, kinds=("coverage", "sweep")):
    """Seeded Poisson stream of uneven requests over the given scenes (name -> scenarios.Workload)."""
    from . import scenarios as S
    rng = S.SplitMix64(seed)
    names = sorted(scenes)
    t = 0.0
    out = []
    for i in range(n):
        t += -math.log(max(rng.uniform(), 1e-300)) / rate_hz
        w = scenes[names[int(rng.uniform() * len(names)) % len(names)]]
        grid = [16, 32, 64, 128][int(rng.uniform() * 4) % 4]
        C = [1, 4, 16, 64][int(rng.uniform() * 4) % 4]
        kind = kinds[int(rng.uniform() * len(kinds)) % len(kinds)]
        rx = S.linspace_grid(0.15, 5.85, grid, 0.15, 3.85, grid, 1.2, jitter=True)
        g = S.phase_configs(rng, C, w.n_elem)
        out.append((t, Request(kind, w.name, w.ris, w.tx, w.rx, rx, g, w.freq_hz, 1, 1, True)))
    return out
