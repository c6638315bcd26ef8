"""Continuous-batching request server for RIS field queries on one GPU.

Requests (coverage maps and configuration sweeps over scenes of uneven size) are admitted while a
stream slot is free and their estimated device-memory footprint fits the budget; every admitted
request runs on its own CUDA stream through its own library context, so the work of requests that
arrived at different times overlaps on the device. Scene BVHs stay resident in a cache shared by
all slots, and so do channel matrices: sweep requests that name the same channel (scene, RIS, Tx and
receiver grid) after the first one skip the trace and the matrix build, reuse the matrix packed for
the tensor cores, and replay a CUDA graph of the sweep captured for their configuration count. A
request's arithmetic does not depend on what else runs (per-request buffers, fixed reduction
orders, and a resident sweep computes exactly what the full one does), so its result is bitwise the
same alone or in a mix.

The admission policy (AdmissionController) is plain host logic and is tested without a GPU.
"""
from __future__ import annotations

import collections
import itertools
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
    channel_key: str | None = None   # same key: same scene, RIS, Tx and receivers (sweeps reuse the channel)
    arrival: float = 0.0
    rid: int = -1
    meta: dict = field(default_factory=dict)


class Overloaded(RuntimeError):
    """A request shed by the server's load limits (queue full, or not admitted in time)."""


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
    cap = 512
    n_ids = n_faces + (n_faces * n_faces if max(req.max_order_rx, req.max_order_tx) >= 2 else 0)
    # path records: valid paths per receiver are few (about 12 in the room at order 2, 5 in the
    # office at order 1); PATHS_PER_RX_EST per receiver is assumed, the 20% of memory left outside the
    # budget absorbs a request above it
    paths = n * min(PATHS_PER_RX_EST, 1 + n_ids)
    b = paths * 96 + n * ((M + 31) // 32) * 4 + n * 64
    b += 3 * n_ids * 160 + 8 * n * cap * 4 + (64 << 10)   # candidate slabs, work lists of the legs
    b += n * C * 4 * 2 + C * M * 8 + n * 12
    if uses_channel(req):
        Kp = (4 * M + 63) // 64 * 64
        Cw = max(C, CHANNEL_CFG_CAP)
        b += n * M * 8 + ((n + 255) // 256 * 256) * Kp * 2 + ((2 * Cw + 255) // 256 * 256) * Kp * 2 + n * C * 4
    return int(b)


PATHS_PER_RX_EST = 64
# Coverage requests whose direct evaluation would exceed this many (receiver, element,
# configuration) terms run through the channel matrix on the tensor cores instead (split BF16,
# about 1e-5 relative on the field), like sweeps.
DIRECT_EVAL_LIMIT = 2e9
# A channel's workspace is sized for this many configurations (or the request's, if more), so later
# sweeps on it with up to as many configurations reuse the packed matrix.
CHANNEL_CFG_CAP = 512
# Resident sweeps capture a CUDA graph per configuration count when their output is at most this big.
GRAPH_OUT_LIMIT = 512 << 20


def uses_channel(req: Request) -> bool:
    """Sweeps, and coverage requests too large to evaluate term by term, go through A."""
    n, M, C = len(req.rx_xyz), req.gammas.shape[1], req.gammas.shape[0]
    return req.kind == "sweep" or float(n) * M * C > DIRECT_EVAL_LIMIT


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
class _Channel:
    """A resident channel: A [n, M] and E0 on the device, the sweep workspace holding A packed for
    the tensor cores, and the captured sweep graphs per configuration count. One request uses it at
    a time (lock)."""

    def __init__(self, n, M, precision, A, E0, ws, cfg_cap, nbytes):
        self.n, self.M, self.precision = n, M, precision
        self.A, self.E0, self.ws = A, E0, ws
        self.cfg_cap = cfg_cap
        self.bytes = nbytes
        self.graphs = {}
        self.lock = threading.Lock()
        self.dead = False


class Server:
    def __init__(self, device: int = 0, slots: int = 4, budget_bytes: int | None = None, executor=None,
                 cache_fraction: float = 0.25, max_queue: int | None = None, max_wait_s: float | None = None):
        """executor(slot_index, request) -> np.ndarray replaces the GPU path (used by host tests).
        cache_fraction of the budget holds resident channels; the rest is for running requests.
        Load shedding (off by default): with max_queue, a request submitted while that many wait for
        admission fails at once with Overloaded; with max_wait_s, a request still waiting that long
        after its arrival fails with Overloaded instead of being admitted later."""
        self.device = device
        self.max_queue = max_queue
        self.max_wait_s = max_wait_s
        self.shed_full = 0           # rejected at submission, queue full
        self.shed_late = 0           # rejected while waiting, past max_wait_s
        self._n_waiting = 0
        self._wait_lock = threading.Lock()
        self._executor = executor
        if budget_bytes is None:
            import torch
            free, _ = torch.cuda.mem_get_info(device)
            # blocks torch's caching allocator holds but no tensor uses are available to requests too
            idle = torch.cuda.memory_reserved(device) - torch.cuda.memory_allocated(device)
            budget_bytes = int((free + idle) * 0.8)
        self.channel_budget = int(budget_bytes * cache_fraction)
        self.admission = AdmissionController(budget_bytes - self.channel_budget, slots)
        self._channels = {}          # channel_key -> _Channel (insertion order = least recently used first)
        self._chan_lock = threading.Lock()
        self.channel_bytes = 0
        self.channel_hits = 0
        self.graph_replays = 0
        # host wall time of the request phases summed over requests (slot threads overlap): inputs
        # uploaded, trace (synchronous), field or channel + sweep until the stream is idle, read-back
        self.phase_s = {"upload": 0.0, "trace": 0.0, "compute": 0.0, "readback": 0.0}
        self.oom_retries = 0
        self.idle_trims = 0
        self._device_lock = threading.Lock()     # graph captures; releases of cached device memory
        self._phase_lock = threading.Lock()
        self._pending: "queue.Queue[tuple]" = queue.Queue()
        self._next_id = 0
        self._id_lock = threading.Lock()
        self._scenes = {}            # scene_id -> (host Scene, {slot: risrt scene handle})
        self._scene_lock = threading.Lock()
        self._slot_free = queue.Queue()
        self._slot_work = [queue.Queue() for _ in range(slots)]
        self._stop = threading.Event()
        self._contexts = [None] * slots
        for s in range(slots):
            self._slot_free.put(s)
        self._threads = [threading.Thread(target=self._worker, args=(s,), daemon=True) for s in range(slots)]
        for t in self._threads:
            t.start()
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
        with self._wait_lock:
            full = self.max_queue is not None and self._n_waiting >= self.max_queue
            if full:
                self.shed_full += 1
            else:
                self._n_waiting += 1
        if full:
            fut.set_exception(Overloaded(f"{self.max_queue} requests already wait for admission"))
            return fut
        self._pending.put((req, fut, fp))
        return fut

    def _left_queue(self):
        with self._wait_lock:
            self._n_waiting -= 1

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
        waiting = collections.deque()                  # FIFO by arrival
        while not self._stop.is_set():
            try:
                while True:
                    waiting.append(self._pending.get(timeout=0.0005 if waiting else 0.05))
            except queue.Empty:
                pass
            if self.max_wait_s is not None:            # the oldest are at the front
                now = time.perf_counter()
                while waiting and now - waiting[0][0].arrival > self.max_wait_s:
                    req, fut, fp = waiting.popleft()
                    self._left_queue()
                    self.shed_late += 1
                    if not fut.done():                 # done only if cancelled
                        fut.set_exception(Overloaded(f"not admitted within {self.max_wait_s} s"))
            # FIFO: the oldest request that does not fit yet holds back the later ones (no starvation)
            while waiting:
                req, fut, fp = waiting[0]
                if fut.cancelled():
                    waiting.popleft()
                    self._left_queue()
                    continue
                if not self.admission.try_admit(fp):
                    break
                waiting.popleft()
                self._left_queue()
                self._slot_work[self._slot_free.get()].put((req, fut, fp))
        # closed: requests still waiting for admission fail instead of never completing
        while True:
            try:
                waiting.append(self._pending.get_nowait())
            except queue.Empty:
                break
        for req, fut, fp in waiting:
            self._left_queue()
            if not fut.done():
                fut.set_exception(RuntimeError("server closed before the request was admitted"))

    def _worker(self, slot: int):
        """The slot's thread: runs the requests the dispatcher hands to this slot, one at a time."""
        while True:
            item = self._slot_work[slot].get()
            if item is None:
                return
            self._run(slot, *item)

    def _run(self, slot: int, req: Request, fut: Future, fp: int):
        t_start = time.perf_counter()
        try:
            if not fut.set_running_or_notify_cancel():
                return
            run = self._executor if self._executor is not None else self._gpu_execute
            self._trim_idle_memory(fp)
            try:
                P = run(slot, req)
            except Exception as e:                # noqa: BLE001 - retried once, else reported
                if not _is_oom(e):
                    raise
                # device memory is shared by torch's caching allocator and the library's own
                # blocks; what one side caches the other cannot get, so release torch's idle blocks
                # and run the request once more
                self._release_idle_memory()
                self.oom_retries += 1
                P = run(slot, req)
            t_end = time.perf_counter()
            fut.set_result(Result(req.rid, P, t_end - req.arrival, t_start - req.arrival, fp))
        except BaseException as e:                    # noqa: BLE001 - reported through the future
            if not fut.done():
                fut.set_exception(e)
        finally:
            self.admission.release(fp)
            self._slot_free.put(slot)

    def _release_idle_memory(self):
        """Return torch's idle cached blocks to the driver. Held under the device lock, which graph
        captures also hold: freeing memory waits on the device, and a wait on a stream that is
        capturing would invalidate that capture."""
        if self._executor is not None:
            return
        import torch
        with self._device_lock:
            torch.cuda.empty_cache()

    def _trim_idle_memory(self, fp: int):
        """Before a request of at least a GiB: if torch's idle cached blocks exceed half of the
        running-request budget, release them (the library allocates outside torch's cache)."""
        if self._executor is not None or fp < (1 << 30):
            return
        import torch
        idle = torch.cuda.memory_reserved(self.device) - torch.cuda.memory_allocated(self.device)
        if idle > self.admission.budget // 2:
            self._release_idle_memory()
            self.idle_trims += 1

    def _context(self, slot: int):
        if self._contexts[slot] is None:
            import torch
            from . import risrt as R
            stream = torch.cuda.Stream(device=self.device)
            self._contexts[slot] = (R.Context(self.device, stream.cuda_stream), stream)
        return self._contexts[slot]

    def _phase_done(self, name: str, t0: float) -> float:
        t = time.perf_counter()
        with self._phase_lock:
            self.phase_s[name] += t - t0
        return t

    def _gpu_execute(self, slot: int, req: Request) -> np.ndarray:
        import torch
        ctx, stream = self._context(slot)
        with torch.cuda.stream(stream):
            t = time.perf_counter()
            n, C, M = len(req.rx_xyz), req.gammas.shape[0], req.gammas.shape[1]
            dev = f"cuda:{self.device}"
            G = torch.from_numpy(np.ascontiguousarray(req.gammas, np.complex64)).to(dev, non_blocking=False)
            if req.kind == "sweep" and req.channel_key is not None:
                ch = self._channel_acquire(req.channel_key, n, M, C, req.precision)
                if ch is not None:
                    try:
                        t = self._phase_done("upload", t)
                        return self._sweep_resident(ctx, stream, ch, G, t)
                    finally:
                        ch.lock.release()
            scene = self._scene_handle(slot, ctx, req.scene_id)
            handles = []
            try:
                return self._trace_and_evaluate(ctx, stream, scene, req, G, handles, t)
            finally:
                for h in reversed(handles):
                    h.close()

    def _trace_and_evaluate(self, ctx, stream, scene, req, G, handles, t):
        """Upload, trace and evaluate one request on its slot's stream; the handles it creates go to
        `handles` so the caller closes them whatever happens."""
        import torch
        from . import risrt as R
        n, C, M = len(req.rx_xyz), req.gammas.shape[0], req.gammas.shape[1]
        dev = G.device
        ris = ctx.ris_upload(req.ris.elem_uv, req.ris.center, req.ris.t1, req.ris.t2, req.ris.dy, req.ris.dz,
                             req.ris.elem_gain, req.ris.host_face)
        handles.append(ris)
        ctx.antenna_set(R.TX, req.tx.pos, req.tx.orient, req.tx.power_w, req.tx.gain_lin, req.tx.pattern)
        ctx.antenna_set(R.RX, None, req.rx.orient, req.rx.power_w, req.rx.gain_lin, req.rx.pattern)
        rx = ctx.rx_upload(req.rx_xyz)
        handles.append(rx)
        t = self._phase_done("upload", t)
        flags = R.FLAG_ENV_PATHS if req.env_paths else 0
        ps = ctx.trace_paths(scene, ris, rx, req.freq_hz, req.max_order_tx, req.max_order_rx, flags)
        handles.append(ps)
        t = self._phase_done("trace", t)
        keep = None
        if not uses_channel(req):
            E = torch.empty((C, n), dtype=torch.complex64, device=dev)
            P = torch.empty((C, n), dtype=torch.float32, device=dev)
            ctx.eval_field(ps, G, E, P)
            out = P.t().contiguous()
        else:
            A = torch.empty((n, M), dtype=torch.complex64, device=dev)
            E0 = torch.empty(n, dtype=torch.complex64, device=dev)
            ctx.build_A(ps, A, E0)
            out = torch.empty((n, C), dtype=torch.float32, device=dev)
            prec = req.precision if req.kind == "sweep" else R.PREC_BF16X2
            ws = ctx.sweep_workspace(n, M, max(C, CHANNEL_CFG_CAP), prec)
            ctx.sweep_configs(A, E0, G, out, prec, ws)
            if req.kind == "sweep" and req.channel_key is not None and prec in (R.PREC_BF16, R.PREC_BF16X2):
                keep = (A, E0, ws, prec, max(C, CHANNEL_CFG_CAP))
        stream.synchronize()
        t = self._phase_done("compute", t)
        host = _read_back(out, stream)
        if keep is not None:
            self._channel_store(req.channel_key, n, M, *keep)
        self._phase_done("readback", t)
        return host

    # -- resident channels --------------------------------------------------------------------------
    def _channel_acquire(self, key, n, M, C, precision):
        """The resident channel of this key, locked for this request, or None (not resident, or for
        other sizes / precision, or too many configurations for its workspace)."""
        with self._chan_lock:
            ch = self._channels.get(key)
            if ch is None or (ch.n, ch.M, ch.precision) != (n, M, precision) or C > ch.cfg_cap:
                return None
            self._channels[key] = self._channels.pop(key)        # most recently used last
        ch.lock.acquire()
        if ch.dead:                                              # evicted meanwhile
            ch.lock.release()
            return None
        self.channel_hits += 1
        return ch

    def _sweep_resident(self, ctx, stream, ch, G, t):
        """Sweep on a resident channel: A stays packed in its workspace; a CUDA graph of the sweep is
        captured once per configuration count and replayed with the new configurations."""
        import torch
        n, C = ch.n, G.shape[0]
        if n * C * 4 <= GRAPH_OUT_LIMIT:
            gr = ch.graphs.get(C)
            if gr is None:
                G_static = torch.empty_like(G)
                P_static = torch.empty((n, C), dtype=torch.float32, device=G.device)
                # capture on this slot's stream without torch.cuda.graph's device-wide synchronize and
                # allocator cache release, which would stall every other slot
                g = torch.cuda.CUDAGraph()
                with self._device_lock:
                    g.capture_begin(capture_error_mode="thread_local")
                    try:
                        ctx.sweep_configs(ch.A, ch.E0, G_static, P_static, ch.precision, ch.ws, keep_a=True,
                                          defer_check=True)
                    finally:
                        g.capture_end()
                gr = ch.graphs[C] = (g, G_static, P_static)
                with self._chan_lock:
                    extra = G_static.numel() * 8 + P_static.numel() * 4
                    ch.bytes += extra
                    self.channel_bytes += extra
            g, G_static, P_static = gr
            G_static.copy_(G)
            g.replay()
            ctx.sweep_check(ch.ws)
            self.graph_replays += 1
            t = self._phase_done("compute", t)
            host = _read_back(P_static, stream)
            self._phase_done("readback", t)
            return host
        out = torch.empty((n, C), dtype=torch.float32, device=G.device)
        ctx.sweep_configs(ch.A, ch.E0, G, out, ch.precision, ch.ws, keep_a=True)
        stream.synchronize()
        t = self._phase_done("compute", t)
        host = _read_back(out, stream)
        self._phase_done("readback", t)
        return host

    def _channel_store(self, key, n, M, A, E0, ws, precision, cfg_cap):
        """Keep a channel resident if it fits the channel budget after evicting least recently used
        channels that no request is using."""
        nbytes = A.numel() * 8 + E0.numel() * 8 + ws.numel()
        if nbytes > self.channel_budget:
            return
        with self._chan_lock:
            if key in self._channels:
                return
            for k in list(self._channels):
                if self.channel_bytes + nbytes <= self.channel_budget:
                    break
                old = self._channels[k]
                if old.lock.acquire(blocking=False):
                    old.dead = True
                    old.graphs.clear()
                    self.channel_bytes -= old.bytes
                    del self._channels[k]
                    old.lock.release()
            if self.channel_bytes + nbytes > self.channel_budget:
                return
            self._channels[key] = _Channel(n, M, precision, A, E0, ws, cfg_cap, nbytes)
            self.channel_bytes += nbytes

    # -- lifecycle ----------------------------------------------------------------------------------
    def drain(self, futures, timeout: float = 600.0):
        return [f.result(timeout=timeout) for f in futures]

    def close(self):
        self._stop.set()
        self._dispatcher.join(timeout=5)
        for q in self._slot_work:
            q.put(None)
        for t in self._threads:
            t.join(timeout=60)
        with self._scene_lock:
            for _, handles in self._scenes.values():
                for h in handles.values():
                    h.close()
        with self._chan_lock:
            for ch in self._channels.values():
                ch.dead = True
                ch.graphs.clear()
            self._channels.clear()
            self.channel_bytes = 0
        for c in self._contexts:
            if c is not None:
                c[0].close()


def _read_back(out, stream) -> np.ndarray:
    """The result copied into page-locked host memory from torch's caching host allocator: the copy
    runs at the link's rate instead of through a staging buffer, and the block goes back to the
    cache for a later result once the caller drops the array (the array keeps its tensor alive)."""
    import torch
    host = torch.empty(out.shape, dtype=out.dtype, pin_memory=True)
    host.copy_(out, non_blocking=True)
    stream.synchronize()
    return host.numpy()


def _is_oom(e: BaseException) -> bool:
    """A device allocation failure of the library (RISRT_ERR_OOM) or of torch."""
    if getattr(e, "code", None) == 2 and type(e).__name__ == "RisrtError":
        return True
    return type(e).__name__ == "OutOfMemoryError"


def latency_stats(results) -> dict:
    """Latency (arrival to result), queueing (arrival to start) and service (start to result), ms."""
    lat = np.array([r.latency_s for r in results]) * 1e3
    q = np.array([r.queue_s for r in results]) * 1e3
    sv = lat - q
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "queue_p50_ms": float(np.percentile(q, 50)),
            "queue_p99_ms": float(np.percentile(q, 99)), "service_p50_ms": float(np.percentile(sv, 50)),
            "service_p99_ms": float(np.percentile(sv, 99)), "n": int(len(lat))}


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


def _ris_of_size(w, n_elem: int):
    """A RIS of n_elem elements (37 / 127 hexagonal, 1,024 / 4,096 square, lambda/2 pitch) with the
    frame and host face of workload w's RIS."""
    from . import scenarios as S
    lam = S.C0 / w.freq_hz
    layouts = {37: lambda: S.hex_layout(3, lam / 2), 127: lambda: S.hex_layout(6, lam / 2),
               1024: lambda: S.square_layout(32, lam / 2), 4096: lambda: S.square_layout(64, lam / 2)}
    r = w.ris
    return S.RIS(layouts[n_elem](), r.center, r.t1, r.t2, lam / 2, lam / 2, 0.0, r.host_face)


POOL_CFGS = 1024


def mixed_requests(seed: int, n: int, rate_hz: float, scenes: dict, **kw):
    """The first n requests of iter_mixed_requests (a list of (arrival time, Request))."""
    return list(itertools.islice(iter_mixed_requests(seed, rate_hz, scenes, **kw), n))


def iter_mixed_requests(seed: int, rate_hz: float, scenes: dict, rx_range=(1e3, 1e6), cfg_range=(1, 512),
                        ris_sizes=(37, 127, 1024, 4096), n_channels: int = 4, reuse: float = 0.5,
                        shared_inputs: bool = False):
    """Seeded Poisson stream of the serving mix, generated as it is consumed: per request a scene
    (name -> scenarios.Workload), a RIS of one of ris_sizes elements on that scene's RIS wall, a
    receiver grid of log-uniform size in rx_range over the scene's floor (margin 0.15 m) at 1.2 m, a
    log-uniform configuration count in cfg_range, and coverage or sweep with equal odds; a fraction
    `reuse` of the sweeps query one of n_channels fixed channels (same scene, RIS, Tx and receivers,
    new configurations).

    shared_inputs: generate at thousands of requests per second. Receiver counts are rounded to
    1/16 of a decade and each (scene, count) grid is built once; each request's configurations are
    C consecutive rows, from a random row, of one seeded pool of POOL_CFGS configurations per RIS
    size (arrays shared between requests, never written). The sizes and the work per request keep
    the mix's distributions."""
    from . import scenarios as S
    rng = S.SplitMix64(seed)
    names = sorted(scenes)
    grids, rises, pools = {}, {}, {}

    def log_uniform(lo, hi):
        return math.exp(math.log(lo) + rng.uniform() * (math.log(hi) - math.log(lo)))

    def grid(w, n):
        if shared_inputs:
            n = 10.0 ** (round(16 * math.log10(n)) / 16)
        side = max(1, int(round(math.sqrt(n))))
        key = (w.name, side)
        if key in grids:
            return grids[key]
        v = w.scene.verts
        x0, y0 = float(v[:, 0].min()) + 0.15, float(v[:, 1].min()) + 0.15
        x1, y1 = float(v[:, 0].max()) - 0.15, float(v[:, 1].max()) - 0.15
        g = S.linspace_grid(x0, x1, side, y0, y1, side, 1.2, jitter=True)
        if shared_inputs:
            grids[key] = g
        return g

    def ris_of(w, size):
        key = (w.name, size)
        if key not in rises:
            rises[key] = _ris_of_size(w, size)
        return rises[key]

    def setup():
        w = scenes[names[int(rng.uniform() * len(names)) % len(names)]]
        ris = ris_of(w, ris_sizes[int(rng.uniform() * len(ris_sizes)) % len(ris_sizes)])
        return w, ris, grid(w, log_uniform(*rx_range))

    def configs(C, M):
        if not shared_inputs:
            return S.phase_configs(rng, C, M)
        if M not in pools:
            pools[M] = S.phase_configs(S.SplitMix64(seed * 1000003 + M), max(POOL_CFGS, int(cfg_range[1])), M)
        p = pools[M]
        r0 = int(rng.uniform() * (p.shape[0] - C + 1)) % (p.shape[0] - C + 1)
        return p[r0:r0 + C]

    channels = [setup() for _ in range(n_channels)]
    t = 0.0
    while True:
        t += -math.log(max(rng.uniform(), 1e-300)) / rate_hz
        kind = "sweep" if rng.uniform() < 0.5 else "coverage"
        key = None
        if kind == "sweep" and channels and rng.uniform() < reuse:
            k = int(rng.uniform() * len(channels)) % len(channels)
            w, ris, rx = channels[k]
            key = f"channel{k}"
        else:
            w, ris, rx = setup()
        C = max(1, min(int(cfg_range[1]), int(log_uniform(cfg_range[0], cfg_range[1] + 1))))
        g = configs(C, ris.elem_uv.shape[0])
        yield t, Request(kind, w.name, ris, w.tx, w.rx, rx, g, w.freq_hz, 1, 1, True, channel_key=key)

