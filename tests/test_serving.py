"""Continuous-batching server: admission by stream slots and device-memory budget (host logic with a
fake executor, no GPU), and on the GPU that every result is bitwise the same alone and in a mix of
concurrent requests of uneven size."""
import threading
import time

import numpy as np
import pytest

from paper_2402_13034_gb300 import scenarios as S
from paper_2402_13034_gb300 import serve


def _room_workloads():
    a = S.room(grid=8, n_boxes=10)
    a.name = "room_a"
    b = S.room(grid=8, n_boxes=25, seed_index=5)
    b.name = "room_b"
    b.ris.elem_uv = S.hex_layout(3, S.C0 / b.freq_hz / 2)
    b.gammas = b.gammas[:, :37]
    return {"room_a": a, "room_b": b}


def _requests(ws, n=10, seed=11):
    reqs = serve.poisson_requests(seed, n, 2000.0, ws)
    return [r for _, r in reqs]


class _Fake:
    """Executor that sleeps and records concurrency; returns a deterministic array."""

    def __init__(self):
        self.lock = threading.Lock()
        self.active = 0
        self.max_active = 0

    def __call__(self, slot, req):
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)
        time.sleep(0.01)
        with self.lock:
            self.active -= 1
        return np.full((len(req.rx_xyz), req.gammas.shape[0]), float(req.rid), np.float32)


def test_admission_respects_budget_and_slots():
    ws = _room_workloads()
    reqs = _requests(ws, 24)
    fps = [serve.estimate_footprint(r, ws[r.scene_id].scene.n_faces) for r in reqs]
    budget = int(max(fps) * 1.5)          # at most one large request at a time
    fake = _Fake()
    srv = serve.Server(slots=3, budget_bytes=budget, executor=fake)
    for name, w in ws.items():
        srv.add_scene(name, w.scene)
    futs = [srv.submit(r) for r in reqs]
    res = srv.drain(futs)
    srv.close()
    assert [r.rid for r in res] == [r.rid for r in reqs]
    assert srv.admission.peak <= budget
    assert 1 <= fake.max_active <= 3
    assert srv.admission.in_use == 0 and srv.admission.running == 0
    for r, q in zip(res, reqs):
        assert r.P.shape == (len(q.rx_xyz), q.gammas.shape[0]) and np.all(r.P == q.rid)


def test_admission_rejects_oversize_and_malformed():
    ws = _room_workloads()
    reqs = _requests(ws, 4)
    srv = serve.Server(slots=2, budget_bytes=1000, executor=_Fake())
    for name, w in ws.items():
        srv.add_scene(name, w.scene)
    f = srv.submit(reqs[0])
    with pytest.raises(MemoryError):
        f.result(timeout=5)
    bad = reqs[1]
    bad.kind = "hologram"
    with pytest.raises(ValueError):
        srv.submit(bad).result(timeout=5)
    r2 = reqs[2]
    r2.scene_id = "nope"
    with pytest.raises(ValueError):
        srv.submit(r2).result(timeout=5)
    srv.close()


def test_executor_failure_is_isolated():
    ws = _room_workloads()
    reqs = _requests(ws, 6)

    def flaky(slot, req):
        if req.rid == 2:
            raise RuntimeError("injected failure")
        return np.zeros((len(req.rx_xyz), req.gammas.shape[0]), np.float32)

    srv = serve.Server(slots=2, budget_bytes=1 << 40, executor=flaky)
    for name, w in ws.items():
        srv.add_scene(name, w.scene)
    futs = [srv.submit(r) for r in reqs]
    for i, f in enumerate(futs):
        if i == 2:
            with pytest.raises(RuntimeError):
                f.result(timeout=10)
        else:
            assert f.result(timeout=10).P.shape[0] == len(reqs[i].rx_xyz)
    assert srv.admission.running == 0
    srv.close()


class RisrtError(RuntimeError):
    """Stands in for the binding's error class (same name and code attribute)."""
    def __init__(self, code):
        super().__init__(f"risrt error {code}")
        self.code = code


def test_allocation_failure_retried_once():
    """A request whose first run fails to allocate (library code 2) runs once more; a second
    allocation failure, or any other error, reaches the caller; nothing else is retried."""
    ws = _room_workloads()
    reqs = _requests(ws, 4)
    calls = {}

    def executor(slot, req):
        calls[req.rid] = calls.get(req.rid, 0) + 1
        if req.rid == 0 and calls[0] == 1:
            raise RisrtError(2)
        if req.rid == 1:
            raise RisrtError(2)
        if req.rid == 2:
            raise RisrtError(3)
        return np.zeros((len(req.rx_xyz), req.gammas.shape[0]), np.float32)

    srv = serve.Server(slots=1, budget_bytes=1 << 40, executor=executor)
    for name, w in ws.items():
        srv.add_scene(name, w.scene)
    futs = [srv.submit(r) for r in reqs]
    assert futs[0].result(timeout=10).P.shape[0] == len(reqs[0].rx_xyz)
    for i in (1, 2):
        with pytest.raises(RisrtError):
            futs[i].result(timeout=10)
    assert futs[3].result(timeout=10) is not None
    srv.close()
    assert calls == {0: 2, 1: 2, 2: 1, 3: 1}
    assert srv.oom_retries == 2
    assert srv.admission.running == 0


@pytest.mark.gpu
def test_results_identical_alone_and_in_mix():
    from paper_2402_13034_gb300 import build as B
    B.build()
    ws = _room_workloads()
    reqs = _requests(ws, 10, seed=3)
    alone = []
    srv = serve.Server(slots=1)
    for name, w in ws.items():
        srv.add_scene(name, w.scene)
    for r in reqs:
        alone.append(srv.submit(r).result(timeout=300).P)
    srv.close()
    srv = serve.Server(slots=4)
    for name, w in ws.items():
        srv.add_scene(name, w.scene)
    futs = [srv.submit(r) for r in reqs]
    mixed = [f.result(timeout=300).P for f in futs]
    srv.close()
    for a, m in zip(alone, mixed):
        assert np.array_equal(a, m)


def test_mixed_requests_span_the_serving_mix():
    """The serving mix: receiver grids of 1k-1M points, 1-512 configurations, RIS of 37 to 4,096
    elements, coverage and sweep, some sweeps on fixed channels (same scene, RIS and receivers)."""
    w = S.room(grid=4)
    w.name = "room"
    reqs = [r for _, r in serve.mixed_requests(5, 200, 2000.0, {"room": w})]
    n = np.array([len(r.rx_xyz) for r in reqs])
    C = np.array([r.gammas.shape[0] for r in reqs])
    M = {r.gammas.shape[1] for r in reqs}
    assert n.min() >= 31 ** 2 and n.max() <= 1000 ** 2 and n.max() > 100_000 and n.min() < 5_000
    assert C.min() >= 1 and C.max() <= 512 and C.max() > 100
    assert M == {37, 127, 1024, 4096}
    keyed = [r for r in reqs if r.channel_key is not None]
    assert keyed and all(r.kind == "sweep" for r in keyed)
    for r in keyed:                       # a channel is one scene, RIS and receiver grid
        first = next(q for q in keyed if q.channel_key == r.channel_key)
        assert r.rx_xyz is first.rx_xyz and r.ris is first.ris
    assert any(serve.uses_channel(r) for r in reqs if r.kind == "coverage")
    assert any(not serve.uses_channel(r) for r in reqs if r.kind == "coverage")


@pytest.mark.gpu
def test_resident_channel_and_graph_replay():
    """Sweeps naming the same channel: the first traces, builds A and packs it for the tensor cores;
    the later ones reuse it and replay a captured graph of the sweep per configuration count. Every
    result is bitwise what the full computation (no channel key) gives for its configurations."""
    from paper_2402_13034_gb300 import build as B
    B.build()
    w = S.room(grid=24, n_boxes=10)
    w.name = "room_c"
    reqs = []
    for i, C in enumerate((8, 8, 3, 8, 3, 20)):
        g = S.phase_configs(S.SplitMix64(100 + i), C, w.n_elem)
        reqs.append(serve.Request("sweep", "room_c", w.ris, w.tx, w.rx, w.rx_xyz, g, w.freq_hz, 1, 1, True,
                                  channel_key="c0"))
    srv = serve.Server(slots=2)
    srv.add_scene("room_c", w.scene)
    got = [srv.submit(r).result(timeout=300).P for r in reqs]
    hits, replays = srv.channel_hits, srv.graph_replays
    srv.close()
    assert hits == 5 and replays == 5
    for r in reqs:
        r.channel_key = None
    srv = serve.Server(slots=2)
    srv.add_scene("room_c", w.scene)
    ref = [srv.submit(r).result(timeout=300).P for r in reqs]
    srv.close()
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_channel_cache_lru_and_locks():
    """Resident channels (host bookkeeping on CPU tensors): a channel is kept while it fits the channel
    budget, least recently used ones that no request holds are evicted first, a held one is never
    evicted, and a lookup with other sizes, precision or more configurations than the workspace was
    sized for misses."""
    import torch
    srv = serve.Server(slots=1, budget_bytes=4 << 20, executor=_Fake(), cache_fraction=0.25)   # 1 MiB of channels

    def chan(key, n=64, M=128, ws_bytes=200_000, cfg_cap=512):
        A = torch.zeros((n, M), dtype=torch.complex64)              # 64 KiB
        E0 = torch.zeros(n, dtype=torch.complex64)
        ws = torch.zeros(ws_bytes, dtype=torch.uint8)
        srv._channel_store(key, n, M, A, E0, ws, 2, cfg_cap)

    for k in ("a", "b", "c", "d"):
        chan(k)                                                      # ~266 KB each: 3 fit in 1 MiB
    assert list(srv._channels) == ["b", "c", "d"] and srv.channel_bytes <= srv.channel_budget
    ch = srv._channel_acquire("b", 64, 128, 8, 2)                   # held by a request (most recent now)
    assert ch is not None and srv.channel_hits == 1
    chan("e")                                                        # evicts c, the least recent unheld
    assert list(srv._channels) == ["d", "b", "e"]
    chan("f")                                                        # evicts d; b stays while held
    assert "b" in srv._channels and "d" not in srv._channels
    ch.lock.release()
    assert srv._channel_acquire("e", 64, 127, 8, 2) is None         # other element count
    assert srv._channel_acquire("e", 64, 128, 8, 1) is None         # other precision
    assert srv._channel_acquire("e", 64, 128, 513, 2) is None       # more configurations than its workspace
    chan("big", ws_bytes=2 << 20)                                    # larger than the channel budget: not kept
    assert "big" not in srv._channels
    srv.close()
    assert srv.channel_bytes == 0 and not srv._channels


@pytest.mark.gpu
def test_served_results_match_oracle():
    """A sample of served requests against the FP64 oracle: coverage (direct field evaluation) and
    sweep (channel matrix on the tensor cores, split BF16, with 2-bit configurations, which BF16
    carries exactly) on two scenes, the room (492 triangles, order 2) and the office (19,932
    triangles, order 1), with a resident-channel repeat. The served power gives |E|; it must be within
    5e-5 of the incoherent magnitude S(r) of the oracle's field on every receiver without an ambiguous
    decision (Eqs. 9, 10)."""
    from oracle import oracle as O
    from paper_2402_13034_gb300 import build as B
    B.build()
    room = S.room(grid=6, n_boxes=12)
    room.name = "room_o"
    office = S.office()
    office.name = "office_o"
    office.rx_xyz = office.rx_xyz[::1024]                     # 16 receivers spread over the target area
    reqs = []
    for w, orders in ((room, (2, 2)), (office, (1, 1))):
        codes, g2 = S.two_bit_configs(S.SplitMix64(7), 5, w.n_elem)
        gph = S.phase_configs(S.SplitMix64(8), 3, w.n_elem)
        for kind, g, key in (("coverage", gph, None), ("sweep", g2, "c_" + w.name), ("sweep", g2[:2], "c_" + w.name)):
            reqs.append((w, serve.Request(kind, w.name, w.ris, w.tx, w.rx, w.rx_xyz, g, w.freq_hz, orders[0],
                                          orders[1], True, channel_key=key)))
    srv = serve.Server(slots=3)
    for w in (room, office):
        srv.add_scene(w.name, w.scene)
    # the repeat sweeps go in after the first ones have stored their channels
    first = [i for i in range(len(reqs)) if i % 3 != 2]
    got = [None] * len(reqs)
    for batch in (first, [i for i in range(len(reqs)) if i % 3 == 2]):
        futs = {i: srv.submit(reqs[i][1]) for i in batch}
        for i, f in futs.items():
            got[i] = f.result(timeout=600).P
    hits = srv.channel_hits
    srv.close()
    assert hits >= 2
    checked = 0
    for (w, r), P in zip(reqs, got):
        wo = S.Workload(w.name, w.freq_hz, w.scene, w.ris, w.tx, w.rx, w.rx_xyz, r.gammas, r.max_order_tx,
                        r.max_order_rx, True)
        fld = O.Oracle(wo).field(wo.rx_xyz)
        E_ref, P_ref, S_ref = O.Oracle.evaluate(fld, r.gammas)
        ok = ~fld["amb"][:, None] & (S_ref > 0)
        dE = np.abs(np.sqrt(P.astype(np.float64) * 2 * 120 * np.pi) - np.abs(E_ref)) / np.where(S_ref > 0, S_ref, 1.0)
        assert dE[ok].max() <= 5e-5, (r.kind, w.name, dE[ok].max())
        checked += int(ok.sum())
    assert checked > 100


def _blocking_executor():
    """An executor whose requests run until `release` is set; `started` is set when one starts."""
    started, release = threading.Event(), threading.Event()

    def run(slot, req):
        started.set()
        assert release.wait(timeout=10)
        return np.zeros((len(req.rx_xyz), req.gammas.shape[0]), np.float32)
    return run, started, release


def test_load_shedding_queue_bound():
    """With max_queue = 2 and the only slot busy, two requests wait and later ones fail at once with
    Overloaded; the waiting ones are served once the slot frees."""
    ws = _room_workloads()
    reqs = _requests(ws, 6)
    run, started, release = _blocking_executor()
    srv = serve.Server(slots=1, budget_bytes=1 << 40, executor=run, max_queue=2)
    for name, w in ws.items():
        srv.add_scene(name, w.scene)
    first = srv.submit(reqs[0])
    assert started.wait(timeout=10)
    futs = [srv.submit(r) for r in reqs[1:]]
    for f in futs[2:]:
        with pytest.raises(serve.Overloaded):
            f.result(timeout=1)
    release.set()
    for f in [first] + futs[:2]:
        assert f.result(timeout=10) is not None
    assert srv.shed_full == 3 and srv.shed_late == 0
    srv.close()
    assert srv.admission.running == 0


def test_load_shedding_wait_limit():
    """With max_wait_s, a request that cannot be admitted within the limit fails with Overloaded
    and never runs; the running one completes."""
    ws = _room_workloads()
    reqs = _requests(ws, 3)
    run, started, release = _blocking_executor()
    ran = []

    def executor(slot, req):
        ran.append(req.rid)
        return run(slot, req)

    srv = serve.Server(slots=1, budget_bytes=1 << 40, executor=executor, max_wait_s=0.1)
    for name, w in ws.items():
        srv.add_scene(name, w.scene)
    first = srv.submit(reqs[0])
    assert started.wait(timeout=10)
    late = [srv.submit(r) for r in reqs[1:]]
    for f in late:
        with pytest.raises(serve.Overloaded):
            f.result(timeout=5)
    release.set()
    assert first.result(timeout=10) is not None
    srv.close()
    assert ran == [0] and srv.shed_late == 2 and srv.shed_full == 0


def test_close_fails_waiting_requests():
    """No request is left pending by close: requests still waiting for admission when the server
    closes fail with an error (those admitted meanwhile complete), and the running one completes."""
    ws = _room_workloads()
    reqs = _requests(ws, 4)
    run, started, release = _blocking_executor()
    srv = serve.Server(slots=1, budget_bytes=1 << 40, executor=run)
    for name, w in ws.items():
        srv.add_scene(name, w.scene)
    first = srv.submit(reqs[0])
    assert started.wait(timeout=10)
    waiting = [srv.submit(r) for r in reqs[1:]]
    time.sleep(0.1)
    release.set()
    srv.close()
    assert first.result(timeout=10) is not None
    for f in waiting:
        assert f.done()
        if f.exception() is not None:               # else admitted before the close took effect
            assert "closed" in str(f.exception())


def test_shared_input_mix_keeps_distributions():
    """The shared-input mix draws sizes from the same distributions (receiver counts within 1/32 of
    a decade of a log-uniform draw, C in range, configurations rows of one pool per RIS size) and
    reuses grid arrays."""
    ws = _room_workloads()
    scenes = {}
    for name, w in ws.items():
        w.name = name
        scenes[name] = w
    reqs = serve.mixed_requests(5, 300, 2000.0, scenes, rx_range=(100, 4000), shared_inputs=True)
    n = np.array([len(r.rx_xyz) for _, r in reqs])
    assert n.min() >= 0.8 * 100 and n.max() <= 1.2 * 4000
    logs = np.log10(n)
    assert abs(np.median(logs) - 0.5 * (2 + np.log10(4000))) < 0.2
    ids = {id(r.rx_xyz) for _, r in reqs}
    assert len(ids) < len(reqs) // 2
    for _, r in reqs:
        assert 1 <= r.gammas.shape[0] <= 512 and r.gammas.flags.c_contiguous
        assert np.allclose(np.abs(r.gammas), 1.0, atol=1e-6)
    t = np.array([a for a, _ in reqs])
    assert np.all(np.diff(t) > 0) and abs(len(t) / t[-1] - 2000.0) < 400
