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
