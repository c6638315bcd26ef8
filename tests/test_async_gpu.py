"""The path search without host synchronisation or device allocation (risrt_trace_paths_async): its
path sets and fields equal the regular trace's bit for bit, a limit that is too small is reported by
risrt_trace_check, and the trace and the field evaluation can be captured into one CUDA graph and
replayed with new configurations and receiver positions."""
import numpy as np
import pytest

from paper_2402_13034_gb300 import scenarios as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2402_13034_gb300 import build as B
    B.build()


def _ctx():
    import torch
    from paper_2402_13034_gb300 import risrt as R
    return R.Context(0, torch.cuda.current_stream().cuda_stream)


def _same_paths(a, b):
    for key in ("seqs", "env"):
        assert all(np.array_equal(x, y) for x, y in zip(a[key], b[key])), key
    assert np.array_equal(np.asarray(a["los"]), np.asarray(b["los"]))
    assert np.array_equal(a["vis"], b["vis"])
    assert np.array_equal(a["tx_seqs"], b["tx_seqs"]) and np.array_equal(a["tx_vis"], b["tx_vis"])


@pytest.mark.parametrize("case", ["room", "office_order1", "free_space"])
def test_async_trace_equals_regular(case):
    import torch
    from paper_2402_13034_gb300 import risrt as R
    if case == "room":
        w = S.room(grid=24)
    elif case == "office_order1":
        w = S.office()
        w.rx_xyz = w.rx_xyz[::16]
    else:
        w = S.free_space()
    ctx = _ctx()
    scene, ris, rx = R.upload_workload(ctx, w)
    flags = R.flags_of(w)
    ps_ref = ctx.trace_paths(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, flags)
    ws, lim = ctx.trace_workspace(scene, ris, rx, w.max_order_tx, w.max_order_rx, flags, cand_cap=1024)
    ps = ctx.trace_paths_async(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, flags, ws, lim)
    G = torch.from_numpy(np.ascontiguousarray(w.gammas, np.complex64)).cuda()
    E1 = torch.empty((G.shape[0], w.n_rx), dtype=torch.complex64, device="cuda")
    E2 = torch.empty_like(E1)
    ctx.eval_field(ps, G, E2)                 # enqueued behind the asynchronous trace, before the check
    ctx.trace_check(ps)
    ctx.eval_field(ps_ref, G, E1)
    torch.cuda.synchronize()
    _same_paths(ps.export(), ps_ref.export())
    assert torch.equal(E1, E2)
    a, b = ps.stats(), ps_ref.stats()
    assert (a.n_rx_paths, a.n_env_paths, a.n_tx_paths, a.units) == (b.n_rx_paths, b.n_env_paths, b.n_tx_paths, b.units)


def test_async_trace_limits_reported():
    import torch
    from paper_2402_13034_gb300 import risrt as R
    w = S.room(grid=12)
    ctx = _ctx()
    scene, ris, rx = R.upload_workload(ctx, w)
    flags = R.flags_of(w)
    for kw in (dict(cand_cap=8), dict(max_paths=2), dict(max_env=1)):
        ws, lim = ctx.trace_workspace(scene, ris, rx, w.max_order_tx, w.max_order_rx, flags, **kw)
        ps = ctx.trace_paths_async(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, flags, ws, lim)
        with pytest.raises(R.RisrtError) as e:
            ctx.trace_check(ps)
        assert e.value.code == 6, kw
    with pytest.raises(R.RisrtError):             # a workspace that is too small is refused
        ws, lim = ctx.trace_workspace(scene, ris, rx, w.max_order_tx, w.max_order_rx, flags)
        ctx.trace_paths_async(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, flags, ws[: ws.numel() // 2], lim)


def test_trace_and_eval_captured_in_a_graph():
    """One CUDA graph holds the whole request (trace + field evaluation). Replays with new
    configurations and new receiver positions (a shifted grid within the measured extent) give what a
    regular trace and evaluation of the same inputs give, bit for bit."""
    import torch
    from paper_2402_13034_gb300 import risrt as R
    w = S.room(grid=16, n_boxes=20)
    stream = torch.cuda.Stream()                 # graphs are captured on a stream of their own
    ctx = R.Context(0, stream.cuda_stream)
    with torch.cuda.stream(stream):
        _capture_and_replay(ctx, stream, w)


def _capture_and_replay(ctx, stream, w):
    import torch
    from paper_2402_13034_gb300 import risrt as R
    sc = w.scene
    scene = ctx.scene_upload(sc.verts, sc.tris, sc.face_id, sc.mat_id, sc.mats)
    ris = ctx.ris_upload(w.ris.elem_uv, w.ris.center, w.ris.t1, w.ris.t2, w.ris.dy, w.ris.dz, w.ris.elem_gain,
                         w.ris.host_face)
    ctx.antenna_set(R.TX, w.tx.pos, w.tx.orient, w.tx.power_w, w.tx.gain_lin, w.tx.pattern)
    ctx.antenna_set(R.RX, None, w.rx.orient, w.rx.power_w, w.rx.gain_lin, w.rx.pattern)
    rx_dev = torch.from_numpy(w.rx_xyz).cuda()
    rx = ctx.rx_bind(rx_dev)
    flags = R.flags_of(w)
    ws, lim = ctx.trace_workspace(scene, ris, rx, w.max_order_tx, w.max_order_rx, flags, cand_cap=1024)
    G = torch.from_numpy(np.ascontiguousarray(w.gammas, np.complex64)).cuda()
    E = torch.empty((G.shape[0], w.n_rx), dtype=torch.complex64, device="cuda")
    P = torch.empty((G.shape[0], w.n_rx), dtype=torch.float32, device="cuda")
    # a first trace of this context creates its side streams and kernel attributes (not capturable)
    ps = ctx.trace_paths_async(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, flags, ws, lim)
    ctx.trace_check(ps)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    g.capture_begin(capture_error_mode="thread_local")
    try:
        ctx.trace_paths_async(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, flags, ws, lim, reuse=ps)
        ctx.eval_field(ps, G, E, P)
    finally:
        g.capture_end()
    for k in range(3):
        G.copy_(torch.from_numpy(S.phase_configs(S.SplitMix64(50 + k), G.shape[0], w.n_elem)).cuda())
        shift = np.array([0.013 * k, -0.007 * k, 0.0], np.float32)
        rx_dev.copy_(torch.from_numpy(w.rx_xyz + shift).cuda())
        g.replay()
        with pytest.raises(R.RisrtError) as e:   # host copies of the replayed trace not read yet
            ps.stats()
        assert e.value.code == 5
        ctx.trace_check(ps)
        torch.cuda.synchronize()
        rx_ref = ctx.rx_upload(rx_dev.cpu().numpy())
        ps_ref = ctx.trace_paths(scene, ris, rx_ref, w.freq_hz, w.max_order_tx, w.max_order_rx, flags)
        E_ref = torch.empty_like(E)
        P_ref = torch.empty_like(P)
        ctx.eval_field(ps_ref, G, E_ref, P_ref)
        torch.cuda.synchronize()
        _same_paths(ps.export(), ps_ref.export())
        assert torch.equal(E, E_ref) and torch.equal(P, P_ref), k
