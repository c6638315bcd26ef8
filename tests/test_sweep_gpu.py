"""Configuration sweep E = E0 + A . Gamma, P = |E|^2 / (2 eta0) (Eq. 9 linear in Gamma, Eq. 10):
the FP32 CUDA-core path and the tcgen05 tensor-core paths (BF16, split BF16, scaled FP16) against FP64
on random inputs, and end to end (trace -> build_A -> sweep) against the FP64 oracle's channel rows."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2402_13034_gb300 import scenarios as S

pytestmark = pytest.mark.gpu

ETA0 = 120 * math.pi
# field error bound relative to S = |E0| + sum |A||Gamma| per precision: FP32 accumulation order,
# split-BF16 (2^-17 on A, Gamma exact), FP16 (2^-11 on A after power-of-two scaling), BF16 (2^-8)
TOL = {0: 5e-5, 2: 5e-5, 3: 1e-3, 1: 4e-3}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2402_13034_gb300 import build as B
    B.build()


def _ctx():
    import torch
    from paper_2402_13034_gb300 import risrt as R
    return R.Context(0, torch.cuda.current_stream().cuda_stream)


def _run(ctx, A, E0, G, prec):
    import torch
    n, C = A.shape[0], G.shape[0]
    P = torch.full((n, C), -1.0, dtype=torch.float32, device="cuda")
    ws = ctx.sweep_workspace(n, A.shape[1], C, prec)
    ctx.sweep_configs(torch.from_numpy(A).cuda(), None if E0 is None else torch.from_numpy(E0).cuda(),
                      torch.from_numpy(G).cuda(), P, prec, ws)
    torch.cuda.synchronize()
    return P.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n,M,C", [(1, 1, 1), (129, 37, 5), (1000, 300, 300), (4097, 1024, 129)])
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_sweep_vs_fp64(n, M, C, prec):
    rng = np.random.default_rng(n + M + C)
    A = ((rng.standard_normal((n, M)) + 1j * rng.standard_normal((n, M))) * 1e-3).astype(np.complex64)
    E0 = ((rng.standard_normal(n) + 1j * rng.standard_normal(n)) * 1e-3).astype(np.complex64)
    G = np.array([1, 1j, -1, -1j], np.complex64)[rng.integers(0, 4, (C, M))]
    E = E0[:, None].astype(np.complex128) + A.astype(np.complex128) @ G.T.astype(np.complex128)
    Sx = np.abs(E0)[:, None] + np.abs(A).astype(np.float64) @ np.abs(G).T.astype(np.float64)
    P = _run(_ctx(), A, E0, G, prec)
    dE = np.abs(np.sqrt(np.maximum(P, 0) * 2 * ETA0) - np.abs(E)) / Sx
    assert P.min() >= 0 and np.isfinite(P).all()
    assert dE.max() <= TOL[prec], dE.max()


def test_sweep_general_gamma_and_no_e0():
    """Uniform phases and amplitudes (not exact in 16 bits) and no E0."""
    rng = np.random.default_rng(9)
    n, M, C = 300, 100, 70
    A = ((rng.standard_normal((n, M)) + 1j * rng.standard_normal((n, M))) * 1e-3).astype(np.complex64)
    G = (1.25 * np.exp(2j * np.pi * rng.random((C, M)))).astype(np.complex64)
    E = A.astype(np.complex128) @ G.T.astype(np.complex128)
    Sx = np.abs(A).astype(np.float64) @ np.abs(G).T.astype(np.float64)
    for prec in (0, 1, 2, 3):
        P = _run(_ctx(), A, None, G, prec)
        dE = np.abs(np.sqrt(P * 2 * ETA0) - np.abs(E)) / Sx
        assert dE.max() <= max(TOL[prec], 4e-3 if prec == 2 else 0), (prec, dE.max())


def test_sweep_room_against_oracle():
    """trace -> build_A -> sweep on the sweep room (32x32 RIS); the oracle's FP64 channel rows
    give the reference for every configuration; power error statistics per precision."""
    import torch
    from paper_2402_13034_gb300 import risrt as R
    w = S.sweep(n_cfg=96, grid=12)
    ctx = _ctx()
    scene, ris, rx = R.upload_workload(ctx, w)
    ps = ctx.trace_paths(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, R.flags_of(w))
    A = torch.empty((w.n_rx, w.n_elem), dtype=torch.complex64, device="cuda")
    E0 = torch.empty(w.n_rx, dtype=torch.complex64, device="cuda")
    ctx.build_A(ps, A, E0)
    torch.cuda.synchronize()
    fld = O.Oracle(w).field(w.rx_xyz)
    E_ref, P_ref, S_ref = O.Oracle.evaluate(fld, w.gammas)
    ok = ~fld["amb"]
    G = torch.from_numpy(w.gammas).cuda()
    for prec in (0, 1, 2, 3):
        P = torch.empty((w.n_rx, G.shape[0]), dtype=torch.float32, device="cuda")
        ctx.sweep_configs(A, E0, G, P, prec, ctx.sweep_workspace(w.n_rx, w.n_elem, G.shape[0], prec))
        torch.cuda.synchronize()
        Pg = P.cpu().numpy().astype(np.float64)
        dE = np.abs(np.sqrt(Pg * 2 * ETA0) - np.abs(E_ref)) / np.where(S_ref > 0, S_ref, 1)
        assert dE[ok].max() <= TOL[prec] + 5e-5, (prec, dE[ok].max())
        # dB error where the power is within 30 dB of the configuration's peak
        strong = ok[:, None] & (P_ref >= 1e-3 * P_ref.max(0, keepdims=True))
        db = np.abs(10 * np.log10(Pg[strong] / P_ref[strong]))
        if prec in (0, 2):
            assert np.percentile(db, 99) < 0.01
        if prec == 3:
            assert np.percentile(db, 99) < 0.01


def test_sweep_invalid_arguments():
    import torch
    from paper_2402_13034_gb300 import risrt as R
    ctx = _ctx()
    A = torch.zeros((4, 3), dtype=torch.complex64, device="cuda")
    G = torch.zeros((2, 3), dtype=torch.complex64, device="cuda")
    P = torch.zeros((4, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(R.RisrtError):
        ctx.sweep_configs(A, None, G, P, 7, None)
    with pytest.raises(R.RisrtError):          # tensor-core precision without a workspace
        ctx.sweep_configs(A, None, G, P, 1, None)


@pytest.mark.parametrize("n,M,C", [(1000, 300, 300), (4097, 1024, 129), (16384, 256, 1024)])
@pytest.mark.parametrize("prec", [1, 3])
def test_pair_and_single_cta_kernels(n, M, C, prec, monkeypatch):
    """The two-CTA persistent kernel (256 x 256 tiles, double-buffered accumulators, several tiles per
    cluster at the largest size) and the one-CTA-per-tile kernel agree, and both stay within the
    precision's bound against FP64 on sampled receivers (ragged last tile: 4097 rows leaves the second
    CTA of the last pair without receivers)."""
    rng = np.random.default_rng(n * 7 + M + C)
    A = ((rng.standard_normal((n, M)) + 1j * rng.standard_normal((n, M))) * 1e-3).astype(np.complex64)
    E0 = ((rng.standard_normal(n) + 1j * rng.standard_normal(n)) * 1e-3).astype(np.complex64)
    G = np.array([1, 1j, -1, -1j], np.complex64)[rng.integers(0, 4, (C, M))]
    rows = np.unique(np.concatenate([np.arange(min(n, 64)), rng.integers(0, n, 384), [n - 1]]))
    E = E0[rows, None].astype(np.complex128) + A[rows].astype(np.complex128) @ G.T.astype(np.complex128)
    Sx = np.abs(E0[rows])[:, None] + np.abs(A[rows]).astype(np.float64) @ np.abs(G).T.astype(np.float64)
    out = {}
    for pair in ("1", "0"):
        monkeypatch.setenv("RISRT_SWEEP_PAIR", pair)
        P = _run(_ctx(), A, E0, G, prec)
        assert P.min() >= 0 and np.isfinite(P).all()
        dE = np.abs(np.sqrt(P[rows] * 2 * ETA0) - np.abs(E)) / Sx
        assert dE.max() <= TOL[prec], (pair, dE.max())
        out[pair] = P
    scale = max(out["0"].max(), 1e-30)
    assert np.abs(out["1"] - out["0"]).max() <= 1e-6 * scale


@pytest.mark.parametrize("prec", [1, 2])
def test_sweep_keep_a_and_graph_replay(prec):
    """RISRT_SWEEP_KEEP_A reuses the packed channel matrix (only Gamma is packed), and
    RISRT_SWEEP_DEFER_CHECK makes the sweep capturable: a CUDA graph of it, replayed on new
    configurations written into its input buffer, gives bitwise the results of a full sweep; fewer
    configurations than the workspace was sized for also reuse it."""
    import torch
    from paper_2402_13034_gb300 import risrt as R
    rng = np.random.default_rng(11)
    n, M, Cmax = 3000, 700, 96
    A = torch.from_numpy(((rng.standard_normal((n, M)) + 1j * rng.standard_normal((n, M))) * 1e-3).astype(np.complex64)).cuda()
    E0 = torch.from_numpy(((rng.standard_normal(n) + 1j * rng.standard_normal(n)) * 1e-2).astype(np.complex64)).cuda()
    gam = [torch.from_numpy(np.exp(2j * np.pi * rng.random((Cmax, M))).astype(np.complex64)).cuda() for _ in range(3)]
    s = torch.cuda.Stream()
    ctx = R.Context(0, s.cuda_stream)
    ref_ctx = _ctx()

    def full(G):
        P = torch.empty((n, G.shape[0]), dtype=torch.float32, device="cuda")
        ref_ctx.sweep_configs(A, E0, G, P, prec, ref_ctx.sweep_workspace(n, M, G.shape[0], prec))
        torch.cuda.synchronize()
        return P.cpu().numpy()

    ws = ctx.sweep_workspace(n, M, Cmax, prec)
    P = torch.empty((n, Cmax), dtype=torch.float32, device="cuda")
    with torch.cuda.stream(s):
        ctx.sweep_configs(A, E0, gam[0], P, prec, ws)                       # packs A into ws
        ctx.sweep_configs(A, E0, gam[1], P, prec, ws, keep_a=True)
    s.synchronize()
    assert np.array_equal(P.cpu().numpy(), full(gam[1]))
    C2 = 33                                                                   # fewer configurations, same ws
    P2 = torch.empty((n, C2), dtype=torch.float32, device="cuda")
    with torch.cuda.stream(s):
        ctx.sweep_configs(A, E0, gam[2][:C2].contiguous(), P2, prec, ws, keep_a=True)
    s.synchronize()
    assert np.array_equal(P2.cpu().numpy(), full(gam[2][:C2].contiguous()))
    # capture (A stays packed), then replay on new configurations
    G_static = gam[0].clone()
    P_static = torch.empty((n, Cmax), dtype=torch.float32, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ctx.sweep_configs(A, E0, G_static, P_static, prec, ws, keep_a=True, defer_check=True)
    for G in (gam[1], gam[2]):
        with torch.cuda.stream(s):
            G_static.copy_(G)
            g.replay()
        ctx.sweep_check(ws)
        assert np.array_equal(P_static.cpu().numpy(), full(G))


def test_sweep_options_rejected_for_fp16():
    import torch
    from paper_2402_13034_gb300 import risrt as R
    ctx = _ctx()
    A = torch.zeros((128, 64), dtype=torch.complex64, device="cuda")
    G = torch.zeros((4, 64), dtype=torch.complex64, device="cuda")
    P = torch.empty((128, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(R.RisrtError):
        ctx.sweep_configs(A, None, G, P, 3, ctx.sweep_workspace(128, 64, 4, 3), keep_a=True)
