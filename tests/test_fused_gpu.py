"""Fused channel tile -> tensor-core sweep (risrt_sweep_fused): the channel matrix built tile by tile in
shared memory and consumed by the tensor cores without going to memory. Against the FP64 oracle's
channel rows at the BF16 bound (|dE| <= 4e-3 of |E0| + sum |A||Gamma|, 2^-8 on A), and against the
unfused path (build_A, then the BF16 sweep) on the same path set, which rounds the same FP32 channel
entries to BF16 and differs only in the order of the FP32 accumulation."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2402_13034_gb300 import scenarios as S

pytestmark = pytest.mark.gpu
ETA0 = 120 * math.pi
BF16_TOL = 4e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2402_13034_gb300 import build as B
    B.build()


def _setup(w):
    import torch
    from paper_2402_13034_gb300 import risrt as R
    ctx = R.Context(0, torch.cuda.current_stream().cuda_stream)
    scene, ris, rx = R.upload_workload(ctx, w)
    ps = ctx.trace_paths(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, R.flags_of(w))
    return ctx, (scene, ris, rx, ps)


def _fused(ctx, ps, G, n_rx, codes=None, amp=1.0):
    import torch
    C = G.shape[0] if G is not None else codes.shape[0]
    P = torch.full((n_rx, C), -1.0, dtype=torch.float32, device="cuda")
    E = torch.empty((n_rx, C), dtype=torch.complex64, device="cuda")
    g = None if G is None else torch.from_numpy(np.ascontiguousarray(G, np.complex64)).cuda()
    c = None if codes is None else torch.from_numpy(np.ascontiguousarray(codes)).cuda()
    ctx.sweep_fused(ps, g, P, gamma_2bit=c, amp=amp, E_out=E)
    torch.cuda.synchronize()
    return P.cpu().numpy().astype(np.float64), E.cpu().numpy().astype(np.complex128)


def _unfused(ctx, ps, G, n_rx, M):
    import torch
    from paper_2402_13034_gb300 import risrt as R
    A = torch.empty((n_rx, M), dtype=torch.complex64, device="cuda")
    E0 = torch.empty(n_rx, dtype=torch.complex64, device="cuda")
    ctx.build_A(ps, A, E0)
    C = G.shape[0]
    E = torch.empty((n_rx, C), dtype=torch.complex64, device="cuda")
    ws = ctx.sweep_workspace(n_rx, M, C, R.PREC_BF16)
    ctx.sweep_configs(A, E0, torch.from_numpy(np.ascontiguousarray(G, np.complex64)).cuda(), None, R.PREC_BF16, ws,
                      E_out=E)
    torch.cuda.synchronize()
    return E.cpu().numpy().astype(np.complex128), A.cpu().numpy(), E0.cpu().numpy()


@pytest.mark.parametrize("grid,C", [(9, 1), (12, 5), (16, 128)])
def test_fused_room_against_oracle_and_unfused(grid, C):
    """The room (127 elements: four K blocks, the last one ragged) on grids whose receiver count is not a
    multiple of 128."""
    w = S.room(grid=grid, n_boxes=12)
    G = S.phase_configs(S.SplitMix64(20 + C), C, w.n_elem)
    ctx, h = _setup(w)
    ps = h[3]
    P, E = _fused(ctx, ps, G, w.n_rx)
    assert np.isfinite(P).all() and P.min() >= 0
    assert np.allclose(P, np.abs(E) ** 2 / (2 * ETA0), rtol=1e-5, atol=0)
    Eu, A, E0 = _unfused(ctx, ps, G, w.n_rx, w.n_elem)
    Sx = np.abs(E0)[:, None] + np.abs(A).astype(np.float64) @ np.abs(G).T.astype(np.float64)
    Sd = np.where(Sx > 0, Sx, 1.0)
    assert np.max(np.abs(E - Eu) / Sd) <= 1e-5          # same BF16 entries, another FP32 summation order
    o = O.Oracle(w)
    fld = o.field(w.rx_xyz)
    E_ref, _, S_ref = O.Oracle.evaluate(fld, G)
    ok = ~fld["amb"]
    err = np.abs(E - E_ref) / np.where(S_ref > 0, S_ref, 1.0)
    assert np.max(err[ok]) <= BF16_TOL, np.max(err[ok])
    print(f"fused room grid {grid}, C {C}: max |dE|/S vs oracle {np.max(err[ok]):.2e}")


def test_fused_square_ris_two_bit_codes():
    """The sweep workload's 32 x 32 RIS (32 K blocks) with 2-bit codes (Gamma = amp j^q) equals the
    same configurations given as complex values, and the unfused sweep."""
    w = S.sweep(n_cfg=64, grid=24)
    q, G = w.extra["codes"], w.gammas
    codes = np.zeros((q.shape[0], (q.shape[1] + 3) // 4), np.uint8)        # four codes per byte
    for k in range(4):
        part = q[:, k::4]
        codes[:, : part.shape[1]] |= (part << (2 * k)).astype(np.uint8)
    ctx, h = _setup(w)
    ps = h[3]
    P1, E1 = _fused(ctx, ps, G, w.n_rx)
    P2, E2 = _fused(ctx, ps, None, w.n_rx, codes=codes)
    assert np.array_equal(E1, E2) and np.array_equal(P1, P2)
    Eu, A, E0 = _unfused(ctx, ps, G, w.n_rx, w.n_elem)
    Sx = np.abs(E0)[:, None] + np.abs(A).astype(np.float64) @ np.abs(G).T.astype(np.float64)
    assert np.max(np.abs(E1 - Eu) / np.where(Sx > 0, Sx, 1.0)) <= 1e-5


def test_fused_rejects_more_than_128_configurations():
    import torch
    from paper_2402_13034_gb300 import risrt as R
    w = S.room(grid=4, n_boxes=4)
    ctx, h = _setup(w)
    G = torch.ones((129, w.n_elem), dtype=torch.complex64, device="cuda")
    P = torch.empty((w.n_rx, 129), dtype=torch.float32, device="cuda")
    with pytest.raises(R.RisrtError) as e:
        ctx.sweep_fused(h[3], G, P)
    assert e.value.code == 1
