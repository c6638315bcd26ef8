"""C ABI on the GPU: the context's device-memory budget, resident channel matrices (risrt_build_A with
no output array, risrt_amat_*), 2-bit configuration codes with an amplitude, and the complex field
output of the configuration sweep (Eqs. 9, 10)."""
import numpy as np
import pytest

from paper_2402_13034_gb300 import scenarios as S

pytestmark = pytest.mark.gpu
ETA0 = 120 * np.pi


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2402_13034_gb300 import build as B
    B.build()


def _traced(w, ctx):
    from paper_2402_13034_gb300 import risrt as R
    scene, ris, rx = R.upload_workload(ctx, w)
    ps = ctx.trace_paths(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, R.flags_of(w))
    return (scene, ris, rx), ps


def _ctx(budget=0):
    import torch
    from paper_2402_13034_gb300 import risrt as R
    return R.Context(0, torch.cuda.current_stream().cuda_stream, hbm_budget=budget)


def test_hbm_budget_bounds_context_memory():
    """A context created with a budget refuses an allocation that would take it past the budget
    (RISRT_ERR_OOM) and keeps working afterwards; without a budget the same request succeeds. A trace
    of 32x32 receivers fits 192 MiB; one of 256x256 does not (its two candidate slabs alone take
    2 x 65,536 x 512 x 4 B = 256 MiB)."""
    from paper_2402_13034_gb300 import risrt as R
    ctx = _ctx(budget=192 << 20)
    handles, ps = _traced(S.room(grid=32), ctx)
    with pytest.raises(R.RisrtError) as e:
        _traced(S.room(grid=256), ctx)
    assert e.value.code == 2
    amat = ctx.build_A(ps)                          # the context still works after the refusal
    assert amat.n_rx == 32 * 32
    amat.close()
    ctx2 = _ctx()
    _traced(S.room(grid=256), ctx2)


def test_device_allocation_failure_leaves_context_usable():
    """A trace whose device allocation really fails (the GPU's memory held by torch's allocator)
    returns RISRT_ERR_OOM; once the memory is back, the same context on the same thread traces
    normally: the failed allocation's error is not reported again by a later launch check."""
    import torch
    from paper_2402_13034_gb300 import risrt as R
    ctx = _ctx()
    w32 = S.room(grid=32)
    handles, ps = _traced(w32, ctx)                 # kernels loaded, context warm
    ref = ps.export()
    for h in (ps, *handles):
        h.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    hog = torch.empty(free - (256 << 20), dtype=torch.uint8, device="cuda")
    try:
        with pytest.raises(R.RisrtError) as e:
            _traced(S.room(grid=256), ctx)          # two candidate slabs alone take 256 MiB
        assert e.value.code == 2
    finally:
        del hog
        torch.cuda.empty_cache()
    handles, ps = _traced(w32, ctx)
    got = ps.export()
    for k in ("los", "vis", "tx_seqs", "tx_vis"):
        assert np.array_equal(ref[k], got[k]), k
    for k in ("seqs", "env"):
        assert all(np.array_equal(a, b) for a, b in zip(ref[k], got[k], strict=True)), k


def test_resident_channel_matrix_matches_caller_memory():
    """build_A without an output array keeps A and E0 in the library; its contents, and sweeps and
    gradients through the handle, are bitwise those of the caller-memory path."""
    import torch
    from paper_2402_13034_gb300 import risrt as R
    w = S.sweep(n_cfg=40, grid=12)
    ctx = _ctx()
    handles, ps = _traced(w, ctx)
    A = torch.empty((w.n_rx, w.n_elem), dtype=torch.complex64, device="cuda")
    E0 = torch.empty(w.n_rx, dtype=torch.complex64, device="cuda")
    assert ctx.build_A(ps, A, E0) is None
    amat = ctx.build_A(ps)
    Ar, E0r = amat.tensors()
    torch.cuda.synchronize()
    assert torch.equal(Ar, A) and torch.equal(E0r, E0)
    G = torch.from_numpy(w.gammas).cuda()
    for prec in (0, 1, 2):
        ws = ctx.sweep_workspace(w.n_rx, w.n_elem, G.shape[0], prec)
        P1 = torch.empty((w.n_rx, G.shape[0]), device="cuda")
        P2 = torch.empty_like(P1)
        ctx.sweep_configs(A, E0, G, P1, prec, ws)
        ctx.sweep_configs(amat, None, G, P2, prec, ws)
        torch.cuda.synchronize()
        assert torch.equal(P1, P2), prec
    ph = torch.rand((3, w.n_elem), device="cuda") * 6.283
    J1, J2 = torch.empty(3, device="cuda"), torch.empty(3, device="cuda")
    g1, g2 = torch.empty((3, w.n_elem), device="cuda"), torch.empty((3, w.n_elem), device="cuda")
    ctx.grad_phases(A, E0, None, ph, None, J1, g1)
    ctx.grad_phases(amat, None, None, ph, None, J2, g2)
    torch.cuda.synchronize()
    assert torch.equal(J1, J2) and torch.equal(g1, g2)
    amat.close()


@pytest.mark.parametrize("M", [64, 37])
def test_two_bit_codes_equal_complex_gamma(M):
    """Configurations given as 2-bit codes (Gamma = amp j^q, four codes per byte) give bitwise the
    results of the same configurations given as complex values, at every precision; with M not a
    multiple of 4 the unused bits of each row's last byte are ignored."""
    import torch
    rng = np.random.default_rng(M)
    n, C, amp = 700, 37, 1.25
    A = ((rng.standard_normal((n, M)) + 1j * rng.standard_normal((n, M))) * 1e-3).astype(np.complex64)
    E0 = ((rng.standard_normal(n) + 1j * rng.standard_normal(n)) * 1e-3).astype(np.complex64)
    q = rng.integers(0, 4, (C, M)).astype(np.uint8)
    nb = (M + 3) // 4
    packed = np.zeros((C, nb), np.uint8)
    for m in range(M):
        packed[:, m // 4] |= q[:, m] << (2 * (m % 4))
    if M % 4:
        packed[:, -1] |= np.uint8(0xFF) << np.uint8(2 * (M % 4))     # garbage in the unused bits
    G = (amp * np.array([1, 1j, -1, -1j], np.complex64)[q]).astype(np.complex64)
    ctx = _ctx()
    Ad, E0d = torch.from_numpy(A).cuda(), torch.from_numpy(E0).cuda()
    for prec in (0, 1, 2, 3):
        ws = ctx.sweep_workspace(n, M, C, prec)
        P1 = torch.empty((n, C), device="cuda")
        P2 = torch.empty_like(P1)
        ctx.sweep_configs(Ad, E0d, torch.from_numpy(G).cuda(), P1, prec, ws)
        ctx.sweep_configs(Ad, E0d, None, P2, prec, ws, gamma_2bit=torch.from_numpy(packed).cuda(), amp=amp)
        torch.cuda.synchronize()
        assert torch.equal(P1, P2), prec


# field error relative to sum |A||Gamma| + |E0| per precision, the bounds of the sweep tests for
# configurations of arbitrary phase (rounded to BF16 / FP16 on the tensor cores)
E_TOL = {0: 5e-5, 1: 4e-3, 2: 4e-3, 3: 1e-3}


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_sweep_complex_output(prec):
    """E_out = E0 + A Gamma against FP64 within the precision's error bound, and |E_out|^2 / (2 eta0)
    equal to P_out; a call with E_out only (no power) gives the same field."""
    import torch
    rng = np.random.default_rng(5 + prec)
    n, M, C = 1000, 300, 130
    A = ((rng.standard_normal((n, M)) + 1j * rng.standard_normal((n, M))) * 1e-3).astype(np.complex64)
    E0 = ((rng.standard_normal(n) + 1j * rng.standard_normal(n)) * 1e-2).astype(np.complex64)
    G = np.exp(2j * np.pi * rng.random((C, M))).astype(np.complex64)
    ref = E0.astype(np.complex128)[:, None] + A.astype(np.complex128) @ G.T.astype(np.complex128)
    S_ = np.abs(E0)[:, None] + np.abs(A).astype(np.float64) @ np.abs(G).T.astype(np.float64)
    ctx = _ctx()
    Ad, E0d, Gd = (torch.from_numpy(x).cuda() for x in (A, E0, G))
    ws = ctx.sweep_workspace(n, M, C, prec)
    P = torch.empty((n, C), device="cuda")
    E = torch.empty((n, C), dtype=torch.complex64, device="cuda")
    E2 = torch.empty_like(E)
    ctx.sweep_configs(Ad, E0d, Gd, P, prec, ws, E_out=E)
    ctx.sweep_configs(Ad, E0d, Gd, None, prec, ws, E_out=E2)
    torch.cuda.synchronize()
    Eg = E.cpu().numpy().astype(np.complex128)
    err = np.abs(Eg - ref) / S_
    assert err.max() <= E_TOL[prec], err.max()
    Pg = P.cpu().numpy().astype(np.float64)
    assert np.allclose(Pg, np.abs(Eg) ** 2 / (2 * ETA0), rtol=1e-5, atol=0)
    assert torch.equal(E, E2)


def test_sweep_rejects_both_or_no_gamma():
    import torch
    from paper_2402_13034_gb300 import risrt as R
    ctx = _ctx()
    A = torch.zeros((4, 8), dtype=torch.complex64, device="cuda")
    G = torch.zeros((2, 8), dtype=torch.complex64, device="cuda")
    codes = torch.zeros((2, 2), dtype=torch.uint8, device="cuda")
    P = torch.zeros((4, 2), device="cuda")
    with pytest.raises(R.RisrtError):
        ctx.sweep_configs(A, None, G, P, 0, None, gamma_2bit=codes)
    with pytest.raises(R.RisrtError):
        ctx.sweep_configs(A, None, G, None, 0, None)          # neither P nor E requested
