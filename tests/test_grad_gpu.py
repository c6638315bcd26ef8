"""Adjoint phase gradient: the CUDA path (risrt_grad_phases) against the FP64 oracle's analytic
gradient; the oracle's gradient is pinned by central finite differences of its own objective."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2402_13034_gb300 import scenarios as S


def _room_fields(grid=10):
    w = S.sweep(n_cfg=4, grid=grid)
    fld = O.Oracle(w).field(w.rx_xyz)
    return w, fld


def test_oracle_gradient_matches_finite_differences():
    w, fld = _room_fields(grid=6)
    ok = ~fld["amb"] & (fld["S0"] + fld["SA"].sum(1) > 0)
    f = {k: (v[ok] if isinstance(v, np.ndarray) and v.shape[:1] == ok.shape else v) for k, v in fld.items()}
    rng = np.random.default_rng(2)
    ph = rng.random((2, w.n_elem)) * 2 * np.pi
    J, g = O.log_power_and_grad(f, ph)
    h = 1e-4
    for m in rng.integers(0, w.n_elem, 6):
        e = np.zeros_like(ph)
        e[:, m] = h
        Jp, _ = O.log_power_and_grad(f, ph + e)
        Jm, _ = O.log_power_and_grad(f, ph - e)
        fd = (Jp - Jm) / (2 * h)
        assert np.allclose(fd, g[:, m], rtol=1e-6, atol=1e-8 * np.abs(g).max())


@pytest.mark.gpu
def test_grad_phases_against_oracle():
    import torch
    from paper_2402_13034_gb300 import build as B
    from paper_2402_13034_gb300 import risrt as R
    B.build()
    w, fld = _room_fields(grid=10)
    ctx = R.Context(0, torch.cuda.current_stream().cuda_stream)
    scene, ris, rx = R.upload_workload(ctx, w)
    ps = ctx.trace_paths(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, R.flags_of(w))
    A = torch.empty((w.n_rx, w.n_elem), dtype=torch.complex64, device="cuda")
    E0 = torch.empty(w.n_rx, dtype=torch.complex64, device="cuda")
    ctx.build_A(ps, A, E0)
    ok = np.where(~fld["amb"] & (fld["S0"] + fld["SA"].sum(1) > 0))[0]
    target = torch.from_numpy(ok.astype(np.int32)).cuda()
    rng = np.random.default_rng(4)
    Bn = 5
    ph = (rng.random((Bn, w.n_elem)) * 2 * np.pi).astype(np.float32)
    amp = (0.5 + rng.random(w.n_elem)).astype(np.float32)
    J = torch.empty(Bn, device="cuda")
    g = torch.empty((Bn, w.n_elem), device="cuda")
    ctx.grad_phases(A, E0, target, torch.from_numpy(ph).cuda(), torch.from_numpy(amp).cuda(), J, g)
    f = {"E0": fld["E0"][ok], "A": fld["A"][ok]}
    J_ref, g_ref = O.log_power_and_grad(f, ph.astype(np.float64), amp.astype(np.float64))
    Jg, gg = J.cpu().numpy().astype(np.float64), g.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(Jg - J_ref) <= 1e-4 * np.abs(J_ref) + 1e-3)
    rel = np.linalg.norm(gg - g_ref, axis=1) / np.linalg.norm(g_ref, axis=1)
    assert rel.max() <= 1e-4, rel


@pytest.mark.gpu
def test_grad_phases_rejects_bad_target():
    import torch
    from paper_2402_13034_gb300 import risrt as R
    ctx = R.Context(0, torch.cuda.current_stream().cuda_stream)
    A = torch.zeros((4, 3), dtype=torch.complex64, device="cuda")
    ph = torch.zeros((1, 3), device="cuda")
    with pytest.raises(R.RisrtError):
        ctx.grad_phases(A, None, torch.tensor([0, 9], dtype=torch.int32, device="cuda"), ph, None,
                        torch.empty(1, device="cuda"), torch.empty((1, 3), device="cuda"))
