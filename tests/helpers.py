"""Shared helpers for the GPU parity tests: run the CUDA path through the binding and compare it
with the FP64 oracle on the same seeded inputs."""
import numpy as np


# Tolerances (field error relative to the incoherent magnitude S(r) everywhere; power and phase
# where the coherent field is not a deep null).
FIELD_TOL = 5e-5
POWER_RTOL = 1e-4
PHASE_TOL = 1e-3
STRONG = 0.05


def run_gpu(w, gammas=None, want_A=False, keep=False):
    import torch
    from paper_2402_13034_gb300 import risrt as R
    ctx = R.Context(0, torch.cuda.current_stream().cuda_stream)
    scene, ris, rx = R.upload_workload(ctx, w)
    ps = ctx.trace_paths(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, R.flags_of(w))
    g = torch.from_numpy(np.ascontiguousarray(w.gammas if gammas is None else gammas, np.complex64)).cuda()
    if g.dim() == 1:
        g = g[None]
    E = torch.empty((g.shape[0], w.n_rx), dtype=torch.complex64, device="cuda")
    P = torch.empty((g.shape[0], w.n_rx), dtype=torch.float32, device="cuda")
    ctx.eval_field(ps, g, E, P)
    out = dict(E=E.cpu().numpy().T, P=P.cpu().numpy().T, paths=ps.export())
    if want_A:
        A = torch.empty((w.n_rx, w.n_elem), dtype=torch.complex64, device="cuda")
        E0 = torch.empty(w.n_rx, dtype=torch.complex64, device="cuda")
        ctx.build_A(ps, A, E0)
        out["A"] = A.cpu().numpy()
        out["E0"] = E0.cpu().numpy()
    torch.cuda.synchronize()
    if keep:
        out["handles"] = (ctx, scene, ris, rx, ps)
    return out


def compare_fields(E, P, E_ref, P_ref, S_ref, mask=None):
    """Returns a dict of error statistics and asserts the tolerances on the masked receivers."""
    E, P = np.atleast_2d(E), np.atleast_2d(P)
    if mask is None:
        mask = np.ones(E.shape[0], bool)
    m = mask[:, None] & np.ones_like(S_ref, bool)
    S = np.where(S_ref > 0, S_ref, 1.0)
    ferr = np.abs(E - E_ref) / S
    assert np.all(ferr[m] <= FIELD_TOL), f"field error {ferr[m].max():.3e} > {FIELD_TOL}"
    strong = m & (np.abs(E_ref) >= STRONG * S_ref) & (S_ref > 0)
    perr = np.abs(P - P_ref) / np.where(P_ref > 0, P_ref, 1.0)
    aerr = np.abs(np.angle(E * np.conj(E_ref)))
    if strong.any():
        assert np.all(perr[strong] <= POWER_RTOL), f"power error {perr[strong].max():.3e}"
        assert np.all(aerr[strong] <= PHASE_TOL), f"phase error {aerr[strong].max():.3e}"
    # receivers with no path at all must be exactly zero on both sides
    zero = m & (S_ref == 0)
    assert np.all(np.abs(E[zero]) == 0)
    return dict(max_field=float(ferr[m].max()) if m.any() else 0.0,
                max_power=float(perr[strong].max()) if strong.any() else 0.0,
                max_phase=float(aerr[strong].max()) if strong.any() else 0.0,
                strong_frac=float(strong.sum() / max(m.sum(), 1)))


def compare_pathsets(gp, op, amb, tx_ref=None):
    """Bit-exact comparison of path sets on receivers without ambiguous decisions."""
    n = len(op["seqs"])
    bad = []
    for i in range(n):
        if amb[i]:
            continue
        if not np.array_equal(np.sort(gp["seqs"][i]), np.sort(op["seqs"][i])):
            bad.append(("rx_seq", i))
        if not np.array_equal(np.sort(gp["env"][i]), np.sort(op["env"][i])):
            bad.append(("env", i))
        if gp["los"][i] != op["los"][i]:
            bad.append(("los", i))
        if not np.array_equal(gp["vis"][i], op["vis"][i]):
            bad.append(("vis", i))
    if tx_ref is not None and not tx_ref["amb"]:
        if not np.array_equal(np.sort(gp["tx_seqs"]), np.sort(tx_ref["seqs"])):
            bad.append(("tx_seq", -1))
        if not np.array_equal(gp["tx_vis"], tx_ref["vis"]):
            bad.append(("tx_vis", -1))
    return bad
