"""Shared helpers for the GPU parity tests: run the CUDA path through the binding and compare it
with the FP64 oracle on the same seeded inputs."""
import numpy as np


# Tolerances (field error relative to the incoherent magnitude S(r) everywhere; power and phase
# where the coherent field is not a deep null).
FIELD_TOL = 5e-5
POWER_RTOL = 1e-4
PHASE_TOL = 1e-3
STRONG = 0.05


def run_gpu(w, gammas=None, want_A=False, keep=False, A_rows=None):
    """Trace and evaluate workload ``w`` through the C ABI. With ``want_A`` also the channel matrix
    and E0 (with ``A_rows`` only those rows of A are copied back; the others are zero)."""
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
    if gammas is not None:
        out["gammas_used"] = np.atleast_2d(np.asarray(gammas))
    if want_A:
        A = torch.empty((w.n_rx, w.n_elem), dtype=torch.complex64, device="cuda")
        E0 = torch.empty(w.n_rx, dtype=torch.complex64, device="cuda")
        ctx.build_A(ps, A, E0)
        if A_rows is None:
            out["A"] = A.cpu().numpy()
        else:
            rows = torch.as_tensor(np.asarray(A_rows), device="cuda")
            out["A"] = np.zeros((w.n_rx, w.n_elem), np.complex64)
            out["A"][np.asarray(A_rows)] = A[rows].cpu().numpy()
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


# Ambiguous decisions (those within the oracle's band of flipping) may be excluded from bit-exact
# comparison; there must be at most this many per decision taken.
AMB_RATE_MAX = 1e-5


def _popcount(words) -> int:
    return int(sum(bin(int(x)).count("1") for x in np.asarray(words).ravel()))


def compare_pathsets(gp, op, tx_ref=None):
    """Decision-by-decision comparison of the GPU's path sets with the oracle's.

    Every Rx-leg and environment sequence, every element's direct visibility bit and the LOS bit of
    every receiver (and, with ``tx_ref``, every Tx-leg sequence and element) is one decision. The two
    sides must agree bit for bit on every decision the oracle does not flag ambiguous. Returns
    ``bad`` (unexplained differences), ``differ`` (receivers whose GPU path set differs from the
    oracle's on some ambiguous decision; all of them if the Tx leg differs), and the counts ``n_dec``
    and ``n_amb`` of decisions and of ambiguous decisions."""
    n = len(op["seqs"])
    bad = []
    differ = np.zeros(n, bool)
    for i in range(n):
        for key, akey in (("seqs", "amb_seqs"), ("env", "amb_env")):
            d = np.setxor1d(np.asarray(gp[key][i], np.int64), op[key][i])
            if d.size:
                differ[i] = True
                unexplained = np.setdiff1d(d, op[akey][i])
                if unexplained.size:
                    bad.append((key, i, unexplained[:4].tolist()))
        if bool(gp["los"][i]) != bool(op["los"][i]):
            differ[i] = True
            if not op["los_amb"][i]:
                bad.append(("los", i))
        dv = np.asarray(gp["vis"][i], np.uint32) ^ op["vis"][i]
        if dv.any():
            differ[i] = True
            if (dv & ~op["vis_amb"][i]).any():
                bad.append(("vis", i))
    n_dec = int(op["n_dec"].sum())
    n_amb = sum(len(a) for a in op["amb_seqs"]) + sum(len(a) for a in op["amb_env"]) + \
        int(op["los_amb"].sum()) + _popcount(op["vis_amb"])
    if tx_ref is not None:
        tx_differ = False
        d = np.setxor1d(np.asarray(gp["tx_seqs"], np.int64), tx_ref["seqs"])
        if d.size:
            tx_differ = True
            if np.setdiff1d(d, tx_ref["amb_seqs"]).size:
                bad.append(("tx_seq", -1, d[:4].tolist()))
        dv = np.asarray(gp["tx_vis"], bool) != tx_ref["vis"]
        if dv.any():
            tx_differ = True
            if (dv & ~tx_ref["vis_amb"]).any():
                bad.append(("tx_vis", -1))
        if tx_differ:
            differ[:] = True
        n_dec += tx_ref["n_dec"]
        n_amb += len(tx_ref["amb_seqs"]) + int(tx_ref["vis_amb"].sum())
    return dict(bad=bad, differ=differ, n_dec=n_dec, n_amb=n_amb, amb_rate=n_amb / max(n_dec, 1))


def subset_paths(gp, idx):
    """The exported GPU path set restricted to the receivers ``idx``."""
    out = {k: [gp[k][i] for i in idx] for k in ("seqs", "env")}
    out["los"] = np.asarray(gp["los"])[idx]
    out["vis"] = np.asarray(gp["vis"])[idx]
    out["tx_seqs"] = gp["tx_seqs"]
    out["tx_vis"] = gp["tx_vis"]
    return out


def compare_A(A, fld, mask, tol=FIELD_TOL):
    """Channel matrix element by element: |A_gpu[r,m] - A_ref[r,m]| <= tol * SA[r,m], the incoherent
    sum of element m's terms at receiver r; entries without any path are exactly zero."""
    SA = fld["SA"][mask]
    err = np.abs(A[mask] - fld["A"][mask])
    pos = SA > 0
    assert np.all(err[pos] <= tol * SA[pos]), f"A error {np.max(err[pos] / SA[pos]):.3e} > {tol}"
    assert np.all(np.abs(A[mask][~pos]) == 0)
    return float(np.max(err[pos] / SA[pos])) if pos.any() else 0.0


def oracle_parity(w, g, idx=None, check_A=False, amb_rate_max=AMB_RATE_MAX, min_compared=0.9):
    """The full check of one GPU run ``g`` (from run_gpu) against the oracle on the receivers ``idx``
    (all by default): path sets decision by decision, fields on every receiver whose path set equals
    the oracle's, and with ``check_A`` the channel matrix and E0 element by element."""
    from oracle import oracle as O
    idx = np.arange(w.n_rx) if idx is None else np.asarray(idx)
    rx = w.rx_xyz[idx]
    o = O.Oracle(w)
    op = o.rx_paths(rx)
    tx = o.tx_leg()
    pc = compare_pathsets(subset_paths(g["paths"], idx), op, tx)
    assert not pc["bad"], pc["bad"][:10]
    assert pc["amb_rate"] <= amb_rate_max, f"ambiguous decisions {pc['n_amb']} of {pc['n_dec']}"
    keep = ~pc["differ"]
    assert keep.mean() >= min_compared, f"only {keep.sum()} of {len(keep)} receivers comparable"
    fld = o.field(rx)
    E, P, Sx = O.Oracle.evaluate(fld, w.gammas if "gammas_used" not in g else g["gammas_used"])
    st = compare_fields(g["E"][idx], g["P"][idx], E, P, Sx, mask=keep)
    st.update(n_dec=pc["n_dec"], n_amb=pc["n_amb"], amb_rate=pc["amb_rate"],
              excluded=int((~keep).sum()), n_rx=len(idx))
    if check_A:
        st["max_A"] = compare_A(g["A"][idx], fld, keep)
        e0 = np.abs(g["E0"][idx] - fld["E0"])[keep]
        S0 = np.where(fld["S0"] > 0, fld["S0"], 1.0)[keep]
        assert np.all(e0 <= FIELD_TOL * S0)
    print(f"parity {w.name}: {st}")
    return st, o, op, fld
