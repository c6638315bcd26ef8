"""Vector field with polarisation on the GPU (risrt_eval_field_vec, risrt_build_A_vec) against the
oracle's vector mode: received values within 5e-5 of their incoherent magnitude (power and phase
where the field is strong), field vectors component by component within 5e-5 of the incoherent sum
of the terms' norms, channel rows element by element. Cases: the room at order 2 with a horn Tx and a
tilted-axis monopole Rx (TE and TM parts on every bounce), the paper's reflective set-up with the
horn's aperture axis, a conducting ground with oblique dipoles, and the TE co-polarised world where
the vector field equals the scalar one."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2402_13034_gb300 import scenarios as S
from tests.helpers import FIELD_TOL, compare_A, compare_fields, compare_pathsets, subset_paths

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2402_13034_gb300 import build as B
    B.build()


def _unit(v):
    v = np.asarray(v, np.float64)
    return (v / np.linalg.norm(v)).astype(np.float32)


def _run_vec(w, want_A=False):
    import torch
    from paper_2402_13034_gb300 import risrt as R
    ctx = R.Context(0, torch.cuda.current_stream().cuda_stream)
    scene, ris, rx = R.upload_workload(ctx, w)
    ps = ctx.trace_paths(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, R.flags_of(w))
    g = torch.from_numpy(np.ascontiguousarray(w.gammas, np.complex64)).cuda()
    C = g.shape[0]
    E = torch.empty((C, w.n_rx), dtype=torch.complex64, device="cuda")
    E3 = torch.empty((C, w.n_rx, 3), dtype=torch.complex64, device="cuda")
    P = torch.empty((C, w.n_rx), dtype=torch.float32, device="cuda")
    ctx.eval_field_vec(scene, rx, ps, g, E, E3, P)
    out = dict(E=E.cpu().numpy().T, P=P.cpu().numpy().T, E3=E3.cpu().numpy().transpose(1, 0, 2),
               paths=ps.export())
    # the received values alone (no field vectors) are the same numbers
    E_only = torch.empty_like(E)
    ctx.eval_field_vec(scene, rx, ps, g, E_only)
    out["E_only"] = E_only.cpu().numpy().T
    if want_A:
        A = torch.empty((w.n_rx, w.n_elem), dtype=torch.complex64, device="cuda")
        E0 = torch.empty(w.n_rx, dtype=torch.complex64, device="cuda")
        ctx.build_A_vec(scene, rx, ps, A, E0)
        # the sweep on the vector channel matrix gives the evaluated received power
        Psw = torch.empty((w.n_rx, C), dtype=torch.float32, device="cuda")
        ctx.sweep_configs(A, E0, g, Psw, R.PREC_FP32)
        out.update(A=A.cpu().numpy(), E0=E0.cpu().numpy(), P_sweep=Psw.cpu().numpy())
    torch.cuda.synchronize()
    return out


def _check_vec(w, g, want_A=False):
    o = O.Oracle(w, vector=True)
    op = o.rx_paths(w.rx_xyz)
    pc = compare_pathsets(subset_paths(g["paths"], np.arange(w.n_rx)), op, o.tx_leg())
    assert not pc["bad"], pc["bad"][:5]
    keep = ~pc["differ"]
    assert keep.mean() >= 0.9
    fld = o.field_vec(w.rx_xyz)
    E, P, Sx, E3, S3 = O.Oracle.evaluate_vec(fld, w.gammas)
    st = compare_fields(g["E"], g["P"], E, P, Sx, mask=keep)
    assert np.array_equal(g["E_only"], g["E"])
    S3s = np.where(S3 > 0, S3, 1.0)[..., None]
    err3 = np.abs(g["E3"] - E3) / S3s
    assert np.all(err3[keep] <= FIELD_TOL), f"field vector error {err3[keep].max():.3e}"
    st["max_E3"] = float(err3[keep].max())
    if want_A:
        st["max_A"] = compare_A(g["A"], fld, keep)
        S0 = np.where(fld["S0"] > 0, fld["S0"], 1.0)
        assert np.all((np.abs(g["E0"] - fld["E0"]) <= FIELD_TOL * S0)[keep])
        strong = (np.abs(E) >= 0.05 * Sx) & keep[:, None]
        rel = np.abs(g["P_sweep"] - g["P"]) / np.where(g["P"] > 0, g["P"], 1.0)
        assert np.all(rel[strong] <= 1e-4), rel[strong].max()
    # polarisation matters in these cases: the vector field is not the scalar one
    fs = O.Oracle(w).field(w.rx_xyz)
    Es = O.Oracle.evaluate(fs, w.gammas)[0]
    st["vs_scalar"] = float(np.median(np.abs(E - Es) / np.where(Sx > 0, Sx, 1.0)))
    print(f"vector {w.name}: {st}")
    return st


def _room_polarised(grid=8):
    w = S.room(grid=grid, n_boxes=12)
    w.tx = S.Antenna(w.tx.pos, S.orient_towards(w.tx.pos, w.ris.center), 1.0, 10.0, S.PATTERN_COS_POW,
                     pol=_unit((0.3, 0.2, 0.93)))
    w.rx = S.Antenna(np.zeros(3, np.float32), S.identity_orient(), 1.0, 1.0, S.PATTERN_MONOPOLE_QW,
                     pol=np.array([0.0, 0.0, 1.0], np.float32))
    w.gammas = S.phase_configs(S.SplitMix64(3), 3, w.n_elem)
    w.name = "room_polarised"
    return w


def test_vector_room_order2_against_oracle():
    w = _room_polarised()
    st = _check_vec(w, _run_vec(w, want_A=True), want_A=True)
    assert st["vs_scalar"] > 1e-3


def test_vector_room_tilted_rx_axis():
    """An Rx axis tilted out of every symmetry plane, five configurations (two kernel passes)."""
    w = _room_polarised(grid=6)
    w.rx.pol = _unit((0.5, -0.4, 0.77))
    w.gammas = S.phase_configs(S.SplitMix64(4), 5, w.n_elem)
    _check_vec(w, _run_vec(w))


def test_vector_paper_reflective():
    """Sec. III's reflective set-up: metal walls, blocking panel, horn Tx with its aperture field along
    its local x axis, vertical monopole Rx, RIS -> Rx reflections up to order 2."""
    w = S.paper_reflective(grid_step=0.1)
    w.tx.pol = np.asarray(w.tx.orient, np.float32)[0].copy()
    w.rx.pol = np.array([0.0, 0.0, 1.0], np.float32)
    _check_vec(w, _run_vec(w))


def test_vector_conducting_ground_oblique_dipoles():
    """A conducting ground under oblique dipoles (LOS and the ground's environment path in E0, the
    RIS's direct and reflected legs)."""
    from tests.test_oracle_vector_pins import _ground_world
    w = _ground_world(np.array([0.2, -0.4, 1.3], np.float32), (0.6, -0.3, 0.7), (-0.2, 0.5, 0.8))
    w.ris.center = np.array([0.0, 0.0, 0.8], np.float32)
    w.ris.t1 = np.array([0, 1, 0], np.float32)
    w.ris.t2 = np.array([0, 0, 1], np.float32)                 # normal +x, vertical RIS above the ground
    w.tx.pos = np.array([1.5, -0.7, 1.3], np.float32)
    w.rx_xyz = S.linspace_grid(0.5, 3.0, 7, -1.5, 1.5, 7, 1.1, jitter=True)
    w.gammas = S.phase_configs(S.SplitMix64(6), 2, w.n_elem)
    w.name = "ground_oblique"
    _check_vec(w, _run_vec(w, want_A=True), want_A=True)


def test_vector_te_copolarised_equals_scalar():
    """Every ray horizontal, every axis vertical: the vector field equals the scalar (TE) one."""
    from tests.test_oracle_vector_pins import _horizontal_world
    w = _horizontal_world()
    w.gammas = S.phase_configs(S.SplitMix64(8), 2, w.n_elem)
    g = _run_vec(w)
    st = _check_vec(w, g)
    assert st["vs_scalar"] < 1e-9
    assert np.max(np.abs(g["E3"][..., :2])) <= 1e-6 * np.max(np.abs(g["E3"][..., 2]))
