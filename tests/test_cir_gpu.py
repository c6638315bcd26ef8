"""Channel impulse response of the RIS part (risrt_eval_cir) and the paper's reflective set-up on the
GPU, against the FP64 oracle: every tap (Rx-leg path q, Tx-leg path p) within 5e-5 of its own
incoherent magnitude, delays through the RIS centre within the FP32 rounding of the stored Rx-leg
length, and the taps plus E0 equal to the evaluated field (Sec. II-B, Eq. 9)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2402_13034_gb300 import scenarios as S
from tests.helpers import FIELD_TOL, compare_pathsets, oracle_parity, run_gpu, subset_paths

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2402_13034_gb300 import build as B
    B.build()


def _check_cir(w, idx, gamma):
    import torch
    g = run_gpu(w, gammas=gamma[None], keep=True)
    ctx, scene, ris, rx, ps = g["handles"]
    taps, rxd, txd = ctx.eval_cir(ps, torch.from_numpy(np.ascontiguousarray(gamma, np.complex64)).cuda())
    torch.cuda.synchronize()
    taps, rxd, txd = taps.cpu().numpy(), rxd.cpu().numpy(), txd.cpu().numpy()
    P = taps.shape[1]
    off = np.concatenate([[0], np.cumsum([1 + len(s) for s in g["paths"]["seqs"]])])
    o = O.Oracle(w)
    op = o.rx_paths(w.rx_xyz[idx])
    pc = compare_pathsets(subset_paths(g["paths"], idx), op, o.tx_leg())
    assert not pc["bad"], pc["bad"][:5]
    ref = o.cir(w.rx_xyz[idx], gamma)
    n_taps = worst = 0
    for k, i in enumerate(idx):
        if pc["differ"][k]:
            continue
        rows = taps[off[i]:off[i + 1]]                  # [Q, P]
        assert rows.size == len(ref[k]["amp"])
        a = rows.reshape(-1)
        err = np.abs(a - ref[k]["amp"])
        sa = ref[k]["sabs"]
        assert np.all(err[sa > 0] <= FIELD_TOL * sa[sa > 0]), np.max(err[sa > 0] / sa[sa > 0])
        assert np.all(a[sa == 0] == 0)
        worst = max(worst, float(np.max(err[sa > 0] / sa[sa > 0])) if (sa > 0).any() else 0.0)
        tau = (txd[None, :] + rxd[off[i]:off[i + 1], None]).reshape(-1)
        assert np.all(np.abs(tau - ref[k]["delay"]) <= 1e-6 * ref[k]["delay"])
        n_taps += a.size
    # the taps of each receiver plus E0 give the evaluated field
    E0 = torch.empty(w.n_rx, dtype=torch.complex64, device="cuda")
    A = torch.empty((w.n_rx, w.n_elem), dtype=torch.complex64, device="cuda")
    ctx.build_A(ps, A, E0)
    E0 = E0.cpu().numpy()
    tap_sum = np.add.reduceat(taps.sum(1), off[:-1])
    fld = o.field(w.rx_xyz)
    _, _, Sx = O.Oracle.evaluate(fld, gamma)
    assert np.all(np.abs(tap_sum + E0 - g["E"][:, 0]) <= FIELD_TOL * np.where(Sx > 0, Sx, 1.0))
    print(f"CIR {w.name}: {n_taps} taps, P = {P}, max tap error / incoherent magnitude {worst:.2e}")
    return taps, rxd, txd


def test_cir_room_with_tx_leg_reflections():
    """The room at order 2 on both legs: several Tx-leg paths per element, so each Rx-leg entry has
    one tap per Tx-leg path."""
    w = S.room(grid=6, n_boxes=12)
    rng = np.random.default_rng(3)
    gamma = np.exp(2j * np.pi * rng.random(w.n_elem)).astype(np.complex64)
    taps, _, txd = _check_cir(w, np.arange(w.n_rx), gamma)
    assert taps.shape[1] > 3


def test_cir_paper_reflective():
    """The reflective set-up of Sec. III (metal walls, blocking panel, horn Tx, monopole Rx, RIS -> Rx
    reflections up to order 2) on a coarse grid of its receiver region."""
    w = S.paper_reflective(grid_step=0.1)
    _check_cir(w, np.arange(w.n_rx), w.gammas[0])


def test_reflective_closeup_parity_and_fading():
    """The close-up of Fig. 5 (101 x 101 receivers at 2 mm): fields match the oracle on every receiver,
    and along x the GPU's received power fades with a dominant period of about lambda/2 (Sec. IV-B)."""
    w = S.paper_reflective(closeup=True)
    g = run_gpu(w)
    oracle_parity(w, g)
    lam = S.C0 / w.freq_hz
    P = g["P"][:, 0].reshape(101, 101)                   # rows: y, columns: x (x fastest)
    step = 0.002
    periods = []
    for row in P[45:56]:
        spec = np.abs(np.fft.rfft(row - row.mean()))
        f = np.fft.rfftfreq(len(row), step)
        periods.append(1.0 / f[1 + np.argmax(spec[1:])])
    med = float(np.median(periods))
    print(f"close-up fading period along x: median {med * 1e3:.2f} mm, lambda/2 = {lam / 2 * 1e3:.2f} mm")
    assert 0.5 * lam <= med <= 0.75 * lam
