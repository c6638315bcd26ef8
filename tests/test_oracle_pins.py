"""Pins of the FP64 oracle against results the paper and the mathematics fix independently.

Each test checks the oracle against something other than itself: textbook closed forms (Friis,
Fresnel in its Snell-law form, Brewster's angle), the Tang22 path-loss formula the paper says its
model reduces to (Sec. II-A), the far-field law of a phase-aligned RIS, pattern normalisation,
brute-force Fermat minimisation for the image method, reciprocity, and values printed in the paper.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import oracle as O
from paper_2402_13034_gb300 import scenarios as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ETA0 = 120 * math.pi


def _free(freq=28e9, M_rings=3, pitch=None, tx=(0.0, -1.5, 2.0), tx_pat=S.PATTERN_ISO, tx_gain=1.0,
          rx_pat=S.PATTERN_ISO, rx_gain=1.0, tx_orient=None, rx_orient=None, power=1.0, elem_gain=0.0,
          layout=None, d=None):
    lam = S.C0 / freq
    pitch = pitch or lam / 2
    d = d or lam / 2
    uv = layout if layout is not None else S.hex_layout(M_rings, pitch)
    ris = S.RIS(uv, np.zeros(3, np.float32), np.array([1, 0, 0], np.float32),
                np.array([0, 1, 0], np.float32), d, d, elem_gain, -1)
    txa = S.Antenna(np.asarray(tx, np.float32), tx_orient if tx_orient is not None else S.identity_orient(),
                    power, tx_gain, tx_pat)
    rxa = S.Antenna(np.zeros(3, np.float32), rx_orient if rx_orient is not None else S.identity_orient(),
                    1.0, rx_gain, rx_pat)
    return S.Workload("t", freq, S.empty_scene(), ris, txa, rxa, np.zeros((1, 3), np.float32),
                      np.ones((1, len(uv)), np.complex64), 0, 0, False)


def _plane_scene(z=0.0, half=50.0, eps=5.3, sigma=0.0, extra_planes=()):
    mb = S._MeshBuilder()
    mats = [(eps, sigma)]
    mb.quad((-half, -half, z), (half, -half, z), (half, half, z), (-half, half, z), 0)
    for zz in extra_planes:
        mb.quad((-half, -half, zz), (-half, half, zz), (half, half, zz), (half, -half, zz), 0)
    return mb.scene(mats)


# ------------------------------------------------------------------------------------------------
# T1: Friis (Eq. 4 + Eq. 8 with no RIS factor) - power and phase sign
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("rx", [(0.3, 0.7, 1.5), (-1.9, 1.2, 1.5), (2.0, -2.0, 1.5)])
def test_friis_los(rx):
    w = _free(power=0.37, tx_gain=1.0, rx_gain=1.0)
    o = O.Oracle(w)
    f = o.field(np.array([rx], np.float32))
    E, P, _ = o.evaluate(f, np.zeros(w.n_elem))
    lam = S.C0 / w.freq_hz
    d = np.linalg.norm(np.asarray(rx, np.float32).astype(np.float64) - w.tx.pos.astype(np.float64))
    P_friis = float(np.float32(0.37)) * (lam / (4 * math.pi * d)) ** 2
    assert abs(P[0] / P_friis - 1) < 1e-12
    # phase -k d (e^{+j omega t} convention, Eq. 3)
    ph = (-2 * math.pi * d / lam) % (2 * math.pi)
    assert abs(np.angle(E[0] * np.exp(-1j * ph))) < 1e-9


def test_friis_with_patterns():
    """Directive Tx (cos^(G/2-1), Sec. III-B) and monopole Rx: P = Pt Gt Ft Gr Fr (lambda/4 pi d)^2."""
    txp = np.array([0.0, -1.5, 2.0])
    rxp = np.array([0.4, 0.5, 1.1], np.float32)
    w = _free(tx_pat=S.PATTERN_COS_POW, tx_gain=10 ** 1.9, rx_pat=S.PATTERN_MONOPOLE_QW,
              tx_orient=S.orient_towards(txp, (0, 0, 0)))
    o = O.Oracle(w)
    E, P, _ = o.evaluate(o.field(rxp[None]), np.zeros(w.n_elem))
    dvec = rxp.astype(np.float64) - w.tx.pos.astype(np.float64)
    d = np.linalg.norm(dvec)
    zt = w.tx.orient[2].astype(np.float64)
    cos_t = dvec @ zt / d / np.linalg.norm(zt)
    Gt = np.float32(10 ** 1.9)
    Ft = cos_t ** (float(Gt) / 2 - 1)
    cos_r = -dvec[2] / d
    Fr = (math.cos(math.pi / 2 * cos_r) / math.sqrt(1 - cos_r ** 2)) ** 2
    lam = S.C0 / w.freq_hz
    assert abs(P[0] / (float(Gt) * Ft * Fr * (lam / (4 * math.pi * d)) ** 2) - 1) < 1e-10


# ------------------------------------------------------------------------------------------------
# T2: reduction to the Tang22 model (Sec. II-A, last paragraph)
# ------------------------------------------------------------------------------------------------
def _tang22_power(w, rx, gamma, G):
    """Tang et al. 2022 RIS path loss, P = Pt Gt Gr G dx dy lambda^2/(64 pi^3) |sum F^1/2 Gamma e^{-jk(rt+rr)}/(rt rr)|^2."""
    lam = S.C0 / w.freq_hz
    k = 2 * math.pi / lam
    ris = w.ris
    c = ris.center.astype(np.float64)
    t1, t2 = ris.t1.astype(np.float64), ris.t2.astype(np.float64)
    n = np.cross(t1, t2)
    n /= np.linalg.norm(n)
    e = c + ris.elem_uv[:, :1].astype(np.float64) * t1 + ris.elem_uv[:, 1:].astype(np.float64) * t2
    T = w.tx.pos.astype(np.float64)
    R = np.asarray(rx, np.float32).astype(np.float64)
    rt = np.linalg.norm(e - T, axis=1)
    rr = np.linalg.norm(R - e, axis=1)
    cos_in = ((T - e) @ n) / rt
    cos_out = ((R - e) @ n) / rr
    zt = w.tx.orient[2].astype(np.float64)
    zt /= np.linalg.norm(zt)
    cos_tx = ((e - T) @ zt) / rt
    Gt = float(np.float32(w.tx.gain_lin))
    Ft = np.where(cos_tx > 0, np.abs(cos_tx) ** (Gt / 2 - 1), 0) if w.tx.pattern == S.PATTERN_COS_POW else 1.0
    zr = w.rx.orient[2].astype(np.float64)
    cos_rx = ((e - R) @ zr) / rr
    Fr = (np.cos(math.pi / 2 * cos_rx) / np.sqrt(1 - cos_rx ** 2)) ** 2 \
        if w.rx.pattern == S.PATTERN_MONOPOLE_QW else 1.0
    Fc = Ft * Fr * cos_in * cos_out
    s = np.sum(np.sqrt(Fc) * gamma * np.exp(-1j * k * (rt + rr)) / (rt * rr))
    Pt, Gr = float(np.float32(w.tx.power_w)), float(np.float32(w.rx.gain_lin))
    dx, dy = float(np.float32(ris.dy)), float(np.float32(ris.dz))
    return Pt * Gt * Gr * G * dx * dy * lam ** 2 / (64 * math.pi ** 3) * abs(s) ** 2


@pytest.mark.parametrize("elem_gain", [0.0, 3.7])
def test_tang22_reduction(elem_gain):
    w = S.paper_anechoic()
    w.ris.elem_gain = elem_gain
    o = O.Oracle(w)
    rng = np.random.default_rng(5)
    gamma = 1.25 * np.exp(2j * np.pi * rng.random(w.n_elem))
    rx = np.array([[1.33, 0.23, 0.11], [1.0, 0.8, 0.114], [1.5, 0.05, 0.2]], np.float32)
    f = o.field(rx)
    lam = S.C0 / w.freq_hz
    dy = float(np.float32(w.ris.dy))
    G = float(np.float32(elem_gain)) if elem_gain > 0 else 4 * math.pi * dy * dy / lam ** 2
    for i in range(len(rx)):
        E_ris = f["A"][i] @ gamma      # RIS part only (LOS is separate in E0)
        P_ris = abs(E_ris) ** 2 / (2 * ETA0)
        assert abs(P_ris / _tang22_power(w, rx[i], gamma, G) - 1) < 1e-11


def test_tang22_default_gain_form():
    """With G = 4 pi dy dz / lambda^2 the prefactor becomes Pt Gt Gr (dy dz)^2 / (16 pi^2) (Sec. II-A)."""
    w = _free()
    lam = S.C0 / w.freq_hz
    d = float(np.float32(w.ris.dy))
    G = 4 * math.pi * d * d / lam ** 2
    assert abs(G * d * d * lam ** 2 / (64 * math.pi ** 3) / ((d * d) ** 2 / (16 * math.pi ** 2)) - 1) < 1e-14
    o = O.Oracle(w)
    rx = np.array([[0.5, 0.2, 1.5]], np.float32)
    g = np.exp(1j * np.linspace(0, 3, w.n_elem))
    P = abs(o.field(rx)["A"][0] @ g) ** 2 / (2 * ETA0)
    assert abs(P / _tang22_power(w, rx[0], g, G) - 1) < 1e-11


# ------------------------------------------------------------------------------------------------
# T3/T4: coherent focusing, N^2 gain and the far-field law
# ------------------------------------------------------------------------------------------------
def _far_field_case(s, rings):
    """Tx and Rx at distances s*d1, s*d2 on fixed directions; geometric phase alignment."""
    freq = 28e9
    lam = S.C0 / freq
    d1, d2 = 1.0, 1.3
    ut = np.array([0.3, -0.4, 1.0]); ut /= np.linalg.norm(ut)
    ur = np.array([-0.5, 0.2, 1.0]); ur /= np.linalg.norm(ur)
    tx = (s * d1 * ut).astype(np.float32)
    rx = (s * d2 * ur).astype(np.float32)
    w = _free(freq=freq, M_rings=rings, tx=tx)
    o = O.Oracle(w)
    e = o.element_positions()
    dt = np.linalg.norm(e - tx.astype(np.float64), axis=1)
    dr = np.linalg.norm(rx.astype(np.float64) - e, axis=1)
    k = 2 * math.pi / lam
    gamma = np.exp(1j * k * (dt + dr))
    f = o.field(rx[None])
    A = f["A"][0]
    E_ris = A @ gamma
    dtt = np.linalg.norm(tx.astype(np.float64))
    drr = np.linalg.norm(rx.astype(np.float64))
    cos_i = tx.astype(np.float64)[2] / dtt
    cos_r = rx.astype(np.float64)[2] / drr
    N = w.n_elem
    d = float(np.float32(w.ris.dy))
    P_far = N ** 2 * (d * d) ** 2 * cos_i * cos_r / (16 * math.pi ** 2)  # Pt = Gt = Gr = 1
    return abs(E_ris) ** 2 / (2 * ETA0) * dtt ** 2 * drr ** 2, P_far, A, gamma


def test_coherent_sum_is_incoherent_sum_when_aligned():
    _, _, A, gamma = _far_field_case(4.0, 3)
    assert abs(abs(A @ gamma) / np.sum(np.abs(A)) - 1) < 1e-12


def test_far_field_law_and_n2_gain():
    errs = []
    for s in (1.0, 4.0, 16.0, 64.0):
        p, pf, _, _ = _far_field_case(s, 3)
        errs.append(abs(p / pf - 1))
    assert errs[-1] < 1e-4
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1))
    # error falls at least quadratically in 1/s between s=16 and s=64
    assert errs[-1] < errs[-2] / 8
    p37, _, _, _ = _far_field_case(64.0, 3)
    p127, _, _, _ = _far_field_case(64.0, 6)
    assert abs(p127 / p37 / (127 / 37) ** 2 - 1) < 1e-3


# ------------------------------------------------------------------------------------------------
# T5: pattern normalisation pins "Gt linear" and the exponent Gt/2 - 1 (Sec. III-B)
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("gain_db", [10.0, 19.0, 25.0])
def test_cos_pow_directivity(gain_db):
    G = 10 ** (gain_db / 10)
    th = np.linspace(0, math.pi, 200001)
    F = np.array([O.pattern(S.PATTERN_COS_POW, G, math.cos(t)) for t in th])
    integral = 2 * math.pi * np.trapezoid(F * np.sin(th), th)
    assert abs(4 * math.pi / integral / G - 1) < 1e-6


def test_monopole_shape():
    assert O.pattern(S.PATTERN_MONOPOLE_QW, 1.0, 0.0) == pytest.approx(1.0, abs=1e-15)
    assert O.pattern(S.PATTERN_MONOPOLE_QW, 1.0, 1.0) == 0.0
    # symmetric about the horizontal plane and small near the axis
    for c in (0.1, 0.5, 0.9):
        assert O.pattern(S.PATTERN_MONOPOLE_QW, 1.0, c) == pytest.approx(O.pattern(S.PATTERN_MONOPOLE_QW, 1.0, -c))
    assert O.pattern(S.PATTERN_MONOPOLE_QW, 1.0, 0.99999) < 1e-4


def test_element_pattern_front_hemisphere():
    """F(theta)=cos(theta) (Sec. III-C): an Rx behind the RIS plane receives nothing through the RIS."""
    w = _free()
    o = O.Oracle(w)
    f = o.field(np.array([[0.2, 0.1, -1.0]], np.float32))
    assert np.all(f["A"] == 0)


# ------------------------------------------------------------------------------------------------
# T6: Fresnel and the image method on brute-force tiny scenes
# ------------------------------------------------------------------------------------------------
def test_fresnel_te_snell_form():
    """TE coefficient against its Snell's-law form (n1 cos i - n2 cos t)/(n1 cos i + n2 cos t)."""
    for eps in (2.0, 5.3, 9.0):
        n2 = math.sqrt(eps)
        for th in np.linspace(0, 1.5, 13):
            tt = math.asin(math.sin(th) / n2)
            R = (math.cos(th) - n2 * math.cos(tt)) / (math.cos(th) + n2 * math.cos(tt))
            assert O.fresnel(math.cos(th), eps, 0.0, 28e9) == pytest.approx(R, abs=1e-13)


def test_fresnel_limits():
    eps = 5.3
    assert O.fresnel(1.0, eps, 0.0, 28e9) == pytest.approx((1 - math.sqrt(eps)) / (1 + math.sqrt(eps)), abs=1e-14)
    assert O.fresnel(1e-9, eps, 0.0, 28e9) == pytest.approx(-1.0, abs=1e-8)
    # PEC limit: metal eps_r = 1, sigma = 1e7 S/m at 23.8 GHz (Table 1)
    for th in (0.0, 0.5, 1.2):
        assert abs(abs(O.fresnel(math.cos(th), 1.0, 1e7, 23.8e9)) - 1) < 1e-3
    # TM vanishes at Brewster's angle tan(theta_B) = sqrt(eps)
    thb = math.atan(math.sqrt(eps))
    assert abs(O.fresnel(math.cos(thb), eps, 0.0, 28e9, tm=True)) < 1e-14


def _one_plane_workload(tx, eps=5.3, sigma=0.0):
    w = _free(tx=tx)
    w.scene = _plane_scene(0.0, 50.0, eps, sigma)
    # lift the RIS off the plane so it does not sit in the floor; the plane is face 0
    w.ris.center = np.array([0.0, 0.0, 1.0], np.float32)
    w.max_order_rx = 1
    w.env_paths = True
    return w


@pytest.mark.parametrize("tx,rx", [((0.0, -1.5, 2.0), (1.2, 0.7, 0.6)), ((3.0, 1.0, 0.3), (-2.0, 0.5, 2.5))])
def test_image_method_fermat_and_fresnel(tx, rx):
    w = _one_plane_workload(tx)
    o = O.Oracle(w)
    T = np.asarray(tx, np.float32).astype(np.float64)
    R = np.asarray(rx, np.float32).astype(np.float64)
    ok, amb, pts = o.validate(T, -1, R, -1, 0)
    assert ok and not amb
    L_img = np.linalg.norm(pts[1] - T) + np.linalg.norm(R - pts[1])
    # brute force Fermat: shortest T -> (x, y, 0) -> R over the plane
    res = minimize(lambda p: np.linalg.norm(np.array([p[0], p[1], 0]) - T) + np.linalg.norm(R - np.array([p[0], p[1], 0])),
                   x0=[0.0, 0.0], method="Nelder-Mead", options=dict(xatol=1e-12, fatol=1e-14, maxiter=20000))
    assert abs(res.fun - L_img) < 1e-9
    assert np.allclose(pts[1][:2], res.x, atol=1e-5)
    # field: E0 = LOS + R_TE(theta_i) * Friis(L1 + L2) (Eq. 4 + Eq. 8 along the unfolded path)
    f = o.field(R.astype(np.float32)[None])
    lam = S.C0 / w.freq_hz
    k = 2 * math.pi / lam
    d = np.linalg.norm(R - T)
    cos_i = abs(T[2] - pts[1][2]) / np.linalg.norm(pts[1] - T)
    n2 = math.sqrt(float(np.float32(5.3)))   # materials travel as float32
    sin_i = math.sqrt(1 - cos_i ** 2)
    cos_t = math.sqrt(1 - (sin_i / n2) ** 2)
    Rte = (cos_i - n2 * cos_t) / (cos_i + n2 * cos_t)
    amp = lambda L: math.sqrt(2 * ETA0) * lam / (4 * math.pi * L)
    E_exp = amp(d) * np.exp(-1j * k * d) + Rte * amp(L_img) * np.exp(-1j * k * L_img)
    assert abs(f["E0"][0] - E_exp) < 1e-12 * abs(E_exp)


def test_image_method_finite_wall_brute_force():
    """A 1x1 m wall: the image-method path is valid iff the Fermat point lies inside the wall."""
    mb = S._MeshBuilder()
    mb.quad((0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), 0)
    w = _free()
    w.scene = mb.scene([(5.3, 0.0)])
    o = O.Oracle(w)
    rng = np.random.default_rng(1)
    n_valid = 0
    for _ in range(200):
        T = np.array([rng.uniform(-1, 2), rng.uniform(-1, 2), rng.uniform(0.2, 2)], np.float32).astype(np.float64)
        R = np.array([rng.uniform(-1, 2), rng.uniform(-1, 2), rng.uniform(0.2, 2)], np.float32).astype(np.float64)
        ok, amb, pts = o.validate(T, -1, R, -1, 0)
        res = minimize(lambda p: np.linalg.norm(np.array([p[0], p[1], 0]) - T) + np.linalg.norm(R - np.array([p[0], p[1], 0])),
                       x0=[0.5, 0.5], method="Nelder-Mead", options=dict(xatol=1e-11, fatol=1e-13, maxiter=20000))
        inside = 0 <= res.x[0] <= 1 and 0 <= res.x[1] <= 1
        margin = min(res.x[0], 1 - res.x[0], res.x[1], 1 - res.x[1])
        if abs(margin) > 1e-6:
            assert ok == inside
            n_valid += ok
    assert n_valid > 20


def test_two_parallel_planes_order2_lengths():
    """Floor z=0 and ceiling z=H: second-order unfolded lengths sqrt(rho^2 + (2H +- (a - b))^2)."""
    H = 3.0
    w = _free()
    w.scene = _plane_scene(0.0, 50.0, extra_planes=(H,))
    o = O.Oracle(w)
    T = np.array([0.2, -1.0, 1.1], np.float32).astype(np.float64)
    R = np.array([2.5, 1.7, 2.2], np.float32).astype(np.float64)
    a, b = T[2], R[2]
    rho = np.linalg.norm((R - T)[:2])
    for (f1, f2), dz in [((0, 1), 2 * H + a - b), ((1, 0), 2 * H - a + b)]:
        ok, amb, pts = o.validate(T, -1, R, -1, o.seq_id(f1, f2))
        assert ok and not amb
        L = sum(np.linalg.norm(pts[i + 1] - pts[i]) for i in range(3))
        assert abs(L - math.hypot(rho, dz)) < 1e-12


def test_occlusion_unit_box():
    mb = S._MeshBuilder()
    mb.box((0, 0, 0), (1, 1, 1), 0)
    w = _free()
    w.scene = mb.scene([(3.0, 0.0)])
    o = O.Oracle(w)
    assert o.segment_blocked((-1, 0.5, 0.5), (2, 0.5, 0.5)) == (True, False)
    assert o.segment_blocked((-1, 1.5, 0.5), (2, 1.5, 0.5)) == (False, False)
    assert o.segment_blocked((-1, 0.3, 0.4), (2, 0.6, 0.7)) == (True, False)
    # through two opposite corners only: both hits sit on vertices, so the decision is ambiguous
    assert o.segment_blocked((-1, -1, -1), (2, 2, 2))[1]
    # a segment ending exactly on a face is not blocked by that face when the face is ignored
    assert o.segment_blocked((-1, 0.5, 0.5), (0, 0.5, 0.5), -1, 0) == (False, False)
    # grazing an edge is ambiguous
    blocked, amb = o.segment_blocked((-1, 1.0, 0.5), (2, 1.0, 0.5))
    assert amb


# ------------------------------------------------------------------------------------------------
# T7: reciprocity
# ------------------------------------------------------------------------------------------------
def test_reciprocity_room():
    w = S.room(grid=4)
    rng = np.random.default_rng(3)
    g = np.exp(2j * np.pi * rng.random(w.n_elem))
    a = np.array([3.0, 0.5, 2.5], np.float32)
    b = np.array([4.1, 2.9, 1.2], np.float32)
    w.tx.pos = a
    Ea, _, _ = O.Oracle.evaluate(O.Oracle(w).field(b[None]), g)
    w.tx.pos = b
    Eb, _, _ = O.Oracle.evaluate(O.Oracle(w).field(a[None]), g)
    assert abs(Ea[0]) > 0
    assert abs(Ea[0] - Eb[0]) < 1e-12 * abs(Ea[0])


# ------------------------------------------------------------------------------------------------
# T8: coordinate conventions and the paper's printed numbers
# ------------------------------------------------------------------------------------------------
def test_paper_coordinates():
    g = json.load(open(os.path.join(GOLD, "paper_coordinates.json")))
    u = g["ris_centre"]
    tol = g["printed_precision_m"] / 2 + 1e-3
    t = S.spherical_to_cartesian(u, **{k: g["tx_spherical"][k] for k in ("r",)},
                                 phi_deg=g["tx_spherical"]["phi_deg"], theta_deg=g["tx_spherical"]["theta_deg"])
    r = S.spherical_to_cartesian(u, g["rx_spherical"]["r"], g["rx_spherical"]["phi_deg"], g["rx_spherical"]["theta_deg"])
    assert np.allclose(t, g["tx_cartesian_fig3"], atol=0.05)
    assert np.allclose(r, g["rx_cartesian_fig3"], atol=tol)
    assert abs(r[2] - g["rx_grid_height_m"]) < 1e-3


def test_element_frame():
    """Elements lie at c + a t1 + b t2 (hex grid in the yz plane for the paper's RIS, Fig. 1)."""
    w = S.paper_anechoic()
    o = O.Oracle(w)
    e = o.element_positions()
    assert np.allclose(e[:, 0], 0.0)
    assert np.allclose(e.mean(0), w.ris.center, atol=1e-7)
    assert len(e) == 127


def test_paper_beam_level():
    """Anechoic Table-1 set-up with an on/off configuration that switches on the elements whose
    contribution at the intended Rx points within 90 degrees of a common phase (the best of 64
    offsets): the Rx power must fall in the paper's simulated beam level (Sec. IV-B)."""
    g = json.load(open(os.path.join(GOLD, "paper_levels.json")))
    w = S.paper_anechoic()
    o = O.Oracle(w)
    rx = np.asarray(g["intended_rx"], np.float32)[None]
    f = o.field(rx)
    A = f["A"][0]
    best = -1
    for psi in np.linspace(0, 2 * math.pi, 64, endpoint=False):
        on = np.cos(np.angle(A) - psi) > 0
        gamma = np.where(on, 1.25, 0.0)
        _, P, _ = O.Oracle.evaluate(f, gamma)
        best = max(best, P[0])
    dbm = 10 * math.log10(best) + 30
    assert g["beam_dbm_low"] - g["slack_db"] <= dbm <= g["beam_dbm_high"] + g["slack_db"]


def test_ris_legs_with_one_wall_image_closed_form():
    """RIS at the origin facing +z, one large wall x = 1 (eps 5.3). Each element sees the Tx directly
    and through the wall, and reaches the Rx directly and through the wall; by the image method the
    channel coefficient is the Cartesian sum of four Tang22-type terms with mirrored endpoints and a
    Fresnel factor (Snell form) per bounce (Sec. II-B)."""
    mb = S._MeshBuilder()
    h = 40.0
    mb.quad((1.0, -h, -h), (1.0, h, -h), (1.0, h, h), (1.0, -h, h), 0)
    w = _free()
    w.scene = mb.scene([(5.3, 0.0)])
    w.max_order_tx = 1
    w.max_order_rx = 1
    o = O.Oracle(w)
    R = np.array([0.3, 0.2, 1.5], np.float32).astype(np.float64)
    A = o.field(R.astype(np.float32)[None])["A"][0]
    lam = S.C0 / w.freq_hz
    k = 2 * math.pi / lam
    e = o.element_positions()
    T = w.tx.pos.astype(np.float64)
    mir = lambda p: np.array([2.0 - p[0], p[1], p[2]])
    n2 = math.sqrt(float(np.float32(5.3)))

    def fres(cos_i):
        sin_i = math.sqrt(max(0.0, 1 - cos_i ** 2))
        cos_t = math.sqrt(1 - (sin_i / n2) ** 2)
        return (cos_i - n2 * cos_t) / (cos_i + n2 * cos_t)

    d = float(np.float32(w.ris.dy))
    G = 4 * math.pi * d * d / lam ** 2
    exp = np.zeros(len(e), complex)
    for m in range(len(e)):
        for Ts, tref in ((T, False), (mir(T), True)):
            for Rs, rref in ((R, False), (mir(R), True)):
                rt = np.linalg.norm(e[m] - Ts)
                rr = np.linalg.norm(Rs - e[m])
                cin = (Ts - e[m])[2] / rt
                cout = (Rs - e[m])[2] / rr
                amp = math.sqrt(2 * ETA0) * math.sqrt(G * cin * cout * d * d / (4 * math.pi)) / rt * lam / (4 * math.pi * rr)
                f = 1.0
                if tref:
                    f *= fres(abs((e[m] - Ts)[0]) / rt)
                if rref:
                    f *= fres(abs((Rs - e[m])[0]) / rr)
                exp[m] += amp * f * np.exp(-1j * k * (rt + rr))
    assert np.max(np.abs(A - exp)) < 1e-12 * np.max(np.abs(exp))


def test_two_parallel_planes_order2_field():
    """Order-2 environment paths between floor and ceiling: E0 = LOS + sum over the two sequences of
    R_TE(theta)^2 * Friis(L) with L = sqrt(rho^2 + (2H +- (a - b))^2) and the same incidence angle at
    both bounces (Sec. II-B with the Fresnel factor per bounce); order-1 paths add R * Friis."""
    H = 3.0
    w = _free()
    w.scene = _plane_scene(0.0, 50.0, extra_planes=(H,))
    w.max_order_rx = 2
    w.env_paths = True
    w.ris.center = np.array([0.0, 0.0, 1.0], np.float32)
    w.tx.pos = np.array([0.2, -1.0, 1.1], np.float32)
    o = O.Oracle(w)
    T = w.tx.pos.astype(np.float64)
    R = np.array([2.5, 1.7, 2.2], np.float32).astype(np.float64)
    a, b = T[2], R[2]
    rho = np.linalg.norm((R - T)[:2])
    lam = S.C0 / w.freq_hz
    k = 2 * math.pi / lam
    n2 = math.sqrt(float(np.float32(5.3)))

    def fres(ci):
        si = math.sqrt(1 - ci * ci)
        ct = math.sqrt(1 - (si / n2) ** 2)
        return (ci - n2 * ct) / (ci + n2 * ct)

    def friis(L):
        return math.sqrt(2 * ETA0) * lam / (4 * math.pi * L) * np.exp(-1j * k * L)

    E = friis(np.linalg.norm(R - T))
    for dz, nb in [(a + b, 1), (2 * H - a - b, 1), (2 * H + a - b, 2), (2 * H - a + b, 2)]:
        L = math.hypot(rho, dz)
        E += fres(dz / L) ** nb * friis(L)
    f = o.field(R.astype(np.float32)[None])
    assert abs(f["E0"][0] - E) < 1e-12 * abs(E)


def test_shell_faces_never_block_inside_the_scene_box():
    """The GPU traversal skips shell triangles (planes with the whole scene box on one closed side:
    the room's walls, floor and ceiling and the box bottoms lying in the floor) for segments whose
    two ends lie in the scene box. In the oracle, removing those triangles from the room changes no
    unambiguous occlusion decision of such segments: reflection points on faces to receivers inside
    the room, and segments between random points of the box."""
    w = S.room(grid=4, n_boxes=12)
    V = w.scene.verts.astype(np.float64)
    lo, hi = V.min(0), V.max(0)
    corners = np.array([[(lo, hi)[(c >> k) & 1][k] for k in range(3)] for c in range(8)])
    shell = []
    for t in w.scene.tris:
        p = V[t]
        n = np.cross(p[1] - p[0], p[2] - p[0])
        n /= np.linalg.norm(n)
        sd = corners @ n - n @ p[0]
        shell.append(sd.min() >= -1e-9 or sd.max() <= 1e-9)
    shell = np.array(shell)
    assert shell.sum() == 12 + 2 * 12       # 6 room faces + 12 box bottoms, two triangles each
    w2 = S.room(grid=4, n_boxes=12)
    keep = ~shell
    w2.scene = S.Scene(w.scene.verts, w.scene.tris[keep], w.scene.face_id[keep], w.scene.mat_id[keep], w.scene.mats)
    full, inner = O.Oracle(w), O.Oracle(w2)
    rng = np.random.default_rng(7)
    tris = V[w.scene.tris]
    n_blocked = n_checked = 0
    for _ in range(400):
        if rng.random() < 0.5:                  # a point on a random triangle (its face ignored) to a receiver
            t = rng.integers(len(tris))
            u, v = rng.random(2)
            if u + v > 1:
                u, v = 1 - u, 1 - v
            a = tris[t][0] + u * (tris[t][1] - tris[t][0]) + v * (tris[t][2] - tris[t][0])
            f = int(w.scene.face_id[t])
            b = np.array([rng.uniform(lo[0], hi[0]), rng.uniform(lo[1], hi[1]), 1.2])
            # the reduced scene keeps the face ids of the triangles it keeps
            r_full = full.segment_blocked(a, b, f, -1)
            r_in = inner.segment_blocked(a, b, f, -1)
        else:
            a = lo + rng.random(3) * (hi - lo)
            b = lo + rng.random(3) * (hi - lo)
            r_full = full.segment_blocked(a, b)
            r_in = inner.segment_blocked(a, b)
        if r_full[1] or r_in[1]:
            continue
        n_checked += 1
        n_blocked += r_full[0]
        assert r_full[0] == r_in[0], (a, b)
    assert n_checked > 150 and 0 < n_blocked < n_checked


# ------------------------------------------------------------------------------------------------
# Directional antennas on reflected legs: pattern angles come from the real (un-mirrored) segments
# ------------------------------------------------------------------------------------------------
def _tilted_plane_scene(normal, height, half=40.0, eps=5.3):
    """One large planar quad through (0, 0, height) with unit normal `normal` (a tilted ceiling)."""
    n = np.asarray(normal, np.float64)
    n /= np.linalg.norm(n)
    a = np.cross(n, [1.0, 0.0, 0.0])
    a /= np.linalg.norm(a)
    b = np.cross(n, a)
    c = np.array([0.0, 0.0, height])
    corners = [c - half * a - half * b, c + half * a - half * b, c + half * a + half * b, c - half * a + half * b]
    mb = S._MeshBuilder()
    mb.quad(*[tuple(p) for p in corners], 0)
    return mb.scene([(eps, 0.0)])


def _tilted_ceiling_case():
    w = _free(tx=(0.4, -1.5, 1.0), tx_pat=S.PATTERN_COS_POW, tx_gain=10.0, rx_pat=S.PATTERN_MONOPOLE_QW,
              tx_orient=S.orient_towards((0.4, -1.5, 1.0), (0.4, 1.0, 1.25)),
              rx_orient=S.orient_towards((0.0, 0.0, 0.0), (0.3, 0.4, 1.0)))
    w.scene = _tilted_plane_scene((0.15, -0.25, -1.0), 2.4)
    w.max_order_tx = w.max_order_rx = 1
    w.env_paths = True
    return w


def _tilted_ceiling_expected(w, R, wrong=None):
    """Closed form of the tilted-ceiling case built from explicit reflection points: the channel row
    A[m] (four leg pairings per element) and E0 (LOS plus the ceiling path), with the Tx pattern,
    both element patterns and the Rx pattern evaluated on the real segment next to each antenna or
    element. Fresnel TE in its Snell form per bounce (Sec. II-B; Eqs. 4, 7, 8).
    `wrong` names one angle to take from a plausible misreading instead, to show the pin detects it:
    "ft" / "fout" - the departure direction at the Tx / at the element taken on the straight line from
    the source's image to the destination; "fin" / "fr" - the arrival direction at the element / at
    the Rx taken on the straight line between the leg's two ends, as if there were no bounce."""
    V = w.scene.verts.astype(np.float64)
    tri = V[w.scene.tris[0]]
    nw = np.cross(tri[1] - tri[0], tri[2] - tri[0])
    nw /= np.linalg.norm(nw)
    dw = nw @ tri[0]
    mirror = lambda p: p - 2 * (p @ nw - dw) * nw
    hit = lambda a, b: a + (dw - a @ nw) / ((b - a) @ nw) * (b - a)      # line a->b meets the plane
    unit = lambda v: v / np.linalg.norm(v)
    lam = S.C0 / w.freq_hz
    k = 2 * math.pi / lam
    n2 = math.sqrt(float(np.float32(5.3)))

    def fres(cos_i):
        sin_i = math.sqrt(max(0.0, 1 - cos_i ** 2))
        cos_t = math.sqrt(1 - (sin_i / n2) ** 2)
        return (cos_i - n2 * cos_t) / (cos_i + n2 * cos_t)

    def leg(src, dst, reflected, wrong_dep=False, wrong_back=False):
        """(length, unit direction leaving src, unit direction from dst back along the last segment,
        Fresnel factor)"""
        if not reflected:
            return np.linalg.norm(dst - src), unit(dst - src), unit(src - dst), 1.0
        img = mirror(src)
        P = hit(img, dst)
        L = np.linalg.norm(P - src) + np.linalg.norm(dst - P)
        f = fres(abs(unit(P - src) @ nw))
        dep = unit(dst - img) if wrong_dep else unit(P - src)
        back = unit(src - dst) if wrong_back else unit(P - dst)
        return L, dep, back, f

    def monopole(c):
        return (math.cos(math.pi / 2 * c) / math.sqrt(1 - c * c)) ** 2

    T = w.tx.pos.astype(np.float64)
    zt = w.tx.orient[2].astype(np.float64)
    zt /= np.linalg.norm(zt)
    zr = w.rx.orient[2].astype(np.float64)
    zr /= np.linalg.norm(zr)
    Gt = float(np.float32(w.tx.gain_lin))
    Ft = lambda d: max(d @ zt, 0.0) ** (Gt / 2 - 1)
    Fr = lambda d: monopole(d @ zr)
    nr = np.array([0.0, 0.0, 1.0])                      # RIS normal t1 x t2
    d = float(np.float32(w.ris.dy))
    G = 4 * math.pi * d * d / lam ** 2
    e = O.Oracle(w).element_positions()
    A = np.zeros(len(e), complex)
    for m in range(len(e)):
        for tref in (False, True):
            Lt, dep_t, back_t, ft = leg(T, e[m], tref, wrong == "ft", wrong == "fin")
            for rref in (False, True):
                Lr, dep_r, back_r, fr = leg(e[m], R, rref, wrong == "fout", wrong == "fr")
                amp = math.sqrt(2 * ETA0 * Gt * Ft(dep_t)) \
                    * math.sqrt(G * max(back_t @ nr, 0) * max(dep_r @ nr, 0) * d * d / (4 * math.pi)) / Lt \
                    * math.sqrt(Fr(back_r)) * lam / (4 * math.pi * Lr)
                A[m] += amp * ft * fr * np.exp(-1j * k * (Lt + Lr))
    E0 = 0j
    for ref in (False, True):
        L, dep, back, f = leg(T, R, ref, wrong == "ft", wrong == "fr")
        E0 += math.sqrt(2 * ETA0 * Gt * Ft(dep)) * math.sqrt(Fr(back)) * lam / (4 * math.pi * L) * f \
            * np.exp(-1j * k * L)
    return A, E0


def test_reflected_legs_directional_patterns_tilted_ceiling():
    """Horn Tx (cos^(Gt/2-1), Sec. III-B) and a tilted quarter-wave monopole Rx under one large tilted
    ceiling: every element sees the Tx directly and through the ceiling and reaches the Rx directly and
    through it. The oracle's channel row and E0 equal the closed form whose four pattern factors (Ft,
    F_in, F_out, Fr) are evaluated on the explicit, un-mirrored segments (reading 7). Taking any one of
    those angles from a misreading (the image line at a departure, the end-to-end line at an arrival)
    changes the closed form far beyond the tolerance, so each factor is pinned."""
    w = _tilted_ceiling_case()
    o = O.Oracle(w)
    for R in ([0.6, 0.8, 1.2], [-0.9, 0.3, 0.7], [0.2, -0.6, 1.6]):
        R = np.asarray(R, np.float32).astype(np.float64)
        f = o.field(R.astype(np.float32)[None])
        assert not f["amb"][0]
        A_exp, E0_exp = _tilted_ceiling_expected(w, R)
        assert np.max(np.abs(f["A"][0] - A_exp)) < 1e-11 * np.max(np.abs(A_exp))
        assert abs(f["E0"][0] - E0_exp) < 1e-11 * abs(E0_exp)
        for wrong in ("ft", "fin", "fout", "fr"):
            A_bad, E0_bad = _tilted_ceiling_expected(w, R, wrong)
            dA = np.max(np.abs(A_bad - A_exp)) / np.max(np.abs(A_exp))
            assert dA > 1e-3, (wrong, dA)


def test_ambiguity_only_without_a_robust_failure():
    """A validity decision is ambiguous only when some condition sits within the tolerance band of
    flipping and no condition fails robustly (Sec. II-B conditions: reflection point in its face,
    neighbours on the same side, segments unblocked)."""
    mb = S._MeshBuilder()
    mb.quad((0, -10, 0), (0, -10, 3), (0, 10, 3), (0, 10, 0), 0)          # wall x = 0, face 0
    mb.quad((10, 1, 0), (11, 1, 0), (11, 1, 3), (10, 1, 3), 0)            # small plate y = 1, face 1
    mb.quad((-5, 0, -2), (5, 0, -2), (5, 2, -2), (-5, 2, -2), 0)          # floor patch z = -2, y in [0, 2]
    w = _free()
    w.scene = mb.scene([(5.3, 0.0)])
    o = O.Oracle(w)
    # source on the wall, sequence (plate, wall): the second bounce lies on the source's own plane
    # (a boundary case of the same-side test), but the first reflection point is 10 m outside the
    # plate, so the sequence is rejected robustly
    ok, amb, _ = o.validate((0, 3, 1.5), 0, (5, 5, 1.2), -1, o.seq_id(1, 0))
    assert not ok and not amb
    # a reflection point exactly on the edge y = 0 of the floor patch: marginal, nothing fails robustly
    ok, amb, pts = o.validate((1, 0.5, 1), -1, (1, -0.5, 1), -1, 2)
    assert amb and abs(pts[1][1]) < 1e-12
    # well inside: robust
    ok, amb, _ = o.validate((1, 1.5, 1), -1, (1, 0.5, 1), -1, 2)
    assert ok and not amb


def test_cir_taps_one_wall_closed_form():
    """Channel impulse response of the one-wall case: exactly four RIS taps (direct / wall on each
    leg), each the closed-form sum of its leg pairing over the elements (with an arbitrary
    configuration), delayed by the travel time through the RIS centre between the image-method end
    points (|T_p - c| + |R_q - c|) / c0, and the taps plus E0 give E (Sec. II-B, Eq. 9)."""
    mb = S._MeshBuilder()
    h = 40.0
    mb.quad((1.0, -h, -h), (1.0, h, -h), (1.0, h, h), (1.0, -h, h), 0)
    w = _free()
    w.scene = mb.scene([(5.3, 0.0)])
    w.max_order_tx = w.max_order_rx = 1
    o = O.Oracle(w)
    R = np.array([0.3, 0.2, 1.5], np.float32).astype(np.float64)
    rng = np.random.default_rng(12)
    gam = 1.25 * np.exp(2j * np.pi * rng.random(w.n_elem))
    taps = o.cir(R.astype(np.float32)[None], gam)[0]
    assert list(taps["q"]) == [-1, -1, 0, 0] and list(taps["p"]) == [-1, 0, -1, 0]
    lam = S.C0 / w.freq_hz
    k = 2 * math.pi / lam
    e = o.element_positions()
    T = w.tx.pos.astype(np.float64)
    c = w.ris.center.astype(np.float64)
    mir = lambda p: np.array([2.0 - p[0], p[1], p[2]])
    n2 = math.sqrt(float(np.float32(5.3)))

    def fres(cos_i):
        sin_i = math.sqrt(max(0.0, 1 - cos_i ** 2))
        cos_t = math.sqrt(1 - (sin_i / n2) ** 2)
        return (cos_i - n2 * cos_t) / (cos_i + n2 * cos_t)

    d = float(np.float32(w.ris.dy))
    G = 4 * math.pi * d * d / lam ** 2
    for j, (rref, tref) in enumerate([(False, False), (False, True), (True, False), (True, True)]):
        Ts = mir(T) if tref else T
        Rs = mir(R) if rref else R
        a = 0j
        for m in range(len(e)):
            rt = np.linalg.norm(e[m] - Ts)
            rr = np.linalg.norm(Rs - e[m])
            cin = (Ts - e[m])[2] / rt
            cout = (Rs - e[m])[2] / rr
            amp = math.sqrt(2 * ETA0) * math.sqrt(G * cin * cout * d * d / (4 * math.pi)) / rt * lam / (4 * math.pi * rr)
            f = (fres(abs((e[m] - Ts)[0]) / rt) if tref else 1.0) * (fres(abs((Rs - e[m])[0]) / rr) if rref else 1.0)
            a += gam[m] * amp * f * np.exp(-1j * k * (rt + rr))
        assert abs(taps["amp"][j] - a) < 1e-12 * abs(a)
        tau = (np.linalg.norm(Ts - c) + np.linalg.norm(Rs - c)) / S.C0
        assert abs(taps["delay"][j] - tau) < 1e-15 * tau + 1e-21
    f = o.field(R.astype(np.float32)[None])
    E, _, _ = O.Oracle.evaluate(f, gam)
    assert abs(taps["amp"].sum() + f["E0"][0] - E[0]) < 1e-13 * abs(E[0])


def test_reflective_closeup_fading_period():
    """The paper's reflective set-up (Sec. III, Table 2): along x through the close-up region of Fig. 5
    the received power fades with a dominant period of about lambda/2 (Sec. IV-B)."""
    g = json.load(open(os.path.join(GOLD, "paper_closeup_fading.json")))
    w = S.paper_reflective(closeup=True)
    o = O.Oracle(w)
    lam = S.C0 / w.freq_hz
    xs = np.arange(g["x_range_m"][0], g["x_range_m"][1] + 1e-9, g["step_m"])
    yc = 0.5 * sum(g["y_range_m"])
    line = np.stack([xs, np.full(len(xs), yc), np.full(len(xs), g["rx_height_m"])], 1).astype(np.float32)
    f = o.field(line)
    _, P, _ = O.Oracle.evaluate(f, w.gammas[0])
    spec = np.abs(np.fft.rfft(P - P.mean()))
    freqs = np.fft.rfftfreq(len(P), g["step_m"])
    period = 1.0 / freqs[1 + np.argmax(spec[1:])]
    lo, hi = g["accepted_period_over_lambda"]
    assert lo * lam <= period <= hi * lam, period / lam
    # the interference is deep: a range of well over 10 dB along the line
    assert 10 * np.log10(P.max() / P.min()) > 10


@pytest.mark.parametrize("leg", ["rx", "tx"])
def test_strict_element_validation_finite_wall(leg):
    """Strict mode (each element's reflected legs validated at the element itself, instead of once at
    the RIS centre as in Sec. II-B): a finite wall x = 1 whose top edge splits the elements' own
    reflection points on one leg. Each element's validity comes from brute-force Fermat minimisation
    over the wall plane; the strict channel row equals the closed form over the valid pairings per
    element, the centre-validated row the closed form with the centre's validity for every element."""
    lam = S.C0 / 28e9
    k0 = 2 * math.pi / lam
    T = np.array([0.0, -1.5, 2.0], np.float32).astype(np.float64)
    R = np.array([0.3, 0.2, 1.5], np.float32).astype(np.float64)
    base = _free()
    e = O.Oracle(base).element_positions()
    c = base.ris.center.astype(np.float64)

    def fermat(a, b):
        f = lambda p: np.linalg.norm(np.array([1.0, p[0], p[1]]) - a) + np.linalg.norm(b - np.array([1.0, p[0], p[1]]))
        x0 = [0.5 * (a[1] + b[1]), 0.5 * (a[2] + b[2])]
        res = minimize(f, x0=x0, method="Nelder-Mead", options=dict(xatol=1e-12, fatol=1e-14, maxiter=40000))
        return res.x
    end = R if leg == "rx" else T
    zs = np.array([fermat(em, end)[1] for em in e])
    zc = fermat(c, end)[1]
    rows = np.unique(np.round(zs, 5))                   # elements of one hex row share a height
    mid = len(rows) // 2
    z1 = float(np.float32(0.5 * (rows[mid - 1] + rows[mid])))   # edge between two rows
    assert np.min(np.abs(zs - z1)) > 1e-4
    mb = S._MeshBuilder()
    mb.quad((1.0, -40.0, -40.0), (1.0, 40.0, -40.0), (1.0, 40.0, z1), (1.0, -40.0, z1), 0)
    w = _free()
    w.scene = mb.scene([(5.3, 0.0)])
    w.max_order_tx = w.max_order_rx = 1
    other = T if leg == "rx" else R
    other_in = [fermat(em, other)[1] <= z1 for em in e]      # the other leg's validity per element

    mir = lambda p: np.array([2.0 - p[0], p[1], p[2]])
    n2 = math.sqrt(float(np.float32(5.3)))

    def fres(cos_i):
        sin_i = math.sqrt(max(0.0, 1 - cos_i ** 2))
        cos_t = math.sqrt(1 - (sin_i / n2) ** 2)
        return (cos_i - n2 * cos_t) / (cos_i + n2 * cos_t)

    d = float(np.float32(w.ris.dy))
    G = 4 * math.pi * d * d / lam ** 2

    def row(valid_leg, valid_other):
        out = np.zeros(len(e), complex)
        for m in range(len(e)):
            tx_ok = valid_leg[m] if leg == "tx" else valid_other[m]
            rx_ok = valid_leg[m] if leg == "rx" else valid_other[m]
            for Ts, tref in ((T, False), (mir(T), True)):
                if tref and not tx_ok:
                    continue
                for Rs, rref in ((R, False), (mir(R), True)):
                    if rref and not rx_ok:
                        continue
                    rt = np.linalg.norm(e[m] - Ts)
                    rr = np.linalg.norm(Rs - e[m])
                    cin, cout = (Ts - e[m])[2] / rt, (Rs - e[m])[2] / rr
                    amp = math.sqrt(2 * ETA0) * math.sqrt(G * cin * cout * d * d / (4 * math.pi)) / rt * lam / (4 * math.pi * rr)
                    f = (fres(abs((e[m] - Ts)[0]) / rt) if tref else 1.0) * (fres(abs((Rs - e[m])[0]) / rr) if rref else 1.0)
                    out[m] += amp * f * np.exp(-1j * k0 * (rt + rr))
        return out

    strict_valid = zs <= z1
    A_strict = O.Oracle(w, strict=True).field(R.astype(np.float32)[None])
    A_centre = O.Oracle(w).field(R.astype(np.float32)[None])
    assert not A_strict["amb"][0] and not A_centre["amb"][0]
    exp_s = row(strict_valid, other_in)
    centre_other = [fermat(c, other)[1] <= z1] * len(e)
    exp_c = row([zc <= z1] * len(e), centre_other)
    scale = np.max(np.abs(exp_s))
    assert np.max(np.abs(A_strict["A"][0] - exp_s)) < 1e-11 * scale
    assert np.max(np.abs(A_centre["A"][0] - exp_c)) < 1e-11 * scale
    assert 0 < strict_valid.sum() < len(e)
    assert np.max(np.abs(exp_s - exp_c)) > 1e-3 * scale
