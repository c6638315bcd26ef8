"""Pins of the oracle's vector (polarisation) mode against results fixed independently of it: the
scalar model it must reduce to when every field is TE and co-polarised, image theory over a
perfectly conducting plane for dipoles of any orientation, Brewster's angle and the Snell-form TE
coefficient, the closed-form factors of the RIS re-radiation (cos(theta) loss of an anomalous beam,
cross-polar zeros, a PEC mirror at Gamma = -1) and reciprocity under exchange of Tx and Rx."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2402_13034_gb300 import scenarios as S
from tests.test_oracle_pins import _free, _plane_scene

ETA0 = 120 * math.pi


def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def _pol(a, k):
    """unit(P(k) a): an antenna's field direction for propagation direction k."""
    p = np.asarray(a, np.float64) - np.dot(a, k) * k
    n = np.linalg.norm(p)
    return p / n if n > 1e-12 else np.zeros(3)


def _amp_free(w, L):
    """Eq. 4 + Eq. 8 amplitude of a path of unfolded length L between isotropic antennas."""
    lam = S.C0 / w.freq_hz
    return (math.sqrt(2 * ETA0 * float(np.float32(w.tx.power_w)) * float(np.float32(w.tx.gain_lin)))
            * math.sqrt(float(np.float32(w.rx.gain_lin))) * lam / (4 * math.pi * L)
            * np.exp(-1j * 2 * math.pi * L / lam))


# ------------------------------------------------------------------------------------------------
# V1: every field TE and co-polarised -> the scalar model (TE Fresnel)
# ------------------------------------------------------------------------------------------------
def _horizontal_world():
    """Vertical walls only, Tx, RIS row and receivers at one height, antennas polarised along z: every
    ray is horizontal, so every bounce is TE, the RIS keeps the (tangential) z field and every
    projection onto a wavefront keeps z."""
    freq = 28e9
    lam = S.C0 / freq
    mb = S._MeshBuilder()
    h = 20.0
    mb.quad((-4.0, -1.0, -h), (-4.0, 8.0, -h), (-4.0, 8.0, h), (-4.0, -1.0, h), 0)   # x = -4
    mb.quad((4.0, 8.0, -h), (4.0, -1.0, -h), (4.0, -1.0, h), (4.0, 8.0, h), 1)       # x = +4
    mb.quad((4.0, 6.0, -h), (-4.0, 6.0, -h), (-4.0, 6.0, h), (4.0, 6.0, h), 0)       # y = 6
    scene = mb.scene([(5.3, 0.4), (3.1, 0.0)])
    uv = np.stack([np.arange(-4, 5) * lam / 2, np.zeros(9)], 1).astype(np.float32)
    ris = S.RIS(uv, np.array([0.0, 0.0, 1.5], np.float32), np.array([-1, 0, 0], np.float32),
                np.array([0, 0, 1], np.float32), lam / 2, lam / 2, 0.0, -1)
    z = np.array([0, 0, 1], np.float32)
    tx = S.Antenna(np.array([-1.5, 3.0, 1.5], np.float32), S.identity_orient(), 1.0, 1.0, S.PATTERN_ISO, pol=z)
    rx = S.Antenna(np.zeros(3, np.float32), S.identity_orient(), 1.0, 1.0, S.PATTERN_ISO, pol=z)
    g = S.linspace_grid(-3.0, 3.0, 5, 0.5, 5.0, 4, 1.5)
    return S.Workload("horizontal", freq, scene, ris, tx, rx, g, np.ones((1, 9), np.complex64), 2, 2, True)


def test_vector_reduces_to_scalar_te_when_copolarised():
    w = _horizontal_world()
    fs = O.Oracle(w).field(w.rx_xyz)
    fv = O.Oracle(w, vector=True).field_vec(w.rx_xyz)
    assert fs["SA"].sum() > 0 and (fs["SA"] > 0).sum(1).min() > 0
    tol = 1e-12
    assert np.all(np.abs(fv["E0"] - fs["E0"]) <= tol * fs["S0"])
    assert np.all(np.abs(fv["A"] - fs["A"]) <= tol * fs["SA"] + 1e-300)
    # the field vectors lie along z and carry the received values
    assert np.all(np.abs(fv["E03"][:, 2] - fs["E0"]) <= tol * fs["S0"])
    assert np.all(np.abs(fv["A3"][..., 2] - fs["A"]) <= tol * fs["SA"] + 1e-300)
    assert np.all(np.abs(fv["A3"][..., :2]) <= tol * fs["SA"][..., None] + 1e-300)
    # several paths per receiver (environment and RIS legs reflected twice)
    nz = np.count_nonzero(np.abs(fv["A"]) > 0)
    assert nz == fv["A"].size


# ------------------------------------------------------------------------------------------------
# V2: image theory over a perfect conductor (sigma -> infinity: R_TE -> -1, R_TM -> +1)
# ------------------------------------------------------------------------------------------------
def _ground_world(tx, a_t, a_r, eps=1.0, sigma=1e12):
    w = _free(tx=tx)
    w.scene = _plane_scene(z=0.0, eps=eps, sigma=sigma)
    w.ris.center = np.array([0.0, 60.0, 5.0], np.float32)   # far away: only E0 is checked
    w.env_paths = True
    w.max_order_rx = 1                          # environment paths go up to the Rx-leg order
    w.tx.pol = np.asarray(a_t, np.float32)
    w.rx.pol = np.asarray(a_r, np.float32)
    return w


@pytest.mark.parametrize("a_t,a_r", [((0, 0, 1), (0, 0, 1)), ((1, 0, 0), (1, 0, 0)), ((0, 1, 0), (0.3, 0.8, 0.2)),
                                     ((0.6, -0.3, 0.7), (-0.2, 0.5, 0.8))])
def test_vector_pec_ground_image_dipole(a_t, a_r):
    """Over a PEC plane the reflected field is that of the image dipole: mirrored position, axis
    2 (a.z) z - a (a horizontal dipole's image is reversed, a vertical one's is not)."""
    T = np.array([0.2, -0.4, 1.3], np.float32)
    w = _ground_world(T, a_t, a_r)
    rng = np.random.default_rng(7)
    R = np.stack([rng.uniform(-3, 3, 6), rng.uniform(-3, 3, 6), rng.uniform(0.3, 2.5, 6)], 1).astype(np.float32)
    f = O.Oracle(w, vector=True).field_vec(R)
    at = _unit(np.asarray(a_t, np.float32))
    ar = _unit(np.asarray(a_r, np.float32))
    z = np.array([0.0, 0.0, 1.0])
    a_img = 2 * np.dot(at, z) * z - at
    T64 = T.astype(np.float64)
    Ti = T64 * np.array([1, 1, -1])
    for i, r in enumerate(R.astype(np.float64)):
        d = np.linalg.norm(r - T64)
        k = (r - T64) / d
        L = np.linalg.norm(r - Ti)
        ki = (r - Ti) / L
        v_los = _amp_free(w, d) * _pol(at, k)
        v_img = _amp_free(w, L) * _pol(a_img, ki)
        E3 = v_los + v_img
        E = np.dot(v_los, _pol(ar, k)) + np.dot(v_img, _pol(ar, ki))
        scale = abs(_amp_free(w, d)) + abs(_amp_free(w, L))
        assert abs(f["E0"][i] - E) <= 2e-5 * scale, (i, f["E0"][i], E)
        assert np.max(np.abs(f["E03"][i] - E3)) <= 2e-5 * scale


# ------------------------------------------------------------------------------------------------
# V3: Brewster's angle (TM reflection vanishes) and the Snell-form TE coefficient at the same angle
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("pol,R_expected", [((0, 0, 1), 0.0), ((0, 1, 0), -0.6)])
def test_vector_brewster_angle(pol, R_expected):
    """eps_r = 4: tan(theta_B) = 2, so Tx (0, 0, 1) and Rx (4, 0, 1) meet the plane z = 0 at Brewster's
    angle. A vertical dipole radiates TM in that plane: no reflection. A y dipole is TE:
    R_TE = (cos - sqrt(eps - sin^2)) / (cos + sqrt(eps - sin^2)) = -0.6 there."""
    w = _ground_world(np.array([0.0, 0.0, 1.0], np.float32), pol, pol, eps=4.0, sigma=0.0)
    R = np.array([[4.0, 0.0, 1.0]], np.float32)
    f = O.Oracle(w, vector=True).field_vec(R)
    d = 4.0
    L = math.sqrt(16.0 + 4.0)
    los = _amp_free(w, d)                        # LOS along x: both axes transverse, co-polarised
    env = f["E0"][0] - los
    assert abs(env - R_expected * _amp_free(w, L)) <= 1e-12 * abs(_amp_free(w, L))


# ------------------------------------------------------------------------------------------------
# V4: the RIS re-radiation in closed form (one element at the origin, normal +z)
# ------------------------------------------------------------------------------------------------
def _one_element(tx, a_t, a_r):
    w = _free(tx=tx, layout=np.zeros((1, 2), np.float32))
    w.tx.pol = np.asarray(a_t, np.float32)
    w.rx.pol = np.asarray(a_r, np.float32)
    return w


@pytest.mark.parametrize("theta_deg", [0.0, 20.0, 50.0])
def test_vector_ris_anomalous_beam_factors(theta_deg):
    """Normal incidence (Tx on the normal), receiver at theta in the xz plane: an x-polarised field
    keeps its tangential x component, which the outgoing wavefront reduces by cos(theta); a y field is
    transverse to every outgoing direction of the plane (factor 1); crossed axes receive nothing."""
    th = math.radians(theta_deg)
    R = np.array([[2 * math.sin(th), 0.0, 2 * math.cos(th)]], np.float32)
    k_out = _unit(R[0].astype(np.float64))
    ref = O.Oracle(_one_element((0.0, 0.0, 2.0), (1, 0, 0), (1, 0, 0))).field(R)["A"][0, 0]
    assert abs(ref) > 0
    cos_t = math.sqrt(1.0 - k_out[0] ** 2)            # of the receiver's FP32 position
    cases = [((1, 0, 0), (1, 0, 0), cos_t), ((0, 1, 0), (0, 1, 0), 1.0), ((1, 0, 0), (0, 1, 0), 0.0),
             ((0, 1, 0), (1, 0, 0), 0.0)]
    for a_t, a_r, factor in cases:
        f = O.Oracle(_one_element((0.0, 0.0, 2.0), a_t, a_r), vector=True).field_vec(R)
        assert abs(f["A"][0, 0] - factor * ref) <= 1e-12 * abs(ref), (a_t, a_r)
    # the field vector of the x-polarised case: P(k_out) x, unnormalised
    f = O.Oracle(_one_element((0.0, 0.0, 2.0), (1, 0, 0), (1, 0, 0)), vector=True).field_vec(R)
    x = np.array([1.0, 0.0, 0.0])
    assert np.max(np.abs(f["A3"][0, 0] - ref * (x - np.dot(x, k_out) * k_out))) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("alpha_deg", [15.0, 40.0])
def test_vector_ris_specular_is_a_mirror(alpha_deg):
    """At the specular direction the re-radiated field is the incident one with its normal component
    reversed: a y (TE) dipole is received with factor +1 and a z (TM) dipole pair with factor -1, so
    Gamma = -1 reproduces a perfect conductor's image dipoles (horizontal reversed, vertical kept)."""
    al = math.radians(alpha_deg)
    T = (-2 * math.sin(al), 0.0, 2 * math.cos(al))
    R = np.array([[2 * math.sin(al), 0.0, 2 * math.cos(al)]], np.float32)
    ref = O.Oracle(_one_element(T, (0, 1, 0), (0, 1, 0))).field(R)["A"][0, 0]
    for a, factor in [((0, 1, 0), 1.0), ((0, 0, 1), -1.0)]:
        f = O.Oracle(_one_element(T, a, a), vector=True).field_vec(R)
        assert abs(f["A"][0, 0] - factor * ref) <= 1e-6 * abs(ref), (a, f["A"][0, 0] / ref)


# ------------------------------------------------------------------------------------------------
# V5: reciprocity (Tx and Rx exchanged together with their polarisation axes)
# ------------------------------------------------------------------------------------------------
def test_vector_reciprocity_room():
    w = S.room(grid=4)
    rng = np.random.default_rng(11)
    g = np.exp(2j * np.pi * rng.random(w.n_elem))
    a = np.array([3.0, 0.5, 2.5], np.float32)
    b = np.array([4.1, 2.9, 1.2], np.float32)
    pa = np.array([0.3, -0.5, 0.8], np.float32)
    pb = np.array([0.9, 0.1, -0.4], np.float32)
    w.tx.pos, w.tx.pol, w.rx.pol = a, pa, pb
    fa = O.Oracle(w, vector=True).field_vec(b[None])
    Ea = O.Oracle.evaluate(fa, g)[0]
    w.tx.pos, w.tx.pol, w.rx.pol = b, pb, pa
    Eb = O.Oracle.evaluate(O.Oracle(w, vector=True).field_vec(a[None]), g)[0]
    assert abs(Ea[0]) > 0 and (np.abs(fa["A"]) > 0).sum() > 0
    assert abs(Ea[0] - Eb[0]) < 1e-12 * abs(Ea[0])
    # polarisation matters here: the vector field differs from the scalar one
    Es = O.Oracle.evaluate(O.Oracle(w).field(a[None]), g)[0]
    assert abs(Es[0] - Eb[0]) > 1e-3 * abs(Es[0])
