"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Path and visibility sets must agree bit for bit on every decision the oracle does not flag as
ambiguous, and ambiguous decisions must be at most 1e-5 of all decisions; fields must agree within
5e-5 of the incoherent magnitude S(r) on every receiver whose path set equals the oracle's, and
power within 1e-4 relative and phase within 1e-3 rad where |E| >= 0.05 S(r); channel-matrix entries
within 5e-5 of their own incoherent sum.
"""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2402_13034_gb300 import scenarios as S
from tests.helpers import compare_fields, compare_pathsets, oracle_parity, run_gpu, subset_paths

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2402_13034_gb300 import build as B
    B.build()


def _oracle_all(w, rx_idx=None, gammas=None):
    o = O.Oracle(w)
    rx = w.rx_xyz if rx_idx is None else w.rx_xyz[rx_idx]
    fld = o.field(rx)
    g = w.gammas if gammas is None else gammas
    E, P, Sx = O.Oracle.evaluate(fld, g)
    return o, fld, E, P, Sx


def test_free_space_full_grid():
    w = S.free_space()
    g = run_gpu(w)
    _, fld, E, P, Sx = _oracle_all(w)
    st = compare_fields(g["E"], g["P"], E, P, Sx)
    assert st["strong_frac"] > 0.5
    # the focused configuration peaks at the focus point (grid centre region)
    assert g["paths"]["stats"].units == w.n_rx * w.n_elem


def test_free_space_single_rx_and_ragged():
    w = S.free_space(grid=5)                 # 25 receivers: not a multiple of a warp or a block
    g = run_gpu(w)
    _, fld, E, P, Sx = _oracle_all(w)
    compare_fields(g["E"], g["P"], E, P, Sx)
    w1 = S.free_space(grid=1)
    w1.rx_xyz = np.array([[0.3, -0.2, 1.5]], np.float32)
    g1 = run_gpu(w1)
    _, _, E1, P1, S1 = _oracle_all(w1)
    compare_fields(g1["E"], g1["P"], E1, P1, S1)


def test_single_element_and_behind_ris():
    w = S.free_space(grid=4)
    w.ris.elem_uv = w.ris.elem_uv[:1]
    w.gammas = w.gammas[:, :1]
    w.rx_xyz = np.concatenate([w.rx_xyz, [[0.1, 0.2, -1.0]]]).astype(np.float32)   # behind the RIS
    g = run_gpu(w)
    _, fld, E, P, Sx = _oracle_all(w)
    compare_fields(g["E"], g["P"], E, P, Sx)


def test_paper_patterns_anechoic():
    """Horn Tx (cos^(Gt/2-1)) aimed at the RIS and monopole Rx: Table 1 set-up (Sec. III)."""
    w = S.paper_anechoic(grid_step=0.05)
    rng = np.random.default_rng(7)
    gam = (1.25 * (rng.random((3, w.n_elem)) > 0.5)).astype(np.complex64)
    g = run_gpu(w, gammas=gam)
    _, fld, E, P, Sx = _oracle_all(w, gammas=gam)
    compare_fields(g["E"], g["P"], E, P, Sx)


@pytest.mark.parametrize("grid", [12, 24])
def test_room_pathsets_bit_exact(grid):
    w = S.room(grid=grid)
    g = run_gpu(w)
    st, *_ = oracle_parity(w, g)
    # a room of this kind has many reflected paths per receiver
    n_ref = np.array([len(s) for s in g["paths"]["seqs"]])
    assert n_ref.max() > 5


@pytest.mark.parametrize("side", [32, 64])
def test_tiled_direct_legs(side, monkeypatch):
    """Square RIS of 1,024 and 4,096 elements in the room with its boxes, so that many receivers see
    part of the aperture: element -> receiver visibility decided through pyramids over spatial tiles
    of 32 elements (rays only for undecided tiles) equals one ray per element (RISRT_TILES=0) bit for
    bit, and the path sets and fields match the oracle."""
    w = S.room(grid=12, square_side=side)
    g = run_gpu(w)
    monkeypatch.setenv("RISRT_TILES", "0")
    g0 = run_gpu(w)
    monkeypatch.delenv("RISRT_TILES")
    assert np.array_equal(g["paths"]["vis"], g0["paths"]["vis"])
    assert np.array_equal(g["P"], g0["P"])
    seen = np.array([sum(bin(int(x)).count("1") for x in row) for row in g["paths"]["vis"]])
    assert np.any((seen > 0) & (seen < side * side))     # partly shadowed receivers exist
    oracle_parity(w, g)


def test_tiled_direct_legs_at_scale(monkeypatch):
    """200x200 receivers against a 4,096-element RIS: many undecided tiles, rays whose FP32 walk meets
    triangles too close to call (settled in FP64 after the walk) — the visibility bits equal one ray
    per element (RISRT_TILES=0), whose settlements run in the walk."""
    import torch
    from paper_2402_13034_gb300 import risrt as R
    w = S.room(grid=200, square_side=64)
    ctx = R.Context(0, torch.cuda.current_stream().cuda_stream)
    scene, ris, rx = R.upload_workload(ctx, w)
    bits = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("RISRT_TILES", mode)
        ps = ctx.trace_paths(scene, ris, rx, w.freq_hz, w.max_order_tx, w.max_order_rx, R.flags_of(w))
        bits[mode] = ps.export()["vis"]
        ps.close()
    monkeypatch.delenv("RISRT_TILES")
    assert np.array_equal(bits["1"], bits["0"])
    seen = np.unpackbits(bits["1"].view(np.uint8), axis=1).sum(axis=1)
    assert np.any((seen > 0) & (seen < 4096))


def test_two_level_culling_same_paths(monkeypatch):
    """The room at 600x600 receivers (352 super-patches of 1,024 receivers, so the sequences are culled
    for groups of 16 super-patches first): path sets and fields equal those of culling every
    super-patch against every sequence (RISRT_CULL_LEVELS=1)."""
    w = S.room(grid=600)
    g = run_gpu(w)
    monkeypatch.setenv("RISRT_CULL_LEVELS", "1")
    g1 = run_gpu(w)
    monkeypatch.delenv("RISRT_CULL_LEVELS")
    for k in ("los", "vis", "tx_seqs", "tx_vis"):
        assert np.array_equal(g["paths"][k], g1["paths"][k]), k
    for k in ("seqs", "env"):
        assert all(np.array_equal(a, b) for a, b in zip(g["paths"][k], g1["paths"][k], strict=True)), k
    assert np.array_equal(g["P"], g1["P"])


def test_room_field_parity():
    w = S.room(grid=16)
    g = run_gpu(w, want_A=True)
    oracle_parity(w, g, check_A=True)


def test_room_directional_antennas():
    """The room with the paper's horn Tx (cos^(Gt/2-1), Gt 10 dB) aimed at the RIS and a quarter-wave
    monopole Rx whose axis is tilted away from the vertical, so that mirroring across the walls,
    floor and ceiling changes every pattern angle of a reflected leg (Sec. III-B; Eqs. 4, 7, 8):
    path sets, fields, and A and E0 element by element."""
    w = S.room(grid=16, n_boxes=20)
    w.tx = S.Antenna(w.tx.pos, S.orient_towards(w.tx.pos, w.ris.center), 1.0, 10.0, S.PATTERN_COS_POW)
    w.rx = S.Antenna(np.zeros(3, np.float32), S.orient_towards((0, 0, 0), (0.3, 0.4, 1.0)), 1.0, 1.0,
                     S.PATTERN_MONOPOLE_QW)
    g = run_gpu(w, want_A=True)
    st, *_ = oracle_parity(w, g, check_A=True)
    assert st["strong_frac"] > 0.3


def test_tilted_ceiling_directional():
    """The oracle pin's tilted-ceiling case (horn Tx, tilted monopole Rx, one tilted reflecting plane,
    order 1 on both legs and environment paths) on a receiver grid."""
    from tests.test_oracle_pins import _tilted_ceiling_case
    w = _tilted_ceiling_case()
    w.rx_xyz = S.linspace_grid(-1.2, 1.2, 9, -1.2, 1.2, 9, 1.1, jitter=True)
    w.gammas = S.phase_configs(S.SplitMix64(11), 2, w.n_elem)
    g = run_gpu(w, want_A=True)
    st, *_ = oracle_parity(w, g, check_A=True)
    assert st["excluded"] == 0


def test_room_full_size_sampled():
    """The benchmark's full 256x256 room, traced and evaluated in one launch configuration on the GPU;
    the oracle evaluates a deterministic sample of receivers one by one."""
    w = S.room()
    g = run_gpu(w)
    idx = np.unique(np.linspace(0, w.n_rx - 1, 97).astype(int))
    oracle_parity(w, g, idx=idx)


def test_plate_corridor_wide_candidate_slab():
    """Two stacks of 20 parallel plates: about 840 geometric candidates per receiver and leg, more than
    the first candidate slab holds, so the trace retries with a wider one; most candidates are occluded
    by the inner plates. Path sets and fields match the oracle."""
    w = S.plate_corridor()
    g = run_gpu(w)
    st = g["paths"]["stats"]
    assert st.n_candidates > 512 * w.n_rx
    oracle_parity(w, g)


@pytest.mark.parametrize("case", ["office_order1", "office_1206faces_order2", "hall_order1"])
def test_large_scenes_sampled(case):
    """Scenes above the 1,024 faces whose outlines the candidate search stages in shared memory (so the
    search reads them from global memory), with deep trees and large triangles split over the
    reference grid: the office (9,966 faces, 64x64 RIS, order 1), an office of 200 boxes at order 2
    (1,206 faces) and the hall (99,606 faces, 199,212 triangles, order 1). The whole receiver grid is
    traced on the GPU; the oracle checks 16 receivers spread over it."""
    if case == "office_order1":
        w = S.office()
    elif case == "office_1206faces_order2":
        w = S.office(n_boxes=200)
        w.max_order_tx = w.max_order_rx = 2
    else:
        w = S.hall()
        w.gammas = w.gammas[:1]
    w.gammas = w.gammas[:2]
    assert w.scene.n_faces > 1024
    idx = np.unique(np.linspace(0, w.n_rx - 1, 16).astype(int))
    g = run_gpu(w, want_A=True, A_rows=idx)
    st, *_ = oracle_parity(w, g, idx=idx, check_A=True)
    assert st["excluded"] <= 1


def test_metal_room_tm_and_lossy():
    """Lossy metal walls (eps_r 1, sigma 1e7 S/m, Table 1) make the Fresnel coefficients complex."""
    w = S.room(grid=8, n_boxes=6)
    w.scene.mats[0] = (1.0, 1e7)
    w.scene.mats[1:, 1] = 0.5
    g = run_gpu(w)
    oracle_parity(w, g)


def test_empty_scene_with_orders():
    w = S.free_space(grid=4)
    w.max_order_tx = w.max_order_rx = 2
    g = run_gpu(w)
    _, fld, E, P, Sx = _oracle_all(w)
    compare_fields(g["E"], g["P"], E, P, Sx)


def test_single_triangle_occluder():
    """A scene of one triangle (a BVH whose root is a leaf): it blocks the LOS of some receivers and
    reflects on order-1 paths of both legs and of the environment; path sets and fields match."""
    w = S.free_space(grid=12)
    w.scene = S.Scene(np.array([[-1.0, -1.2, 1.75], [1.0, -1.2, 1.75], [0.0, 0.0, 1.75]], np.float32),
                      np.array([[0, 1, 2]], np.int32), np.zeros(1, np.int32), np.zeros(1, np.int32),
                      np.array([[5.3, 0.1]], np.float32))
    w.max_order_tx = w.max_order_rx = 1
    w.env_paths = True
    g = run_gpu(w)
    st, o, op, fld = oracle_parity(w, g)
    # the triangle removes the LOS of some receivers and not of others
    los = np.asarray(op["los"], bool)
    assert los.any() and (~los).any()


def test_invalid_arguments():
    import torch
    from paper_2402_13034_gb300 import risrt as R
    ctx = R.Context(0, torch.cuda.current_stream().cuda_stream)
    w = S.room(grid=2, n_boxes=2)
    with pytest.raises(R.RisrtError) as e:
        ctx.ris_upload(np.zeros((0, 2)), w.ris.center, w.ris.t1, w.ris.t2, 1e-3, 1e-3)
    assert e.value.code == 1
    scene = ctx.scene_upload(w.scene.verts, w.scene.tris, w.scene.face_id, w.scene.mat_id, w.scene.mats)
    ris = ctx.ris_upload(w.ris.elem_uv, w.ris.center, w.ris.t1, w.ris.t2, w.ris.dy, w.ris.dz, 0, 0)
    rx = ctx.rx_upload(w.rx_xyz)
    with pytest.raises(R.RisrtError) as e:      # antennas not set
        ctx.trace_paths(scene, ris, rx, w.freq_hz, 1, 1)
    assert e.value.code == 5
    ctx.antenna_set(R.TX, w.tx.pos, w.tx.orient, 1.0, 1.0, 0)
    ctx.antenna_set(R.RX, None, w.rx.orient, 1.0, 1.0, 0)
    with pytest.raises(R.RisrtError) as e:
        ctx.trace_paths(scene, ris, rx, w.freq_hz, 3, 1)
    assert e.value.code == 1
    with pytest.raises(R.RisrtError):
        ctx.scene_upload(w.scene.verts, w.scene.tris + 10000, w.scene.face_id, w.scene.mat_id, w.scene.mats)


def test_visibility_maps_change_no_decision(monkeypatch):
    """The first-segment visibility maps and the receiver aperture pyramids decide occlusion without
    traversal; with them forced on and off the path sets are bit-identical, the fields equal, and
    both match the oracle."""
    w = S.room(grid=48)
    out = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("RISRT_MAPS", flag)
        out[flag] = run_gpu(w)
    a, b = out["1"]["paths"], out["0"]["paths"]
    for key in ("seqs", "env"):
        assert all(np.array_equal(np.sort(x), np.sort(y)) for x, y in zip(a[key], b[key]))
    assert np.array_equal(np.asarray(a["los"]), np.asarray(b["los"]))
    assert all(np.array_equal(x, y) for x, y in zip(a["vis"], b["vis"]))
    assert np.array_equal(out["1"]["E"], out["0"]["E"])
    oracle_parity(w, out["1"])


@pytest.mark.parametrize("switch", ["RISRT_SHELL", "RISRT_OVERLAP"])
def test_switches_change_no_decision(monkeypatch, switch):
    """RISRT_SHELL: the room's walls, floor and ceiling (and the box bottoms lying in the floor) have the
    whole scene on one side, so segments with both ends in the scene box skip them. RISRT_OVERLAP: the
    Tx leg, the visibility maps and the direct legs run on side streams beside the receiver legs. With
    either switched off the path sets are bit-identical and the fields equal."""
    w = S.room(grid=40)
    out = {}
    for flag in ("1", "0"):
        monkeypatch.setenv(switch, flag)
        out[flag] = run_gpu(w)
    a, b = out["1"]["paths"], out["0"]["paths"]
    for key in ("seqs", "env"):
        assert all(np.array_equal(np.sort(x), np.sort(y)) for x, y in zip(a[key], b[key]))
    assert np.array_equal(np.asarray(a["los"]), np.asarray(b["los"]))
    assert all(np.array_equal(x, y) for x, y in zip(a["vis"], b["vis"]))
    assert np.array_equal(out["1"]["E"], out["0"]["E"])


@pytest.mark.parametrize("maps", ["1", "0"])
def test_endpoints_outside_scene_box(monkeypatch, maps):
    """A room without its ceiling, the Tx outside wall x = 6 above the wall tops' height and receivers
    outside the room: segments with an end outside the scene box must still be tested against the walls
    (some pass over them, some are stopped); path sets and fields match the oracle."""
    monkeypatch.setenv("RISRT_MAPS", maps)
    w = S.room(grid=10, n_boxes=8)
    keep = w.scene.face_id != 5                   # face 5 is the ceiling (z = 3)
    fid = w.scene.face_id[keep]
    w.scene = S.Scene(w.scene.verts, w.scene.tris[keep], np.where(fid > 5, fid - 1, fid).astype(np.int32),
                      w.scene.mat_id[keep], w.scene.mats)
    w.tx.pos = np.array([6.45, 1.7, 3.42], np.float32)
    extra = np.array([[6.5, 1.0, 1.2], [3.0, 4.5, 1.2], [3.0, 2.0, 3.3], [-0.4, 2.0, 1.5], [2.0, 1.0, -0.3]],
                     np.float32)
    w.rx_xyz = np.concatenate([w.rx_xyz, extra]).astype(np.float32)
    w.env_paths = True
    g = run_gpu(w)
    st, o, op, fld = oracle_parity(w, g)
    los = np.asarray(op["los"], bool)
    assert los.any() and (~los).any()             # the Tx sees over the walls into part of the room


def test_plain_fp32_baseline_error():
    """The plain FP32 baseline of the field evaluation (absolute FP32 phase 2 pi L / lambda with sincosf)
    against the oracle on the room. Its phase error per term is bounded by the FP32 rounding of L and of
    k L (L <= 12 m, k L <= 7.1e3 rad, so a few 1e-4 rad), i.e. a field error of at most about 1e-3 S;
    the element-major kernel with the FP64 per-path phase reference stays within 5e-5 S."""
    import torch
    from paper_2402_13034_gb300 import risrt as R
    w = S.room(grid=16)
    g = run_gpu(w, keep=True)
    ctx, scene, ris, rx, ps = g["handles"]
    gam = torch.from_numpy(w.gammas).cuda()
    E = torch.empty((gam.shape[0], w.n_rx), dtype=torch.complex64, device="cuda")
    ctx.eval_field_plain(ps, gam, E)
    torch.cuda.synchronize()
    Ep = E.cpu().numpy().T
    _, fld, E_ref, P_ref, S_ref = _oracle_all(w)
    ok = ~fld["amb"][:, None] & (S_ref > 0)
    Sd = np.where(S_ref > 0, S_ref, 1.0)
    err_plain = (np.abs(Ep - E_ref) / Sd)[ok].max()
    err_fast = (np.abs(g["E"] - E_ref) / Sd)[ok].max()
    print(f"max |dE|/S: plain FP32 {err_plain:.2e}, eval_field {err_fast:.2e}")
    assert err_fast <= 5e-5
    assert err_plain <= 1e-3


def test_microbenchmarks_positive():
    import torch
    from paper_2402_13034_gb300 import risrt as R
    ctx = R.Context(0, torch.cuda.current_stream().cuda_stream)
    rates = {k: ctx.microbench(k, 64)[0] for k in range(8)}
    assert all(v > 1e9 for v in rates.values()), rates
    assert rates[R.MB_FFMA] > rates[R.MB_MUFU_SIN]


def test_order2_above_10k_faces_sampled():
    """Order 2 on both legs and environment paths in an office of 10,008 faces: about 10^8 face
    sequences per source, pruned on the GPU to those whose second face the beam through the first can
    reach (per source, then per super-patch of receivers) before the per-receiver candidate search.
    The whole 128x128 grid is traced; the oracle, which enumerates every sequence without pruning,
    checks the path sets of 6 receivers spread over it decision by decision."""
    w = S.office(n_boxes=1667)
    w.max_order_tx = w.max_order_rx = 2
    w.gammas = w.gammas[:1]
    assert w.scene.n_faces >= 10000
    g = run_gpu(w)
    idx = np.unique(np.linspace(0, w.n_rx - 1, 6).astype(int))
    o = O.Oracle(w)
    op = o.rx_paths(w.rx_xyz[idx])
    pc = compare_pathsets(subset_paths(g["paths"], idx), op, o.tx_leg())
    assert not pc["bad"], pc["bad"][:10]
    assert pc["amb_rate"] <= 1e-5
    n2 = sum(int(np.sum(s >= w.scene.n_faces)) for s in op["seqs"])
    print(f"order 2 at {w.scene.n_faces} faces: {pc['n_dec']} decisions, {pc['n_amb']} ambiguous, "
          f"{sum(len(s) for s in op['seqs'])} Rx-leg paths ({n2} of order 2), {len(g['paths']['tx_seqs'])} Tx-leg paths")
    assert n2 > 0
