"""Seeded synthetic inputs for the RIS field path (geometry, RIS layout, antennas, Rx grids, configs).

This module is input tooling only: it places triangles, RIS elements, antennas and receiver
points and draws reflection-coefficient configurations from a seeded SplitMix64 stream. It holds
none of the propagation model's arithmetic (no path lengths, patterns, Fresnel terms or fields),
so both the CUDA path and the FP64 CPU oracle can consume exactly the same arrays.

Workloads (paper "Ray Tracing Algorithm for Reconfigurable Intelligent Surfaces", arXiv 2402.13034):

* ``free_space``   - 37-element hexagonal RIS at the origin (normal +z), Tx (0,-1.5,2), 32x32 Rx grid
  on z=1.5 over [-2,2]^2, 28 GHz, line of sight plus the single RIS bounce.
* ``room``         - 6x4x3 m shoebox (concrete, eps_r 5.3) with 40 random axis-aligned boxes
  (eps_r ~ U[2,6]), 127-element hexagonal RIS on wall x=0, 256x256 Rx grid at 1.2 m,
  specular order <= 2 on both legs.
* ``sweep``        - the room with a 32x32 square RIS and 4,096 two-bit phase configurations.
* ``office``       - 20x12x3 m room with ~1,660 boxes (~20k triangles), 64x64 RIS, 128x128 target grid.
* ``paper_anechoic`` / ``paper_reflective`` - Table 1 parameters (Sec. III) with the horn Tx
  (cos^(Gt/2-1) pattern) and quarter-wave monopole Rx.

Conventions: SI units, gains linear, rows of an orientation matrix are the antenna's local
x, y, z axes in global coordinates (theta is measured from the local z axis, Sec. II-A).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C0 = 299_792_458.0  # m/s, used only to turn "lambda/2 pitch" into metres when placing elements

PATTERN_ISO = 0
PATTERN_COS_POW = 1
PATTERN_MONOPOLE_QW = 2

SEED_BASE = 240213034

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 counter generator (Steele, Lea, Flood 2014); doubles from the top 53 bits."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))

    def uniforms(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """n draws in stream order (vectorised SplitMix64, identical to n calls of uniform())."""
        if n == 0:
            return np.zeros(0, dtype=np.float64)
        with np.errstate(over="ignore"):
            k = np.arange(1, n + 1, dtype=np.uint64)
            s = np.uint64(self.state) + k * np.uint64(0x9E3779B97F4A7C15)
            z = s
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        self.state = int(s[-1])
        u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def ints(self, n: int, k: int) -> np.ndarray:
        """n integers uniform on {0..k-1} (floor of a uniform double; k small)."""
        return np.minimum((self.uniforms(n) * k).astype(np.int64), k - 1)


# ----------------------------------------------------------------------------------------------
# Scene containers
# ----------------------------------------------------------------------------------------------

@dataclass
class Scene:
    verts: np.ndarray      # float32 [V,3]
    tris: np.ndarray       # int32 [T,3]
    face_id: np.ndarray    # int32 [T]   planar face each triangle belongs to
    mat_id: np.ndarray     # int32 [T]
    mats: np.ndarray       # float32 [n_mat,2] (eps_r, sigma S/m)

    @property
    def n_faces(self) -> int:
        return int(self.face_id.max()) + 1 if len(self.face_id) else 0


@dataclass
class RIS:
    elem_uv: np.ndarray    # float32 [M,2] element centres in the RIS plane, (a_m, b_m) along (t1, t2)
    center: np.ndarray     # float32 [3]
    t1: np.ndarray         # float32 [3]
    t2: np.ndarray         # float32 [3]   normal n = t1 x t2
    dy: float
    dz: float
    elem_gain: float = 0.0  # <= 0: use 4*pi*dy*dz/lambda^2 (the Tang22 assumption of Sec. II-A)
    host_face: int = -1


@dataclass
class Antenna:
    pos: np.ndarray        # float32 [3] (ignored for the Rx: positions come from the grid)
    orient: np.ndarray     # float32 [3,3] rows = local x, y, z axes
    power_w: float = 1.0
    gain_lin: float = 1.0
    pattern: int = PATTERN_ISO
    pol: np.ndarray | None = None   # float32 [3] polarisation axis (global), for the vector field; None: unset


@dataclass
class Workload:
    name: str
    freq_hz: float
    scene: Scene
    ris: RIS
    tx: Antenna
    rx: Antenna
    rx_xyz: np.ndarray     # float32 [N,3]
    gammas: np.ndarray     # complex64 [C,M]
    max_order_tx: int = 0
    max_order_rx: int = 0
    env_paths: bool = False
    extra: dict = field(default_factory=dict)

    @property
    def n_rx(self) -> int:
        return int(self.rx_xyz.shape[0])

    @property
    def n_elem(self) -> int:
        return int(self.ris.elem_uv.shape[0])


# ----------------------------------------------------------------------------------------------
# Building blocks
# ----------------------------------------------------------------------------------------------

def empty_scene() -> Scene:
    return Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), np.zeros(0, np.int32),
                 np.zeros(0, np.int32), np.array([[1.0, 0.0]], np.float32))


def hex_layout(rings: int, pitch: float) -> np.ndarray:
    """Hexagonal grid of 1+3R(R+1) points: axial (q,r) with max(|q|,|r|,|q+r|) <= R,
    position pitch*(q + r/2, r*sqrt(3)/2); ordered by r then q (Sec. II, Fig. 1 hex grid)."""
    pts = []
    for r in range(-rings, rings + 1):
        for q in range(-rings, rings + 1):
            if max(abs(q), abs(r), abs(q + r)) <= rings:
                pts.append((pitch * (q + 0.5 * r), pitch * r * math.sqrt(3.0) / 2.0))
    return np.asarray(pts, dtype=np.float32)


def square_layout(n_side: int, pitch: float) -> np.ndarray:
    """n_side x n_side row-major grid centred on the RIS centre (first coordinate fastest)."""
    c = (np.arange(n_side) - (n_side - 1) / 2.0) * pitch
    b, a = np.meshgrid(c, c, indexing="ij")
    return np.stack([a.ravel(), b.ravel()], axis=1).astype(np.float32)


def linspace_grid(x0, x1, nx, y0, y1, ny, z, jitter=False) -> np.ndarray:
    """Inclusive linspace grid, row-major with x fastest. With ``jitter`` the whole grid is shifted
    by 0.37*(sqrt(2)-1) of a spacing in x and y so receivers avoid exact geometric alignments."""
    xs = np.linspace(x0, x1, nx)
    ys = np.linspace(y0, y1, ny)
    if jitter:
        off = 0.37 * (math.sqrt(2.0) - 1.0)
        xs = xs + off * (xs[1] - xs[0] if nx > 1 else 0.0)
        ys = ys + off * (ys[1] - ys[0] if ny > 1 else 0.0)
    yy, xx = np.meshgrid(ys, xs, indexing="ij")
    return np.stack([xx.ravel(), yy.ravel(), np.full(xx.size, z)], axis=1).astype(np.float32)


def identity_orient() -> np.ndarray:
    return np.eye(3, dtype=np.float32)


def orient_towards(pos, target) -> np.ndarray:
    """Orientation whose local z axis points from ``pos`` to ``target`` (main lobe aimed, Sec. III-B)."""
    z = np.asarray(target, np.float64) - np.asarray(pos, np.float64)
    z /= np.linalg.norm(z)
    ref = np.array([0.0, 0.0, 1.0]) if abs(z[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    x = np.cross(ref, z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return np.stack([x, y, z]).astype(np.float32)


def spherical_to_cartesian(origin, r, phi_deg, theta_deg) -> np.ndarray:
    """(r, phi, theta) about ``origin``: theta from +z, phi from +x (Sec. II-A, Sec. III)."""
    ph, th = math.radians(phi_deg), math.radians(theta_deg)
    o = np.asarray(origin, np.float64)
    return o + r * np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])


class _MeshBuilder:
    def __init__(self):
        self.verts, self.tris, self.face, self.mat = [], [], [], []
        self.n_faces = 0

    def quad(self, p0, p1, p2, p3, mat):
        """Planar quad p0-p1-p2-p3 as two triangles of one face."""
        b = len(self.verts)
        self.verts += [p0, p1, p2, p3]
        self.tris += [(b, b + 1, b + 2), (b, b + 2, b + 3)]
        self.face += [self.n_faces, self.n_faces]
        self.mat += [mat, mat]
        self.n_faces += 1
        return self.n_faces - 1

    def box(self, lo, hi, mat):
        """Axis-aligned box: six faces, order x-, x+, y-, y+, z-, z+. Returns the first face id."""
        x0, y0, z0 = lo
        x1, y1, z1 = hi
        f = self.quad((x0, y0, z0), (x0, y0, z1), (x0, y1, z1), (x0, y1, z0), mat)
        self.quad((x1, y0, z0), (x1, y1, z0), (x1, y1, z1), (x1, y0, z1), mat)
        self.quad((x0, y0, z0), (x1, y0, z0), (x1, y0, z1), (x0, y0, z1), mat)
        self.quad((x0, y1, z0), (x0, y1, z1), (x1, y1, z1), (x1, y1, z0), mat)
        self.quad((x0, y0, z0), (x0, y1, z0), (x1, y1, z0), (x1, y0, z0), mat)
        self.quad((x0, y0, z1), (x1, y0, z1), (x1, y1, z1), (x0, y1, z1), mat)
        return f

    def scene(self, mats) -> Scene:
        return Scene(np.asarray(self.verts, np.float32).reshape(-1, 3),
                     np.asarray(self.tris, np.int32).reshape(-1, 3),
                     np.asarray(self.face, np.int32), np.asarray(self.mat, np.int32),
                     np.asarray(mats, np.float32).reshape(-1, 2))


def _aabb_point_dist(lo, hi, p) -> float:
    d = np.maximum(np.maximum(np.asarray(lo) - p, 0.0), np.asarray(p) - np.asarray(hi))
    return float(np.linalg.norm(d))


def room_with_boxes(rng: SplitMix64, size, n_boxes, keepout_pts, keepout=0.3,
                    wall_eps=5.3, box_eps=(2.0, 6.0), sxy=(0.2, 1.0), sz=(0.3, 2.0)) -> tuple:
    """Shoebox [0,X]x[0,Y]x[0,Z] (room walls are faces 0..5: x=0, x=X, y=0, y=Y, z=0, z=Z) plus
    ``n_boxes`` axis-aligned boxes resting on the floor, inside the room, at least ``keepout`` from
    every keep-out point. Material 0 is the wall; box i has material i+1 with eps_r ~ U[box_eps]."""
    X, Y, Z = size
    mb = _MeshBuilder()
    mb.quad((0, 0, 0), (0, 0, Z), (0, Y, Z), (0, Y, 0), 0)        # x = 0
    mb.quad((X, 0, 0), (X, Y, 0), (X, Y, Z), (X, 0, Z), 0)        # x = X
    mb.quad((0, 0, 0), (X, 0, 0), (X, 0, Z), (0, 0, Z), 0)        # y = 0
    mb.quad((0, Y, 0), (0, Y, Z), (X, Y, Z), (X, Y, 0), 0)        # y = Y
    mb.quad((0, 0, 0), (0, Y, 0), (X, Y, 0), (X, 0, 0), 0)        # z = 0
    mb.quad((0, 0, Z), (X, 0, Z), (X, Y, Z), (0, Y, Z), 0)        # z = Z
    mats = [(wall_eps, 0.0)]
    placed = 0
    while placed < n_boxes:
        bx, by = rng.uniform(*sxy), rng.uniform(*sxy)
        bz = min(rng.uniform(*sz), Z - 0.05)
        x0, y0 = rng.uniform(0.0, X - bx), rng.uniform(0.0, Y - by)
        lo, hi = (x0, y0, 0.0), (x0 + bx, y0 + by, bz)
        if any(_aabb_point_dist(lo, hi, np.asarray(p)) < keepout for p in keepout_pts):
            continue
        mats.append((rng.uniform(*box_eps), 0.0))
        mb.box(lo, hi, len(mats) - 1)
        placed += 1
    return mb.scene(mats), 0  # host face of a RIS on wall x = 0


def phase_configs(rng: SplitMix64, n_cfg: int, M: int, amp: float = 1.0) -> np.ndarray:
    """Uniform phases on [0, 2pi) per element; Gamma = amp * exp(j phi). complex64 [C,M]."""
    ph = rng.uniforms(n_cfg * M, 0.0, 2.0 * math.pi).reshape(n_cfg, M)
    return (amp * np.exp(1j * ph)).astype(np.complex64)


def two_bit_configs(rng: SplitMix64, n_cfg: int, M: int) -> tuple:
    """2-bit phase codes q ~ U{0..3}, Gamma = j^q (amplitude 1). Returns (codes uint8 [C,M], complex64)."""
    q = rng.ints(n_cfg * M, 4).reshape(n_cfg, M).astype(np.uint8)
    table = np.array([1, 1j, -1, -1j], dtype=np.complex64)
    return q, table[q]


def focus_phase_config(ris: RIS, tx_pos, focus, freq_hz, amp=1.0) -> np.ndarray:
    """Geometric beam-focusing profile: each element's phase cancels its direct Tx->element->focus
    path length, Gamma_m = amp*exp(+j*2*pi*(d_t+d_r)/lambda). Computed in float64 from the same
    float32 element coordinates both implementations receive. complex64 [M]."""
    lam = C0 / freq_hz
    c = ris.center.astype(np.float64)
    e = c + ris.elem_uv[:, :1].astype(np.float64) * ris.t1.astype(np.float64) \
          + ris.elem_uv[:, 1:].astype(np.float64) * ris.t2.astype(np.float64)
    d = np.linalg.norm(e - np.asarray(tx_pos, np.float64), axis=1) + \
        np.linalg.norm(e - np.asarray(focus, np.float64), axis=1)
    frac = np.mod(d / lam, 1.0)
    return (amp * np.exp(2j * math.pi * frac)).astype(np.complex64)


# ----------------------------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------------------------

def free_space(n_cfg_random: int = 8, grid: int = 32) -> Workload:
    """37-element hex RIS (3 rings, lambda/2 pitch, 28 GHz) at the origin in z=0; Tx (0,-1.5,2);
    Rx grid x grid on z=1.5 over [-2,2]^2; LOS + single RIS bounce; uniform-phase configs + a focus."""
    rng = SplitMix64(SEED_BASE + 0)
    f = 28e9
    lam = C0 / f
    ris = RIS(hex_layout(3, lam / 2), np.zeros(3, np.float32), np.array([1, 0, 0], np.float32),
              np.array([0, 1, 0], np.float32), lam / 2, lam / 2, 0.0, -1)
    tx = Antenna(np.array([0.0, -1.5, 2.0], np.float32), identity_orient(), 1.0, 1.0, PATTERN_ISO)
    rx = Antenna(np.zeros(3, np.float32), identity_orient(), 1.0, 1.0, PATTERN_ISO)
    rx_xyz = linspace_grid(-2, 2, grid, -2, 2, grid, 1.5)
    g = phase_configs(rng, n_cfg_random, len(ris.elem_uv))
    foc = focus_phase_config(ris, tx.pos, (0.0, 0.0, 1.5), f)
    return Workload("free_space_37el_32x32", f, empty_scene(), ris, tx, rx, rx_xyz,
                    np.concatenate([g, foc[None]], 0), 0, 0, False)


def room(grid: int = 256, n_boxes: int = 40, n_cfg_random: int = 1, square_side: int = 0,
         seed_index: int = 1) -> Workload:
    """6x4x3 m concrete room + 40 random boxes, 127-element hex RIS (6 rings, lambda/2) on wall x=0
    centred (0,2,1.5) with normal +x, Tx (3.0,0.5,2.5) isotropic 1 W, Rx grid at z=1.2 over
    [0.1,5.9]x[0.1,3.9] (jittered), specular order <= 2 on both legs, 28 GHz.
    ``square_side`` > 0 replaces the hex RIS with a square one of that side (the sweep workload)."""
    rng = SplitMix64(SEED_BASE + seed_index)
    f = 28e9
    lam = C0 / f
    center = np.array([0.0, 2.0, 1.5], np.float32)
    txp = np.array([3.0, 0.5, 2.5], np.float32)
    scene, host = room_with_boxes(rng, (6.0, 4.0, 3.0), n_boxes, [txp, center])
    layout = square_layout(square_side, lam / 2) if square_side else hex_layout(6, lam / 2)
    ris = RIS(layout, center, np.array([0, 1, 0], np.float32), np.array([0, 0, 1], np.float32),
              lam / 2, lam / 2, 0.0, host)
    tx = Antenna(txp, identity_orient(), 1.0, 1.0, PATTERN_ISO)
    rx = Antenna(np.zeros(3, np.float32), identity_orient(), 1.0, 1.0, PATTERN_ISO)
    rx_xyz = linspace_grid(0.1, 5.9, grid, 0.1, 3.9, grid, 1.2, jitter=True)
    g = phase_configs(rng, n_cfg_random, len(layout))
    foc = focus_phase_config(ris, txp, (3.0, 2.0, 1.2), f)
    name = f"room_{len(layout)}el_{grid}x{grid}_order2"
    return Workload(name, f, scene, ris, tx, rx, rx_xyz, np.concatenate([g, foc[None]], 0),
                    2, 2, True)


def sweep(n_cfg: int = 4096, grid: int = 256) -> Workload:
    """The room with a 32x32 square RIS (lambda/2) replacing the hex one; 2-bit phase configs."""
    w = room(grid=grid, square_side=32, n_cfg_random=0)
    rng = SplitMix64(SEED_BASE + 2)
    codes, g = two_bit_configs(rng, n_cfg, w.n_elem)
    w.gammas = g
    w.extra["codes"] = codes
    w.name = f"sweep_{w.n_elem}el_{w.n_rx}rx_{n_cfg}cfg"
    return w


def office(n_boxes: int = 1660, target_grid: int = 128, n_start: int = 64, ris_side: int = 64) -> Workload:
    """20x12x3 m office with ~1,660 random boxes (~20k triangles), 64x64 RIS on wall x=0 centred
    (0,6,1.5), Tx (10,2,2.5), 128x128 target Rx over [6,10]x[4,8] at 1.2 m, order <= 1."""
    rng = SplitMix64(SEED_BASE + 3)
    f = 28e9
    lam = C0 / f
    center = np.array([0.0, 6.0, 1.5], np.float32)
    txp = np.array([10.0, 2.0, 2.5], np.float32)
    scene, host = room_with_boxes(rng, (20.0, 12.0, 3.0), n_boxes, [txp, center],
                                  sxy=(0.2, 0.8), sz=(0.3, 1.0))
    ris = RIS(square_layout(ris_side, lam / 2), center, np.array([0, 1, 0], np.float32),
              np.array([0, 0, 1], np.float32), lam / 2, lam / 2, 0.0, host)
    tx = Antenna(txp, identity_orient(), 1.0, 1.0, PATTERN_ISO)
    rx = Antenna(np.zeros(3, np.float32), identity_orient(), 1.0, 1.0, PATTERN_ISO)
    rx_xyz = linspace_grid(6.0, 10.0, target_grid, 4.0, 8.0, target_grid, 1.2, jitter=True)
    phases = rng.uniforms(n_start * ris.elem_uv.shape[0], 0.0, 2 * math.pi)
    phases = phases.reshape(n_start, -1).astype(np.float32)
    w = Workload(f"office_{ris.elem_uv.shape[0]}el_{len(scene.tris)}tri", f, scene, ris, tx, rx,
                 rx_xyz, np.exp(1j * phases).astype(np.complex64), 1, 1, True)
    w.extra["phases"] = phases
    return w


def hall(n_boxes: int = 16600, target_grid: int = 256) -> Workload:
    """60x40x3 m hall with ~16,600 random boxes (~200k triangles), the largest scene of the serving
    mix: 64x64 RIS on wall x=0 centred (0,20,1.5), Tx (30,10,2.5), 256x256 Rx over the floor at
    1.2 m, order <= 1."""
    rng = SplitMix64(SEED_BASE + 5)
    f = 28e9
    lam = C0 / f
    center = np.array([0.0, 20.0, 1.5], np.float32)
    txp = np.array([30.0, 10.0, 2.5], np.float32)
    scene, host = room_with_boxes(rng, (60.0, 40.0, 3.0), n_boxes, [txp, center], sxy=(0.2, 0.8), sz=(0.3, 1.0))
    ris = RIS(square_layout(64, lam / 2), center, np.array([0, 1, 0], np.float32),
              np.array([0, 0, 1], np.float32), lam / 2, lam / 2, 0.0, host)
    tx = Antenna(txp, identity_orient(), 1.0, 1.0, PATTERN_ISO)
    rx = Antenna(np.zeros(3, np.float32), identity_orient(), 1.0, 1.0, PATTERN_ISO)
    rx_xyz = linspace_grid(0.2, 59.8, target_grid, 0.2, 39.8, target_grid, 1.2, jitter=True)
    g = phase_configs(rng, 1, ris.elem_uv.shape[0])
    return Workload(f"hall_{ris.elem_uv.shape[0]}el_{len(scene.tris)}tri", f, scene, ris, tx, rx, rx_xyz, g, 1, 1, True)


def paper_anechoic(grid_step: float = 0.01) -> Workload:
    """Table 1 set-up without walls: 127-element hex RIS (12 cm / 13 pitch) centred u=(0,0,0.5),
    normal +x, d_y=d_z=6.6 mm, 23.8 GHz, Pt 10 dBm, horn Tx Gt 19 dB aimed at u, monopole Rx
    (0 dB, vertical); Rx grid 0.92<=x<=1.52, 0.02<=y<=0.92 at z=11.4 cm (Sec. III)."""
    f = 23.8e9
    u = np.array([0.0, 0.0, 0.5])
    txp = spherical_to_cartesian(u, 1.86, -36.0, 90.0).astype(np.float32)
    ris = RIS(hex_layout(6, 0.12 / 13), u.astype(np.float32), np.array([0, 1, 0], np.float32),
              np.array([0, 0, 1], np.float32), 6.6e-3, 6.6e-3, 0.0, -1)
    tx = Antenna(txp, orient_towards(txp, u), 0.01, 10 ** 1.9, PATTERN_COS_POW)
    rx = Antenna(np.zeros(3, np.float32), identity_orient(), 1.0, 1.0, PATTERN_MONOPOLE_QW)
    nx = int(round((1.52 - 0.92) / grid_step)) + 1
    ny = int(round((0.92 - 0.02) / grid_step)) + 1
    rx_xyz = linspace_grid(0.92, 1.52, nx, 0.02, 0.92, ny, 0.114)
    return Workload("paper_anechoic", f, empty_scene(), ris, tx, rx, rx_xyz,
                    np.ones((1, 127), np.complex64) * 1.25, 0, 0, False)


def paper_reflective(grid_step: float = 0.01, closeup: bool = False, wall: float = 0.05) -> Workload:
    """The reflective set-up of Sec. III (Table 2): three metal walls (eps_r 1, sigma 1e7 S/m) of a
    2 x 2.4 x 1 m room (blocks ``wall`` thick: x = 2 opposite the RIS, y = +-1.2 at the sides; the
    side x = 0 is the opening holding the RIS), a 0.9 x 0.05 x 1 m metal panel centred (1.55, -0.475,
    0.5) that blocks the Tx -> Rx line, the 127-element hex RIS (12 cm / 13 pitch, 6.6 mm elements)
    centred u = (0, 0, 0.5) with normal +x, 23.8 GHz, horn Tx (Gt 19 dB, 10 dBm) at
    t = (1.86 m, -36 deg, 90 deg) about u aimed at u, vertical monopole Rx. Receivers on z = 11.4 cm
    over 0.92 <= x <= 1.52, 0.02 <= y <= 0.92 at ``grid_step`` (Fig. 4 c), or with ``closeup`` over
    1.1 <= x <= 1.3, 0.25 <= y <= 0.45 at 2 mm (Fig. 5). RIS -> Rx reflections up to order 2, no
    Tx-leg reflections, no environment paths (every multipath component from the RIS, Sec. III).
    Configuration: each element on (Gamma = 1.25) when its direct Tx -> element -> intended-Rx path
    phase lies within a quarter turn of zero, else off (Eq. 11 alphabet; a geometric stand-in for the
    configuration algorithm the paper cites), intended Rx r = (1.4 m, 10 deg, 106 deg) about u."""
    f = 23.8e9
    u = np.array([0.0, 0.0, 0.5])
    mb = _MeshBuilder()
    mats = [(1.0, 1e7)]
    mb.box((2.0, -1.2, 0.0), (2.0 + wall, 1.2, 1.0), 0)                 # opposite the RIS
    mb.box((0.0, -1.2 - wall, 0.0), (2.0 + wall, -1.2, 1.0), 0)         # side walls
    mb.box((0.0, 1.2, 0.0), (2.0 + wall, 1.2 + wall, 1.0), 0)
    mb.box((1.1, -0.5, 0.0), (2.0, -0.45, 1.0), 0)                      # blocking panel
    scene = mb.scene(mats)
    txp = spherical_to_cartesian(u, 1.86, -36.0, 90.0).astype(np.float32)
    ris = RIS(hex_layout(6, 0.12 / 13), u.astype(np.float32), np.array([0, 1, 0], np.float32),
              np.array([0, 0, 1], np.float32), 6.6e-3, 6.6e-3, 0.0, -1)
    tx = Antenna(txp, orient_towards(txp, u), 0.01, 10 ** 1.9, PATTERN_COS_POW)
    rx = Antenna(np.zeros(3, np.float32), identity_orient(), 1.0, 1.0, PATTERN_MONOPOLE_QW)
    if closeup:
        rx_xyz = linspace_grid(1.1, 1.3, 101, 0.25, 0.45, 101, 0.114)
    else:
        nx = int(round((1.52 - 0.92) / grid_step)) + 1
        ny = int(round((0.92 - 0.02) / grid_step)) + 1
        rx_xyz = linspace_grid(0.92, 1.52, nx, 0.02, 0.92, ny, 0.114)
    target = spherical_to_cartesian(u, 1.4, 10.0, 106.0)
    foc = focus_phase_config(ris, txp, target, f)
    gam = np.where(np.real(foc) > 0, 1.25, 0.0).astype(np.complex64)
    name = "paper_reflective_closeup" if closeup else "paper_reflective"
    w = Workload(name, f, scene, ris, tx, rx, rx_xyz, gam[None], 0, 2, False)
    w.extra["intended_rx"] = target
    return w


def plate_corridor(n_side: int = 20, grid: int = 8, spacing: float = 0.25, half: float = 60.0) -> Workload:
    """37-element hex RIS (lambda/2, 28 GHz) at the origin facing +y between two stacks of ``n_side``
    large parallel plates (planes x = +-(0.5 + i*spacing), eps_r 3): every receiver has about
    2 n_side^2 + 2 n_side geometric order-2 candidates on each receiver leg (one per plate pair on
    opposite sides), most of them occluded by the inner plates. Tx (0.2, 3, 0.4) isotropic;
    grid x grid receivers over [-0.4, 0.4]^2 in x and z at y = 2; order <= 2 on both legs."""
    rng = SplitMix64(SEED_BASE + 6)
    f = 28e9
    lam = C0 / f
    mb = _MeshBuilder()
    for i in range(n_side):
        x = 0.5 + i * spacing
        mb.quad((x, -half, -half), (x, half, -half), (x, half, half), (x, -half, half), 0)
        mb.quad((-x, -half, -half), (-x, -half, half), (-x, half, half), (-x, half, -half), 0)
    scene = mb.scene([(3.0, 0.0)])
    ris = RIS(hex_layout(3, lam / 2), np.zeros(3, np.float32), np.array([0, 0, 1], np.float32),
              np.array([1, 0, 0], np.float32), lam / 2, lam / 2, 0.0, -1)
    tx = Antenna(np.array([0.2, 3.0, 0.4], np.float32), identity_orient(), 1.0, 1.0, PATTERN_ISO)
    rx = Antenna(np.zeros(3, np.float32), identity_orient(), 1.0, 1.0, PATTERN_ISO)
    g = linspace_grid(-0.4, 0.4, grid, -0.4, 0.4, grid, 2.0, jitter=True)
    rx_xyz = np.stack([g[:, 0], g[:, 2], g[:, 1]], axis=1).astype(np.float32)
    return Workload(f"plate_corridor_{2 * n_side}faces_{grid}x{grid}", f, scene, ris, tx, rx, rx_xyz,
                    phase_configs(rng, 1, len(ris.elem_uv)), 2, 2, True)


WORKLOADS = {
    "free_space": free_space,
    "room": room,
    "sweep": sweep,
    "office": office,
    "paper_anechoic": paper_anechoic,
    "paper_reflective": paper_reflective,
}
