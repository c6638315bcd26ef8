"""Python front end of the FP64 CPU oracle (``ris_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it. It never touches the CUDA library and the CUDA library never touches it.

The oracle evaluates the paper's RIS path-loss model (Eqs. 4-10, arXiv 2402.13034) as the plain,
unfactored triple sum over elements, Tx-leg paths and Rx-leg paths, with the image method of
Sec. II-B (validation between the RIS centre and each endpoint) and Fresnel reflection per bounce.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ris_oracle.c")
_LIB = os.path.join(_HERE, "libris_oracle.so")
_lock = threading.Lock()
_lib = None

ETA0 = 120.0 * np.pi


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, OpenMP over receivers)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("verts", C.c_void_p), ("n_verts", C.c_int64),
        ("tris", C.c_void_p), ("face_id", C.c_void_p), ("mat_id", C.c_void_p), ("n_tris", C.c_int64),
        ("mats", C.c_void_p), ("n_mat", C.c_int32),
        ("elem_uv", C.c_void_p), ("M", C.c_int32),
        ("center", C.c_float * 3), ("t1", C.c_float * 3), ("t2", C.c_float * 3),
        ("dy", C.c_float), ("dz", C.c_float), ("elem_gain", C.c_float), ("host_face", C.c_int32),
        ("tx_pos", C.c_float * 3), ("tx_orient", C.c_float * 9), ("tx_power", C.c_float),
        ("tx_gain", C.c_float), ("tx_pattern", C.c_int32),
        ("rx_orient", C.c_float * 9), ("rx_gain", C.c_float), ("rx_pattern", C.c_int32),
        ("freq", C.c_double),
        ("max_order_tx", C.c_int32), ("max_order_rx", C.c_int32), ("env_paths", C.c_int32),
        ("fresnel_tm", C.c_int32), ("strict_elements", C.c_int32),
        ("vector_pol", C.c_int32), ("tx_pol", C.c_float * 3), ("rx_pol", C.c_float * 3),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            lib.or_create.restype = C.c_void_p
            lib.or_create.argtypes = [C.POINTER(_Problem)]
            lib.or_destroy.argtypes = [C.c_void_p]
            lib.or_pattern.restype = C.c_double
            lib.or_pattern.argtypes = [C.c_int, C.c_double, C.c_double]
            lib.or_fresnel.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_int,
                                       C.POINTER(C.c_double), C.POINTER(C.c_double)]
            lib.or_set_amb_tol.argtypes = [C.c_double]
            lib.or_n_faces.argtypes = [C.c_void_p]
            lib.or_tx_leg.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                      C.c_void_p]
            lib.or_rx_paths.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int32,
                                        C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_int32, C.c_void_p, C.c_void_p]
            lib.or_field.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
            lib.or_field_vec.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            lib.or_cir.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            lib.or_element_positions.argtypes = [C.c_void_p, C.c_void_p]
            lib.or_element_paths.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                             C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int32,
                                             C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]
            lib.or_segment_blocked.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                               C.c_void_p]
            lib.or_validate.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                                        C.c_int64, C.c_void_p, C.c_void_p]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None and a.size else None


def pattern(pat: int, gain: float, cos_t: float) -> float:
    return _load().or_pattern(pat, gain, cos_t)


def fresnel(cos_i: float, eps_r: float, sigma: float, freq: float, tm: bool = False) -> complex:
    re, im = C.c_double(), C.c_double()
    _load().or_fresnel(cos_i, eps_r, sigma, freq, int(tm), C.byref(re), C.byref(im))
    return complex(re.value, im.value)


def set_amb_tol(tol: float) -> None:
    _load().or_set_amb_tol(tol)


class Oracle:
    """FP64 oracle bound to one workload (scene, RIS, antennas, frequency, orders, flags)."""

    def __init__(self, w, fresnel_tm: bool = False, strict: bool = False, vector: bool = False):
        lib = _load()
        self.w = w
        sc, ris = w.scene, w.ris
        # keep contiguous copies alive for the lifetime of the C context
        self._keep = dict(
            verts=np.ascontiguousarray(sc.verts, np.float32),
            tris=np.ascontiguousarray(sc.tris, np.int32),
            face=np.ascontiguousarray(sc.face_id, np.int32),
            mat=np.ascontiguousarray(sc.mat_id, np.int32),
            mats=np.ascontiguousarray(sc.mats, np.float32),
            uv=np.ascontiguousarray(ris.elem_uv, np.float32),
        )
        k = self._keep
        P = _Problem()
        P.verts, P.n_verts = _ptr(k["verts"]), len(k["verts"])
        P.tris, P.face_id, P.mat_id, P.n_tris = _ptr(k["tris"]), _ptr(k["face"]), _ptr(k["mat"]), len(k["tris"])
        P.mats, P.n_mat = _ptr(k["mats"]), len(k["mats"])
        P.elem_uv, P.M = _ptr(k["uv"]), len(k["uv"])
        P.center[:] = [float(x) for x in ris.center]
        P.t1[:] = [float(x) for x in ris.t1]
        P.t2[:] = [float(x) for x in ris.t2]
        P.dy, P.dz, P.elem_gain, P.host_face = ris.dy, ris.dz, ris.elem_gain, ris.host_face
        P.tx_pos[:] = [float(x) for x in w.tx.pos]
        P.tx_orient[:] = [float(x) for x in np.asarray(w.tx.orient, np.float32).ravel()]
        P.tx_power, P.tx_gain, P.tx_pattern = w.tx.power_w, w.tx.gain_lin, w.tx.pattern
        P.rx_orient[:] = [float(x) for x in np.asarray(w.rx.orient, np.float32).ravel()]
        P.rx_gain, P.rx_pattern = w.rx.gain_lin, w.rx.pattern
        P.freq = w.freq_hz
        P.max_order_tx, P.max_order_rx = w.max_order_tx, w.max_order_rx
        P.env_paths, P.fresnel_tm = int(w.env_paths), int(fresnel_tm)
        P.strict_elements = int(strict)
        P.vector_pol = int(vector)
        if vector:
            if w.tx.pol is None or w.rx.pol is None:
                raise ValueError("the vector field needs the Tx and Rx polarisation axes")
            P.tx_pol[:] = [float(x) for x in np.asarray(w.tx.pol, np.float32)]
            P.rx_pol[:] = [float(x) for x in np.asarray(w.rx.pol, np.float32)]
        self.vector = bool(vector)
        self._P = P
        self._ctx = lib.or_create(C.byref(P))
        self.F = lib.or_n_faces(self._ctx)
        self.M = w.n_elem

    def __del__(self):
        try:
            if getattr(self, "_ctx", None):
                _load().or_destroy(self._ctx)
        except Exception:
            pass

    # --- geometry -----------------------------------------------------------------------------
    def element_positions(self) -> np.ndarray:
        out = np.zeros((self.M, 3))
        _load().or_element_positions(self._ctx, _ptr(out))
        return out

    def segment_blocked(self, a, b, ign0: int = -1, ign1: int = -1):
        a = np.asarray(a, np.float64)
        b = np.asarray(b, np.float64)
        amb = np.zeros(1, np.int32)
        r = _load().or_segment_blocked(self._ctx, _ptr(a), _ptr(b), ign0, ign1, _ptr(amb))
        return bool(r), bool(amb[0])

    def validate(self, src, src_face, dst, dst_face, seq_id: int):
        src = np.asarray(src, np.float64)
        dst = np.asarray(dst, np.float64)
        k = 1 if seq_id < self.F else 2
        pts = np.zeros((k + 2, 3))
        amb = np.zeros(1, np.int32)
        ok = _load().or_validate(self._ctx, _ptr(src), src_face, _ptr(dst), dst_face, seq_id,
                                 _ptr(amb), _ptr(pts))
        return bool(ok), bool(amb[0]), pts

    def seq_id(self, *faces) -> int:
        if len(faces) == 1:
            return faces[0]
        return self.F + faces[0] * self.F + faces[1]

    # --- path sets ----------------------------------------------------------------------------
    def tx_leg(self, cap: int = 1 << 16, amb_cap: int = 1 << 12):
        """Valid reflected Tx-leg sequences and per-element direct visibility. ``amb`` is set if any
        decision is ambiguous; ``vis_amb`` / ``amb_seqs`` name the ambiguous decisions; ``n_dec``
        counts every decision (elements plus allowed sequences)."""
        ids = np.zeros(cap, np.int64)
        n = np.zeros(1, np.int64)
        vis = np.zeros(self.M, np.uint8)
        amb = np.zeros(1, np.int32)
        vis_amb = np.zeros(self.M, np.uint8)
        amb_ids = np.zeros(amb_cap, np.int64)
        n_amb = np.zeros(1, np.int64)
        n_dec = np.zeros(1, np.int64)
        _load().or_tx_leg(self._ctx, _ptr(ids), cap, _ptr(n), _ptr(vis), _ptr(amb), _ptr(vis_amb),
                          _ptr(amb_ids), amb_cap, _ptr(n_amb), _ptr(n_dec))
        if n[0] > cap or n_amb[0] > amb_cap:
            raise RuntimeError("oracle Tx-leg capacity exceeded")
        return dict(seqs=ids[: int(n[0])].copy(), vis=vis.astype(bool), amb=bool(amb[0]),
                    vis_amb=vis_amb.astype(bool), amb_seqs=amb_ids[: int(n_amb[0])].copy(),
                    n_dec=int(n_dec[0]))

    ENV_TAG = 1 << 62

    def rx_paths(self, rx_xyz: np.ndarray, cap: int = 512, env_cap: int = 512, amb_cap: int = 256):
        """Per receiver: valid Rx-leg and environment sequences, LOS, direct visibility bits, whether
        any decision is ambiguous (``amb``), and per decision: ``los_amb``, ``vis_amb`` bits,
        ``amb_seqs`` (Rx-leg ids) / ``amb_env`` (environment ids) whose validity is ambiguous, and
        ``n_dec``, the number of decisions taken."""
        rx = np.ascontiguousarray(rx_xyz, np.float32).reshape(-1, 3)
        n = len(rx)
        W = (self.M + 31) // 32
        seq = np.full((n, cap), -1, np.int64)
        env = np.full((n, env_cap), -1, np.int64)
        n_seq = np.zeros(n, np.int32)
        n_env = np.zeros(n, np.int32)
        los = np.zeros(n, np.uint8)
        vis = np.zeros((n, W), np.uint32)
        amb = np.zeros(n, np.int32)
        los_amb = np.zeros(n, np.uint8)
        vis_amb = np.zeros((n, W), np.uint32)
        amb_ids = np.full((n, amb_cap), -1, np.int64)
        n_amb = np.zeros(n, np.int32)
        n_dec = np.zeros(n, np.int64)
        _load().or_rx_paths(self._ctx, _ptr(rx), n, _ptr(seq), cap, _ptr(n_seq), _ptr(env), env_cap,
                            _ptr(n_env), _ptr(los), _ptr(vis), _ptr(amb), _ptr(los_amb), _ptr(vis_amb),
                            _ptr(amb_ids), amb_cap, _ptr(n_amb), _ptr(n_dec))
        if (n_seq > cap).any() or (n_env > env_cap).any() or (n_amb > amb_cap).any():
            raise RuntimeError("oracle path capacity exceeded")
        amb_rx, amb_env = [], []
        for i in range(n):
            a = amb_ids[i, : n_amb[i]]
            tagged = (a & self.ENV_TAG) != 0
            amb_rx.append(a[~tagged].copy())
            amb_env.append((a[tagged] & ~self.ENV_TAG).copy())
        return dict(seqs=[seq[i, : n_seq[i]].copy() for i in range(n)],
                    env=[env[i, : n_env[i]].copy() for i in range(n)],
                    los=los.astype(bool), vis=vis, amb=amb.astype(bool), los_amb=los_amb.astype(bool),
                    vis_amb=vis_amb, amb_seqs=amb_rx, amb_env=amb_env, n_dec=n_dec)

    def element_paths(self, m: int, rx_xyz: np.ndarray, cap: int = 512, amb_cap: int = 256):
        """Strict mode's path sets of element m (reflected legs validated at the element itself): the
        valid Tx-leg ids, and per receiver the valid Rx-leg ids, each with the ambiguous decisions, and
        the number of decisions."""
        rx = np.ascontiguousarray(rx_xyz, np.float32).reshape(-1, 3)
        n = len(rx)
        tx = np.zeros(1 << 16, np.int64)
        tx_amb = np.zeros(1 << 12, np.int64)
        n_tx, n_tx_amb, n_dec = np.zeros(1, np.int64), np.zeros(1, np.int64), np.zeros(1, np.int64)
        seq = np.full((n, cap), -1, np.int64)
        amb = np.full((n, amb_cap), -1, np.int64)
        n_seq, n_amb = np.zeros(n, np.int32), np.zeros(n, np.int32)
        _load().or_element_paths(self._ctx, int(m), _ptr(rx), n, _ptr(tx), len(tx), _ptr(n_tx), _ptr(tx_amb), len(tx_amb),
                                 _ptr(n_tx_amb), _ptr(seq), cap, _ptr(n_seq), _ptr(amb), amb_cap, _ptr(n_amb), _ptr(n_dec))
        if (n_seq > cap).any() or (n_amb > amb_cap).any() or n_tx[0] > len(tx) or n_tx_amb[0] > len(tx_amb):
            raise RuntimeError("oracle path capacity exceeded")
        return dict(tx_seqs=tx[: int(n_tx[0])].copy(), tx_amb=tx_amb[: int(n_tx_amb[0])].copy(),
                    seqs=[seq[i, : n_seq[i]].copy() for i in range(n)],
                    amb_seqs=[amb[i, : n_amb[i]].copy() for i in range(n)], n_dec=int(n_dec[0]))

    # --- field --------------------------------------------------------------------------------
    def field(self, rx_xyz: np.ndarray):
        """E0 (LOS + environment), S0, channel rows A [n, M] (E = E0 + A @ Gamma), SA, ambiguity."""
        rx = np.ascontiguousarray(rx_xyz, np.float32).reshape(-1, 3)
        n = len(rx)
        E0 = np.zeros((n, 2))
        S0 = np.zeros(n)
        A = np.zeros((n, self.M, 2))
        SA = np.zeros((n, self.M))
        amb = np.zeros(n, np.int32)
        _load().or_field(self._ctx, _ptr(rx), n, _ptr(E0), _ptr(S0), _ptr(A), _ptr(SA), _ptr(amb), 0)
        return dict(E0=E0[:, 0] + 1j * E0[:, 1], S0=S0, A=A[..., 0] + 1j * A[..., 1], SA=SA,
                    amb=amb.astype(bool))

    def field_vec(self, rx_xyz: np.ndarray):
        """Vector mode: ``field``'s entries for the received values (co-polarised with the Rx axis) plus
        the field vectors E03 [n, 3], A3 [n, M, 3] and their incoherent magnitudes S03, SA3."""
        if not self.vector:
            raise ValueError("the oracle was built without vector=True")
        rx = np.ascontiguousarray(rx_xyz, np.float32).reshape(-1, 3)
        n = len(rx)
        E0 = np.zeros((n, 2))
        S0 = np.zeros(n)
        A = np.zeros((n, self.M, 2))
        SA = np.zeros((n, self.M))
        amb = np.zeros(n, np.int32)
        E03 = np.zeros((n, 3, 2))
        S03 = np.zeros(n)
        A3 = np.zeros((n, self.M, 3, 2))
        SA3 = np.zeros((n, self.M))
        rc = _load().or_field_vec(self._ctx, _ptr(rx), n, _ptr(E0), _ptr(S0), _ptr(A), _ptr(SA), _ptr(amb), _ptr(E03),
                                  _ptr(S03), _ptr(A3), _ptr(SA3))
        if rc:
            raise RuntimeError("or_field_vec failed")
        return dict(E0=E0[:, 0] + 1j * E0[:, 1], S0=S0, A=A[..., 0] + 1j * A[..., 1], SA=SA, amb=amb.astype(bool),
                    E03=E03[..., 0] + 1j * E03[..., 1], S03=S03, A3=A3[..., 0] + 1j * A3[..., 1], SA3=SA3)

    @staticmethod
    def evaluate_vec(fld: dict, gamma: np.ndarray):
        """Vector mode for configurations gamma [C, M]: received E, P = |E|^2 / (2 eta0), S (as
        ``evaluate``), the field vectors E3 [n, C, 3] and their incoherent magnitudes S3 [n, C]."""
        g = np.atleast_2d(np.asarray(gamma, np.complex128))
        E, P, S = Oracle.evaluate(fld, g)
        E3 = fld["E03"][:, None, :] + np.einsum("rmj,cm->rcj", fld["A3"], g)
        S3 = fld["S03"][:, None] + fld["SA3"] @ np.abs(g).T
        return E, P, S, E3, S3

    def cir(self, rx_xyz: np.ndarray, gamma: np.ndarray, cap: int = 4096):
        """RIS channel impulse response per receiver: a list of taps (Rx-leg id q, Tx-leg id p, delay in
        seconds through the RIS centre, complex amplitude sum_m Gamma_m e_mpq and its incoherent
        magnitude sabs), q-major in ascending ids (-1 = direct leg first)."""
        rx = np.ascontiguousarray(rx_xyz, np.float32).reshape(-1, 3)
        n = len(rx)
        g = np.asarray(gamma, np.complex128).ravel()
        gi = np.ascontiguousarray(np.stack([g.real, g.imag], 1))
        amp = np.zeros((n, cap, 2))
        sabs = np.zeros((n, cap))
        delay = np.zeros((n, cap))
        p_id = np.zeros((n, cap), np.int64)
        q_id = np.zeros((n, cap), np.int64)
        cnt = np.zeros(n, np.int32)
        _load().or_cir(self._ctx, _ptr(rx), n, _ptr(gi), cap, _ptr(amp), _ptr(sabs), _ptr(delay), _ptr(p_id), _ptr(q_id),
                       _ptr(cnt))
        if (cnt > cap).any():
            raise RuntimeError("oracle CIR capacity exceeded")
        return [dict(q=q_id[i, : cnt[i]].copy(), p=p_id[i, : cnt[i]].copy(), delay=delay[i, : cnt[i]].copy(),
                     amp=amp[i, : cnt[i], 0] + 1j * amp[i, : cnt[i], 1], sabs=sabs[i, : cnt[i]].copy())
                for i in range(n)]

    @staticmethod
    def evaluate(fld: dict, gamma: np.ndarray):
        """E, P (Eq. 9, Eq. 10) and the incoherent magnitude S for configuration(s) gamma [.., M]."""
        g = np.asarray(gamma, np.complex128)
        E = fld["E0"][:, None] + fld["A"] @ g.reshape(-1, g.shape[-1]).T
        S = fld["S0"][:, None] + fld["SA"] @ np.abs(g.reshape(-1, g.shape[-1])).T
        P = np.abs(E) ** 2 / (2 * ETA0)
        if g.ndim == 1:
            return E[:, 0], P[:, 0], S[:, 0]
        return E, P, S


def log_power_and_grad(fld: dict, phases: np.ndarray, amp=None):
    """Objective J_b = sum_r log P_b(r) over the receivers of ``fld`` and its analytic gradient with
    respect to every element phase, in FP64 (from Eq. 9 and Eq. 10):
    dJ/dphi_bm = sum_r 2 Re(conj(E_b(r)) dE_b(r)/dphi_bm) / |E_b(r)|^2, dE/dphi_bm = j A[r][m] Gamma_bm.
    |E|^2 is clamped below at 1e-30 of its maximum over the receivers of each configuration."""
    ph = np.atleast_2d(np.asarray(phases, np.float64))
    a = np.ones(ph.shape[1]) if amp is None else np.asarray(amp, np.float64)
    G = a[None, :] * np.exp(1j * ph)                       # [B, M]
    E = fld["E0"][None, :] + G @ fld["A"].T                # [B, n]
    p2 = np.abs(E) ** 2
    p2 = np.maximum(p2, 1e-30 * p2.max(axis=1, keepdims=True))
    J = np.sum(np.log(p2 / (2 * ETA0)), axis=1)
    dE = 1j * G[:, None, :] * fld["A"][None, :, :]         # [B, n, M]
    grad = np.sum(2 * np.real(np.conj(E)[:, :, None] * dE) / p2[:, :, None], axis=1)
    return J, grad
