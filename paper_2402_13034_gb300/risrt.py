"""Thin Python binding of the risrt C ABI (include/risrt.h).

Argument marshalling only: every step of the path runs in the CUDA library. Device buffers are
torch tensors (complex64 for complex arrays); host inputs are numpy arrays. If the compiled
library is missing, loading fails with an error instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librisrt.so")

OK = 0
TX, RX = 0, 1
PATTERN_ISO, PATTERN_COS_POW, PATTERN_MONOPOLE_QW = 0, 1, 2
FLAG_ENV_PATHS, FLAG_FRESNEL_TM = 1, 2
PREC_FP32, PREC_BF16, PREC_BF16X2, PREC_FP16 = 0, 1, 2, 3
GRAD_KEEP_A = 0x100
GRAD_DEFER_CHECK = 0x200
SWEEP_KEEP_A = 0x100
SWEEP_DEFER_CHECK = 0x200
MB_FFMA, MB_MUFU_SIN, MB_MUFU_COS, MB_MUFU_RSQ, MB_MUFU_RCP, MB_MUFU_SQRT, MB_MUFU_EX2, MB_DFMA = range(8)

_lock = threading.Lock()
_lib = None

# Every symbol the header declares, with (restype, argtypes).
_P = C.c_void_p
_SIGS = {
    "risrt_create": (C.c_int, [C.POINTER(_P), C.c_int, _P, C.c_size_t]),
    "risrt_set_stream": (C.c_int, [_P, _P]),
    "risrt_destroy": (C.c_int, [_P]),
    "risrt_last_error": (C.c_char_p, [_P]),
    "risrt_scene_upload": (C.c_int, [_P, _P, C.c_int64, _P, _P, _P, C.c_int64, _P, C.c_int32, C.POINTER(_P)]),
    "risrt_ris_upload": (C.c_int, [_P, _P, C.c_int32, _P, _P, _P, C.c_float, C.c_float, C.c_float, C.c_int32,
                                   C.POINTER(_P)]),
    "risrt_antenna_set": (C.c_int, [_P, C.c_int, _P, _P, C.c_float, C.c_float, C.c_int]),
    "risrt_rx_upload": (C.c_int, [_P, _P, C.c_int64, C.POINTER(_P)]),
    "risrt_rx_bind": (C.c_int, [_P, _P, C.c_int64, C.POINTER(_P)]),
    "risrt_trace_paths": (C.c_int, [_P, _P, _P, _P, C.c_double, C.c_int32, C.c_int32, C.c_uint32, C.POINTER(_P)]),
    "risrt_trace_workspace_size": (C.c_int, [_P, _P, _P, _P, C.c_int32, C.c_int32, C.c_uint32, _P, C.POINTER(C.c_size_t)]),
    "risrt_trace_paths_async": (C.c_int, [_P, _P, _P, _P, C.c_double, C.c_int32, C.c_int32, C.c_uint32, _P, _P,
                                          C.c_size_t, C.POINTER(_P)]),
    "risrt_trace_check": (C.c_int, [_P, _P]),
    "risrt_pathset_stats_get": (C.c_int, [_P, _P]),
    "risrt_pathset_export": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "risrt_eval_field": (C.c_int, [_P, _P, _P, C.c_int32, _P, _P]),
    "risrt_eval_field_plain": (C.c_int, [_P, _P, _P, C.c_int32, _P, _P]),
    "risrt_eval_cir": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "risrt_eval_field_strict": (C.c_int, [_P, _P, _P, _P, C.c_double, C.c_int32, C.c_int32, C.c_uint32, _P, C.c_int32,
                                          _P, _P]),
    "risrt_antenna_set_polarization": (C.c_int, [_P, C.c_int, _P]),
    "risrt_eval_field_vec": (C.c_int, [_P, _P, _P, _P, _P, C.c_int32, _P, _P, _P]),
    "risrt_build_A_vec": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "risrt_microbench": (C.c_int, [_P, C.c_int, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "risrt_build_A": (C.c_int, [_P, _P, _P, _P, C.POINTER(_P)]),
    "risrt_amat_wrap": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int32, C.POINTER(_P)]),
    "risrt_amat_data": (C.c_int, [_P, C.POINTER(_P), C.POINTER(_P), C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "risrt_amat_destroy": (C.c_int, [_P, _P]),
    "risrt_sweep_workspace_size": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.c_int, C.POINTER(C.c_size_t)]),
    "risrt_sweep_configs": (C.c_int, [_P, _P, _P, _P, C.c_float, C.c_int32, C.c_int, _P, _P, _P, C.c_size_t]),
    "risrt_sweep_fused": (C.c_int, [_P, _P, _P, _P, C.c_float, C.c_int32, _P, _P]),
    "risrt_sweep_check": (C.c_int, [_P, _P, C.c_size_t]),
    "risrt_grad_workspace_size": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int, C.POINTER(C.c_size_t)]),
    "risrt_grad_phases": (C.c_int, [_P, _P, _P, C.c_int32, _P, _P, C.c_int32, _P, _P, _P, C.c_size_t, C.c_int]),
    "risrt_grad_check": (C.c_int, [_P, _P, C.c_size_t]),
    "risrt_find_paths_noalloc": (C.c_int, [_P, _P, _P, C.c_int32, _P, C.c_int32, C.c_int32, _P, C.c_int32,
                                           C.POINTER(C.c_int32)]),
    "risrt_profile_enable": (C.c_int, [_P, C.c_int]),
    "risrt_profile_only": (C.c_int, [_P, C.c_char_p]),
    "risrt_profile_query": (C.c_int, [_P, C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "risrt_profile_names": (C.c_int, [_P, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "risrt_profile_reset": (C.c_int, [_P]),
    "risrt_launch_count": (C.c_int, [C.POINTER(C.c_int64)]),
    "risrt_scene_destroy": (C.c_int, [_P, _P]),
    "risrt_ris_destroy": (C.c_int, [_P, _P]),
    "risrt_rxset_destroy": (C.c_int, [_P, _P]),
    "risrt_pathset_destroy": (C.c_int, [_P, _P]),
}


class TraceLimits(C.Structure):
    _fields_ = [("cand_cap", C.c_int32), ("max_paths_per_rx", C.c_int32), ("max_env_paths_per_rx", C.c_int32)]


class RisrtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"risrt error {code}: {msg}")
        self.code = code


class PathsetStats(C.Structure):
    _fields_ = [("n_rx", C.c_int64), ("M", C.c_int32), ("n_faces", C.c_int32), ("n_rx_paths", C.c_int64),
                ("n_env_paths", C.c_int64), ("n_tx_paths", C.c_int32), ("units", C.c_int64),
                ("fp64_refines", C.c_int64), ("n_candidates", C.c_int64), ("n_segments", C.c_int64),
                ("node_visits", C.c_int64), ("tri_tests", C.c_int64)]


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load the compiled library (build it with paper_2402_13034_gb300.build.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RisrtError(-1, f"CUDA library not built: {path} is missing")
            lib = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _f32(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} floats, got {a.size}")
    return a


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p)
    return C.c_void_p(a.data_ptr())     # torch tensor


def _dev_ptr(t, dtype_name: str, numel: int | None = None):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("device arguments must be CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("device tensors must be contiguous")
    if str(t.dtype) != dtype_name:
        raise TypeError(f"expected {dtype_name}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


class _Handle:
    def __init__(self, ctx: "Context", ptr: C.c_void_p, destroy: str):
        self._ctx, self._ptr, self._destroy = ctx, ptr, destroy

    @property
    def ptr(self):
        return self._ptr

    def close(self):
        if self._ptr and self._ctx._ptr:
            getattr(load(), self._destroy)(self._ctx._ptr, self._ptr)
        self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Scene(_Handle):
    pass


class RIS(_Handle):
    def __init__(self, ctx, ptr, M):
        super().__init__(ctx, ptr, "risrt_ris_destroy")
        self.M = M


class RxSet(_Handle):
    def __init__(self, ctx, ptr, n, keep=None):
        super().__init__(ctx, ptr, "risrt_rxset_destroy")
        self.n = n
        self._keep = keep


class AMat(_Handle):
    """A channel matrix A [n_rx, M] and E0 [n_rx] on the device (owned by the library or a view)."""

    def __init__(self, ctx, ptr, n_rx, M, keep=None):
        super().__init__(ctx, ptr, "risrt_amat_destroy")
        self.n_rx, self.M = n_rx, M
        self._keep = keep

    def tensors(self):
        """(A, E0) as complex64 CUDA tensors sharing the device memory (E0 None if absent); valid while
        the handle lives."""
        import torch
        a, e = C.c_void_p(), C.c_void_p()
        rc = load().risrt_amat_data(self._ptr, C.byref(a), C.byref(e), None, None)
        if rc:
            raise RisrtError(rc, "amat data")

        def view(ptr, n):
            if not ptr.value:
                return None
            return torch.as_tensor(_DevBytes(ptr.value, n * 8), device=f"cuda:{self._ctx.device}").view(torch.complex64)
        A = view(a, self.n_rx * self.M)
        return A.view(self.n_rx, self.M), view(e, self.n_rx)


class _DevBytes:
    """A device byte range exposed through __cuda_array_interface__ (no copy, no ownership)."""

    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False), "version": 3}


class PathSet(_Handle):
    def stats(self) -> PathsetStats:
        st = PathsetStats()
        rc = load().risrt_pathset_stats_get(self._ptr, C.byref(st))
        if rc:
            raise RisrtError(rc, "pathset stats")
        return st

    def export(self) -> dict:
        st = self.stats()
        n, M = st.n_rx, st.M
        W = (M + 31) // 32
        rx_count = np.zeros(n, np.int32)
        rx_seq = np.zeros(max(st.n_rx_paths - n, 1), np.int64)
        env_count = np.zeros(n, np.int32)
        env_seq = np.zeros(max(st.n_env_paths, 1), np.int64)
        los = np.zeros(n, np.uint8)
        vis = np.zeros((n, W), np.uint32)
        tx_seq = np.zeros(max(st.n_tx_paths, 1), np.int64)
        tx_vis = np.zeros(M, np.uint8)
        rc = load().risrt_pathset_export(self._ptr, _ptr(rx_count), _ptr(rx_seq), _ptr(env_count), _ptr(env_seq),
                                         _ptr(los), _ptr(vis), _ptr(tx_seq), _ptr(tx_vis))
        if rc:
            raise RisrtError(rc, "pathset export")
        ro = np.concatenate([[0], np.cumsum(rx_count)])
        eo = np.concatenate([[0], np.cumsum(env_count)])
        return dict(seqs=[rx_seq[ro[i]:ro[i + 1]] for i in range(n)],
                    env=[env_seq[eo[i]:eo[i + 1]] for i in range(n)],
                    los=los.astype(bool), vis=vis, tx_seqs=tx_seq[: st.n_tx_paths], tx_vis=tx_vis.astype(bool),
                    stats=st)


class Context:
    """One device + stream. Methods mirror the C ABI; see include/risrt.h for semantics."""

    def __init__(self, device: int = 0, stream=None, hbm_budget: int = 0):
        lib = load()
        self._ptr = C.c_void_p()
        s = None if stream is None else C.c_void_p(stream)
        rc = lib.risrt_create(C.byref(self._ptr), device, s, int(hbm_budget))
        if rc:
            raise RisrtError(rc, lib.risrt_last_error(None).decode())
        self.device = device
        self.stream = stream

    def _check(self, rc: int):
        if rc:
            raise RisrtError(rc, load().risrt_last_error(self._ptr).decode())

    def close(self):
        if self._ptr:
            load().risrt_destroy(self._ptr)
        self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_handle: int | None):
        self._check(load().risrt_set_stream(self._ptr, None if stream_handle is None else C.c_void_p(stream_handle)))
        self.stream = stream_handle

    # --- tracing -------------------------------------------------------------------------------
    def profile_enable(self, on: bool = True):
        self._check(load().risrt_profile_enable(self._ptr, int(on)))

    def profile_only(self, name=None):
        """Bracket only the kernels called `name` while profiling (None: all kernels)."""
        self._check(load().risrt_profile_only(self._ptr, name.encode() if name else None))

    def profile_reset(self):
        self._check(load().risrt_profile_reset(self._ptr))

    def profile(self) -> dict:
        """{kernel name: (total ms, launches)} since the last reset (synchronises)."""
        need = C.c_size_t()
        self._check(load().risrt_profile_names(self._ptr, None, 0, C.byref(need)))
        buf = C.create_string_buffer(need.value)
        self._check(load().risrt_profile_names(self._ptr, buf, need.value, None))
        out = {}
        for name in filter(None, buf.value.decode().split(",")):
            ms, n = C.c_double(), C.c_int64()
            self._check(load().risrt_profile_query(self._ptr, name.encode(), C.byref(ms), C.byref(n)))
            out[name] = (ms.value, n.value)
        return out

    # --- inputs --------------------------------------------------------------------------------
    def scene_upload(self, verts, tris, face_id, mat_id, mats) -> Scene:
        v = _f32(verts)
        t = np.ascontiguousarray(tris, np.int32)
        f = np.ascontiguousarray(face_id, np.int32)
        m = np.ascontiguousarray(mat_id, np.int32)
        mt = _f32(mats)
        out = C.c_void_p()
        self._check(load().risrt_scene_upload(self._ptr, _ptr(v), v.size // 3, _ptr(t), _ptr(f), _ptr(m),
                                              t.size // 3, _ptr(mt), mt.size // 2, C.byref(out)))
        return Scene(self, out, "risrt_scene_destroy")

    def ris_upload(self, elem_uv, center, t1, t2, dy, dz, elem_gain=0.0, host_face=-1) -> RIS:
        uv = _f32(elem_uv)
        out = C.c_void_p()
        self._check(load().risrt_ris_upload(self._ptr, _ptr(uv), uv.size // 2, _ptr(_f32(center, 3)),
                                            _ptr(_f32(t1, 3)), _ptr(_f32(t2, 3)), float(dy), float(dz),
                                            float(elem_gain), int(host_face), C.byref(out)))
        return RIS(self, out, uv.size // 2)

    def antenna_set(self, which, pos, orient, power_w, gain_lin, pattern):
        p = _f32(pos if pos is not None else np.zeros(3), 3)
        o = _f32(orient, 9)
        self._check(load().risrt_antenna_set(self._ptr, which, _ptr(p), _ptr(o), float(power_w), float(gain_lin),
                                             int(pattern)))

    def antenna_set_polarization(self, which, axis):
        """Polarisation axis (global frame) of the Tx or Rx antenna for the vector field."""
        a = _f32(axis, 3)
        self._check(load().risrt_antenna_set_polarization(self._ptr, which, _ptr(a)))

    def rx_upload(self, rx_xyz) -> RxSet:
        r = _f32(rx_xyz)
        out = C.c_void_p()
        self._check(load().risrt_rx_upload(self._ptr, _ptr(r), r.size // 3, C.byref(out)))
        return RxSet(self, out, r.size // 3)

    def rx_bind(self, rx_xyz_dev) -> RxSet:
        out = C.c_void_p()
        self._check(load().risrt_rx_bind(self._ptr, _dev_ptr(rx_xyz_dev, "torch.float32"), rx_xyz_dev.numel() // 3,
                                         C.byref(out)))
        return RxSet(self, out, rx_xyz_dev.numel() // 3, keep=rx_xyz_dev)

    # --- path finding and fields -----------------------------------------------------------------
    def trace_paths(self, scene: Scene, ris: RIS, rxset: RxSet, freq_hz: float, max_order_tx: int,
                    max_order_rx: int, flags: int = 0, reuse: PathSet | None = None) -> PathSet:
        ptr = reuse.ptr if reuse is not None else C.c_void_p()
        self._check(load().risrt_trace_paths(self._ptr, scene.ptr, ris.ptr, rxset.ptr, float(freq_hz),
                                             int(max_order_tx), int(max_order_rx), int(flags), C.byref(ptr)))
        return reuse if reuse is not None else PathSet(self, ptr, "risrt_pathset_destroy")

    def trace_workspace(self, scene: Scene, ris: RIS, rxset: RxSet, max_order_tx: int, max_order_rx: int,
                        flags: int = 0, cand_cap: int = 512, max_paths: int = 64, max_env: int = 64):
        """(workspace tensor, limits) for trace_paths_async."""
        import torch
        lim = TraceLimits(cand_cap, max_paths, max_env)
        nb = C.c_size_t()
        self._check(load().risrt_trace_workspace_size(self._ptr, scene.ptr, ris.ptr, rxset.ptr, int(max_order_tx),
                                                      int(max_order_rx), int(flags), C.byref(lim), C.byref(nb)))
        return torch.empty(nb.value + 256, dtype=torch.uint8, device=f"cuda:{self.device}"), lim

    def trace_paths_async(self, scene: Scene, ris: RIS, rxset: RxSet, freq_hz: float, max_order_tx: int,
                          max_order_rx: int, flags: int, workspace, limits, reuse: PathSet | None = None) -> PathSet:
        """Enqueue a trace into the workspace (no synchronisation, no allocation); trace_check before reading
        counts or exporting."""
        ptr = reuse.ptr if reuse is not None else C.c_void_p()
        base = (workspace.data_ptr() + 255) // 256 * 256
        nbytes = workspace.numel() - (base - workspace.data_ptr())
        self._check(load().risrt_trace_paths_async(self._ptr, scene.ptr, ris.ptr, rxset.ptr, float(freq_hz),
                                                   int(max_order_tx), int(max_order_rx), int(flags), C.byref(limits),
                                                   C.c_void_p(base), nbytes, C.byref(ptr)))
        if reuse is not None:
            return reuse
        ps = PathSet(self, ptr, "risrt_pathset_destroy")
        ps._keep = workspace
        return ps

    def trace_check(self, ps: PathSet):
        self._check(load().risrt_trace_check(self._ptr, ps.ptr))

    def eval_field(self, ps: PathSet, gamma, E_out, P_out=None):
        """gamma: complex64 CUDA [C, M]; E_out: complex64 CUDA [C, n_rx]; P_out: float32 CUDA [C, n_rx]."""
        n_cfg = gamma.shape[0] if gamma.dim() == 2 else 1
        self._check(load().risrt_eval_field(self._ptr, ps.ptr, _dev_ptr(gamma, "torch.complex64"), n_cfg,
                                            _dev_ptr(E_out, "torch.complex64"), _dev_ptr(P_out, "torch.float32")))

    def eval_field_plain(self, ps: PathSet, gamma, E_out, P_out=None):
        """The plain FP32 baseline of eval_field (same arguments and outputs)."""
        n_cfg = gamma.shape[0] if gamma.dim() == 2 else 1
        self._check(load().risrt_eval_field_plain(self._ptr, ps.ptr, _dev_ptr(gamma, "torch.complex64"), n_cfg,
                                                  _dev_ptr(E_out, "torch.complex64"), _dev_ptr(P_out, "torch.float32")))

    def eval_field_strict(self, scene: Scene, ris: RIS, rxset: RxSet, freq_hz: float, max_order_tx: int,
                          max_order_rx: int, flags: int, gamma, E_out, P_out=None):
        """The field with every element's reflected legs validated at the element itself (strict mode);
        gamma complex64 CUDA [C, M], E_out complex64 [C, n_rx], P_out float32 [C, n_rx] or None."""
        n_cfg = gamma.shape[0] if gamma.dim() == 2 else 1
        self._check(load().risrt_eval_field_strict(self._ptr, scene.ptr, ris.ptr, rxset.ptr, float(freq_hz),
                                                   int(max_order_tx), int(max_order_rx), int(flags),
                                                   _dev_ptr(gamma, "torch.complex64"), n_cfg,
                                                   _dev_ptr(E_out, "torch.complex64"), _dev_ptr(P_out, "torch.float32")))

    def eval_field_vec(self, scene: Scene, rxset: RxSet, ps: PathSet, gamma, E_out, E3_out=None, P_out=None):
        """Vector field with polarisation over the paths of ps (traced with scene and rxset): received
        values E_out complex64 [C, n_rx], field vectors E3_out complex64 [C, n_rx, 3] or None, P_out
        float32 [C, n_rx] or None; gamma complex64 CUDA [C, M]."""
        n_cfg = gamma.shape[0] if gamma.dim() == 2 else 1
        self._check(load().risrt_eval_field_vec(self._ptr, scene.ptr, rxset.ptr, ps.ptr,
                                                _dev_ptr(gamma, "torch.complex64"), n_cfg,
                                                _dev_ptr(E_out, "torch.complex64"), _dev_ptr(E3_out, "torch.complex64"),
                                                _dev_ptr(P_out, "torch.float32")))

    def build_A_vec(self, scene: Scene, rxset: RxSet, ps: PathSet, A_out, E0_out=None):
        """Channel matrix of the vector field's received values into A_out [n_rx, M] and E0_out [n_rx]
        (complex64 CUDA)."""
        self._check(load().risrt_build_A_vec(self._ptr, scene.ptr, rxset.ptr, ps.ptr, _dev_ptr(A_out, "torch.complex64"),
                                             _dev_ptr(E0_out, "torch.complex64")))

    def eval_cir(self, ps: PathSet, gamma):
        """RIS channel impulse response for one configuration gamma (complex64 CUDA [M]): returns
        (taps complex64 [n_rx_paths, n_tx_paths + 1], rx_delay float64 [n_rx_paths], tx_delay float64
        [n_tx_paths + 1]) as CUDA tensors (entries receiver-major as in PathSet.export)."""
        import torch
        st = ps.stats()
        P = st.n_tx_paths + 1
        dev = f"cuda:{self.device}"
        taps = torch.empty((st.n_rx_paths, P), dtype=torch.complex64, device=dev)
        rxd = torch.empty(st.n_rx_paths, dtype=torch.float64, device=dev)
        txd = torch.empty(P, dtype=torch.float64, device=dev)
        self._check(load().risrt_eval_cir(self._ptr, ps.ptr, _dev_ptr(gamma, "torch.complex64"),
                                          _dev_ptr(taps, "torch.complex64"), _dev_ptr(rxd, "torch.float64"),
                                          _dev_ptr(txd, "torch.float64")))
        return taps, rxd, txd

    def microbench(self, kind: int, iters: int = 4096):
        """Issue rate of one pipe (MB_* kinds): (lane operations per second, ms of the best launch)."""
        ops, ms = C.c_double(), C.c_double()
        self._check(load().risrt_microbench(self._ptr, int(kind), int(iters), C.byref(ops), C.byref(ms)))
        return ops.value, ms.value

    def sweep_workspace(self, n_rx: int, M: int, n_cfg: int, precision: int):
        """A device workspace tensor for sweep_configs (None for FP32)."""
        import torch
        nb = C.c_size_t()
        rc = load().risrt_sweep_workspace_size(int(n_rx), int(M), int(n_cfg), int(precision), C.byref(nb))
        if rc:
            raise RisrtError(rc, "sweep workspace size")
        if nb.value == 0:
            return None
        return torch.empty(nb.value, dtype=torch.uint8, device=f"cuda:{self.device}")

    def amat(self, A, E0=None) -> "AMat":
        """A channel-matrix handle viewing the complex64 CUDA tensors A [n_rx, M] and E0 [n_rx] (or None)."""
        n_rx, M = A.shape
        out = C.c_void_p()
        self._check(load().risrt_amat_wrap(self._ptr, _dev_ptr(A, "torch.complex64"), _dev_ptr(E0, "torch.complex64"),
                                           int(n_rx), int(M), C.byref(out)))
        return AMat(self, out, int(n_rx), int(M), keep=(A, E0))

    def _as_amat(self, A, E0):
        return A if isinstance(A, AMat) else self.amat(A, E0)

    def sweep_fused(self, ps: PathSet, gamma, P_out=None, gamma_2bit=None, amp: float = 1.0, E_out=None):
        """Fused channel tile -> tensor-core sweep over a path set (A never materialised), at most 128
        configurations: gamma complex64 CUDA [C, M] (or gamma_2bit uint8 [C, ceil(M/4)] with amp);
        P_out float32 [n_rx, C] and/or E_out complex64 [n_rx, C]."""
        n_cfg = gamma.shape[0] if gamma is not None else gamma_2bit.shape[0]
        self._check(load().risrt_sweep_fused(self._ptr, ps.ptr, _dev_ptr(gamma, "torch.complex64"),
                                             _dev_ptr(gamma_2bit, "torch.uint8"), float(amp), int(n_cfg),
                                             _dev_ptr(P_out, "torch.float32"), _dev_ptr(E_out, "torch.complex64")))

    def sweep_configs(self, A, E0, gamma, P_out, precision: int, workspace=None, keep_a: bool = False,
                      defer_check: bool = False, gamma_2bit=None, amp: float = 1.0, E_out=None):
        """A: complex64 CUDA [n_rx, M] (with E0 complex64 [n_rx] or None) or an AMat handle (E0 ignored);
        gamma: complex64 [C, M], or None with gamma_2bit: uint8 CUDA [C, ceil(M/4)] codes (Gamma = amp j^q);
        P_out: float32 [n_rx, C] or None; E_out: complex64 [n_rx, C] or None. keep_a: reuse A as packed into
        the workspace by an earlier call; defer_check: enqueue only (capturable), check later with
        sweep_check."""
        h = self._as_amat(A, E0)
        n_cfg = gamma.shape[0] if gamma is not None else gamma_2bit.shape[0]
        ws_ptr = None if workspace is None else C.c_void_p(workspace.data_ptr())
        ws_n = 0 if workspace is None else workspace.numel()
        opts = (SWEEP_KEEP_A if keep_a else 0) | (SWEEP_DEFER_CHECK if defer_check else 0)
        self._check(load().risrt_sweep_configs(self._ptr, h.ptr, _dev_ptr(gamma, "torch.complex64"),
                                               _dev_ptr(gamma_2bit, "torch.uint8"), float(amp), int(n_cfg),
                                               int(precision) | opts, _dev_ptr(P_out, "torch.float32"),
                                               _dev_ptr(E_out, "torch.complex64"), ws_ptr, ws_n))

    def sweep_check(self, workspace):
        """Waits for the stream; raises RisrtError if a deferred-check sweep on this workspace timed out."""
        self._check(load().risrt_sweep_check(self._ptr, C.c_void_p(workspace.data_ptr()), workspace.numel()))

    def grad_workspace(self, n_target: int, B: int, M: int, precision: int = PREC_FP32):
        import torch
        nb = C.c_size_t()
        rc = load().risrt_grad_workspace_size(int(n_target), int(B), int(M), int(precision), C.byref(nb))
        if rc:
            raise RisrtError(rc, "grad workspace size")
        return torch.empty(nb.value, dtype=torch.uint8, device=f"cuda:{self.device}")

    def grad_phases(self, A, E0, target, phases, amp, J_out, grad_out, workspace=None, precision: int = PREC_FP32,
                    keep_a: bool = False, defer_check: bool = False):
        """A: complex64 CUDA [n_rx, M] (with E0) or an AMat; target: int32 CUDA [n_t] or None (first n_t rows given by
        phases' companion J); phases: float32 [B, M]; amp: float32 [M] or None; J_out [B]; grad_out [B, M];
        precision PREC_FP32 (CUDA cores) or PREC_BF16X2 (tensor cores, split BF16); keep_a: A, E0 and target
        are those of the previous call with this workspace (its packed A is reused); defer_check: enqueue only (no
        synchronisation), check later with grad_check."""
        h = self._as_amat(A, E0)
        n_rx, M = h.n_rx, h.M
        B = phases.shape[0]
        n_t = target.numel() if target is not None else n_rx
        ws = workspace if workspace is not None else self.grad_workspace(n_t, B, M, precision)
        self._check(load().risrt_grad_phases(self._ptr, h.ptr, _dev_ptr(target, "torch.int32"), int(n_t),
                                             _dev_ptr(phases, "torch.float32"), _dev_ptr(amp, "torch.float32"), int(B),
                                             _dev_ptr(J_out, "torch.float32"), _dev_ptr(grad_out, "torch.float32"),
                                             C.c_void_p(ws.data_ptr()), ws.numel(),
                                             int(precision) | (GRAD_KEEP_A if keep_a else 0)
                                             | (GRAD_DEFER_CHECK if defer_check else 0)))

    def grad_check(self, workspace):
        """Timeout flag of the last deferred grad_phases on this workspace (waits for the stream)."""
        self._check(load().risrt_grad_check(self._ptr, C.c_void_p(workspace.data_ptr()), workspace.numel()))

    def find_paths_noalloc(self, scene: Scene, src, src_face: int, dst, dst_face: int, max_order: int,
                           cap: int = 4096) -> np.ndarray:
        """Reflected face-sequence ids between two points without any device allocation."""
        ids = np.zeros(max(cap, 1), np.int64)
        n = C.c_int32()
        self._check(load().risrt_find_paths_noalloc(self._ptr, scene.ptr, _ptr(_f32(src, 3)), int(src_face),
                                                     _ptr(_f32(dst, 3)), int(dst_face), int(max_order), _ptr(ids),
                                                     int(cap), C.byref(n)))
        return ids[: n.value].copy()

    def build_A(self, ps: PathSet, A_out=None, E0_out=None, resident: bool = False):
        """Channel matrix into A_out [n_rx, M] / E0_out [n_rx] (complex64 CUDA). With A_out None the
        library keeps A and E0 resident and an AMat owning them is returned; with resident=True and
        A_out given, an AMat viewing A_out / E0_out is returned."""
        out = C.c_void_p()
        want = A_out is None or resident
        self._check(load().risrt_build_A(self._ptr, ps.ptr, _dev_ptr(A_out, "torch.complex64"),
                                         _dev_ptr(E0_out, "torch.complex64"), C.byref(out) if want else None))
        if not want:
            return None
        st = ps.stats()
        return AMat(self, out, st.n_rx, st.M, keep=(A_out, E0_out) if A_out is not None else None)


def launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    n = C.c_int64()
    rc = load().risrt_launch_count(C.byref(n))
    if rc:
        raise RisrtError(rc, "launch count")
    return n.value


def flags_of(w) -> int:
    return FLAG_ENV_PATHS if w.env_paths else 0


def upload_workload(ctx: Context, w, rx_device=None):
    """Upload a scenarios.Workload (scene, RIS, antennas, receivers). Receivers come from host
    memory unless ``rx_device`` (a float32 CUDA tensor [n,3]) is given."""
    sc = w.scene
    scene = ctx.scene_upload(sc.verts, sc.tris, sc.face_id, sc.mat_id, sc.mats)
    ris = ctx.ris_upload(w.ris.elem_uv, w.ris.center, w.ris.t1, w.ris.t2, w.ris.dy, w.ris.dz, w.ris.elem_gain,
                         w.ris.host_face)
    ctx.antenna_set(TX, w.tx.pos, w.tx.orient, w.tx.power_w, w.tx.gain_lin, w.tx.pattern)
    ctx.antenna_set(RX, None, w.rx.orient, w.rx.power_w, w.rx.gain_lin, w.rx.pattern)
    if getattr(w.tx, "pol", None) is not None:
        ctx.antenna_set_polarization(TX, w.tx.pol)
    if getattr(w.rx, "pol", None) is not None:
        ctx.antenna_set_polarization(RX, w.rx.pol)
    rx = ctx.rx_bind(rx_device) if rx_device is not None else ctx.rx_upload(w.rx_xyz)
    return scene, ris, rx
