"""Thin ctypes binding of ``libaxlbm`` (include/axlbm.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  The functions keep the C names; :class:`Domain` bundles a handle
with PyTorch-owned device memory and the caller's CUDA stream.  Importing this
module loads the library and raises ``RuntimeError`` if it is missing; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import inputs as _inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libaxlbm.so")

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, EUNSUPPORTED = range(7)
FP64, FP32, FP16_DEV, BF16_DEV = range(4)
PRECISIONS = {"fp64": FP64, "fp32": FP32, "fp16": FP16_DEV, "bf16": BF16_DEV}
INNER_AXIS, INNER_WALL, INNER_AXIS_NODE = 0, 1, 2
Z_PERIODIC, Z_WALL, Z_FREE, Z_MIXED, Z_NEE, Z_HALO = range(6)
FACE_INNER, FACE_OUTER, FACE_LO, FACE_HI = range(4)
OUTER_BB, OUTER_NEE, OUTER_ZOUHE = 0, 1, 2
RHO, UR, UZ, UTH, T = 1, 2, 4, 8, 16
F64, F32 = 0, 1
BGK, MRT = 0, 1
_ZKIND = {"periodic": Z_PERIODIC, "wall": Z_WALL, "free": Z_FREE, "mixed": Z_MIXED, "nee": Z_NEE, "halo": Z_HALO}
_OUTER = {"wall": OUTER_BB, "nee": OUTER_NEE, "zou_he": OUTER_ZOUHE}
_INNER = {"axis": INNER_AXIS, "wall": INNER_WALL, "axis_node": INNER_AXIS_NODE}


class axlbm_grid(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int32), ("nz", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("with_swirl", ctypes.c_int32), ("with_temperature", ctypes.c_int32),
                ("collision", ctypes.c_int32), ("r0", ctypes.c_double)]


class axlbm_forcing(ctypes.Structure):
    _fields_ = [("rho0", ctypes.c_double), ("az0", ctypes.c_double), ("omega_t", ctypes.c_double),
                ("gbeta", ctypes.c_double), ("t_ref", ctypes.c_double), ("tau_t", ctypes.c_double),
                ("t_init", ctypes.c_double), ("mrt_s_eps", ctypes.c_double), ("mrt_s_q", ctypes.c_double)]


class axlbm_ws_domain(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int32), ("nz", ctypes.c_int32), ("r_first", ctypes.c_double),
                ("r_wall", ctypes.c_double), ("z_first", ctypes.c_double), ("z_bottom", ctypes.c_double),
                ("height", ctypes.c_double), ("rho0", ctypes.c_double), ("u_scale", ctypes.c_double),
                ("t_ref", ctypes.c_double)]


class axlbm_boundary(ctypes.Structure):
    _fields_ = [("inner", ctypes.c_int32), ("z_lo", ctypes.c_int32), ("z_hi", ctypes.c_int32),
                ("t_dirichlet", ctypes.c_int32 * 4), ("outer", ctypes.c_int32),
                ("r_split", ctypes.c_double), ("omega", ctypes.c_double * 4),
                ("t_wall", ctypes.c_double * 4)]


class axlbm_domain(ctypes.Structure):
    _fields_ = [("grid", axlbm_grid), ("tau", ctypes.c_double), ("forcing", axlbm_forcing),
                ("boundary", axlbm_boundary)]


class AxlbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"axlbm status {status}: {message}")
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libaxlbm; raises RuntimeError when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libaxlbm is not built ({LIB_PATH} missing); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        H = ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        L.axlbm_abi_version.restype = ctypes.c_int32
        L.axlbm_abi_version.argtypes = []
        L.axlbm_status_string.restype = ctypes.c_char_p
        L.axlbm_status_string.argtypes = [ctypes.c_int]
        L.axlbm_state_bytes.argtypes = [ctypes.POINTER(axlbm_grid), ctypes.POINTER(ctypes.c_size_t)]
        L.axlbm_create.argtypes = [ctypes.POINTER(axlbm_grid), ctypes.c_double, ctypes.POINTER(axlbm_forcing),
                                   ctypes.POINTER(axlbm_boundary), ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_size_t, ctypes.POINTER(H)]
        L.axlbm_step.argtypes = [H, ctypes.c_int64]
        L.axlbm_moments.argtypes = [H, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]
        L.axlbm_residual.argtypes = [H, dp, dp, dp]
        L.axlbm_set_fields.argtypes = [H, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]
        L.axlbm_get_populations.argtypes = [H, dp, dp, dp]
        L.axlbm_set_populations.argtypes = [H, dp, dp, dp, ctypes.c_int64]
        L.axlbm_time.argtypes = [H, ctypes.POINTER(ctypes.c_int64)]
        L.axlbm_destroy.argtypes = [H]
        L.axlbm_kernel_timing.argtypes = [H, ctypes.c_int32]
        L.axlbm_use_graphs.argtypes = [H, ctypes.c_int32]
        L.axlbm_set_residual_lag.argtypes = [H, ctypes.c_int32]
        L.axlbm_halo_bytes.argtypes = [H, ctypes.POINTER(ctypes.c_size_t)]
        L.axlbm_halo_send.argtypes = [H, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32]
        L.axlbm_halo_recv.argtypes = [H, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32]
        L.axlbm_batch_set_residual_lag.argtypes = [H, ctypes.c_int32]
        L.axlbm_graph_stats.argtypes = [H, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        L.axlbm_kernel_times.argtypes = [H, ctypes.POINTER(ctypes.c_int64), dp, dp, ctypes.POINTER(ctypes.c_int64)]
        L.axlbm_check_static.argtypes = [ctypes.POINTER(axlbm_grid), ctypes.c_double,
                                         ctypes.POINTER(axlbm_forcing), ctypes.POINTER(axlbm_boundary),
                                         ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p]
        L.axlbm_last_error.restype = ctypes.c_char_p
        L.axlbm_last_error.argtypes = [H]
        DP = ctypes.POINTER(axlbm_domain)
        L.axlbm_batch_state_bytes.argtypes = [DP, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]
        L.axlbm_batch_create.argtypes = [DP, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_size_t, ctypes.POINTER(H)]
        L.axlbm_batch_step.argtypes = [H, ctypes.c_int64]
        L.axlbm_batch_residuals.argtypes = [H, dp]
        L.axlbm_batch_moments.argtypes = [H, ctypes.c_int32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.c_int32]
        L.axlbm_batch_set_fields.argtypes = [H, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]
        L.axlbm_batch_get_populations.argtypes = [H, ctypes.c_int32, dp, dp, dp]
        L.axlbm_batch_set_fields_all.argtypes = [H, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]
        L.axlbm_batch_moments_all.argtypes = [H, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]
        L.axlbm_batch_set_populations.argtypes = [H, ctypes.c_int32, dp, dp, dp]
        L.axlbm_batch_time.argtypes = [H, ctypes.POINTER(ctypes.c_int64)]
        L.axlbm_batch_tile_shape.argtypes = [H, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
        L.axlbm_selftest_bounded_wait.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                                                  ctypes.POINTER(ctypes.c_uint32)]
        L.axlbm_selftest_rcp.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        L.axlbm_batch_set_tile_shape.argtypes = [H, ctypes.c_int32, ctypes.c_int32]
        L.axlbm_batch_set_tile_shapes.argtypes = [H, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
        L.axlbm_batch_tile_shapes.argtypes = [H, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
        L.axlbm_batch_set_fields_all_async.argtypes = [H, ctypes.c_void_p, ctypes.c_int32]
        L.axlbm_batch_moments_all_async.argtypes = [H, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int32]
        L.axlbm_batch_sync.argtypes = [H]
        L.axlbm_batch_use_graphs.argtypes = [H, ctypes.c_int32]
        L.axlbm_batch_set_time.argtypes = [H, ctypes.c_int64]
        for pre in ("axlbm_", "axlbm_batch_"):
            getattr(L, pre + "save").argtypes = [H, ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
            getattr(L, pre + "save").restype = ctypes.c_int
            getattr(L, pre + "load").argtypes = [H, ctypes.c_void_p, ctypes.c_size_t]
            getattr(L, pre + "load").restype = ctypes.c_int
        L.axlbm_batch_copy_domain.argtypes = [H, ctypes.c_int32, H, ctypes.c_int32]
        L.axlbm_batch_graph_stats.argtypes = [H, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        L.axlbm_batch_kernel_timing.argtypes = [H, ctypes.c_int32]
        L.axlbm_batch_kernel_times.argtypes = [H, ctypes.POINTER(ctypes.c_int64), dp, dp, ctypes.POINTER(ctypes.c_int64)]
        L.axlbm_batch_kernel_times_by_parity.argtypes = [H, ctypes.POINTER(ctypes.c_int64), dp, dp]
        L.axlbm_batch_destroy.argtypes = [H]
        L.axlbm_batch_last_error.restype = ctypes.c_char_p
        L.axlbm_batch_last_error.argtypes = [H]
        V = ctypes.c_void_p
        L.axlbm_ws_weight_count.restype = ctypes.c_size_t
        L.axlbm_ws_weight_count.argtypes = []
        L.axlbm_ws_create.argtypes = [V, ctypes.c_size_t, V, ctypes.POINTER(V)]
        L.axlbm_ws_predict.argtypes = [V, V, ctypes.c_int32, V]
        L.axlbm_ws_fields.argtypes = [V, V, ctypes.c_int32, ctypes.POINTER(axlbm_ws_domain), V]
        L.axlbm_ws_destroy.argtypes = [V]
        L.axlbm_ws_to_canvas.argtypes = [V, V, ctypes.c_int32, ctypes.POINTER(axlbm_ws_domain), V]
        L.axlbm_ws_train_step.argtypes = [V, V, V, ctypes.c_int32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                          ctypes.c_float, ctypes.POINTER(ctypes.c_double)]
        L.axlbm_ws_loss.argtypes = [V, V, V, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
        L.axlbm_ws_get_weights.argtypes = [V, V]
        L.axlbm_ws_last_gradient.argtypes = [V, V]
        L.axlbm_ws_last_error.restype = ctypes.c_char_p
        L.axlbm_ws_last_error.argtypes = [V]
        for name in ("axlbm_ws_create", "axlbm_ws_predict", "axlbm_ws_fields", "axlbm_ws_destroy", "axlbm_ws_to_canvas",
                     "axlbm_ws_train_step", "axlbm_ws_loss", "axlbm_ws_get_weights", "axlbm_ws_last_gradient"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("axlbm_batch_state_bytes", "axlbm_batch_create", "axlbm_batch_step", "axlbm_batch_residuals",
                     "axlbm_batch_moments", "axlbm_batch_set_fields", "axlbm_batch_get_populations",
                     "axlbm_batch_set_populations", "axlbm_batch_time", "axlbm_batch_tile_shape",
                     "axlbm_batch_set_tile_shape", "axlbm_batch_set_tile_shapes", "axlbm_batch_tile_shapes", "axlbm_batch_use_graphs", "axlbm_batch_graph_stats",
                     "axlbm_batch_set_time", "axlbm_batch_copy_domain", "axlbm_batch_set_residual_lag",
                     "axlbm_batch_set_fields_all_async", "axlbm_batch_moments_all_async", "axlbm_batch_sync",
                     "axlbm_batch_kernel_timing", "axlbm_batch_kernel_times", "axlbm_batch_kernel_times_by_parity",
                     "axlbm_batch_destroy",
                     "axlbm_batch_set_fields_all", "axlbm_batch_moments_all"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("axlbm_state_bytes", "axlbm_create", "axlbm_step", "axlbm_moments", "axlbm_residual",
                     "axlbm_set_fields", "axlbm_get_populations", "axlbm_set_populations", "axlbm_time",
                     "axlbm_destroy", "axlbm_kernel_timing", "axlbm_kernel_times", "axlbm_check_static",
                     "axlbm_use_graphs", "axlbm_graph_stats", "axlbm_set_residual_lag",
                     "axlbm_halo_bytes", "axlbm_halo_send", "axlbm_halo_recv",
                     "axlbm_selftest_bounded_wait", "axlbm_selftest_rcp"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(status: int, handle=None) -> int:
    if status != OK:
        msg = lib().axlbm_last_error(handle).decode(errors="replace")
        raise AxlbmError(status, msg or lib().axlbm_status_string(status).decode())
    return status


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ----------------------------------------------------------------------------- C-named wrappers


def axlbm_abi_version() -> int:
    return int(lib().axlbm_abi_version())


def axlbm_state_bytes(grid: axlbm_grid) -> int:
    n = ctypes.c_size_t()
    _check(lib().axlbm_state_bytes(ctypes.byref(grid), ctypes.byref(n)))
    return int(n.value)


def axlbm_create(grid: axlbm_grid, tau: float, forcing: axlbm_forcing, boundary: axlbm_boundary,
                 stream: int = 0, state_mem: int = 0, state_bytes: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().axlbm_create(ctypes.byref(grid), float(tau), ctypes.byref(forcing), ctypes.byref(boundary),
                              ctypes.c_void_p(stream or None), ctypes.c_void_p(state_mem or None),
                              ctypes.c_size_t(state_bytes), ctypes.byref(h)))
    return h


def axlbm_step(h, n: int) -> None:
    _check(lib().axlbm_step(h, int(n)), h)


def axlbm_moments(h, mask: int, out_ptr: int, out_dtype: int, out_on_device: int) -> None:
    _check(lib().axlbm_moments(h, int(mask), ctypes.c_void_p(out_ptr), int(out_dtype), int(out_on_device)), h)


def axlbm_residual(h, allow_nonfinite: bool = False):
    r, m, b = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    st = lib().axlbm_residual(h, ctypes.byref(r), ctypes.byref(m), ctypes.byref(b))
    if not (allow_nonfinite and st == ENONFINITE):
        _check(st, h)
    return r.value, m.value, b.value


def axlbm_set_fields(h, ptr: int, in_dtype: int, on_device: int) -> None:
    _check(lib().axlbm_set_fields(h, ctypes.c_void_p(ptr), int(in_dtype), int(on_device)), h)


def axlbm_get_populations(h, f: np.ndarray, g: Optional[np.ndarray], t_pop: Optional[np.ndarray]) -> None:
    _check(lib().axlbm_get_populations(h, _dptr(f), _dptr(g), _dptr(t_pop)), h)


def axlbm_set_populations(h, f: np.ndarray, g: Optional[np.ndarray], t_pop: Optional[np.ndarray],
                          time: int) -> None:
    _check(lib().axlbm_set_populations(h, _dptr(f), _dptr(g), _dptr(t_pop), int(time)), h)


def axlbm_time(h) -> int:
    t = ctypes.c_int64()
    _check(lib().axlbm_time(h, ctypes.byref(t)), h)
    return int(t.value)


def axlbm_kernel_timing(h, enable: bool) -> None:
    _check(lib().axlbm_kernel_timing(h, int(bool(enable))), h)


def axlbm_kernel_times(h):
    """(bulk launches, bulk device ms, bulk algorithmic bytes, all launches)."""
    nb, na = ctypes.c_int64(), ctypes.c_int64()
    ms, by = ctypes.c_double(), ctypes.c_double()
    _check(lib().axlbm_kernel_times(h, ctypes.byref(nb), ctypes.byref(ms), ctypes.byref(by), ctypes.byref(na)), h)
    return int(nb.value), ms.value, by.value, int(na.value)


def axlbm_check_static(grid: axlbm_grid, tau: float, forcing: axlbm_forcing, bc, f_ptr: int, g_ptr: int,
                       t_ptr: int, a_z: float, speed_prev_ptr: int, speed_out_ptr: int, out_ptr: int,
                       stream: int = 0) -> None:
    """Check-step statistics over caller device buffers, without allocating
    (bc: an axlbm_boundary, or None for the half-spacing grid)."""
    vp = lambda p: ctypes.c_void_p(p or None)
    bcp = ctypes.byref(bc) if bc is not None else None
    _check(lib().axlbm_check_static(ctypes.byref(grid), float(tau), ctypes.byref(forcing), bcp, vp(f_ptr), vp(g_ptr),
                                    vp(t_ptr), float(a_z), vp(speed_prev_ptr), vp(speed_out_ptr), vp(out_ptr),
                                    vp(stream)))


def axlbm_destroy(h) -> None:
    _check(lib().axlbm_destroy(h))


# ----------------------------------------------------------------------------- structs from a Problem


def structs(pb: "_inputs.Problem", precision: str = "fp32"):
    """(grid, tau, forcing, boundary) for a Problem."""
    g = axlbm_grid(nr=pb.nr, nz=pb.nz, precision=PRECISIONS[precision], with_swirl=int(bool(pb.swirl)),
                   with_temperature=int(bool(pb.temperature)), collision={"bgk": BGK, "mrt": MRT}[pb.collision],
                   r0=float(pb.r0))
    f = axlbm_forcing(rho0=pb.rho0, az0=pb.az0, omega_t=pb.omega_t, gbeta=pb.gbeta, t_ref=pb.t_ref,
                      tau_t=pb.tau_t, t_init=pb.t_ref, mrt_s_eps=float(pb.s_eps), mrt_s_q=float(pb.s_q))
    b = axlbm_boundary()
    b.inner = _INNER[pb.inner]
    b.z_lo, b.z_hi = _ZKIND[pb.z_lo], _ZKIND[pb.z_hi]
    b.outer = _OUTER[getattr(pb, "outer", "wall")]
    b.r_split = float(pb.r_split)
    for i, face in enumerate(_inputs.FACES):
        b.t_dirichlet[i] = int(pb.t_dirichlet(face))
        b.omega[i] = pb.omega_of(face)
        b.t_wall[i] = pb.t_value(face)
    return g, float(pb.tau), f, b


class Domain:
    """One axisymmetric domain on the current CUDA device.

    Device memory comes from PyTorch (a uint8 tensor handed to the library as
    caller-owned state memory) and work runs on the current PyTorch stream.
    """

    def __init__(self, pb: "_inputs.Problem", precision: str = "fp32", stream=None):
        import torch

        self.pb = pb
        self.precision = precision
        self.grid, self.tau, self.forcing, self.boundary = structs(pb, precision)
        nbytes = axlbm_state_bytes(self.grid)
        self._mem = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = axlbm_create(self.grid, self.tau, self.forcing, self.boundary,
                                   stream=self.stream.cuda_stream, state_mem=self._mem.data_ptr(),
                                   state_bytes=nbytes)

    def close(self) -> None:
        if getattr(self, "handle", None) is not None:
            axlbm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- stepping
    def step(self, n: int) -> None:
        axlbm_step(self.handle, n)

    def use_graphs(self, enable: bool) -> None:
        """Replay runs of plain steps from captured CUDA graphs (default) or launch every kernel."""
        _check(lib().axlbm_use_graphs(self.handle, int(bool(enable))), self.handle)

    def set_residual_lag(self, lag: int) -> None:
        """1: Eq. 57 between consecutive levels (default); 2: half the change over two levels."""
        _check(lib().axlbm_set_residual_lag(self.handle, int(lag)), self.handle)

    # -- cut faces (z-slab decomposition)
    def halo_bytes(self) -> int:
        n = ctypes.c_size_t()
        _check(lib().axlbm_halo_bytes(self.handle, ctypes.byref(n)), self.handle)
        return int(n.value)

    def halo_send(self, face: int, out) -> None:
        """Message of cut face `face` (FACE_LO / FACE_HI) into `out`: a uint8
        numpy array (host, synchronises) or a uint8 CUDA tensor (queued)."""
        if isinstance(out, np.ndarray):
            _check(lib().axlbm_halo_send(self.handle, int(face), out.ctypes.data, 0), self.handle)
        else:
            _check(lib().axlbm_halo_send(self.handle, int(face), out.data_ptr(), 1), self.handle)

    def halo_recv(self, face: int, msg) -> None:
        """Store the neighbouring slab's message for cut face `face`."""
        if isinstance(msg, np.ndarray):
            m = np.ascontiguousarray(msg)
            _check(lib().axlbm_halo_recv(self.handle, int(face), m.ctypes.data, 0), self.handle)
        else:
            _check(lib().axlbm_halo_recv(self.handle, int(face), msg.data_ptr(), 1), self.handle)

    def graph_stats(self):
        """(captures, launches) of the step graphs since creation."""
        c, n = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().axlbm_graph_stats(self.handle, ctypes.byref(c), ctypes.byref(n)), self.handle)
        return int(c.value), int(n.value)

    @property
    def time(self) -> int:
        return axlbm_time(self.handle)

    def residual(self, allow_nonfinite: bool = False):
        """(residual of Eq. 57, mass, budget) of the last check step."""
        return axlbm_residual(self.handle, allow_nonfinite)

    # -- data movement
    def moments(self, mask: int = RHO | UR | UZ, dtype=np.float64) -> np.ndarray:
        """Selected fields on the host, shape [nfields][nz][nr]."""
        nf = bin(mask).count("1")
        out = np.empty((nf, self.pb.nz, self.pb.nr), dtype=dtype)
        axlbm_moments(self.handle, mask, out.ctypes.data, F64 if dtype == np.float64 else F32, 0)
        return out

    def moments_device(self, mask: int, out) -> None:
        """Selected fields into a CUDA tensor (float32 or float64), asynchronously."""
        import torch

        axlbm_moments(self.handle, mask, out.data_ptr(), F32 if out.dtype == torch.float32 else F64, 1)

    def set_fields(self, fields) -> None:
        """Equilibrium reset from fields [5][nz][nr] (numpy on the host or a CUDA tensor)."""
        if isinstance(fields, np.ndarray):
            a = np.ascontiguousarray(fields, dtype=np.float64)
            axlbm_set_fields(self.handle, a.ctypes.data, F64, 0)
        else:
            import torch

            axlbm_set_fields(self.handle, fields.data_ptr(), F32 if fields.dtype == torch.float32 else F64, 1)

    def get_populations(self):
        shape = (self.pb.nz, self.pb.nr)
        f = np.empty((9,) + shape)
        g = np.empty((4,) + shape) if self.pb.swirl else None
        h = np.empty((4,) + shape) if self.pb.temperature else None
        axlbm_get_populations(self.handle, f, g, h)
        return f, g, h

    def set_populations(self, f, g=None, h=None, time: int = 0) -> None:
        cast = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)
        axlbm_set_populations(self.handle, cast(f), cast(g), cast(h), time)

    # -- checkpoint / resume
    def save(self) -> np.ndarray:
        """Checkpoint of the whole state (axlbm_save) as a uint8 array."""
        return _save(lib().axlbm_save, self.handle, _check)

    def load(self, checkpoint) -> None:
        """Resume from a checkpoint of a domain with the same grid and storage (axlbm_load)."""
        _load(lib().axlbm_load, self.handle, checkpoint, _check)


# Checkpoint header fields (name, byte offset, struct format), as include/axlbm.h lays them out.
CHECKPOINT_HEADER = (("magic", 0, "8s"), ("version", 8, "I"), ("kind", 12, "I"), ("fingerprint", 16, "Q"),
                     ("state_bytes", 24, "Q"), ("time", 32, "q"), ("parity", 40, "i"), ("flags", 44, "I"),
                     ("aux", 48, "i"))
CHECKPOINT_HEADER_BYTES = 64


def checkpoint_info(checkpoint) -> dict:
    """The header fields of a checkpoint (axlbm_save / axlbm_batch_save), read on the host."""
    import struct

    raw = bytes(np.frombuffer(checkpoint, dtype=np.uint8)[:CHECKPOINT_HEADER_BYTES])
    if len(raw) < CHECKPOINT_HEADER_BYTES or raw[:8] != b"AXLBMCK\0":
        raise ValueError("not a checkpoint")
    info = {name: struct.unpack_from("<" + fmt, raw, off)[0] for name, off, fmt in CHECKPOINT_HEADER}
    info["kind"] = {1: "domain", 2: "batch"}.get(info["kind"], info["kind"])
    return info


def _save(fn, handle, check) -> np.ndarray:
    n = ctypes.c_size_t()
    check(fn(handle, None, 0, ctypes.byref(n)), handle)
    out = np.empty(n.value, dtype=np.uint8)
    check(fn(handle, out.ctypes.data, out.size, ctypes.byref(n)), handle)
    return out


def _load(fn, handle, checkpoint, check) -> None:
    a = np.ascontiguousarray(np.frombuffer(checkpoint, dtype=np.uint8) if isinstance(checkpoint, (bytes, bytearray))
                             else checkpoint, dtype=np.uint8)
    check(fn(handle, a.ctypes.data, a.size), handle)


# ----------------------------------------------------------------------------- batches


def _bcheck(status: int, batch=None) -> int:
    if status != OK:
        msg = lib().axlbm_batch_last_error(batch).decode(errors="replace")
        raise AxlbmError(status, msg or lib().axlbm_status_string(status).decode())
    return status


def domain_array(problems):
    """ctypes array of axlbm_domain for a list of Problems."""
    arr = (axlbm_domain * len(problems))()
    for i, pb in enumerate(problems):
        g, tau, f, b = structs(pb, "fp32")
        arr[i].grid, arr[i].tau, arr[i].forcing, arr[i].boundary = g, tau, f, b
    return arr


def axlbm_batch_state_bytes(domains, precision: int) -> int:
    n = ctypes.c_size_t()
    _bcheck(lib().axlbm_batch_state_bytes(domains, len(domains), int(precision), ctypes.byref(n)))
    return int(n.value)


def axlbm_batch_create(domains, precision: int, stream: int = 0, state_mem: int = 0, state_bytes: int = 0):
    h = ctypes.c_void_p()
    _bcheck(lib().axlbm_batch_create(domains, len(domains), int(precision), ctypes.c_void_p(stream or None),
                                     ctypes.c_void_p(state_mem or None), ctypes.c_size_t(state_bytes),
                                     ctypes.byref(h)))
    return h


def axlbm_batch_step(b, n: int) -> None:
    _bcheck(lib().axlbm_batch_step(b, int(n)), b)


def axlbm_batch_residuals(b, n_domains: int, allow_nonfinite: bool = False) -> np.ndarray:
    out = np.empty((n_domains, 3))
    st = lib().axlbm_batch_residuals(b, _dptr(out))
    if not (allow_nonfinite and st == ENONFINITE):
        _bcheck(st, b)
    return out


def axlbm_batch_moments(b, d: int, mask: int, out_ptr: int, out_dtype: int, out_on_device: int) -> None:
    _bcheck(lib().axlbm_batch_moments(b, int(d), int(mask), ctypes.c_void_p(out_ptr), int(out_dtype),
                                      int(out_on_device)), b)


def axlbm_batch_set_fields(b, d: int, ptr: int, in_dtype: int, on_device: int) -> None:
    _bcheck(lib().axlbm_batch_set_fields(b, int(d), ctypes.c_void_p(ptr), int(in_dtype), int(on_device)), b)


def axlbm_batch_set_fields_all(b, ptr: int, in_dtype: int, on_device: int) -> None:
    _bcheck(lib().axlbm_batch_set_fields_all(b, ctypes.c_void_p(ptr), int(in_dtype), int(on_device)), b)


def axlbm_batch_moments_all(b, mask: int, out_ptr: int, out_dtype: int, out_on_device: int) -> None:
    _bcheck(lib().axlbm_batch_moments_all(b, int(mask), ctypes.c_void_p(out_ptr), int(out_dtype),
                                          int(out_on_device)), b)


def _host_array(a):
    """(dtype code, address) of a contiguous FP32/FP64 host array (numpy or CPU tensor)."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous or a.dtype not in (np.float32, np.float64):
            raise ValueError("a contiguous float32 or float64 array is needed")
        return (F32 if a.dtype == np.float32 else F64), a.ctypes.data
    import torch

    if a.device.type != "cpu" or not a.is_contiguous() or a.dtype not in (torch.float32, torch.float64):
        raise ValueError("a contiguous float32 or float64 CPU tensor is needed")
    return (F32 if a.dtype == torch.float32 else F64), a.data_ptr()


def axlbm_batch_set_fields_all_async(b, host_ptr: int, in_dtype: int) -> None:
    _bcheck(lib().axlbm_batch_set_fields_all_async(b, ctypes.c_void_p(host_ptr), int(in_dtype)), b)


def axlbm_batch_moments_all_async(b, mask: int, host_ptr: int, out_dtype: int) -> None:
    _bcheck(lib().axlbm_batch_moments_all_async(b, int(mask), ctypes.c_void_p(host_ptr), int(out_dtype)), b)


def axlbm_batch_sync(b) -> None:
    _bcheck(lib().axlbm_batch_sync(b), b)


def axlbm_batch_get_populations(b, d: int, f, g, t_pop) -> None:
    _bcheck(lib().axlbm_batch_get_populations(b, int(d), _dptr(f), _dptr(g), _dptr(t_pop)), b)


def axlbm_batch_set_populations(b, d: int, f, g, t_pop) -> None:
    _bcheck(lib().axlbm_batch_set_populations(b, int(d), _dptr(f), _dptr(g), _dptr(t_pop)), b)


def axlbm_batch_time(b) -> int:
    t = ctypes.c_int64()
    _bcheck(lib().axlbm_batch_time(b, ctypes.byref(t)), b)
    return int(t.value)


def axlbm_batch_tile_shape(b):
    r, c = ctypes.c_int32(), ctypes.c_int32()
    _bcheck(lib().axlbm_batch_tile_shape(b, ctypes.byref(r), ctypes.byref(c)), b)
    return int(r.value), int(c.value)


def axlbm_batch_kernel_timing(b, enable: bool) -> None:
    _bcheck(lib().axlbm_batch_kernel_timing(b, int(bool(enable))), b)


def axlbm_batch_kernel_times(b):
    nb, na = ctypes.c_int64(), ctypes.c_int64()
    ms, by = ctypes.c_double(), ctypes.c_double()
    _bcheck(lib().axlbm_batch_kernel_times(b, ctypes.byref(nb), ctypes.byref(ms), ctypes.byref(by),
                                           ctypes.byref(na)), b)
    return int(nb.value), ms.value, by.value, int(na.value)


def axlbm_batch_kernel_times_by_parity(b):
    """([even, odd] launches, [even, odd] ms, [even, odd] algorithmic bytes) of the bulk kernel."""
    nb = (ctypes.c_int64 * 2)()
    ms, by = (ctypes.c_double * 2)(), (ctypes.c_double * 2)()
    _bcheck(lib().axlbm_batch_kernel_times_by_parity(b, nb, ms, by), b)
    return list(nb), list(ms), list(by)


def axlbm_selftest_rcp(x) -> tuple:
    """(scalar, paired) FP32 reciprocals of the collision evaluated on the device for the values x."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(2 * x.size, dtype=np.float32)
    _check(lib().axlbm_selftest_rcp(x.ctypes.data, x.size, out.ctypes.data), None)
    return out[:x.size], out[x.size:]


def axlbm_selftest_bounded_wait(max_cycles: int):
    """(threads that gave up, error word) of a warp whose bounded wait can never complete."""
    n, err = ctypes.c_int32(), ctypes.c_uint32()
    _check(lib().axlbm_selftest_bounded_wait(int(max_cycles), ctypes.byref(n), ctypes.byref(err)), None)
    return int(n.value), int(err.value)


def axlbm_batch_destroy(b) -> None:
    _bcheck(lib().axlbm_batch_destroy(b))


class Batch:
    """Many domains advanced together, on PyTorch-owned device memory and stream."""

    def __init__(self, problems, precision: str = "fp32", stream=None):
        import torch

        self.problems = list(problems)
        self.domains = domain_array(self.problems)
        self.precision = PRECISIONS[precision]
        nbytes = axlbm_batch_state_bytes(self.domains, self.precision)
        self._mem = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._in_flight = []  # host arrays of queued asynchronous copies, kept alive until sync()
        self.handle = axlbm_batch_create(self.domains, self.precision, stream=self.stream.cuda_stream,
                                         state_mem=self._mem.data_ptr(), state_bytes=nbytes)

    def close(self) -> None:
        if getattr(self, "handle", None) is not None:
            axlbm_batch_destroy(self.handle)  # waits for the copies in flight
            self.handle = None
            self._in_flight = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int) -> None:
        axlbm_batch_step(self.handle, n)

    @property
    def time(self) -> int:
        return axlbm_batch_time(self.handle)

    @property
    def tile_shape(self):
        return axlbm_batch_tile_shape(self.handle)

    @tile_shape.setter
    def tile_shape(self, shape):
        """Use this tile shape (rows, nodes) in even and odd steps."""
        _bcheck(lib().axlbm_batch_set_tile_shape(self.handle, int(shape[0]), int(shape[1])), self.handle)

    @property
    def tile_shapes(self):
        """((rows, nodes) of even steps, (rows, nodes) of odd steps)."""
        r, n = (ctypes.c_int32 * 2)(), (ctypes.c_int32 * 2)()
        _bcheck(lib().axlbm_batch_tile_shapes(self.handle, r, n), self.handle)
        return (int(r[0]), int(n[0])), (int(r[1]), int(n[1]))

    @tile_shapes.setter
    def tile_shapes(self, shapes):
        """Use shapes[0] in even steps and shapes[1] in odd steps."""
        r = (ctypes.c_int32 * 2)(int(shapes[0][0]), int(shapes[1][0]))
        n = (ctypes.c_int32 * 2)(int(shapes[0][1]), int(shapes[1][1]))
        _bcheck(lib().axlbm_batch_set_tile_shapes(self.handle, r, n), self.handle)

    def use_graphs(self, enable: bool) -> None:
        """Replay runs of plain steps from captured CUDA graphs (default) or launch every kernel."""
        _bcheck(lib().axlbm_batch_use_graphs(self.handle, int(bool(enable))), self.handle)

    def set_residual_lag(self, lag: int) -> None:
        """1: Eq. 57 between consecutive levels (default); 2: half the change over two levels."""
        _bcheck(lib().axlbm_batch_set_residual_lag(self.handle, int(lag)), self.handle)

    def set_time(self, t: int) -> None:
        """Move the batch (at an even level) to the even time level t."""
        _bcheck(lib().axlbm_batch_set_time(self.handle, int(t)), self.handle)

    def copy_domain(self, d: int, src: "Batch", sd: int) -> None:
        """Copy domain sd of batch src (same storage, time level and grid) into domain d."""
        _bcheck(lib().axlbm_batch_copy_domain(self.handle, int(d), src.handle, int(sd)), self.handle)

    def graph_stats(self):
        """(captures, launches) of the step graphs since creation."""
        c, n = ctypes.c_int64(), ctypes.c_int64()
        _bcheck(lib().axlbm_batch_graph_stats(self.handle, ctypes.byref(c), ctypes.byref(n)), self.handle)
        return int(c.value), int(n.value)

    def residuals(self, allow_nonfinite: bool = False) -> np.ndarray:
        """[n][3]: residual (Eq. 57), mass, budget of each domain's last check step."""
        return axlbm_batch_residuals(self.handle, len(self.problems), allow_nonfinite)

    def moments(self, d: int, mask: int = RHO | UR | UZ, dtype=np.float64) -> np.ndarray:
        pb = self.problems[d]
        out = np.empty((bin(mask).count("1"), pb.nz, pb.nr), dtype=dtype)
        axlbm_batch_moments(self.handle, d, mask, out.ctypes.data, F64 if dtype == np.float64 else F32, 0)
        return out

    def set_fields(self, d: int, fields) -> None:
        if isinstance(fields, np.ndarray):
            a = np.ascontiguousarray(fields, dtype=np.float64)
            axlbm_batch_set_fields(self.handle, d, a.ctypes.data, F64, 0)
        else:
            import torch

            axlbm_batch_set_fields(self.handle, d, fields.data_ptr(),
                                   F32 if fields.dtype == torch.float32 else F64, 1)

    def set_fields_all(self, fields) -> None:
        """Fields of every domain, packed in domain order ([5][nz][nr] each); numpy or CUDA tensor."""
        if isinstance(fields, np.ndarray):
            a = np.ascontiguousarray(fields, dtype=np.float64)
            axlbm_batch_set_fields_all(self.handle, a.ctypes.data, F64, 0)
        else:
            import torch

            axlbm_batch_set_fields_all(self.handle, fields.data_ptr(), F32 if fields.dtype == torch.float32 else F64,
                                       0 if fields.device.type == "cpu" else 1)

    def moments_all(self, mask: int, out) -> None:
        """Selected fields of every domain into a packed buffer (numpy or torch, host or CUDA)."""
        if isinstance(out, np.ndarray):
            axlbm_batch_moments_all(self.handle, mask, out.ctypes.data, F64 if out.dtype == np.float64 else F32, 0)
        else:
            import torch

            axlbm_batch_moments_all(self.handle, mask, out.data_ptr(), F32 if out.dtype == torch.float32 else F64,
                                    0 if out.device.type == "cpu" else 1)

    def set_fields_all_async(self, fields) -> None:
        """As set_fields_all from host memory (numpy or CPU tensor, FP32 or FP64), the copy queued on the
        batch's copy stream; the array is kept alive, and must stay unchanged, until sync()."""
        dt, ptr = _host_array(fields)
        axlbm_batch_set_fields_all_async(self.handle, ptr, dt)
        self._in_flight.append(fields)

    def moments_all_async(self, mask: int, out) -> None:
        """As moments_all into host memory (numpy or CPU tensor); `out` is filled when sync() returns."""
        dt, ptr = _host_array(out)
        axlbm_batch_moments_all_async(self.handle, mask, ptr, dt)
        self._in_flight.append(out)

    def sync(self) -> None:
        """Wait for the batch's steps and every asynchronous copy."""
        axlbm_batch_sync(self.handle)
        self._in_flight.clear()

    def get_populations(self, d: int):
        pb = self.problems[d]
        shape = (pb.nz, pb.nr)
        f, g = np.empty((9,) + shape), np.empty((4,) + shape)
        h = np.empty((4,) + shape) if pb.temperature else None
        axlbm_batch_get_populations(self.handle, d, f, g, h)
        return f, g, h

    def set_populations(self, d: int, f, g, h=None) -> None:
        cast = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)
        axlbm_batch_set_populations(self.handle, d, cast(f), cast(g), cast(h))

    # -- checkpoint / resume
    def save(self) -> np.ndarray:
        """Checkpoint of every domain's state (axlbm_batch_save) as a uint8 array."""
        return _save(lib().axlbm_batch_save, self.handle, _bcheck)

    def load(self, checkpoint) -> None:
        """Resume from a checkpoint of a batch of the same domains and storage (axlbm_batch_load)."""
        _load(lib().axlbm_batch_load, self.handle, checkpoint, _bcheck)


# ----------------------------------------------------------------------------- warm start

WS_FEATURES = 6
WS_CANVAS = (256, 128)  # rows (z), columns (r)


def ws_domain(pb) -> axlbm_ws_domain:
    """Canvas geometry of a Problem (see inputs.warm_start_geometry)."""
    g = _inputs.warm_start_geometry(pb)
    return axlbm_ws_domain(nr=pb.nr, nz=pb.nz, r_first=g["r_first"], r_wall=g["r_wall"], z_first=g["z_first"],
                           z_bottom=g["z_bottom"], height=g["height"], rho0=pb.rho0, u_scale=g["u_scale"],
                           t_ref=pb.t_ref)


class WarmStart:
    """The warm-start network on the current CUDA device (weights: uint16 BF16
    bit patterns, axlbm_ws_weight_count() of them, packed as in axlbm.h)."""

    def __init__(self, weights, stream=None):
        import torch
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.uint16).ravel())
        self.count = int(lib().axlbm_ws_weight_count())
        if w.size != self.count:
            raise ValueError(f"need {self.count} weights, got {w.size}")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = lib().axlbm_ws_create(w.ctypes.data, w.size, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != OK:
            raise AxlbmError(st, lib().axlbm_ws_last_error(None).decode(errors="replace"))
        self.handle = h

    def _check(self, st):
        if st != OK:
            raise AxlbmError(st, lib().axlbm_ws_last_error(self.handle).decode(errors="replace"))

    def predict(self, features):
        """Canvases [n][4][256][128] (torch FP32 on the device) of features [n][6]."""
        import torch
        f = np.ascontiguousarray(np.asarray(features, dtype=np.float32).reshape(-1, WS_FEATURES))
        out = torch.empty((f.shape[0], 4) + WS_CANVAS, dtype=torch.float32, device="cuda")
        self._check(lib().axlbm_ws_predict(self.handle, f.ctypes.data, f.shape[0], out.data_ptr()))
        return out

    def fields(self, canvas, problems):
        """Packed fields of every problem (torch FP32 on the device, the layout of
        axlbm_batch_set_fields_all) from their canvases."""
        import torch
        doms = (axlbm_ws_domain * len(problems))(*[ws_domain(pb) for pb in problems])
        out = torch.empty(sum(5 * pb.cells for pb in problems), dtype=torch.float32, device="cuda")
        self._check(lib().axlbm_ws_fields(self.handle, canvas.data_ptr(), len(problems), doms, out.data_ptr()))
        return out

    def to_canvas(self, moments, problems):
        """Canvases [n][4][256][128] (torch FP32 on the device) of every problem's
        moments (device FP32, u_r, u_z, u_theta, T as [4][nz][nr] per problem, packed)."""
        import torch
        doms = (axlbm_ws_domain * len(problems))(*[ws_domain(pb) for pb in problems])
        out = torch.empty((len(problems), 4) + WS_CANVAS, dtype=torch.float32, device="cuda")
        self._check(lib().axlbm_ws_to_canvas(self.handle, moments.data_ptr(), len(problems), doms, out.data_ptr()))
        return out

    def train_step(self, features, target, lr, betas=(0.9, 0.999), eps=1e-8) -> float:
        """One Adam step on 1..16 canvases (features and targets as torch FP32 on the
        device); returns the mean squared error before the update."""
        loss = ctypes.c_double()
        self._check(lib().axlbm_ws_train_step(self.handle, features.data_ptr(), target.data_ptr(), features.shape[0],
                                              float(lr), float(betas[0]), float(betas[1]), float(eps),
                                              ctypes.byref(loss)))
        return loss.value

    def loss(self, features, target) -> float:
        """Mean squared error on any number of canvases (torch FP32 on the device)."""
        loss = ctypes.c_double()
        self._check(lib().axlbm_ws_loss(self.handle, features.data_ptr(), target.data_ptr(), features.shape[0],
                                        ctypes.byref(loss)))
        return loss.value

    def last_gradient(self) -> np.ndarray:
        """FP32 gradient of the last training step's loss, in the weight packing."""
        out = np.empty(self.count, dtype=np.float32)
        self._check(lib().axlbm_ws_last_gradient(self.handle, out.ctypes.data))
        return out

    def weights(self) -> np.ndarray:
        """The current weights as BF16 bit patterns (uint16)."""
        out = np.empty(self.count, dtype=np.uint16)
        self._check(lib().axlbm_ws_get_weights(self.handle, out.ctypes.data))
        return out

    def start(self, batch, problems):
        """Initialise a Batch (at an even level) from the network's fields."""
        canvas = self.predict([_inputs.warm_start_features(pb) for pb in problems])
        fields = self.fields(canvas, problems)
        axlbm_batch_set_fields_all(batch.handle, fields.data_ptr(), F32, 1)
        return canvas

    def close(self):
        if getattr(self, "handle", None):
            lib().axlbm_ws_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
