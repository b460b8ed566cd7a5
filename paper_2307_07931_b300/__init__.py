"""Python binding of libprotox.so, the B300 fused periodic Poisson relaxation
library (ProtoX, Sec. IV). Argument marshalling only: every step of the
computation runs in the library's CUDA kernels. PyTorch supplies device
memory and streams.

The names mirror the C ABI in include/protox.h:
    create / destroy / last_error          px_create / px_destroy / px_last_error
    apply_stencil(ctx, phi, lphi)          px_apply_stencil
    relax_n(ctx, phi_in, phi_out, rho,...) px_relax_n
    residual_norm(ctx, phi, rho)           px_residual_norm
Fields are CUDA tensors of shape (ny, nx) (ghost=0) or (ny + 2, nx + 2)
(ghost=1), dtype float64 or float32, unit stride along x; the row stride is
passed as the pitch ld.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))

LIB_PATH = os.path.join(HERE, "libprotox.so")
LIB_CHECKED_PATH = os.path.join(HERE, "libprotox_checked.so")  # -DPX_CHECKED variant

PX_OK, PX_EINVAL, PX_ECUDA, PX_ENOMEM, PX_ENOCONV, PX_ETIMEOUT, PX_EMEAN, PX_ENAN, \
    PX_EUNSUPPORTED = range(9)
PX_F64, PX_F32 = 0, 1
(PX_OPT_FP32_FAMILY, PX_OPT_RB_SWEEPS_PER_LAUNCH, PX_OPT_BATCH_LAUNCHES, PX_OPT_RB_FP64_PASSES,
 PX_OPT_MG_PROLONG) = 1, 2, 3, 4, 5


class PxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_name(status)}: {msg}")
        self.status = status


PX_SOLVE_PLAIN, PX_SOLVE_REFINE = 0, 1


class SolveOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("tblock", ctypes.c_int32), ("omega", ctypes.c_double),
                ("rtol", ctypes.c_double), ("max_sweeps", ctypes.c_int64),
                ("check_every", ctypes.c_int32), ("inner_sweeps", ctypes.c_int32),
                ("timeout_ms", ctypes.c_int64), ("check_mean", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int64), ("cycles", ctypes.c_int64), ("checks", ctypes.c_int64),
                ("rel_resid", ctypes.c_double), ("wall_ms", ctypes.c_double)]


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("ld", ctypes.c_int64),
                ("ghost", ctypes.c_int32), ("dtype", ctypes.c_int32), ("h", ctypes.c_double)]


class Grid3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("ld", ctypes.c_int64), ("lp", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("h", ctypes.c_double)]


_lib = None
_vp = ctypes.c_void_p


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libprotox.so (build it first with paper_2307_07931_b300.build).
    Raises ImportError if the library is absent: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libprotox.so not found at {path}; run "
                          "`python -m paper_2307_07931_b300.build` (nvcc, sm_103a)")
    lib = ctypes.CDLL(path)
    gp = ctypes.POINTER(Grid)
    i, d = ctypes.c_int, ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    lib.px_create.argtypes = [ctypes.POINTER(_vp), i]
    lib.px_destroy.argtypes = [_vp]
    lib.px_last_error.argtypes = [_vp]
    lib.px_last_error.restype = ctypes.c_char_p
    lib.px_status_string.argtypes = [i]
    lib.px_status_string.restype = ctypes.c_char_p
    lib.px_apply_stencil.argtypes = [_vp, gp, _vp, _vp, _vp]
    lib.px_relax_n.argtypes = [_vp, gp, _vp, _vp, _vp, d, i, i, _vp, i, _vp]
    lib.px_rbsor_n.argtypes = [_vp, gp, _vp, _vp, _vp, d, i, _vp, i, _vp]
    lib.px_mg_solve.argtypes = [_vp, gp, _vp, _vp, i, i, i, d, i, i, _vp, _vp]
    lib.px_relax3_n.argtypes = [_vp, ctypes.POINTER(Grid3), _vp, _vp, _vp, d, i, _vp, i, _vp]
    lib.px_residual_norm.argtypes = [_vp, gp, _vp, _vp, dp, dp, _vp]
    lib.px_residual_norm_async.argtypes = [_vp, gp, _vp, _vp, _vp, _vp]
    ip = ctypes.POINTER(ctypes.c_int)
    lib.px_relax_plan.argtypes = [_vp, gp, _vp, _vp, _vp, i, i, ip, ip]
    lib.px_relax_n_static.argtypes = [gp, _vp, _vp, _vp, d, i, i, _vp, i, _vp]
    lib.px_batch_plan.argtypes = [_vp, i, gp, i, d, i, ctypes.c_char_p, i, ctypes.POINTER(_vp)]
    lib.px_batch_run.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp, _vp]
    lib.px_batch_describe.argtypes = [_vp]
    lib.px_batch_describe.restype = ctypes.c_char_p
    lib.px_batch_destroy.argtypes = [_vp]
    fp = ctypes.POINTER(ctypes.c_float)
    lib.px_cnn_param_count.restype = ctypes.c_size_t
    lib.px_cnn_create.argtypes = [_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(_vp)]
    lib.px_cnn_destroy.argtypes = [_vp]
    lib.px_cnn_get_params.argtypes = [_vp, fp, ctypes.c_size_t]
    lib.px_cnn_set_params.argtypes = [_vp, fp, ctypes.c_size_t]
    lib.px_cnn_forward.argtypes = [_vp, _vp, _vp, i, i, i, _vp]
    lib.px_cnn_state_count.restype = ctypes.c_size_t
    lib.px_cnn_get_state.argtypes = [_vp, fp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int64)]
    lib.px_cnn_set_state.argtypes = [_vp, fp, ctypes.c_size_t, ctypes.c_int64]
    lib.px_cnn_grads.argtypes = [_vp, _vp, _vp, i, i, i, fp, dp, _vp]
    lib.px_cnn_train_step.argtypes = [_vp, _vp, _vp, i, i, i, ctypes.c_float, dp, _vp]
    lib.px_cnn_prepare.argtypes = [_vp, _vp, _vp, _vp, _vp, i, i, i, d, dp, _vp]
    lib.px_cnn_guess.argtypes = [_vp, _vp, _vp, i, i, i, d, _vp]
    lib.px_cnn_get_hidden.argtypes = [_vp, i, i, ctypes.POINTER(ctypes.c_uint16), ctypes.c_size_t,
                                      _vp]
    lib.px_cnn_set_wait_limit.argtypes = [_vp, ctypes.c_uint32]
    lib.px_cnn_set_staging.argtypes = [_vp, i]
    lib.px_cnn_set_relabel.argtypes = [_vp, i]
    lib.px_set_option.argtypes = [_vp, i, i]
    lib.px_is_checked_build.restype = i
    lib.px_checked_faults.argtypes = [_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
    lib.px_get_option.argtypes = [_vp, i, ip]
    eg = ctypes.POINTER(EulerGrid)
    lib.px_euler_step.argtypes = [_vp, eg, _vp, _vp, d, d, i, d, _vp, _vp]
    lib.px_euler_conserved.argtypes = [_vp, eg, _vp, _vp, d, _vp]
    for name in ("px_cnn_get_hidden", "px_cnn_set_wait_limit", "px_cnn_set_staging",
                 "px_cnn_set_relabel",
                 "px_set_option", "px_get_option", "px_checked_faults",
                 "px_euler_step", "px_euler_conserved"):
        getattr(lib, name).restype = i
    for name in ("px_cnn_get_state", "px_cnn_set_state",
                 "px_cnn_create", "px_cnn_destroy", "px_cnn_get_params", "px_cnn_set_params",
                 "px_cnn_forward", "px_cnn_grads", "px_cnn_train_step", "px_cnn_prepare",
                 "px_cnn_guess"):
        getattr(lib, name).restype = i
    lib.px_solve.argtypes = [_vp, gp, _vp, _vp, ctypes.POINTER(SolveOpts),
                             ctypes.POINTER(SolveInfo), _vp]
    for name in ("px_create", "px_destroy", "px_apply_stencil", "px_relax_n", "px_rbsor_n",
                 "px_mg_solve", "px_relax3_n",
                 "px_residual_norm", "px_residual_norm_async", "px_relax_plan",
                 "px_relax_n_static", "px_solve", "px_batch_plan", "px_batch_run",
                 "px_batch_destroy"):
        getattr(lib, name).restype = i
    _lib = lib
    return lib


def status_name(s: int) -> str:
    return load_library().px_status_string(int(s)).decode()


# ----------------------------------------------------------------- contexts
class Context:
    """Owns one px_ctx (device scratch and reduction slots) on one device."""

    def __init__(self, device: int = 0):
        lib = load_library()
        h = _vp()
        s = lib.px_create(ctypes.byref(h), int(device))
        if s != PX_OK:
            raise PxError(s, lib.px_last_error(None).decode())
        self.handle = h
        self.device = int(device)

    def check(self, s: int):
        if s != PX_OK:
            raise PxError(s, load_library().px_last_error(self.handle).decode())

    def set_option(self, option: int, value: int):
        """px_set_option: per-context kernel selection (PX_OPT_*)."""
        self.check(load_library().px_set_option(self.handle, int(option), int(value)))

    def checked_faults(self):
        """(count, first) of the checked build's bounds violations since the last
        call (px_checked_faults; PxError PX_EUNSUPPORTED in the normal build)."""
        cnt, first = ctypes.c_uint64(), ctypes.c_uint64()
        self.check(load_library().px_checked_faults(self.handle, ctypes.byref(cnt), ctypes.byref(first)))
        return cnt.value, first.value

    def get_option(self, option: int) -> int:
        v = ctypes.c_int()
        self.check(load_library().px_get_option(self.handle, int(option), ctypes.byref(v)))
        return v.value

    def close(self):
        if self.handle:
            load_library().px_destroy(self.handle)
            self.handle = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default: dict[int, Context] = {}


def context(device: int | None = None) -> Context:
    """The process-wide default Context of a device (created on first use)."""
    import torch
    dev = torch.cuda.current_device() if device is None else int(device)
    if dev not in _default:
        _default[dev] = Context(dev)
    return _default[dev]


# ----------------------------------------------------------------- marshalling
def grid_of(t, h: float, ghost: int = 0) -> Grid:
    """px_grid describing tensor t of shape (ny + 2 ghost, nx + 2 ghost)."""
    import torch
    if t.dim() != 2:
        raise ValueError("fields are 2D tensors (ny, nx)")
    if t.stride(1) != 1:
        raise ValueError("fields need unit stride along x")
    if t.dtype == torch.float64:
        dt = PX_F64
    elif t.dtype == torch.float32:
        dt = PX_F32
    else:
        raise TypeError(f"unsupported dtype {t.dtype}")
    ny, nx = t.shape[0] - 2 * ghost, t.shape[1] - 2 * ghost
    return Grid(nx, ny, t.stride(0) if t.shape[0] > 1 else t.shape[1] + 0, ghost, dt, float(h))


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _stream(stream) -> int | None:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _same_layout(a, b):
    if a.shape != b.shape or a.dtype != b.dtype or a.stride() != b.stride():
        raise ValueError("fields of one call must share shape, dtype and strides")


# ----------------------------------------------------------------- the calls
def apply_stencil(phi, lphi, h: float, ghost: int = 0, ctx: Context | None = None,
                  stream=None):
    """lphi = L phi (px_apply_stencil)."""
    _same_layout(phi, lphi)
    ctx = ctx or context(phi.device.index)
    g = grid_of(phi, h, ghost)
    ctx.check(load_library().px_apply_stencil(ctx.handle, ctypes.byref(g), _ptr(phi),
                                              _ptr(lphi), _stream(stream)))
    return lphi


def relax_n(phi_in, phi_out, rho, h: float, omega: float, nsweeps: int, tblock: int = 0,
            resid=None, report_every: int = 0, ghost: int = 0, ctx: Context | None = None,
            stream=None):
    """nsweeps fused sweeps phi_in -> phi_out (px_relax_n). `resid`, if given,
    is a float64 CUDA tensor of ceil(nsweeps / report_every) entries."""
    _same_layout(phi_in, phi_out)
    _same_layout(phi_in, rho)
    ctx = ctx or context(phi_in.device.index)
    g = grid_of(phi_in, h, ghost)
    if resid is not None:
        import torch
        need = (nsweeps + report_every - 1) // report_every if report_every > 0 else 0
        if resid.dtype != torch.float64 or not resid.is_cuda or resid.numel() < need \
                or not resid.is_contiguous():
            raise ValueError(f"resid must be a contiguous CUDA float64 tensor of >= {need}")
    ctx.check(load_library().px_relax_n(ctx.handle, ctypes.byref(g), _ptr(phi_in),
                                        _ptr(phi_out), _ptr(rho), float(omega), int(nsweeps),
                                        int(tblock), _ptr(resid), int(report_every),
                                        _stream(stream)))
    return phi_out


def rbsor_n(phi_in, phi_out, rho, h: float, omega: float, nsweeps: int, resid=None,
            report_every: int = 0, ctx: Context | None = None, stream=None):
    """nsweeps red-black SOR sweeps phi_in -> phi_out (px_rbsor_n): red cells
    ((x + y) even) then black cells, in place within a sweep; nx, ny even.
    `resid`, if given, is a float64 CUDA tensor of ceil(nsweeps /
    report_every) entries (residual of each reported sweep's input state)."""
    _same_layout(phi_in, phi_out)
    _same_layout(phi_in, rho)
    ctx = ctx or context(phi_in.device.index)
    g = grid_of(phi_in, h, 0)
    if resid is not None:
        import torch
        need = (nsweeps + report_every - 1) // report_every if report_every > 0 else 0
        if resid.dtype != torch.float64 or not resid.is_cuda or resid.numel() < need \
                or not resid.is_contiguous():
            raise ValueError(f"resid must be a contiguous CUDA float64 tensor of >= {need}")
    ctx.check(load_library().px_rbsor_n(ctx.handle, ctypes.byref(g), _ptr(phi_in),
                                        _ptr(phi_out), _ptr(rho), float(omega), int(nsweeps),
                                        _ptr(resid), int(report_every), _stream(stream)))
    return phi_out


def mg_solve(phi, rho, h: float, ncycles: int, nu1: int = 2, nu2: int = 2, omega: float = 1.0,
             coarse_sweeps: int = 0, max_levels: int = 0, resid=None,
             ctx: Context | None = None, stream=None):
    """ncycles multigrid V-cycles on phi in place (px_mg_solve). `resid`, if
    given, is a float64 CUDA tensor of ncycles + 1 entries: the residual
    max-norm after 0, 1, ..., ncycles cycles."""
    _same_layout(phi, rho)
    ctx = ctx or context(phi.device.index)
    g = grid_of(phi, h, 0)
    if resid is not None:
        import torch
        if resid.dtype != torch.float64 or not resid.is_cuda or resid.numel() < ncycles + 1 \
                or not resid.is_contiguous():
            raise ValueError(f"resid must be a contiguous CUDA float64 tensor of >= {ncycles + 1}")
    ctx.check(load_library().px_mg_solve(ctx.handle, ctypes.byref(g), _ptr(phi), _ptr(rho),
                                         int(ncycles), int(nu1), int(nu2), float(omega),
                                         int(coarse_sweeps), int(max_levels), _ptr(resid),
                                         _stream(stream)))
    return phi


def grid3_of(t, h: float) -> Grid3:
    """px_grid3 describing a 3D tensor t of shape (nz, ny, nx)."""
    import torch
    if t.dim() != 3:
        raise ValueError("3D fields are tensors (nz, ny, nx)")
    if t.stride(2) != 1:
        raise ValueError("fields need unit stride along x")
    if t.dtype == torch.float64:
        dt = PX_F64
    elif t.dtype == torch.float32:
        dt = PX_F32
    else:
        raise TypeError(f"unsupported dtype {t.dtype}")
    nz, ny, nx = t.shape
    ld = t.stride(1) if ny > 1 else nx
    lp = t.stride(0) if nz > 1 else max(ny - 1, 0) * ld + nx
    return Grid3(nx, ny, nz, ld, lp, dt, float(h))


def relax3_n(phi_in, phi_out, rho, h: float, omega: float, nsweeps: int, resid=None,
             report_every: int = 0, ctx: Context | None = None, stream=None):
    """nsweeps fused 3D sweeps phi_in -> phi_out (px_relax3_n); tensors of
    shape (nz, ny, nx). `resid`, if given, is a float64 CUDA tensor of
    ceil(nsweeps / report_every) entries."""
    _same_layout(phi_in, phi_out)
    _same_layout(phi_in, rho)
    ctx = ctx or context(phi_in.device.index)
    g = grid3_of(phi_in, h)
    if resid is not None:
        import torch
        need = (nsweeps + report_every - 1) // report_every if report_every > 0 else 0
        if resid.dtype != torch.float64 or not resid.is_cuda or resid.numel() < need \
                or not resid.is_contiguous():
            raise ValueError(f"resid must be a contiguous CUDA float64 tensor of >= {need}")
    ctx.check(load_library().px_relax3_n(ctx.handle, ctypes.byref(g), _ptr(phi_in),
                                         _ptr(phi_out), _ptr(rho), float(omega), int(nsweeps),
                                         _ptr(resid), int(report_every), _stream(stream)))
    return phi_out


def relax_n_static(phi_in, phi_out, rho, h: float, omega: float, nsweeps: int,
                   tblock: int = 0, resid=None, report_every: int = 0, ghost: int = 0,
                   stream=None):
    """px_relax_n_static: relax_n for callers that cannot allocate device memory
    (no context; the ping-pong field comes from a fixed 16 MiB array in the
    library). Runs on the current device; fields up to 16 MiB."""
    _same_layout(phi_in, phi_out)
    _same_layout(phi_in, rho)
    g = grid_of(phi_in, h, ghost)
    lib = load_library()
    st = lib.px_relax_n_static(ctypes.byref(g), _ptr(phi_in), _ptr(phi_out), _ptr(rho),
                               float(omega), int(nsweeps), int(tblock), _ptr(resid),
                               int(report_every), _stream(stream))
    if st != PX_OK:
        raise PxError(st, lib.px_last_error(None).decode())
    return phi_out


def relax_plan(phi_in, phi_out, rho, h: float, nsweeps: int, tblock: int = 0, ghost: int = 0,
               ctx: Context | None = None) -> tuple[int, int]:
    """(sweeps per launch, kernel launches) that relax_n would use (px_relax_plan)."""
    ctx = ctx or context(phi_in.device.index)
    g = grid_of(phi_in, h, ghost)
    tb, nl = ctypes.c_int(), ctypes.c_int()
    ctx.check(load_library().px_relax_plan(ctx.handle, ctypes.byref(g), _ptr(phi_in),
                                           _ptr(phi_out), _ptr(rho), int(nsweeps), int(tblock),
                                           ctypes.byref(tb), ctypes.byref(nl)))
    return tb.value, nl.value


def residual_norm(phi, rho, h: float, ghost: int = 0, ctx: Context | None = None,
                  stream=None) -> tuple[float, float]:
    """(||rho - L phi||_inf, ||rho||_inf) in FP64 (px_residual_norm; synchronises)."""
    _same_layout(phi, rho)
    ctx = ctx or context(phi.device.index)
    g = grid_of(phi, h, ghost)
    r, p = ctypes.c_double(), ctypes.c_double()
    ctx.check(load_library().px_residual_norm(ctx.handle, ctypes.byref(g), _ptr(phi),
                                              _ptr(rho), ctypes.byref(r), ctypes.byref(p),
                                              _stream(stream)))
    return r.value, p.value


def residual_norm_async(phi, rho, out, h: float, ghost: int = 0, ctx: Context | None = None,
                        stream=None):
    """out[0:2] = (||rho - L phi||_inf, ||rho||_inf) on the device, no sync."""
    _same_layout(phi, rho)
    ctx = ctx or context(phi.device.index)
    g = grid_of(phi, h, ghost)
    ctx.check(load_library().px_residual_norm_async(ctx.handle, ctypes.byref(g), _ptr(phi),
                                                    _ptr(rho), _ptr(out), _stream(stream)))
    return out


def solve(phi, rho, h: float, mode: str = "plain", omega: float = 2.0 / 3.0, rtol: float = 1e-8,
          max_sweeps: int = 10**7, check_every: int = 1000, inner_sweeps: int = 500,
          tblock: int = 0, timeout_ms: int = 0, check_mean: bool = False, ghost: int = 0,
          ctx: Context | None = None, stream=None) -> dict:
    """px_solve: relax phi in place until ||rho - L phi|| <= rtol ||rho|| (FP64
    check). mode "plain" sweeps in the tensors' dtype; "refine" runs FP32-storage
    sweeps inside an FP64 refinement loop (FP64 tensors). Returns the info as a
    dict; raises PxError (with .info) on any status other than PX_OK."""
    _same_layout(phi, rho)
    ctx = ctx or context(phi.device.index)
    g = grid_of(phi, h, ghost)
    o = SolveOpts(PX_SOLVE_PLAIN if mode == "plain" else PX_SOLVE_REFINE, int(tblock),
                  float(omega), float(rtol), int(max_sweeps), int(check_every),
                  int(inner_sweeps), int(timeout_ms), 1 if check_mean else 0, 0)
    info = SolveInfo()
    st = load_library().px_solve(ctx.handle, ctypes.byref(g), _ptr(phi), _ptr(rho),
                                 ctypes.byref(o), ctypes.byref(info), _stream(stream))
    d = {k: getattr(info, k) for k, _ in SolveInfo._fields_}
    d["status"] = status_name(st)
    if st != PX_OK:
        err = PxError(st, load_library().px_last_error(ctx.handle).decode())
        err.info = d
        raise err
    return d


class EulerGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("ld", ctypes.c_int64),
                ("cs", ctypes.c_int64), ("dtype", ctypes.c_int32), ("dx", ctypes.c_double),
                ("dy", ctypes.c_double)]


def euler_grid_of(u, dx: float, dy: float) -> EulerGrid:
    """px_euler_grid of a (4, ny, nx) tensor (component planes, x fastest)."""
    import torch
    if u.dim() != 3 or u.shape[0] != 4:
        raise ValueError("Euler states are (4, ny, nx) tensors: rho, rho u, rho v, E")
    if u.dtype not in (torch.float64, torch.float32) or not u.is_cuda:
        raise ValueError("Euler states are CUDA float64 or float32 tensors")
    if u.stride(2) != 1:
        raise ValueError("x must be contiguous")
    dt = PX_F64 if u.dtype == torch.float64 else PX_F32
    return EulerGrid(int(u.shape[2]), int(u.shape[1]), int(u.stride(1)), int(u.stride(0)), dt,
                     float(dx), float(dy))


def euler_step(u_in, u_out, dx: float, dy: float, nsteps: int = 1, gamma: float = 1.4,
               cfl: float = 0.4, dt_fixed: float = 0.0, dt=None, ctx: Context | None = None,
               stream=None):
    """nsteps fused SSP-RK2 finite-volume steps of the 2D Euler equations
    u_in -> u_out (px_euler_step). `dt`, if given, is a float64 CUDA tensor of
    nsteps entries receiving each step's time step."""
    _same_layout(u_in, u_out)
    ctx = ctx or context(u_in.device.index)
    g = euler_grid_of(u_in, dx, dy)
    if dt is not None:
        import torch
        if dt.dtype != torch.float64 or not dt.is_cuda or dt.numel() < nsteps or not dt.is_contiguous():
            raise ValueError(f"dt must be a contiguous CUDA float64 tensor of >= {nsteps}")
    ctx.check(load_library().px_euler_step(ctx.handle, ctypes.byref(g), _ptr(u_in), _ptr(u_out),
                                           float(gamma), float(cfl), int(nsteps), float(dt_fixed),
                                           _ptr(dt), _stream(stream)))
    return u_out


def euler_conserved(w, u, dx: float = 1.0, dy: float = 1.0, gamma: float = 1.4,
                    ctx: Context | None = None, stream=None):
    """Conserved planes (rho, rho u, rho v, E) from primitive planes (rho, u, v, p)."""
    _same_layout(w, u)
    ctx = ctx or context(w.device.index)
    g = euler_grid_of(w, dx, dy)
    ctx.check(load_library().px_euler_conserved(ctx.handle, ctypes.byref(g), _ptr(w), _ptr(u),
                                                float(gamma), _stream(stream)))
    return u


class Batch:
    """px_batch_plan / px_batch_run: many independent instances in one persistent
    launch replayed from a CUDA graph. `grids` are Grid layouts (or tensors,
    whose layout is taken with h = 1 / nx)."""

    def __init__(self, grids, nsweeps: int, omega: float = 2.0 / 3.0, report_every: int = 0,
                 tune_cache: str | None = None, tune: bool = False, ctx: Context | None = None):
        self.ctx = ctx or context()
        gs = [g if isinstance(g, Grid) else grid_of(g, 1.0 / g.shape[1]) for g in grids]
        self.n = len(gs)
        self.nsweeps = int(nsweeps)
        self.every = int(report_every)
        self.nrep = (self.nsweeps + self.every - 1) // self.every if self.every > 0 else 0
        arr = (Grid * self.n)(*gs)
        h = _vp()
        self.ctx.check(load_library().px_batch_plan(
            self.ctx.handle, self.n, arr, self.nsweeps, float(omega), self.every,
            tune_cache.encode() if tune_cache else None, 1 if tune else 0, ctypes.byref(h)))
        self.handle = h

    def describe(self) -> dict:
        import json
        return json.loads(load_library().px_batch_describe(self.handle).decode())

    def run(self, phis, rhos, resid=None, stream=None):
        if len(phis) != self.n or len(rhos) != self.n:
            raise ValueError("one phi and one rho per instance")
        pa = (_vp * self.n)(*[p.data_ptr() for p in phis])
        ra = (_vp * self.n)(*[r.data_ptr() for r in rhos])
        if resid is not None and resid.numel() < self.n * self.nrep:
            raise ValueError("resid needs n * nrep entries")
        self.ctx.check(load_library().px_batch_run(self.handle, pa, ra, _ptr(resid),
                                                   _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            load_library().px_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Cnn:
    """The learned initial-guess network (px_cnn_*): 6 periodic 3x3 conv layers,
    BF16 on the tensor cores, trained with Adam by the library's kernels.
    Images are CUDA tensors (B, H, W); H % 4 == 0 and W % 64 == 0."""

    def __init__(self, seed: int = 0, dilations=None, ctx: Context | None = None):
        self.ctx = ctx or context()
        h = _vp()
        self.dilations = tuple(dilations) if dilations is not None else (1,) * 6
        dil = (ctypes.c_int32 * 6)(*self.dilations)
        self.ctx.check(load_library().px_cnn_create(self.ctx.handle, int(seed), dil,
                                                    ctypes.byref(h)))
        self.handle = h
        self.nparams = int(load_library().px_cnn_param_count())

    def params(self):
        import numpy as np
        out = np.empty(self.nparams, dtype=np.float32)
        self.ctx.check(load_library().px_cnn_get_params(
            self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), self.nparams))
        return out

    def set_params(self, p):
        import numpy as np
        p = np.ascontiguousarray(p, dtype=np.float32)
        self.ctx.check(load_library().px_cnn_set_params(
            self.handle, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), self.nparams))

    def state(self):
        """(flat FP32 parameters + Adam moments, step) for checkpoints."""
        import numpy as np
        n = int(load_library().px_cnn_state_count())
        out = np.empty(n, dtype=np.float32)
        step = ctypes.c_int64()
        self.ctx.check(load_library().px_cnn_get_state(
            self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n, ctypes.byref(step)))
        return out, step.value

    def set_state(self, flat, step: int):
        import numpy as np
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        self.ctx.check(load_library().px_cnn_set_state(
            self.handle, flat.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), flat.size, int(step)))

    def forward(self, x, y, stream=None):
        B, H, W = x.shape
        self.ctx.check(load_library().px_cnn_forward(self.handle, x.data_ptr(), y.data_ptr(),
                                                     B, H, W, _stream(stream)))
        return y

    def grads(self, x, t, stream=None):
        import numpy as np
        B, H, W = x.shape
        g = np.empty(self.nparams, dtype=np.float32)
        loss = ctypes.c_double()
        self.ctx.check(load_library().px_cnn_grads(
            self.handle, x.data_ptr(), t.data_ptr(), B, H, W,
            g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(loss), _stream(stream)))
        return g, loss.value

    def train_step(self, x, t, lr: float, want_loss: bool = True, stream=None):
        B, H, W = x.shape
        loss = ctypes.c_double()
        self.ctx.check(load_library().px_cnn_train_step(
            self.handle, x.data_ptr(), t.data_ptr(), B, H, W, float(lr),
            ctypes.byref(loss) if want_loss else None, _stream(stream)))
        return loss.value if want_loss else None

    def prepare(self, rho, phi, x, t, h: float, stream=None):
        import numpy as np
        B, H, W = rho.shape
        sc = np.empty(B, dtype=np.float64)
        self.ctx.check(load_library().px_cnn_prepare(
            self.handle, rho.data_ptr(), _ptr(phi), x.data_ptr(), _ptr(t), B, H, W, float(h),
            sc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream(stream)))
        return sc

    def hidden(self, layer: int, which: str, shape, stream=None):
        """Hidden tensor of the last forward pass as a (B, H, W, 32) float32 array
        of its BF16 values: which = "a" (activation) or "z" (pre-activation)."""
        import numpy as np
        B, H, W = shape
        n = B * H * W * 32
        raw = np.empty(n, dtype=np.uint16)
        self.ctx.check(load_library().px_cnn_get_hidden(
            self.handle, int(layer), 0 if which == "a" else 1,
            raw.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)), n, _stream(stream)))
        f = (raw.astype(np.uint32) << 16).view(np.float32).reshape(B, 4, H, W, 8)
        return f.transpose(0, 2, 3, 1, 4).reshape(B, H, W, 32)

    def set_wait_limit(self, polls: int):
        """px_cnn_set_wait_limit: polls per handshake wait of the tensor-core
        kernels (0 = default)."""
        self.ctx.check(load_library().px_cnn_set_wait_limit(self.handle, int(polls)))

    def set_staging(self, mode: int):
        """px_cnn_set_staging: 1 tensor-memory-accelerator boxes for in-image tap
        tiles (default), 0 per-pixel copies only."""
        self.ctx.check(load_library().px_cnn_set_staging(self.handle, int(mode)))

    def set_relabel(self, on: bool):
        """px_cnn_set_relabel: 1 dilated layers over relabelled activations
        (unit-offset taps, the default), 0 natural order with offset tap tiles."""
        self.ctx.check(load_library().px_cnn_set_relabel(self.handle, int(on)))

    def guess(self, rho, phi0, h: float, stream=None):
        B, H, W = rho.shape
        self.ctx.check(load_library().px_cnn_guess(self.handle, rho.data_ptr(), phi0.data_ptr(),
                                                   B, H, W, float(h), _stream(stream)))
        return phi0

    def close(self):
        if getattr(self, "handle", None):
            load_library().px_cnn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cnn_unflatten(p):
    """Flat parameter vector -> [(W (Cout, Cin, 3, 3), b (Cout,))] per layer."""
    import numpy as np
    widths = (1, 32, 32, 32, 32, 32, 1)
    out, o = [], 0
    for cin, cout in zip(widths[:-1], widths[1:]):
        w = np.asarray(p[o:o + cout * cin * 9]).reshape(cout, cin, 3, 3)
        o += cout * cin * 9
        b = np.asarray(p[o:o + cout])
        o += cout
        out.append((w, b))
    return out
