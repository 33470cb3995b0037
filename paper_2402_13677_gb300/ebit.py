"""Thin ctypes binding of libebit.so (include/ebit.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module only converts numpy arrays
and torch tensors to pointers, fills the C structs and turns status codes into exceptions.
There is no CPU fallback: importing works anywhere, but load() raises if the compiled
library is missing.

PyTorch is used for device memory (the library allocates its arena through a torch-backed
allocator callback) and for the CUDA stream the work is ordered on.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libebit.so")

# status codes
EBIT_OK, EBIT_EINVAL, EBIT_ENOMEM, EBIT_ENOCONV, EBIT_ETOPO, EBIT_ECUDA, EBIT_ECFL, EBIT_ENONFINITE = (
    0, -1, -2, -3, -4, -5, -6, -7)
STATUS_NAMES = {0: "EBIT_OK", -1: "EBIT_EINVAL", -2: "EBIT_ENOMEM", -3: "EBIT_ENOCONV", -4: "EBIT_ETOPO",
                -5: "EBIT_ECUDA", -6: "EBIT_ECFL", -7: "EBIT_ENONFINITE"}
EBIT_FP64, EBIT_MIXED = 0, 1

# field ids
(F_T_L, F_T_V, F_U_L, F_U_V, F_UFX_L, F_UFX_V, F_UFY_L, F_UFY_V, F_P, F_GC, F_MDOT, F_VF, F_CCOL, F_BAND, F_NB,
 F_VCOL, F_HX_POS, F_VY_POS, F_TSTAR_L, F_TSTAR_V, F_CSEG, F_UG) = range(22)
FIELD_DTYPES = {F_CCOL: np.uint8, F_BAND: np.uint8, F_VCOL: np.uint8, F_CSEG: np.uint16}

# stages
(STAGE_PREPARE, STAGE_RECONSTRUCT, STAGE_ADVECT_T, STAGE_EXTEND_TSTAR, STAGE_ADVANCE_INTERFACE, STAGE_SOLVE_ENERGY,
 STAGE_EXTEND_T, STAGE_MASS_FLUX, STAGE_GHOST_VELOCITY, STAGE_MOMENTUM, STAGE_DIAGNOSTICS) = range(11)

EXPORTS = ["ebit_init", "ebit_set_phase_props", "ebit_set_interface", "ebit_set_field", "ebit_get_field",
           "ebit_set_fields", "ebit_get_fields", "ebit_field_shape", "ebit_set_time", "ebit_run_stage", "ebit_step", "ebit_get_diagnostics",
           "ebit_launch_count", "ebit_timing_begin", "ebit_timing_end", "ebit_set_option", "ebit_solve_system",
           "ebit_solve_system_noalloc", "ebit_autotune", "ebit_get_schedule", "ebit_last_error",
           "ebit_destroy", "ebit_version"]
EBIT_OPT_GRAPH = 1
EBIT_OPT_TMA = 2
EBIT_OPT_COOP = 3
EBIT_OPT_BARRIER_SPIN = 4
EBIT_OPT_EXT_BLOCK = 5
EBIT_KT_SMOOTH_L0 = 1


class ebit_config(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("x0", C.c_double), ("y0", C.c_double), ("h", C.c_double),
                ("bc", C.c_int * 4), ("T_fixed", C.c_int * 4), ("T_wall", C.c_double * 4), ("dt", C.c_double),
                ("precision", C.c_int), ("rtol", C.c_double), ("max_iter", C.c_int), ("extend_iters", C.c_int),
                ("theta_min", C.c_double), ("sweep_order", C.c_int), ("energy", C.c_int),
                ("mdot_fixed", C.c_double), ("one_fluid", C.c_int), ("axisymmetric", C.c_int)]


class ebit_phase_props(C.Structure):
    _fields_ = [("rho", C.c_double), ("mu", C.c_double), ("lambda_", C.c_double), ("cp", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class ebit_allocator(C.Structure):
    _fields_ = [("alloc_fn", ALLOC_FN), ("free_fn", FREE_FN), ("user", C.c_void_p)]


class EbitError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libebit.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libebit.so not built ({path}); run __graft_entry__.build() first")
    lib = C.CDLL(path)
    vp, i32, f64 = C.c_void_p, C.c_int, C.c_double
    lib.ebit_init.argtypes = [C.POINTER(ebit_config), i32, vp, C.POINTER(ebit_allocator), C.POINTER(vp)]
    lib.ebit_set_phase_props.argtypes = [vp, i32, C.POINTER(ebit_phase_props), C.POINTER(ebit_phase_props), f64, f64,
                                         f64, f64, f64]
    lib.ebit_set_interface.argtypes = [vp, i32, vp, vp, vp, i32]
    lib.ebit_set_field.argtypes = [vp, i32, i32, vp, i32]
    lib.ebit_get_field.argtypes = [vp, i32, i32, vp, i32]
    lib.ebit_set_fields.argtypes = [vp, i32, i32, C.POINTER(C.c_int), C.POINTER(vp), i32]
    lib.ebit_get_fields.argtypes = [vp, i32, i32, C.POINTER(C.c_int), C.POINTER(vp), i32]
    lib.ebit_field_shape.argtypes = [vp, i32, i32, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
    lib.ebit_set_time.argtypes = [vp, i32, f64]
    lib.ebit_run_stage.argtypes = [vp, i32]
    lib.ebit_step.argtypes = [vp, i32]
    lib.ebit_get_diagnostics.argtypes = [vp, i32, C.POINTER(C.c_double), i32]
    lib.ebit_launch_count.argtypes = [vp]
    lib.ebit_launch_count.restype = C.c_uint64
    lib.ebit_timing_begin.argtypes = [vp, i32]
    lib.ebit_set_option.argtypes = [vp, i32, i32]
    lib.ebit_solve_system.argtypes = [vp, i32, vp, vp, vp, vp, vp, i32, i32, f64, i32, C.POINTER(C.c_int),
                                      C.POINTER(C.c_double)]
    lib.ebit_solve_system_noalloc.argtypes = [i32, i32, vp, vp, vp, vp, vp, i32, i32, f64, i32, vp,
                                              C.POINTER(C.c_int), C.POINTER(C.c_double)]
    lib.ebit_timing_end.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_uint64), C.POINTER(C.c_double)]
    lib.ebit_autotune.argtypes = [vp, i32]
    lib.ebit_get_schedule.argtypes = [vp, i32, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_int),
                                      C.POINTER(C.c_int)]
    lib.ebit_last_error.argtypes = [vp]
    lib.ebit_last_error.restype = C.c_char_p
    lib.ebit_destroy.argtypes = [vp]
    lib.ebit_destroy.restype = None
    lib.ebit_version.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("ebit_launch_count", "ebit_last_error", "ebit_destroy", "ebit_version"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(ctx, status):
    if status != EBIT_OK:
        raise EbitError(status, load().ebit_last_error(ctx).decode())
    return status


def check(ctx, status):
    """Raise EbitError for a non-OK status returned by a direct call into the library."""
    _check(ctx, status)


# ------------------------------------------------------------------ torch-backed device memory
class TorchAllocator:
    """Device allocator callback backed by torch tensors (kept alive until freed)."""

    def __init__(self, device=None):
        import torch
        self.torch = torch
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.live = {}
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)
        self.struct = ebit_allocator(self._alloc, self._free, None)

    def _do_alloc(self, nbytes, user):
        t = self.torch.empty(int(nbytes) + 256, dtype=self.torch.uint8, device=self.device)
        ptr = t.data_ptr()
        aligned = (ptr + 255) & ~255
        self.live[aligned] = t
        return aligned

    def _do_free(self, ptr, user):
        self.live.pop(ptr, None)


# ------------------------------------------------------------------ same-name marshalling wrappers
def ebit_init(cfgs, stream=None, allocator=None):
    lib = load()
    arr = (ebit_config * len(cfgs))(*cfgs)
    out = C.c_void_p()
    _check(None, lib.ebit_init(arr, len(cfgs), C.c_void_p(stream or 0),
                               C.byref(allocator.struct) if allocator is not None else None, C.byref(out)))
    return out


def ebit_set_phase_props(ctx, inst, liq, vap, T_sat, h_lg, sigma, gx, gy):
    _check(ctx, load().ebit_set_phase_props(ctx, inst, C.byref(liq), C.byref(vap), T_sat, h_lg, sigma, gx, gy))


def _host_ptr(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


def ebit_set_interface(ctx, inst, vcol, hx_pos, vy_pos):
    v, pv = _host_ptr(vcol, np.uint8)
    hp, ph = _host_ptr(hx_pos, np.float64)
    vp_, pvv = _host_ptr(vy_pos, np.float64)
    _check(ctx, load().ebit_set_interface(ctx, inst, pv, ph, pvv, 0))


def ebit_set_field(ctx, inst, field, data):
    """data: numpy array (host) or torch CUDA tensor (device)."""
    if hasattr(data, "data_ptr") and getattr(data, "is_cuda", False):
        _check(ctx, load().ebit_set_field(ctx, inst, field, data.data_ptr(), 1))
        return
    a, p = _host_ptr(data, FIELD_DTYPES.get(field, np.float64))
    _check(ctx, load().ebit_set_field(ctx, inst, field, p, 0))


def ebit_field_shape(ctx, inst, field):
    n, e = C.c_size_t(), C.c_size_t()
    _check(ctx, load().ebit_field_shape(ctx, inst, field, C.byref(n), C.byref(e)))
    return n.value, e.value


def _field_batch(fields, ptrs):
    n = len(fields)
    ids = (C.c_int * n)(*fields)
    pp = (C.c_void_p * n)(*ptrs)
    return n, ids, pp


def ebit_set_fields(ctx, inst, fields, ptrs, on_device):
    """Copy several fields in with one call: fields (ids) and raw pointers (host page-locked or
    device, per on_device), one synchronisation for host pointers."""
    n, ids, pp = _field_batch(fields, ptrs)
    _check(ctx, load().ebit_set_fields(ctx, inst, n, ids, pp, 1 if on_device else 0))


def ebit_get_fields(ctx, inst, fields, ptrs, on_device):
    """Copy several fields out with one call (raw pointers as for ebit_set_fields)."""
    n, ids, pp = _field_batch(fields, ptrs)
    _check(ctx, load().ebit_get_fields(ctx, inst, n, ids, pp, 1 if on_device else 0))


def ebit_get_field(ctx, inst, field, out=None):
    """Copy a field to host (numpy, flat) or into a torch CUDA tensor `out`."""
    if out is not None and hasattr(out, "data_ptr") and getattr(out, "is_cuda", False):
        _check(ctx, load().ebit_get_field(ctx, inst, field, out.data_ptr(), 1))
        return out
    n, e = ebit_field_shape(ctx, inst, field)
    dt = FIELD_DTYPES.get(field, np.float64)
    count = n * e // np.dtype(dt).itemsize
    a = np.empty(count, dtype=dt)
    _check(ctx, load().ebit_get_field(ctx, inst, field, a.ctypes.data, 0))
    return a


def ebit_set_time(ctx, inst, t):
    _check(ctx, load().ebit_set_time(ctx, inst, t))


def ebit_run_stage(ctx, stage):
    return _check(ctx, load().ebit_run_stage(ctx, stage))


def ebit_step(ctx, nsteps, allow_noconv=False):
    s = load().ebit_step(ctx, nsteps)
    if s == EBIT_ENOCONV and allow_noconv:
        return s
    return _check(ctx, s)


def ebit_get_diagnostics(ctx, inst, n=14):
    buf = (C.c_double * n)()
    _check(ctx, load().ebit_get_diagnostics(ctx, inst, buf, n))
    return np.array(buf[:])


def ebit_launch_count(ctx):
    return int(load().ebit_launch_count(ctx))


def ebit_timing_begin(ctx, kernel_class=EBIT_KT_SMOOTH_L0):
    _check(ctx, load().ebit_timing_begin(ctx, kernel_class))


def ebit_timing_end(ctx):
    """(total kernel ms, launches, algorithmic bytes per launch) of the timed kernel class."""
    ms, n, b = C.c_double(), C.c_uint64(), C.c_double()
    _check(ctx, load().ebit_timing_end(ctx, C.byref(ms), C.byref(n), C.byref(b)))
    return ms.value, n.value, b.value


def ebit_set_option(ctx, option, value):
    _check(ctx, load().ebit_set_option(ctx, option, value))


def ebit_autotune(ctx, trial_steps=2):
    """Time candidate multigrid schedules per batch / instance, keep the fastest (state restored)."""
    _check(ctx, load().ebit_autotune(ctx, trial_steps))


def ebit_get_schedule(ctx, inst):
    """(single-block level size, inner FP32 tolerance, TMA staging, cooperative coarse cycle)."""
    sm, it, tm, co = C.c_int(), C.c_double(), C.c_int(), C.c_int()
    _check(ctx, load().ebit_get_schedule(ctx, inst, C.byref(sm), C.byref(it), C.byref(tm), C.byref(co)))
    return sm.value, it.value, tm.value, co.value


def ebit_solve_system(ctx, inst, D, wl, wb, b, x0=None, nr=1, precision=EBIT_FP64, rtol=1e-10, max_iter=500,
                      allow_noconv=False):
    """Solve the five-point system (D, wl, wb cell arrays) for b (nr interleaved RHS); returns (x, iters, relres)."""
    Dp = np.ascontiguousarray(D, np.float64)
    wlp = np.ascontiguousarray(wl, np.float64)
    wbp = np.ascontiguousarray(wb, np.float64)
    bp = np.ascontiguousarray(b, np.float64)
    x = np.zeros_like(bp) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    it, rr = C.c_int(), C.c_double()
    s = load().ebit_solve_system(ctx, inst, Dp.ctypes.data, wlp.ctypes.data, wbp.ctypes.data, bp.ctypes.data,
                                 x.ctypes.data, nr, precision, rtol, max_iter, C.byref(it), C.byref(rr))
    if not (s == EBIT_ENOCONV and allow_noconv):
        _check(ctx, s)
    return x, it.value, rr.value


def ebit_solve_system_noalloc(nx, ny, D, wl, wb, b, x, nr=1, precision=EBIT_FP64, rtol=1e-10, max_iter=500,
                              stream=None):
    """Allocation-free solve on caller-owned device tensors (x is updated in place).
    Returns (status, iters, relres); the status is returned, not raised (no context holds a message)."""
    it, rr = C.c_int(), C.c_double()
    s = load().ebit_solve_system_noalloc(nx, ny, D.data_ptr(), wl.data_ptr(), wb.data_ptr(), b.data_ptr(),
                                         x.data_ptr(), nr, precision, rtol, max_iter, C.c_void_p(stream or 0),
                                         C.byref(it), C.byref(rr))
    return s, it.value, rr.value


def ebit_last_error(ctx):
    return load().ebit_last_error(ctx).decode()


def ebit_destroy(ctx):
    load().ebit_destroy(ctx)


def ebit_version():
    return load().ebit_version().decode()


# ------------------------------------------------------------------ problem marshalling helpers
def config_from_problem(pb, precision=EBIT_FP64, rtol=1e-8, max_iter=200):
    """ebit_config of a workloads.Problem (grid, boundaries, time step, solver settings)."""
    c = ebit_config()
    c.nx, c.ny, c.x0, c.y0, c.h = pb.nx, pb.ny, pb.x0, pb.y0, pb.h
    for s in range(4):
        c.bc[s] = int(pb.bc[s])
        c.T_fixed[s] = 0 if pb.T_bc[s] is None else 1
        c.T_wall[s] = 0.0 if pb.T_bc[s] is None else float(pb.T_bc[s])
    c.dt = pb.dt
    c.precision = precision
    c.rtol = rtol
    c.max_iter = max_iter
    c.extend_iters = pb.extend_iters
    c.theta_min = pb.theta_min
    c.sweep_order = pb.sweep_order
    c.energy = 1 if pb.energy else 0
    c.mdot_fixed = pb.mdot_fixed
    c.one_fluid = 1 if getattr(pb, "one_fluid", False) else 0
    c.axisymmetric = 1 if getattr(pb, "axi", False) else 0
    return c


def props_from_problem(pb):
    return (ebit_phase_props(pb.rho_l, pb.mu_l, pb.lam_l, pb.cp_l),
            ebit_phase_props(pb.rho_v, pb.mu_v, pb.lam_v, pb.cp_v))


STATE_FIELDS = {"T_l": F_T_L, "T_v": F_T_V, "u_l": F_U_L, "u_v": F_U_V, "ufx_l": F_UFX_L, "ufx_v": F_UFX_V,
                "ufy_l": F_UFY_L, "ufy_v": F_UFY_V, "p": F_P, "gc": F_GC, "mdot": F_MDOT}


def upload_state(ctx, inst, pb, vcol, hx_pos, vy_pos, fields, t):
    """Interface + every field given in `fields` (name -> array), properties and time."""
    liq, vap = props_from_problem(pb)
    ebit_set_phase_props(ctx, inst, liq, vap, pb.T_sat, pb.h_lg, getattr(pb, "sigma", 0.0), pb.gx, pb.gy)
    ebit_set_interface(ctx, inst, vcol, hx_pos, vy_pos)
    for name, arr in fields.items():
        if arr is not None:
            ebit_set_field(ctx, inst, STATE_FIELDS[name], arr)
    ebit_set_time(ctx, inst, t)


def download(ctx, inst, nx, ny, names=None):
    """Fields as numpy arrays in their natural shapes."""
    shapes = {F_T_L: (ny, nx), F_T_V: (ny, nx), F_P: (ny, nx), F_MDOT: (ny, nx), F_VF: (ny, nx),
              F_TSTAR_L: (ny, nx), F_TSTAR_V: (ny, nx), F_CCOL: (ny, nx), F_BAND: (ny, nx), F_CSEG: (ny, nx),
              F_U_L: (ny, nx, 2), F_U_V: (ny, nx, 2), F_GC: (ny, nx, 2), F_NB: (ny, nx, 2), F_UG: (ny, nx, 2),
              F_UFX_L: (ny, nx + 1), F_UFX_V: (ny, nx + 1), F_VY_POS: (ny, nx + 1),
              F_UFY_L: (ny + 1, nx), F_UFY_V: (ny + 1, nx), F_HX_POS: (ny + 1, nx), F_VCOL: (ny + 1, nx + 1)}
    key = {"T_l": F_T_L, "T_v": F_T_V, "p": F_P, "mdot": F_MDOT, "vf": F_VF, "Ts_l": F_TSTAR_L,
           "Ts_v": F_TSTAR_V, "ccol": F_CCOL, "band": F_BAND, "cseg": F_CSEG, "u_l": F_U_L, "u_v": F_U_V,
           "gc": F_GC, "nb": F_NB, "uG": F_UG, "ufx_l": F_UFX_L, "ufx_v": F_UFX_V, "vy_pos": F_VY_POS,
           "ufy_l": F_UFY_L, "ufy_v": F_UFY_V, "hx_pos": F_HX_POS, "vcol": F_VCOL}
    out = {}
    for name in (names or key.keys()):
        f = key[name]
        out[name] = ebit_get_field(ctx, inst, f).reshape(shapes[f])
    return out
