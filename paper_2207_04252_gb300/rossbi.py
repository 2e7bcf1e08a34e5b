"""Thin ctypes binding of librossbi.so (C ABI in include/rossbi.h).

Argument marshalling only: every step of the update runs in the library's
CUDA kernels.  The functions carry the C names.  State arguments are either a
CUDA tensor of shape (nfields, nz, nth, nr) or a sequence of per-field CUDA
tensors; their dtype must match the grid's precision form (float64 for
ROSSBI_FP64 / ROSSBI_FP64_PERT, float32 for ROSSBI_FP32_PERT).

Importing this module does not need a GPU; loading the library does.  There is
no CPU fallback: if the library is missing, load() raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librossbi.so")

ROSSBI_OK, ROSSBI_ERR_ARG, ROSSBI_ERR_CUDA, ROSSBI_ERR_OOM, ROSSBI_ERR_NONPHYSICAL, ROSSBI_ERR_RIEMANN, \
    ROSSBI_ERR_UNSUPPORTED = range(7)
ROSSBI_GEOM_BOX, ROSSBI_GEOM_CYL = 0, 1
ROSSBI_BC_PERIODIC, ROSSBI_BC_OUTFLOW, ROSSBI_BC_EQUILIBRIUM = 0, 1, 2
ROSSBI_FP64, ROSSBI_FP32_PERT, ROSSBI_FP64_PERT = 0, 1, 2
ROSSBI_RECON_CONSERVATIVE, ROSSBI_RECON_PRIMITIVE = 0, 1

# every function declared in include/rossbi.h
EXPORTS = (
    "rossbi_init_grid", "rossbi_set_equilibrium", "rossbi_set_indirect", "rossbi_indirect_moments", "rossbi_set_damping", "rossbi_set_vertical_damping", "rossbi_set_dust_species", "rossbi_pack_theta_rows",
    "rossbi_unpack_theta_rows", "rossbi_get_equilibrium", "rossbi_cfl_dt", "rossbi_step",
    "rossbi_step_host", "rossbi_step_noalloc", "rossbi_adjoint_step", "rossbi_adjoint_dstokes",
    "rossbi_conservation_sums", "rossbi_fallback_count", "rossbi_take_status", "rossbi_profile_enable",
    "rossbi_measure_fma_peak",
    "rossbi_profile_read", "rossbi_nfields", "rossbi_precision", "rossbi_destroy", "rossbi_status_string",
)


class rossbi_grid_desc(ctypes.Structure):
    _fields_ = [("geometry", ctypes.c_int), ("nr", ctypes.c_int), ("nth", ctypes.c_int), ("nz", ctypes.c_int),
                ("x0", ctypes.c_double * 3), ("x1", ctypes.c_double * 3),
                ("bc_lo", ctypes.c_int * 3), ("bc_hi", ctypes.c_int * 3),
                ("gamma", ctypes.c_double), ("gm", ctypes.c_double), ("omega_frame", ctypes.c_double),
                ("cfl", ctypes.c_double), ("n_dust", ctypes.c_int), ("precision", ctypes.c_int),
                ("recon", ctypes.c_int)]


class rossbi_disc_params(ctypes.Structure):
    _fields_ = [("sigma0", ctypes.c_double), ("beta_sigma", ctypes.c_double), ("T0", ctypes.c_double),
                ("beta_T", ctypes.c_double), ("bump_delta", ctypes.c_double), ("bump_r0", ctypes.c_double),
                ("bump_width", ctypes.c_double)]


class rossbi_dust_params(ctypes.Structure):
    _fields_ = [("stokes", ctypes.c_double), ("drag_law", ctypes.c_int), ("kappa", ctypes.c_double)]


class rossbi_damping_params(ctypes.Structure):
    _fields_ = [("r_edge_in", ctypes.c_double), ("r_edge_out", ctypes.c_double), ("period_factor", ctypes.c_double)]


class rossbi_vertical_damping_params(ctypes.Structure):
    _fields_ = [("z_edge", ctypes.c_double), ("period_factor", ctypes.c_double)]


class RossbiError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} ({code})")


_lib = None
_VP = ctypes.c_void_p
_PP = ctypes.POINTER(ctypes.c_void_p)
_DP = ctypes.POINTER(ctypes.c_double)


def load(path: str = LIB_PATH):
    """Load librossbi.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librossbi.so not found at {path}; build it with paper_2207_04252_gb300.build")
    L = ctypes.CDLL(path)
    L.rossbi_init_grid.argtypes = [ctypes.POINTER(rossbi_grid_desc), _VP, ctypes.POINTER(_VP)]
    L.rossbi_set_equilibrium.argtypes = [_VP, ctypes.POINTER(rossbi_disc_params)]
    L.rossbi_set_indirect.argtypes = [_VP, ctypes.c_double]
    L.rossbi_indirect_moments.argtypes = [_VP, _PP, _DP]
    L.rossbi_set_damping.argtypes = [_VP, ctypes.POINTER(rossbi_damping_params)]
    L.rossbi_set_dust_species.argtypes = [_VP, _DP, ctypes.c_int]
    L.rossbi_set_vertical_damping.argtypes = [_VP, ctypes.POINTER(rossbi_vertical_damping_params)]
    L.rossbi_pack_theta_rows.argtypes = [_VP, _PP, ctypes.c_int, ctypes.c_int, _VP]
    L.rossbi_unpack_theta_rows.argtypes = [_VP, _PP, ctypes.c_int, ctypes.c_int, _VP]
    L.rossbi_get_equilibrium.argtypes = [_VP, _DP]
    L.rossbi_cfl_dt.argtypes = [_VP, _PP, _DP]
    L.rossbi_step.argtypes = [_VP, _PP, _PP, ctypes.c_double, ctypes.POINTER(rossbi_dust_params), _DP]
    L.rossbi_step_host.argtypes = [_VP, _PP, ctypes.c_double, ctypes.POINTER(rossbi_dust_params), _DP]
    L.rossbi_step_noalloc.argtypes = [_VP, _PP, ctypes.c_double, ctypes.POINTER(rossbi_dust_params), _DP]
    L.rossbi_adjoint_step.argtypes = [_VP, _PP, ctypes.c_double, ctypes.POINTER(rossbi_dust_params), _PP, _PP, _DP]
    L.rossbi_adjoint_dstokes.argtypes = [_VP, _DP, ctypes.c_int]
    L.rossbi_conservation_sums.argtypes = [_VP, _PP, _DP]
    L.rossbi_take_status.argtypes = [_VP]
    L.rossbi_fallback_count.argtypes = [_VP, ctypes.POINTER(ctypes.c_ulonglong)]
    L.rossbi_measure_fma_peak.argtypes = [ctypes.c_int, _VP, ctypes.POINTER(ctypes.c_double)]
    L.rossbi_profile_enable.argtypes = [_VP, ctypes.c_int]
    L.rossbi_profile_read.argtypes = [_VP, _DP, ctypes.POINTER(ctypes.c_int)]
    L.rossbi_nfields.argtypes = [_VP]
    L.rossbi_precision.argtypes = [_VP]
    L.rossbi_destroy.argtypes = [_VP]
    L.rossbi_destroy.restype = None
    L.rossbi_status_string.argtypes = [ctypes.c_int]
    L.rossbi_status_string.restype = ctypes.c_char_p
    _lib = L
    return L


def status_string(code: int) -> str:
    return load().rossbi_status_string(int(code)).decode()


def _check(code, where):
    if code != ROSSBI_OK:
        raise RossbiError(code, where)


def _fields(state, nf):
    if state is None:
        return None
    if hasattr(state, "data_ptr") and getattr(state, "dim", lambda: 0)() == 4:
        assert state.shape[0] == nf and state.is_contiguous()
        ptrs = [state[f].data_ptr() for f in range(nf)]
    elif isinstance(state, np.ndarray):
        assert state.shape[0] == nf and state.flags.c_contiguous
        step = state[0].nbytes
        ptrs = [state.ctypes.data + f * step for f in range(nf)]
    else:
        ptrs = [t.data_ptr() if hasattr(t, "data_ptr") else int(t) for t in state]
        assert len(ptrs) == nf
    return (ctypes.c_void_p * nf)(*ptrs)


def _stream_handle(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)


def make_desc(geometry, n, x0, x1, bc_lo, bc_hi, gamma=1.4, gm=1.0, omega_frame=0.0, cfl=0.5, n_dust=0,
              precision=ROSSBI_FP64, recon=ROSSBI_RECON_CONSERVATIVE) -> rossbi_grid_desc:
    return rossbi_grid_desc(geometry, n[0], n[1], n[2], (ctypes.c_double * 3)(*x0), (ctypes.c_double * 3)(*x1),
                            (ctypes.c_int * 3)(*bc_lo), (ctypes.c_int * 3)(*bc_hi), gamma, gm, omega_frame, cfl,
                            n_dust, precision, recon)


def rossbi_init_grid(desc: rossbi_grid_desc, stream=None):
    h = ctypes.c_void_p()
    _check(load().rossbi_init_grid(ctypes.byref(desc), _stream_handle(stream), ctypes.byref(h)), "rossbi_init_grid")
    return h


def rossbi_set_equilibrium(grid, disc):
    # four power-law parameters, optionally followed by the bump's three
    p = None if disc is None else ctypes.byref(rossbi_disc_params(*disc))
    _check(load().rossbi_set_equilibrium(grid, p), "rossbi_set_equilibrium")


def rossbi_nfields(grid) -> int:
    return load().rossbi_nfields(grid)


def rossbi_precision(grid) -> int:
    return load().rossbi_precision(grid)


def rossbi_get_equilibrium(grid, nz, nr) -> np.ndarray:
    out = np.zeros((5, nz, nr))
    _check(load().rossbi_get_equilibrium(grid, out.ctypes.data_as(_DP)), "rossbi_get_equilibrium")
    return out


def rossbi_cfl_dt(grid, state) -> float:
    dt = ctypes.c_double()
    _check(load().rossbi_cfl_dt(grid, _fields(state, rossbi_nfields(grid)), ctypes.byref(dt)), "rossbi_cfl_dt")
    return dt.value


def rossbi_step(grid, state, scratch=None, dt=0.0, dust=None, want_next_dt=False):
    """One RK2 step in place.  Returns the next CFL dt when want_next_dt (synchronising), else None."""
    nf = rossbi_nfields(grid)
    d = None if dust is None else ctypes.byref(rossbi_dust_params(*dust))
    nd = ctypes.c_double()
    code = load().rossbi_step(grid, _fields(state, nf), _fields(scratch, nf), float(dt), d,
                              ctypes.byref(nd) if want_next_dt else None)
    _check(code, "rossbi_step")
    return nd.value if want_next_dt else None


def rossbi_step_noalloc(grid, state, dt=0.0, dust=None, want_next_dt=False):
    """rossbi_step with its scratch in the library's fixed device array (no allocation).
    For callers that cannot allocate device memory while stepping; see include/rossbi.h
    for the size limit and the rule that overlapping calls must be serialised."""
    nf = rossbi_nfields(grid)
    d = None if dust is None else ctypes.byref(rossbi_dust_params(*dust))
    nd = ctypes.c_double()
    _check(load().rossbi_step_noalloc(grid, _fields(state, nf), float(dt), d,
                                      ctypes.byref(nd) if want_next_dt else None), "rossbi_step_noalloc")
    return nd.value if want_next_dt else None


def rossbi_adjoint_step(grid, state, dt, dust, lam_np1, lam_n, want_dstokes=False):
    """Cotangent of E^n from the cotangent of E^{n+1} for one FP64 step of length dt
    (lam_n may be lam_np1).  Returns this step's lambda . dE^{n+1}/dSt if
    want_dstokes (the call then synchronises), else None; the library also keeps
    a running total (rossbi_adjoint_dstokes)."""
    nf = rossbi_nfields(grid)
    d = None if dust is None else ctypes.byref(rossbi_dust_params(*dust))
    v = ctypes.c_double(0.0)
    _check(load().rossbi_adjoint_step(grid, _fields(state, nf), float(dt), d, _fields(lam_np1, nf),
                                      _fields(lam_n, nf), ctypes.byref(v) if want_dstokes else None),
           "rossbi_adjoint_step")
    return v.value if want_dstokes else None


def rossbi_set_indirect(grid, x_ref):
    """Indirect gravity of Sect. 2.10 with constant X_ref (0 switches it off)."""
    _check(load().rossbi_set_indirect(grid, float(x_ref)), "rossbi_set_indirect")


def rossbi_set_damping(grid, zones):
    """Wave-killing zones (r_edge_in, r_edge_out, period_factor), or None for off."""
    p = None if zones is None else ctypes.byref(rossbi_damping_params(*map(float, zones)))
    _check(load().rossbi_set_damping(grid, p), "rossbi_set_damping")


def rossbi_set_vertical_damping(grid, zone):
    """Vertical sheared damped boundary (z_edge, period_factor), or None for off."""
    p = None if zone is None else ctypes.byref(rossbi_vertical_damping_params(*map(float, zone)))
    _check(load().rossbi_set_vertical_damping(grid, p), "rossbi_set_vertical_damping")


def rossbi_set_dust_species(grid, stokes_factors):
    """Stokes-number factors of the dust species (factor[0] must be 1)."""
    f = np.ascontiguousarray(stokes_factors, dtype=np.float64)
    _check(load().rossbi_set_dust_species(grid, f.ctypes.data_as(_DP), len(f)), "rossbi_set_dust_species")


def rossbi_pack_theta_rows(grid, state, j0, rows, buf):
    """Copy theta rows j0 .. j0 + rows - 1 of every field into the device buffer buf."""
    _check(load().rossbi_pack_theta_rows(grid, _fields(state, rossbi_nfields(grid)), int(j0), int(rows),
                                         ctypes.c_void_p(buf.data_ptr())), "rossbi_pack_theta_rows")


def rossbi_unpack_theta_rows(grid, state, j0, rows, buf):
    """Copy the device buffer buf into theta rows j0 .. j0 + rows - 1 of every field."""
    _check(load().rossbi_unpack_theta_rows(grid, _fields(state, rossbi_nfields(grid)), int(j0), int(rows),
                                           ctypes.c_void_p(buf.data_ptr())), "rossbi_unpack_theta_rows")


def rossbi_indirect_moments(grid, state) -> np.ndarray:
    """(A_disc, B_disc) of Sect. 2.10 of a state (without X_ref)."""
    out = np.zeros(2)
    _check(load().rossbi_indirect_moments(grid, _fields(state, rossbi_nfields(grid)), out.ctypes.data_as(_DP)),
           "rossbi_indirect_moments")
    return out


def rossbi_adjoint_dstokes(grid, reset=False) -> float:
    """Running total of d/dSt over the adjoint steps since the last reset."""
    v = ctypes.c_double()
    _check(load().rossbi_adjoint_dstokes(grid, ctypes.byref(v), int(bool(reset))), "rossbi_adjoint_dstokes")
    return v.value


def rossbi_step_host(grid, host_state, dt=0.0, dust=None):
    """Step a host-resident state (numpy array (nf, nz, nth, nr)); returns the next dt."""
    nf = rossbi_nfields(grid)
    d = None if dust is None else ctypes.byref(rossbi_dust_params(*dust))
    nd = ctypes.c_double()
    _check(load().rossbi_step_host(grid, _fields(host_state, nf), float(dt), d, ctypes.byref(nd)),
           "rossbi_step_host")
    return nd.value


def rossbi_conservation_sums(grid, state) -> np.ndarray:
    nf = rossbi_nfields(grid)
    out = np.zeros(nf)
    _check(load().rossbi_conservation_sums(grid, _fields(state, nf), out.ctypes.data_as(_DP)),
           "rossbi_conservation_sums")
    return out


def rossbi_measure_fma_peak(fp64: bool, stream=None) -> float:
    """Measured FMA throughput of the device in FLOP/s (FP32 or FP64)."""
    v = ctypes.c_double()
    _check(load().rossbi_measure_fma_peak(int(bool(fp64)), _stream_handle(stream), ctypes.byref(v)),
           "rossbi_measure_fma_peak")
    return v.value


def rossbi_fallback_count(grid) -> int:
    n = ctypes.c_ulonglong()
    _check(load().rossbi_fallback_count(grid, ctypes.byref(n)), "rossbi_fallback_count")
    return n.value


def rossbi_take_status(grid) -> int:
    return load().rossbi_take_status(grid)


def rossbi_profile_enable(grid, enable=True):
    _check(load().rossbi_profile_enable(grid, int(bool(enable))), "rossbi_profile_enable")


def rossbi_profile_read(grid):
    """(summed stage-kernel device ms, number of stage launches) since the last read."""
    ms = ctypes.c_double()
    n = ctypes.c_int()
    _check(load().rossbi_profile_read(grid, ctypes.byref(ms), ctypes.byref(n)), "rossbi_profile_read")
    return ms.value, n.value


def rossbi_destroy(grid):
    if grid:
        load().rossbi_destroy(grid)
