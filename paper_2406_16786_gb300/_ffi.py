"""ctypes declarations of the sphbuf C ABI (include/sphbuf.h).  Marshalling only."""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsphbuf.so")

c_u64 = ctypes.c_uint64
c_u32 = ctypes.c_uint32
c_i32 = ctypes.c_int32
c_dbl = ctypes.c_double
P = ctypes.POINTER
vp = ctypes.c_void_p


class DomainDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("lo", c_dbl * 3), ("hi", c_dbl * 3), ("dp", c_dbl),
                ("h_over_dp", c_dbl), ("rho0", c_dbl), ("c0", c_dbl), ("nu", c_dbl), ("dt", c_dbl),
                ("capacity", c_u64)]


class BcParams(ctypes.Structure):
    _fields_ = [("umax", c_dbl), ("half_width", c_dbl), ("p_b", c_dbl), ("p_amp", c_dbl),
                ("p_omega", c_dbl), ("p_phase", c_dbl)]


# name -> (restype, argtypes); every entry point declared in include/sphbuf.h
SIGNATURES = {
    "sphbuf_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "sphbuf_error_message": (ctypes.c_char_p, [vp]),
    "sphbuf_create_domain": (ctypes.c_int, [P(DomainDesc), vp, P(vp)]),
    "sphbuf_destroy": (ctypes.c_int, [vp]),
    "sphbuf_set_walls": (ctypes.c_int, [vp, vp, c_u64]),
    "sphbuf_set_fluid": (ctypes.c_int, [vp, vp, vp, vp, c_u64]),
    "sphbuf_write_particles": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp, c_u64, c_u32]),
    "sphbuf_add_inout_buffer": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_int, P(BcParams), P(ctypes.c_int)]),
    "sphbuf_rotation_from_normal": (ctypes.c_int, [vp, c_dbl, vp]),
    "sphbuf_set_buffer_rotation": (ctypes.c_int, [vp, ctypes.c_int, vp, vp, c_dbl]),
    "sphbuf_set_windkessel": (ctypes.c_int, [vp, ctypes.c_int, c_dbl, c_dbl, c_dbl, c_dbl]),
    "sphbuf_set_background_pressure": (ctypes.c_int, [vp, c_dbl]),
    "sphbuf_set_transport_velocity": (ctypes.c_int, [vp, c_dbl]),
    "sphbuf_set_dual_time_stepping": (ctypes.c_int, [vp, ctypes.c_int]),
    "sphbuf_read_boundary_pressure": (ctypes.c_int, [vp, ctypes.c_int, P(c_dbl), P(c_dbl), P(c_dbl)]),
    "sphbuf_step": (ctypes.c_int, [vp, ctypes.c_int]),
    "sphbuf_step_phases": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_uint]),
    "sphbuf_use_graph": (ctypes.c_int, [vp, ctypes.c_int]),
    "sphbuf_sync": (ctypes.c_int, [vp]),
    "sphbuf_count": (ctypes.c_int, [vp, P(c_u64)]),
    "sphbuf_grid_info": (ctypes.c_int, [vp, vp, P(c_dbl), P(c_u64)]),
    "sphbuf_read_particles": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp, c_u64, P(c_u64)]),
    "sphbuf_read_positions": (ctypes.c_int, [vp, vp, c_u64, P(c_u64)]),
    "sphbuf_read_cell_start": (ctypes.c_int, [vp, vp, c_u64]),
    "sphbuf_read_counters": (ctypes.c_int, [vp, ctypes.c_int, P(c_u64), P(c_u64), P(c_dbl), P(c_dbl), P(c_dbl)]),
    "sphbuf_read_global": (ctypes.c_int, [vp, P(c_u64), P(c_u64), P(c_u32)]),
    "sphbuf_last_decisions": (ctypes.c_int, [vp, vp, vp, vp, P(c_u64), vp, vp, P(c_u64), c_u64]),
    "sphbuf_enable_phase_timing": (ctypes.c_int, [vp, ctypes.c_int]),
    "sphbuf_read_phase_times": (ctypes.c_int, [vp, vp, P(c_u64)]),
    "sphbuf_candidate_count": (ctypes.c_int, [vp, ctypes.c_int, P(c_u64), P(c_u64)]),
    "sphbuf_read_launch_count": (ctypes.c_int, [vp, P(c_u64)]),
    "sphbuf_batch_create": (ctypes.c_int, [vp, ctypes.c_int, vp, P(vp)]),
    "sphbuf_batch_step": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_uint]),
    "sphbuf_batch_use_graph": (ctypes.c_int, [vp, ctypes.c_int]),
    "sphbuf_batch_autotune": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_uint, P(ctypes.c_int), vp]),
    "sphbuf_batch_set_grid": (ctypes.c_int, [vp, ctypes.c_int]),
    "sphbuf_batch_get_config": (ctypes.c_int, [vp, vp]),
    "sphbuf_batch_set_config": (ctypes.c_int, [vp, vp]),
    "sphbuf_batch_set_persistent": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_longlong]),
    "sphbuf_set_list_reuse": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_int]),
    "sphbuf_read_list_builds": (ctypes.c_int, [vp, P(ctypes.c_uint64)]),
    "sphbuf_read_boundary_flags": (ctypes.c_int, [vp, vp, c_u64, P(c_u64)]),
    "sphbuf_write_particles_async": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp, ctypes.c_uint64, ctypes.c_uint32]),
    "sphbuf_read_particles_async": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp, ctypes.c_uint64, P(ctypes.c_uint64)]),
    "sphbuf_io_wait": (ctypes.c_int, [vp]),
    "sphbuf_batch_sync": (ctypes.c_int, [vp]),
    "sphbuf_batch_destroy": (ctypes.c_int, [vp]),
    "sphbuf_cell_list_build": (ctypes.c_int, [vp, vp, vp, c_u64, c_u64, vp, vp, vp]),
    "sphbuf_cell_list_build_noalloc": (ctypes.c_int, [vp, vp, vp, c_u64, c_u64, vp, vp, vp]),
}

PHASE_PHYSICS = 1
PHASE_KINEMATIC = 2
PHASE_BUFFER = 4
PHASE_FULL_CHECK = 8
PHASE_BUFFER_KERNEL = 16

# sphbuf_kernel (the configurable batched kernels) and sphbuf_batch_config's layout
KERNELS = ["neighbours", "density", "force", "drift", "viscous", "acoustic", "dual_finish", "buffer", "buffer_full",
           "hist", "keys", "scatter"]
STEP_DEFAULT = PHASE_PHYSICS | PHASE_BUFFER

_lib = None


def load(path: str = LIB_PATH):
    """Loads libsphbuf.so; raises if it has not been built (there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libsphbuf.so is not built (%s); run `python -m paper_2406_16786_gb300.build`" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
