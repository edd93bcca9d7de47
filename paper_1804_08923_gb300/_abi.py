"""ctypes declarations mirroring ``include/lbcm.h`` (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbcm.so")
MAX_BUFFERS = 8

BC_PERIODIC, BC_FREESLIP, BC_INLET, BC_CONVECTIVE = 0, 1, 2, 3
INIT_UNIFORM, INIT_DROPLET, INIT_JET, INIT_FIELDS = 0, 1, 2, 3
STORE_FP32, STORE_FP16, STORE_FP16_FIT = 0, 1, 2
FIELD_NAMES = ("rho_r", "rho_b", "phi", "ux", "uy", "uz", "p")
STATUS = {0: "LB_OK", 1: "LB_EINVAL", 2: "LB_ENOMEM", 3: "LB_ECUDA", 4: "LB_EUNSTABLE", 5: "LB_ETIMEOUT",
          6: "LB_ESTATE", 7: "LB_ENOTIMPL"}

# every entry point declared in include/lbcm.h
EXPORTS = ("lb_params_default", "lb_buffer_sizes", "lb_create", "lb_create_with_buffers", "lb_init", "lb_step",
           "lb_step_count", "lb_fields", "lb_populations", "lb_history", "lb_mass", "lb_mass_noalloc", "lb_save", "lb_load",
           "lb_profile_enable", "lb_profile_read", "lb_kernel_launches", "lb_set_params", "lb_adjoint",
           "lb_adjoint_state", "lb_fragments", "lb_step_gather", "lb_step_collide", "lb_halo_bytes",
           "lb_halo_pack", "lb_halo_unpack", "lb_mass_planes", "lb_selftest", "lb_last_error", "lb_destroy")
SELFTEST_FUSED_WAIT = 1
HALO_POPULATIONS, HALO_PHASE = 0, 1
ADJ_NOUT = 21  # LB_ADJ_NOUT: J and 20 parameter gradients


class FragmentStats(C.Structure):
    _fields_ = [("n_fragments", C.c_int64), ("column_volume", C.c_int64), ("total_volume", C.c_int64),
                ("mass_median_diameter", C.c_double)]
KERNEL_NAMES = ("boundary_kernel", "moment_kernel", "collide_kernel", "step_kernel")


class LBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("bc_zlo", C.c_int32), ("bc_zhi", C.c_int32), ("bc_x", C.c_int32), ("bc_y", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("rho_r0", C.c_double), ("rho_b0", C.c_double), ("nu_r", C.c_double), ("nu_b", C.c_double),
                ("sigma", C.c_double), ("beta", C.c_double), ("g", C.c_double * 3),
                ("s0", C.c_double), ("s1", C.c_double), ("s2b", C.c_double), ("s3", C.c_double),
                ("s4", C.c_double), ("s5", C.c_double), ("s6", C.c_double),
                ("u_in", C.c_double), ("d_in", C.c_double), ("noise_amp", C.c_double),
                ("seed", C.c_uint64), ("eps_grad", C.c_double), ("storage", C.c_int32),
                ("check_every", C.c_int32), ("fourier", C.c_double * 16), ("step_kernel", C.c_int32),
                ("alpha_mix", C.c_int32)]


_lock = threading.Lock()
_lib = None


def library(path: str = LIB_PATH):
    """Load liblbcm.so and declare its signatures.  Raises if it was not built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
        L = C.CDLL(path)
        vp, gp, pp = C.c_void_p, C.POINTER(Grid), C.POINTER(Params)
        fp, dp = C.POINTER(C.c_float), C.POINTER(C.c_double)
        L.lb_params_default.argtypes = [pp]
        L.lb_params_default.restype = None
        L.lb_buffer_sizes.argtypes = [gp, pp, C.POINTER(C.c_size_t), C.POINTER(C.c_int32)]
        L.lb_create.argtypes = [gp, pp, vp, C.POINTER(vp)]
        L.lb_create_with_buffers.argtypes = [gp, pp, vp, C.POINTER(vp), C.POINTER(C.c_size_t), C.c_int32,
                                             C.POINTER(vp)]
        L.lb_init.argtypes = [vp, C.c_int32, dp, C.c_int32, fp, fp, fp, C.c_int32]
        L.lb_step.argtypes = [vp, C.c_int64]
        L.lb_step_count.argtypes = [vp]
        L.lb_step_count.restype = C.c_int64
        L.lb_fields.argtypes = [vp, C.c_uint32, C.POINTER(fp), C.c_int32]
        L.lb_populations.argtypes = [vp, fp, C.c_int32]
        L.lb_history.argtypes = [vp, fp, C.c_int32]
        L.lb_mass.argtypes = [vp, dp]
        L.lb_mass_noalloc.argtypes = [vp, C.c_int64, vp, vp]
        L.lb_save.argtypes = [vp, vp, C.POINTER(C.c_size_t)]
        L.lb_load.argtypes = [vp, C.c_char_p, C.c_size_t]
        L.lb_profile_enable.argtypes = [vp, C.c_int32]
        L.lb_profile_read.argtypes = [vp, dp, C.POINTER(C.c_int64), C.c_int32]
        L.lb_kernel_launches.argtypes = [vp]
        L.lb_kernel_launches.restype = C.c_int64
        L.lb_set_params.argtypes = [vp, pp]
        L.lb_adjoint.argtypes = [vp, C.c_int32, C.c_int64, dp, dp, C.c_int32]
        L.lb_adjoint_state.argtypes = [vp, fp, C.c_int32]
        L.lb_fragments.argtypes = [vp, C.c_int32, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64), dp,
                                   C.c_int64, C.POINTER(FragmentStats)]
        L.lb_step_gather.argtypes = [vp]
        L.lb_step_collide.argtypes = [vp]
        L.lb_halo_bytes.argtypes = [vp, C.c_int32, C.POINTER(C.c_size_t)]
        L.lb_halo_pack.argtypes = [vp, C.c_int32, C.c_int32, vp, C.c_int32]
        L.lb_halo_unpack.argtypes = [vp, C.c_int32, C.c_int32, vp, C.c_int32]
        L.lb_mass_planes.argtypes = [vp, C.c_int32, C.c_int32, dp]
        L.lb_last_error.argtypes = []
        L.lb_last_error.restype = C.c_char_p
        L.lb_destroy.argtypes = [vp]
        L.lb_destroy.restype = None
        for name in EXPORTS:
            fn = getattr(L, name)
            if fn.restype is C.c_int:  # default restype: status codes are C ints
                fn.restype = C.c_int
        _lib = L
        return _lib


def check(status: int):
    if status != 0:
        msg = _lib.lb_last_error().decode() if _lib is not None else ""
        raise LBError(status, msg)


def make_grid(nx, ny, nz, bc_zlo=BC_PERIODIC, bc_zhi=BC_PERIODIC, bc_x=BC_PERIODIC, bc_y=BC_PERIODIC) -> Grid:
    """Extents and boundaries: z ends, x and y sides (PERIODIC or FREESLIP walls)."""
    return Grid(nx, ny, nz, bc_zlo, bc_zhi, bc_x, bc_y)


def make_params(d: dict) -> Params:
    """lb_params from a dict; missing entries take lb_params_default's values."""
    p = Params()
    library().lb_params_default(C.byref(p))
    for k, v in d.items():
        if k == "g":
            p.g[0], p.g[1], p.g[2] = v
        elif k == "fourier":
            vals = list(v) + [0.0] * 16
            for m in range(16):
                p.fourier[m] = float(vals[m])
        elif k in ("seed", "storage", "check_every", "alpha_mix", "step_kernel"):
            setattr(p, k, int(v))
        elif k in dict(Params._fields_):
            setattr(p, k, float(v))
        else:
            raise KeyError(f"unknown lattice parameter {k!r}")
    return p
