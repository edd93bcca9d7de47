"""GB300 colour-gradient lattice Boltzmann with nonorthogonal central moments
(arXiv:1804.08923): Python binding of the C ABI in ``include/lbcm.h``.

The binding only marshals arguments: every step of the method runs in the CUDA kernels
of ``liblbcm.so``.  PyTorch supplies device memory (``lb_create_with_buffers``) and the
CUDA stream.  There is no CPU fallback: without the compiled library or a GPU, creating
a lattice raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _abi
from ._abi import (BC_CONVECTIVE, BC_FREESLIP, BC_INLET, BC_PERIODIC, FIELD_NAMES, INIT_DROPLET, INIT_FIELDS,
                   INIT_JET, INIT_UNIFORM, STORE_FP16, STORE_FP16_FIT, STORE_FP32, LBError, library, make_grid,
                   make_params)

__all__ = ["Lattice", "LBError", "library", "make_grid", "make_params", "BC_PERIODIC", "BC_FREESLIP",
           "BC_INLET", "BC_CONVECTIVE", "STORE_FP32", "STORE_FP16", "STORE_FP16_FIT", "FIELD_NAMES", "GRAD_NAMES",
           "OBJECTIVES"]

# order of the gradient entries lb_adjoint returns after J
GRAD_NAMES = ("u_in", "sigma", "nu_r", "nu_b") + tuple(f"{ab}{m}" for m in range(1, 9) for ab in "ab")
OBJECTIVES = {"area": 0, "penetration": 1}


def _torch():
    import torch
    return torch


class Lattice:
    """One D3Q27 two-colour lattice resident on a CUDA device.

    grid: (nx, ny, nz); bc: (bc_zlo, bc_zhi) or (bc_zlo, bc_zhi, bc_x, bc_y) with x and y
    PERIODIC or FREESLIP side walls; params: dict of lb_params fields.
    Buffers are torch uint8 tensors owned by this object (PyTorch's caching allocator);
    the library works on them through lb_create_with_buffers.
    """

    def __init__(self, grid, params: dict, bc=(BC_PERIODIC, BC_PERIODIC), device=None, stream=None):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("paper_1804_08923_gb300 needs a CUDA device; no CPU fallback exists")
        self.lib = library()
        self.device = torch.device(device if device is not None else "cuda")
        self.nx, self.ny, self.nz = (int(v) for v in grid)
        self.shape = (self.nz, self.ny, self.nx)
        self.nodes = self.nx * self.ny * self.nz
        self._g = make_grid(self.nx, self.ny, self.nz, *bc)
        self.params = dict(params)
        self._p = make_params(params)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            sizes = (C.c_size_t * _abi.MAX_BUFFERS)()
            n = C.c_int32()
            _abi.check(self.lib.lb_buffer_sizes(C.byref(self._g), C.byref(self._p), sizes, C.byref(n)))
            self._bufs = [torch.empty(int(sizes[j]), dtype=torch.uint8, device=self.device) for j in range(n.value)]
            ptrs = (C.c_void_p * n.value)(*[b.data_ptr() for b in self._bufs])
            szs = (C.c_size_t * n.value)(*[int(sizes[j]) for j in range(n.value)])
            ctx = C.c_void_p()
            _abi.check(self.lib.lb_create_with_buffers(C.byref(self._g), C.byref(self._p),
                                                       C.c_void_p(self.stream.cuda_stream), ptrs, szs, n,
                                                       C.byref(ctx)))
            self._ctx = ctx

    # ------------------------------------------------------------------ lifecycle
    def close(self):
        if getattr(self, "_ctx", None):
            self.lib.lb_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------ init
    def init_uniform(self, rho_r, rho_b, u=(0.0, 0.0, 0.0)):
        args = (C.c_double * 5)(rho_r, rho_b, *u)
        _abi.check(self.lib.lb_init(self._ctx, INIT_UNIFORM, args, 5, None, None, None, 0))

    def init_droplet(self, R, W=4.0):
        args = (C.c_double * 2)(R, W)
        _abi.check(self.lib.lb_init(self._ctx, INIT_DROPLET, args, 2, None, None, None, 0))

    def init_jet(self):
        _abi.check(self.lib.lb_init(self._ctx, INIT_JET, None, 0, None, None, None, 0))

    def init_fields(self, rho_r, rho_b, u):
        """Fields as numpy arrays (host) or CUDA float32 tensors (device); shapes
        (nz, ny, nx) and (3, nz, ny, nx)."""
        torch = _torch()
        if isinstance(rho_r, torch.Tensor) and rho_r.is_cuda:
            ts = [t.to(self.device, torch.float32).contiguous() for t in (rho_r, rho_b, u)]
            ps = [C.cast(C.c_void_p(t.data_ptr()), C.POINTER(C.c_float)) for t in ts]
            _abi.check(self.lib.lb_init(self._ctx, INIT_FIELDS, None, 0, ps[0], ps[1], ps[2], 1))
            self.stream.synchronize()
        else:
            arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (rho_r, rho_b, u)]
            assert arrs[0].size == self.nodes and arrs[1].size == self.nodes and arrs[2].size == 3 * self.nodes
            ps = [a.ctypes.data_as(C.POINTER(C.c_float)) for a in arrs]
            _abi.check(self.lib.lb_init(self._ctx, INIT_FIELDS, None, 0, ps[0], ps[1], ps[2], 0))

    # ------------------------------------------------------------------ stepping
    def step(self, n=1):
        _abi.check(self.lib.lb_step(self._ctx, C.c_int64(n)))

    def step_gather(self):
        """First half of a step (boundary planes, gather pass); see lb_step_gather."""
        _abi.check(self.lib.lb_step_gather(self._ctx))

    def step_collide(self):
        """Second half of a step (collision); see lb_step_collide."""
        _abi.check(self.lib.lb_step_collide(self._ctx))

    def halo_bytes(self, kind: int) -> int:
        n = C.c_size_t()
        _abi.check(self.lib.lb_halo_bytes(self._ctx, int(kind), C.byref(n)))
        return int(n.value)

    def halo_pack(self, kind: int, z: int, buf):
        """Copies halo plane z into buf: a CUDA uint8 tensor (device) or a numpy uint8 array
        (host) of halo_bytes(kind) bytes."""
        dev, ptr = self._buffer(buf, self.halo_bytes(kind))
        _abi.check(self.lib.lb_halo_pack(self._ctx, int(kind), int(z), ptr, dev))

    def halo_unpack(self, kind: int, z: int, buf):
        dev, ptr = self._buffer(buf, self.halo_bytes(kind))
        _abi.check(self.lib.lb_halo_unpack(self._ctx, int(kind), int(z), ptr, dev))

    def _buffer(self, buf, nbytes):
        torch = _torch()
        if isinstance(buf, torch.Tensor):
            assert buf.is_contiguous() and buf.numel() * buf.element_size() >= nbytes
            return (1 if buf.is_cuda else 0), C.c_void_p(buf.data_ptr())
        assert buf.flags.c_contiguous and buf.nbytes >= nbytes
        return 0, C.c_void_p(buf.ctypes.data)

    def mass_planes(self, z_begin: int, z_end: int):
        out = (C.c_double * 2)()
        _abi.check(self.lib.lb_mass_planes(self._ctx, int(z_begin), int(z_end), out))
        return np.array([out[0], out[1]])

    def selftest_fused_wait(self):
        """Runs the fused step kernel's plane wait against a target nothing reaches (lb_selftest):
        returns (status the host read, milliseconds the wait lasted)."""
        res, ms = C.c_int32(), C.c_double()
        _abi.check(self.lib.lb_selftest(self._ctx, _abi.SELFTEST_FUSED_WAIT, C.byref(res), C.byref(ms)))
        return int(res.value), float(ms.value)

    @property
    def step_count(self) -> int:
        return int(self.lib.lb_step_count(self._ctx))

    # ------------------------------------------------------------------ outputs
    def fields(self, names=FIELD_NAMES, device=True, out=None):
        """Dict of macroscopic fields (float32, shape (nz, ny, nx)) as CUDA tensors
        (device=True) or numpy arrays (device=False); `out` may supply the arrays."""
        torch = _torch()
        mask, outs, keep = 0, (C.POINTER(C.c_float) * len(FIELD_NAMES))(), {}
        for j, nm in enumerate(FIELD_NAMES):
            if nm not in names:
                continue
            mask |= 1 << j
            if device:
                t = out[nm] if out else torch.empty(self.shape, dtype=torch.float32, device=self.device)
                assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == self.nodes
                outs[j] = C.cast(C.c_void_p(t.data_ptr()), C.POINTER(C.c_float))
            else:
                t = out[nm] if out else np.empty(self.shape, dtype=np.float32)
                assert t.dtype == np.float32 and t.flags.c_contiguous and t.size == self.nodes
                outs[j] = t.ctypes.data_as(C.POINTER(C.c_float))
            keep[nm] = t
        _abi.check(self.lib.lb_fields(self._ctx, C.c_uint32(mask), outs, 1 if device else 0))
        return keep

    def populations(self, device=True):
        """Current populations, shape (2, 27, nz, ny, nx), float32."""
        torch = _torch()
        shp = (2, 27) + self.shape
        if device:
            t = torch.empty(shp, dtype=torch.float32, device=self.device)
            _abi.check(self.lib.lb_populations(self._ctx, C.cast(C.c_void_p(t.data_ptr()), C.POINTER(C.c_float)), 1))
            return t
        a = np.empty(shp, dtype=np.float32)
        _abi.check(self.lib.lb_populations(self._ctx, a.ctypes.data_as(C.POINTER(C.c_float)), 0))
        return a

    def history(self):
        """Outflow history plane, shape (2, 27, ny, nx), float32 numpy."""
        a = np.empty((2, 27, self.ny, self.nx), dtype=np.float32)
        _abi.check(self.lib.lb_history(self._ctx, a.ctypes.data_as(C.POINTER(C.c_float)), 0))
        return a

    def mass(self):
        out = (C.c_double * 2)()
        _abi.check(self.lib.lb_mass(self._ctx, out))
        return np.array([out[0], out[1]])

    def save(self) -> bytes:
        n = C.c_size_t()
        _abi.check(self.lib.lb_save(self._ctx, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _abi.check(self.lib.lb_save(self._ctx, buf, C.byref(n)))
        return buf.raw[: n.value]

    # ------------------------------------------------------------------ profiling
    def profile_enable(self, capacity: int):
        _abi.check(self.lib.lb_profile_enable(self._ctx, int(capacity)))

    def profile_read(self) -> dict:
        """{kernel name: (total device ms, launches)} since profile_enable / the last read."""
        nk = len(_abi.KERNEL_NAMES)
        ms = (C.c_double * nk)()
        cnt = (C.c_int64 * nk)()
        _abi.check(self.lib.lb_profile_read(self._ctx, ms, cnt, nk))
        return {_abi.KERNEL_NAMES[k]: (ms[k], int(cnt[k])) for k in range(nk)}

    @property
    def kernel_launches(self) -> int:
        return int(self.lib.lb_kernel_launches(self._ctx))

    # ------------------------------------------------------------------ parameters, adjoint
    def set_params(self, **changes):
        """Changes lb_params fields of the context (grid, storage and state are kept)."""
        params = dict(self.params)
        params.update(changes)
        p = make_params(params)
        _abi.check(self.lib.lb_set_params(self._ctx, C.byref(p)))
        self.params, self._p = params, p

    def adjoint(self, T: int, objective: str = "area", args=(1e-3,), checkpoint: int = 0):
        """Runs T steps and returns (J, grad): J the objective of the state T steps ahead and
        grad (float64, 20) its gradient w.r.t. GRAD_NAMES.  checkpoint = segment length
        (0: ceil(sqrt(T)))."""
        a = list(args)[:2] + [0.0] * (2 - len(list(args)[:2]))
        obj_args = (C.c_double * 4)(a[0], a[1], float(checkpoint), 0.0)
        out = (C.c_double * _abi.ADJ_NOUT)()
        _abi.check(self.lib.lb_adjoint(self._ctx, C.c_int32(OBJECTIVES[objective]), C.c_int64(int(T)), obj_args,
                                       out, C.c_int32(_abi.ADJ_NOUT)))
        return float(out[0]), np.array(out[1:], dtype=np.float64)

    def adjoint_state(self, device=False):
        """dJ/dS of the state the last adjoint started from, shape (2, 27, nz, ny, nx), float32."""
        torch = _torch()
        shp = (2, 27) + self.shape
        if device:
            t = torch.empty(shp, dtype=torch.float32, device=self.device)
            _abi.check(self.lib.lb_adjoint_state(self._ctx, C.cast(C.c_void_p(t.data_ptr()), C.POINTER(C.c_float)), 1))
            return t
        a = np.empty(shp, dtype=np.float32)
        _abi.check(self.lib.lb_adjoint_state(self._ctx, a.ctypes.data_as(C.POINTER(C.c_float)), 0))
        return a

    # ------------------------------------------------------------------ fragments
    def fragments(self, connectivity: int = 6, exclude_inlet: bool = True) -> dict:
        """Fragments of the current state (lb_fragments): roots (smallest node index), volumes,
        equivalent diameters (6V/pi)^(1/3), the excluded column volume and the mass-median
        diameter, all computed by the library."""
        st = _abi.FragmentStats()
        _abi.check(self.lib.lb_fragments(self._ctx, int(connectivity), int(bool(exclude_inlet)), None, None, None, 0,
                                         C.byref(st)))
        n = int(st.n_fragments)
        roots, vols, diam = np.zeros(n, np.int64), np.zeros(n, np.int64), np.zeros(n, np.float64)
        if n:
            _abi.check(self.lib.lb_fragments(self._ctx, int(connectivity), int(bool(exclude_inlet)),
                                             roots.ctypes.data_as(C.POINTER(C.c_int64)),
                                             vols.ctypes.data_as(C.POINTER(C.c_int64)),
                                             diam.ctypes.data_as(C.POINTER(C.c_double)), n, C.byref(st)))
        return {"roots": roots, "volumes": vols, "diameters": diam,
                "mass_median_diameter": float(st.mass_median_diameter), "column_volume": int(st.column_volume),
                "total_volume": int(st.total_volume)}

    def load(self, blob: bytes):
        _abi.check(self.lib.lb_load(self._ctx, blob, C.c_size_t(len(blob))))
