"""FP64 CPU oracle for the colour-gradient central-moment LBM step (arXiv:1804.08923).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of the
benchmark are the only callers.  The CUDA product path never imports this package and
this package never imports the product; they share only the seeded input generators
in ``workloads``.

The arithmetic lives in ``lbcm_oracle.c`` (plain C, FP64, dense 27x27 matrices, every
step in the paper's order).  This module compiles it with gcc and wraps it with ctypes.

Parity unpinned: the inlet ghost placement (reading R7 in the C file) is fixed by no closed
form or printed value; only the uniform-state invariants of the boundary tests constrain it.
The convective outflow (R8) is pinned by the advection equation it discretises (harmonic and
step responses, tests/test_oracle_outflow.py); its clamp of lambda to [0, 1] under backflow is
a reading the paper is silent on.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbcm_oracle.c")
_LIB = os.path.join(_HERE, "liblbcm_oracle.so")
_lock = threading.Lock()
_lib = None

BC_PERIODIC, BC_FREESLIP, BC_INLET, BC_CONVECTIVE = 0, 1, 2, 3


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("bc_zlo", C.c_int32), ("bc_zhi", C.c_int32), ("bc_x", C.c_int32), ("bc_y", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("rho_r0", C.c_double), ("rho_b0", C.c_double),
                ("nu_r", C.c_double), ("nu_b", C.c_double),
                ("sigma", C.c_double), ("beta", C.c_double),
                ("g", C.c_double * 3),
                ("s0", C.c_double), ("s1", C.c_double), ("s2b", C.c_double),
                ("s3", C.c_double), ("s4", C.c_double), ("s5", C.c_double), ("s6", C.c_double),
                ("u_in", C.c_double), ("d_in", C.c_double), ("noise_amp", C.c_double),
                ("seed", C.c_uint64), ("eps_grad", C.c_double), ("alpha_b", C.c_double),
                ("fourier", C.c_double * 16), ("alpha_mix", C.c_int32)]


_Z = C.c_double * 2  # double _Complex: (real, imaginary)


class CSParams(C.Structure):
    """orc_params of the complex-step build: every real field complex."""
    _fields_ = [(name, (_Z * ct._length_) if hasattr(ct, "_length_") else _Z)
                if ct not in (C.c_uint64, C.c_int32) else (name, ct) for name, ct in Params._fields_]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP over nodes)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            flags = ["-O2", "-std=c11", "-fPIC", "-fopenmp", "-ffp-contract=off", "-fno-fast-math"]
            objs = [tmp + ".real.o", tmp + ".cs.o"]  # FP64, and the complex-step tangent build
            subprocess.run(["gcc", "-c", _SRC, "-o", objs[0]] + flags, check=True)
            subprocess.run(["gcc", "-c", _SRC, "-o", objs[1], "-DORC_COMPLEX_STEP"] + flags, check=True)
            subprocess.run(["gcc", "-shared", "-fopenmp", "-o", tmp] + objs + ["-lm"], check=True)
            for o in objs:
                os.remove(o)
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        L.orc_build_T.argtypes = [dp, dp]
        L.orc_T_inverse.argtypes = [dp, dp]
        L.orc_T_inverse.restype = C.c_int
        L.orc_equilibrium.argtypes = [C.c_double, dp, C.c_double, C.c_double, dp, dp]
        L.orc_forcing_prime.argtypes = [dp, dp, dp]
        L.orc_collide.argtypes = [dp, dp, dp, dp, dp, dp]
        L.orc_collide.restype = C.c_int
        L.orc_perturbation.argtypes = [C.c_double, dp, C.c_double, dp]
        L.orc_recolor.argtypes = [dp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                  dp, C.c_double, dp, dp]
        L.orc_splitmix64.argtypes = [C.c_uint64]
        L.orc_splitmix64.restype = C.c_uint64
        L.orc_inlet_xi.argtypes = [C.c_uint64, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int32]
        L.orc_inlet_xi.restype = C.c_double
        gp, pp = C.POINTER(Grid), C.POINTER(Params)
        L.orc_stream.argtypes = [gp, pp, dp, dp, C.c_int64, dp, dp]
        L.orc_step.argtypes = [gp, pp, dp, dp, C.c_int64, dp, dp, C.POINTER(C.c_uint8)]
        L.orc_step.restype = C.c_int
        L.orc_init_fields.argtypes = [gp, pp, dp, dp, dp, dp, dp]
        L.orc_droplet_fields.argtypes = [gp, pp, C.c_double, C.c_double, dp, dp]
        L.orc_fields.argtypes = [gp, pp, dp, dp, dp, dp, dp, dp]
        L.orc_mass.argtypes = [gp, dp, dp]
        L.orc_objective.argtypes = [gp, pp, dp, C.c_int, dp]
        L.orc_objective.restype = C.c_double
        L.orc_fragments.argtypes = [gp, pp, dp, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_uint8), C.c_int64]
        L.orc_fragments.restype = C.c_int64
        cpp = C.POINTER(CSParams)
        L.orc_cs_step.argtypes = [gp, cpp, dp, dp, C.c_int64, dp, dp, C.POINTER(C.c_uint8)]
        L.orc_cs_step.restype = C.c_int
        L.orc_cs_objective_parts.argtypes = [gp, cpp, dp, C.c_int, dp, dp]
        L.orc_cs_objective_parts.restype = None
        L.orc_velocity_set.argtypes = [C.POINTER(C.c_int32)]
        L.orc_weights.argtypes = [dp]
        L.orc_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _vec(x, n=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        assert a.size == n
    return a


# ----------------------------------------------------------------- single-node pieces
def velocity_set() -> np.ndarray:
    c = np.zeros((27, 3), dtype=np.int32)
    lib().orc_velocity_set(c.ctypes.data_as(C.POINTER(C.c_int32)))
    return c


def weights() -> np.ndarray:
    w = np.zeros(27)
    lib().orc_weights(_p(w))
    return w


def build_T(u) -> np.ndarray:
    T = np.zeros((27, 27))
    lib().orc_build_T(_p(_vec(u, 3)), _p(T))
    return T


def T_inverse(u) -> np.ndarray:
    Ti = np.zeros((27, 27))
    assert lib().orc_T_inverse(_p(_vec(u, 3)), _p(Ti)) == 0
    return Ti


def equilibrium(rho, u, alpha, nu, grad_rho) -> np.ndarray:
    fe = np.zeros(27)
    lib().orc_equilibrium(float(rho), _p(_vec(u, 3)), float(alpha), float(nu), _p(_vec(grad_rho, 3)), _p(fe))
    return fe


def forcing_prime(u, F) -> np.ndarray:
    Fp = np.zeros(27)
    lib().orc_forcing_prime(_p(_vec(u, 3)), _p(_vec(F, 3)), _p(Fp))
    return Fp


def collide(f, fe, Fp, u, K) -> np.ndarray:
    out = np.zeros(27)
    rc = lib().orc_collide(_p(_vec(f, 27)), _p(_vec(fe, 27)), _p(_vec(Fp, 27)), _p(_vec(u, 3)),
                           _p(_vec(K, 27)), _p(out))
    assert rc == 0
    return out


def perturbation(A, grad_phi, eps) -> np.ndarray:
    out = np.zeros(27)
    lib().orc_perturbation(float(A), _p(_vec(grad_phi, 3)), float(eps), _p(out))
    return out


def recolor(fstar, rho_r, rho_b, alpha_bar, nu_bar, beta, grad_phi, eps):
    fr, fb = np.zeros(27), np.zeros(27)
    lib().orc_recolor(_p(_vec(fstar, 27)), float(rho_r), float(rho_b), float(alpha_bar), float(nu_bar),
                      float(beta), _p(_vec(grad_phi, 3)), float(eps), _p(fr), _p(fb))
    return fr, fb


def splitmix64(state: int) -> int:
    return int(lib().orc_splitmix64(C.c_uint64(state)))


def inlet_xi(seed, step, x, y, nx, ny) -> float:
    return float(lib().orc_inlet_xi(seed, step, x, y, nx, ny))


def num_threads() -> int:
    return int(lib().orc_num_threads())


# ----------------------------------------------------------------------- whole lattice
def make_grid(nx, ny, nz, bc_zlo=BC_PERIODIC, bc_zhi=BC_PERIODIC, bc_x=BC_PERIODIC, bc_y=BC_PERIODIC) -> Grid:
    """Lattice extents and boundaries: z ends (PERIODIC at both or neither), x and y sides
    PERIODIC or FREESLIP walls (reading R14)."""
    return Grid(nx, ny, nz, bc_zlo, bc_zhi, bc_x, bc_y)


def make_params(d: dict) -> Params:
    """Oracle parameter block from a plain dict of lattice parameters (see ``workloads``)."""
    p = Params()
    p.rho_r0, p.rho_b0 = d["rho_r0"], d["rho_b0"]
    p.nu_r, p.nu_b = d["nu_r"], d["nu_b"]
    p.sigma, p.beta = d["sigma"], d.get("beta", 0.7)
    g = d.get("g", (0.0, 0.0, 0.0))
    p.g[0], p.g[1], p.g[2] = g
    p.s0, p.s1 = d.get("s0", 0.0), d.get("s1", 0.0)
    p.s2b, p.s3, p.s4, p.s5, p.s6 = (d.get(k, 1.0) for k in ("s2b", "s3", "s4", "s5", "s6"))
    p.u_in, p.d_in, p.noise_amp = d.get("u_in", 0.0), d.get("d_in", 0.0), d.get("noise_amp", 0.0)
    p.seed = d.get("seed", 0)
    p.eps_grad = d.get("eps_grad", 1e-6)
    p.alpha_b = d.get("alpha_b", 8.0 / 27.0)
    fr = list(d.get("fourier", ())) + [0.0] * 16
    for m in range(16):
        p.fourier[m] = fr[m]
    p.alpha_mix = int(d.get("alpha_mix", 0))
    return p


class Lattice:
    """A whole FP64 lattice advanced by the oracle; populations S[k][i][z][y][x]."""

    def __init__(self, grid: Grid, params: Params):
        self.g, self.p = grid, params
        self.shape = (grid.nz, grid.ny, grid.nx)
        self.nn = grid.nx * grid.ny * grid.nz
        self.S = np.zeros((2, 27) + self.shape)
        self.hist = np.zeros((2, 27, grid.ny, grid.nx))
        self.step_count = 0

    def init_fields(self, rho_r, rho_b, u):
        rr = np.ascontiguousarray(rho_r, dtype=np.float64).reshape(self.shape)
        rb = np.ascontiguousarray(rho_b, dtype=np.float64).reshape(self.shape)
        uu = np.ascontiguousarray(u, dtype=np.float64).reshape((3,) + self.shape)
        lib().orc_init_fields(C.byref(self.g), C.byref(self.p), _p(rr), _p(rb), _p(uu), _p(self.S), _p(self.hist))
        self.step_count = 0

    def init_droplet(self, R, W=4.0):
        rr, rb = np.zeros(self.shape), np.zeros(self.shape)
        lib().orc_droplet_fields(C.byref(self.g), C.byref(self.p), float(R), float(W), _p(rr), _p(rb))
        self.init_fields(rr, rb, np.zeros((3,) + self.shape))

    def init_jet(self):
        z = np.zeros(self.shape)
        self.init_fields(z, np.full(self.shape, self.p.rho_b0), np.zeros((3,) + self.shape))

    def set_state(self, S, hist=None, step=None):
        self.S = np.ascontiguousarray(S, dtype=np.float64).reshape((2, 27) + self.shape).copy()
        if hist is not None:
            self.hist = np.ascontiguousarray(hist, dtype=np.float64).reshape(self.hist.shape).copy()
        if step is not None:
            self.step_count = int(step)

    def stream(self):
        f = np.zeros_like(self.S)
        h = self.hist.copy()
        lib().orc_stream(C.byref(self.g), C.byref(self.p), _p(self.S), _p(self.hist), self.step_count, _p(f), _p(h))
        return f, h

    def step(self, n=1, mask=None):
        mp = None
        if mask is not None:
            m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(self.shape)
            mp = m.ctypes.data_as(C.POINTER(C.c_uint8))
        for _ in range(n):
            out = np.empty_like(self.S)
            h = self.hist.copy()
            rc = lib().orc_step(C.byref(self.g), C.byref(self.p), _p(self.S), _p(self.hist), self.step_count,
                                _p(out), _p(h), mp)
            if rc != 0:
                raise RuntimeError(f"oracle step failed ({rc})")
            self.S, self.hist = out, h
            self.step_count += 1

    def fields(self):
        sh = self.shape
        rr, rb, ph, pr = (np.zeros(sh) for _ in range(4))
        u = np.zeros((3,) + sh)
        lib().orc_fields(C.byref(self.g), C.byref(self.p), _p(self.S), _p(rr), _p(rb), _p(u), _p(ph), _p(pr))
        return {"rho_r": rr, "rho_b": rb, "u": u, "phi": ph, "p": pr}

    def mass(self):
        out = np.zeros(2)
        lib().orc_mass(C.byref(self.g), _p(self.S), _p(out))
        return out

    def fragments(self, connectivity: int = 6, exclude_inlet: bool = True) -> dict:
        """Fragments of the current state (reading R13): roots (smallest node index), volumes,
        equivalent diameters d = (6V/pi)^(1/3), the excluded column volume and the mass-median
        diameter of the kept fragments."""
        n = lib().orc_fragments(C.byref(self.g), C.byref(self.p), _p(self.S), connectivity, None, None, None, 0)
        if n < 0:
            raise MemoryError("oracle fragments")
        roots, vols, touch = np.zeros(n, np.int64), np.zeros(n, np.int64), np.zeros(n, np.uint8)
        if n:
            lib().orc_fragments(C.byref(self.g), C.byref(self.p), _p(self.S), connectivity,
                                roots.ctypes.data_as(C.POINTER(C.c_int64)), vols.ctypes.data_as(C.POINTER(C.c_int64)),
                                touch.ctypes.data_as(C.POINTER(C.c_uint8)), n)
        column = np.zeros(n, bool)
        if exclude_inlet and self.g.bc_zlo == BC_INLET:
            column = touch.astype(bool)
        keep = ~column
        return fragment_stats(roots[keep], vols[keep], int(vols[column].sum()))

    def objective(self, kind: str, args=(1e-3,)):
        """Adjoint objective of the current state (reading R12): "area" (args = eps) or
        "penetration" (args = delta)."""
        a = np.zeros(4)
        a[: len(args)] = args
        k = {"area": 0, "penetration": 1}[kind]
        return float(lib().orc_objective(C.byref(self.g), C.byref(self.p), _p(self.S), k, _p(a)))


def _cs_params(p: dict, dp: dict, h: float) -> CSParams:
    """Complex parameters p + i h dp (dp: field -> direction, "fourier" a sequence of 16)."""
    base = make_params(p)
    out = CSParams()
    for name, ct in Params._fields_:
        v = getattr(base, name)
        if ct in (C.c_uint64, C.c_int32):
            setattr(out, name, v)
            continue
        d = dp.get(name, 0.0)
        if hasattr(ct, "_length_"):
            dd = (list(d) if not np.isscalar(d) else [d] * ct._length_) + [0.0] * ct._length_
            arr = getattr(out, name)
            for k in range(ct._length_):
                arr[k][0], arr[k][1] = v[k], h * dd[k]
        else:
            z = getattr(out, name)
            z[0], z[1] = v, h * d
    return out


def tangent_objective(grid: Grid, params: dict, S0, hist0, T: int, kind: str, args, dparams=None, dS=None,
                      h: float = 1e-30, step0: int = 0):
    """Forward-mode tangent of the oracle by complex step: runs T steps from (S0, hist0) with
    parameters params + i h dparams and state S0 + i h dS and returns (J, dJ), dJ the
    directional derivative of the objective (reading R12) along (dparams, dS)."""
    shape = (grid.nz, grid.ny, grid.nx)
    S = np.zeros((2, 27) + shape + (2,))
    S[..., 0] = np.asarray(S0, dtype=np.float64).reshape((2, 27) + shape)
    if dS is not None:
        S[..., 1] = h * np.asarray(dS, dtype=np.float64).reshape((2, 27) + shape)
    H = np.zeros((2, 27, grid.ny, grid.nx, 2))
    H[..., 0] = np.asarray(hist0, dtype=np.float64).reshape(H.shape[:-1])
    cp = _cs_params(params, dparams or {}, h)
    L = lib()
    for t in range(T):
        out = np.empty_like(S)
        Ho = H.copy()
        rc = L.orc_cs_step(C.byref(grid), C.byref(cp), _p(S), _p(H), step0 + t, _p(out), _p(Ho), None)
        if rc != 0:
            raise RuntimeError(f"oracle tangent step failed ({rc})")
        S, H = out, Ho
    a = np.zeros(4)
    a[: len(args)] = args
    z = np.zeros(2)
    L.orc_cs_objective_parts(C.byref(grid), C.byref(cp), _p(S), {"area": 0, "penetration": 1}[kind], _p(a), _p(z))
    return z[0], z[1] / h


def fragment_stats(roots, volumes, column_volume=0) -> dict:
    """Equivalent diameters and the mass-median diameter (reading R13) of a fragment list."""
    roots, volumes = np.asarray(roots, np.int64), np.asarray(volumes, np.int64)
    d = (6.0 * volumes / np.pi) ** (1.0 / 3.0)
    d_m = 0.0
    if volumes.size:
        order = np.argsort(volumes, kind="stable")
        cum = np.cumsum(volumes[order])
        k = int(np.searchsorted(cum, 0.5 * cum[-1], side="left"))
        d_m = float(d[order][k])
    return {"roots": roots, "volumes": volumes, "diameters": d, "mass_median_diameter": d_m,
            "column_volume": int(column_volume), "total_volume": int(volumes.sum())}
