"""FP64 CPU oracle for the two-component Shan-Chen method of arXiv:2112.02574.

TEST INFRASTRUCTURE ONLY.  This package is the slow reference the CUDA library
is checked against; only the test suite, the smoke check and the benchmark's
CPU-baseline leg and reference arm may import it.  It shares no code with the CUDA library and
never imports it.

* ``sc_oracle.c`` -- the lattice Boltzmann step (section 2: Eqs. lbm, omega_i,
  Guo, feq, u, sc_force), the lattice pressure tensor (Eq. sm:pt), the bulk
  pressure (Eq. bulkp) and the radial / planar / axis profiles (section 3,
  Eq. pt_projection; section 4 for the flat interface).
* ``sigma.py`` -- the generalized surface tension sigma[R] (Eq. gen_sigma), its
  notional derivative (Eq. gen_d_sigma) and the surface of tension R_s.
* ``np_step.py`` -- an independent NumPy transcription of one time step, used
  only to cross-check the C code on tiny lattices.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libsc_oracle.so")

D2Q9, D3Q19 = 0, 1
E4, E6 = 0, 1
PSI_N, PSI_EXP = 0, 1
CS2 = 1.0 / 3.0


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP) into oracle/_build/."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("lattice", ctypes.c_int32), ("stencil", ctypes.c_int32), ("psi_self", ctypes.c_int32),
        ("tau", ctypes.c_double * 2), ("G", ctypes.c_double), ("G_self", ctypes.c_double * 2),
    ]


@dataclass
class Params:
    """Model parameters in the paper's convention (Eq. sc_force: force = -G c_s^2 ...)."""
    shape: tuple  # (nx, ny, nz); nz = 1 for D2Q9
    lattice: int = D3Q19
    stencil: int = E4
    psi_self: int = PSI_EXP
    tau: tuple = (1.0, 1.0)
    G: float = 0.0
    G_self: tuple = (0.0, 0.0)

    @property
    def n_sites(self) -> int:
        nx, ny, nz = self.shape
        return nx * ny * nz

    @property
    def Q(self) -> int:
        return 19 if self.lattice == D3Q19 else 9

    def c(self) -> _Params:
        nx, ny, nz = self.shape
        return _Params(nx, ny, nz, self.lattice, self.stencil, self.psi_self,
                       (ctypes.c_double * 2)(*self.tau), self.G, (ctypes.c_double * 2)(*self.G_self))


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        L.orc_q.argtypes = [ctypes.c_int]
        L.orc_stencil.argtypes = [pp, ctypes.POINTER(ctypes.c_int), dp]
        L.orc_velocity_set.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp]
        L.orc_init.argtypes = [pp, dp, dp, dp]
        L.orc_density.argtypes = [pp, dp, dp, dp]
        L.orc_force.argtypes = [pp, dp, dp, dp, dp]
        L.orc_moments.argtypes = [pp, dp, dp, dp, ctypes.c_void_p]
        L.orc_step.argtypes = [pp, dp, dp, ctypes.c_int]
        L.orc_step_sites.argtypes = [pp, dp, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, dp]
        L.orc_totals.argtypes = [pp, dp, dp, dp]
        L.orc_bulk_pressure.argtypes = [pp, ctypes.c_double, ctypes.c_double]
        L.orc_bulk_pressure.restype = ctypes.c_double
        L.orc_pressure_tensor.argtypes = [pp, dp, dp, dp]
        L.orc_profile.argtypes = [pp, dp, dp, ctypes.c_int, dp, ctypes.c_double, ctypes.c_int, dp]
        L.orc_threads.argtypes = []
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _flat(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))


def threads() -> int:
    """OpenMP threads the oracle's loops run on."""
    return int(lib().orc_threads())


def stencil(p: Params):
    """Full forcing stencil (vectors [n, 3], weights [n]) as the oracle uses it."""
    vec = np.zeros((64, 3), dtype=np.int32)
    W = np.zeros(64)
    n = lib().orc_stencil(ctypes.byref(p.c()), vec.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(W))
    return vec[:n].copy(), W[:n].copy()


def velocity_set(lattice: int):
    """(xi [Q, 3], w [Q]) in the oracle's direction order."""
    xi = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19)
    q = lib().orc_velocity_set(int(lattice), xi.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w))
    return xi[:q].copy(), w[:q].copy()


def init(p: Params, nA, nB) -> np.ndarray:
    """Rest equilibrium populations f[2, Q, N] with f_i = w_i n_J."""
    f = np.zeros((2, p.Q, p.n_sites))
    lib().orc_init(ctypes.byref(p.c()), _dp(_flat(nA)), _dp(_flat(nB)), _dp(f))
    return f


def step(p: Params, f: np.ndarray, nsteps: int = 1) -> np.ndarray:
    """Advance a copy of f by nsteps time steps (Eq. lbm)."""
    f = np.ascontiguousarray(f, dtype=np.float64).copy()
    tmp = np.empty_like(f)
    lib().orc_step(ctypes.byref(p.c()), _dp(f), _dp(tmp), int(nsteps))
    return f


def step_sites(p: Params, f: np.ndarray, sites) -> np.ndarray:
    """f_i^J(site, t+1) for the listed sites only -> [2, Q, len(sites)]."""
    sites = np.ascontiguousarray(np.asarray(sites, dtype=np.int64))
    out = np.zeros((2, p.Q, len(sites)))
    f = np.ascontiguousarray(f, dtype=np.float64)
    lib().orc_step_sites(ctypes.byref(p.c()), _dp(f), sites.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                         len(sites), _dp(out))
    return out


def moments(p: Params, f: np.ndarray, with_u: bool = True):
    """(n_A, n_B, u[3, N]) of state f; u is the common velocity of Eq. u."""
    N = p.n_sites
    nA, nB = np.zeros(N), np.zeros(N)
    u = np.zeros((3, N)) if with_u else None
    f = np.ascontiguousarray(f, dtype=np.float64)
    lib().orc_moments(ctypes.byref(p.c()), _dp(f), _dp(nA), _dp(nB),
                      u.ctypes.data_as(ctypes.c_void_p) if with_u else None)
    return nA, nB, u


def force(p: Params, nA, nB):
    """Shan-Chen forces F_A, F_B ([3, N] each) of Eq. sc_force."""
    N = p.n_sites
    FA, FB = np.zeros((3, N)), np.zeros((3, N))
    lib().orc_force(ctypes.byref(p.c()), _dp(_flat(nA)), _dp(_flat(nB)), _dp(FA), _dp(FB))
    return FA, FB


def totals(p: Params, f: np.ndarray):
    """(mass[2], momentum[3]) summed over the lattice."""
    mass, mom = np.zeros(2), np.zeros(3)
    lib().orc_totals(ctypes.byref(p.c()), _dp(np.ascontiguousarray(f, dtype=np.float64)), _dp(mass), _dp(mom))
    return mass, mom


def bulk_pressure(p: Params, nA: float, nB: float) -> float:
    """Eq. bulkp."""
    return lib().orc_bulk_pressure(ctypes.byref(p.c()), float(nA), float(nB))


def pressure_tensor(p: Params, nA, nB) -> np.ndarray:
    """Eq. sm:pt per site: [6, N] with components (xx, yy, zz, xy, xz, yz)."""
    P = np.zeros((6, p.n_sites))
    lib().orc_pressure_tensor(ctypes.byref(p.c()), _dp(_flat(nA)), _dp(_flat(nB)), _dp(P))
    return P


RADIAL, PLANAR_Z, AXIS_X = 0, 1, 2


def profile(p: Params, nA, nB, kind: int, centre=(0.0, 0.0, 0.0), bin_width: float = 0.5,
            nbins: int = 0) -> np.ndarray:
    """Rows [nbins, 6] = (coordinate, P_N, P_T, n_A, n_B, count); see sc_oracle.c."""
    out = np.zeros((nbins, 6))
    c = np.ascontiguousarray(np.asarray(centre, dtype=np.float64))
    lib().orc_profile(ctypes.byref(p.c()), _dp(_flat(nA)), _dp(_flat(nB)), int(kind), _dp(c), float(bin_width),
                      int(nbins), _dp(out))
    return out
