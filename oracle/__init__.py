"""FP64 CPU oracle of the multi-component pseudo-potential LB step of Peng, Ayala & Ayala
(arXiv:1909.12390): the step itself in plain C++ (lbm_oracle.cpp, loaded here through
ctypes) and the phase-equilibrium calculations in plain Python (thermo.py).

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke(), bench.py's cpu_baseline /
reference leg and the case-writing script beside the golden files may import this package.
It shares no code with the CUDA library (paper_1909_12390_gb300) and imports nothing from it.

Parity status: every function here is pinned by a test against a value the paper prints, a
closed form, an invariant or brute force (see tests/test_oracle_*.py). The MRT collision is
not in the paper; it is pinned by its reduction to BGK when every rate equals 1/tau, by exact
mass conservation and by the orthogonality of its moment basis. The forward-mode derivative
(step_dual) is pinned by central differences of step, by the independence of its two
directions and by the zero split derivative of the total density of identical components
(tests/test_oracle_dual.py), which also pins both split factors through the component
momenta a step produces.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

OK, ERR_ARG, ERR_PSI_DOMAIN, ERR_NONFINITE = 0, -1, -4, -5


def build(force: bool = False) -> str:
    """Compile the C++ oracle with gcc, no fused multiply-add contraction."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c++17",
                               "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _Case(ctypes.Structure):
    _fields_ = [("Q", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("nc", ctypes.c_int), ("tau", ctypes.c_double),
                ("collision", ctypes.c_int), ("s", ctypes.c_double * 19),
                ("T", ctypes.c_double), ("R", ctypes.c_double),
                ("Tc", ctypes.c_double * 4), ("pc", ctypes.c_double * 4),
                ("omega", ctypes.c_double * 4), ("M", ctypes.c_double * 4),
                ("kij", ctypes.c_double * 16), ("gamma", ctypes.c_double * 4),
                ("beta", ctypes.c_double), ("G", ctypes.c_double), ("split", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        cp = ctypes.POINTER(_Case)
        _lib.oracle_step.argtypes = [cp, dp, ctypes.c_int, ip]
        _lib.oracle_step_dual.argtypes = [cp, dp, dp, dp, ctypes.c_int, ip]
        _lib.oracle_fields.argtypes = [cp, dp, dp, dp, dp, dp, dp]
        _lib.oracle_eos.argtypes = [cp, dp, dp, dp]
        _lib.oracle_equilibrium.argtypes = [cp, dp, dp, dp]
        _lib.oracle_lattice.argtypes = [ctypes.c_int, ip, dp]
        _lib.oracle_mrt_matrix.argtypes = [ctypes.c_int, dp, dp]
        _lib.oracle_threads.argtypes = []
        _lib.oracle_set_threads.argtypes = [ctypes.c_int]
        _lib.oracle_set_threads.restype = None
    return _lib


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class OracleError(RuntimeError):
    def __init__(self, status, step=None):
        super().__init__("oracle status %d at step %s" % (status, step))
        self.status = status
        self.step = step


@dataclass
class Case:
    """One lattice problem in lattice units. shape is (nx, ny) or (nx, ny, nz)."""
    Q: int
    shape: tuple
    Tc: list
    pc: list
    omega: list
    M: list
    T: float
    tau: float
    gamma: list
    kij: list = None
    beta: float = 1.0
    G: float = -1.0
    R: float = 1.0
    collision: int = 0
    s: list = None
    split: int = 0  # 0: Eq. distributionforce; 1: Eq. Gong with sqrt(|p0 - ph_i|)

    def __post_init__(self):
        nc = len(self.Tc)
        if self.kij is None:
            self.kij = [[0.0] * nc for _ in range(nc)]

    @property
    def nc(self):
        return len(self.Tc)

    @property
    def D(self):
        return 2 if self.Q == 9 else 3

    @property
    def nsites(self):
        return int(np.prod(self.shape))

    @property
    def grid(self):
        """Array shape of one field, slowest first: (nz, ny, nx) or (ny, nx)."""
        return tuple(reversed(self.shape))

    def cstruct(self) -> _Case:
        c = _Case()
        c.Q = self.Q
        nx, ny = self.shape[0], self.shape[1]
        nz = self.shape[2] if len(self.shape) > 2 else 1
        c.nx, c.ny, c.nz, c.nc = nx, ny, nz, self.nc
        c.tau = self.tau
        c.collision = self.collision
        if self.s is not None:
            for k, v in enumerate(self.s):
                c.s[k] = v
        c.T, c.R = self.T, self.R
        c.split = self.split
        for i in range(self.nc):
            c.Tc[i], c.pc[i], c.omega[i], c.M[i] = self.Tc[i], self.pc[i], self.omega[i], self.M[i]
            c.gamma[i] = self.gamma[i]
            for j in range(self.nc):
                c.kij[i * self.nc + j] = self.kij[i][j]
        c.beta, c.G = self.beta, self.G
        return c


def equilibrium(case: Case, rho: np.ndarray, u: np.ndarray = None) -> np.ndarray:
    """f_eq(rho_s, u) (Eq. equilibrium a), layout (nc, Q, *grid)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(case.nc, -1)
    f = np.empty((case.nc, case.Q, case.nsites))
    uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64).reshape(3, -1)
    st = lib().oracle_equilibrium(ctypes.byref(case.cstruct()), _dp(rho), _dp(uu), _dp(f))
    if st != OK:
        raise OracleError(st)
    return f.reshape((case.nc, case.Q) + case.grid)


def step(case: Case, f: np.ndarray, nsteps: int = 1) -> np.ndarray:
    """Advance populations f (nc, Q, *grid) by nsteps; returns a new array."""
    g = np.array(f, dtype=np.float64, order="C", copy=True)
    fs = ctypes.c_int(-1)
    st = lib().oracle_step(ctypes.byref(case.cstruct()), _dp(g), int(nsteps), ctypes.byref(fs))
    if st != OK:
        raise OracleError(st, fs.value)
    return g


def step_dual(case: Case, f: np.ndarray, df: np.ndarray, dkij: np.ndarray, dgamma: np.ndarray,
              nsteps: int = 1):
    """Forward-mode derivative run. f (nc, Q, *grid); df (2, nc, Q, *grid) the derivatives of
    the initial state; dkij (2, nc, nc) and dgamma (2, nc) the derivatives of zeta_ij and
    gamma_i with respect to two parameters. Returns (f, df) after nsteps."""
    n = f.size
    buf = np.empty(3 * n)
    buf[:n] = f.ravel()
    buf[n:] = np.asarray(df, dtype=np.float64).ravel()
    dk = np.ascontiguousarray(dkij, dtype=np.float64).ravel()
    dg = np.ascontiguousarray(dgamma, dtype=np.float64).ravel()
    fs = ctypes.c_int(-1)
    st = lib().oracle_step_dual(ctypes.byref(case.cstruct()), _dp(dk), _dp(dg), _dp(buf),
                                int(nsteps), ctypes.byref(fs))
    if st != OK:
        raise OracleError(st, fs.value)
    return buf[:n].reshape(f.shape), buf[n:].reshape((2,) + f.shape)


@dataclass
class Fields:
    rho: np.ndarray  # (nc, *grid)
    u: np.ndarray    # (3, *grid)
    p: np.ndarray    # (*grid)
    psi: np.ndarray  # (*grid)
    F: np.ndarray    # (3, *grid)


def fields(case: Case, f: np.ndarray) -> Fields:
    g = np.ascontiguousarray(f, dtype=np.float64)
    N = case.nsites
    rho = np.empty(case.nc * N)
    u = np.empty(3 * N)
    p = np.empty(N)
    psi = np.empty(N)
    F = np.empty(3 * N)
    st = lib().oracle_fields(ctypes.byref(case.cstruct()), _dp(g), _dp(rho), _dp(u), _dp(p),
                             _dp(psi), _dp(F))
    if st != OK:
        raise OracleError(st)
    gr = case.grid
    return Fields(rho.reshape((case.nc,) + gr), u.reshape((3,) + gr), p.reshape(gr),
                  psi.reshape(gr), F.reshape((3,) + gr))


def eos(case: Case, rho_c) -> tuple:
    """(p_EOS, psi^2) of one site with cell-volume densities rho_c."""
    r = np.ascontiguousarray(rho_c, dtype=np.float64)
    p = ctypes.c_double()
    q = ctypes.c_double()
    st = lib().oracle_eos(ctypes.byref(case.cstruct()), _dp(r), ctypes.byref(p), ctypes.byref(q))
    if st not in (OK, ERR_PSI_DOMAIN):
        raise OracleError(st)
    return p.value, q.value


def lattice(Q: int):
    e = np.zeros(19 * 3, dtype=np.int32)
    w = np.zeros(19)
    D = lib().oracle_lattice(Q, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w))
    return D, e.reshape(19, 3)[:Q], w[:Q]


def mrt_matrix(Q: int):
    M = np.zeros(Q * Q)
    Mi = np.zeros(Q * Q)
    st = lib().oracle_mrt_matrix(Q, _dp(M), _dp(Mi))
    if st != OK:
        raise OracleError(st)
    return M.reshape(Q, Q), Mi.reshape(Q, Q)


def threads() -> int:
    """OpenMP threads the oracle's loops use (set OMP_NUM_THREADS before the first call)."""
    return int(lib().oracle_threads())


def set_threads(n: int) -> None:
    """Threads of the oracle's later loops (results do not depend on it)."""
    lib().oracle_set_threads(int(n))


def mass(f: np.ndarray) -> np.ndarray:
    """Per-component total mass sum_x sum_a f (FP64)."""
    nc, Q = f.shape[:2]
    return f.reshape(nc, -1).sum(axis=1)
