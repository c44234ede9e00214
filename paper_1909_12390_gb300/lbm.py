"""Python binding of liblbm.so (include/lbm.h): argument marshalling only.

Every step of the lattice Boltzmann path runs in the library's CUDA kernels. There is no
CPU fallback: if the library is missing or cannot be loaded, the import fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# LBM_LIBRARY overrides the library file (e.g. a build with other compile-time tile options)
LIB_PATH = os.environ.get("LBM_LIBRARY") or os.path.join(_PKG, "liblbm.so")

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_PSI_DOMAIN, ERR_NONFINITE, ERR_TIMEOUT = 0, -1, -2, -3, -4, -5, -6
D2Q9, D3Q19 = 9, 19
BGK, MRT = 0, 1
FP64, FP32_SHIFTED = 0, 1

# the entry points include/lbm.h declares
EXPORTS = ("lbm_create", "lbm_destroy", "lbm_set_stream", "lbm_init", "lbm_step", "lbm_time",
           "lbm_fields", "lbm_mass", "lbm_get_f", "lbm_set_f", "lbm_state_bytes", "lbm_save",
           "lbm_restore", "lbm_last_error", "lbm_scale_to_lattice", "lbm_profile",
           "lbm_profile_read", "lbm_set_path", "lbm_get_path", "lbm_get_fused_kind", "lbm_test_silence_block",

           "lbm_step_static", "lbm_step_static_error", "lbm_batch_create", "lbm_batch_destroy",
           "lbm_batch_init", "lbm_batch_step", "lbm_batch_case_status", "lbm_batch_fields",
           "lbm_batch_get_f", "lbm_batch_tune", "lbm_batch_tune_report", "lbm_batch_sites",
           "lbm_batch_last_error", "lbm_record", "lbm_adjoint", "lbm_set_adjoint_memory", "lbm_test_adjoint_overlap", "lbm_revolve_steps", "lbm_queue_schedule", "lbm_flash", "lbm_flash_error", "lbm_diagnostics")
STATIC_MAX_SITES = 1048576
PATH_AUTO, PATH_TWO_KERNEL, PATH_FUSED, PATH_TRAILING, PATH_QUEUE = 0, 1, 2, 3, 4
FUSED_TILES, FUSED_PLANES = 1, 3
SPLIT_VOLATILITY, SPLIT_GONG = 0, 1


class LBMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("lbm status %d: %s" % (status, msg))
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("lattice", ctypes.c_int)]


class Component(ctypes.Structure):
    _fields_ = [("Tc", ctypes.c_double), ("pc", ctypes.c_double), ("omega", ctypes.c_double),
                ("M", ctypes.c_double)]


_DP = ctypes.POINTER(ctypes.c_double)


class Eos(ctypes.Structure):
    _fields_ = [("T", ctypes.c_double), ("R", ctypes.c_double), ("kij", _DP), ("gamma", _DP),
                ("beta", ctypes.c_double), ("G", ctypes.c_double), ("collision", ctypes.c_int),
                ("mrt_rates", _DP), ("precision", ctypes.c_int), ("rho_ref", _DP), ("split", ctypes.c_int)]


class FlashCase(ctypes.Structure):
    _fields_ = [("T", ctypes.c_double), ("p", ctypes.c_double), ("z", ctypes.c_double * 4),
                ("kij", ctypes.c_double * 16)]


class FlashResult(ctypes.Structure):
    _fields_ = [("V", ctypes.c_double), ("x", ctypes.c_double * 4), ("y", ctypes.c_double * 4),
                ("K", ctypes.c_double * 4), ("Zl", ctypes.c_double), ("Zv", ctypes.c_double),
                ("residual", ctypes.c_double), ("rho_l", ctypes.c_double * 4),
                ("rho_v", ctypes.c_double * 4), ("gamma", ctypes.c_double * 4),
                ("iterations", ctypes.c_int), ("status", ctypes.c_int)]


FLASH_TWO_PHASE, FLASH_SINGLE, FLASH_NOT_CONVERGED = 0, 1, 2


class DiagParams(ctypes.Structure):
    _fields_ = [("threshold", ctypes.c_double), ("erode", ctypes.c_int)]


class DiagResult(ctypes.Structure):
    _fields_ = [("threshold", ctypes.c_double), ("rho_max", ctypes.c_double), ("rho_min", ctypes.c_double),
                ("rho_l", ctypes.c_double * 4), ("rho_v", ctypes.c_double * 4), ("p_l", ctypes.c_double),
                ("p_v", ctypes.c_double), ("x", ctypes.c_double * 4), ("y", ctypes.c_double * 4),
                ("residual", ctypes.c_double), ("radius", ctypes.c_double), ("dp", ctypes.c_double),
                ("n_l", ctypes.c_int64), ("n_v", ctypes.c_int64), ("liquid_cells", ctypes.c_int64)]

_lib = None


def lib() -> ctypes.CDLL:
    """Loads liblbm.so; raises if it is absent (build it with __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("liblbm.so not built: %s (run __graft_entry__.build())" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        L.lbm_create.argtypes = [ctypes.POINTER(Grid), ctypes.c_int, ctypes.POINTER(Component),
                                 ctypes.POINTER(Eos), ctypes.c_double, ctypes.POINTER(vp)]
        L.lbm_destroy.argtypes = [vp]
        L.lbm_destroy.restype = None
        L.lbm_set_stream.argtypes = [vp, vp]
        L.lbm_init.argtypes = [vp, _DP, _DP]
        L.lbm_step.argtypes = [vp, ctypes.c_int64]
        L.lbm_time.argtypes = [vp]
        L.lbm_time.restype = ctypes.c_int64
        L.lbm_fields.argtypes = [vp, _DP, _DP, _DP, _DP]
        L.lbm_mass.argtypes = [vp, _DP]
        L.lbm_get_f.argtypes = [vp, _DP]
        L.lbm_set_f.argtypes = [vp, _DP]
        L.lbm_state_bytes.argtypes = [vp]
        L.lbm_state_bytes.restype = ctypes.c_size_t
        L.lbm_save.argtypes = [vp, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int64)]
        L.lbm_restore.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_int64]
        L.lbm_profile.argtypes = [vp, ctypes.c_int]
        L.lbm_profile_read.argtypes = [vp, ctypes.c_int, _DP, ctypes.POINTER(ctypes.c_int64)]
        L.lbm_set_path.argtypes = [vp, ctypes.c_int]
        L.lbm_get_path.argtypes = [vp]
        L.lbm_get_fused_kind.argtypes = [vp]
        L.lbm_test_silence_block.argtypes = [vp, ctypes.c_int]
        L.lbm_step_static.argtypes = [ctypes.POINTER(Grid), ctypes.c_int, ctypes.POINTER(Component),
                                      ctypes.POINTER(Eos), ctypes.c_double, vp, ctypes.c_int64, ctypes.c_int64,
                                      vp, ctypes.POINTER(ctypes.c_int64)]
        L.lbm_step_static_error.argtypes = []
        L.lbm_flash.argtypes = [ctypes.c_int, ctypes.POINTER(Component), ctypes.c_int, ctypes.POINTER(FlashCase),
                                ctypes.c_double, ctypes.c_double, ctypes.c_int, vp, ctypes.POINTER(FlashResult)]
        L.lbm_diagnostics.argtypes = [vp, ctypes.POINTER(DiagParams), ctypes.POINTER(DiagResult)]
        L.lbm_flash_error.argtypes = []
        L.lbm_flash_error.restype = ctypes.c_char_p
        L.lbm_step_static_error.restype = ctypes.c_char_p
        L.lbm_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(Grid), ctypes.c_int,
                                       ctypes.POINTER(Component), ctypes.POINTER(Eos), _DP, ctypes.POINTER(vp)]
        L.lbm_batch_destroy.argtypes = [vp]
        L.lbm_batch_destroy.restype = None
        L.lbm_batch_init.argtypes = [vp, _DP, _DP]
        L.lbm_batch_step.argtypes = [vp, ctypes.c_int64]
        L.lbm_batch_case_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64)]
        L.lbm_batch_fields.argtypes = [vp, _DP, _DP, _DP]
        L.lbm_batch_get_f.argtypes = [vp, ctypes.c_int, _DP]
        L.lbm_batch_tune.argtypes = [vp, ctypes.c_int]
        L.lbm_batch_tune_report.argtypes = [vp]
        L.lbm_batch_tune_report.restype = ctypes.c_char_p
        L.lbm_batch_sites.argtypes = [vp]
        L.lbm_batch_sites.restype = ctypes.c_int64
        L.lbm_batch_last_error.argtypes = [vp]
        L.lbm_batch_last_error.restype = ctypes.c_char_p
        L.lbm_record.argtypes = [vp, ctypes.c_int64, ctypes.c_int]
        L.lbm_adjoint.argtypes = [vp, _DP, _DP, _DP, _DP]
        L.lbm_set_adjoint_memory.argtypes = [vp, ctypes.c_int]
        L.lbm_test_adjoint_overlap.argtypes = [vp, ctypes.c_int]
        L.lbm_revolve_steps.argtypes = [ctypes.c_int64, ctypes.c_int]
        L.lbm_revolve_steps.restype = ctypes.c_int64
        L.lbm_queue_schedule.argtypes = [ctypes.c_int] * 5 + [vp, vp]
        L.lbm_queue_schedule.restype = ctypes.c_int
        L.lbm_last_error.argtypes = [vp]
        L.lbm_last_error.restype = ctypes.c_char_p
        L.lbm_scale_to_lattice.argtypes = [ctypes.c_int, ctypes.POINTER(Component), ctypes.c_double,
                                           ctypes.c_double, ctypes.POINTER(Component), _DP, _DP]
        _lib = L
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(_DP)


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def make_args(shape, components, T, gamma=None, kij=None, beta=1.0, G=-1.0, collision=BGK,
              mrt_rates=None, precision=FP64, rho_ref=None, R=1.0, split=0):
    """The lbm_grid, lbm_component[] and lbm_eos of one lattice (plus arrays to keep alive)."""
    shape = tuple(int(s) for s in shape)
    Q = D2Q9 if len(shape) == 2 else D3Q19
    nx, ny = shape[0], shape[1]
    nz = shape[2] if len(shape) == 3 else 1
    nc = len(components)
    comps = (Component * nc)(*[Component(*c) for c in components])
    keep = []

    def arr(v, n):
        if v is None:
            return None
        a = _f64(v, n)
        keep.append(a)
        return _dp(a)

    eos = Eos(T=T, R=R, kij=arr(None if kij is None else np.asarray(kij, dtype=float).ravel(), nc * nc),
              gamma=arr(gamma, nc), beta=beta, G=G, collision=collision,
              mrt_rates=arr(mrt_rates, Q), precision=precision, rho_ref=arr(rho_ref, nc), split=int(split))
    return Grid(nx, ny, nz, Q), comps, eos, keep


QUEUE_MAX_NBR = 16


def queue_schedule(nx: int, ny: int, nz: int, chunk: int = 0, lag: int = 0):
    """lbm_queue_schedule: (nch, nbr[nch, QUEUE_MAX_NBR], tasks[2 nz nch]) of the task-queue
    step on an nx x ny x nz grid, or None when the grid is not served."""
    L = lib()
    nch = int(L.lbm_queue_schedule(nx, ny, nz, chunk, lag, None, None))
    if nch < 0:
        return None
    nbr = np.empty((nch, QUEUE_MAX_NBR), dtype=np.int32)
    tasks = np.empty(2 * nz * nch, dtype=np.int32)
    L.lbm_queue_schedule(nx, ny, nz, chunk, lag, nbr.ctypes.data_as(ctypes.c_void_p),
                         tasks.ctypes.data_as(ctypes.c_void_p))
    return nch, nbr, tasks


def revolve_steps(n: int, snapshots: int) -> int:
    """lbm_revolve_steps: forward steps the adjoint's reverse sweep recomputes for a segment of
    n steps with the given state slots."""
    return int(lib().lbm_revolve_steps(int(n), int(snapshots)))


def step_static(shape, components, T, tau, f_device_ptr: int, t0: int, n: int, stream: int = 0, **kw):
    """lbm_step_static on caller-owned device populations at address f_device_ptr; returns the
    step index reached (t0 + completed steps). Raises LBMError on failure; its `time` attribute
    is then the index of the failing step (None when the call failed before running)."""
    grid, comps, eos, keep = make_args(shape, components, T, **kw)
    tout = ctypes.c_int64()
    st = lib().lbm_step_static(ctypes.byref(grid), len(components), comps, ctypes.byref(eos), tau,
                               ctypes.c_void_p(f_device_ptr), int(t0), int(n), ctypes.c_void_p(stream or None),
                               ctypes.byref(tout))
    if st != OK:
        err = LBMError(st, lib().lbm_step_static_error().decode())
        err.time = tout.value if st in (ERR_PSI_DOMAIN, ERR_NONFINITE, ERR_TIMEOUT) else None
        raise err
    return tout.value


def flash(components, T, p, z, kij=None, R=1.0, tol=1e-13, maxit=20000, stream: int = 0):
    """lbm_flash over the cases (T[k], p[k], z[k], kij[k]) of one set of components
    ((Tc, pc, omega, M) tuples). T, p: (ncase,); z: (ncase, nc); kij: (ncase, nc, nc) or None.
    Returns a dict of arrays: V, x, y, K, Zl, Zv, residual, rho_l, rho_v, gamma, iterations,
    status (FLASH_TWO_PHASE, FLASH_SINGLE, FLASH_NOT_CONVERGED)."""
    nc = len(components)
    if not 1 <= nc <= 4:
        raise LBMError(ERR_ARG, "nc must be 1..4")
    T = np.atleast_1d(np.asarray(T, dtype=np.float64))
    p = np.atleast_1d(np.asarray(p, dtype=np.float64))
    z = np.asarray(z, dtype=np.float64).reshape(len(T), nc)
    kij = np.zeros((len(T), nc, nc)) if kij is None else np.asarray(kij, dtype=np.float64).reshape(len(T), nc, nc)
    n = len(T)
    comps = (Component * nc)(*[Component(*map(float, c)) for c in components])
    cases = (FlashCase * max(n, 1))()
    for k in range(n):
        cases[k].T, cases[k].p = T[k], p[k]
        for i in range(nc):
            cases[k].z[i] = z[k, i]
            for j in range(nc):
                cases[k].kij[i * nc + j] = kij[k, i, j]
    out = (FlashResult * max(n, 1))()
    st = lib().lbm_flash(nc, comps, n, cases, float(R), float(tol), int(maxit), ctypes.c_void_p(stream or None), out)
    if st != OK:
        raise LBMError(st, lib().lbm_flash_error().decode())
    res = {}
    for name in ("V", "Zl", "Zv", "residual"):
        res[name] = np.array([getattr(out[k], name) for k in range(n)])
    for name in ("x", "y", "K", "rho_l", "rho_v", "gamma"):
        res[name] = np.array([list(getattr(out[k], name))[:nc] for k in range(n)]).reshape(n, nc)
    res["iterations"] = np.array([out[k].iterations for k in range(n)])
    res["status"] = np.array([out[k].status for k in range(n)])
    return res


class Lattice:
    """One periodic lattice with nc components, behind lbm_create / lbm_destroy.

    shape is (nx, ny) for D2Q9 or (nx, ny, nz) for D3Q19; fields are returned with array
    shape (nc, nz, ny, nx) / (nc, ny, nx) (x fastest), populations as (nc, Q, *grid)."""

    def __init__(self, shape, components, T, tau, gamma=None, kij=None, beta=1.0, G=-1.0,
                 collision=BGK, mrt_rates=None, precision=FP64, rho_ref=None, R=1.0, split=0):
        L = lib()
        grid, comps, eos, keep = make_args(shape, components, T, gamma=gamma, kij=kij, beta=beta, G=G,
                                           collision=collision, mrt_rates=mrt_rates, precision=precision,
                                           rho_ref=rho_ref, R=R, split=split)
        self._keep = keep
        shape = tuple(int(s) for s in shape)
        self.Q = grid.lattice
        self.shape = shape
        self.grid = tuple(reversed(shape))
        self.N = grid.nx * grid.ny * grid.nz
        self.nc = len(components)
        h = ctypes.c_void_p()
        st = L.lbm_create(ctypes.byref(grid), self.nc, comps, ctypes.byref(eos), tau, ctypes.byref(h))
        if st != OK:
            raise LBMError(st, L.lbm_last_error(None).decode())
        self._h = h
        self.precision = precision

    def _check(self, st):
        if st != OK:
            raise LBMError(st, lib().lbm_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_handle: int):
        self._check(lib().lbm_set_stream(self._h, ctypes.c_void_p(stream_handle)))

    def init(self, rho, u=None):
        r = _f64(rho, self.nc * self.N)
        uu = None if u is None else _f64(u, 3 * self.N)
        self._check(lib().lbm_init(self._h, _dp(r), _dp(uu)))

    def step(self, n: int = 1):
        self._check(lib().lbm_step(self._h, int(n)))

    @property
    def time(self) -> int:
        return int(lib().lbm_time(self._h))

    def fields(self, rho=True, u=True, p=True, psi=True):
        out = {}
        bufs = {}
        if rho:
            bufs["rho"] = np.empty((self.nc,) + self.grid)
        if u:
            bufs["u"] = np.empty((3,) + self.grid)
        if p:
            bufs["p"] = np.empty(self.grid)
        if psi:
            bufs["psi"] = np.empty(self.grid)
        self._check(lib().lbm_fields(self._h, _dp(bufs.get("rho")), _dp(bufs.get("u")),
                                     _dp(bufs.get("p")), _dp(bufs.get("psi"))))
        out.update(bufs)
        return out

    def fields_into(self, rho=None, u=None, p=None, psi=None):
        """Writes the fields into caller-provided C-contiguous float64 host arrays."""
        self._check(lib().lbm_fields(self._h, _dp(rho), _dp(u), _dp(p), _dp(psi)))

    def diagnostics(self, erode: int = 8, threshold: float = 0.0) -> dict:
        """lbm_diagnostics: bulk phases, compositions, iso-fugacity residual, radius, Laplace
        jump of the current state (see include/lbm.h)."""
        r = DiagResult()
        self._check(lib().lbm_diagnostics(self._h, ctypes.byref(DiagParams(float(threshold), int(erode))),
                                          ctypes.byref(r)))
        out = {k: getattr(r, k) for k in ("threshold", "rho_max", "rho_min", "p_l", "p_v", "residual", "radius",
                                          "dp", "n_l", "n_v", "liquid_cells")}
        for k in ("rho_l", "rho_v", "x", "y"):
            out[k] = np.array(list(getattr(r, k))[:self.nc])
        return out

    def mass(self) -> np.ndarray:
        m = np.empty(self.nc)
        self._check(lib().lbm_mass(self._h, _dp(m)))
        return m

    def get_f(self) -> np.ndarray:
        f = np.empty((self.nc, self.Q) + self.grid)
        self._check(lib().lbm_get_f(self._h, _dp(f)))
        return f

    def set_f(self, f):
        a = _f64(f, self.nc * self.Q * self.N)
        self._check(lib().lbm_set_f(self._h, _dp(a)))

    def set_path(self, path: int):
        self._check(lib().lbm_set_path(self._h, int(path)))

    @property
    def path(self) -> int:
        return int(lib().lbm_get_path(self._h))

    @property
    def fused_kind(self) -> int:
        """FUSED_TILES or FUSED_PLANES on the fused path, else 0."""
        return int(lib().lbm_get_fused_kind(self._h))

    def test_silence_block(self, block: int):
        self._check(lib().lbm_test_silence_block(self._h, int(block)))

    def profile(self, on: bool):
        self._check(lib().lbm_profile(self._h, 1 if on else 0))

    def profile_read(self, kernel: int):
        """(total milliseconds, launches) of kernel kind 0 (psi pass), 1 (collide pass) or 2
        (fused step)."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(lib().lbm_profile_read(self._h, kernel, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def record(self, n: int, checkpoint_every: int):
        """Advance n steps keeping checkpoints for lbm_adjoint."""
        self._check(lib().lbm_record(self._h, int(n), int(checkpoint_every)))

    def set_adjoint_memory(self, snapshots: int):
        """State slots of lbm_adjoint's reverse sweep per segment: 0 keeps every state of a
        segment; fewer than checkpoint_every selects revolve-style binomial checkpointing."""
        self._check(lib().lbm_set_adjoint_memory(self._h, int(snapshots)))

    def test_adjoint_overlap(self, on: bool):
        """Test hook: False runs each segment's replay and reverse sweep one after the other."""
        self._check(lib().lbm_test_adjoint_overlap(self._h, int(bool(on))))

    def adjoint(self, drho):
        """Back-propagate dL/drho(final) (array (nc, *grid)) through the recorded steps.
        Returns (dL/dzeta (nc, nc), dL/dgamma (nc,), dL/drho(start) (nc, *grid))."""
        d = _f64(drho, self.nc * self.N)
        dk = np.zeros(self.nc * self.nc)
        dg = np.zeros(self.nc)
        d0 = np.empty((self.nc,) + self.grid)
        self._check(lib().lbm_adjoint(self._h, _dp(d), _dp(dk), _dp(dg), _dp(d0)))
        return dk.reshape(self.nc, self.nc), dg, d0

    def save(self):
        n = int(lib().lbm_state_bytes(self._h))
        buf = np.empty(n, dtype=np.uint8)
        t = ctypes.c_int64()
        self._check(lib().lbm_save(self._h, buf.ctypes.data_as(ctypes.c_void_p), n, ctypes.byref(t)))
        return buf, t.value

    def restore(self, buf, t):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._check(lib().lbm_restore(self._h, buf.ctypes.data_as(ctypes.c_void_p), buf.size, int(t)))


class Batch:
    """Many independent D2Q9 lattices behind lbm_batch_create. `cases` is a list of dicts with
    keys shape (nx, ny), components [(Tc, pc, omega, M)], T, tau and optional gamma, kij,
    beta, G, mrt_rates, rho_ref; collision and precision are common to all cases."""

    def __init__(self, cases, collision=BGK, precision=FP64):
        L = lib()
        n = len(cases)
        nc = len(cases[0]["components"])
        self.nc = nc
        self.shapes = [tuple(int(v) for v in c["shape"]) for c in cases]
        self.sizes = [s[0] * s[1] for s in self.shapes]
        grids = (Grid * n)()
        comps = (Component * (n * nc))()
        eoss = (Eos * n)()
        taus = np.array([float(c["tau"]) for c in cases])
        self._keep = [taus]
        for i, c in enumerate(cases):
            g, cp, e, keep = make_args(c["shape"], c["components"], c["T"], gamma=c.get("gamma"),
                                       kij=c.get("kij"), beta=c.get("beta", 1.0), G=c.get("G", -1.0),
                                       collision=collision, mrt_rates=c.get("mrt_rates"),
                                       precision=precision, rho_ref=c.get("rho_ref"), split=c.get("split", 0))
            grids[i] = g
            for k in range(nc):
                comps[i * nc + k] = cp[k]
            eoss[i] = e
            self._keep.append(keep)
        h = ctypes.c_void_p()
        st = L.lbm_batch_create(n, grids, nc, comps, eoss, _dp(taus), ctypes.byref(h))
        if st != OK:
            raise LBMError(st, L.lbm_batch_last_error(None).decode())
        self._h = h
        self.ncase = n

    def _check(self, st):
        if st != OK:
            raise LBMError(st, lib().lbm_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, rho_list):
        """rho_list[i]: array (nc, ny, nx) of case i."""
        flat = np.concatenate([np.ascontiguousarray(r, dtype=np.float64).ravel() for r in rho_list])
        self._check(lib().lbm_batch_init(self._h, _dp(flat), None))

    def step(self, n):
        self._check(lib().lbm_batch_step(self._h, int(n)))

    def tune(self, trial_steps=20):
        self._check(lib().lbm_batch_tune(self._h, int(trial_steps)))
        return lib().lbm_batch_tune_report(self._h).decode()

    def case_status(self):
        st = (ctypes.c_int * self.ncase)()
        t = (ctypes.c_int64 * self.ncase)()
        self._check(lib().lbm_batch_case_status(self._h, st, t))
        return list(st), list(t)

    def rho(self):
        """List of (nc, ny, nx) density arrays, one per case."""
        total = sum(self.sizes) * self.nc
        out = np.empty(total)
        self._check(lib().lbm_batch_fields(self._h, _dp(out), None, None))
        res, off = [], 0
        for (nx, ny), n in zip(self.shapes, self.sizes):
            res.append(out[off:off + self.nc * n].reshape(self.nc, ny, nx))
            off += self.nc * n
        return res

    def rho_into(self, out):
        self._check(lib().lbm_batch_fields(self._h, _dp(out), None, None))

    def get_f(self, i):
        nx, ny = self.shapes[i]
        f = np.empty((self.nc, 9, ny, nx))
        self._check(lib().lbm_batch_get_f(self._h, int(i), _dp(f)))
        return f


def scale_to_lattice(components, T_phys, p_phys):
    """Section 4.2 scaling (see include/lbm.h). components: list of (Tc, pc, omega, M)."""
    nc = len(components)
    src = (Component * nc)(*[Component(*c) for c in components])
    dst = (Component * nc)()
    T = ctypes.c_double()
    p = ctypes.c_double()
    st = lib().lbm_scale_to_lattice(nc, src, T_phys, p_phys, dst, ctypes.byref(T), ctypes.byref(p))
    if st != OK:
        raise LBMError(st, "lbm_scale_to_lattice")
    return [(d.Tc, d.pc, d.omega, d.M) for d in dst], T.value, p.value
