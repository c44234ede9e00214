"""Peng-Robinson phase-equilibrium oracle (plain FP64 Python), Section 3.2 of
Peng, Ayala & Ayala, arXiv:1909.12390.

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke(), bench.py's cpu_baseline /
reference leg and the case-writing script beside the golden files may import this module.
It shares no code with the CUDA library.

What it computes, in the paper's notation:
  * a_i, b_i, alpha_i(T), m_i                                  (Section 3.2, after Eq. randommixingrule)
  * A_i, B_i, A_ij, A, B and the cubic in Z                     (Eq. cubiccoeff, Eq. PRcubic)
  * the Gibbs-energy choice between the smallest and largest root (Eq. solutionselection)
  * ln phi_i                                                   (Eq. fugacitycoeff2)
  * fugacities and the iso-fugacity residual                   (Eq. fugacity, Eq. error)
  * a two-phase flash at (T, p, z): Wilson start, Rachford-Rice (negative flash allowed),
    successive substitution K_i = phi_li / phi_vi until the residual vanishes
  * the volatility coefficients gamma_i                        (Eq. gamma, generalised)
  * pure-substance saturation by equal fugacity (the Maxwell rule of Section 4.1)
  * the scaling of physical critical constants into lattice units (Section 4.2)

Readings of garbled or silent passages (each pinned by Table 2 in the tests):
  * Eq. PRcubic is printed with wrong coefficients. The cubic used is the one that follows
    from Eq. MCPengRobinson: Z^3 - (1 - B) Z^2 + (A - 3B^2 - 2B) Z - (AB - B^2 - B^3) = 0.
  * Eq. cubiccoeff prints A_i with p_ri / T_ri; the dimensionless attraction parameter is
    A_i = Omega_a alpha_i p_ri / T_ri^2 (from A = [a alpha]_m p / (RT)^2).
  * Eq. solutionselection: dG = 0 takes Z_max (the "otherwise" branch).
  * Eq. gamma is derived for two components; for n_c > 2 the same per-component hydrostatic
    balance gives gamma_i = ln(rho_il / rho_iv) / ln(rho_hl / rho_hv), h the least volatile
    component (smallest K), gamma_h = 1.
  * Lattice units: a_1 = 2/49, b_1 = 2/21, M_1 = 1, R = 1 fix T_c1 and p_c1; the other
    components keep the physical ratios T_ci / T_c1, p_ci / p_c1, M_i / M_1, and temperature
    and pressure are scaled by T_c1 and p_c1, so every reduced quantity is unchanged.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

OMEGA_A = 0.45724
OMEGA_B = 0.0778
SQ2 = math.sqrt(2.0)

# lattice-unit attraction and co-volume of component 1 (Section 4.1 and Section 4.2)
A1_LB = 2.0 / 49.0
B1_LB = 2.0 / 21.0


@dataclass
class Component:
    name: str
    Tc: float
    pc: float
    omega: float
    M: float


def m_factor(omega: float) -> float:
    """m_i of Section 3.2 (two branches in the acentric factor)."""
    if omega <= 0.49:
        return 0.374640 + 1.54226 * omega - 0.26992 * omega ** 2
    return 0.379642 + 1.48503 * omega - 0.164423 * omega ** 2 + 0.016666 * omega ** 3


def alpha(comp: Component, T: float) -> float:
    return (1.0 + m_factor(comp.omega) * (1.0 - math.sqrt(T / comp.Tc))) ** 2


def a_b(comp: Component, R: float):
    """a_i = Omega_a R^2 Tc^2 / pc and b_i = Omega_b R Tc / pc."""
    return OMEGA_A * R * R * comp.Tc ** 2 / comp.pc, OMEGA_B * R * comp.Tc / comp.pc


def pressure(comps, kij, T, R, nmol):
    """Mixture PR pressure (Eq. MCPengRobinson) from the component molar densities nmol."""
    nt = sum(nmol)
    c = [ni / nt for ni in nmol]
    aa = [a_b(k, R)[0] * alpha(k, T) for k in comps]
    bb = [a_b(k, R)[1] for k in comps]
    nc = len(comps)
    am = sum(c[i] * c[j] * math.sqrt(aa[i] * aa[j]) * (1.0 - kij[i][j])
             for i in range(nc) for j in range(nc))
    bm = sum(c[i] * bb[i] for i in range(nc))
    return nt * R * T / (1.0 - bm * nt) - am * nt * nt / (1.0 + 2 * bm * nt - bm * bm * nt * nt)


def coefficients(comps, kij, T, p, c):
    """A_i, B_i, A_ij, A, B of Eq. cubiccoeff for composition c."""
    nc = len(comps)
    Ai = [OMEGA_A * alpha(k, T) * (p / k.pc) / (T / k.Tc) ** 2 for k in comps]
    Bi = [OMEGA_B * (p / k.pc) / (T / k.Tc) for k in comps]
    Aij = [[math.sqrt(Ai[i] * Ai[j]) * (1.0 - kij[i][j]) for j in range(nc)] for i in range(nc)]
    A = sum(c[i] * c[j] * Aij[i][j] for i in range(nc) for j in range(nc))
    B = sum(c[i] * Bi[i] for i in range(nc))
    return Ai, Bi, Aij, A, B


def z_roots(A: float, B: float):
    """Real roots above B of Z^3 - (1-B) Z^2 + (A - 3B^2 - 2B) Z - (AB - B^2 - B^3) = 0,
    ascending, each polished by Newton steps on the cubic."""
    coef = [1.0, -(1.0 - B), A - 3 * B * B - 2 * B, -(A * B - B * B - B ** 3)]
    out = []
    for r in np.roots(coef):
        if abs(r.imag) > 1e-7 * max(1.0, abs(r.real)):
            continue
        z = float(r.real)
        for _ in range(3):
            f = ((z + coef[1]) * z + coef[2]) * z + coef[3]
            d = (3 * z + 2 * coef[1]) * z + coef[2]
            if d != 0:
                z -= f / d
        if z > B:
            out.append(z)
    return sorted(out)


def gibbs_dG(zmin: float, zmax: float, A: float, B: float) -> float:
    """dG/RT of Eq. solutionselection (G at Z_max minus G at Z_min)."""
    return ((zmax - zmin) + math.log((zmin - B) / (zmax - B))
            + A / (2 * SQ2 * B) * math.log(((zmin + (1 + SQ2) * B) * (zmax + (1 - SQ2) * B))
                                            / ((zmin + (1 - SQ2) * B) * (zmax + (1 + SQ2) * B))))


def select_root(roots, A, B) -> float:
    if len(roots) == 1:
        return roots[0]
    zmin, zmax = roots[0], roots[-1]
    return zmin if gibbs_dG(zmin, zmax, A, B) > 0 else zmax


def ln_phi(Z, A, B, Aij, Bi, c):
    """ln phi_i of Eq. fugacitycoeff2."""
    nc = len(c)
    out = []
    lg = math.log((Z + (1 - SQ2) * B) / (Z + (1 + SQ2) * B))
    for i in range(nc):
        s = sum(Aij[i][j] * c[j] for j in range(nc))
        out.append(-math.log(Z - B) + Bi[i] / B * (Z - 1)
                   + A / (2 * SQ2 * B) * (2 * s / A - Bi[i] / B) * lg)
    return out


def phase_state(comps, kij, T, p, c, which=None):
    """Z and ln phi of a phase of composition c at (T, p). which = 'l' / 'v' forces the
    smallest / largest root; None applies Eq. solutionselection."""
    _, Bi, Aij, A, B = coefficients(comps, kij, T, p, c)
    roots = z_roots(A, B)
    if which == "l":
        Z = roots[0]
    elif which == "v":
        Z = roots[-1]
    else:
        Z = select_root(roots, A, B)
    return Z, ln_phi(Z, A, B, Aij, Bi, c)


def fugacities(comps, kij, T, p, c, which=None):
    """f_i = phi_i c_i p (Eq. fugacity)."""
    Z, lp = phase_state(comps, kij, T, p, c, which)
    return [math.exp(l) * ci * p for l, ci in zip(lp, c)], Z


def iso_fugacity_residual(fl, fv) -> float:
    """Eq. error: sum_i (f_li / f_vi - 1)^2."""
    return sum((a / b - 1.0) ** 2 for a, b in zip(fl, fv))


def wilson_k(comps, T, p):
    return [k.pc / p * math.exp(5.373 * (1 + k.omega) * (1 - k.Tc / T)) for k in comps]


def rachford_rice(z, K):
    """Vapour mole fraction V solving sum z_i (K_i - 1) / (1 + V (K_i - 1)) = 0 by bisection on
    the interval between the poles (negative flash: V may leave [0, 1])."""
    kmax, kmin = max(K), min(K)
    if kmax <= 1.0 or kmin >= 1.0:
        return None
    lo = 1.0 / (1.0 - kmax)
    hi = 1.0 / (1.0 - kmin)

    def g(V):
        return sum(zi * (Ki - 1) / (1 + V * (Ki - 1)) for zi, Ki in zip(z, K))

    for _ in range(400):
        mid = 0.5 * (lo + hi)
        if mid == lo or mid == hi:
            break
        if g(mid) > 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


@dataclass
class FlashResult:
    V: float
    x: list
    y: list
    Zl: float
    Zv: float
    K: list
    residual: float
    iterations: int
    trivial: bool
    extra: dict = field(default_factory=dict)


def flash(comps, kij, T, p, z, K0=None, tol=1e-13, maxit=20000) -> FlashResult:
    """Two-phase flash at (T, p, z) by successive substitution on K_i = phi_li / phi_vi."""
    K = list(K0) if K0 is not None else wilson_k(comps, T, p)
    V = None
    x = y = list(z)
    Zl = Zv = float("nan")
    it = 0
    for it in range(1, maxit + 1):
        V = rachford_rice(z, K)
        if V is None:
            break
        x = [zi / (1 + V * (Ki - 1)) for zi, Ki in zip(z, K)]
        y = [Ki * xi for Ki, xi in zip(K, x)]
        sx, sy = sum(x), sum(y)
        x = [v / sx for v in x]
        y = [v / sy for v in y]
        Zl, lpl = phase_state(comps, kij, T, p, x)
        Zv, lpv = phase_state(comps, kij, T, p, y)
        Knew = [math.exp(a - b) for a, b in zip(lpl, lpv)]
        step = max(abs(math.log(a / b)) for a, b in zip(Knew, K))
        K = Knew
        if step < tol:
            break
    trivial = V is None or max(abs(math.log(k)) for k in K) < 1e-4
    res = float("nan")
    if not trivial:
        fl, _ = fugacities(comps, kij, T, p, x)
        fv, _ = fugacities(comps, kij, T, p, y)
        res = iso_fugacity_residual(fl, fv)
    return FlashResult(V if V is not None else float("nan"), x, y, Zl, Zv, K, res, it, trivial)


def phase_partial_densities(comps, T, p, R, fr: FlashResult):
    """Cell-volume densities of each component in each phase (Section 2.2 relations):
    rho_il = n_l x_i M_i, rho_iv = n_v y_i M_i with n = p / (Z R T)."""
    nl = p / (fr.Zl * R * T)
    nv = p / (fr.Zv * R * T)
    rl = [nl * xi * k.M for xi, k in zip(fr.x, comps)]
    rv = [nv * yi * k.M for yi, k in zip(fr.y, comps)]
    return rl, rv, nl, nv


def gamma_coefficients(rho_l, rho_v, K):
    """Volatility coefficients of Eq. gamma, normalised so that the least volatile
    component (smallest K) has gamma = 1."""
    h = int(np.argmin(K))
    den = math.log(rho_l[h] / rho_v[h])
    return [math.log(a / b) / den for a, b in zip(rho_l, rho_v)], h


def pure_saturation(comp: Component, T: float, R: float = 1.0):
    """Saturation pressure and molar densities of a pure PR fluid at T from equal fugacity
    of the smallest and largest cubic roots (the Maxwell rule). Returns (p, n_l, n_v)."""
    kij = [[0.0]]

    def h(p):
        _, Bi, Aij, A, B = coefficients([comp], kij, T, p, [1.0])
        r = z_roots(A, B)
        if len(r) < 3:
            return None
        zl, zv = r[0], r[-1]
        return ln_phi(zl, A, B, Aij, Bi, [1.0])[0] - ln_phi(zv, A, B, Aij, Bi, [1.0])[0], zl, zv

    ps = np.geomspace(1e-4 * comp.pc, comp.pc, 4000)
    vals = [(p, h(p)) for p in ps]
    br = None
    for (p0, h0), (p1, h1) in zip(vals, vals[1:]):
        if h0 is not None and h1 is not None and h0[0] * h1[0] <= 0:
            br = (p0, p1)
            break
    if br is None:
        raise ValueError("no saturation bracket")
    lo, hi = br
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        hm = h(mid)
        hl = h(lo)
        if hm is None or hl is None:
            break
        if hl[0] * hm[0] <= 0:
            hi = mid
        else:
            lo = mid
    p = 0.5 * (lo + hi)
    _, zl, zv = h(p)
    return p, p / (zl * R * T), p / (zv * R * T)


def lattice_components(phys):
    """Scale physical components to lattice units (a_1 = 2/49, b_1 = 2/21, M_1 = 1, R = 1).
    Returns (components in lattice units, T scale, p scale) with T_LB = T_phys * T scale."""
    Tc1 = (OMEGA_B / OMEGA_A) * (A1_LB / B1_LB)
    pc1 = OMEGA_B * Tc1 / B1_LB
    ts = Tc1 / phys[0].Tc
    ps = pc1 / phys[0].pc
    out = [Component(k.name, k.Tc * ts, k.pc * ps, k.omega, k.M / phys[0].M) for k in phys]
    return out, ts, ps


def liquid_volume_fraction(fr: FlashResult, nl: float, nv: float) -> float:
    V = min(max(fr.V, 0.0), 1.0)
    vl = (1 - V) / nl
    vv = V / nv
    return vl / (vl + vv)


def pressure_for_liquid_fraction(comps, kij, T, z, target, R=1.0, npts=120):
    """Pressure inside the two-phase window at which the flash's liquid volume fraction
    equals `target`, found by a scan followed by bisection. Returns (p, FlashResult)."""
    pmax = 1.5 * max(k.pc for k in comps)
    pmin = 1e-3 * min(k.pc for k in comps)
    ps = np.geomspace(pmin, pmax, npts)

    def frac(p, K0=None):
        fr = flash(comps, kij, T, p, z, K0=K0)
        if fr.trivial:
            return None, fr
        if fr.V >= 1.0:
            return 0.0, fr
        if fr.V <= 0.0:
            return 1.0, fr
        _, _, nl, nv = phase_partial_densities(comps, T, p, R, fr)
        return liquid_volume_fraction(fr, nl, nv), fr

    prev = None
    br = None
    for p in ps:
        fv, fr = frac(p)
        if fv is None:
            prev = None
            continue
        if prev is not None and (prev[1] - target) * (fv - target) <= 0:
            br = (prev[0], p, fr.K)
            break
        prev = (p, fv)
    if br is None:
        raise ValueError("no two-phase window reaches the target liquid fraction")
    lo, hi, K = br
    flo = frac(lo)[0]
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        fm, fr = frac(mid, K)
        if fm is None:
            fm, fr = frac(mid)
        if fm is None:
            raise ValueError("flash collapsed inside the bracket")
        K = fr.K
        if (flo - target) * (fm - target) <= 0:
            hi = mid
        else:
            lo, flo = mid, fm
        if hi - lo < 1e-14 * hi:
            break
    p = 0.5 * (lo + hi)
    fr = flash(comps, kij, T, p, z, K0=K)
    return p, fr
