"""Pins of the oracle's forward-mode derivative (oracle_step_dual, the Dual type) and of its
split factors, against what the mathematics fixes rather than against the oracle itself:

* the dual-number derivative of a run equals central finite differences of the plain FP64
  step (oracle.step), for the binary interaction coefficient zeta_12 (Eq. randommixingrule),
  the split-factor scale s (gamma_i -> s gamma_i, Eq. distributionforce) and a perturbation
  of the initial populations, with BGK and MRT collisions (D2Q9, and D3Q19 with MRT);
* the two derivative directions are independent: swapping the seeds swaps the results
  bit for bit, and a seed scaled by two gives exactly twice the derivative;
* with identical components the total density obeys the single-fluid LBE whatever the split
  (Section 4.1), so its derivative with respect to s is zero, while each component's is not;
* the split factor the step applies, read back from the component momenta after one step
  through the first moment of the Guo term (sum_a e_a Fbar_a = F_s), equals chi_i of
  Eq. distributionforce, and that of Eq. Gong: the molar composition when the components
  differ only in molar mass, and c_i sqrt(|n R T - p_i(n)|) normalised, with p_i(n) the
  pure-component pressure taken from the oracle's EOS (itself pinned to Table 2)."""
import numpy as np
import pytest

import lbm_inputs
import oracle
from conftest import read_table
from oracle import thermo as th


def _case(c, shape, **kw):
    comps = c["components"]
    args = dict(Q=9, shape=tuple(shape), Tc=[d["Tc"] for d in comps], pc=[d["pc"] for d in comps],
                omega=[d["omega"] for d in comps], M=[d["M"] for d in comps], T=c["T"], tau=c["tau"],
                gamma=list(c["gamma"]), kij=[row[:] for row in c["kij"]], beta=c["beta"], G=c["G"])
    args.update(kw)
    return oracle.Case(**args)


def _droplet(case, c, radius=2.6, width=2.0):
    rho = lbm_inputs.ball_fields(case.grid, c["rho_l"], c["rho_v"], radius, width,
                                 center=[g / 2 - 0.3 for g in case.grid])
    return oracle.equilibrium(case, rho)


def _with(case, kij=None, gamma=None):
    kw = dict(case.__dict__)
    if kij is not None:
        kw["kij"] = kij
    if gamma is not None:
        kw["gamma"] = gamma
    return oracle.Case(**kw)


def _seeds(nc, h_idx, gamma0):
    """Direction 0: d/dzeta_12 (both symmetric entries); direction 1: d/ds with
    gamma_i = s gamma0_i for i != h."""
    dk = np.zeros((2, nc, nc))
    dk[0, 0, 1] = dk[0, 1, 0] = 1.0
    dg = np.zeros((2, nc))
    for i in range(nc):
        if i != h_idx:
            dg[1, i] = gamma0[i]
    return dk, dg


MRT9 = [1.25, 1.0, 1.0, 1.25, 1.2, 1.25, 1.2, 1.25, 1.25]


@pytest.mark.parametrize("collision", [0, 1])
def test_dual_derivatives_equal_central_differences(cases, collision):
    c = cases["c5"]
    k12, steps, h = 0.01, 12, 1e-6
    base = _case(c, (8, 8), collision=collision, s=MRT9 if collision else None,
                 kij=[[0.0, k12], [k12, 0.0]])
    f0 = _droplet(base, c)
    g0 = np.array(c["gamma"], dtype=float)
    hv = int(c["least_volatile"])
    dk, dg = _seeds(2, hv, g0)
    f, df = oracle.step_dual(base, f0, np.zeros((2,) + f0.shape), dk, dg, steps)
    assert np.array_equal(f, oracle.step(base, f0, steps))  # values are the plain step's

    def run_zeta(z):
        return oracle.step(_with(base, kij=[[0.0, z], [z, 0.0]]), f0, steps)

    def run_s(s):
        g = g0.copy()
        g[np.arange(2) != hv] *= s
        return oracle.step(_with(base, gamma=list(g)), f0, steps)

    fd = [(run_zeta(k12 + h) - run_zeta(k12 - h)) / (2 * h), (run_s(1 + h) - run_s(1 - h)) / (2 * h)]
    for d in range(2):
        scale = np.max(np.abs(df[d]))
        assert scale > 1e-6  # the derivative is not trivially zero
        err = np.max(np.abs(df[d] - fd[d])) / scale
        assert err < 1e-6, (d, err)


def test_dual_derivatives_equal_central_differences_d3q19_mrt(cases):
    """The same pin on D3Q19 with the MRT collision and three components (the sphere
    workload's mixture and rates) on a 4 x 4 x 4 grid. Here d f / d zeta_12 is about 2e-4 of
    the populations, so h = 1e-6 leaves the difference to rounding (2.8e-6 relative, falling as
    1 / h); h = 1e-4 gives 3e-8."""
    c = cases["c3"]
    nc = len(c["gamma"])
    k12, steps, h = 0.01, 6, 1e-4
    kij = np.zeros((nc, nc))
    kij[0, 1] = kij[1, 0] = k12
    base = _case(c, (4, 4, 4), Q=19, collision=1, s=list(c["mrt_s"]), kij=kij.tolist())
    f0 = _droplet(base, c, radius=1.4, width=1.5)
    g0 = np.array(c["gamma"], dtype=float)
    hv = int(c["least_volatile"])
    dk, dg = _seeds(nc, hv, g0)
    f, df = oracle.step_dual(base, f0, np.zeros((2,) + f0.shape), dk, dg, steps)
    assert np.array_equal(f, oracle.step(base, f0, steps))

    def run_zeta(z):
        k = kij.copy()
        k[0, 1] = k[1, 0] = z
        return oracle.step(_with(base, kij=k.tolist()), f0, steps)

    def run_s(s):
        g = g0.copy()
        g[np.arange(nc) != hv] *= s
        return oracle.step(_with(base, gamma=list(g)), f0, steps)

    fd = [(run_zeta(k12 + h) - run_zeta(k12 - h)) / (2 * h), (run_s(1 + h) - run_s(1 - h)) / (2 * h)]
    for d in range(2):
        scale = np.max(np.abs(df[d]))
        assert scale > 1e-8
        err = np.max(np.abs(df[d] - fd[d])) / scale
        assert err < 1e-6, (d, err)


def test_dual_derivative_along_an_initial_state_direction(cases):
    """J v for a perturbation v of the initial populations, against central differences."""
    c = cases["c5"]
    steps, h = 8, 1e-6
    base = _case(c, (8, 8))
    f0 = _droplet(base, c)
    v = (lbm_inputs.uniform01(77, f0.size).reshape(f0.shape) - 0.5) * np.abs(f0)
    df0 = np.zeros((2,) + f0.shape)
    df0[0] = v
    df0[1] = -2.0 * v
    zero_k, zero_g = np.zeros((2, 2, 2)), np.zeros((2, 2))
    _, df = oracle.step_dual(base, f0, df0, zero_k, zero_g, steps)
    fd = (oracle.step(base, f0 + h * v, steps) - oracle.step(base, f0 - h * v, steps)) / (2 * h)
    scale = np.max(np.abs(fd))
    assert np.max(np.abs(df[0] - fd)) < 1e-6 * scale
    assert np.array_equal(df[1], -2.0 * df[0])  # a seed scaled by -2 (exact) scales the result


def test_dual_directions_do_not_mix(cases):
    c = cases["c5"]
    base = _case(c, (8, 8), kij=[[0.0, 0.01], [0.01, 0.0]])
    f0 = _droplet(base, c)
    g0 = np.array(c["gamma"], dtype=float)
    dk, dg = _seeds(2, int(c["least_volatile"]), g0)
    z = np.zeros((2,) + f0.shape)
    _, a = oracle.step_dual(base, f0, z, dk, dg, 6)
    _, b = oracle.step_dual(base, f0, z, dk[::-1].copy(), dg[::-1].copy(), 6)
    assert np.array_equal(a[0], b[1]) and np.array_equal(a[1], b[0])
    dk2 = dk.copy()
    dk2[1] = 2.0 * dk[0]
    dg2 = np.zeros_like(dg)
    _, d = oracle.step_dual(base, f0, z, dk2, dg2, 6)
    assert np.array_equal(d[1], 2.0 * a[0])


@pytest.mark.parametrize("collision", [0, 1])
def test_identical_components_total_density_has_zero_split_derivative(collision):
    """Section 4.1: with one tau and identical components, sum_s of the LBE is the
    single-component LBE and the EOS depends on the total only, so the total density does not
    depend on gamma: d(rho_1 + rho_2)/ds = 0 up to rounding, while d rho_1/ds is O(1)."""
    comps = {r[0]: th.Component(r[0], r[2], r[1], r[3], r[4]) for r in read_table("table1_components.txt")}
    lb, _, _ = th.lattice_components([comps["C3"], comps["C3"]])
    T = 0.9 * lb[0].Tc
    case = oracle.Case(Q=9, shape=(10, 8), Tc=[k.Tc for k in lb], pc=[k.pc for k in lb],
                       omega=[k.omega for k in lb], M=[k.M for k in lb], T=T, tau=0.8,
                       gamma=[0.4, 1.0], beta=1.5, G=-1.0, collision=collision,
                       s=MRT9 if collision else None)
    grid = case.grid
    u = lbm_inputs.uniform01(5, 2 * int(np.prod(grid))).reshape((2,) + grid)
    rho = 0.5 + 3.0 * u
    f0 = oracle.equilibrium(case, rho)
    dk, dg = _seeds(2, 1, [0.4, 1.0])
    f, df = oracle.step_dual(case, f0, np.zeros((2,) + f0.shape), dk, dg, 10)
    drho = df.sum(axis=2)  # (direction, component, *grid)
    tot = drho[1, 0] + drho[1, 1]
    comp = np.max(np.abs(drho[1, 0]))
    assert comp > 1e-4
    assert np.max(np.abs(tot)) < 1e-12 * comp
    # zeta_12 changes the mixing rule: its derivative of the total is not zero
    assert np.max(np.abs(drho[0, 0] + drho[0, 1])) > 1e-6


# ---------------------------------------------------------------------------------------------
# the split factor as applied by the step

def _applied_split(case, f0):
    """chi_s(x) read back from one BGK step started at rest: the component momentum after the
    collision is J*_s = (1 - 1/tau) j_s + rho_s u / tau + (1 - 1/(2 tau)) chi_s F (the first
    moments of f_eq and of the Guo term are rho_s u and F_s), and streaming moves
    f*_a(x) to x + e_a, so J*_s(x) = sum_a e_a f_new[s, a, x + e_a]."""
    fl = oracle.fields(case, f0)
    f1 = oracle.step(case, f0, 1)
    _, e, _ = oracle.lattice(case.Q)
    nc, tau = case.nc, case.tau
    D = case.D
    J = np.zeros((nc, D) + case.grid)
    for s in range(nc):
        for a in range(case.Q):
            g = f1[s, a]
            for d in range(D):
                g = np.roll(g, -int(e[a][d]), axis=len(case.grid) - 1 - d)
            for d in range(D):
                J[s, d] += e[a][d] * g
    F = fl.F[:D]
    d = np.argmax(np.abs(F), axis=0)  # per site, the force component with the largest magnitude
    Fd = np.take_along_axis(F, d[None], 0)[0]
    mask = np.abs(Fd) > 1e-3 * np.max(np.abs(Fd))
    chi = np.zeros((nc,) + case.grid)
    for s in range(nc):
        Js = np.take_along_axis(J[s], d[None], 0)[0]
        ud = np.take_along_axis(fl.u[:D], d[None], 0)[0]
        chi[s] = (Js - fl.rho[s] * ud / tau) / ((1 - 0.5 / tau) * np.where(mask, Fd, 1.0))
    return chi, fl, mask


def _rand_state(case, seed):
    u = lbm_inputs.uniform01(seed, case.nc * case.nsites).reshape((case.nc,) + case.grid)
    return oracle.equilibrium(case, 0.5 + 4.0 * u)


def test_applied_split_is_eq_distributionforce(cases):
    c = cases["c5"]
    case = _case(c, (12, 10), tau=0.8, gamma=[0.3, 1.0])
    f0 = _rand_state(case, 3)
    chi, fl, mask = _applied_split(case, f0)
    g = np.array([0.3, 1.0]).reshape(2, 1, 1)
    want = g * fl.rho / np.sum(g * fl.rho, axis=0)
    assert mask.sum() > 50
    assert np.max(np.abs(chi - want)[:, mask]) < 1e-9


def _table1():
    return {r[0]: th.Component(r[0], r[2], r[1], r[3], r[4]) for r in read_table("table1_components.txt")}


def test_gong_split_weights_are_molar():
    """Two components with the same critical constants and acentric factor but different molar
    masses have the same molar EOS, so the pure-component pressures of Eq. Gong are equal and
    chi_i is the molar composition (rho_i / M_i) / sum_j (rho_j / M_j), not the mass fraction."""
    lb, _, _ = th.lattice_components([_table1()["C3"]])
    k = lb[0]
    case = oracle.Case(Q=9, shape=(12, 10), Tc=[k.Tc, k.Tc], pc=[k.pc, k.pc], omega=[k.omega, k.omega],
                       M=[1.0, 2.5], T=0.9 * k.Tc, tau=0.8, gamma=[1.0, 1.0], beta=1.5, G=-1.0, split=1)
    f0 = _rand_state(case, 4)
    chi, fl, mask = _applied_split(case, f0)
    n = fl.rho / np.array([1.0, 2.5]).reshape(2, 1, 1)
    want = n / n.sum(axis=0)
    mass_frac = fl.rho / fl.rho.sum(axis=0)
    assert mask.sum() > 50
    assert np.max(np.abs(chi - want)[:, mask]) < 1e-9
    assert np.max(np.abs(chi - mass_frac)[:, mask]) > 1e-2


def test_gong_split_uses_pure_component_pressures_at_the_mixture_density():
    """Eq. Gong for C3 / nC5 with unequal molar masses: chi_i proportional to
    c_i sqrt(|n R T - p_i(n)|), p_i(n) the Peng-Robinson pressure of pure i at the mixture's
    molar density, taken here from the oracle's single-component EOS (Table 2 pins it)."""
    t1 = _table1()
    lb, _, _ = th.lattice_components([t1["C3"], t1["nC5"]])
    T = 0.9 * lb[0].Tc
    kw = dict(Q=9, shape=(12, 10), Tc=[k.Tc for k in lb], pc=[k.pc for k in lb],
              omega=[k.omega for k in lb], M=[k.M for k in lb], T=T, tau=0.8, gamma=[1.0, 1.0],
              beta=1.5, G=-1.0)
    assert abs(lb[1].M / lb[0].M - 1) > 0.3
    case = oracle.Case(**kw, split=1)
    f0 = _rand_state(case, 6)
    chi, fl, mask = _applied_split(case, f0)
    M = np.array([k.M for k in lb])
    nmol = fl.rho / M.reshape(2, 1, 1)
    n = nmol.sum(axis=0)
    pure = [oracle.Case(Q=9, shape=(1, 1), Tc=[k.Tc], pc=[k.pc], omega=[k.omega], M=[k.M], T=T,
                        tau=0.8, gamma=[1.0]) for k in lb]
    w = np.zeros_like(fl.rho)
    for i in range(2):
        p_i = np.vectorize(lambda nn: oracle.eos(pure[i], [nn * M[i]])[0])(n)
        w[i] = nmol[i] / n * np.sqrt(np.abs(n * T - p_i))
    want = w / w.sum(axis=0)
    assert mask.sum() > 50
    assert np.max(np.abs(chi - want)[:, mask]) < 1e-9
