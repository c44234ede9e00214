"""torch.autograd.Function around lbm_record / lbm_adjoint (argument marshalling only).

LatticeRun.apply(zeta, s, spec) runs the lattice described by `spec` for spec["steps"] steps
with the binary interaction coefficient of the pair spec["pair"] set to `zeta` and the
volatility coefficients gamma_i (i != least volatile) scaled by `s`, and returns the final
cell-volume densities (nc, *grid) as a float64 CPU tensor. Its backward runs the library's
hand-written adjoint with checkpoints every spec["checkpoint_every"] steps and returns dL/dzeta
and dL/ds. spec["collision"] (lbm.BGK, the default, or lbm.MRT with spec["mrt_rates"]) selects
the collision.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbm


def _gamma(spec, s):
    """(scaled gamma, unscaled gamma, least-volatile index h): gamma_i = s gamma0_i for i != h.
    h is spec["least_volatile"], else the one entry of gamma0 equal to 1 (Eq. gamma normalises
    the least volatile component's coefficient to 1)."""
    g0 = np.array(spec["gamma"], dtype=float)
    if "least_volatile" in spec:
        h = int(spec["least_volatile"])
    else:
        ones = np.flatnonzero(g0 == 1.0)
        if len(ones) != 1:
            raise ValueError("spec needs 'least_volatile': gamma has %d entries equal to 1" % len(ones))
        h = int(ones[0])
    scale = np.full(len(g0), float(s))
    scale[h] = 1.0
    return g0 * scale, g0, h


def _kij(spec, zeta):
    k = np.array(spec.get("kij", np.zeros((len(spec["components"]),) * 2)), dtype=float).copy()
    i, j = spec.get("pair", (0, 1))
    k[i, j] = k[j, i] = float(zeta)
    return k


class LatticeRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, zeta, s, spec):
        g, g0, h = _gamma(spec, s.item())
        lat = lbm.Lattice(tuple(spec["shape"]), spec["components"], T=spec["T"], tau=spec["tau"], gamma=g,
                          kij=_kij(spec, zeta.item()), beta=spec["beta"], G=spec.get("G", -1.0),
                          collision=spec.get("collision", lbm.BGK), mrt_rates=spec.get("mrt_rates"),
                          precision=spec.get("precision", lbm.FP32_SHIFTED))
        lat.init(spec["rho0"])
        lat.record(spec["steps"], spec.get("checkpoint_every", 55))
        rho = lat.fields(u=False, p=False, psi=False)["rho"]
        ctx.lat = lat
        ctx.gamma0 = g0
        ctx.h = h
        ctx.pair = spec.get("pair", (0, 1))
        return torch.from_numpy(rho)

    @staticmethod
    def backward(ctx, grad_rho):
        dk, dg, _ = ctx.lat.adjoint(grad_rho.detach().cpu().numpy())
        i, j = ctx.pair
        dzeta = dk[i, j] + dk[j, i]
        # gamma_k = s gamma0_k (k != h): dL/ds = sum_k dL/dgamma_k gamma0_k
        ds = sum(dg[k] * ctx.gamma0[k] for k in range(len(dg)) if k != ctx.h)
        ctx.lat.close()
        return (torch.tensor(dzeta, dtype=torch.float64), torch.tensor(ds, dtype=torch.float64), None)
