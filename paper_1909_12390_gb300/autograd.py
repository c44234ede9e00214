"""torch.autograd.Function around lbm_record / lbm_adjoint (argument marshalling only).

LatticeRun.apply(zeta, s, spec) runs the lattice described by `spec` for spec["steps"] steps
with the binary interaction coefficient of the pair spec["pair"] set to `zeta` and the
volatility coefficients gamma_i (i != least volatile) scaled by `s`, and returns the final
cell-volume densities (nc, *grid) as a float64 CPU tensor. Its backward runs the library's
hand-written adjoint with checkpoints every spec["checkpoint_every"] steps and returns dL/dzeta
and dL/ds.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbm


def _gamma(spec, s):
    g = np.array(spec["gamma"], dtype=float)
    h = int(np.argmax(g == 1.0)) if "least_volatile" not in spec else int(spec["least_volatile"])
    scale = np.full(len(g), float(s))
    scale[h] = 1.0
    return g * scale, h


def _kij(spec, zeta):
    k = np.array(spec.get("kij", np.zeros((len(spec["components"]),) * 2)), dtype=float).copy()
    i, j = spec.get("pair", (0, 1))
    k[i, j] = k[j, i] = float(zeta)
    return k


class LatticeRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, zeta, s, spec):
        g, h = _gamma(spec, s.item())
        lat = lbm.Lattice(tuple(spec["shape"]), spec["components"], T=spec["T"], tau=spec["tau"], gamma=g,
                          kij=_kij(spec, zeta.item()), beta=spec["beta"], G=spec.get("G", -1.0),
                          precision=spec.get("precision", lbm.FP32_SHIFTED))
        lat.init(spec["rho0"])
        lat.record(spec["steps"], spec.get("checkpoint_every", 55))
        rho = lat.fields(u=False, p=False, psi=False)["rho"]
        ctx.lat = lat
        ctx.gamma = g
        ctx.h = h
        ctx.pair = spec.get("pair", (0, 1))
        return torch.from_numpy(rho)

    @staticmethod
    def backward(ctx, grad_rho):
        dk, dg, _ = ctx.lat.adjoint(grad_rho.detach().cpu().numpy())
        i, j = ctx.pair
        dzeta = dk[i, j] + dk[j, i]
        ds = sum(dg[k] * ctx.gamma[k] for k in range(len(dg)) if k != ctx.h) / 1.0
        ctx.lat.close()
        return (torch.tensor(dzeta, dtype=torch.float64), torch.tensor(ds, dtype=torch.float64), None)
