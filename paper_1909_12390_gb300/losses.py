"""Loss of the adjoint workload, as torch operations on the densities LatticeRun returns.

The workload differentiates the bulk-phase compositions and the density profile of a droplet
with respect to the binary interaction coefficient and the split-factor scale (Sections 4.2
and 4.3 measure both; the loss itself is the workload's choice):

    L = sum_i (x_i - x_i^T)^2 + sum_i (y_i - y_i^T)^2 + mean_x (rho(x) - rho^T(x))^2,

x and y the molar compositions of the mean bulk liquid and vapour partial densities, rho the
total density, ^T the same quantities of a target state. Bulk cells lie farther than `erode`
cells (L-infinity, periodic) from the (max + min) / 2 contour of the total density; the masks
are piecewise constant in the densities and are taken as fixed (no gradient flows through
them). Host-side and cheap: the lattice work is in LatticeRun's forward and adjoint passes.
"""
from __future__ import annotations

import torch


def bulk_masks(rho: torch.Tensor, erode: int = 8):
    """(liquid, vapour) bulk masks of densities rho (nc, *grid)."""
    with torch.no_grad():
        tot = rho.sum(0)
        liq = tot > 0.5 * (tot.max() + tot.min())
        all_l, any_l = liq.clone(), liq.clone()
        for axis in range(liq.dim()):
            a2 = torch.ones_like(all_l)
            b2 = torch.zeros_like(any_l)
            for d in range(-erode, erode + 1):
                a2 &= torch.roll(all_l, d, dims=axis)
                b2 |= torch.roll(any_l, d, dims=axis)
            all_l, any_l = a2, b2
    return all_l, ~any_l


def _composition(rho: torch.Tensor, mask: torch.Tensor, M: torch.Tensor) -> torch.Tensor:
    mean = torch.stack([rho[c][mask].mean() for c in range(rho.shape[0])])
    n = mean / M
    return n / n.sum()


def composition_profile_loss(rho: torch.Tensor, target: torch.Tensor, M, erode: int = 8) -> torch.Tensor:
    """L above for densities rho (nc, *grid) against target (same shape); M the molar masses."""
    M = torch.as_tensor(M, dtype=rho.dtype, device=rho.device)
    bl, bv = bulk_masks(rho.detach(), erode)
    tl, tv = bulk_masks(target, erode)
    x, y = _composition(rho, bl, M), _composition(rho, bv, M)
    with torch.no_grad():
        xT, yT = _composition(target, tl, M), _composition(target, tv, M)
    prof = ((rho.sum(0) - target.sum(0)) ** 2).mean()
    return ((x - xT) ** 2).sum() + ((y - yT) ** 2).sum() + prof
