"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and bench.py.

This module holds no arithmetic of the lattice Boltzmann method itself: it only builds
initial component-density fields (tanh slabs, discs and spheres, as in the paper's Eqs.
initialden, initialdensity and initialdensity_droplet, with liquid inside), the
multiplicative site noise, and the per-case random draws of the batched flash sweep.
The phase densities that go into the profiles are arguments; they come from a flash
calculation, never from here.

Randomness is SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), used in counter form: output i of a generator seeded with s is
mix(s + (i + 1) * 0x9E3779B97F4A7C15), so every array is reproducible element by element.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

DEFAULT_SEED = 20191912


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+n-1 of SplitMix64 seeded with `seed`, as uint64."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits each."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


class Stream:
    """Sequential draws from one SplitMix64 counter stream."""

    def __init__(self, seed: int):
        self.seed = seed
        self.pos = 0

    def uniform(self, n: int = 1) -> np.ndarray:
        u = uniform01(self.seed, n, self.pos)
        self.pos += n
        return u


def _grid(shape):
    """Coordinate arrays (z, y, x) or (y, x) of the site centres, x fastest."""
    return np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")


def slab_profile(shape, axis: int, lo: float, hi: float, width: float,
                 rho_l: float, rho_v: float) -> np.ndarray:
    """Liquid between coordinates lo and hi along `axis` (periodic domain), tanh walls of
    thickness `width`: v + (l - v) * (tanh(2(s - lo)/W) - tanh(2(s - hi)/W)) / 2."""
    s = _grid(shape)[axis]
    prof = 0.5 * (np.tanh(2.0 * (s - lo) / width) - np.tanh(2.0 * (s - hi) / width))
    return rho_v + (rho_l - rho_v) * prof


def ball_profile(shape, center, radius: float, width: float,
                 rho_l: float, rho_v: float) -> np.ndarray:
    """Disc (2-D) or sphere (3-D) of liquid: (l + v)/2 - (l - v)/2 * tanh(2(r - R)/W)."""
    g = _grid(shape)
    r2 = sum((gi - ci) ** 2 for gi, ci in zip(g, center))
    r = np.sqrt(r2)
    return 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * np.tanh(2.0 * (r - radius) / width)


def multiplicative_noise(field: np.ndarray, amp: float, seed: int, offset: int = 0) -> np.ndarray:
    """field * (1 + amp * (2U - 1)), U drawn per element in C order."""
    u = uniform01(seed, field.size, offset).reshape(field.shape)
    return field * (1.0 + amp * (2.0 * u - 1.0))


def slab_fields(shape, rho_l, rho_v, lo, hi, width=4.0, noise=0.0, seed=DEFAULT_SEED,
                axis=0) -> np.ndarray:
    """Per-component slab fields, array (nc, *shape). Component k draws its noise from the
    counter range [k*N, (k+1)*N) of the seed's stream."""
    nc = len(rho_l)
    n = int(np.prod(shape))
    out = np.empty((nc,) + tuple(shape))
    for k in range(nc):
        f = slab_profile(shape, axis, lo, hi, width, rho_l[k], rho_v[k])
        if noise:
            f = multiplicative_noise(f, noise, seed, offset=k * n)
        out[k] = f
    return out


def ball_fields(shape, rho_l, rho_v, radius, width=4.0, center=None) -> np.ndarray:
    """Per-component droplet fields, array (nc, *shape), centred at shape/2 by default."""
    if center is None:
        center = [s / 2.0 for s in shape]
    return np.stack([ball_profile(shape, center, radius, width, rho_l[k], rho_v[k])
                     for k in range(len(rho_l))])


def droplet_radius(seed: int, lo: float = 40.0, hi: float = 120.0) -> float:
    """Radius drawn uniformly in [lo, hi) from the first output of the seed's stream."""
    return float(lo + (hi - lo) * uniform01(seed, 1)[0])


BATCH_LX_CHOICES = (64, 96, 128, 192, 256)


def batch_case_draws(n_cases: int, seed: int, accept=None):
    """Draw (Lx, T/T_pc, z_1) per case in the order Lx, T, z from one stream. `accept` is an
    optional predicate on a draw; rejected draws are redrawn from the same stream, so the
    sequence is deterministic under the seed."""
    st = Stream(seed)
    out = []
    while len(out) < n_cases:
        u = st.uniform(3)
        lx = BATCH_LX_CHOICES[min(int(u[0] * len(BATCH_LX_CHOICES)), len(BATCH_LX_CHOICES) - 1)]
        tfrac = 0.75 + 0.20 * u[1]
        z1 = 0.1 + 0.5 * u[2]
        d = (lx, float(tfrac), float(z1))
        if accept is None or accept(d):
            out.append(d)
    return out
