"""Seeded synthetic initial fields for the two-component Shan-Chen workloads.

This module only builds input density fields n_A(x), n_B(x) (host FP64 arrays,
x fastest, shape [nz, ny, nx]); it holds none of the lattice Boltzmann
arithmetic.  The CUDA library and the CPU oracle both consume its output.

* droplet: the tanh radial profile of the paper's initial condition
  (section 4, "n_J(r, R) = ...") around a centre node, minimum-image radius;
* slab: the paper's flat-strip initial condition (section 4), evaluated as
  printed -- it puts the value called "l" inside the strip, so an A-rich band
  passes the rich value as ``n_inside``;
* noise: independent uniform noise in [-a, a] per component and per site from
  a counter-based generator (SplitMix64 of a 64-bit counter built from the
  seed, the component and the site index; top 53 bits -> [0, 1)).
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 20211206

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea and Flood, OOPSLA 2014) on uint64 arrays."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, comp: int, n: int) -> np.ndarray:
    """n draws in [0, 1) for component ``comp``: counter = seed<<32 ^ comp<<62 ^ site."""
    site = np.arange(n, dtype=np.uint64)
    ctr = (np.uint64(seed) << np.uint64(32)) ^ (np.uint64(comp) << np.uint64(62)) ^ site
    return (splitmix64(ctr) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def noise(shape, amplitude: float, seed: int, comp: int) -> np.ndarray:
    """Uniform noise in [-amplitude, amplitude] on a [nz, ny, nx] lattice."""
    n = int(np.prod(shape))
    return (amplitude * (2.0 * uniform01(seed, comp, n) - 1.0)).reshape(shape)


def min_image_radius(shape, centre) -> np.ndarray:
    """Distance of every node from ``centre`` (x, y, z) with periodic minimum image."""
    nz, ny, nx = shape
    out = np.zeros(shape)
    for axis, (L, c) in enumerate(zip((nx, ny, nz), centre)):
        d = np.arange(L, dtype=np.float64) - c
        d -= L * np.floor(d / L + 0.5)
        sh = [1, 1, 1]
        sh[2 - axis] = L
        out = out + (d.reshape(sh)) ** 2
    return np.sqrt(out)


def droplet(shape, centre, radius: float, n_in: float = 0.95, n_out: float = 0.05, amplitude: float = 1e-3,
            seed: int = DEFAULT_SEED, a_rich: bool = True):
    """(n_A, n_B) for a droplet of radius ``radius``; shape = (nz, ny, nx).

    n_J(r) = (in + out)/2 - (in - out)/2 tanh(r - R); the A-rich droplet has
    (in, out) = (n_in, n_out) for A and the complement for B (swapped when
    ``a_rich`` is False).  Noise is added after the profile."""
    r = min_image_radius(shape, centre)
    prof = lambda a, b: 0.5 * (a + b) - 0.5 * (a - b) * np.tanh(r - radius)
    rich, poor = prof(n_in, n_out), prof(n_out, n_in)
    nA, nB = (rich, poor) if a_rich else (poor, rich)
    if amplitude:
        nA = nA + noise(shape, amplitude, seed, 0)
        nB = nB + noise(shape, amplitude, seed, 1)
    return np.ascontiguousarray(nA), np.ascontiguousarray(nB)


def droplet_ab(shape, centre, radius: float, a_in: float, a_out: float, b_in: float, b_out: float,
               amplitude: float = 1e-3, seed: int = DEFAULT_SEED):
    """(n_A, n_B) of a droplet with separate inner and outer densities per component (section 4: the
    values of a flat-interface run); shape = (nz, ny, nx); tanh profile of unit width plus noise."""
    r = min_image_radius(shape, centre)
    prof = lambda a, b: 0.5 * (a + b) - 0.5 * (a - b) * np.tanh(r - radius)
    nA, nB = prof(a_in, a_out), prof(b_in, b_out)
    if amplitude:
        nA = nA + noise(shape, amplitude, seed, 0)
        nB = nB + noise(shape, amplitude, seed, 1)
    return np.ascontiguousarray(nA), np.ascontiguousarray(nB)


def strip_profile(coord: np.ndarray, x0: float, width: float, n_outside: float, n_inside: float) -> np.ndarray:
    """The paper's three-tanh flat-strip profile, as printed, with n_h = n_outside and n_l = n_inside."""
    h, l = n_outside, n_inside
    return (0.5 * (h + l) - 0.5 * (h - l) * np.tanh(coord - (x0 - 0.5 * width))
            + 0.5 * (h - l) * (np.tanh(coord - (x0 + 0.5 * width)) + 1.0))


def slab(shape, width: float, n_rich: float = 0.95, n_poor: float = 0.05, amplitude: float = 0.0,
         seed: int = DEFAULT_SEED, axis: str = "z"):
    """(n_A, n_B) for an A-rich band of ``width`` centred in the box along ``axis``."""
    nz, ny, nx = shape
    L = {"x": nx, "y": ny, "z": nz}[axis]
    c = np.arange(L, dtype=np.float64)
    pa = strip_profile(c, 0.5 * L, width, n_outside=n_poor, n_inside=n_rich)
    pb = strip_profile(c, 0.5 * L, width, n_outside=n_rich, n_inside=n_poor)
    sh = {"x": (1, 1, L), "y": (1, L, 1), "z": (L, 1, 1)}[axis]
    nA = np.broadcast_to(pa.reshape(sh), shape).astype(np.float64)
    nB = np.broadcast_to(pb.reshape(sh), shape).astype(np.float64)
    if amplitude:
        nA = nA + noise(shape, amplitude, seed, 0)
        nB = nB + noise(shape, amplitude, seed, 1)
    return np.ascontiguousarray(nA), np.ascontiguousarray(nB)


def uniform(shape, nA: float, nB: float):
    """A uniform mixture."""
    return np.full(shape, float(nA)), np.full(shape, float(nB))
