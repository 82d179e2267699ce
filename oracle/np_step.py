"""Second, independent transcription of the time step in NumPy (np.roll).

TEST INFRASTRUCTURE ONLY (part of the oracle).  It exists to cross-check
sc_oracle.c on tiny lattices: it builds its velocity set by enumeration, keeps
fields as [z, y, x] arrays and uses whole-array shifts instead of index
arithmetic, so a slip in either transcription shows up as a mismatch in the
moments (which do not depend on the order of the velocities).
Section 2: Eqs. lbm, omega_i, Guo, feq, u and sc_force; c_s^2 = 1/3.
"""
from __future__ import annotations

import itertools

import numpy as np

CS2 = 1.0 / 3.0


def velocity_set(dim: int):
    """D2Q9 / D3Q19: every vector with components in {-1, 0, 1} and |xi|^2 <= 2."""
    vs = [v for v in itertools.product((-1, 0, 1), repeat=dim) if sum(c * c for c in v) <= 2]
    w0, w1, w2 = (4 / 9, 1 / 9, 1 / 36) if dim == 2 else (1 / 3, 1 / 18, 1 / 36)
    w = [w0 if sum(c * c for c in v) == 0 else (w1 if sum(c * c for c in v) == 1 else w2) for v in vs]
    vs = [tuple(v) + (0,) * (3 - dim) for v in vs]
    return np.array(vs, dtype=np.int64), np.array(w)


def forcing_set(dim: int, extended: bool):
    """(vectors, W) of the forcing stencil: W = w / c_s^2 on the velocity set, or E6."""
    if not extended:
        xi, w = velocity_set(dim)
        keep = np.any(xi != 0, axis=1)
        return xi[keep], w[keep] / CS2
    Wtab = {1: 2 / 15, 2: 1 / 15, 3: 1 / 60, 4: 1 / 120}
    vs, W = [], []
    for v in itertools.product(range(-2, 3), repeat=3):
        l2 = sum(c * c for c in v)
        if l2 in Wtab and max(abs(c) for c in v) <= 2 and not (l2 == 4 and sorted(map(abs, v)) != [0, 0, 2]):
            vs.append(v)
            W.append(Wtab[l2])
    return np.array(vs, dtype=np.int64), np.array(W)


def shift(a: np.ndarray, v) -> np.ndarray:
    """a(x + v) for a periodic field a[z, y, x]."""
    return np.roll(a, shift=(-v[2], -v[1], -v[0]), axis=(0, 1, 2))


def step(f, dim: int, tau, G: float, G_self, psi_exp: bool, extended: bool = False):
    """One time step.  f: dict J -> [Q, nz, ny, nx] in velocity_set(dim) order."""
    xi, w = velocity_set(dim)
    fv, W = forcing_set(dim, extended)
    n = {J: f[J].sum(axis=0) for J in (0, 1)}
    j = {J: np.einsum("iq,izyx->qzyx", xi.astype(float), f[J]) for J in (0, 1)}
    psi = {J: (np.exp(-1.0 / n[J]) if psi_exp else n[J]) for J in (0, 1)}

    def grad_sum(a):  # sum_a W(|xi_a|^2) a(x + xi_a) xi_a
        return np.stack([sum(Wa * va[m] * shift(a, va) for va, Wa in zip(fv, W)) for m in range(3)])

    F = {}
    for J, K in ((0, 1), (1, 0)):
        F[J] = -G * CS2 * n[J] * grad_sum(n[K]) - G_self[J] * CS2 * psi[J] * grad_sum(psi[J])
    u = sum(j[J] + 0.5 * F[J] for J in (0, 1)) / (n[0] + n[1])
    out = {}
    uu = (u * u).sum(axis=0)
    for J in (0, 1):
        uF = (u * F[J]).sum(axis=0)
        post = np.empty_like(f[J])
        for i in range(len(w)):
            xu = sum(xi[i, m] * u[m] for m in range(3))
            xF = sum(xi[i, m] * F[J][m] for m in range(3))
            feq = n[J] * w[i] * (1 + xu / CS2 + (xu * xu - CS2 * uu) / (2 * CS2 * CS2))
            Fi = w[i] * (xF / CS2 + (xu * xF - CS2 * uF) / (CS2 * CS2))
            post[i] = f[J][i] - (f[J][i] - feq) / tau[J] + (1 - 1 / (2 * tau[J])) * Fi
        # streaming: f_i(x + xi_i) <- post_i(x)
        out[J] = np.stack([shift(post[i], -xi[i]) for i in range(len(w))])
    return out


def init(nA, nB, dim: int):
    """f_i = w_i n_J for fields [nz, ny, nx]."""
    _, w = velocity_set(dim)
    return {0: w[:, None, None, None] * nA[None], 1: w[:, None, None, None] * nB[None]}


def moments(f, dim: int, G: float, G_self, psi_exp: bool, extended: bool = False):
    """(n_A, n_B, u[3]) with the common velocity of Eq. u."""
    xi, _ = velocity_set(dim)
    fv, W = forcing_set(dim, extended)
    n = {J: f[J].sum(axis=0) for J in (0, 1)}
    j = {J: np.einsum("iq,izyx->qzyx", xi.astype(float), f[J]) for J in (0, 1)}
    psi = {J: (np.exp(-1.0 / n[J]) if psi_exp else n[J]) for J in (0, 1)}

    def grad_sum(a):
        return np.stack([sum(Wa * va[m] * shift(a, va) for va, Wa in zip(fv, W)) for m in range(3)])

    F = {J: -G * CS2 * n[J] * grad_sum(n[K]) - G_self[J] * CS2 * psi[J] * grad_sum(psi[J])
         for J, K in ((0, 1), (1, 0))}
    u = sum(j[J] + 0.5 * F[J] for J in (0, 1)) / (n[0] + n[1])
    return n[0], n[1], u
