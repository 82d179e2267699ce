"""Tolman length and rigidity from a sweep of droplets (section 4, Eq. sigma_c).

Droplets of several radii, rich in component A (positive curvature) or in B
(negative curvature), are stepped together as one batch (one step-kernel launch
per time step).  For each member the device computes the radial pressure-tensor
profile (Eq. sm:pt), the bulk pressures at the centre node and at the far corner
(Eq. bulkp) and the sigma[R] minimum (Eqs. gen_sigma, gen_d_sigma), which give
(R_s, sigma_s = dP R_s / 2).  A periodic slab gives the flat-interface tension
sigma_0 (sc_sigma0_flat) and sc_curvature_fit fits Eq. sigma_c,
sigma(R_s) = sigma_0 (1 - 2 delta / R_s + (2 kbar + k) / R_s^2).

All arithmetic runs in the library's kernels; this module only sets the runs up
and moves the small result tensors.  Initial fields come from a caller-supplied
function, so any initial profile can be used (section 4 uses a tanh droplet).
"""
from __future__ import annotations

import math

import torch

from . import binding as B


def droplet_side(R: float) -> int:
    """Cube side about 4 R: 4 ceil(R), a multiple of 4, so that every storage mode takes the staged kernel."""
    return 4 * math.ceil(R)


def droplet_sweep(radii, signs, make_fields, params_kw, steps: int, check_every: int = 2048, bin_width=0.5,
                  device="cuda"):
    """Step one droplet per (R, sign) as a batch and return, per droplet, a dict with the side L, the sign
    (+1: A-rich, -1: B-rich), R, and from the device: dP, R_s, sigma_s, P_in, P_out, and dP_change =
    |dP(steps) - dP(steps - check_every)| / dP(steps - check_every) (the convergence measure of section 4).

    make_fields(shape_zyx, centre_xyz, R, a_rich) -> (n_A, n_B); params_kw: make_params keywords shared by
    every member (storage, G, G_self, tau, psi_self, ...)."""
    members = [(R, s, droplet_side(R)) for R in radii for s in signs]
    plist = [B.make_params((L, L, L), **params_kw) for _, _, L in members]
    fields = [make_fields((L, L, L), (L // 2,) * 3, R, s > 0) for R, s, L in members]
    batch = B.Batch(plist, fields, device=device)
    first = max(0, steps - check_every)
    batch.step(first)
    before = _analyse(batch, members, bin_width)
    batch.step(steps - first)
    after = _analyse(batch, members, bin_width)
    for m in batch.members:
        B.sc_sync(m.ctx)  # raises on a non-finite or non-positive density
    before, after = before.cpu().numpy(), after.cpu().numpy()
    out = []
    for k, (R, s, L) in enumerate(members):
        o, p = after[k], before[k]
        out.append({"L": L, "sign": s, "R": R, "dP": float(o[0]), "R_s": float(o[2]), "sigma_s": float(o[3]),
                    "P_in": float(o[6]), "P_out": float(o[7]),
                    "dP_change": float(abs(o[0] - p[0]) / abs(p[0])) if p[0] != 0 else float("nan")})
    return out


def _analyse(batch, members, bin_width):
    outs = []
    for m, (_, _, L) in zip(batch.members, members):
        _, o = B.surface_of_tension(m, (L // 2,) * 3, bin_width)
        outs.append(o)
    return torch.stack(outs)


def flat_sigma0(shape, make_fields, params_kw, steps: int, device="cuda"):
    """sigma_0 of a periodic slab (an A-rich band along z) after `steps` steps: a CUDA tensor [1]."""
    nA, nB = make_fields(tuple(shape[::-1]))
    sim = B.Simulation(B.make_params(tuple(shape), **params_kw), nA, nB, device=device)
    sim.step(steps)
    _, s0 = B.sigma0_flat(sim)
    B.sc_sync(sim.ctx)
    return s0


def fit(droplets, sigma0=None, order: int = 2, device="cuda"):
    """Eq. sigma_c over the droplets of droplet_sweep (R_s signed by the droplet's component), on the
    device; sigma0 a CUDA tensor [1] (held fixed) or None (fitted).  Returns a dict sigma0, delta,
    rigidity (2 kbar + k), rms."""
    Rs = torch.tensor([d["sign"] * d["R_s"] for d in droplets], dtype=torch.float64, device=device)
    sg = torch.tensor([d["sigma_s"] for d in droplets], dtype=torch.float64, device=device)
    o = B.curvature_fit(Rs, sg, order=order, sigma0=sigma0).cpu().numpy()
    return {"sigma0": float(o[0]), "delta": float(o[1]), "rigidity": float(o[2]), "rms": float(o[3])}
