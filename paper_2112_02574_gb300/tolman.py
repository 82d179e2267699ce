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
    """Step one droplet per (R, sign) in a cube of side droplet_side(R) as a batch; see sweep().

    make_fields(shape_zyx, centre_xyz, R, a_rich) -> (n_A, n_B); params_kw: make_params keywords shared by
    every member (storage, G, G_self, tau, psi_self, ...)."""
    members = []
    for R in radii:
        for s in signs:
            L = droplet_side(R)
            members.append({"L": L, "R": R, "sign": s, "params": params_kw,
                            "fields": make_fields((L, L, L), (L // 2,) * 3, R, s > 0)})
    return sweep(members, steps, check_every, bin_width, device)


def sweep(members, steps: int, check_every: int = 2048, bin_width=0.5, device="cuda"):
    """Step the droplets described by `members` as one batch and return, per member, a dict with its side
    L, sign (+1: A-rich, -1: B-rich), R and tag, and from the device: dP, R_s, sigma_s, P_in, P_out, and
    dP_change = |dP(steps) - dP(steps - check_every)| / dP(steps - check_every) (the convergence measure
    of section 4).  Each member is a dict with L (cube side), R, sign, params (make_params keywords),
    fields ((n_A, n_B) initial densities) and optionally tag."""
    plist = [B.make_params((m["L"],) * 3, **m["params"]) for m in members]
    batch = B.Batch(plist, [m["fields"] for m in members], device=device)
    first = max(0, steps - check_every)
    batch.step(first)
    before = _analyse(batch, [m["L"] for m in members], bin_width)
    batch.step(steps - first)
    after = _analyse(batch, [m["L"] for m in members], bin_width)
    for m in batch.members:
        B.sc_sync(m.ctx)  # raises on a non-finite or non-positive density
    before, after = before.cpu().numpy(), after.cpu().numpy()
    out = []
    for k, m in enumerate(members):
        o, p = after[k], before[k]
        out.append({"L": m["L"], "sign": m["sign"], "R": m["R"], "tag": m.get("tag"), "dP": float(o[0]),
                    "R_s": float(o[2]), "sigma_s": float(o[3]), "P_in": float(o[6]), "P_out": float(o[7]),
                    "dP_change": float(abs(o[0] - p[0]) / abs(p[0])) if p[0] != 0 else float("nan")})
    return out


def _analyse(batch, sides, bin_width):
    outs = []
    for m, L in zip(batch.members, sides):
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


def flat_densities(shape, make_fields, params_kw, steps: int, device="cuda"):
    """The flat-interface pre-run of section 4: a periodic slab (an A-rich band along z, centred) stepped
    `steps` times; returns the bulk densities {"A_in", "A_out", "B_in", "B_out"} read at the slab's
    centre plane (inside the band) and at z = 0 (outside), plus sigma_0 -- the inner and outer values
    that initialise the droplets of the same couplings."""
    nA, nB = make_fields(tuple(shape[::-1]))
    sim = B.Simulation(B.make_params(tuple(shape), **params_kw), nA, nB, device=device)
    sim.step(steps)
    a, b, _ = sim.moments(with_u=False)
    _, s0 = B.sigma0_flat(sim)
    B.sc_sync(sim.ctx)
    nx, ny, nz = shape
    mid, edge = (nz // 2) * nx * ny, 0
    v = torch.stack([a[mid], a[edge], b[mid], b[edge], s0[0]]).cpu().numpy()
    return {"A_in": float(v[0]), "A_out": float(v[1]), "B_in": float(v[2]), "B_out": float(v[3]),
            "sigma0": float(v[4])}


def usable(d, max_change: float = 1e-3) -> bool:
    """A droplet enters the fit if it is one: a positive pressure jump and a positive surface-of-tension
    radius within a factor two of its initial radius, and dP settled to max_change over the last check
    interval (section 4 converges to 1e-5; a droplet that dissolved or whose interface fills the box
    fails one of these)."""
    ok = d["dP"] > 0 and 0.5 * d["R"] < d["R_s"] < 2.0 * d["R"]
    return bool(ok and d["dP_change"] < max_change)


def fit(droplets, sigma0=None, order: int = 2, device="cuda", select=usable):
    """Eq. sigma_c over the droplets of sweep() that pass `select` (R_s signed by the droplet's component),
    on the device; sigma0 a CUDA tensor [1] (held fixed) or None (fitted).  Returns a dict sigma0, delta,
    rigidity (2 kbar + k), rms, used (droplets in the fit)."""
    ds = [d for d in droplets if select is None or select(d)]
    need = order + (0 if sigma0 is not None else 1)
    if len(ds) < need:
        return {"sigma0": float("nan"), "delta": float("nan"), "rigidity": float("nan"), "rms": float("nan"),
                "used": len(ds)}
    Rs = torch.tensor([d["sign"] * d["R_s"] for d in ds], dtype=torch.float64, device=device)
    sg = torch.tensor([d["sigma_s"] for d in ds], dtype=torch.float64, device=device)
    o = B.curvature_fit(Rs, sg, order=order, sigma0=sigma0).cpu().numpy()
    return {"sigma0": float(o[0]), "delta": float(o[1]), "rigidity": float(o[2]), "rms": float(o[3]),
            "used": len(ds)}
