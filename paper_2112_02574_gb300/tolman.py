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


def sweep(members, steps: int, check_every: int = 2048, bin_width=0.5, device="cuda", converge: bool = False,
          dp_tol: float = 1e-5, du_tol: float = 1e-12):
    """Step the droplets described by `members` as one batch and return, per member, a dict with its side
    L, sign (+1: A-rich, -1: B-rich), R and tag, and from the device: dP, R_s, sigma_s, P_in, P_out,
    dP_change = |dP(t) - dP(t - check_every)| / dP(t - check_every), steps (run), converged, and
    com_offset (largest coordinate distance of the droplet component's centre of mass from the centre
    node).  Each member is a dict with L (cube side), R, sign, params (make_params keywords), fields
    ((n_A, n_B) initial densities) and optionally tag.

    converge=False: every member runs `steps` steps.  converge=True: section 4's criteria are checked
    every check_every (= 2^11) steps -- a member has converged when the relative change of dP is below
    dp_tol or the velocity change dU below du_tol -- and converged members are retired from the batch;
    the rest run to `steps` at most."""
    plist = [B.make_params((m["L"],) * 3, **m["params"]) for m in members]
    batch = B.Batch(plist, [m["fields"] for m in members], device=device)
    n = len(members)
    ran = [0] * n
    done = [False] * n
    change = [float("nan")] * n
    if not converge:
        first = max(0, steps - check_every)
        batch.step(first)
        before = _pressure_jumps(batch, [m["L"] for m in members]).cpu().numpy()
        batch.step(steps - first)
        after = _pressure_jumps(batch, [m["L"] for m in members]).cpu().numpy()
        for k in range(n):
            ran[k] = steps
            change[k] = float(abs(after[k] - before[k]) / abs(before[k])) if before[k] != 0 else float("nan")
    else:
        u_prev = [m.moments()[2].clone() for m in batch.members]
        prev = None
        t = 0
        while t < steps and batch.active > 0:
            w = min(check_every, steps - t)
            batch.step(w)
            t += w
            live = [k for k in range(n) if not done[k]]
            dps = _pressure_jumps(batch, [members[k]["L"] for k in live], live)
            dus = torch.cat([batch.members[k].velocity_change(u_prev[k]) for k in live])
            dps, dus = dps.cpu().numpy(), dus.cpu().numpy()
            for j, k in enumerate(live):
                ran[k] = t
                if prev is not None and prev[k] != 0:
                    change[k] = float(abs(dps[j] - prev[k]) / abs(prev[k]))
                if change[k] < dp_tol or dus[j] < du_tol:
                    done[k] = True
                    batch.retire(k)
            prev = {k: dps[j] for j, k in enumerate(live)}
    for m in batch.members:
        B.sc_sync(m.ctx)  # raises on a non-finite or non-positive density
    final = _analyse(batch, [m["L"] for m in members], bin_width).cpu().numpy()
    out = []
    for k, m in enumerate(members):
        o = final[k]
        out.append({"L": m["L"], "sign": m["sign"], "R": m["R"], "tag": m.get("tag"), "dP": float(o[0]),
                    "R_s": float(o[2]), "sigma_s": float(o[3]), "P_in": float(o[6]), "P_out": float(o[7]),
                    "dP_change": change[k], "steps": ran[k], "converged": done[k] if converge else None,
                    "com_offset": _com_offset(batch.members[k], m["L"], m["sign"])})
    return out


def _pressure_jumps(batch, sides, which=None):
    """P(centre node) - P(far corner) (Eq. bulkp, section 4) of the members `which` (all by default)."""
    which = range(len(sides)) if which is None else which
    out = []
    for k, L in zip(which, sides):
        m = batch.members[k]
        out.append(m.bulk_pressure((L // 2,) * 3) - m.bulk_pressure((L - 1,) * 3))
    return torch.cat(out)


def _com_offset(member, L, sign):
    """Largest coordinate distance between the centre node and the centre of mass of the droplet's
    component (A for an A-rich droplet), counted above its density at the far corner (section 4 accepts
    a run when this is below 1e-3)."""
    comp = 0 if sign > 0 else 1
    n = member.moments(with_u=False)[comp]
    bg = float(n[L * L * L - 1].item())
    c = member.centre_of_mass(comp, bg).cpu().numpy()
    return float(max(abs(c[i] - L // 2) for i in range(3)))


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
