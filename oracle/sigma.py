"""Generalized surface tension and surface of tension (paper section 3), FP64.

TEST INFRASTRUCTURE ONLY (part of the oracle; see oracle/__init__.py).

Discrete definitions shared by the oracle and the pins (readings of section 3):
* a profile is a list of sample points r_k (bin mean radius, ascending, r_0 may
  be 0) with the tangential pressure P_T,k;
* r_max is the last sample point; the integrals of Eq. gen_sigma and
  Eq. gen_d_sigma run over [0, r_max] (the paper's R_in -> 0, R_out -> infinity,
  cut where the profile ends);
* the pressure-jump function P_J(r; R) = P_in for r < R and P_out for r > R is
  integrated exactly, the measured P_T by the trapezoid rule over the samples.
With those, sigma[R] = dP R/3 + C/R^2 where C = int_0^r_max r^2 (P_out - P_T) dr,
so the minimum is at R_s = (6 C / dP)^(1/3) with sigma_s = dP R_s / 2 (Laplace at
the surface of tension, Eq. f-statio-Rs).  In two dimensions the weight r^2/R^2
becomes r/R: sigma[R] = dP R/2 + C2/R, R_s = (2 C2/dP)^(1/2), sigma_s = dP R_s.
"""
from __future__ import annotations

import numpy as np

__all__ = ["trapezoid", "surface_of_tension", "sigma_of_R", "notional_derivative", "argmin_on_grid",
           "sigma0_flat", "curvature_fit", "clean_profile"]


def trapezoid(y, x) -> float:
    """Plain trapezoid rule, summed left to right."""
    y = np.asarray(y, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    return float(np.sum(0.5 * (y[1:] + y[:-1]) * (x[1:] - x[:-1])))


def clean_profile(rows: np.ndarray):
    """(r, P_N, P_T, n_A, n_B) of the non-empty rows of a profile [nbins, 6]."""
    rows = np.asarray(rows)
    keep = rows[:, 5] > 0
    return tuple(rows[keep, c] for c in range(5))


def _pj_moment(R: float, r_max: float, P_in: float, P_out: float, power: int) -> float:
    """int_0^r_max r^power P_J(r; R) dr, exactly, for 0 < R <= r_max."""
    k = power + 1
    return P_in * R**k / k + P_out * (r_max**k - R**k) / k


def sigma_of_R(R, r, PT, P_in: float, P_out: float, dim: int = 3):
    """Eq. gen_sigma: sigma[R] = int_0^r_max (r/R)^(dim-1) [P_J(r;R) - P_T(r)] dr."""
    r = np.asarray(r, dtype=np.float64)
    w = r ** (dim - 1)
    T = trapezoid(w * PT, r)
    R = np.atleast_1d(np.asarray(R, dtype=np.float64))
    out = np.array([(_pj_moment(x, r[-1], P_in, P_out, dim - 1) - T) / x ** (dim - 1) for x in R])
    return out if out.size > 1 else float(out[0])


def notional_derivative(R, r, PT, P_in: float, P_out: float):
    """Eq. gen_d_sigma (three dimensions): -(2/R^3) int_0^r_max r (r - R) [P_J - P_T] dr."""
    r = np.asarray(r, dtype=np.float64)
    R = np.atleast_1d(np.asarray(R, dtype=np.float64))
    out = []
    for x in R:
        pj = _pj_moment(x, r[-1], P_in, P_out, 2) - x * _pj_moment(x, r[-1], P_in, P_out, 1)
        pt = trapezoid(r * (r - x) * PT, r)
        out.append(-2.0 / x**3 * (pj - pt))
    out = np.array(out)
    return out if out.size > 1 else float(out[0])


def surface_of_tension(r, PT, P_in: float, P_out: float, dim: int = 3) -> dict:
    """Closed-form minimum of sigma[R] (see module docstring)."""
    r = np.asarray(r, dtype=np.float64)
    dP = P_in - P_out
    r_max = r[-1]
    C = P_out * r_max**dim / dim - trapezoid(r ** (dim - 1) * PT, r)
    if dim == 3:
        Rs = np.cbrt(6.0 * C / dP)
        sig = 0.5 * dP * Rs
    else:
        Rs = np.sqrt(2.0 * C / dP)
        sig = dP * Rs
    return {"dP": dP, "C": C, "Rs": float(Rs), "sigma_s": float(sig)}


def argmin_on_grid(r, PT, P_in: float, P_out: float, R_lo: float, R_hi: float, step: float = 0.01,
                   dim: int = 3):
    """The paper's procedure (section 3): evaluate sigma[R] on a grid and
    interpolate the position of its minimum with a parabola through the
    smallest grid value and its two neighbours.  Returns (R_min, sigma_min)."""
    grid = np.arange(R_lo, R_hi + 0.5 * step, step)
    s = np.asarray(sigma_of_R(grid, r, PT, P_in, P_out, dim))
    k = int(np.clip(np.argmin(s), 1, len(grid) - 2))
    y0, y1, y2 = s[k - 1], s[k], s[k + 1]
    den = y0 - 2.0 * y1 + y2
    off = 0.5 * (y0 - y2) / den if den != 0 else 0.0
    Rm = grid[k] + off * step
    return float(Rm), float(y1 - 0.25 * (y0 - y2) * off)


def sigma0_flat(PN, PT) -> float:
    """Flat-interface tension of section 4: sum over the upper half of the
    planar profile of (P_N - P_T), one sample per lattice plane (the integrand
    vanishes at both ends of the half, so rectangle and trapezoid agree)."""
    PN = np.asarray(PN, dtype=np.float64)
    PT = np.asarray(PT, dtype=np.float64)
    L = len(PN)
    return float(np.sum(PN[L // 2:] - PT[L // 2:]))


def curvature_fit(Rs, sigma_s, order: int = 2, sigma0=None) -> dict:
    """Least-squares fit of Eq. sigma_c, sigma(R_s) = sigma_0 (1 - 2 delta/R_s + (2kbar + k)/R_s^2),
    as a polynomial in 1/R_s (negative R_s for droplets of the other component).  With sigma0
    given (the flat-interface value) only delta and 2kbar + k are fitted, to sigma_s/sigma_0 - 1."""
    x = 1.0 / np.asarray(Rs, dtype=np.float64)
    y = np.asarray(sigma_s, dtype=np.float64)
    if sigma0 is None:
        c = np.polynomial.polynomial.polyfit(x, y, order)
        s0 = c[0]
        out = {"sigma0": float(s0), "delta": float(-c[1] / (2.0 * s0))}
        if order >= 2:
            out["rigidity"] = float(c[2] / s0)
        return out
    s0 = float(sigma0)
    A = np.stack([x ** p for p in range(1, order + 1)], axis=1)
    b, *_ = np.linalg.lstsq(A, y / s0 - 1.0, rcond=None)
    out = {"sigma0": s0, "delta": float(-b[0] / 2.0)}
    if order >= 2:
        out["rigidity"] = float(b[1])
    return out
