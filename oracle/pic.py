"""Plain FP64 numpy oracle of the particle side of the space-charge step
(Sec. 4.1 domain transform and Fig. sc_workflow; Eqs. potential_transform,
efield_transform, rms_sigma and halo) and of the kick-drift push around it.

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the product path.
It shares no code with the CUDA path; each function is the formula written
out, evaluated in numpy FP64 in the order stated.
"""
from __future__ import annotations

import numpy as np


def domain_transform(x, y, z, centre=(0.0, 0.0, 0.0), delta=0.2):
    """Sec. 4.1: Gamma_i = max_d |x_i,d - c_d| (the paper's Gamma with
    l = (1, 1, 1), a cubic computation space), s = (1 + delta) max_i Gamma_i,
    x* = (x - c) / s in [-1, 1]^3 / (1 + delta); mapped onto the unit cube
    the solver covers, u = 1/2 + x* / 2 = 1/2 + (x - c) / S with S = 2 s.
    Returns (u, v, w, S)."""
    c = [float(v) for v in centre]
    d = [np.asarray(a, np.float64) - cv for a, cv in zip((x, y, z), c)]
    ext = max(float(np.abs(a).max()) for a in d)
    s = (1.0 + delta) * ext
    S = 2.0 * s
    inv = 1.0 / S
    return (*(0.5 + a * inv for a in d), S)


def rescale_fields(H, S):
    """Fig. sc_workflow, back to particle space on the grid: phi / S
    (Eq. potential_transform) and E / S^2 (Eq. efield_transform) on every
    level of the oracle hierarchy H."""
    f1, f2 = 1.0 / S, 1.0 / (S * S)
    for l in range(H.nlevels):
        H.set(l, "phi", H.get(l, "phi") * f1)
        for f in ("ex", "ey", "ez"):
            H.set(l, f, H.get(l, f) * f2)


def push(pos, mom, field, q_over_m, dt):
    """Kick-drift step: p <- p + (q/m dt) E, then x <- x + dt p; returns the
    new (pos, mom) as lists of arrays."""
    k = q_over_m * dt
    mom = [p + k * e for p, e in zip(mom, field)]
    pos = [x + dt * p for x, p in zip(pos, mom)]
    return pos, mom


def moments(x, y, z):
    """Eqs. rms_sigma and halo about the centroid: <w>, sigma_w =
    sqrt(<(w - <w>)^2>), xi_w = <(w - <w>)^4> / <(w - <w>)^2>^2."""
    out = {"centroid": [], "sigma": [], "xi": []}
    for a in (x, y, z):
        a = np.asarray(a, np.float64)
        m = a.mean()
        d = a - m
        m2, m4 = (d ** 2).mean(), (d ** 4).mean()
        out["centroid"].append(m)
        out["sigma"].append(np.sqrt(m2))
        out["xi"].append(m4 / (m2 * m2) if m2 > 0 else 0.0)
    return {k: np.array(v) for k, v in out.items()}

