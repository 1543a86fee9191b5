"""The score kernel's band, restated from its derivation for the tests.

A query whose FP32 value satisfies |f| > eps(q) B(q) keeps its FP32 label, so
eps(q) must bound |f32 - f| / B(q) on every query.  The derivation (the
library's score_band; Sec. III-B's label rule, the RQ summand of Eq. 3 in
the FK kernel of Eq. 4) gives eps(q) = eps0 + eps1 (|p(q)| + |s|max) with
|p(q)| the largest norm of the query's configuration-dependent control
points and |s|max that of the support set's, in coordinates scaled by
sqrt(gamma/2), u = 2^-24:

  eps1 = 2 u (1 + u) (1 + 2^-10)                 control points rounded once
  eps0 = (A u + (16 + 3) u + n_c^2 u^2 / 2 + 4 e_fk) (1 + 2^-10)
  A    = max(15 + 2, 10 + 2 * 2) + Mv - NP + 1    summands, NP = (Mv + 5) // 14
  n_c  = npair / 16 + npair / 32 + 2, npair = (ns + 1) // 2 + 1
  e_fk = 2^-32 (1 + sqrt(gamma/2) reach)          pair-arithmetic kinematics

The half-precision kernel takes uh = 2^-11 for the coordinates (eps1 with
uh + u) and 10 uh for t, an absolute 4 sqrt(3) 2^-25 for FP16 underflow,
and a factor 1 + 1/16.

Circle form (FP32 kernel): when the first configuration-dependent point sits
on frame 1 of a revolute joint 1, it moves on a circle of radius rho about
that joint's axis (Eq. 1 for link 1, then Eq. 2), and the kernel computes its
summand from sin and cos of half the joint angle.  That summand's error is
at most 12 u (1 + u) rho g + 6u + 2 rho_rcp, which eps(q) covers when it
takes max(|p(q)| + |s|max, cnorm) with cnorm = 6 rho g (rounded up):

  cnorm = 6 rho g (1 + 2^-20), if 0 < rho g <= 4 and |S| >= 128, else 0
  rho   = |(a_1 + t_x, cos(alpha_1) t_y - sin(alpha_1) t_z)|
"""
from __future__ import annotations

import math

import numpy as np

U = 2.0 ** -24
UH = 2.0 ** -11
RCP = 2.0 ** -23


def reach(arm) -> float:
    """Lever-arm bound of the chain in metres (base offset, |a| + |d| per link,
    a prismatic joint's travel counted to 2^10, the largest point offset)."""
    dh = np.asarray(arm.dh, dtype=np.float64)
    r = float(np.linalg.norm(np.asarray(arm.base, dtype=np.float64)[:3, 3]))
    r += float(np.sum(np.abs(dh[:, 0]) + np.abs(dh[:, 2]) + np.where(dh[:, 4] == 1, 1024.0, 0.0)))
    r += float(np.max(np.linalg.norm(np.asarray(arm.cp_off, dtype=np.float64), axis=1)))
    return float(np.float32(r * (1.0 + 1e-6)))


def constants(arm, gamma: float, ns: int, half: bool = False):
    """(eps0, eps1) as float32 values, for an arm with Mv configuration-dependent points."""
    mv = int(np.sum(np.asarray(arm.cp_joint) != 0))
    npp = (mv + 5) // 14
    t_err = 10.0 * (UH if half else U)
    pair = t_err + 5.0 * U + RCP if npp > 0 else 0.0
    single = t_err + 2.0 * RCP if mv > 2 * npp else 0.0
    term = max(pair, single) + (mv - npp + 1) * U
    npair = float((ns + 1) // 2 + 1)
    nc = npair / 16 + npair / 32 + 2.0
    acc = (16 + 3) * U + 0.5 * nc * nc * U * U
    efk = 2.0 ** -32 * (1.0 + np.sqrt(0.5 * gamma) * reach(arm))
    pos_abs = 4.0 * np.sqrt(3.0) * 2.0 ** -25 if half else 0.0
    factor = 1.0 + (1.0 / 16 if half else 2.0 ** -10)
    eps0 = (term + acc + 4.0 * efk + pos_abs) * factor
    eps1 = 2.0 * ((UH if half else 0.0) + U) * (1.0 + U) * factor
    return float(np.float32(eps0)), float(np.float32(eps1))


def circle_radius(arm):
    """rho of the first configuration-dependent point when it moves on the
    circle of a revolute joint 1 (metres), else None."""
    cj = np.asarray(arm.cp_joint)
    dep = np.flatnonzero(cj != 0)
    dh = np.asarray(arm.dh, dtype=np.float64)
    if len(dep) == 0 or cj[dep[0]] != 1 or dh[0, 4] != 0:
        return None
    t = np.asarray(arm.cp_off, dtype=np.float64)[dep[0]]
    a, al = float(dh[0, 0]), float(dh[0, 1])
    return math.hypot(a + t[0], math.cos(al) * t[1] - math.sin(al) * t[2])


CIRCLE_MIN_SUPPORT = 128


def circle_norm(arm, gamma: float, ns: int, on: bool = True) -> float:
    """cnorm of the FP32 band for a support set of ns points (0.0: every point
    in the direct form)."""
    rho = circle_radius(arm) if on else None
    if rho is None or ns < CIRCLE_MIN_SUPPORT:
        return 0.0
    rg = rho * math.sqrt(0.5 * gamma)
    if not (0.0 < rg <= 4.0):
        return 0.0
    return float(np.nextafter(np.float32(6.0 * rg * (1.0 + 2.0 ** -20)), np.float32(np.inf)))


def dependent(arm, cp):
    """The configuration-dependent control points of an (n, M, 3) array."""
    return np.asarray(cp)[:, np.asarray(arm.cp_joint) != 0, :]


def per_query(arm, gamma: float, eps0: float, eps1: float, cps, cpq, cnorm: float = 0.0):
    """eps(q) for every query from FP64 control points (n, M, 3) of the support
    set (cps) and of the queries (cpq); cnorm: the circle term."""
    g = np.sqrt(0.5 * gamma)
    smax = g * np.max(np.linalg.norm(dependent(arm, cps), axis=2)) if len(cps) else 0.0
    pn = g * np.max(np.linalg.norm(dependent(arm, cpq), axis=2), axis=1)
    return eps0 + eps1 * np.maximum(pn + smax, cnorm)
