"""Exact solution of the 1D relativistic Riemann problem for p = e/3.

Independent of the oracle: it is derived from the relativistic Euler
equations of Sec. 2 (conservation of T^{mu nu} and of the baryon current),
not from the SHASTA scheme.  Both initial states are at rest with e_L > e_R,
so the solution is a left-moving rarefaction, a contact and a right-moving
shock.

* Rarefaction (simple wave, Riemann invariant conserved across it):
  atanh(v) + (sqrt(3)/4) ln e = (sqrt(3)/4) ln e_L, and inside the fan the
  local sound cone gives v(xi) = (xi + c_s)/(1 + xi c_s), c_s = 1/sqrt(3).
  Baryons follow the isentrope n ~ e^(3/4).
* Shock into the state at rest: relative velocity across a shock between two
  states a, b of an ideal fluid,
  v^2 = (p_b - p_a)(e_b - e_a) / ((e_a + p_b)(e_b + p_a)).
  The shock speed follows from the jump of T^{00}: v_s = M_2 / (E_2 - E_R),
  the baryon density behind it from the jump of J^0:
  n_2 gamma_2 (v_s - v_2) = n_R v_s.
* Contact: equal pressure, i.e. equal e for p = e/3, and equal velocity.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq

CS = 1.0 / math.sqrt(3.0)


def v_rarefaction(e, e_l):
    return math.tanh(math.sqrt(3.0) / 4.0 * math.log(e_l / e))


def v_shock(e, e_r):
    p, pr = e / 3.0, e_r / 3.0
    return math.sqrt((p - pr) * (e - e_r) / ((e_r + p) * (e + pr)))


def solve(e_l=1.0, e_r=0.01, n_l=1.0, n_r=0.01):
    """Return the star state and wave speeds as a dict."""
    f = lambda e: v_rarefaction(e, e_l) - v_shock(e, e_r)
    e_star = brentq(f, e_r * (1 + 1e-12), e_l * (1 - 1e-12), xtol=1e-15, rtol=1e-15)
    v_star = v_rarefaction(e_star, e_l)
    g2 = 1.0 / (1.0 - v_star * v_star)
    p_star = e_star / 3.0
    E2 = (e_star + p_star) * g2 - p_star
    M2 = (e_star + p_star) * g2 * v_star
    v_s = M2 / (E2 - e_r)
    n2 = n_r * v_s / (math.sqrt(g2) * (v_s - v_star))
    n3 = n_l * (e_star / e_l) ** 0.75
    xi_tail = (v_star - CS) / (1.0 - v_star * CS)
    return dict(e_star=e_star, v_star=v_star, v_shock=v_s, n2=n2, n3=n3,
                xi_head=-CS, xi_tail=xi_tail, e_l=e_l, e_r=e_r, n_l=n_l, n_r=n_r)


def profile(xi, sol):
    """e, v, n at similarity coordinates xi = (x - x0)/t."""
    xi = np.asarray(xi, dtype=np.float64)
    e = np.empty_like(xi)
    v = np.empty_like(xi)
    n = np.empty_like(xi)
    for i, s in enumerate(xi.flat):
        if s < sol["xi_head"]:
            e.flat[i], v.flat[i], n.flat[i] = sol["e_l"], 0.0, sol["n_l"]
        elif s < sol["xi_tail"]:
            vv = (s + CS) / (1.0 + s * CS)
            ee = sol["e_l"] * ((1.0 - vv) / (1.0 + vv)) ** (2.0 / math.sqrt(3.0))
            e.flat[i], v.flat[i] = ee, vv
            n.flat[i] = sol["n_l"] * (ee / sol["e_l"]) ** 0.75
        elif s < sol["v_star"]:
            e.flat[i], v.flat[i], n.flat[i] = sol["e_star"], sol["v_star"], sol["n3"]
        elif s < sol["v_shock"]:
            e.flat[i], v.flat[i], n.flat[i] = sol["e_star"], sol["v_star"], sol["n2"]
        else:
            e.flat[i], v.flat[i], n.flat[i] = sol["e_r"], 0.0, sol["n_r"]
    return e, v, n
