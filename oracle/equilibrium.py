"""Constant-enthalpy, constant-pressure chemical equilibrium by Gibbs minimisation.

TEST INFRASTRUCTURE ONLY (an oracle-side reference used to pin the kinetics:
a long adiabatic integration must relax to the state this module finds).

For an ideal-gas mixture at (T, p), the equilibrium composition minimises
G = sum_k n_k (g_k/RT + ln(n_k/N) + ln(p/P0)) subject to the linear invariants
of the kinetics. Those invariants are the left null space of the net
stoichiometric matrix S (K x I): any vector b with b^T S = 0 is conserved by
every reaction, so the kinetic equilibrium is the Gibbs minimum under
B^T n = B^T n0 with B a basis of that null space (element conservation and the
inertness of N2 are both contained in it). The first-order conditions give
n_k = N exp(sum_r lambda_r B_kr - g_k/RT - ln(p/P0)); (lambda, ln N) are found by
Newton's method on the convex dual for a fixed total N, with a 1-D root for N
(an element-potential method in the sense of Gordon & McBride, NASA RP-1311,
Ch. 2). The outer problem finds the
temperature whose equilibrium composition has the initial mass enthalpy.

The NASA-7 polynomials are evaluated here by this module's own code.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.optimize

RC = 8.31446261815324e7
P0 = 1.01325e6


def _coeffs(mech, T):
    lo = T < mech.T_mid
    return np.where(lo[:, None], mech.nasa_lo, mech.nasa_hi)


def h_RT(mech, T):
    a = _coeffs(mech, T)
    return (a[:, 0] + a[:, 1] * T / 2 + a[:, 2] * T ** 2 / 3 + a[:, 3] * T ** 3 / 4
            + a[:, 4] * T ** 4 / 5 + a[:, 5] / T)


def s_R(mech, T):
    a = _coeffs(mech, T)
    return (a[:, 0] * np.log(T) + a[:, 1] * T + a[:, 2] * T ** 2 / 2 + a[:, 3] * T ** 3 / 3
            + a[:, 4] * T ** 4 / 4 + a[:, 6])


def h_mass(mech, T, Y):
    return float(np.sum(Y * h_RT(mech, T) * RC * T / mech.W))


def _dual_min(B, c, mu_eff, lam, tol=1e-15, max_iter=500):
    """Minimise F(lam) = -c.lam + sum_k exp(B_k lam - mu_eff_k) (strictly convex)
    by Newton's method with backtracking; returns (lam, n = exp(B lam - mu_eff))."""
    def val(l):
        n = np.exp(np.clip(B @ l - mu_eff, -745.0, 700.0))
        return -c @ l + n.sum(), n

    F, n = val(lam)
    cs = np.abs(c).sum()
    for _ in range(max_iter):
        g = B.T @ n - c
        if np.abs(g).max() <= tol * cs:
            break
        H = (B * n[:, None]).T @ B
        H = H + 1e-14 * np.trace(H) * np.eye(H.shape[0])
        d = -np.linalg.solve(H, g)
        t = 1.0
        while True:
            l1 = lam + t * d
            F1, n1 = val(l1)
            if F1 <= F + 1e-4 * t * (g @ d) or t < 1e-14:
                break
            t *= 0.5
        lam, F, n = l1, F1, n1
    return lam, n


def gibbs_tp(mech, T, p, n0, B=None):
    """Equilibrium moles per gram at fixed (T, p) under the kinetic invariants.

    For a fixed total N the problem is the strictly convex dual above with
    mu_eff = g/RT + ln(p/P0) - ln N; the outer 1-D root finds the N that equals
    the sum of the resulting moles.
    """
    if B is None:
        B = scipy.linalg.null_space(mech.net_stoich().T.astype(np.float64))
    c = B.T @ n0
    mu = h_RT(mech, T) - s_R(mech, T) + np.log(p / P0)
    N0 = n0.sum()
    state = {"lam": np.zeros(B.shape[1])}

    def resid(lnN):
        lam, n = _dual_min(B, c, mu - lnN, state["lam"])
        state["lam"], state["n"] = lam, n
        return np.log(n.sum()) - lnN

    lo, hi = np.log(0.2 * N0), np.log(5.0 * N0)
    lnN = scipy.optimize.brentq(resid, lo, hi, xtol=1e-15, rtol=1e-15)
    resid(lnN)
    return state["n"]


def equilibrium_hp(mech, T0, p, Y0, T_bracket=(300.0, 5500.0)):
    """(T_eq, Y_eq) with the mass enthalpy of (T0, Y0) at pressure p."""
    Y0 = np.asarray(Y0, dtype=np.float64)
    n0 = Y0 / mech.W
    B = scipy.linalg.null_space(mech.net_stoich().T.astype(np.float64))
    h0 = h_mass(mech, T0, Y0)

    def g(T):
        n = gibbs_tp(mech, T, p, n0, B)
        return h_mass(mech, T, n * mech.W) - h0

    T_eq = scipy.optimize.brentq(g, *T_bracket, xtol=1e-12, rtol=1e-14)
    n = gibbs_tp(mech, T_eq, p, n0, B)
    return T_eq, n * mech.W
