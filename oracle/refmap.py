"""Reference mapping by Bilger's mixture fraction: the FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` (and nothing on the GPU path).

The paper (Methodology, "DLBFoam: Dynamic load balancing") states that, with
Bilger's mixture fraction Z, the chemistry of a cell is either solved or mapped
from a reference solution of the domain with a similar Z. The readings used on
both sides (they are listed with the design notes):

- zone: cells with |Z - Z_center| <= Z_tol, Z of the initial state;
- reference: the zone cell with the lowest index; it is integrated;
- mapped: the other zone cells whose initial T is within T_tol of the
  reference's; each receives the reference's change over the step
  (T += T_ref(dt) - T_ref(0), Y_k += Y_ref,k(dt) - Y_ref,k(0)); if the reference
  failed, a mapped cell keeps its initial state and takes the reference's status;
- every other cell is integrated.

Z is computed here from Bilger's definition as printed in the literature: the
element mass fractions Z_e = sum_k a_ek W_e Y_k / W_k, the coupling function
beta = 2 Z_C / W_C + Z_H / (2 W_H) - Z_O / W_O, and
Z = (beta - beta_ox) / (beta_fuel - beta_ox). (The GPU path folds the atomic
masses away into one coefficient per species; this side keeps them.)

Pinned by ``tests/test_refmap_oracle.py``: beta = 0 for stoichiometric
fuel/oxygen mixtures and their complete-combustion products (both fuels), Z = 0
and 1 on the streams and Z = w on stream blends, Z conserved by the oracle's
integration, the selection rule by brute force on hand-made cases, and the
mapped result of a cell identical to the reference.
"""
from __future__ import annotations

import numpy as np

from . import integrate

# atomic masses (g/mol); they cancel in Z and only need to be positive
_W_ATOM = {"C": 12.011, "H": 1.008, "O": 15.999}


def element_mass_fractions(mech, Y):
    """Z_e[n, E] = sum_k a_ek W_e Y_k / W_k for the elements C, H, O the mechanism has."""
    Y = np.atleast_2d(np.asarray(Y, dtype=np.float64))
    out = {}
    for e, w_e in _W_ATOM.items():
        if e in mech.elements:
            a = mech.elem[:, list(mech.elements).index(e)].astype(np.float64)
            out[e] = (Y * (a * w_e / mech.W)).sum(axis=1)
    return out


def coupling_beta(mech, Y):
    """Bilger's coupling function beta = 2 Z_C/W_C + Z_H/(2 W_H) - Z_O/W_O."""
    Ze = element_mass_fractions(mech, Y)
    n = np.atleast_2d(Y).shape[0]
    beta = np.zeros(n)
    if "C" in Ze:
        beta += 2.0 * Ze["C"] / _W_ATOM["C"]
    if "H" in Ze:
        beta += Ze["H"] / (2.0 * _W_ATOM["H"])
    if "O" in Ze:
        beta -= Ze["O"] / _W_ATOM["O"]
    return beta


def mixture_fraction(mech, Y, Y_fuel, Y_ox):
    """Z = (beta - beta_ox) / (beta_fuel - beta_ox)."""
    bf = coupling_beta(mech, Y_fuel)[0]
    bo = coupling_beta(mech, Y_ox)[0]
    return (coupling_beta(mech, Y) - bo) / (bf - bo)


def select(Z, T, Z_center, Z_tol, T_tol):
    """(zone[n] bool, reference index or -1, mapped[n] bool) by the rule above."""
    Z = np.asarray(Z, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    zone = np.abs(Z - Z_center) <= Z_tol
    idx = np.flatnonzero(zone)
    if idx.size == 0:
        return zone, -1, np.zeros_like(zone)
    ref = int(idx[0])
    mapped = zone & (np.abs(T - T[ref]) <= T_tol)
    mapped[ref] = False
    return zone, ref, mapped


def integrate_mapped(mech, T, p, Y, dt, Y_fuel, Y_ox, Z_center, Z_tol, T_tol, rtol=1e-8, atol=1e-12,
                     max_steps=100000, n_threads=0):
    """One step of the batch with reference mapping; the integrated cells go to the
    oracle integrator. Returns the result arrays plus Z, mapped and ref."""
    T = np.asarray(T, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    Y = np.atleast_2d(np.asarray(Y, dtype=np.float64))
    Z = mixture_fraction(mech, Y, Y_fuel, Y_ox)
    zone, ref, mapped = select(Z, T, Z_center, Z_tol, T_tol)
    solve = np.flatnonzero(~mapped)
    r = integrate(mech, T[solve], p[solve], Y[solve], dt, rtol=rtol, atol=atol, max_steps=max_steps,
                  n_threads=n_threads)
    n = T.shape[0]
    T_out, Y_out = T.copy(), Y.copy()
    status = np.zeros(n, dtype=np.int32)
    substeps = np.zeros(n, dtype=np.int32)
    T_out[solve], Y_out[solve] = r["T"], r["Y"]
    status[solve], substeps[solve] = r["status"], r["substeps"]
    if ref >= 0 and mapped.any():
        status[mapped] = status[ref]
        if status[ref] == 0:
            T_out[mapped] = T[mapped] + (T_out[ref] - T[ref])
            Y_out[mapped] = Y[mapped] + (Y_out[ref] - Y[ref])
    return {"T": T_out, "Y": Y_out, "status": status, "substeps": substeps, "Z": Z, "zone": zone,
            "mapped": mapped, "ref": ref}
