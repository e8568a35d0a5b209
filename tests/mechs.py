"""Small hand-built mechanisms with closed-form behaviour, for pinning the oracle
and for GPU-vs-oracle parity on special cases."""
from __future__ import annotations

import numpy as np

from paper_2112_05834_gb300.synth import ATOMIC_MASS, Mechanism


def build(species, formulas, nasa, reactions, elements=("C", "H", "O", "N")):
    """species: names; formulas: list of dicts; nasa: [K,7] (lo = hi, T_mid 1000 K);
    reactions: list of dicts with keys reac [(k, nu)], prod [(k, nu)], type, A, b, Ea_R,
    optional A0, b0, Ea0_R, troe (4), eff (K), reversible."""
    K = len(species)
    I = len(reactions)
    elem = np.array([[f.get(e, 0) for e in elements] for f in formulas], dtype=np.int32)
    W = np.array([sum(f.get(e, 0) * ATOMIC_MASS[e] for e in elements) for f in formulas])
    nasa = np.asarray(nasa, dtype=np.float64)
    ri = -np.ones((I, 2), np.int32)
    rn = np.zeros((I, 2), np.int32)
    pi = -np.ones((I, 2), np.int32)
    pn = np.zeros((I, 2), np.int32)
    arr = {k: np.zeros(I) for k in ("A", "b", "Ea_R", "A0", "b0", "Ea0_R")}
    troe = np.zeros((I, 4))
    eff = np.ones((I, K))
    typ = np.zeros(I, np.int32)
    rev = np.ones(I, np.int32)
    for i, r in enumerate(reactions):
        for s, (k, nu) in enumerate(r["reac"]):
            ri[i, s], rn[i, s] = k, nu
        for s, (k, nu) in enumerate(r["prod"]):
            pi[i, s], pn[i, s] = k, nu
        typ[i] = r.get("type", 0)
        rev[i] = r.get("reversible", 1)
        for k in arr:
            arr[k][i] = r.get(k, 0.0)
        if "troe" in r:
            troe[i] = r["troe"]
        if "eff" in r:
            eff[i] = r["eff"]
    return Mechanism(
        species=list(species), elements=list(elements), W=W, elem=elem, nasa_lo=nasa.copy(),
        nasa_hi=nasa.copy(), T_lo=np.full(K, 300.0), T_mid=np.full(K, 1000.0),
        T_hi=np.full(K, 3000.0), rxn_type=typ, reac_idx=ri, reac_nu=rn, prod_idx=pi, prod_nu=pn,
        reversible=rev, A=arr["A"], b=arr["b"], Ea_R=arr["Ea_R"], A0=arr["A0"], b0=arr["b0"],
        Ea0_R=arr["Ea0_R"], troe=troe, eff=eff, roles={"inert": 0})


def isomerization(kind="elementary", dS_R=0.7, A=2.0e5, Ea_R=3000.0, eff=(1.0, 2.5, 0.5)):
    """N2 bath + isomers A, B (same formula written as two species, same W, same
    H; S differs by dS_R). A <=> B (elementary) or A + M <=> B + M (third body)."""
    base = [3.5, 1e-4, 0.0, 0.0, 0.0, -1000.0, 4.0]
    nA = [3.8, 2e-4, 1e-8, 0.0, 0.0, -5000.0, 6.0]
    nB = list(nA)
    nB[6] += dS_R
    r = {"reac": [(1, 1)], "prod": [(2, 1)], "type": 0 if kind == "elementary" else 1,
         "A": A, "b": 0.0, "Ea_R": Ea_R, "eff": np.array(eff, dtype=np.float64)}
    return build(["N2", "A", "B"], [{"N": 2}, {"C": 1, "H": 2, "O": 1}, {"C": 1, "H": 2, "O": 1}],
                 [base, nA, nB], [r])


def dimerization(A=5.0e9, Ea_R=2000.0):
    """N2 bath + 2A -> B, irreversible and thermo-neutral (NASA a1..a6 of B twice
    those of A, W_B = 2 W_A): T stays constant at constant pressure."""
    base = [3.5, 1e-4, 0.0, 0.0, 0.0, -1000.0, 4.0]
    nA = [3.6, 3e-4, 2e-8, 0.0, 0.0, 2000.0, 5.0]
    nB = [2 * a for a in nA[:6]] + [7.0]
    r = {"reac": [(1, 2)], "prod": [(2, 1)], "type": 0, "A": A, "b": 0.0, "Ea_R": Ea_R,
         "reversible": 0}
    return build(["N2", "A", "B"], [{"N": 2}, {"C": 1, "H": 1}, {"C": 2, "H": 2}],
                 [base, nA, nB], [r])


def falloff_single(kind="troe", troe=(0.6, 300.0, 1500.0, 4000.0), A=1e13, b=0.3, Ea_R=1200.0,
                   A0=1e17, b0=-0.8, Ea0_R=300.0, eff=(1.0, 1.3, 2.0, 0.7)):
    """N2 bath + X + Y <=> XY (+M) with a Lindemann or Troe falloff."""
    base = [3.5, 1e-4, 0.0, 0.0, 0.0, -1000.0, 4.0]
    nX = [2.5, 0.0, 0.0, 0.0, 0.0, 20000.0, 3.0]
    nY = [3.6, 2e-4, 0.0, 0.0, 0.0, 5000.0, 6.0]
    nXY = [4.2, 4e-4, 1e-8, 0.0, 0.0, -15000.0, 7.0]
    r = {"reac": [(1, 1), (2, 1)], "prod": [(3, 1)], "type": 3 if kind == "troe" else 2,
         "A": A, "b": b, "Ea_R": Ea_R, "A0": A0, "b0": b0, "Ea0_R": Ea0_R,
         "troe": np.array(troe, dtype=np.float64), "eff": np.array(eff, dtype=np.float64)}
    return build(["N2", "X", "Y", "XY"],
                 [{"N": 2}, {"H": 1}, {"C": 1, "H": 3}, {"C": 1, "H": 4}],
                 [base, nX, nY, nXY], [r])


def with_high_branch(mech, seed=7, delta=0.3):
    """Copy of ``mech`` whose high-temperature NASA coefficients differ from the low
    ones (a1 shifted by delta, a6 and a7 re-matched so that cp/R jumps but H/RT and
    S/R are continuous at T_mid). Used to exercise the T_mid branch."""
    import copy

    m = copy.deepcopy(mech)
    rng = np.random.default_rng(seed)
    Tm = m.T_mid
    for k in range(m.n_species):
        d = delta * rng.uniform(0.5, 1.0)
        hi = m.nasa_lo[k].copy()
        hi[0] += d
        # H/RT continuity: a6 term absorbs d * T_mid; S/R continuity: a7 absorbs d ln T_mid.
        hi[5] -= d * Tm[k]
        hi[6] -= d * np.log(Tm[k])
        m.nasa_hi[k] = hi
    return m
