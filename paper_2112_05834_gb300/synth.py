"""Seeded synthetic inputs: reaction mechanisms and per-cell thermochemical states.

This module is the only code shared by the CUDA path and the CPU oracle. It
draws random numbers and does atom bookkeeping; it evaluates none of the
method's arithmetic (no thermodynamic polynomial, no rate, no Jacobian). Every
bound it promises (cp/R range, atom balance, element conservation of blended
states) holds by construction, not by evaluating the quantities.

The paper's workloads (a 54-species/269-reaction n-dodecane mechanism, GRI-3.0
methane chemistry, a 2D shear layer and the ECN Spray A LES; Results section)
are not available; these generators stand in for them with the same sizes and
the same kinds of structure: reversible elementary, third-body and Troe falloff
reactions over a C/H/O/N species set, and cells that are cold, igniting or burnt.

Units are cgs-molar: mol, cm^3, s, K, erg; pressure in dyn/cm^2.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

ATOMIC_MASS = {"C": 12.011, "H": 1.008, "O": 15.999, "N": 14.007}

ATM = 1.01325e6  # dyn/cm^2
BAR = 1.0e6      # dyn/cm^2

# Reaction types, in the order the C-ABI uses.
RXN_ELEMENTARY, RXN_THIRD_BODY, RXN_LINDEMANN, RXN_TROE = 0, 1, 2, 3


@dataclass
class Mechanism:
    """Struct-of-arrays reaction mechanism (the layout the C-ABI takes).

    Reactants/products are stored as up to two (species index, stoichiometric
    coefficient) slots per side; index -1 marks an empty slot. A species that
    appears twice on one side (2A) is one slot with coefficient 2.
    """

    species: list
    elements: list
    W: np.ndarray          # [K] g/mol, sum of atomic masses
    elem: np.ndarray       # [K, E] int32 atom counts
    nasa_lo: np.ndarray    # [K, 7]
    nasa_hi: np.ndarray    # [K, 7]
    T_lo: np.ndarray       # [K]
    T_mid: np.ndarray      # [K]
    T_hi: np.ndarray       # [K]
    rxn_type: np.ndarray   # [I] int32
    reac_idx: np.ndarray   # [I, 2] int32
    reac_nu: np.ndarray    # [I, 2] int32
    prod_idx: np.ndarray   # [I, 2] int32
    prod_nu: np.ndarray    # [I, 2] int32
    reversible: np.ndarray  # [I] int32
    A: np.ndarray          # [I] high-pressure (or only) pre-exponential, cgs
    b: np.ndarray          # [I] temperature exponent
    Ea_R: np.ndarray       # [I] activation temperature, K
    A0: np.ndarray         # [I] low-pressure limit (falloff only)
    b0: np.ndarray         # [I]
    Ea0_R: np.ndarray      # [I]
    troe: np.ndarray       # [I, 4] alpha, T***, T*, T**
    eff: np.ndarray        # [I, K] third-body efficiencies
    roles: dict = field(default_factory=dict)

    @property
    def n_species(self) -> int:
        return len(self.species)

    @property
    def n_reactions(self) -> int:
        return int(self.rxn_type.shape[0])

    @property
    def n_elements(self) -> int:
        return len(self.elements)

    def net_stoich(self) -> np.ndarray:
        """[K, I] net stoichiometric matrix (products minus reactants)."""
        K, I = self.n_species, self.n_reactions
        nu = np.zeros((K, I), dtype=np.int64)
        for i in range(I):
            for s in range(2):
                if self.reac_idx[i, s] >= 0:
                    nu[self.reac_idx[i, s], i] -= self.reac_nu[i, s]
                if self.prod_idx[i, s] >= 0:
                    nu[self.prod_idx[i, s], i] += self.prod_nu[i, s]
        return nu

    def arrays(self) -> dict:
        """Contiguous arrays keyed by the C-ABI field names."""
        out = {}
        for name in ("W", "nasa_lo", "nasa_hi", "T_lo", "T_mid", "T_hi", "A", "b", "Ea_R",
                     "A0", "b0", "Ea0_R", "troe", "eff"):
            out[name] = np.ascontiguousarray(getattr(self, name), dtype=np.float64)
        for name in ("elem", "rxn_type", "reac_idx", "reac_nu", "prod_idx", "prod_nu",
                     "reversible"):
            out[name] = np.ascontiguousarray(getattr(self, name), dtype=np.int32)
        return out


# --------------------------------------------------------------------------
# species sets
# --------------------------------------------------------------------------

def _formula_name(counts: dict) -> str:
    return "".join(f"{e}{c if c > 1 else ''}" for e, c in counts.items() if c > 0)


# Formation-enthalpy offsets a6 (K) for the designated species; realistic orders of
# magnitude so that fuel + oxidiser -> products releases heat.
_CORE_A6 = {
    "N2": -1000.0, "O2": -1000.0, "H2": -900.0, "H2O": -29000.0, "CO2": -47600.0,
    "CO": -14300.0, "H": 25500.0, "O": 29000.0, "OH": 3500.0, "HO2": 300.0,
    "H2O2": -16500.0, "CH4": -9000.0,
}
_ATOM_H = {"H": 26000.0, "O": 30000.0, "C": 86000.0, "N": 57000.0}


def _core_species(atoms):
    """Designated species (formula dicts) always present, by role."""
    def f(**kw):
        return {e: kw.get(e, 0) for e in atoms}
    core = {
        "inert": ("N2", f(N=2)),
        "oxidizer": ("O2", f(O=2)),
        "H2": ("H2", f(H=2)),
        "H2O": ("H2O", f(H=2, O=1)),
        "H": ("H", f(H=1)),
        "O": ("O", f(O=1)),
        "OH": ("OH", f(H=1, O=1)),
        "HO2": ("HO2", f(H=1, O=2)),
        "H2O2": ("H2O2", f(H=2, O=2)),
    }
    if "C" in atoms:
        core["fuel"] = ("CH4", f(C=1, H=4))
        core["CO2"] = ("CO2", f(C=1, O=2))
        core["CO"] = ("CO", f(C=1, O=1))
    else:
        core["fuel"] = core["H2"]
    return core


def _draw_nasa(rng, n_atoms: int):
    """NASA-7 coefficients with cp/R inside [2.5, 6] on 300-3000 K by construction.

    cp/R = a1 + a2 T + a3 T^2 + a4 T^3 + a5 T^4. Atoms get cp/R = 2.5 exactly.
    Otherwise a1 in [3, 4]; the non-negative a2, a3 terms add at most Delta <= 1.8
    at 3000 K; |a4 T^3| <= 0.1 and |a5 T^4| <= 0.05 there. Hence cp/R lies in
    [a1 - 0.15, a1 + Delta + 0.15], a subset of [2.85, 5.95].
    """
    a = np.zeros(7)
    if n_atoms == 1:
        a[0] = 2.5
    else:
        a1 = rng.uniform(3.0, 4.0)
        delta = rng.uniform(0.0, 1.8)
        u = rng.uniform(0.3, 1.0)
        a[0] = a1
        a[1] = delta * u / 3000.0
        a[2] = delta * (1.0 - u) / 3000.0 ** 2
        a[3] = rng.uniform(-1.0, 1.0) * 0.1 / 3000.0 ** 3
        a[4] = rng.uniform(-1.0, 1.0) * 0.05 / 3000.0 ** 4
    # a7: entropy constant, larger for larger molecules.
    a[6] = rng.uniform(-4.0, 8.0) + 1.5 * (n_atoms - 1)
    return a


def _species_set(rng, atoms, n_species):
    core = _core_species(atoms)
    names, formulas, roles = [], [], {}
    for role, (nm, fm) in core.items():
        if nm not in names:
            names.append(nm)
            formulas.append(fm)
        roles[role] = names.index(nm)
    if len(names) > n_species:
        raise ValueError(f"n_species={n_species} is below the {len(names)} designated species")
    reactive = [e for e in atoms if e != "N"]
    hmax = 3 if "C" not in atoms else 8
    cmax = 3 if "C" in atoms else 0
    pool = []
    for c in range(cmax + 1):
        for h in range(hmax + 1):
            for o in range(4):
                fm = {e: 0 for e in atoms}
                if "C" in atoms:
                    fm["C"] = c
                fm["H"], fm["O"] = h, o
                if sum(fm.values()) == 0:
                    continue
                if any(all(fm[e] == g[e] for e in atoms) for g in formulas):
                    continue
                pool.append(fm)
    need = n_species - len(names)
    if need > len(pool):
        raise ValueError("not enough distinct formulas for the requested species count")
    pick = rng.choice(len(pool), size=need, replace=False)
    for j in sorted(pick.tolist()):
        formulas.append(pool[j])
        names.append(_formula_name(pool[j]))
    del reactive
    return names, formulas, roles


# --------------------------------------------------------------------------
# mechanism generator
# --------------------------------------------------------------------------

def gen_mechanism(seed: int = 0, atoms=("H", "O", "N"), n_species: int = 10,
                  n_reactions: int = 25, n_third_body: int = 4, n_troe: int = 0,
                  n_lindemann: int = 0, A_range=(1e6, 1e14), b_range=(-1.0, 1.5),
                  Ea_R_max: float = 25000.0, eff_range=(0.5, 3.0)) -> Mechanism:
    """Seeded, atom-conserving, reversible synthetic mechanism.

    Every reaction has 1-2 reactant and 1-2 product species, balances every
    element, and is written in the direction whose enthalpy-offset sum
    (products minus reactants of a6) is negative, so that reverse rates obtained
    from equilibrium constants stay bounded. N2 is inert: it enters only as a
    collision partner.
    """
    rng = np.random.default_rng(seed)
    atoms = tuple(atoms)
    names, formulas, roles = _species_set(rng, atoms, n_species)
    K = len(names)
    E = len(atoms)
    elem = np.array([[fm[e] for e in atoms] for fm in formulas], dtype=np.int32)
    W = np.array([sum(fm[e] * ATOMIC_MASS[e] for e in atoms) for fm in formulas])
    n_atoms = elem.sum(axis=1)

    nasa = np.zeros((K, 7))
    for k in range(K):
        nasa[k] = _draw_nasa(rng, int(n_atoms[k]))
        nm = names[k]
        if nm in _CORE_A6:
            nasa[k, 5] = _CORE_A6[nm]
        else:
            bond = rng.uniform(45000.0, 60000.0)
            a6 = sum(formulas[k][e] * _ATOM_H[e] for e in atoms) - (n_atoms[k] - 1) * bond
            nasa[k, 5] = float(np.clip(a6 + rng.uniform(-5000.0, 5000.0), -6.0e4, 6.0e4))

    # Candidate atom-balanced (reactants, products) pairs among reactive species.
    reactive = [k for k in range(K) if k != roles["inert"]]
    groups = {}
    for r in range(1, 3):
        for combo in itertools.combinations_with_replacement(reactive, r):
            key = tuple(int(x) for x in elem[list(combo)].sum(axis=0))
            groups.setdefault(key, []).append(combo)
    pairs = []
    for combos in groups.values():
        for a, b_ in itertools.combinations(combos, 2):
            pairs.append((a, b_))
    if len(pairs) < n_reactions:
        raise ValueError(f"only {len(pairs)} atom-balanced pairs for {n_reactions} reactions")
    # Association/dissociation pairs (2 <-> 1 species) carry third-body and falloff forms.
    assoc = [j for j, (a, b_) in enumerate(pairs) if {len(a), len(b_)} == {1, 2}]
    other = [j for j, (a, b_) in enumerate(pairs) if {len(a), len(b_)} != {1, 2}]
    n_pressure = n_third_body + n_troe + n_lindemann
    n_assoc = min(len(assoc), max(n_pressure, int(round(0.35 * n_reactions))))
    n_assoc = min(n_assoc, n_reactions)
    pick_assoc = list(rng.choice(len(assoc), size=n_assoc, replace=False)) if n_assoc else []
    rest = n_reactions - n_assoc
    picked = set(int(j) for j in pick_assoc)
    pool_other = other + [assoc[j] for j in range(len(assoc)) if j not in picked]
    pick_other = list(rng.choice(len(pool_other), size=rest, replace=False)) if rest else []
    chosen = [pairs[assoc[j]] for j in pick_assoc] + [pairs[pool_other[j]] for j in pick_other]
    is_assoc = [True] * n_assoc + [False] * rest

    I = n_reactions
    rxn_type = np.zeros(I, dtype=np.int32)
    reac_idx = -np.ones((I, 2), dtype=np.int32)
    prod_idx = -np.ones((I, 2), dtype=np.int32)
    reac_nu = np.zeros((I, 2), dtype=np.int32)
    prod_nu = np.zeros((I, 2), dtype=np.int32)
    A = np.zeros(I)
    b = np.zeros(I)
    Ea_R = np.zeros(I)
    A0 = np.zeros(I)
    b0 = np.zeros(I)
    Ea0_R = np.zeros(I)
    troe = np.zeros((I, 4))
    eff = np.ones((I, K))

    # Pressure-dependent forms go to association reactions first, then to others.
    types = [RXN_THIRD_BODY] * n_third_body + [RXN_TROE] * n_troe + [RXN_LINDEMANN] * n_lindemann
    if len(types) > I:
        raise ValueError("more pressure-dependent reactions than reactions")
    assoc_slots = [j for j in range(I) if is_assoc[j]]
    other_slots = [j for j in range(I) if not is_assoc[j]]
    slots = ([assoc_slots[j] for j in rng.permutation(len(assoc_slots))]
             + [other_slots[j] for j in rng.permutation(len(other_slots))])
    for t, j in zip(types, slots):
        rxn_type[j] = t

    stable = {roles[r] for r in ("fuel", "oxidizer", "H2O", "H2") if r in roles}
    for r in ("CO2", "CO"):
        if r in roles:
            stable.add(roles[r])

    def side(combo):
        idx, nu = [-1, -1], [0, 0]
        uniq = sorted(set(combo))
        for s, k in enumerate(uniq):
            idx[s] = int(k)
            nu[s] = int(combo.count(k))
        return idx, nu

    for i, (ra, pa) in enumerate(chosen):
        dh = sum(nasa[k, 5] for k in pa) - sum(nasa[k, 5] for k in ra)
        if dh > 0:  # write in the exothermic direction
            ra, pa = pa, ra
        reac_idx[i], reac_nu[i] = side(ra)
        prod_idx[i], prod_nu[i] = side(pa)
        A[i] = np.exp(rng.uniform(np.log(A_range[0]), np.log(A_range[1])))
        b[i] = rng.uniform(*b_range)
        # Reactions between two stable molecules are slow (high activation temperature).
        if len(ra) == 2 and all(k in stable for k in ra):
            Ea_R[i] = rng.uniform(0.5, 1.0) * Ea_R_max
        else:
            Ea_R[i] = rng.uniform(0.0, Ea_R_max)
        if rxn_type[i] in (RXN_THIRD_BODY, RXN_LINDEMANN, RXN_TROE):
            eff[i] = rng.uniform(*eff_range, size=K)
        if rxn_type[i] in (RXN_LINDEMANN, RXN_TROE):
            A0[i] = A[i] * np.exp(rng.uniform(np.log(1e2), np.log(1e6)))
            b0[i] = rng.uniform(*b_range)
            Ea0_R[i] = Ea_R[i] * rng.uniform(0.0, 1.0)
        if rxn_type[i] == RXN_TROE:
            troe[i, 0] = rng.uniform(0.3, 0.9)
            troe[i, 1:4] = np.exp(rng.uniform(np.log(1e1), np.log(1e4), size=3))

    T_lo = np.full(K, 300.0)
    T_mid = np.full(K, 1000.0)
    T_hi = np.full(K, 3000.0)
    return Mechanism(
        species=names, elements=list(atoms), W=W, elem=elem,
        nasa_lo=nasa.copy(), nasa_hi=nasa.copy(), T_lo=T_lo, T_mid=T_mid, T_hi=T_hi,
        rxn_type=rxn_type, reac_idx=reac_idx, reac_nu=reac_nu, prod_idx=prod_idx,
        prod_nu=prod_nu, reversible=np.ones(I, dtype=np.int32), A=A, b=b, Ea_R=Ea_R,
        A0=A0, b0=b0, Ea0_R=Ea0_R, troe=troe, eff=eff, roles=roles)


def mechanism_preset(name: str, seed: int = 0) -> Mechanism:
    """The synthetic mechanisms of the benchmark workloads, by size.

    ``h2_10``: 10 species, 25 reactions, H/O/N, 4 third-body, Ea/R <= 25000 K.
    ``c_32``, ``c_54``, ``c_100``: C/H/O/N with 5 (5.2 for 100) reactions per
    species, 20 % third-body, 10 % Troe falloff, Ea/R <= 40000 K.
    """
    if name == "h2_10":
        return gen_mechanism(seed, ("H", "O", "N"), 10, 25, n_third_body=4)
    sizes = {"c_32": (32, 160), "c_54": (54, 270), "c_100": (100, 520)}
    if name not in sizes:
        raise KeyError(name)
    K, I = sizes[name]
    return gen_mechanism(seed, ("C", "H", "O", "N"), K, I,
                         n_third_body=int(round(0.2 * I)), n_troe=int(round(0.1 * I)),
                         Ea_R_max=40000.0)


# --------------------------------------------------------------------------
# cell states
# --------------------------------------------------------------------------

def _mole_to_mass(X, W):
    m = X * W
    return m / m.sum(axis=-1, keepdims=True)


def unreacted_mixture(mech: Mechanism, ratio, x_inert=0.7):
    """Mass fractions of fuel/oxidiser/N2 mixtures; ratio = X_fuel / X_O2."""
    ratio = np.atleast_1d(np.asarray(ratio, dtype=np.float64))
    K = mech.n_species
    X = np.zeros((ratio.size, K))
    rest = 1.0 - x_inert
    X[:, mech.roles["inert"]] = x_inert
    X[:, mech.roles["fuel"]] += rest * ratio / (1.0 + ratio)
    X[:, mech.roles["oxidizer"]] += rest / (1.0 + ratio)
    return _mole_to_mass(X, mech.W)


def streams(mech: Mechanism, x_inert=0.7):
    """(Y_fuel, Y_ox): the pure fuel stream and the oxidiser stream O2/N2 with
    X_N2 = x_inert (the two streams whose mixing the mixture fraction measures)."""
    K = mech.n_species
    Xf = np.zeros(K)
    Xf[mech.roles["fuel"]] = 1.0
    Xo = np.zeros(K)
    Xo[mech.roles["inert"]] = x_inert
    Xo[mech.roles["oxidizer"]] = 1.0 - x_inert
    return _mole_to_mass(Xf, mech.W), _mole_to_mass(Xo, mech.W)


def burnt_products(mech: Mechanism, Y):
    """Complete-combustion products of mixtures Y (atom bookkeeping only).

    Atoms per unit mass are conserved exactly: N -> N2; C -> CO then CO2 and
    H -> H2O as far as oxygen allows (C to CO first, then H to H2O, then CO to
    CO2); left-over O -> O2, left-over H -> H2, left-over C stays as CO only if
    oxygen allows (generated fuels never leave bare carbon).
    """
    Y = np.atleast_2d(Y)
    el = list(mech.elements)
    moles = Y / mech.W  # species mol per gram
    atoms = moles @ mech.elem  # [N, E] element mol per gram
    K = mech.n_species
    out = np.zeros((Y.shape[0], K))
    r = mech.roles
    for c in range(Y.shape[0]):
        a = dict(zip(el, atoms[c]))
        n = np.zeros(K)
        if "N" in a:
            n[r["inert"]] += a["N"] / 2.0
        o = a.get("O", 0.0)
        h = a.get("H", 0.0)
        cc = a.get("C", 0.0)
        co = min(cc, o)
        o -= co
        h2o = min(h / 2.0, o)
        o -= h2o
        co2 = min(co, o)
        o -= co2
        co -= co2
        if "CO2" in r:
            n[r["CO2"]] += co2
            n[r["CO"]] += co
        n[r["H2O"]] += h2o
        n[r["H2"]] += (h - 2.0 * h2o) / 2.0
        n[r["oxidizer"]] += o / 2.0
        out[c] = n * mech.W
    return out / out.sum(axis=1, keepdims=True)


@dataclass
class CellStates:
    T: np.ndarray   # [N] K
    p: np.ndarray   # [N] dyn/cm^2
    Y: np.ndarray   # [N, K] mass fractions
    kind: np.ndarray  # [N] int8: 0 unreacted/cold, 1 igniting, 2 burnt, 3 oxidiser


def gen_states(mech: Mechanism, n_cells: int, seed: int = 1, p: float = ATM,
               classes=((1.0, "unreacted", 1000.0, 1800.0),), ratio_range=(0.5, 2.0),
               x_inert: float = 0.7, shuffle: bool = True) -> CellStates:
    """Seeded cell states at constant pressure.

    ``classes`` is a sequence of (fraction, kind, T_low, T_high) with kind in
    {"unreacted", "igniting", "burnt"}:
    unreacted = fuel/O2/N2 with X_fuel/X_O2 ~ U(ratio_range) and X_N2 = x_inert;
    burnt = complete-combustion products blended with the unreacted mixture
    at a weight <= 1e-3; igniting = convex blend (1-c) unreacted + c burnt with
    c ~ U[0.1, 0.9]; oxidiser = the oxidiser stream of ``streams`` blended with
    the unreacted mixture at a weight <= 1e-4 (the air side of a mixing layer,
    mixture fraction near 0). Blends are in mass fractions, so element mass
    fractions are those of the blended inputs. Cells are shuffled (seeded) so cost is
    spatially mixed, as in a decomposed CFD domain.
    """
    rng = np.random.default_rng(seed)
    kinds = {"unreacted": 0, "igniting": 1, "burnt": 2, "oxidiser": 3}
    fr = np.array([c[0] for c in classes], dtype=np.float64)
    counts = np.floor(fr / fr.sum() * n_cells).astype(np.int64)
    counts[0] += n_cells - counts.sum()
    T_all, Y_all, k_all = [], [], []
    for (frac, kind, tlo, thi), m in zip(classes, counts):
        if m == 0:
            continue
        ratio = rng.uniform(*ratio_range, size=m)
        Yu = unreacted_mixture(mech, ratio, x_inert)
        if kind == "unreacted":
            Y = Yu
        elif kind == "oxidiser":
            w = rng.uniform(0.0, 1e-4, size=(m, 1))
            Y = (1.0 - w) * streams(mech, x_inert)[1] + w * Yu
        else:
            Yb = burnt_products(mech, Yu)
            if kind == "burnt":
                w = rng.uniform(0.0, 1e-3, size=(m, 1))
                Y = (1.0 - w) * Yb + w * Yu
            elif kind == "igniting":
                c = rng.uniform(0.1, 0.9, size=(m, 1))
                Y = (1.0 - c) * Yu + c * Yb
            else:
                raise ValueError(kind)
        T_all.append(rng.uniform(tlo, thi, size=m))
        Y_all.append(Y)
        k_all.append(np.full(m, kinds[kind], dtype=np.int8))
    T = np.concatenate(T_all) if T_all else np.zeros(0)
    Y = np.concatenate(Y_all) if Y_all else np.zeros((0, mech.n_species))
    kind = np.concatenate(k_all) if k_all else np.zeros(0, dtype=np.int8)
    if shuffle and n_cells > 0:
        perm = rng.permutation(n_cells)
        T, Y, kind = T[perm], Y[perm], kind[perm]
    return CellStates(T=np.ascontiguousarray(T), p=np.full(n_cells, float(p)),
                      Y=np.ascontiguousarray(Y), kind=kind)


MIXED_CLASSES = ((0.6, "unreacted", 700.0, 900.0), (0.3, "igniting", 1000.0, 1600.0),
                 (0.1, "burnt", 2000.0, 2700.0))

# the mixed classes beside an oxidiser zone of 40 % of the cells at 800 +- 5 K
OXZONE_CLASSES = ((0.4, "oxidiser", 795.0, 805.0), (0.36, "unreacted", 700.0, 900.0),
                  (0.18, "igniting", 1000.0, 1600.0), (0.06, "burnt", 2000.0, 2700.0))


def perturb_states(states: CellStates, seed: int, dT: float = 50.0, w_max: float = 0.1,
                   T_range=(300.0, 3000.0)):
    """Mixing perturbation between CFD steps: T += U[-dT, dT], reflected at the ends of
    T_range (the NASA fits' range: over many steps the perturbation is a random walk,
    which would otherwise carry a few of a million cells out of it);
    Y <- (1 - w) Y + w Y_partner with a seeded random partner cell and w ~ U[0, w_max]."""
    rng = np.random.default_rng(seed)
    n = states.T.shape[0]
    T = states.T + rng.uniform(-dT, dT, size=n)
    lo, hi = T_range
    T = np.where(T < lo, 2.0 * lo - T, T)
    T = np.where(T > hi, 2.0 * hi - T, T)
    partner = rng.integers(0, n, size=n)
    w = rng.uniform(0.0, w_max, size=(n, 1))
    Y = (1.0 - w) * states.Y + w * states.Y[partner]
    return CellStates(T=np.ascontiguousarray(T), p=states.p.copy(), Y=np.ascontiguousarray(Y),
                      kind=states.kind.copy())


# --------------------------------------------------------------------------
# workloads (sizes of the benchmark configurations)
# --------------------------------------------------------------------------

WORKLOADS = {
    # name: (mechanism preset, n_cells, pressure, classes, dt)
    "h2_10_1k": ("h2_10", 1024, ATM, ((1.0, "unreacted", 1000.0, 1800.0),), 1e-5),
    "c54_65k": ("c_54", 65536, 60 * BAR, MIXED_CLASSES, 1e-6),
    "c54_262k": ("c_54", 262144, 60 * BAR, MIXED_CLASSES, 1e-6),
    "c54_65k_oxzone": ("c_54", 65536, 60 * BAR, OXZONE_CLASSES, 1e-6),
    "c100_262k": ("c_100", 262144, 40 * BAR, MIXED_CLASSES, 1e-6),
    "c100_1m": ("c_100", 1048576, 40 * BAR, MIXED_CLASSES, 1e-6),
}


def workload(name: str, n_cells: int | None = None, mech_seed: int = 0, state_seed: int = 1):
    """(mechanism, states, dt) for a named workload, optionally with fewer cells."""
    preset, n, p, classes, dt = WORKLOADS[name]
    mech = mechanism_preset(preset, mech_seed)
    st = gen_states(mech, n if n_cells is None else n_cells, seed=state_seed, p=p, classes=classes)
    return mech, st, dt
