"""Pins of the reference-mapping oracle (oracle/refmap.py) to what Bilger's definition
and the selection rule fix, independent of the oracle's own formulas.

- beta = 0 at stoichiometry: a stoichiometric fuel/O2 mixture (fuel C_x H_y O_z with
  x + y/4 - z/2 moles of O2) and its complete-combustion products (CO2, H2O) have a
  zero coupling function, for the H2 and the CH4 mechanisms; rich mixtures positive,
  lean ones negative. A wrong weight, sign or element column fails here.
- Z = 0 on the oxidiser, 1 on the fuel, and w on a mass-fraction blend (Z is linear).
- Z is conserved by the oracle's integration (Bilger's Z is a conserved scalar of
  element-balanced kinetics).
- The selection rule by hand on small cases (zone boundary inclusive, NaN excluded,
  lowest-index reference, temperature window, empty zone).
- A zone cell identical to the reference ends where the reference (and its own plain
  integration) ends; mapped cells keep their Z and sum of Y; a failed reference maps
  nothing (mapped cells keep their initial state and take its status).
"""
import numpy as np
import pytest

from paper_2112_05834_gb300 import synth

rm = pytest.importorskip("oracle.refmap")


def _fuel_formula(m):
    el = list(m.elements)
    k = m.roles["fuel"]
    return {e: int(m.elem[k, el.index(e)]) if e in el else 0 for e in ("C", "H", "O")}


@pytest.mark.parametrize("preset", ["h2_10", "c_54"])
def test_beta_zero_at_stoichiometry(preset):
    m = synth.mechanism_preset(preset)
    f = _fuel_formula(m)
    nu_o2 = f["C"] + f["H"] / 4.0 - f["O"] / 2.0
    assert nu_o2 > 0
    K = m.n_species
    for x_n2 in (0.0, 3.76 * nu_o2):
        X = np.zeros(K)
        X[m.roles["fuel"]] = 1.0
        X[m.roles["oxidizer"]] = nu_o2
        X[m.roles["inert"]] = x_n2
        Y = X * m.W / (X * m.W).sum()
        b = rm.coupling_beta(m, Y)[0]
        ze = rm.element_mass_fractions(m, Y)
        scale = sum(abs(v) for v in ze.values())
        assert abs(b) <= 1e-15 * scale + 1e-18, (x_n2, b)
        # complete-combustion products of the same mixture
        Yb = synth.burnt_products(m, Y)[0]
        assert abs(rm.coupling_beta(m, Yb)[0]) <= 1e-15 * scale + 1e-18
        # rich / lean
        for fac, sign in ((0.5, 1.0), (2.0, -1.0)):
            X2 = X.copy()
            X2[m.roles["oxidizer"]] = fac * nu_o2
            Y2 = X2 * m.W / (X2 * m.W).sum()
            assert np.sign(rm.coupling_beta(m, Y2)[0]) == sign


@pytest.mark.parametrize("preset", ["h2_10", "c_54"])
def test_Z_streams_and_blends(preset):
    m = synth.mechanism_preset(preset)
    yf, yo = synth.streams(m)
    assert rm.mixture_fraction(m, yf, yf, yo)[0] == pytest.approx(1.0, abs=1e-14)
    assert rm.mixture_fraction(m, yo, yf, yo)[0] == pytest.approx(0.0, abs=1e-14)
    w = np.array([0.0, 1e-6, 0.03, 0.5, 0.97, 1.0])
    Y = (1.0 - w)[:, None] * yo + w[:, None] * yf
    np.testing.assert_allclose(rm.mixture_fraction(m, Y, yf, yo), w, rtol=1e-12, atol=1e-14)


def test_Z_conserved_by_integration(oracle_lib):
    m, st, dt = synth.workload("c54_65k", n_cells=6, state_seed=4)
    yf, yo = synth.streams(m)
    r = oracle_lib.integrate(m, st.T, st.p, st.Y, dt)
    assert np.all(r["status"] == 0)
    Z0 = rm.mixture_fraction(m, st.Y, yf, yo)
    Z1 = rm.mixture_fraction(m, r["Y"], yf, yo)
    np.testing.assert_allclose(Z1, Z0, rtol=0, atol=1e-12)


def test_select_by_hand():
    Z = np.array([0.5, 1e-5, 2e-5, 3e-4, 0.0, 1e-4, np.nan, -5e-5])
    T = np.array([800.0, 800.0, 801.5, 800.0, 803.0, 799.0, 800.0, 802.0])
    zone, ref, mapped = rm.select(Z, T, 0.0, 1e-4, 2.0)
    assert zone.tolist() == [False, True, True, False, True, True, False, True]
    assert ref == 1
    assert np.flatnonzero(mapped).tolist() == [2, 5, 7]
    # a zone around another centre; the lowest zone index is the reference
    zone, ref, mapped = rm.select(Z, T, 0.5, 0.01, 0.0)
    assert np.flatnonzero(zone).tolist() == [0] and ref == 0 and not mapped.any()
    # empty zone
    zone, ref, mapped = rm.select(Z, T, 0.9, 1e-3, 2.0)
    assert ref == -1 and not zone.any() and not mapped.any()
    # T_tol = 0: only cells at exactly T_ref are mapped
    zone, ref, mapped = rm.select(Z, T, 0.0, 1e-4, 0.0)
    assert np.flatnonzero(mapped).tolist() == []


def test_identical_cell_takes_the_reference_result(oracle_lib):
    m, st, dt = synth.workload("c54_65k_oxzone", n_cells=40, state_seed=5)
    yf, yo = synth.streams(m)
    zc = np.flatnonzero(st.kind == 3)
    assert zc.size >= 3
    r0 = zc[0]
    T, Y = st.T.copy(), st.Y.copy()
    T[zc[2]], Y[zc[2]] = T[r0], Y[r0]  # a copy of the reference cell
    res = rm.integrate_mapped(m, T, st.p, Y, dt, yf, yo, 0.0, 1e-4, 2.0)
    assert res["ref"] == r0 and res["mapped"][zc[2]]
    plain = oracle_lib.integrate(m, T[[r0]], st.p[[r0]], Y[[r0]], dt)
    assert res["T"][zc[2]] == pytest.approx(plain["T"][0], rel=1e-14)
    np.testing.assert_allclose(res["Y"][zc[2]], plain["Y"][0], rtol=0, atol=1e-15)
    assert res["substeps"][zc[2]] == 0 and res["substeps"][r0] > 0


def test_mapped_cells_keep_Z_and_sum(oracle_lib):
    m, st, dt = synth.workload("c54_65k_oxzone", n_cells=48, state_seed=6)
    yf, yo = synth.streams(m)
    res = rm.integrate_mapped(m, st.T, st.p, st.Y, dt, yf, yo, 0.0, 1e-4, 5.0)
    mp = res["mapped"]
    assert mp.sum() >= 3
    Z1 = rm.mixture_fraction(m, res["Y"][mp], yf, yo)
    np.testing.assert_allclose(Z1, res["Z"][mp], rtol=0, atol=1e-12)
    np.testing.assert_allclose(res["Y"][mp].sum(axis=1), st.Y[mp].sum(axis=1), rtol=0, atol=1e-13)
    # the integrated cells are exactly the plain oracle's
    solve = np.flatnonzero(~mp)
    plain = oracle_lib.integrate(m, st.T[solve], st.p[solve], st.Y[solve], dt)
    assert np.array_equal(res["T"][solve], plain["T"])
    assert np.array_equal(res["Y"][solve], plain["Y"])


def test_failed_reference_leaves_mapped_cells(oracle_lib):
    """A reference that fails (step budget of one step) maps nothing: the mapped cells keep
    their initial state and take the reference's status."""
    m, st, dt = synth.workload("c54_65k_oxzone", n_cells=40, state_seed=5)
    yf, yo = synth.streams(m)
    res = rm.integrate_mapped(m, st.T, st.p, st.Y, dt, yf, yo, 0.0, 1e-4, 10.0, max_steps=1)
    mp, r = res["mapped"], res["ref"]
    assert r >= 0 and mp.sum() >= 3
    assert res["status"][r] != 0
    assert np.all(res["status"][mp] == res["status"][r])
    assert np.array_equal(res["Y"][mp], st.Y[mp]) and np.array_equal(res["T"][mp], st.T[mp])
