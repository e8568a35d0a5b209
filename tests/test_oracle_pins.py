"""Pins of the CPU oracle to things other than itself: order conditions and
published node sums, closed-form solutions, conservation laws, Gibbs-minimum
equilibrium, LAPACK, complex-step derivatives, thermodynamic identities, and a
tight-tolerance brute-force integration. Each test names what fixes it.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.optimize

import mechs
from paper_2112_05834_gb300 import synth

RC = 8.31446261815324e7
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ tableau
def _order_conditions(alpha, gam, b):
    """Residuals of the Rosenbrock (ROW) order conditions up to order 4 for a method
    with constant diagonal gamma (Hairer & Wanner II, Sec. IV.7, Table 7.1), with
    beta_ij = alpha_ij + gamma_ij (j < i), alpha_i = sum_j alpha_ij, beta'_i = sum_j beta_ij."""
    g = gam[0, 0]
    beta = alpha + np.tril(gam, -1)
    ai = alpha.sum(axis=1)
    bp = beta.sum(axis=1)
    return np.array([
        b.sum() - 1.0,
        b @ bp - (0.5 - g),
        b @ ai ** 2 - 1.0 / 3.0,
        b @ (beta @ bp) - (1.0 / 6.0 - g + g * g),
        b @ ai ** 3 - 0.25,
        (b * ai) @ (alpha @ bp) - (1.0 / 8.0 - g / 3.0),
        b @ (beta @ ai ** 2) - (1.0 / 12.0 - g / 3.0),
        b @ (beta @ (beta @ bp)) - (1.0 / 24.0 - g / 2.0 + 1.5 * g * g - g ** 3),
    ])


def test_rodas4_order_conditions(oracle_lib):
    alpha, gam, b, bhat = oracle_lib.tableau()
    main = _order_conditions(alpha, gam, b)
    emb = _order_conditions(alpha, gam, bhat)
    assert np.abs(main).max() < 1e-14, main          # order 4
    assert np.abs(emb[:4]).max() < 1e-14, emb        # embedded order 3 ...
    assert np.abs(emb[4:]).max() > 1e-4              # ... and not 4 (a genuine error estimate)
    # constant diagonal, lower triangular
    np.testing.assert_allclose(np.diag(gam), 0.25, rtol=0, atol=1e-15)
    assert np.all(np.triu(alpha) == 0) and np.all(np.triu(gam, 1) == 0)
    # stiffly accurate: b_j = beta_6j (j < 6), b_6 = gamma; bhat_j = beta_5j, bhat_5 = gamma
    beta = alpha + np.tril(gam, -1)
    np.testing.assert_allclose(b[:5], beta[5, :5], atol=1e-13)
    np.testing.assert_allclose(bhat[:4], beta[4, :4], atol=1e-13)
    assert abs(b[5] - 0.25) < 1e-13 and abs(bhat[4] - 0.25) < 1e-13 and abs(bhat[5]) < 1e-13


def test_rodas4_published_nodes(oracle_lib):
    ref = json.load(open(os.path.join(GOLDEN, "rodas4_nodes.json")))
    alpha, gam, b, bhat = oracle_lib.tableau()
    np.testing.assert_allclose(alpha.sum(axis=1), ref["alpha_i"], atol=1e-13)
    np.testing.assert_allclose(gam.sum(axis=1), ref["gamma_i"], atol=1e-13)


def test_rodas4_empirical_local_order(oracle_lib):
    """Local error of one step against a 256-substep reference on a smooth nonlinear
    problem: slope ~5 for the order-4 solution and ~4 for the order-3 embedded one."""
    M = oracle_lib.Mech(mechs.dimerization())
    y0 = np.array([1000.0, 0.6, 0.4, 0.0])
    p = 1e6
    hs = [2e-5 * 2.0 ** -k for k in range(1, 5)]
    em, ee = [], []
    for h in hs:
        y1, yh = oracle_lib.rodas_step(M, p, y0, h)
        y = y0.copy()
        for _ in range(256):
            y, _ = oracle_lib.rodas_step(M, p, y, h / 256)
        em.append(np.abs(y1 - y)[1:].max())
        ee.append(np.abs(yh - y)[1:].max())
    sm = np.polyfit(np.log(hs), np.log(em), 1)[0]
    se = np.polyfit(np.log(hs), np.log(ee), 1)[0]
    assert 4.6 < sm < 5.4, (sm, em)
    assert 3.6 < se < 4.4, (se, ee)


def _w_order_conditions(alpha, gam, b):
    """Residuals of the order conditions up to order 3 of a W-method (W any matrix in
    place of the Jacobian). Expanding the stages k_i = h f(y0 + sum alpha_ij k_j) +
    h W sum_{j<=i} gamma_ij k_j in powers of h, with a_i = sum_j alpha_ij and
    g_i = sum_{j<=i} gamma_ij: order h^2 carries f'f (weight b.a) and W f (b.g), order
    h^3 carries f''(f,f) (b.a^2 / 2), f'f'f (b A a), f'W f (b A g), W f'f (b G a) and
    W W f (b G g). Every term containing W must vanish and the others must match the
    exact solution's Taylor series (1, 1/2, 1/6 (f''(f,f) + f'f'f))."""
    A = np.tril(alpha, -1)
    a = A.sum(axis=1)
    g = gam.sum(axis=1)
    return np.array([b.sum() - 1.0, b @ a - 0.5, b @ g,
                     b @ a ** 2 - 1.0 / 3.0, b @ (A @ a) - 1.0 / 6.0, b @ (A @ g), b @ (gam @ a), b @ (gam @ g)])


def test_ros34pw2_order_conditions(oracle_lib):
    """ROS34PW2 (Rang & Angermann 2005): W-order 3 for the main solution and W-order 2
    (and not 3) for the embedded one; hence also Rosenbrock order 3 with the exact
    Jacobian; stiffly accurate (b = last row of alpha + Gamma); L-stable, with gamma the
    root of 6 g^3 - 18 g^2 + 9 g - 1 near 0.4359 (R(z) -> 0 as z -> -inf)."""
    alpha, gam, b, bhat, q = oracle_lib.tableau_of("ros34pw2")
    assert alpha.shape == (4, 4) and q == 3.0
    main = _w_order_conditions(alpha, gam, b)
    emb = _w_order_conditions(alpha, gam, bhat)
    assert np.abs(main).max() < 1e-14, main
    assert np.abs(emb[:3]).max() < 1e-14, emb
    assert np.abs(emb[3:]).max() > 1e-3
    assert np.abs(_order_conditions(alpha, gam, b)[:4]).max() < 1e-14
    g = gam[0, 0]
    np.testing.assert_allclose(np.diag(gam), g, rtol=0, atol=0)
    assert abs(6 * g ** 3 - 18 * g ** 2 + 9 * g - 1) < 1e-14 and abs(g - 0.4358665215) < 1e-10
    beta = alpha + gam
    np.testing.assert_allclose(b, beta[3], atol=1e-15)
    # stability function at -infinity: R = 1 - b^T (alpha + Gamma)^-1 1
    r_inf = 1.0 - b @ np.linalg.solve(beta, np.ones(4))
    assert abs(r_inf) < 1e-13
    # RODAS4 is not a W-method: already the order-2 W condition b.g = 0 fails
    a4, g4, b4, _, _ = oracle_lib.tableau_of("rodas4")
    assert abs(_w_order_conditions(a4, g4, b4)[2]) > 1e-2


def test_w_method_keeps_its_order_with_a_wrong_jacobian(oracle_lib):
    """Local error of one step with W = J + E, E a fixed random matrix of 30 % of |J|'s
    largest entry, against 256 RODAS4 substeps with the exact Jacobian, on the smooth
    dimerisation problem: ROS34PW2 keeps slopes ~4 (order 3) and ~3 (embedded order 2),
    RODAS4 falls to ~2 (order 1)."""
    M = oracle_lib.Mech(mechs.dimerization())
    y0 = np.array([1000.0, 0.6, 0.4, 0.0])
    p = 1e6
    J = oracle_lib.jac(M, p, y0)
    E = np.random.default_rng(0).standard_normal(J.shape) * 0.3 * np.abs(J).max()
    hs = [2e-5 * 2.0 ** -k for k in range(1, 6)]

    def slopes(method):
        em, ee = [], []
        for h in hs:
            y1, yh = oracle_lib.row_step(M, p, y0, h, method, E)
            y = y0.copy()
            for _ in range(256):
                y, _ = oracle_lib.row_step(M, p, y, h / 256, "rodas4")
            em.append(np.abs(y1 - y)[1:].max())
            ee.append(np.abs(yh - y)[1:].max())
        return np.polyfit(np.log(hs), np.log(em), 1)[0], np.polyfit(np.log(hs), np.log(ee), 1)[0]

    sm, se = slopes("ros34pw2")
    assert abs(sm - 4.0) < 0.3 and abs(se - 3.0) < 0.3, (sm, se)
    sm4, _ = slopes("rodas4")
    assert abs(sm4 - 2.0) < 0.3, sm4


# ------------------------------------------------------------------ thermo / rates
def test_thermo_identities(oracle_lib):
    """d(H/R)/dT = cp/R, d(S/R)/dT = cp/(R T) (central differences), including across
    the T_mid branch of a mechanism whose high-T coefficients differ."""
    m = mechs.with_high_branch(synth.mechanism_preset("c_54"))
    M = oracle_lib.Mech(m)
    for T in (400.0, 999.0, 1001.0, 1700.0, 2900.0):
        d = 1e-3
        cp, h, s = oracle_lib.thermo(M, T)
        _, hp, sp = oracle_lib.thermo(M, T + d)
        _, hm, sm = oracle_lib.thermo(M, T - d)
        dH = ((T + d) * hp - (T - d) * hm) / (2 * d)
        dS = (sp - sm) / (2 * d)
        np.testing.assert_allclose(dH, cp, rtol=1e-8)
        np.testing.assert_allclose(dS * T, cp, rtol=1e-8)
    # branch: continuity of H and S at T_mid, cp jumps
    cpl, hl, sl = oracle_lib.thermo(M, 1000.0 - 1e-9)
    cph, hh, sh = oracle_lib.thermo(M, 1000.0)
    np.testing.assert_allclose(hl, hh, rtol=1e-10)
    np.testing.assert_allclose(sl, sh, rtol=1e-10)
    assert np.all(np.abs(cph - cpl) > 0.1)


def _troe_consts(Fcent):
    lF = np.log10(Fcent)
    return lF, -0.4 - 0.67 * lF, 0.75 - 1.27 * lF


@pytest.mark.parametrize("T", [700.0, 1300.0, 2100.0])
def test_troe_special_points(oracle_lib, T):
    """Gilbert-Luther-Troe broadening (Chemkin theory manual): F = Fcent where
    log10 Pr = -c; F = sqrt(Fcent) where log10 Pr + c = n'/1.14; Lindemann (F = 1)
    reaches k0 [M] as Pr -> 0 and k_inf as Pr -> inf."""
    tr = (0.6, 300.0, 1500.0, 4000.0)
    m = mechs.falloff_single("troe", troe=tr)
    M = oracle_lib.Mech(m)
    kinf = m.A[0] * T ** m.b[0] * np.exp(-m.Ea_R[0] / T)
    k0 = m.A0[0] * T ** m.b0[0] * np.exp(-m.Ea0_R[0] / T)
    Fcent = (1 - tr[0]) * np.exp(-T / tr[1]) + tr[0] * np.exp(-T / tr[2]) + np.exp(-tr[3] / T)
    lF, c, nn = _troe_consts(Fcent)
    eff = m.eff[0]
    for target_L, F_expect in ((-c, Fcent), (nn / 1.14 - c, np.sqrt(Fcent))):
        Pr = 10.0 ** target_L
        Mtot = Pr * kinf / k0
        Cc = np.array([Mtot / eff[0], 0.0, 0.0, 0.0])  # [M] carried by the bath
        kf, kr, q = oracle_lib.rates_conc(M, T, Cc)
        np.testing.assert_allclose(kf[0], kinf * Pr / (1 + Pr) * F_expect, rtol=1e-12)
    ml = oracle_lib.Mech(mechs.falloff_single("lindemann"))
    for Mtot, expect in ((1e-14, k0 * 1e-14), (1e14, kinf)):
        Cc = np.array([Mtot / eff[0], 0.0, 0.0, 0.0])
        kf, _, _ = oracle_lib.rates_conc(ml, T, Cc)
        np.testing.assert_allclose(kf[0], expect, rtol=1e-6)


def test_third_body_concentration(oracle_lib):
    """q of a third-body reaction scales with [M] = sum eps_k C_k (linear in each C_k
    of a species that does not react)."""
    m = mechs.isomerization("third_body", eff=(1.0, 2.5, 0.5))
    M = oracle_lib.Mech(m)
    T = 1200.0
    C1 = np.array([1e-5, 2e-6, 1e-6])
    C2 = C1.copy()
    C2[0] *= 3.0
    _, _, q1 = oracle_lib.rates_conc(M, T, C1)
    _, _, q2 = oracle_lib.rates_conc(M, T, C2)
    M1 = 1e-5 + 2.5 * 2e-6 + 0.5 * 1e-6
    M2 = 3e-5 + 2.5 * 2e-6 + 0.5 * 1e-6
    np.testing.assert_allclose(q2 / q1, M2 / M1, rtol=1e-13)


# ------------------------------------------------------------------ closed forms
@pytest.mark.parametrize("kind", ["elementary", "third_body"])
def test_isomerization_closed_form(oracle_lib, kind):
    """A <=> B with equal W and H (T and rho constant): Y_A(t) = Y_A^eq + (Y_A0 - Y_A^eq)
    exp(-(kf + kr) t) with Kc = exp(dS/R) (dnu = 0), kr = kf/Kc; the third-body form
    multiplies both by [M], constant here because A and B have equal efficiencies."""
    dS = 0.7
    # equal efficiencies for A and B keep [M] constant as A converts to B
    m = mechs.isomerization(kind, dS_R=dS, eff=(0.8, 1.7, 1.7))
    M = oracle_lib.Mech(m)
    T0, p = 1100.0, 2e6
    Y0 = np.array([0.5, 0.4, 0.1])
    rho = p / (RC * T0 * np.sum(Y0 / m.W))
    kf = m.A[0] * np.exp(-m.Ea_R[0] / T0)
    if kind == "third_body":
        kf *= np.sum(m.eff[0] * rho * Y0 / m.W)
    kr = kf / np.exp(dS)
    t = 3.0 / (kf + kr)
    Yeq = (Y0[1] + Y0[2]) * kr / (kf + kr)
    expect = Yeq + (Y0[1] - Yeq) * np.exp(-(kf + kr) * t)
    r = oracle_lib.integrate(M, [T0], [p], Y0[None], t, rtol=1e-12, atol=1e-16)
    assert r["status"][0] == 0
    np.testing.assert_allclose(r["Y"][0, 1], expect, rtol=1e-10)
    np.testing.assert_allclose(r["Y"][0, 1] + r["Y"][0, 2], Y0[1] + Y0[2], rtol=1e-13)
    np.testing.assert_allclose(r["T"][0], T0, rtol=1e-12)


def test_dimerization_closed_form(oracle_lib):
    """2A -> B, irreversible, thermo-neutral, at constant T and p. Per unit mass,
    dn_A/dt = -2 k c0 n_A^2 / n_tot with c0 = p/(Rc T), n_tot = n_A/2 + s,
    s = n_A0/2 + n_B0 + n_N2; integrating: (1/2) ln(n_A/n_A0) - s (1/n_A - 1/n_A0) = -2 k c0 t."""
    m = mechs.dimerization()
    M = oracle_lib.Mech(m)
    T, p = 1000.0, 1e6
    Y0 = np.array([0.5, 0.4, 0.1])
    n0 = Y0 / m.W
    k = m.A[0] * np.exp(-m.Ea_R[0] / T)
    c0 = p / (RC * T)
    s = n0[1] / 2 + n0[2] + n0[0]
    t = 4e-4
    g = lambda nA: 0.5 * np.log(nA / n0[1]) - s * (1 / nA - 1 / n0[1]) + 2 * k * c0 * t
    nA = scipy.optimize.brentq(g, 1e-12 * n0[1], n0[1], xtol=1e-30, rtol=1e-15)
    r = oracle_lib.integrate(M, [T], [p], Y0[None], t, rtol=1e-12, atol=1e-16)
    assert r["status"][0] == 0
    np.testing.assert_allclose(r["Y"][0, 1] / m.W[1], nA, rtol=1e-9)
    np.testing.assert_allclose(r["T"][0], T, rtol=1e-12)


# ------------------------------------------------------------------ Jacobian
def _jac_mechs():
    return {
        "h2_10": synth.mechanism_preset("h2_10"),
        "c_54": synth.mechanism_preset("c_54"),
        "falloff_mix": synth.gen_mechanism(5, ("C", "H", "O", "N"), 30, 120, n_third_body=10,
                                           n_troe=8, n_lindemann=8, Ea_R_max=30000.0),
        "branch": mechs.with_high_branch(synth.mechanism_preset("h2_10")),
        "troe_single": mechs.falloff_single("troe"),
    }


@pytest.mark.parametrize("name", list(_jac_mechs().keys()))
def test_jacobian_vs_complex_step_and_fd(oracle_lib, name):
    """Analytic J vs complex-step derivative of the RHS (entry-wise <= 1e-12 relative
    where |J_ij| > 1e-12 max|J|) and vs central differences (<= 1e-3 relative to
    |J_ij| + 1e-6 max|J|)."""
    m = _jac_mechs()[name]
    M = oracle_lib.Mech(m)
    if name == "troe_single":
        states = [(T, 5e6, np.array([0.7, 0.01, 0.2, 0.09])) for T in (800.0, 1200.0, 1700.0)]
    else:
        st = synth.gen_states(m, 6, seed=2, p=40e5, classes=synth.MIXED_CLASSES)
        states = list(zip(st.T, st.p, st.Y))
    for T, p, Y in states:
        y = np.concatenate([[T], Y])
        J = oracle_lib.jac(M, p, y)
        Jc = oracle_lib.jac_cstep(M, p, y)
        Jf = oracle_lib.jac_fd(M, p, y)
        nrm = np.abs(Jc).max()
        mask = np.abs(Jc) > 1e-12 * nrm
        rel = np.abs(J - Jc)[mask] / np.abs(Jc)[mask]
        assert rel.max() < 1e-12, (name, rel.max())
        assert np.all(np.abs(J - Jc)[~mask] <= 1e-12 * nrm)
        assert (np.abs(Jf - Jc) / (np.abs(Jc) + 1e-6 * nrm)).max() < 1e-3


# ------------------------------------------------------------------ LU
@pytest.mark.parametrize("n,cond", [(11, 1e2), (55, 1e3), (101, 1e6), (55, 1e12)])
def test_lu_matches_lapack(oracle_lib, n, cond):
    """Doolittle LU with partial pivoting vs LAPACK getrf (through SciPy): same row
    interchanges, same factors; solves have backward error ~ machine precision."""
    rng = np.random.default_rng(n)
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = U @ np.diag(np.logspace(0, -np.log10(cond), n)) @ V.T
    LU, piv, info = oracle_lib.lu_factor(A)
    assert info == 0
    lu_ref, piv_ref = scipy.linalg.lu_factor(A)
    np.testing.assert_array_equal(piv, piv_ref)
    # factors agree up to the rounding-order difference of LAPACK's blocked algorithm,
    # which grows with the conditioning of the trailing Schur complements
    if cond <= 1e6:
        np.testing.assert_allclose(LU, lu_ref, rtol=0,
                                   atol=1e-15 * n * np.sqrt(cond) * np.abs(lu_ref).max())
    # backward error of the factorisation: P A = L U to rounding
    L = np.tril(LU, -1) + np.eye(n)
    PA = A.copy()
    for k in range(n):
        PA[[k, piv[k]]] = PA[[piv[k], k]]
    assert np.abs(L @ np.triu(LU) - PA).max() <= 1e-15 * n * np.abs(A).max()
    b = rng.standard_normal(n)
    x = oracle_lib.lu_solve(LU, piv, b)
    res = np.abs(A @ x - b).max() / (np.abs(A).max() * np.abs(x).max())
    assert res < 1e-14 * n


def test_lu_tie_break_lowest_row(oracle_lib):
    """Equal |a_ik| candidates: the lowest row index is the pivot (LAPACK idamax)."""
    A = np.array([[1.0, 2.0, 3.0], [-4.0, 1.0, 0.5], [4.0, 7.0, 1.0]])
    _, piv, _ = oracle_lib.lu_factor(A)
    _, piv_ref = scipy.linalg.lu_factor(A)
    np.testing.assert_array_equal(piv, piv_ref)
    assert piv[0] == 1


def test_lu_singular_reports(oracle_lib):
    A = np.array([[1.0, 2.0], [2.0, 4.0]])
    _, _, info = oracle_lib.lu_factor(A)
    assert info == 2


# ------------------------------------------------------------------ integration laws
@pytest.mark.parametrize("name", ["h2_10_1k", "c54_65k"])
def test_conservation(oracle_lib, name):
    """Mass (sum Y = 1) and element conservation are linear invariants a Rosenbrock
    method preserves exactly up to rounding; the mass enthalpy is conserved by the
    ODE (T_ode within tolerance) and exactly by the recovered temperature."""
    m, st, dt = synth.workload(name, n_cells=12, state_seed=11)
    M = oracle_lib.Mech(m)
    r = oracle_lib.integrate(M, st.T, st.p, st.Y, dt, n_threads=4)
    assert np.all(r["status"] == 0)
    steps = r["substeps"][:, None]
    assert np.all(np.abs(r["Y"].sum(axis=1) - 1.0) <= 1e-13 * (1 + r["substeps"]))
    el0 = (st.Y / m.W) @ m.elem
    el1 = (r["Y"] / m.W) @ m.elem
    assert np.all(np.abs(el1 - el0) <= 1e-13 * (1 + steps) * np.abs(el0).max())
    for c in range(12):
        h0 = oracle_lib.enthalpy_mass(M, st.T[c], st.Y[c])
        h_ode = oracle_lib.enthalpy_mass(M, r["T_ode"][c], r["Y"][c])
        h_rec = oracle_lib.enthalpy_mass(M, r["T"][c], r["Y"][c])
        cpm = 1.5e7  # erg/(g K), order of the mixture heat capacity
        assert abs(h_ode - h0) <= 1e-6 * cpm * st.T[c]
        assert abs(h_rec - h0) <= 1e-10 * cpm * st.T[c]
        assert abs(r["T"][c] - r["T_ode"][c]) <= 1e-6 * st.T[c]


def test_relaxes_to_gibbs_equilibrium(oracle_lib):
    """A long adiabatic integration (10 s, rtol 1e-10) reaches the constant-(h, p)
    Gibbs minimum under the kinetic invariants: |dY| <= 1e-8 + 1e-6 Y, |dT| <= 1e-6 T.
    This pins the equilibrium constants (Gibbs energies, the (P0/Rc T)^dnu factor)
    and the temperature equation together."""
    from oracle import equilibrium

    m = synth.mechanism_preset("h2_10")
    M = oracle_lib.Mech(m)
    st = synth.gen_states(m, 3, seed=3, p=synth.ATM, classes=((1.0, "unreacted", 1500.0, 2200.0),))
    r = oracle_lib.integrate(M, st.T, st.p, st.Y, 10.0, rtol=1e-10, atol=1e-14, n_threads=3)
    assert np.all(r["status"] == 0)
    for c in range(3):
        Teq, Yeq = equilibrium.equilibrium_hp(m, st.T[c], st.p[c], st.Y[c])
        assert abs(r["T"][c] - Teq) <= 1e-6 * Teq
        assert np.all(np.abs(r["Y"][c] - Yeq) <= 1e-8 + 1e-6 * Yeq)


def test_tight_tolerance_brute_force(oracle_lib):
    """The oracle at rtol 1e-8 lies inside the parity bound (|dT|/T <= 1e-6,
    |dY| <= 1e-8 + 1e-5 Y) of the same cells integrated at rtol 1e-12."""
    for name, n, tight in (("h2_10_1k", 16, 1e-12), ("c100_262k", 8, 1e-12)):
        m, st, dt = synth.workload(name, n_cells=n, state_seed=21)
        M = oracle_lib.Mech(m)
        a = oracle_lib.integrate(M, st.T, st.p, st.Y, dt, rtol=1e-8, atol=1e-12, n_threads=4)
        b = oracle_lib.integrate(M, st.T, st.p, st.Y, dt, rtol=tight, atol=1e-16, n_threads=4)
        assert np.all(a["status"] == 0) and np.all(b["status"] == 0)
        assert np.all(np.abs(a["T"] - b["T"]) <= 1e-6 * b["T"])
        assert np.all(np.abs(a["Y"] - b["Y"]) <= 1e-8 + 1e-5 * np.abs(b["Y"]))


# ------------------------------------------------------------------ starting step, T recovery
def test_starting_step_closed_form(oracle_lib):
    """Hairer-Wanner starting step on the linear A <=> B problem, where every norm in the
    algorithm has a closed form: f = L y with the constant matrix L, so
    f(y0 + h_a f0) - f0 = h_a L f0."""
    m = mechs.isomerization("elementary", dS_R=0.7, A=2e7)
    M = oracle_lib.Mech(m)
    T0, p = 1100.0, 2e6
    Y0 = np.array([0.5, 0.4, 0.1])
    kf = m.A[0] * np.exp(-m.Ea_R[0] / T0)
    kr = kf / np.exp(0.7)
    L = np.array([[-kf, kr], [kf, -kr]])
    y0 = np.concatenate([[T0], Y0])
    f0 = np.concatenate([[0.0, 0.0], L @ Y0[1:]])
    rtol, atol, dt = 1e-8, 1e-12, 1e-3
    sc = atol + rtol * np.abs(y0)
    nrm = lambda v: np.sqrt(np.mean((v / sc) ** 2))
    d0, d1 = nrm(y0), nrm(f0)
    ha = min(0.01 * d0 / d1, dt)
    d2 = nrm(np.concatenate([[0.0, 0.0], ha * (L @ f0[2:])])) / ha
    hb = (0.01 / max(d1, d2)) ** 0.25
    expect = min(100 * ha, hb, dt)
    got = oracle_lib.h0(M, p, y0, dt, rtol, atol)
    np.testing.assert_allclose(got, expect, rtol=1e-10)
    # vanishing derivative (pure bath gas): the whole interval
    y_bath = np.array([T0, 1.0, 0.0, 0.0])
    assert oracle_lib.h0(M, p, y_bath, dt, rtol, atol) == dt


def test_temperature_recovery(oracle_lib):
    m = synth.mechanism_preset("c_54")
    M = oracle_lib.Mech(m)
    st = synth.gen_states(m, 4, seed=4, classes=synth.MIXED_CLASSES)
    for T, Y in zip(st.T, st.Y):
        h = oracle_lib.enthalpy_mass(M, T, Y)
        Tr = oracle_lib.recover_T(M, Y, h, T + 150.0)
        np.testing.assert_allclose(Tr, T, rtol=1e-11)
