"""GPU path vs the CPU oracle, element by element, through the C ABI.

Bound for integrated states (rtol 1e-8, atol 1e-12): |dT| <= 1e-6 T and
|dY_k| <= 1e-8 + 1e-5 |Y_k|, for the FP64 and the mixed-precision forms.
"""
import numpy as np
import pytest

import mechs
from paper_2112_05834_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-8, 1e-12


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_05834_gb300 import _build

    _build.build()
    import paper_2112_05834_gb300 as p

    p.load()
    return p


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=torch.float64)


def _assert_bound(T, Y, ref, what=""):
    dT = np.abs(T - ref["T"]) / ref["T"]
    dY = np.abs(Y - ref["Y"]) / (1e-8 + 1e-5 * np.abs(ref["Y"]))
    assert dT.max() <= 1e-6, f"{what}: max |dT|/T = {dT.max():.3e} at cell {np.argmax(dT)}"
    assert dY.max() <= 1.0, f"{what}: max |dY|/bound = {dY.max():.3e}"


def _mech_cases():
    return {
        "h2_10": synth.mechanism_preset("h2_10"),
        "c_54": synth.mechanism_preset("c_54"),
        "falloff_mix": synth.gen_mechanism(5, ("C", "H", "O", "N"), 30, 120, n_third_body=10,
                                           n_troe=8, n_lindemann=8, Ea_R_max=30000.0),
        "branch": mechs.with_high_branch(synth.mechanism_preset("c_32")),
    }


def _states(m, n=24, seed=3, p=40e5):
    st = synth.gen_states(m, n, seed=seed, p=p, classes=synth.MIXED_CLASSES)
    # add states straddling T_mid = 1000 K
    st.T[:4] = [999.9, 1000.0, 1000.1, 1300.0]
    return st


# ------------------------------------------------------------------ RHS / Jacobian / h0
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", list(_mech_cases().keys()))
def test_rhs_parity(pkg, orc, name, precision):
    """RHS vs the oracle; the mixed form (precision 1) evaluates the third-body sums in
    float-float arithmetic and must stay within the same 1e-11 relative bound."""
    m = _mech_cases()[name]
    st = _states(m)
    integ = pkg.Integrator(m, precision=precision)
    f = integ.eval_rhs(_dev(st.T), _dev(st.p), _dev(st.Y)).cpu().numpy()
    M = orc.Mech(m)
    nu = np.abs(m.net_stoich())
    for c in range(st.T.shape[0]):
        y = np.concatenate([[st.T[c]], st.Y[c]])
        fr = orc.rhs(M, st.p[c], y)
        _, _, q = orc.rates(M, st.p[c], y)
        rho = st.p[c] / (8.31446261815324e7 * st.T[c] * np.sum(st.Y[c] / m.W))
        gross = np.concatenate([[np.abs(fr[0])], m.W * (nu @ np.abs(q)) / rho])
        gross[0] = max(gross[0], np.abs(fr[0]))
        err = np.abs(f[c] - fr)
        assert np.all(err <= 1e-11 * (np.abs(fr) + gross) + 1e-300), (name, c, np.max(err / (np.abs(fr) + gross + 1e-300)))


@pytest.mark.parametrize("name", list(_mech_cases().keys()))
def test_jacobian_parity(pkg, orc, name):
    m = _mech_cases()[name]
    st = _states(m, n=12)
    M = orc.Mech(m)
    for precision, tol in ((0, 1e-10), (1, 1e-10), (2, 2e-5)):
        integ = pkg.Integrator(m, precision=precision)
        J = integ.eval_jacobian(_dev(st.T), _dev(st.p), _dev(st.Y)).cpu().numpy()
        for c in range(st.T.shape[0]):
            y = np.concatenate([[st.T[c]], st.Y[c]])
            Jr = orc.jac(M, st.p[c], y)
            row = np.abs(Jr).max(axis=1, keepdims=True) + 1e-300
            err = np.abs(J[c] - Jr) / (np.abs(Jr) + row)
            assert err.max() <= tol, (name, precision, c, err.max())


@pytest.mark.parametrize("name", list(_mech_cases().keys()))
def test_float_float_assembly_accuracy(pkg, orc, name):
    """The mixed form assembles the Jacobian in float-float arithmetic on the FP32 pipe
    (about 48 significant bits: one FP32 rounding would leave ~6e-8). Entry by entry,
    relative to |J| plus the row's largest entry, it must agree with the oracle to
    1e-11 and with the FP64 form's assembly to 1e-11: the accuracy RODAS4 needs of its
    Jacobian to keep its order, which a plain FP32 assembly (precision 2) does not have."""
    m = _mech_cases()[name]
    st = _states(m, n=12)
    M = orc.Mech(m)
    J = {}
    for precision in (0, 1):
        integ = pkg.Integrator(m, precision=precision)
        J[precision] = integ.eval_jacobian(_dev(st.T), _dev(st.p), _dev(st.Y)).cpu().numpy()
    worst = {"oracle": 0.0, "fp64": 0.0}
    for c in range(st.T.shape[0]):
        y = np.concatenate([[st.T[c]], st.Y[c]])
        Jr = orc.jac(M, st.p[c], y)
        row = np.abs(Jr).max(axis=1, keepdims=True) + 1e-300
        worst["oracle"] = max(worst["oracle"], (np.abs(J[1][c] - Jr) / (np.abs(Jr) + row)).max())
        worst["fp64"] = max(worst["fp64"], (np.abs(J[1][c] - J[0][c]) / (np.abs(Jr) + row)).max())
    print(name, "float-float assembly: max scaled error vs oracle %.2e, vs FP64 form %.2e" %
          (worst["oracle"], worst["fp64"]))
    assert worst["oracle"] <= 1e-11 and worst["fp64"] <= 1e-11, worst


def _large_gibbs_mechanism():
    """The 54-species mechanism with every formation enthalpy (NASA a6) scaled so the
    largest |a6| is 1.8e5 K: at 300 K the species' |G/RT| reach about 600. Scaling all
    a6 by one factor keeps each reaction's enthalpy sign, so reverse rates stay finite."""
    import copy

    m = copy.deepcopy(synth.mechanism_preset("c_54"))
    s = 1.8e5 / np.abs(m.nasa_lo[:, 5]).max()
    m.nasa_lo[:, 5] *= s
    m.nasa_hi[:, 5] *= s
    return m


def test_rhs_jacobian_large_gibbs_parity(pkg, orc):
    """Cells between 300 K and 2500 K of a mechanism whose species reach |G/RT| ~ 600
    at 300 K: the kernels' reverse-rate ratio (normally a product of per-species
    factors exp(+-G/RT), whose partial products would leave the double range here)
    must match the oracle's one exponential of the reaction's Gibbs energy change, for
    the RHS (1e-11) and the Jacobian (1e-10), FP64 and mixed forms. The mixed form
    assembles in float-float, whose exponent range is FP32's: entries below 2^-126
    (here whole rows of near-inert species at 300 K, next to entries of 1e14) become
    zero, so its Jacobian error is taken net of that floor (64 x 2^-126, against
    diagonal entries of the iteration matrix of at least 1/dt)."""
    m = _large_gibbs_mechanism()
    st = _states(m, n=16)
    st.T[:] = np.geomspace(300.0, 2500.0, 16)
    M = orc.Mech(m)
    g_rt = np.array([[orc.thermo(M, T)[1][k] - orc.thermo(M, T)[2][k] for k in range(m.n_species)]
                     for T in st.T[:2]])
    assert np.abs(g_rt).max() > 300.0  # the range the factor products cannot hold
    nu = np.abs(m.net_stoich())
    for precision in (0, 1):
        integ = pkg.Integrator(m, precision=precision)
        f = integ.eval_rhs(_dev(st.T), _dev(st.p), _dev(st.Y)).cpu().numpy()
        J = integ.eval_jacobian(_dev(st.T), _dev(st.p), _dev(st.Y)).cpu().numpy()
        assert np.all(np.isfinite(f)) and np.all(np.isfinite(J))
        for c in range(st.T.shape[0]):
            y = np.concatenate([[st.T[c]], st.Y[c]])
            fr = orc.rhs(M, st.p[c], y)
            _, _, q = orc.rates(M, st.p[c], y)
            rho = st.p[c] / (8.31446261815324e7 * st.T[c] * np.sum(st.Y[c] / m.W))
            gross = np.concatenate([[np.abs(fr[0])], m.W * (nu @ np.abs(q)) / rho])
            assert np.all(np.abs(f[c] - fr) <= 1e-11 * (np.abs(fr) + gross) + 1e-300), (precision, c)
            Jr = orc.jac(M, st.p[c], y)
            row = np.abs(Jr).max(axis=1, keepdims=True) + 1e-300
            floor = 64 * 2.0 ** -126 if precision == 1 else 0.0
            err = np.maximum(np.abs(J[c] - Jr) - floor, 0.0) / (np.abs(Jr) + row)
            assert err.max() <= 1e-10, (precision, c, err.max())


@pytest.mark.parametrize("name", ["h2_10", "c_54"])
def test_fd_jacobian_vs_oracle(pkg, orc, name):
    """Option jacobian = 1 (forward differences, FP64 form) against the oracle's
    analytical Jacobian: truncation (the quadratic and third-body terms) and rounding
    of a forward difference leave each entry within 5e-3 of its row's largest entry
    (the same difference quotient on the oracle's RHS: 2.8e-3 and 1.6e-3)."""
    m = _mech_cases()[name]
    st = _states(m, n=12)
    M = orc.Mech(m)
    integ = pkg.Integrator(m, precision=0, jacobian=1)
    J = integ.eval_jacobian(_dev(st.T), _dev(st.p), _dev(st.Y)).cpu().numpy()
    worst = 0.0
    for c in range(st.T.shape[0]):
        y = np.concatenate([[st.T[c]], st.Y[c]])
        Jr = orc.jac(M, st.p[c], y)
        row = np.abs(Jr).max(axis=1, keepdims=True) + 1e-300
        worst = max(worst, (np.abs(J[c] - Jr) / row).max())
    print(name, "forward-difference Jacobian: max error / row max", worst)
    assert worst <= 5e-3


@pytest.mark.parametrize("jacobian,pivoting", [(1, 1), (0, 0), (1, 0)])
def test_fd_and_naive_elimination_parity(pkg, orc, jacobian, pivoting):
    """The classical variants of the FP64 form (forward-difference Jacobian and/or
    Gaussian elimination without row interchanges) integrate within the parity bound."""
    for name, n in (("h2_10_1k", 200), ("c54_65k", 64)):
        m, st, dt, ref = _oracle_ref(orc, name, n)
        g = _run(pkg, m, st, dt, precision=0, jacobian=jacobian, pivoting=pivoting)
        assert np.all(g["status"] == 0)
        _assert_bound(g["T"], g["Y"], ref, f"{name} jacobian={jacobian} pivoting={pivoting}")


def test_starting_step_parity(pkg, orc):
    m = synth.mechanism_preset("c_54")
    st = _states(m, n=32)
    integ = pkg.Integrator(m)
    h = integ.eval_h0(_dev(st.T), _dev(st.p), _dev(st.Y), 1e-6, RTOL, ATOL).cpu().numpy()
    M = orc.Mech(m)
    for c in range(32):
        y = np.concatenate([[st.T[c]], st.Y[c]])
        np.testing.assert_allclose(h[c], orc.h0(M, st.p[c], y, 1e-6, RTOL, ATOL), rtol=1e-10)


# ------------------------------------------------------------------ elementary functions
def _ulp_err(y, x, fn):
    ref = fn(x.astype(np.longdouble))
    return np.abs((y.astype(np.longdouble) - ref) / ref).astype(np.float64)


def test_exp_accuracy(pkg):
    """The rate kernels' table-driven exponential against exp in extended precision:
    within 1 ulp over the table/polynomial range, the library's behaviour outside it."""
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.uniform(-671.9, 671.9, 200000), rng.uniform(-60.0, 40.0, 200000),
                        rng.uniform(-0.02, 0.02, 20000),
                        np.arange(-2000, 2001) * (np.log(2.0) / 32.0),  # table nodes
                        [0.0, -0.0, 1e-300, -1e-300, 671.9, -671.9]])
    y = pkg.eval_math("exp", _dev(x)).cpu().numpy()
    rel = _ulp_err(y, x, np.exp)
    print("exp: max relative error", rel.max())
    assert rel.max() <= 2.3e-16
    assert np.all(y[x == 0.0] == 1.0)
    # outside the reduced range: the library exponential (overflow, underflow, inf, NaN)
    xo = np.array([672.0, 700.0, 709.7, -700.0, 710.0, -800.0, np.inf, -np.inf, np.nan])
    yo = pkg.eval_math("exp", _dev(xo)).cpu().numpy()
    np.testing.assert_allclose(yo[:4], np.exp(xo[:4]), rtol=4e-16)
    assert yo[4] == np.inf and yo[5] == 0.0 and yo[6] == np.inf and yo[7] == 0.0 and np.isnan(yo[8])


def test_log_accuracy(pkg):
    """Table-driven logarithm: absolute error within 1 ulp of ln x plus a few ulp of
    the result over the arguments the rate kernels meet (T, F_cent, P_r) and across
    binades; the library's behaviour for zero, negative, subnormal, inf and NaN."""
    rng = np.random.default_rng(12)
    x = np.concatenate([rng.uniform(200.0, 6000.0, 200000), 10.0 ** rng.uniform(-300, 300, 200000),
                        rng.uniform(0.5, 2.0, 100000), 1.0 + np.arange(-64, 129) / 128.0,
                        [1.0, 2.0, 0.5, 1.0 + 2.0 ** -40, 1.0 - 2.0 ** -40, 2.2250738585072014e-308]])
    y = pkg.eval_math("log", _dev(x)).cpu().numpy()
    ref = np.log(x.astype(np.longdouble))
    err = np.abs(y.astype(np.longdouble) - ref).astype(np.float64)
    bound = 2.3e-16 * np.abs(ref.astype(np.float64)) + 2.3e-19
    print("log: max error / bound", (err / bound).max())
    assert np.all(err <= bound)
    assert y[x == 1.0][0] == 0.0
    xo = np.array([0.0, -1.0, 1e-310, np.inf, np.nan])
    yo = pkg.eval_math("log", _dev(xo)).cpu().numpy()
    assert yo[0] == -np.inf and np.isnan(yo[1]) and yo[3] == np.inf and np.isnan(yo[4])
    np.testing.assert_allclose(yo[2], np.log(1e-310), rtol=1e-15)


def test_rcp_accuracy(pkg):
    """Newton reciprocal: within 1 ulp of 1/x; IEEE division outside its range."""
    rng = np.random.default_rng(13)
    x = np.concatenate([10.0 ** rng.uniform(-290, 290, 200000) * rng.choice([-1.0, 1.0], 200000),
                        rng.uniform(1.0, 2.0, 100000), [1.0, -1.0, 3.0, 0.1]])
    y = pkg.eval_math("rcp", _dev(x)).cpu().numpy()
    rel = _ulp_err(y, x, lambda v: 1 / v)
    print("rcp: max relative error", rel.max())
    assert rel.max() <= 2.3e-16
    assert y[x == 1.0][0] == 1.0
    xo = np.array([0.0, -0.0, np.inf, np.nan, 1e-305, 1e305])
    yo = pkg.eval_math("rcp", _dev(xo)).cpu().numpy()
    assert yo[0] == np.inf and yo[1] == -np.inf and yo[2] == 0.0 and np.isnan(yo[3])
    np.testing.assert_allclose(yo[4:], 1 / xo[4:], rtol=2.3e-16)


def test_float_float_split(pkg):
    """The integer-operation split of a double into a float-float pair (the mixed
    form's assembly and refinement inputs), against its definition computed here
    from the bit pattern: hi = x with the low 29 mantissa bits cleared, lo = x - hi
    rounded to FP32 (exactly, where lo is an FP32 normal number; within one subnormal
    unit where it is not, the integer-to-float rounding coming before the scaling);
    in FP32's subnormal range hi = x truncated to a multiple of 2^-149 and lo = 0;
    |x| >= 2^128 gives (+-inf, 0), NaN gives NaN. The widening back to double that
    returns the parts is exact, subnormals included."""
    rng = np.random.default_rng(12)
    x = np.concatenate([10.0 ** rng.uniform(-45, 45, 200000) * rng.choice([-1.0, 1.0], 200000),
                        rng.uniform(-2.0, 2.0, 50000),
                        [2.0 ** -126, np.nextafter(2.0 ** -126, 0.0), 2.0 ** 128, np.nextafter(2.0 ** 128, 0.0),
                         -np.nextafter(2.0 ** 128, 0.0), 1.0, 1.5, -3.0, 2.0 - 2.0 ** -52, 0.0, -0.0,
                         np.inf, -np.inf, np.nan, 2.0 ** -100, 3.0 * 2.0 ** -100, 2.0 ** -149,
                         1.5 * 2.0 ** -140, -2.0 ** -127, 2.0 ** -150]])
    d = _dev(x)
    hi = pkg.eval_math("ff_hi", d).cpu().numpy()
    lo = pkg.eval_math("ff_lo", d).cpu().numpy()
    ax = np.abs(x)
    normal = (ax >= 2.0 ** -126) & (ax < 2.0 ** 128)
    u = x[normal].view(np.uint64)
    hi_ref = (u & ~np.uint64(0x1FFFFFFF)).view(np.float64)
    np.testing.assert_array_equal(hi[normal], hi_ref)
    rem = x[normal] - hi_ref  # exact in double
    lo_ref = rem.astype(np.float32).astype(np.float64)
    sub = np.abs(lo_ref) < 2.0 ** -126
    np.testing.assert_array_equal(lo[normal][~sub], lo_ref[~sub])
    assert np.all(np.abs(lo[normal][sub] - lo_ref[sub]) <= 2.0 ** -149)
    wide = normal & (ax >= 2.0 ** -100)
    assert np.all(np.abs(x[wide] - (hi[wide] + lo[wide])) <= 2.0 ** -48 * ax[wide])
    tiny = ax < 2.0 ** -126
    q = np.floor(ax[tiny] / 2.0 ** -149) * 2.0 ** -149 * np.sign(x[tiny])
    np.testing.assert_array_equal(hi[tiny], q)
    assert np.all(lo[tiny] == 0.0)
    big = (ax >= 2.0 ** 128) & ~np.isnan(x)
    assert np.all(hi[big] == np.sign(x[big]) * np.inf) and np.all(lo[big] == 0.0)
    assert np.isnan(hi[np.isnan(x)]).all()


# ------------------------------------------------------------------ LU
@pytest.mark.parametrize("dim,cond", [(3, 10.0), (55, 1e3), (60, 1e3), (101, 1e4), (128, 1e2)])
def test_lu_solve_parity(pkg, orc, dim, cond):
    rng = np.random.default_rng(dim)
    n_mat = 37
    A = np.empty((n_mat, dim, dim))
    for s in range(n_mat):
        U, _ = np.linalg.qr(rng.standard_normal((dim, dim)))
        V, _ = np.linalg.qr(rng.standard_normal((dim, dim)))
        A[s] = U @ np.diag(np.logspace(0, -np.log10(cond), dim)) @ V.T
    b = rng.standard_normal((n_mat, dim))
    ref = np.stack([orc.lu_solve(*orc.lu_factor(A[s])[:2], b[s]) for s in range(n_mat)])
    # the FP32-assembly form refines towards the FP32-rounded matrix
    A32 = A.astype(np.float32).astype(np.float64)
    ref32 = np.stack([orc.lu_solve(*orc.lu_factor(A32[s])[:2], b[s]) for s in range(n_mat)])
    for precision, ir, tol, r in ((0, 0, 1e-13, ref), (1, 3, 1e-12, ref), (1, 0, 1e-5, ref),
                                  (2, 3, 1e-12, ref32)):
        x, info = pkg.lu_solve_batched(_dev(A), _dev(b), precision=precision, ir_sweeps=ir)
        x = x.cpu().numpy()
        assert np.all(info.cpu().numpy() == 0)
        err = np.abs(x - r).max(axis=1) / np.abs(r).max(axis=1)
        assert err.max() <= tol * cond, (precision, ir, err.max())


def test_lu_singular(pkg):
    A = np.zeros((2, 4, 4))
    A[0] = np.eye(4)
    A[1] = np.eye(4)
    A[1, 2, 2] = 0.0
    b = np.ones((2, 4))
    x, info = pkg.lu_solve_batched(_dev(A), _dev(b))
    assert list(info.cpu().numpy()) == [0, 3]
    assert np.all(np.isnan(x.cpu().numpy()[1]))


# ------------------------------------------------------------------ integration
def _run(pkg, m, st, dt, **opt):
    integ = pkg.Integrator(m, **opt)
    T, p, Y = _dev(st.T), _dev(st.p), _dev(st.Y)
    integ.integrate(T, p, Y, dt, RTOL, ATOL)
    s = integ.stats(st.T.shape[0])
    torch.cuda.synchronize()
    out = {"T": T.cpu().numpy(), "Y": Y.cpu().numpy()}
    out.update({k: v.cpu().numpy() for k, v in s.items()})
    integ.close()
    return out


_REF_CACHE = {}


def _oracle_ref(orc, name, n, seed=1):
    key = (name, n, seed)
    if key not in _REF_CACHE:
        m, st, dt = synth.workload(name, n_cells=n, state_seed=seed)
        _REF_CACHE[key] = (m, st, dt, orc.integrate(m, st.T, st.p, st.Y, dt, RTOL, ATOL))
    return _REF_CACHE[key]


@pytest.mark.parametrize("name,n", [("h2_10_1k", 1000), ("c54_65k", 333), ("c100_262k", 161)])
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_integrate_parity(pkg, orc, name, n, precision):
    m, st, dt, ref = _oracle_ref(orc, name, n)
    assert np.all(ref["status"] == 0)
    g = _run(pkg, m, st, dt, precision=precision)
    assert np.all(g["status"] == 0)
    _assert_bound(g["T"], g["Y"], ref, f"{name} precision={precision}")
    ratio = g["substeps"].sum() / ref["substeps"].sum()
    print(f"{name} precision={precision}: substeps gpu/oracle = {ratio:.4f}, "
          f"rejects gpu {g['rejects'].sum()} oracle {ref['rejects'].sum()}")
    if precision in (0, 1):
        # the same method up to rounding: step counts agree closely
        assert abs(ratio - 1.0) <= 0.05, ratio


_W_REF = {}


def _oracle_w_ref(orc, name, n, seed=1):
    key = (name, n, seed)
    if key not in _W_REF:
        m, st, dt = synth.workload(name, n_cells=n, state_seed=seed)
        _W_REF[key] = orc.integrate(m, st.T, st.p, st.Y, dt, RTOL, ATOL, method="ros34pw2")
    return _W_REF[key]


@pytest.mark.parametrize("name,n", [("h2_10_1k", 1000), ("c54_65k", 333), ("c100_262k", 161)])
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_w_method_parity(pkg, orc, name, n, precision):
    """Option method = 1 (ROS34PW2 W-method) against the oracle's ROS34PW2 and its
    RODAS4, at the parity bound, for the FP64, mixed and FP32-assembly forms. With
    precision 0 and 1 (the same method up to rounding) the step totals agree with the
    oracle's; with precision 2 the FP32-assembled matrix is a W, and because the
    method's order does not rely on W being the exact Jacobian its step total stays
    within 5 % as well (RODAS4 in that form takes about 2.6 times as many)."""
    m, st, dt, ref4 = _oracle_ref(orc, name, n)
    refw = _oracle_w_ref(orc, name, n)
    assert np.all(refw["status"] == 0)
    g = _run(pkg, m, st, dt, precision=precision, method=1)
    assert np.all(g["status"] == 0)
    _assert_bound(g["T"], g["Y"], refw, f"{name} W-method precision={precision} vs oracle ROS34PW2")
    _assert_bound(g["T"], g["Y"], ref4, f"{name} W-method precision={precision} vs oracle RODAS4")
    ratio = g["substeps"].sum() / refw["substeps"].sum()
    print(f"{name} W-method precision={precision}: substeps gpu/oracle = {ratio:.4f} "
          f"(oracle RODAS4 / ROS34PW2 = {ref4['substeps'].sum() / refw['substeps'].sum():.3f}), "
          f"rejects gpu {g['rejects'].sum()} oracle {refw['rejects'].sum()}")
    assert abs(ratio - 1.0) <= 0.05, ratio


def test_w_method_starting_step(pkg, orc):
    """The starting step of method = 1 uses the exponent 1/3 (its embedded order + 1)."""
    m = synth.mechanism_preset("c_54")
    st = _states(m, n=16)
    integ = pkg.Integrator(m, method=1)
    h = integ.eval_h0(_dev(st.T), _dev(st.p), _dev(st.Y), 1e-6, RTOL, ATOL).cpu().numpy()
    M = orc.Mech(m)
    for c in range(16):
        y = np.concatenate([[st.T[c]], st.Y[c]])
        np.testing.assert_allclose(h[c], orc.h0(M, st.p[c], y, 1e-6, RTOL, ATOL, method="ros34pw2"), rtol=1e-10)


@pytest.mark.parametrize("precision", [0, 1])
def test_conservation_on_gpu(pkg, orc, precision):
    m, st, dt, ref = _oracle_ref(orc, "c54_65k", 333)
    g = _run(pkg, m, st, dt, precision=precision)
    print("precision", precision, "max |sum Y - 1| =", np.abs(g["Y"].sum(axis=1) - 1.0).max())
    steps = g["substeps"]
    assert np.all(np.abs(g["Y"].sum(axis=1) - 1.0) <= 1e-13 * (1 + steps))
    el0 = (st.Y / m.W) @ m.elem
    el1 = (g["Y"] / m.W) @ m.elem
    assert np.all(np.abs(el1 - el0) <= 1e-13 * (1 + steps[:, None]) * np.abs(el0).max())


def test_schedulers_bitwise_identical(pkg, orc):
    """Per-cell results do not depend on how cells are scheduled (plain launch,
    static persistent, queue) or on repetition."""
    m, st, dt, ref = _oracle_ref(orc, "c54_65k", 333)
    outs = [_run(pkg, m, st, dt, scheduler=s) for s in (0, 1, 2, 2)]
    for o in outs[1:]:
        np.testing.assert_array_equal(o["T"], outs[0]["T"])
        np.testing.assert_array_equal(o["Y"], outs[0]["Y"])
        np.testing.assert_array_equal(o["substeps"], outs[0]["substeps"])


@pytest.mark.parametrize("block", [64, 256])
def test_block_sizes(pkg, orc, block):
    m, st, dt, ref = _oracle_ref(orc, "c54_65k", 333)
    g = _run(pkg, m, st, dt, block=block, precision=1)
    _assert_bound(g["T"], g["Y"], ref, f"block={block}")


@pytest.mark.parametrize("block", [0, 128, 256])
@pytest.mark.parametrize("precision", [0, 1])
def test_block_sizes_101(pkg, orc, block, precision):
    """100 species (n = 101): the register Gauss-Jordan of 256-thread blocks, the
    shared-memory one of 128-thread blocks, and the automatic choice agree with the oracle."""
    m, st, dt, ref = _oracle_ref(orc, "c100_262k", 161)
    g = _run(pkg, m, st, dt, block=block, precision=precision)
    _assert_bound(g["T"], g["Y"], ref, f"block={block} precision={precision}")


def test_graph_replay(pkg, orc):
    m, st, dt, ref = _oracle_ref(orc, "h2_10_1k", 1000)
    integ = pkg.Integrator(m, graph=1)
    p = _dev(st.p)
    res = []
    for _ in range(3):
        T, Y = _dev(st.T), _dev(st.Y)
        integ.integrate(T, p, Y, dt, RTOL, ATOL)
        torch.cuda.synchronize()
        res.append((T.cpu().numpy(), Y.cpu().numpy()))
    for T, Y in res:
        _assert_bound(T, Y, ref, "graph")
    np.testing.assert_array_equal(res[0][0], res[2][0])


def test_host_entry_point(pkg, orc):
    m, st, dt, ref = _oracle_ref(orc, "h2_10_1k", 1000)
    integ = pkg.Integrator(m)
    T, Y = st.T.copy(), st.Y.copy()
    integ.integrate_host(T, st.p.copy(), Y, dt, RTOL, ATOL)
    g = _run(pkg, m, st, dt)
    np.testing.assert_array_equal(T, g["T"])
    np.testing.assert_array_equal(Y, g["Y"])


def test_multi_mechanism_single_launch(pkg, orc):
    """Four mechanisms (10, 32, 54, 100 species) in one launch give the same
    per-cell results as four separate calls with the same block size (the
    reduction layout depends on it), and match the oracle."""
    names = [("h2_10", 1e-5, synth.ATM), ("c_32", 1e-6, 60e5), ("c_54", 1e-6, 60e5), ("c_100", 1e-6, 40e5)]
    jobs, singles, host = [], [], []
    dt = 1e-6
    for i, (nm, _, p) in enumerate(names):
        m = synth.mechanism_preset(nm)
        st = synth.gen_states(m, 97 + i, seed=10 + i, p=p, classes=synth.MIXED_CLASSES)
        integ = pkg.Integrator(m, block=256)
        jobs.append((integ, _dev(st.T), _dev(st.p), _dev(st.Y)))
        singles.append(_run(pkg, m, st, dt, block=256))
        host.append((m, st))
    pkg.integrate_jobs(jobs, dt, RTOL, ATOL)
    torch.cuda.synchronize()
    for (integ, T, p, Y), s, (m, st) in zip(jobs, singles, host):
        np.testing.assert_array_equal(T.cpu().numpy(), s["T"])
        np.testing.assert_array_equal(Y.cpu().numpy(), s["Y"])
        sub = slice(0, 24)
        ref = orc.integrate(m, st.T[sub], st.p[sub], st.Y[sub], dt, RTOL, ATOL)
        _assert_bound(s["T"][sub], s["Y"][sub], ref, m.species[0])


def test_multi_mechanism_concurrent_launches(pkg):
    """Option job_launch = 1: one launch per job on streams forked from the caller's,
    each with its own handle's block size; per-cell results and statistics bitwise equal
    to separate calls, and work the caller enqueues afterwards on its stream sees them."""
    names = [("h2_10", synth.ATM), ("c_32", 60e5), ("c_54", 60e5), ("c_100", 40e5)]
    dt = 1e-6
    jobs, singles = [], []
    for i, (nm, p) in enumerate(names):
        m = synth.mechanism_preset(nm)
        st = synth.gen_states(m, 300 + 7 * i, seed=20 + i, p=p, classes=synth.MIXED_CLASSES)
        integ = pkg.Integrator(m, precision=1, job_launch=1 if i == 0 else 0)
        jobs.append((integ, _dev(st.T), _dev(st.p), _dev(st.Y)))
        singles.append(_run(pkg, m, st, dt, precision=1))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        pkg.integrate_jobs(jobs, dt, RTOL, ATOL, stream=s)
        sums = [Y.sum(dim=1) for (_, _, _, Y) in jobs]  # ordered after the jobs on s
    s.synchronize()
    for (integ, T, p, Y), r, sm in zip(jobs, singles, sums):
        np.testing.assert_array_equal(T.cpu().numpy(), r["T"])
        np.testing.assert_array_equal(Y.cpu().numpy(), r["Y"])
        np.testing.assert_array_equal(sm.cpu().numpy(), Y.sum(dim=1).cpu().numpy())
        st = integ.stats(T.shape[0])
        np.testing.assert_array_equal(st["substeps"].cpu().numpy(), r["substeps"])


# ------------------------------------------------------------------ edge cases
def test_edge_cases(pkg):
    m = synth.mechanism_preset("h2_10")
    st = synth.gen_states(m, 8, seed=4, classes=synth.MIXED_CLASSES)
    integ = pkg.Integrator(m)
    # zero cells: no-op
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    integ.integrate(e, e, torch.empty((0, m.n_species), dtype=torch.float64, device="cuda"), 1e-6)
    # invalid arguments
    T, p, Y = _dev(st.T), _dev(st.p), _dev(st.Y)
    with pytest.raises(pkg.ChemError):
        integ.integrate(T, p, Y, -1.0)
    with pytest.raises(pkg.ChemError):
        integ.integrate(T, p, Y, 1e-6, rtol=0.0)
    with pytest.raises(pkg.ChemError):
        integ.set_option("block", 96)
    # a non-finite cell is flagged and left alone; the others integrate
    Tn = st.T.copy()
    Tn[3] = np.nan
    T = _dev(Tn)
    integ.integrate(T, p, Y, 1e-6)
    s = integ.stats(8)
    status = s["status"].cpu().numpy()
    assert status[3] == pkg.CELL_NONFINITE and np.all(np.delete(status, 3) == pkg.CELL_OK)
    # step budget exhausted: MAX_STEPS, last accepted state kept (finite, normalised)
    integ.set_option("max_steps", 2)
    T, Y = _dev(st.T), _dev(st.Y)
    integ.integrate(T, p, Y, 1e-3)
    s = integ.stats(8)
    assert np.any(s["status"].cpu().numpy() == pkg.CELL_MAX_STEPS)
    assert np.all(np.isfinite(Y.cpu().numpy()))
    assert integ.totals()["failed"] > 0
    # final temperature outside [200, 6000] K
    integ.set_option("max_steps", 100000)
    Yn2 = np.zeros((1, m.n_species))
    Yn2[0, m.roles["inert"]] = 1.0
    T1 = _dev(np.array([6500.0]))
    integ.integrate(T1, _dev(np.array([synth.ATM])), _dev(Yn2), 1e-6)
    assert integ.stats(1)["status"].cpu().numpy()[0] == pkg.CELL_T_RANGE


# ------------------------------------------------------------------ full size, sampled
def test_full_size_sampled_parity(pkg, orc):
    """The 54-species / 65,536-cell workload in the benchmark's launch
    configuration (queue scheduler, mixed precision); sampled cells (per
    temperature class and the costliest) against the oracle."""
    m, st, dt = synth.workload("c54_65k")
    g = _run(pkg, m, st, dt, precision=1, scheduler=2)
    assert np.all(g["status"] == 0)
    rng = np.random.default_rng(0)
    pick = []
    for k in range(3):
        idx = np.flatnonzero(st.kind == k)
        pick.extend(rng.choice(idx, 8, replace=False))
    pick.extend(np.argsort(g["substeps"])[-8:])
    pick = np.unique(np.array(pick))
    ref = orc.integrate(m, st.T[pick], st.p[pick], st.Y[pick], dt, RTOL, ATOL)
    _assert_bound(g["T"][pick], g["Y"][pick], ref, "c54 full size")
    np.testing.assert_allclose(g["Y"].sum(axis=1), 1.0, atol=1e-10)


@pytest.mark.parametrize("ir", [1, 2, 3])
def test_full_size_c100_mixed_sampled_parity(pkg, orc, ir):
    """100-species / 520-reaction mechanism, 262,144 cells at 40 bar in the mixed form
    with 1, 2 and 3 refinement sweeps; sampled cells against the oracle."""
    m, st, dt = synth.workload("c100_262k")
    g = _run(pkg, m, st, dt, precision=1, scheduler=2, ir_sweeps=ir)
    assert np.all(g["status"] == 0)
    rng = np.random.default_rng(ir)
    pick = []
    for k in range(3):
        idx = np.flatnonzero(st.kind == k)
        pick.extend(rng.choice(idx, 6, replace=False))
    pick.extend(np.argsort(g["substeps"])[-6:])
    pick = np.unique(np.array(pick))
    ref = orc.integrate(m, st.T[pick], st.p[pick], st.Y[pick], dt, RTOL, ATOL)
    _assert_bound(g["T"][pick], g["Y"][pick], ref, f"c100 full size ir={ir}")
    print(f"c100 262k ir={ir}: substeps {g['substeps'].sum()}")


def test_autotune_picks_a_block_and_keeps_parity(pkg, orc, tmp_path, monkeypatch):
    """The autotuner times CTA size x matrix layout x resident CTAs per SM on a sample
    of the call's cells (copies) and keeps the fastest; the caller's cells are
    integrated once, within the bound, and the choice is cached (in the handle and in
    the cache file, one "key block ctas layout" line); a second handle reads the file
    instead of timing and integrates bitwise identically."""
    cache = tmp_path / "autotune.txt"
    monkeypatch.setenv("CHEM_AUTOTUNE_CACHE", str(cache))
    m, st, dt, ref = _oracle_ref(orc, "c54_65k", 333)
    g = _run(pkg, m, st, dt, precision=1, autotune=1)
    _assert_bound(g["T"], g["Y"], ref, "autotune")
    f = cache.read_text().split()
    assert len(f) == 4, f
    block, ctas, layout = int(f[1]), int(f[2]), int(f[3])
    assert block in (64, 128, 256) and 1 <= ctas <= 16 and layout in (0, 1)
    print("autotuned: block", block, "CTAs per SM", ctas, "matrix in", "global slot" if layout else "shared memory")
    g2 = _run(pkg, m, st, dt, precision=1, autotune=1)
    assert len(cache.read_text().split()) == 4  # read, not re-timed
    np.testing.assert_array_equal(g2["T"], g["T"])
    np.testing.assert_array_equal(g2["Y"], g["Y"])
