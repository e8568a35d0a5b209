"""Reference mapping by mixture fraction on the GPU vs the oracle (oracle/refmap.py),
through the C ABI.

- Z per cell against Bilger's definition (FP64 both sides, different formulas).
- Mapped flags and the reference cell bit-exact against the oracle's selection
  (cells within rounding of a zone or temperature boundary are reported, and
  excluded only if present).
- Integrated and mapped cells within the parity bound |dT| <= 1e-6 T,
  |dY| <= 1e-8 + 1e-5 |Y| of the oracle's mapped step.
- Mapped cells bit-exact against the GPU reference's own change (the apply step).
- An empty zone leaves the call bitwise equal to an unmapped call; the work-order
  variants (graph replay, last-call cost order) give bitwise equal results.
"""
import numpy as np
import pytest

from paper_2112_05834_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-8, 1e-12
ZTOL, TTOL = 1e-4, 2.0


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
def rm():
    import oracle
    import oracle.refmap as r

    oracle.build()
    return r


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=torch.float64)


def _bound(T, Y, ref_T, ref_Y, what):
    dT = np.abs(T - ref_T) / ref_T
    dY = np.abs(Y - ref_Y) / (1e-8 + 1e-5 * np.abs(ref_Y))
    assert dT.max(initial=0.0) <= 1e-6, f"{what}: max |dT|/T = {dT.max():.3e}"
    assert dY.max(initial=0.0) <= 1.0, f"{what}: max |dY|/bound = {dY.max():.3e}"


def _run(pkg, m, st, dt, yf, yo, zc=0.0, ztol=ZTOL, ttol=TTOL, mapping=True, **opt):
    integ = pkg.Integrator(m, **opt)
    if mapping:
        integ.set_reference_mapping(yf, yo, zc, ztol, ttol)
    T, p, Y = _dev(st.T), _dev(st.p), _dev(st.Y)
    integ.integrate(T, p, Y, dt, RTOL, ATOL)
    stats = integ.stats(st.T.shape[0])
    out = {"T": T.cpu().numpy(), "Y": Y.cpu().numpy(),
           "substeps": stats["substeps"].cpu().numpy(), "status": stats["status"].cpu().numpy()}
    if mapping:
        mapped, nm, ref = integ.reference_mapping(st.T.shape[0])
        out.update(mapped=mapped.cpu().numpy().astype(bool), n_mapped=nm, ref=ref)
    return integ, out


def _near_boundary(Z, T, ref, zc, ztol, ttol):
    """Cells whose zone or temperature decision is within rounding of its boundary."""
    near = np.abs(np.abs(Z - zc) - ztol) <= 1e-12
    if ref >= 0:
        near |= np.abs(np.abs(T - T[ref]) - ttol) <= 1e-9
    return near


def test_mixture_fraction_matches_oracle(pkg, rm):
    for wl in ("c54_65k_oxzone", "h2_10_1k"):
        m, st, _ = synth.workload(wl, n_cells=777)
        yf, yo = synth.streams(m)
        integ = pkg.Integrator(m)
        integ.set_reference_mapping(yf, yo)
        Z = integ.mixture_fraction(_dev(st.Y)).cpu().numpy()
        Zo = rm.mixture_fraction(m, st.Y, yf, yo)
        np.testing.assert_allclose(Z, Zo, rtol=0, atol=1e-13)
        S = integ.mixture_fraction(_dev(np.stack([yf, yo]))).cpu().numpy()
        np.testing.assert_allclose(S, [1.0, 0.0], rtol=0, atol=1e-14)


@pytest.mark.parametrize("precision", [0, 1])
def test_refmap_parity(pkg, rm, precision):
    m, st, dt = synth.workload("c54_65k_oxzone", n_cells=400, state_seed=7)
    yf, yo = synth.streams(m)
    ref = rm.integrate_mapped(m, st.T, st.p, st.Y, dt, yf, yo, 0.0, ZTOL, TTOL, rtol=RTOL, atol=ATOL)
    near = _near_boundary(ref["Z"], st.T, ref["ref"], 0.0, ZTOL, TTOL)
    assert near.sum() == 0, f"{near.sum()} cells within rounding of a boundary"
    _, g = _run(pkg, m, st, dt, yf, yo, precision=precision)
    assert g["ref"] == ref["ref"]
    assert np.array_equal(g["mapped"], ref["mapped"])
    assert g["n_mapped"] == int(ref["mapped"].sum()) > 50
    mp = g["mapped"]
    assert np.all(g["substeps"][mp] == 0) and np.all(g["substeps"][~mp] > 0)
    assert np.all(g["status"] == 0) and np.all(ref["status"] == 0)
    _bound(g["T"][~mp], g["Y"][~mp], ref["T"][~mp], ref["Y"][~mp], "integrated cells")
    _bound(g["T"][mp], g["Y"][mp], ref["T"][mp], ref["Y"][mp], "mapped cells")
    # the apply step: initial state + the GPU reference's change, bit for bit
    r = g["ref"]
    np.testing.assert_array_equal(g["Y"][mp], st.Y[mp] + (g["Y"][r] - st.Y[r]))
    np.testing.assert_array_equal(g["T"][mp], st.T[mp] + (g["T"][r] - st.T[r]))


def test_refmap_empty_zone_equals_unmapped(pkg):
    m, st, dt = synth.workload("c54_65k_oxzone", n_cells=300, state_seed=8)
    yf, yo = synth.streams(m)
    integ, a = _run(pkg, m, st, dt, yf, yo, zc=0.5, ztol=1e-9, precision=1)
    assert a["n_mapped"] == 0 and a["ref"] == -1 and not a["mapped"].any()
    _, b = _run(pkg, m, st, dt, yf, yo, mapping=False, precision=1)
    assert np.array_equal(a["T"], b["T"]) and np.array_equal(a["Y"], b["Y"])
    assert np.array_equal(a["substeps"], b["substeps"])
    # a zone holding only the reference maps nothing either
    Z = integ.mixture_fraction(_dev(st.Y)).cpu().numpy()
    i = int(np.argmax(Z))
    _, c = _run(pkg, m, st, dt, yf, yo, zc=float(Z[i]), ztol=0.0, precision=1)
    assert c["n_mapped"] == 0 and c["ref"] == i
    assert np.array_equal(c["T"], b["T"]) and np.array_equal(c["Y"], b["Y"])


def test_refmap_work_order_variants(pkg):
    """Graph replay and the last-call cost order change only the work order."""
    m, st, dt = synth.workload("c54_65k_oxzone", n_cells=1500, state_seed=9)
    yf, yo = synth.streams(m)
    _, a = _run(pkg, m, st, dt, yf, yo, precision=1, block=128)
    integ = pkg.Integrator(m, precision=1, block=128, graph=1, order=2)
    integ.set_reference_mapping(yf, yo, 0.0, ZTOL, TTOL)
    for rep in range(3):  # capture, then cost order from the previous call, then replay
        T, p, Y = _dev(st.T), _dev(st.p), _dev(st.Y)
        integ.integrate(T, p, Y, dt, RTOL, ATOL)
        assert np.array_equal(T.cpu().numpy(), a["T"]), rep
        assert np.array_equal(Y.cpu().numpy(), a["Y"]), rep
        mapped, nm, ref = integ.reference_mapping(st.T.shape[0])
        assert nm == a["n_mapped"] and ref == a["ref"]
        assert np.array_equal(mapped.cpu().numpy().astype(bool), a["mapped"])
    # switched off: the next call integrates every cell
    integ.set_reference_mapping(yf, yo, 0.0, -1.0, TTOL)
    T, p, Y = _dev(st.T), _dev(st.p), _dev(st.Y)
    integ.integrate(T, p, Y, dt, RTOL, ATOL)
    assert np.all(integ.stats(st.T.shape[0])["substeps"].cpu().numpy() > 0)
    with pytest.raises(pkg.ChemError):
        integ.reference_mapping(st.T.shape[0])


def test_refmap_argument_errors(pkg):
    m, st, dt = synth.workload("c54_65k_oxzone", n_cells=64)
    yf, yo = synth.streams(m)
    integ = pkg.Integrator(m, scheduler=1)
    with pytest.raises(pkg.ChemError):
        integ.mixture_fraction(_dev(st.Y))  # no streams yet
    with pytest.raises(pkg.ChemError):
        integ.set_reference_mapping(yf, yf)  # equal streams
    with pytest.raises(pkg.ChemError):
        integ.set_reference_mapping(yf, yo, 0.0, float("nan"), 2.0)
    with pytest.raises(pkg.ChemError):
        integ.set_reference_mapping(yf, yo, 0.0, 1e-4, -1.0)
    integ.set_reference_mapping(yf, yo)
    T, p, Y = _dev(st.T), _dev(st.p), _dev(st.Y)
    with pytest.raises(pkg.ChemError):
        integ.integrate(T, p, Y, dt)  # static scheduler
    integ.set_option("scheduler", 2)
    lib = pkg.load()
    rc = lib.chem_integrate_noalloc(integ.h, st.T.shape[0], pkg._dptr(T), pkg._dptr(p), pkg._dptr(Y),
                                    dt, RTOL, ATOL, pkg._stream_ptr(None))
    assert rc == pkg.CHEM_ERR_INVALID_ARG
    other = pkg.Integrator(m)
    with pytest.raises(pkg.ChemError):
        pkg.integrate_jobs([(integ, T, p, Y), (other, _dev(st.T), _dev(st.p), _dev(st.Y))], dt)
    torch.cuda.synchronize()
    assert np.array_equal(T.cpu().numpy(), st.T)  # nothing ran


def test_refmap_full_size(pkg, rm):
    """65,536 cells with a 40 % oxidiser zone, mixed form: the selection equals the
    oracle's, sampled cells meet the bound, and mapping removes work."""
    m, st, dt = synth.workload("c54_65k_oxzone")
    yf, yo = synth.streams(m)
    n = st.T.shape[0]
    Z = rm.mixture_fraction(m, st.Y, yf, yo)
    zone, r, mapped = rm.select(Z, st.T, 0.0, ZTOL, TTOL)
    near = _near_boundary(Z, st.T, r, 0.0, ZTOL, TTOL)
    integ, g = _run(pkg, m, st, dt, yf, yo, precision=1)
    assert g["ref"] == r
    assert np.array_equal(g["mapped"][~near], mapped[~near])
    assert g["n_mapped"] == int(g["mapped"].sum()) > n // 10
    assert np.all(g["status"] == 0)
    _, b = _run(pkg, m, st, dt, yf, yo, mapping=False, precision=1)
    assert g["substeps"].sum() < b["substeps"].sum()
    ok = ~g["mapped"]
    assert np.array_equal(g["T"][ok], b["T"][ok]) and np.array_equal(g["Y"][ok], b["Y"][ok])
    rng = np.random.default_rng(0)
    sample = np.unique(np.concatenate([[r], rng.choice(np.flatnonzero(ok), 24, replace=False)]))
    import oracle

    o = oracle.integrate(m, st.T[sample], st.p[sample], st.Y[sample], dt, rtol=RTOL, atol=ATOL)
    _bound(g["T"][sample], g["Y"][sample], o["T"], o["Y"], "sampled integrated cells")
    mp = np.flatnonzero(g["mapped"])[:64]
    j = int(np.flatnonzero(sample == r)[0])
    _bound(g["T"][mp], g["Y"][mp], st.T[mp] + (o["T"][j] - st.T[r]), st.Y[mp] + (o["Y"][j] - st.Y[r]),
           "sampled mapped cells")


def test_refmap_many_tiles(pkg, rm):
    """1,100,000 hydrogen-mechanism cells (no carbon column): 1,075 partition tiles, so
    the tile-offset scan runs in two chunks of 1,024, and a ragged last tile. Every
    integrated cell is integrated once, every mapped cell is not, the selection equals
    the oracle's and the mapped cells carry the reference's change bit for bit."""
    m = synth.mechanism_preset("h2_10")
    n = 1_100_000
    st = synth.gen_states(m, n, seed=11, p=synth.ATM,
                          classes=((0.9, "oxidiser", 795.0, 805.0), (0.1, "unreacted", 700.0, 900.0)))
    yf, yo = synth.streams(m)
    Z = rm.mixture_fraction(m, st.Y, yf, yo)
    zone, r, mapped = rm.select(Z, st.T, 0.0, ZTOL, 10.0)
    near = _near_boundary(Z, st.T, r, 0.0, ZTOL, 10.0)
    integ = pkg.Integrator(m, precision=1)
    integ.set_reference_mapping(yf, yo, 0.0, ZTOL, 10.0)
    T, p, Y = _dev(st.T), _dev(st.p), _dev(st.Y)
    integ.integrate(T, p, Y, 1e-5, RTOL, ATOL)
    g_mapped, nm, ref = integ.reference_mapping(n)
    g_mapped = g_mapped.cpu().numpy().astype(bool)
    assert ref == r
    assert np.array_equal(g_mapped[~near], mapped[~near])
    assert nm == int(g_mapped.sum()) > n // 2
    sub = integ.stats(n)["substeps"].cpu().numpy()
    assert np.all(sub[g_mapped] == 0) and np.all(sub[~g_mapped] > 0)
    Tg, Yg = T.cpu().numpy(), Y.cpu().numpy()
    np.testing.assert_array_equal(Tg[g_mapped], st.T[g_mapped] + (Tg[r] - st.T[r]))
    np.testing.assert_array_equal(Yg[g_mapped], st.Y[g_mapped] + (Yg[r] - st.Y[r]))
