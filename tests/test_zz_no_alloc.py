"""The allocation-free integration entry point (chem_integrate_noalloc), for callers
that cannot allocate device memory: applications whose device memory is fixed up
front by their own pool, and callers that cannot take the synchronisation an
allocation may imply in the middle of a time step.

Called through the C ABI. With the same handle options and block size it runs the
same kernel on the same cells as chem_integrate, so its output must equal
chem_integrate's bitwise, on two calls in a row (the second reuses the library's
fixed scratch array); the per-cell statistics read after it (chem_get_stats,
chem_get_totals) must be those of its own cells, failures included.

Kept in a file collected last: it must pass alone in a fresh process and after
the rest of the suite."""
import ctypes as C

import numpy as np
import pytest

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


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=torch.float64)


def _noalloc(pkg, integ, T, p, Y, dt, rtol=RTOL, atol=ATOL):
    stream = C.c_void_p(int(torch.cuda.current_stream().cuda_stream))
    return pkg.load().chem_integrate_noalloc(integ.h, T.shape[0], C.c_void_p(T.data_ptr()),
                                             C.c_void_p(p.data_ptr()), C.c_void_p(Y.data_ptr()), dt, rtol,
                                             atol, stream)


def _stats(integ, n):
    s = integ.stats(n)
    return {k: v.cpu().numpy() for k, v in s.items()}


@pytest.mark.parametrize("max_steps", [100000, 3])
def test_noalloc_equals_integrate_bitwise(pkg, max_steps):
    """777 cells of the 54-species workload, mixed precision, work queue, 128-thread
    CTAs on both paths. max_steps = 3 makes most cells fail (status MAX_STEPS, last
    accepted state kept): the no-alloc call must report the same failures."""
    lib = pkg.load()
    m, st, dt = synth.workload("c54_65k", n_cells=777, state_seed=9)
    integ = pkg.Integrator(m, precision=1, scheduler=2, block=128, max_steps=max_steps)
    n = st.T.shape[0]
    Tr, pr, Yr = _dev(st.T), _dev(st.p), _dev(st.Y)
    integ.integrate(Tr, pr, Yr, dt, RTOL, ATOL)
    ref_stats = _stats(integ, n)
    ref_tot = integ.totals()
    Tr, Yr = Tr.cpu().numpy(), Yr.cpu().numpy()
    if max_steps == 3:
        assert ref_tot["failed"] > 0
    for call in range(2):
        T, p, Y = _dev(st.T), _dev(st.p), _dev(st.Y)
        s = _noalloc(pkg, integ, T, p, Y, dt)
        assert s == pkg.CHEM_OK, lib.chem_last_error(integ.h)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(T.cpu().numpy(), Tr)
        np.testing.assert_array_equal(Y.cpu().numpy(), Yr)
        got = _stats(integ, n)
        for k in ("substeps", "rejects", "h_first", "status"):
            np.testing.assert_array_equal(got[k], ref_stats[k], err_msg=f"{k}, call {call}")
        assert integ.totals() == ref_tot
        print("call", call, "bitwise equal;", ref_tot)


def test_noalloc_argument_errors(pkg):
    lib = pkg.load()
    m, st, dt = synth.workload("c54_65k", n_cells=16, state_seed=9)
    integ = pkg.Integrator(m, precision=1, scheduler=2)
    T, p, Y = _dev(st.T), _dev(st.p), _dev(st.Y)
    # the same range checks as chem_integrate: non-finite dt / rtol / atol
    for dt_, rt_, at_ in ((float("inf"), RTOL, ATOL), (dt, float("inf"), ATOL), (dt, RTOL, float("nan")),
                          (0.0, RTOL, ATOL)):
        assert _noalloc(pkg, integ, T, p, Y, dt_, rt_, at_) == pkg.CHEM_ERR_INVALID_ARG
    np.testing.assert_array_equal(T.cpu().numpy(), st.T)
    # more cells than the fixed scratch holds: a clear error, nothing launched
    n_big = 65537
    e = torch.empty(n_big, dtype=torch.float64, device="cuda")
    E = torch.empty((n_big, m.n_species), dtype=torch.float64, device="cuda")
    assert _noalloc(pkg, integ, e, e, E, dt) == pkg.CHEM_ERR_INVALID_ARG
    assert b"scratch capacity" in lib.chem_last_error(integ.h)
    # zero cells: nothing to do, and the statistics then describe zero cells
    z = torch.empty(0, dtype=torch.float64, device="cuda")
    Z = torch.empty((0, m.n_species), dtype=torch.float64, device="cuda")
    assert _noalloc(pkg, integ, z, z, Z, dt) == pkg.CHEM_OK
    assert integ.totals()["n_cells"] == 0
