"""The allocation-free integration entry point (chem_integrate_noalloc), for
callers that cannot allocate device memory (stream capture, fixed memory pools,
no implicit synchronisation). Called through the C ABI; its output must match
chem_integrate's within the parity tolerance the other tests use, on two calls
in a row (the second call reuses the library's fixed scratch array).

Kept in a file collected last: it must pass alone in a fresh process and after
the rest of the suite."""
import ctypes as C

import numpy as np
import pytest

from paper_2112_05834_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-8, 1e-12


def test_noalloc_matches_integrate_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_05834_gb300 import _build

    _build.build()
    import paper_2112_05834_gb300 as pkg

    lib = pkg.load()
    m, st, dt = synth.workload("c54_65k", n_cells=777, state_seed=9)
    integ = pkg.Integrator(m, precision=1, scheduler=2)
    stream = C.c_void_p(int(torch.cuda.current_stream().cuda_stream))

    def dev(a):
        return torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=torch.float64)

    # reference: the allocating entry point
    Tr, pr, Yr = dev(st.T), dev(st.p), dev(st.Y)
    integ.integrate(Tr, pr, Yr, dt, RTOL, ATOL)
    torch.cuda.synchronize()
    Tr, Yr = Tr.cpu().numpy(), Yr.cpu().numpy()
    for call in range(2):
        T, p, Y = dev(st.T), dev(st.p), dev(st.Y)
        s = lib.chem_integrate_noalloc(integ.h, T.shape[0], C.c_void_p(T.data_ptr()), C.c_void_p(p.data_ptr()),
                                       C.c_void_p(Y.data_ptr()), dt, RTOL, ATOL, stream)
        assert s == pkg.CHEM_OK, lib.chem_last_error(integ.h)
        torch.cuda.synchronize()
        Tn, Yn = T.cpu().numpy(), Y.cpu().numpy()
        assert np.all(np.abs(Tn - Tr) <= 1e-6 * Tr), call
        assert np.all(np.abs(Yn - Yr) <= 1e-8 + 1e-5 * np.abs(Yr)), call
        print("call", call, "max |dT| =", np.abs(Tn - Tr).max(), "max |dY| =", np.abs(Yn - Yr).max())
    # more cells than the fixed scratch holds: a clear error, nothing launched
    n_big = 65537
    e = torch.empty(n_big, dtype=torch.float64, device="cuda")
    E = torch.empty((n_big, m.n_species), dtype=torch.float64, device="cuda")
    s = lib.chem_integrate_noalloc(integ.h, n_big, C.c_void_p(e.data_ptr()), C.c_void_p(e.data_ptr()),
                                   C.c_void_p(E.data_ptr()), dt, RTOL, ATOL, stream)
    assert s == pkg.CHEM_ERR_INVALID_ARG
    assert b"scratch capacity" in lib.chem_last_error(integ.h)
