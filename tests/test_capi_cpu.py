"""C ABI checks that need no GPU: the library loads, exports every symbol the
headers declare, validates mechanisms on the host, and reports the Rosenbrock
tableau it integrates with (pinned to the order conditions)."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

import mechs
from paper_2112_05834_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2112_05834_gb300 import _build

    _build.build()
    import paper_2112_05834_gb300 as pkg

    return pkg.load()


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for mm in re.finditer(r"\b(chem_[a-z0-9_]+)\s*\(", text):
            names.add(mm.group(1))
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared_symbols()
    assert "chem_integrate" in names and "chem_create" in names
    for name in sorted(names):
        assert hasattr(lib, name), name


def test_binding_covers_header(lib):
    import paper_2112_05834_gb300 as pkg

    assert _declared_symbols() <= set(pkg.SIGNATURES), _declared_symbols() - set(pkg.SIGNATURES)


def test_tableau_order_conditions(lib):
    """The device tableau (transformed form) maps back to a ROW method satisfying the
    order-4 conditions, with an order-3 embedded method (Hairer & Wanner II, IV.7)."""
    import paper_2112_05834_gb300 as pkg
    from test_oracle_pins import _order_conditions

    g, a, c, m, e = pkg.tableau()
    Gi = np.eye(6) / g - c
    G = np.linalg.inv(Gi)
    alpha = np.tril(a @ G, -1)
    b = m @ G
    bhat = (m - e) @ G
    assert np.abs(_order_conditions(alpha, G, b)).max() < 1e-13
    assert np.abs(_order_conditions(alpha, G, bhat)[:4]).max() < 1e-13


def test_w_method_tableau(lib):
    """The device tableau of option method = 1 (transformed form, converted on the host
    from the published coefficients) maps back to a W-method of order 3 with an
    embedded W-order 2, written independently of the oracle's table."""
    import paper_2112_05834_gb300 as pkg
    from test_oracle_pins import _w_order_conditions

    g, a, c, m, e = pkg.method_tableau(1)
    assert a.shape == (4, 4)
    G = np.linalg.inv(np.eye(4) / g - c)
    alpha = np.tril(a @ G, -1)
    res = _w_order_conditions(alpha, G, m @ G)
    assert np.abs(res).max() < 1e-13, res
    assert np.abs(_w_order_conditions(alpha, G, (m - e) @ G)[:3]).max() < 1e-13
    g0, a0, c0, m0, e0 = pkg.method_tableau(0)
    assert a0.shape == (6, 6) and g0 == 0.25 and np.all(e0 == [0, 0, 0, 0, 0, 1])
    with pytest.raises(ValueError):
        pkg.method_tableau(2)


def _desc(mech):
    import paper_2112_05834_gb300 as pkg

    arr = mech.arrays()
    d = pkg.MechanismDesc()
    d.n_species, d.n_reactions, d.n_elements = mech.n_species, mech.n_reactions, mech.n_elements
    for name, a in arr.items():
        setattr(d, name, a.ctypes.data)
    return d, arr


def test_create_rejects_bad_mechanisms(lib):
    import paper_2112_05834_gb300 as pkg

    h = C.c_void_p()
    assert lib.chem_create(None, C.byref(h)) == pkg.CHEM_ERR_INVALID_ARG
    base = synth.mechanism_preset("h2_10")
    cases = []
    m = synth.mechanism_preset("h2_10")
    m.prod_idx[3, 0] = 99
    cases.append((m, "out of range"))
    m = synth.mechanism_preset("h2_10")
    m.A[2] = -1.0
    cases.append((m, "A > 0"))
    m = synth.mechanism_preset("h2_10")
    k = m.prod_idx[0, 0]
    m.elem[k, 0] += 1  # breaks the element balance of a reaction
    cases.append((m, "not balanced"))
    m = synth.mechanism_preset("h2_10")
    m.nasa_hi[1, 5] += 50.0
    cases.append((m, "discontinuous"))
    m = synth.mechanism_preset("h2_10")
    m.reac_nu[0, 0] = 3
    cases.append((m, "coefficient"))
    for mech, msg in cases:
        d, keep = _desc(mech)
        st = lib.chem_create(C.byref(d), C.byref(h))
        assert st == pkg.CHEM_ERR_BAD_MECHANISM, msg
        assert msg in lib.chem_last_error(None).decode()
    del base


def test_null_handle_is_invalid(lib):
    import paper_2112_05834_gb300 as pkg

    assert lib.chem_set_option(None, b"precision", 1.0) == pkg.CHEM_ERR_INVALID_ARG
    assert lib.chem_integrate(None, 1, None, None, None, 1e-6, 1e-8, 1e-12, None) == pkg.CHEM_ERR_INVALID_ARG
    assert lib.chem_lu_solve_batched(1, 300, None, None, None, None, 0, 0, None) == pkg.CHEM_ERR_INVALID_ARG


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_2112_05834_gb300 as pkg

    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(ImportError):
        pkg.load()
