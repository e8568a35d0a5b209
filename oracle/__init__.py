"""CPU oracle (FP64) for the batched stiff-chemistry integrator.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``. The GPU product path never imports
it, and it imports nothing from the GPU path (only the seeded input generator
``paper_2112_05834_gb300.synth``, which holds no arithmetic of the method).

``oracle.cpp`` is the plain C++ restatement of the method (thermo, rates, RHS,
analytic / finite-difference / complex-step Jacobians, dense partial-pivot LU,
RODAS4 and the ROS34PW2 W-method in their original form, starting step, step
control, temperature recovery). ``equilibrium.py`` (constant-enthalpy Gibbs minimisation) and
``mlp_ref.py`` (FP64 MLP forward/backward) are further oracle-side references.

Every function here is pinned by the ``-m "not gpu"`` tests to something other
than itself (closed forms, conservation laws, order conditions, LAPACK,
complex-step derivatives, brute force); see the test files for each pin.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ST_OK, ST_MAX_STEPS, ST_H_UNDERFLOW, ST_NONFINITE, ST_T_RANGE = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source (g++, -O2, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class OMech(C.Structure):
    _fields_ = [("K", C.c_int32), ("I", C.c_int32), ("E", C.c_int32)] + [
        (name, C.c_void_p) for name in (
            "W", "elem", "nasa_lo", "nasa_hi", "T_lo", "T_mid", "T_hi", "rxn_type", "reac_idx",
            "reac_nu", "prod_idx", "prod_nu", "reversible", "A", "b", "Ea_R", "A0", "b0",
            "Ea0_R", "troe", "eff")
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            P, D, I32, I64 = C.c_void_p, C.c_double, C.c_int32, C.c_int64
            sig = {
                "oracle_thermo": (None, [P, D, P, P, P]),
                "oracle_rates": (None, [P, D, P, P, P, P]),
                "oracle_rates_conc": (None, [P, D, P, P, P, P]),
                "oracle_rhs": (None, [P, D, P, P]),
                "oracle_jac": (None, [P, D, P, P]),
                "oracle_jac_fd": (None, [P, D, P, P, D, D]),
                "oracle_jac_cstep": (None, [P, D, P, P]),
                "oracle_lu_factor": (C.c_int, [C.c_int, P, P]),
                "oracle_lu_solve": (None, [C.c_int, P, P, P]),
                "oracle_tableau": (None, [P, P, P, P]),
                "oracle_rodas_step": (C.c_int, [P, D, P, D, P, P]),
                "oracle_h0": (D, [P, D, P, D, D, D]),
                "oracle_enthalpy_mass": (D, [P, D, P]),
                "oracle_recover_T": (D, [P, P, D, D]),
                "oracle_integrate": (I64, [P, I64, P, P, P, D, D, D, I32, P, P, P, P, P, P, I32, I32]),
                "oracle_tableau_m": (C.c_int, [C.c_int, P, P, P, P, P]),
                "oracle_row_step": (C.c_int, [P, D, P, D, P, P, C.c_int, P]),
                "oracle_h0_m": (D, [P, D, P, D, D, D, C.c_int]),
                "oracle_max_threads": (C.c_int, []),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class Mech:
    """Holds contiguous copies of a synthetic mechanism's arrays and the C view of them."""

    def __init__(self, mech):
        self.mech = mech
        self.arr = mech.arrays()
        self.K = mech.n_species
        self.I = mech.n_reactions
        self.n = self.K + 1
        s = OMech()
        s.K, s.I, s.E = self.K, self.I, mech.n_elements
        for name, a in self.arr.items():
            setattr(s, name, a.ctypes.data)
        self.struct = s
        self.ref = C.byref(s)


def as_mech(m) -> Mech:
    return m if isinstance(m, Mech) else Mech(m)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def thermo(m, T):
    m = as_mech(m)
    cp, h, s = (np.zeros(m.K) for _ in range(3))
    _load().oracle_thermo(m.ref, float(T), _ptr(cp), _ptr(h), _ptr(s))
    return cp, h, s


def rates(m, p, y):
    m = as_mech(m)
    y = _f64(y)
    kf, kr, q = (np.zeros(m.I) for _ in range(3))
    _load().oracle_rates(m.ref, float(p), _ptr(y), _ptr(kf), _ptr(kr), _ptr(q))
    return kf, kr, q


def rates_conc(m, T, Cc):
    m = as_mech(m)
    Cc = _f64(Cc)
    kf, kr, q = (np.zeros(m.I) for _ in range(3))
    _load().oracle_rates_conc(m.ref, float(T), _ptr(Cc), _ptr(kf), _ptr(kr), _ptr(q))
    return kf, kr, q


def rhs(m, p, y):
    m = as_mech(m)
    y = _f64(y)
    f = np.zeros(m.n)
    _load().oracle_rhs(m.ref, float(p), _ptr(y), _ptr(f))
    return f


def jac(m, p, y):
    m = as_mech(m)
    y = _f64(y)
    J = np.zeros((m.n, m.n))
    _load().oracle_jac(m.ref, float(p), _ptr(y), _ptr(J))
    return J


def jac_fd(m, p, y, rel=1e-7, floor=1e-4):
    """Central differences, step rel * max(|y_j|, floor)."""
    m = as_mech(m)
    y = _f64(y)
    J = np.zeros((m.n, m.n))
    _load().oracle_jac_fd(m.ref, float(p), _ptr(y), _ptr(J), float(rel), float(floor))
    return J


def jac_cstep(m, p, y):
    m = as_mech(m)
    y = _f64(y)
    J = np.zeros((m.n, m.n))
    _load().oracle_jac_cstep(m.ref, float(p), _ptr(y), _ptr(J))
    return J


def lu_factor(A):
    A = np.array(A, dtype=np.float64, order="C")
    n = A.shape[0]
    piv = np.zeros(n, dtype=np.int32)
    info = _load().oracle_lu_factor(n, _ptr(A), _ptr(piv))
    return A, piv, info


def lu_solve(LU, piv, b):
    x = np.array(b, dtype=np.float64)
    _load().oracle_lu_solve(LU.shape[0], _ptr(np.ascontiguousarray(LU)), _ptr(piv), _ptr(x))
    return x


def tableau():
    alpha, gam = np.zeros((6, 6)), np.zeros((6, 6))
    b, bhat = np.zeros(6), np.zeros(6)
    _load().oracle_tableau(_ptr(alpha), _ptr(gam), _ptr(b), _ptr(bhat))
    return alpha, gam, b, bhat


METHODS = {"rodas4": 0, "ros34pw2": 1}


def tableau_of(method):
    """(alpha, gamma, b, bhat, q) of a method ("rodas4" or "ros34pw2"), trimmed to its stages."""
    alpha, gam = np.zeros((6, 6)), np.zeros((6, 6))
    b, bhat, q = np.zeros(6), np.zeros(6), C.c_double()
    s = _load().oracle_tableau_m(METHODS[method], _ptr(alpha), _ptr(gam), _ptr(b), _ptr(bhat), C.byref(q))
    return alpha[:s, :s], gam[:s, :s], b[:s], bhat[:s], q.value


def row_step(m, p, y0, h, method="rodas4", E=None):
    """One step with W = J(y0) + E (E: an optional fixed perturbation of the Jacobian)."""
    m = as_mech(m)
    y0 = _f64(y0)
    y1, yh = np.zeros(m.n), np.zeros(m.n)
    Ea = None if E is None else _f64(E, (m.n, m.n))
    info = _load().oracle_row_step(m.ref, float(p), _ptr(y0), float(h), _ptr(y1), _ptr(yh), METHODS[method],
                                   _ptr(Ea))
    if info:
        raise RuntimeError("singular iteration matrix")
    return y1, yh


def rodas_step(m, p, y0, h):
    m = as_mech(m)
    y0 = _f64(y0)
    y1, yh = np.zeros(m.n), np.zeros(m.n)
    info = _load().oracle_rodas_step(m.ref, float(p), _ptr(y0), float(h), _ptr(y1), _ptr(yh))
    if info:
        raise RuntimeError("singular iteration matrix")
    return y1, yh


def h0(m, p, y0, dt, rtol, atol, method="rodas4"):
    m = as_mech(m)
    return _load().oracle_h0_m(m.ref, float(p), _ptr(_f64(y0)), float(dt), float(rtol), float(atol),
                               METHODS[method])


def enthalpy_mass(m, T, Y):
    m = as_mech(m)
    return _load().oracle_enthalpy_mass(m.ref, float(T), _ptr(_f64(Y)))


def recover_T(m, Y, h_target, T_guess):
    m = as_mech(m)
    return _load().oracle_recover_T(m.ref, _ptr(_f64(Y)), float(h_target), float(T_guess))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def integrate(m, T, p, Y, dt, rtol=1e-8, atol=1e-12, max_steps=100000, h0=None, n_threads=0,
              method="rodas4"):
    """Integrate a batch of cells over dt with RODAS4 or the ROS34PW2 W-method. Returns a
    dict of result arrays (inputs untouched)."""
    m = as_mech(m)
    T = np.array(T, dtype=np.float64)
    p = _f64(p)
    Y = np.array(Y, dtype=np.float64, order="C").reshape(-1, m.K)
    n = T.shape[0]
    if p.shape[0] != n or Y.shape[0] != n:
        raise ValueError("T, p, Y disagree on the number of cells")
    sub = np.zeros(n, dtype=np.int32)
    rej = np.zeros(n, dtype=np.int32)
    hf = np.zeros(n)
    st = np.zeros(n, dtype=np.int32)
    Tode = np.zeros(n)
    h0a = None if h0 is None else _f64(h0)
    failed = _load().oracle_integrate(
        m.ref, n, _ptr(T), _ptr(p), _ptr(Y), float(dt), float(rtol), float(atol), int(max_steps),
        _ptr(h0a), _ptr(sub), _ptr(rej), _ptr(hf), _ptr(st), _ptr(Tode), int(n_threads), METHODS[method])
    return {"T": T, "Y": Y, "substeps": sub, "rejects": rej, "h_first": hf, "status": st,
            "T_ode": Tode, "failed": int(failed)}
