"""GB300-native batched stiff-chemistry integrator (sm_103a).

Thin Python binding over the C ABI of ``libchem.so`` (``include/chem.h``):
argument marshalling only, every step of the integration runs in the library's
CUDA kernels. PyTorch supplies device memory and streams. There is no CPU
fallback: if the compiled library is missing, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libchem.so")

CHEM_OK, CHEM_ERR_INVALID_ARG, CHEM_ERR_BAD_MECHANISM, CHEM_ERR_CUDA, CHEM_ERR_CELLS_FAILED, \
    CHEM_ERR_OOM = range(6)
CELL_OK, CELL_MAX_STEPS, CELL_H_UNDERFLOW, CELL_NONFINITE, CELL_T_RANGE = range(5)

# Every symbol include/chem.h (and include/chem_mlp.h) declares, with its ctypes signature.
_P, _D, _I32, _I64 = C.c_void_p, C.c_double, C.c_int32, C.c_int64
SIGNATURES = {
    "chem_create": (C.c_int, [_P, _P]),
    "chem_destroy": (C.c_int, [_P]),
    "chem_integrate": (C.c_int, [_P, _I64, _P, _P, _P, _D, _D, _D, _P]),
    "chem_integrate_host": (C.c_int, [_P, _I64, _P, _P, _P, _D, _D, _D, _P]),
    "chem_integrate_noalloc": (C.c_int, [_P, _I64, _P, _P, _P, _D, _D, _D, _P]),
    "chem_integrate_jobs": (C.c_int, [_P, _I32, _D, _D, _D, _P]),
    "chem_set_option": (C.c_int, [_P, C.c_char_p, _D]),
    "chem_get_option": (C.c_int, [_P, C.c_char_p, _P]),
    "chem_get_stats": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "chem_get_totals": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "chem_last_error": (C.c_char_p, [_P]),
    "chem_n_species": (_I32, [_P]),
    "chem_n_reactions": (_I32, [_P]),
    "chem_eval_rhs": (C.c_int, [_P, _I64, _P, _P, _P, _P, _P]),
    "chem_eval_jacobian": (C.c_int, [_P, _I64, _P, _P, _P, _P, _P]),
    "chem_eval_h0": (C.c_int, [_P, _I64, _P, _P, _P, _D, _D, _D, _P, _P]),
    "chem_lu_solve_batched": (C.c_int, [_I64, _I32, _P, _P, _P, _P, _I32, _I32, _P]),
    "chem_eval_math": (C.c_int, [_I32, _I64, _P, _P, _P]),
    "chem_get_kernel_ms": (C.c_int, [_P, _P]),
    "chem_set_reference_mapping": (C.c_int, [_P, _I32, _I32, _I32, _P, _P, _D, _D, _D]),
    "chem_eval_mixture_fraction": (C.c_int, [_P, _I64, _P, _P, _P]),
    "chem_get_reference_mapping": (C.c_int, [_P, _P, _P, _P, _P]),
    "chem_rosenbrock_tableau": (None, [_P, _P, _P, _P, _P]),
    "chem_method_tableau": (_I32, [_I32, _P, _P, _P, _P, _P]),
    "chem_get_phase_cycles": (C.c_int, [_P, _P, _P, _I32]),
    "chem_mlp_create": (C.c_int, [_I32, C.c_uint64, _P]),
    "chem_mlp_destroy": (C.c_int, [_P]),
    "chem_mlp_train": (C.c_int, [_P, _I64, _P, _P, _P, _P, _P, _I32, _I32, _D, C.c_uint64, _P, _P]),
    "chem_mlp_predict": (C.c_int, [_P, _I64, _P, _P, _P, _P, _P, _P]),
    "chem_mlp_attach": (C.c_int, [_P, _P]),
    "chem_mlp_get_params": (C.c_int, [_P, _P, _P]),
    "chem_mlp_set_params": (C.c_int, [_P, _P, _I64]),
    "chem_mlp_gradient": (C.c_int, [_P, _I64, _P, _P, _P, _P, _P, _P, _P, _P]),
    "chem_mlp_apply_gradient": (C.c_int, [_P, _P, _D, _P]),
}

_lib = None
_lock = threading.Lock()


class ChemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"chem status {status}: {msg}")
        self.status = status


def load():
    """Load ``libchem.so`` (built by ``__graft_entry__.build()`` / ``_build.py``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build the CUDA extension first "
                                  "(python -c 'import __graft_entry__ as g; g.build()')")
            lib = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status, handle=None):
    if status != CHEM_OK:
        msg = load().chem_last_error(handle)
        raise ChemError(status, msg.decode() if msg else "")


class MechanismDesc(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("n_reactions", C.c_int32), ("n_elements", C.c_int32)] + [
        (name, C.c_void_p) for name in (
            "W", "elem", "nasa_lo", "nasa_hi", "T_lo", "T_mid", "T_hi", "rxn_type", "reac_idx",
            "reac_nu", "prod_idx", "prod_nu", "reversible", "A", "b", "Ea_R", "A0", "b0", "Ea0_R",
            "troe", "eff")
    ]


class Job(C.Structure):
    _fields_ = [("h", C.c_void_p), ("n_cells", C.c_int64), ("T", C.c_void_p), ("p", C.c_void_p),
                ("Y", C.c_void_p)]


def _stream_ptr(stream):
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def _dptr(t):
    return C.c_void_p(int(t.data_ptr())) if t is not None else None


def _check_cells(T, p, Y, K):
    import torch

    for name, t in (("T", T), ("p", p), ("Y", Y)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
            raise TypeError(f"{name} must be a CUDA float64 tensor")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    n = T.shape[0]
    if p.shape != (n,) or T.shape != (n,) or Y.shape != (n, K):
        raise ValueError(f"expected T[n], p[n], Y[n, {K}]")
    return n


class Integrator:
    """One mechanism on the current CUDA device (wraps a ``chem_handle``)."""

    def __init__(self, mech, **options):
        lib = load()
        arr = mech.arrays()
        self._arr = arr  # keep host arrays alive during create
        d = MechanismDesc()
        d.n_species, d.n_reactions, d.n_elements = mech.n_species, mech.n_reactions, mech.n_elements
        for name, a in arr.items():
            setattr(d, name, a.ctypes.data)
        h = C.c_void_p()
        _check(lib.chem_create(C.byref(d), C.byref(h)), None)
        self.h = h
        self._elements = list(getattr(mech, "elements", []))
        self.K = mech.n_species
        self.I = mech.n_reactions
        self.n = self.K + 1
        for k, v in options.items():
            self.set_option(k, v)

    def close(self):
        if getattr(self, "h", None):
            load().chem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, key, value):
        _check(load().chem_set_option(self.h, key.encode(), float(value)), self.h)

    def get_option(self, key):
        v = C.c_double()
        _check(load().chem_get_option(self.h, key.encode(), C.byref(v)), self.h)
        return v.value

    def integrate(self, T, p, Y, dt, rtol=1e-8, atol=1e-12, stream=None):
        """In-place integration of device tensors T[n], Y[n, K] (p[n] read only)."""
        n = _check_cells(T, p, Y, self.K)
        _check(load().chem_integrate(self.h, n, _dptr(T), _dptr(p), _dptr(Y), float(dt), float(rtol),
                                     float(atol), _stream_ptr(stream)), self.h)

    def integrate_host(self, T, p, Y, dt, rtol=1e-8, atol=1e-12, stream=None):
        """In-place integration of host numpy arrays (copies inside the call; synchronises)."""
        for name, a in (("T", T), ("p", p), ("Y", Y)):
            if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
                raise TypeError(f"{name} must be a contiguous float64 numpy array")
        n = T.shape[0]
        if p.shape != (n,) or Y.shape != (n, self.K):
            raise ValueError("shape mismatch")
        _check(load().chem_integrate_host(self.h, n, T.ctypes.data_as(C.c_void_p),
                                          p.ctypes.data_as(C.c_void_p), Y.ctypes.data_as(C.c_void_p),
                                          float(dt), float(rtol), float(atol), _stream_ptr(stream)),
               self.h)

    def stats(self, n, stream=None, check=False):
        """Per-cell (substeps, rejects, h_first, status) of the last call as CUDA tensors."""
        import torch

        sub = torch.empty(n, dtype=torch.int32, device="cuda")
        rej = torch.empty(n, dtype=torch.int32, device="cuda")
        hf = torch.empty(n, dtype=torch.float64, device="cuda")
        st = torch.empty(n, dtype=torch.int32, device="cuda")
        s = load().chem_get_stats(self.h, _stream_ptr(stream), _dptr(sub), _dptr(rej), _dptr(hf),
                                  _dptr(st))
        if s not in (CHEM_OK, CHEM_ERR_CELLS_FAILED) or (check and s != CHEM_OK):
            _check(s, self.h)
        return {"substeps": sub, "rejects": rej, "h_first": hf, "status": st}

    def totals(self, stream=None):
        vals = [C.c_int64() for _ in range(4)]
        _check(load().chem_get_totals(self.h, _stream_ptr(stream), *[C.byref(v) for v in vals]),
               self.h)
        return dict(zip(("n_cells", "substeps", "rejects", "failed"), (v.value for v in vals)))

    PHASES = ("load+h0", "rhs+jac data", "assembly", "factorisation", "stage rhs", "stage solves",
              "stage combine+control", "T recovery+store")

    def phase_cycles(self, reset=True, stream=None):
        """Per-phase SM cycles (option "profile" = 1) as a dict."""
        buf = (C.c_uint64 * 8)()
        _check(load().chem_get_phase_cycles(self.h, _stream_ptr(stream), buf, int(bool(reset))), self.h)
        return dict(zip(self.PHASES, (int(v) for v in buf)))

    def kernel_ms(self):
        """Device time (ms) of the last integration kernel launch (option "time_kernel" = 1)."""
        ms = C.c_float()
        _check(load().chem_get_kernel_ms(self.h, C.byref(ms)), self.h)
        return float(ms.value)

    def set_reference_mapping(self, Y_fuel, Y_ox, Z_center=0.0, Z_tol=1e-4, T_tol=2.0):
        """Reference mapping by Bilger mixture fraction (chem_set_reference_mapping);
        Y_fuel / Y_ox are the streams' mass fractions [K]. Z_tol < 0 switches it off."""
        col = {e: (self._elements.index(e) if e in self._elements else -1) for e in ("C", "H", "O")}
        yf = np.ascontiguousarray(Y_fuel, dtype=np.float64)
        yo = np.ascontiguousarray(Y_ox, dtype=np.float64)
        if yf.shape != (self.K,) or yo.shape != (self.K,):
            raise ValueError(f"stream compositions must have shape ({self.K},)")
        _check(load().chem_set_reference_mapping(self.h, col["C"], col["H"], col["O"],
                                                 yf.ctypes.data_as(C.c_void_p),
                                                 yo.ctypes.data_as(C.c_void_p), float(Z_center),
                                                 float(Z_tol), float(T_tol)), self.h)

    def mixture_fraction(self, Y, stream=None):
        """Bilger Z[n] of device Y[n, K] for the streams of set_reference_mapping."""
        import torch

        if not (isinstance(Y, torch.Tensor) and Y.is_cuda and Y.dtype == torch.float64
                and Y.is_contiguous() and Y.dim() == 2 and Y.shape[1] == self.K):
            raise TypeError(f"Y must be a contiguous CUDA float64 tensor [n, {self.K}]")
        Z = torch.empty(Y.shape[0], dtype=torch.float64, device=Y.device)
        _check(load().chem_eval_mixture_fraction(self.h, Y.shape[0], _dptr(Y), _dptr(Z),
                                                 _stream_ptr(stream)), self.h)
        return Z

    def reference_mapping(self, n, stream=None):
        """(mapped[n] int32 CUDA tensor, n_mapped, reference cell or -1) of the last call."""
        import torch

        mapped = torch.empty(n, dtype=torch.int32, device="cuda")
        nm, ref = C.c_int64(), C.c_int64()
        _check(load().chem_get_reference_mapping(self.h, _stream_ptr(stream), _dptr(mapped),
                                                 C.byref(nm), C.byref(ref)), self.h)
        return mapped, nm.value, ref.value

    def eval_rhs(self, T, p, Y, stream=None):
        import torch

        n = _check_cells(T, p, Y, self.K)
        f = torch.empty((n, self.n), dtype=torch.float64, device=T.device)
        _check(load().chem_eval_rhs(self.h, n, _dptr(T), _dptr(p), _dptr(Y), _dptr(f),
                                    _stream_ptr(stream)), self.h)
        return f

    def eval_jacobian(self, T, p, Y, stream=None):
        import torch

        n = _check_cells(T, p, Y, self.K)
        J = torch.empty((n, self.n, self.n), dtype=torch.float64, device=T.device)
        _check(load().chem_eval_jacobian(self.h, n, _dptr(T), _dptr(p), _dptr(Y), _dptr(J),
                                         _stream_ptr(stream)), self.h)
        return J

    def eval_h0(self, T, p, Y, dt, rtol=1e-8, atol=1e-12, stream=None):
        import torch

        n = _check_cells(T, p, Y, self.K)
        h0 = torch.empty(n, dtype=torch.float64, device=T.device)
        _check(load().chem_eval_h0(self.h, n, _dptr(T), _dptr(p), _dptr(Y), float(dt), float(rtol),
                                   float(atol), _dptr(h0), _stream_ptr(stream)), self.h)
        return h0


def integrate_jobs(jobs, dt, rtol=1e-8, atol=1e-12, stream=None):
    """One launch over several (Integrator, T, p, Y) jobs with different mechanisms."""
    arr = (Job * len(jobs))()
    for j, (integ, T, p, Y) in enumerate(jobs):
        n = _check_cells(T, p, Y, integ.K)
        arr[j].h, arr[j].n_cells = integ.h, n
        arr[j].T, arr[j].p, arr[j].Y = int(T.data_ptr()), int(p.data_ptr()), int(Y.data_ptr())
    _check(load().chem_integrate_jobs(arr, len(jobs), float(dt), float(rtol), float(atol),
                                      _stream_ptr(stream)), jobs[0][0].h)


def lu_solve_batched(A, b, precision=0, ir_sweeps=2, stream=None):
    """x[s] = A[s]^-1 b[s] for CUDA float64 A[n, d, d], b[n, d]; returns (x, info)."""
    import torch

    n, d, _ = A.shape
    x = torch.empty((n, d), dtype=torch.float64, device=A.device)
    info = torch.empty(n, dtype=torch.int32, device=A.device)
    _check(load().chem_lu_solve_batched(n, d, _dptr(A.contiguous()), _dptr(b.contiguous()), _dptr(x),
                                        _dptr(info), int(precision), int(ir_sweeps),
                                        _stream_ptr(stream)))
    return x, info


def eval_math(op, x, stream=None):
    """Elementwise exp ("exp"), ln ("log") or 1/x ("rcp") of a CUDA float64 tensor by
    the rate kernels' own routines; "ff_hi" / "ff_lo": the parts of the float-float
    split the mixed form's assembly and refinement use."""
    import torch

    code = {"exp": 0, "log": 1, "rcp": 2, "ff_hi": 3, "ff_lo": 4}[op]
    xc = x.contiguous()
    y = torch.empty_like(xc)
    _check(load().chem_eval_math(code, xc.numel(), _dptr(xc), _dptr(y), _stream_ptr(stream)))
    return y


def tableau():
    """(gamma, a[6,6], c[6,6], m[6], e[6]) as used by the device stepper (host call)."""
    g = C.c_double()
    a, c = np.zeros((6, 6)), np.zeros((6, 6))
    m, e = np.zeros(6), np.zeros(6)
    load().chem_rosenbrock_tableau(C.byref(g), a.ctypes.data_as(C.c_void_p),
                                   c.ctypes.data_as(C.c_void_p), m.ctypes.data_as(C.c_void_p),
                                   e.ctypes.data_as(C.c_void_p))
    return g.value, a, c, m, e


def method_tableau(method):
    """(gamma, a, c, m, e) of option "method" (0 RODAS4, 1 ROS34PW2) in the device
    stepper's transformed form, trimmed to the method's stages (host call)."""
    g = C.c_double()
    a, c = np.zeros((6, 6)), np.zeros((6, 6))
    m, e = np.zeros(6), np.zeros(6)
    s = load().chem_method_tableau(int(method), C.byref(g), a.ctypes.data_as(C.c_void_p),
                                   c.ctypes.data_as(C.c_void_p), m.ctypes.data_as(C.c_void_p),
                                   e.ctypes.data_as(C.c_void_p))
    if s < 0:
        raise ValueError(f"unknown method {method}")
    return g.value, a[:s, :s], c[:s, :s], m[:s], e[:s]


class CostModel:
    """Learned per-cell cost / initial-step model (wraps ``chem_mlp``; include/chem_mlp.h)."""

    def __init__(self, n_species, seed=0):
        h = C.c_void_p()
        _check(load().chem_mlp_create(int(n_species), int(seed), C.byref(h)))
        self.h = h
        self.K = n_species

    def close(self):
        if getattr(self, "h", None):
            load().chem_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def train(self, T, p, Y, substeps, h_first, epochs=20, batch=8192, lr=1e-3, seed=0, stream=None):
        """Adam on the logged (state, substeps, first step) samples; returns per-epoch losses."""
        n = _check_cells(T, p, Y, self.K)
        losses = np.zeros(max(epochs, 1), dtype=np.float32)
        _check(load().chem_mlp_train(self.h, n, _dptr(T), _dptr(p), _dptr(Y), _dptr(substeps), _dptr(h_first),
                                     int(epochs), int(batch), float(lr), int(seed),
                                     losses.ctypes.data_as(C.c_void_p), _stream_ptr(stream)))
        return losses[:epochs]

    def predict(self, T, p, Y, stream=None):
        """(ln substeps, ln first step) per cell as CUDA float32 tensors."""
        import torch

        n = _check_cells(T, p, Y, self.K)
        lc = torch.empty(n, dtype=torch.float32, device=T.device)
        lh = torch.empty(n, dtype=torch.float32, device=T.device)
        _check(load().chem_mlp_predict(self.h, n, _dptr(T), _dptr(p), _dptr(Y), _dptr(lc), _dptr(lh),
                                       _stream_ptr(stream)))
        return lc, lh

    def get_params(self):
        nf = C.c_int64()
        _check(load().chem_mlp_get_params(self.h, None, C.byref(nf)))
        buf = np.zeros(nf.value, dtype=np.float32)
        _check(load().chem_mlp_get_params(self.h, buf.ctypes.data_as(C.c_void_p), C.byref(nf)))
        return buf

    def set_params(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.float32)
        _check(load().chem_mlp_set_params(self.h, buf.ctypes.data_as(C.c_void_p), buf.size))

    def gradient(self, T, p, Y, substeps, h_first, stream=None):
        """(loss, gradient over W1, b1, W2, b2, W3, b3) of one full-batch pass, no update."""
        n = _check_cells(T, p, Y, self.K)
        D = self.K + 2
        nw = 128 * D + 128 + 128 * 128 + 128 + 2 * 128 + 2
        g = np.zeros(nw, dtype=np.float32)
        loss = C.c_float()
        _check(load().chem_mlp_gradient(self.h, n, _dptr(T), _dptr(p), _dptr(Y), _dptr(substeps), _dptr(h_first),
                                        C.byref(loss), g.ctypes.data_as(C.c_void_p), _stream_ptr(stream)))
        return loss.value, g

    def apply_gradient(self, grad, lr=1e-3, stream=None):
        """One Adam update of the master weights with a given gradient (host floats in
        the order of ``gradient``'s output)."""
        g = np.ascontiguousarray(grad, dtype=np.float32)
        D = self.K + 2
        if g.size != 128 * D + 128 + 128 * 128 + 128 + 2 * 128 + 2:
            raise ValueError("gradient has the wrong length")
        _check(load().chem_mlp_apply_gradient(self.h, g.ctypes.data_as(C.c_void_p), float(lr),
                                              _stream_ptr(stream)))

    def attach(self, integrator):
        _check(load().chem_mlp_attach(integrator.h, self.h), integrator.h)
        integrator._model = self


def log_cells(integ, T, p, Y, dt, rtol=1e-8, atol=1e-12):
    """Integrates copies of the given cells with the plain heuristic and index order,
    returning the per-cell logs (substeps, h_first) the cost model trains on."""
    order, h0 = integ.get_option("order"), integ.get_option("h0")
    integ.set_option("order", 0)
    integ.set_option("h0", 0)
    T2, Y2 = T.clone(), Y.clone()
    integ.integrate(T2, p, Y2, dt, rtol, atol)
    s = integ.stats(T.shape[0])
    integ.set_option("order", order)
    integ.set_option("h0", h0)
    return s["substeps"], s["h_first"]


def train_cost_model(integ, mech, workload, n_cells, dt, seed=7, epochs=20, batch=8192, lr=1e-3):
    """Trains a cost model on the logs of a separately seeded batch of the same
    workload distribution and switches the integrator to the learned order and
    initial step. Returns the attached model."""
    import torch

    from . import synth

    _, st, _ = synth.workload(workload, n_cells=n_cells, state_seed=1000 + seed)
    dev = torch.device("cuda", torch.cuda.current_device())
    T = torch.tensor(st.T, device=dev)
    p = torch.tensor(st.p, device=dev)
    Y = torch.tensor(st.Y, device=dev)
    sub, hf = log_cells(integ, T, p, Y, dt)
    model = CostModel(mech.n_species, seed=seed)
    model.train(T, p, Y, sub, hf, epochs=epochs, batch=batch, lr=lr, seed=seed)
    model.attach(integ)
    integ.set_option("order", 1)
    integ.set_option("h0", 1)
    return model
