"""Benchmark: cells x CFD-step / s of the batched stiff-chemistry integrator.

One step = one chem_integrate call over the whole batch (every cell advanced by
one CFD time step dt at rtol 1e-8, atol 1e-12), from the same saved input state
each time. Default workload: the 54-species / 270-reaction synthetic mechanism,
65,536 cells at 60 bar (60 % cold, 30 % igniting, 10 % burnt), dt = 1e-6 s.

Forms timed on the GPU:
  plain_fp64 : FP64 throughout, one CTA per cell (the plain batched baseline)
  headline   : mixed precision (float-float Jacobian assembly, FP32 Gauss-Jordan and
               solves, refinement against the float-float matrix), persistent
               work queue, and (when trained) the learned cost order and initial
               step.
The JSON line's value is the headline form; plain_fp64 is reported beside it.

--impl reference times the CPU oracle (the plain FP64 C++ restatement of the
method) on a bounded sample of the same workload on this machine's host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2112_05834_gb300 import synth  # noqa: E402

RTOL, ATOL = 1e-8, 1e-12
# FP64 peak derived from the unit count and the clock: 2 DFMA per cycle per SM (ncu's
# sm__sass_thread_inst_executed_op_dfma_pred_on peak_sustained on GB300), 152 SMs,
# 2 flop per FMA, 2070 MHz maximum SM clock. The driver's measured peaks have no FP64 entry.
FP64_PEAK_TFLOPS = 2 * 152 * 2 * 2.070e9 / 1e12
# FP32 peak derived the same way: 128 FFMA per cycle per SM
FP32_PEAK_TFLOPS = 128 * 152 * 2 * 2.070e9 / 1e12


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c54_65k")
    ap.add_argument("--cells", type=int, default=None, help="override the number of cells")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU baseline time budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--forms", default="plain_fp64,mixed,w_method,headline",
                    help="plain_fp64: FP64, one CTA per cell; mixed: mixed precision + work queue; "
                         "w_method: the ROS34PW2 W-method with the Jacobian assembled in FP32 (+ queue); "
                         "headline: mixed + queue + learned order/h0")
    ap.add_argument("--compare-steps", type=int, default=3,
                    help="timed steps of each comparison form (the headline form takes --steps)")
    ap.add_argument("--sweep", action="store_true",
                    help="per-cell time vs absolute tolerance for the FP64 form's classical variants "
                         "(forward-difference Jacobian, elimination without pivoting); one JSON line each")
    ap.add_argument("--cfd-loop", action="store_true",
                    help="the learned scheduling configuration: 100 species, 1,048,576 cells, 20 CFD steps "
                         "with mixing between steps, training on steps 1-5; one JSON line per step")
    ap.add_argument("--retrain-every", type=int, default=0,
                    help="with --cfd-loop: retrain the model every N steps on the learned form's own logs "
                         "of the last N steps (0: train once, on steps 1-5)")
    ap.add_argument("--retrain-epochs", type=int, default=20,
                    help="with --retrain-every: epochs of each retraining (continuing from the current "
                         "weights)")
    ap.add_argument("--no-h0-guard", action="store_true",
                    help="with --cfd-loop: the learned initial step as predicted, without the starting-step "
                         "envelope check (option h0_guard = 0)")
    ap.add_argument("--h0-range", type=int, default=10,
                    help="with --cfd-loop: option h0_range (cells with a standardised model input beyond "
                         "this many training standard deviations start from the heuristic; 0 = off)")
    ap.add_argument("--diag-h0", action="store_true",
                    help="with --cfd-loop: per step, the error |ln(h0 / h_first)| of the learned and of the "
                         "heuristic initial step against the first accepted step, for cells whose standardised "
                         "features lie within / beyond 5 training standard deviations")
    ap.add_argument("--no-learned-order", action="store_true",
                    help="with --cfd-loop: learned initial step only, index order")
    ap.add_argument("--refmap", action="store_true",
                    help="reference mapping by mixture fraction: the mixed form on the 54-species workload "
                         "with a 40 %% oxidiser zone (c54_65k_oxzone unless --workload names another), "
                         "without and with mapping; one JSON line each")
    ap.add_argument("--batching", action="store_true",
                    help="the batching configuration, FP64 throughout: 262,144 cells of the 54-species "
                         "workload, plain launch vs work queue + autotuner + CUDA graph; then four "
                         "mechanisms (10, 32, 54, 100 species) in one launch vs four launches")
    ap.add_argument("--precision-forms", action="store_true",
                    help="the precision configuration: 100 species, 262,144 cells at 40 bar (c100_262k unless "
                         "--workload names another): plain FP64, mixed with 1, 2 and 3 refinement sweeps, and the "
                         "W-method with FP32 assembly; sampled same-run parity; one JSON line each")
    ap.add_argument("--no-phases", action="store_true",
                    help="skip the extra untimed step per form with per-phase cycle counters")
    ap.add_argument("--parity-per-class", type=int, default=512,
                    help="same-run parity: cells per temperature class (cold, igniting, burnt) integrated "
                         "by the oracle and compared with every timed GPU form")
    ap.add_argument("--parity-costliest", type=int, default=256,
                    help="same-run parity: also the costliest cells by the headline form's substeps")
    ap.add_argument("--ref-step-cells", type=int, default=256,
                    help="--impl reference: uniformly sampled cells integrated per step")
    return ap.parse_args()


METRIC = "cells*CFD-step/s at rtol 1e-8 (mixed+learned vs plain FP64 GPU)"


# ---------------------------------------------------------------------------- helpers
def algorithmic_fp64_flops_per_step(m, precision, ir_sweeps):
    """Algorithmic FP64 floating-point operations of one Rosenbrock step of one cell.

    Counted from the method's structure (exp/log not counted as flops):
      RHS (6 per step + 1 at the Jacobian point): per species 41 (thermo
        polynomials, concentration, production sum share, enthalpy sums), per
        reaction 22 (rate argument, mass-action products, reverse ratio, net
        rate, production scatter), per third-body reaction 2 K ([M] sums), per
        falloff reaction 30 (Pr, broadening);
      Jacobian data at the step point: 24 per reaction; assembly 6 n^2;
      FP64 form: LU 2 n^3 / 3, 6 solves x 2 n^2, iteration matrix n^2;
      mixed form: 6 solves x ir_sweeps x 2 n^2 refinement residuals (LU and
        triangular solves run in FP32 and are not counted here).
    """
    K, I = m.n_species, m.n_reactions
    n = K + 1
    n_tb = int(np.sum(m.rxn_type >= 1))
    n_fo = int(np.sum(m.rxn_type >= 2))
    rhs = 41 * K + 22 * I + 2 * n_tb * K + 30 * n_fo
    w = 7 * rhs + 24 * I + 6 * n * n
    if precision == 0:
        w += 2 * n ** 3 / 3 + 12 * n * n + n * n
    else:
        w += 6 * ir_sweeps * 2 * n * n
    return float(w)


def float_float_flops_per_step(m, ir_sweeps):
    """The part of algorithmic_fp64_flops_per_step (mixed form) that the kernel runs as
    float-float arithmetic on the FP32 pipe: the third-body sums of the 7 RHS evaluations,
    the Jacobian assembly and the refinement residuals."""
    K = m.n_species
    n = K + 1
    n_tb = int(np.sum(m.rxn_type >= 1))
    return float(7 * 2 * n_tb * K + 6 * n * n + 6 * ir_sweeps * 2 * n * n)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip() == "Active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def kernel_source_digest():
    """sha256 over the integration kernel's device source (the shared device header and
    the translation unit that instantiates the RODAS4 stepper), in that order."""
    import hashlib

    h = hashlib.sha256()
    for f in ("chem_device.cuh", "chem_kernels.cu"):
        h.update(open(os.path.join(ROOT, "paper_2112_05834_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def kernel_traffic(n_cells):
    """DRAM bytes per launch of the integration kernel from the committed ncu summary
    (profiles/k_integrate_traffic.txt), scaled from the captured batch to n_cells (state
    traffic is per cell); None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "k_integrate_traffic.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_source_sha256") != kernel_source_digest():
        return None
    per_cell = (float(kv["dram_bytes_read"]) + float(kv["dram_bytes_write"])) / float(kv["cells"])
    return per_cell * n_cells


def phase_rooflines(m, hd, n, mlp_ms):
    """Per-phase fractions of the headline launch: phase time = the phase's share of the
    CTAs' cycles (option "profile") x the launch's CUDA-event time; algorithmic work per
    Rosenbrock step x the launch's steps. Rates + Jacobian against the FP64 peak; the
    FP32 Gauss-Jordan inverse and the FP32 products of the stage solves against the FP32
    peak; MLP inference (timed alone) against the measured BF16 peak; state streaming
    against the measured HBM bandwidth."""
    K, I = m.n_species, m.n_reactions
    nn = K + 1
    n_tb = int(np.sum(m.rxn_type >= 1))
    n_fo = int(np.sum(m.rxn_type >= 2))
    ph = hd["phases"]
    t = hd["kernel_ms"] / 1e3
    steps = hd["substeps"]
    peaks = measured_peaks()
    out = {}
    rhs = 41 * K + 22 * I + 2 * n_tb * K + 30 * n_fo
    share = ph["rhs+jac data"] + ph["assembly"] + ph["stage rhs"]
    w = (7 * rhs + 24 * I + 6 * nn * nn) * steps
    a = w / (share * t) / 1e12
    out["rates_jacobian"] = {"bound": "alu", "achieved": a, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": a / FP64_PEAK_TFLOPS, "time_share": share}
    share = ph["factorisation"] + ph["stage solves"]
    w = (nn ** 3 + 12 * 2 * nn * nn) * steps  # Gauss-Jordan inverse + 12 FP32 products (1 sweep)
    a = w / (share * t) / 1e12
    out["factor_solve_fp32"] = {"bound": "alu", "achieved": a, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                                "frac": a / FP32_PEAK_TFLOPS, "time_share": share}
    if mlp_ms:
        w = 2.0 * n * ((K + 2) * 128 + 128 * 128 + 128 * 2)
        a = w / (mlp_ms / 1e3) / 1e12
        pk = peaks.get("bf16_tflops", 1900.0)
        out["mlp_inference"] = {"bound": "tensor", "achieved": a, "peak": pk, "unit": "TFLOP/s", "frac": a / pk,
                                "ms": mlp_ms}
    b = n * (2 * K + 3) * 8.0
    a = b / t / 1e9
    pk = peaks.get("hbm_gbs", 6800.0)
    out["state_streaming"] = {"bound": "hbm", "achieved": a, "peak": pk, "unit": "GB/s", "frac": a / pk}
    return out


def cpu_model():
    """The host CPU's model name (x86: "model name"; Arm: implementer / part codes)."""
    import platform

    fields = {}
    try:
        with open("/proc/cpuinfo", errors="replace") as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields.setdefault(k.strip().lower(), v.strip())
    except Exception:  # the model name is informative only
        fields = {}
    if "model name" in fields:
        return fields["model name"]
    if "cpu part" in fields:
        return f"{platform.machine()} (CPU implementer {fields.get('cpu implementer', '?')}, part {fields['cpu part']})"
    return platform.processor() or platform.machine()


_HOST_THREADS = []


def host_threads():
    """The oracle's OpenMP thread count, read once: the oracle's integrate sets the
    process-wide count when given n_threads, so a later read would see the last value."""
    if not _HOST_THREADS:
        import oracle

        _HOST_THREADS.append(oracle.max_threads())
    return _HOST_THREADS[0]


def _oracle_rate(m, st, dt, seconds, order, threads, chunk, keep=None):
    import oracle

    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds and done < order.size:
        idx = order[done:done + chunk]
        r = oracle.integrate(m, st.T[idx], st.p[idx], st.Y[idx], dt, RTOL, ATOL, n_threads=threads)
        if keep is not None:
            keep.append((idx, r))
        done += idx.size
    return done, time.perf_counter() - t0


def cpu_baseline(m, st, dt, seconds, seed=0):
    """Oracle on a bounded uniform sample of the workload's cells (all host cores), plus a
    single-thread rate on a fifth of the time budget (another sample of the same cells)."""
    import oracle

    oracle.build()
    rng = np.random.default_rng(seed)
    order = rng.permutation(st.T.shape[0])
    threads = host_threads()
    keep = []
    done, el = _oracle_rate(m, st, dt, seconds, order, threads, 64, keep)
    rest = order[done:] if done < order.size else order
    done1, el1 = _oracle_rate(m, st, dt, seconds / 5.0, rest, 1, 4, keep)
    return {"value": done / el, "unit": "cells*step/s", "cores": threads, "kind": "oracle",
            "sample": f"{done} uniformly sampled cells of the {st.T.shape[0]}-cell batch, "
                      f"{el:.1f} s on {threads} threads",
            "single_thread": {"value": done1 / el1, "sample": f"{done1} further cells, {el1:.1f} s on 1 thread"},
            "cpu_model": cpu_model(), "_results": keep}


def same_run_parity(m, st, dt, results, per_class, costliest, extra=(), seed=5):
    """The bench's own inputs, integrated by the oracle on a stratified sample (per_class
    cells of each temperature class, plus the costliest cells by the headline form's
    substeps, plus any cells the CPU baseline already integrated), compared with the
    final states of every timed GPU form at the parity bound |dT| <= 1e-6 T,
    |dY_k| <= 1e-8 + 1e-5 |Y_k|."""
    import oracle

    oracle.build()
    rng = np.random.default_rng(seed)
    pick = []
    for k in np.unique(st.kind):
        cls = np.nonzero(st.kind == k)[0]
        pick.append(rng.choice(cls, min(per_class, cls.size), replace=False))
    ref_sub = results.get("headline", next(iter(results.values())))["cell_substeps"]
    pick.append(np.argsort(ref_sub, kind="stable")[::-1][:costliest])
    idx = np.unique(np.concatenate(pick)) if pick else np.zeros(0, dtype=np.int64)
    have = {}
    for cells, r in extra:
        for j, c in enumerate(cells):
            have[int(c)] = (r["T"][j], r["Y"][j], r["status"][j])
    todo = np.array([c for c in idx if int(c) not in have], dtype=np.int64)
    t0 = time.perf_counter()
    if todo.size:
        r = oracle.integrate(m, st.T[todo], st.p[todo], st.Y[todo], dt, RTOL, ATOL, n_threads=host_threads())
        for j, c in enumerate(todo):
            have[int(c)] = (r["T"][j], r["Y"][j], r["status"][j])
    el = time.perf_counter() - t0
    cells = np.array(sorted(have), dtype=np.int64)
    Tr = np.array([have[c][0] for c in cells])
    Yr = np.array([have[c][1] for c in cells])
    ok_ref = np.array([have[c][2] == 0 for c in cells])
    out = {"cells": int(cells.size), "per_class": per_class, "costliest": costliest,
           "oracle_s": round(el, 1), "oracle_failed": int((~ok_ref).sum()), "bound": "|dT|<=1e-6 T, |dY|<=1e-8+1e-5|Y|",
           "forms": {}}
    ok = bool(ok_ref.all())
    for name, res in results.items():
        dT = np.abs(res["T"][cells] - Tr) / Tr
        dY = np.abs(res["Y"][cells] - Yr) / (1e-8 + 1e-5 * np.abs(Yr))
        f = {"max_dT_over_T": float(dT.max()), "max_dY_over_bound": float(dY.max()),
             "cells_outside": int(np.sum((dT > 1e-6) | (dY > 1.0).any(axis=1)))}
        f["ok"] = f["cells_outside"] == 0
        ok = ok and f["ok"]
        out["forms"][name] = f
    out["ok"] = ok
    return out


# ---------------------------------------------------------------------------- GPU arm
def run_ours(args, rank, world):
    import torch

    import paper_2112_05834_gb300 as pkg

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    m, st, dt = synth.workload(args.workload, n_cells=args.cells)
    n = st.T.shape[0]
    T0 = torch.tensor(st.T, device=dev)
    p = torch.tensor(st.p, device=dev)
    Y0 = torch.tensor(st.Y, device=dev)
    T = torch.empty_like(T0)
    Y = torch.empty_like(Y0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    forms = {}
    plain = pkg.Integrator(m, precision=0, scheduler=0)
    mixed = pkg.Integrator(m, precision=1, scheduler=2, ir_sweeps=1)
    wmeth = pkg.Integrator(m, precision=2, scheduler=2, ir_sweeps=1, method=1)
    head = pkg.Integrator(m, precision=1, scheduler=2, ir_sweeps=1)
    for integ in (plain, mixed, wmeth, head):
        integ.set_option("time_kernel", 1)  # CUDA events around the integration kernel
    learned = False
    if not args.no_learned and hasattr(pkg, "train_cost_model"):
        learned = pkg.train_cost_model(head, m, args.workload, n, dt, seed=7)
    want = args.forms.split(",")
    if "plain_fp64" in want:
        forms["plain_fp64"] = plain
    if "mixed" in want:
        forms["mixed"] = mixed
    if "w_method" in want:
        forms["w_method"] = wmeth
    if "headline" in want:
        forms["headline"] = head

    def one(integ):
        T.copy_(T0)
        Y.copy_(Y0)
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        integ.integrate(T, p, Y, dt, RTOL, ATOL)
        e1.record(stream)
        return e0, e1

    results = {}
    clocks = ClockSampler(dev.index)
    clk = None
    for name, integ in forms.items():
        # the headline form is the benchmark (W warm-up, K timed steps); the comparison
        # forms are timed on fewer steps from the same input
        steps = args.steps if name == "headline" else min(args.steps, args.compare_steps)
        for _ in range(args.warmup if name == "headline" else min(args.warmup, 1)):
            one(integ)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        if name == "headline":
            clocks.start()
        evs, kms = [], []
        for _ in range(steps):
            evs.append(one(integ))
            kms.append(integ.kernel_ms())  # waits for this step's integration kernel
        torch.cuda.synchronize()
        if name == "headline":
            clk = clocks.stop()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        tot = integ.totals()
        # every timed step starts from the same input, so the last step's output is the
        # form's result for it (compared with the oracle after the timed region)
        results[name] = {"ms_total": ms, "steps": steps, "kernel_ms": float(np.mean(kms)), "substeps": tot["substeps"],
                         "failed": tot["failed"], "rejects": tot["rejects"],
                         "T": T.cpu().numpy(), "Y": Y.cpu().numpy(),
                         "cell_substeps": integ.stats(n)["substeps"].cpu().numpy()}
        if not args.no_phases:
            integ.set_option("profile", 1)
            one(integ)
            torch.cuda.synchronize()
            ph = integ.phase_cycles()
            integ.set_option("profile", 0)
            tot_c = sum(ph.values())
            results[name]["phases"] = {k: round(v / tot_c, 4) for k, v in ph.items()}
    # end to end through the host entry point (H2D of T, p, Y; D2H of T, Y inside the call)
    Th = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
    ph = torch.tensor(st.p).pin_memory().numpy()
    Yh = torch.empty((n, m.n_species), dtype=torch.float64).pin_memory().numpy()
    e2e_times = []
    for it in range(args.warmup + args.steps):
        Th[:] = st.T
        Yh[:] = st.Y
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        head.integrate_host(Th, ph, Yh, dt, RTOL, ATOL)
        t1 = time.perf_counter()
        if it >= args.warmup:
            e2e_times.append(t1 - t0)
    e2e_s = sum(e2e_times)
    # MLP inference alone on the batch (untimed region; for its roofline)
    mlp_ms = None
    if learned and hasattr(learned, "predict"):
        learned.predict(T0, p, Y0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            learned.predict(T0, p, Y0)
        e1.record(stream)
        torch.cuda.synchronize()
        mlp_ms = e0.elapsed_time(e1) / 5
    if world > 1:
        t = torch.tensor([results["headline"]["ms_total"], e2e_s], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        results["headline"]["ms_total"], e2e_s = float(t[0]), float(t[1])
    return m, st, dt, n, results, clk, e2e_s, learned, head, mlp_ms


def run_sweep(args):
    """Per-cell device time vs atol (rtol 1e-6) on the FP64 form with: forward-difference
    Jacobian + elimination without pivoting, analytical Jacobian + elimination without
    pivoting, analytical Jacobian + partial-pivot LU, and the mixed form for comparison.
    Each point: one warm-up and one timed launch (CUDA events) from the same state."""
    import torch

    import paper_2112_05834_gb300 as pkg

    n = args.cells or 8192
    m, st, dt = synth.workload(args.workload, n_cells=n)
    dev = torch.device("cuda", 0)
    T0, p, Y0 = (torch.tensor(a, device=dev) for a in (st.T, st.p, st.Y))
    variants = [("fd_jacobian+no_pivoting", dict(precision=0, jacobian=1, pivoting=0)),
                ("analytic+no_pivoting", dict(precision=0, jacobian=0, pivoting=0)),
                ("analytic+lu", dict(precision=0, jacobian=0, pivoting=1)),
                ("analytic+mixed", dict(precision=1)),
                ("rodas4+fp32_assembly", dict(precision=2)),
                ("w_method+fp32_assembly", dict(precision=2, method=1))]
    for atol in (1e-6, 1e-8, 1e-10, 1e-12):
        for name, opt in variants:
            integ = pkg.Integrator(m, scheduler=2, time_kernel=1, **opt)
            for _ in range(2):
                T, Y = T0.clone(), Y0.clone()
                integ.integrate(T, p, Y, dt, 1e-6, atol)
                ms = integ.kernel_ms()
            tot = integ.totals()
            print(json.dumps({"sweep": name, "workload": args.workload, "n_cells": n, "rtol": 1e-6, "atol": atol,
                              "us_per_cell": 1e3 * ms / n, "kernel_ms": ms, "substeps": tot["substeps"],
                              "rejects": tot["rejects"], "failed": tot["failed"]}), flush=True)
            integ.close()


def run_refmap(args):
    """Whole-call device time of chem_integrate (CUDA events on the stream, mapping
    kernels included) without and with reference mapping, mixed form, work queue.
    Each variant: one warm-up and three timed calls from the same initial state
    (restored by a device copy outside the timed region); the median is reported."""
    import torch

    import paper_2112_05834_gb300 as pkg

    wl = "c54_65k_oxzone" if args.workload == "c54_65k" else args.workload
    m, st, dt = synth.workload(wl, n_cells=args.cells)
    n = st.T.shape[0]
    yf, yo = synth.streams(m)
    dev = torch.device("cuda", 0)
    T0, p, Y0 = (torch.tensor(a, device=dev) for a in (st.T, st.p, st.Y))
    stream = torch.cuda.current_stream()
    variants = [("no_mapping", None), ("mapping_Ztol1e-4_Ttol2K", (1e-4, 2.0)),
                ("mapping_Ztol1e-4_Ttol10K", (1e-4, 10.0))]
    for name, zt in variants:
        integ = pkg.Integrator(m, precision=1, scheduler=2, time_kernel=1)
        if zt is not None:
            integ.set_reference_mapping(yf, yo, 0.0, zt[0], zt[1])
        times, kms = [], []
        for rep in range(4):
            T, Y = T0.clone(), Y0.clone()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            integ.integrate(T, p, Y, dt, 1e-8, 1e-12)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep > 0:
                times.append(e0.elapsed_time(e1))
                kms.append(integ.kernel_ms())
        tot = integ.totals()
        nm = integ.reference_mapping(n)[1] if zt is not None else 0
        ms = float(np.median(times))
        print(json.dumps({"refmap": name, "workload": wl, "n_cells": n, "rtol": 1e-8, "atol": 1e-12,
                          "cells_per_s": n / (ms * 1e-3), "call_ms": ms,
                          "integration_kernel_ms": float(np.median(kms)), "n_mapped": nm,
                          "substeps": tot["substeps"], "failed": tot["failed"]}), flush=True)
        integ.close()


def run_batching(args):
    """FP64 throughout. (1) 262,144 cells of the 54-species workload: one CTA per cell
    (the plain launch) against persistent CTAs on the device work queue with the block
    size from the autotuner and the launch captured in a CUDA graph. (2) Four mechanisms
    (10, 32, 54, 100 species; a quarter of the cells each, same cell mix at 60 bar) in one
    launch against four launches in sequence and four concurrent launches (option
    job_launch). CUDA events on the stream around each call; one
    warm-up call (for the batching form it includes the autotuner's trials and the graph
    capture, timed separately) and two timed calls from the same initial state."""
    import torch

    import paper_2112_05834_gb300 as pkg

    n = args.cells or 262144
    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", 0)

    def timed(call, inputs, reps=2):
        out = []
        for r in range(1 + reps):
            arrs = [tuple(t.clone() for t in x) for x in inputs]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            call(arrs)
            e1.record(stream)
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
        return out[0], float(np.median(out[1:]))

    m, st, dt = synth.workload("c54_262k", n_cells=n)
    x = [tuple(torch.tensor(a, device=dev) for a in (st.T, st.p, st.Y))]
    res = {}
    for name, opt in (("plain_launch", dict(precision=0, scheduler=0)),
                      ("queue_autotune_graph", dict(precision=0, scheduler=2, autotune=1, graph=1))):
        integ = pkg.Integrator(m, **opt)
        first, ms = timed(lambda a, i=integ: i.integrate(a[0][0], a[0][1], a[0][2], dt, 1e-8, 1e-12), x)
        tot = integ.totals()
        res[name] = ms
        print(json.dumps({"batching": name, "workload": "c54_262k", "n_cells": n, "dtype": "f64",
                          "cells_per_s": n / (ms * 1e-3), "call_ms": ms, "first_call_ms": first,
                          "block": int(integ.get_option("last_block")), "substeps": tot["substeps"],
                          "failed": tot["failed"]}), flush=True)
        integ.close()
    print(json.dumps({"batching": "speedup_queue_autotune_graph_over_plain",
                      "value": res["plain_launch"] / res["queue_autotune_graph"]}), flush=True)

    presets = ("h2_10", "c_32", "c_54", "c_100")
    per = n // len(presets)
    integs, inputs = [], []
    for i, name in enumerate(presets):
        mech = synth.mechanism_preset(name)
        s = synth.gen_states(mech, per, seed=1 + i, p=60 * synth.BAR, classes=synth.MIXED_CLASSES)
        integs.append(pkg.Integrator(mech, precision=0, scheduler=2))
        inputs.append(tuple(torch.tensor(a, device=dev) for a in (s.T, s.p, s.Y)))

    def joint(a):
        pkg.integrate_jobs([(g, *t) for g, t in zip(integs, a)], dt, 1e-8, 1e-12)

    def separate(a):
        for g, t in zip(integs, a):
            g.integrate(*t, dt, 1e-8, 1e-12)

    def concurrent(a):
        integs[0].set_option("job_launch", 1)
        joint(a)
        integs[0].set_option("job_launch", 0)

    for name, call in (("four_mechanisms_one_launch", joint), ("four_mechanisms_four_launches", separate),
                       ("four_mechanisms_concurrent_launches", concurrent)):
        _, ms = timed(call, inputs)
        sub = sum(g.totals()["substeps"] for g in integs)
        print(json.dumps({"batching": name, "mechanisms": list(presets), "cells_each": per, "dtype": "f64",
                          "cells_per_s": len(presets) * per / (ms * 1e-3), "call_ms": ms,
                          "block": int(integs[0].get_option("last_block")), "substeps": sub}), flush=True)


def run_precision_forms(args):
    """The precision configuration: each form integrates the same 262,144-cell batch of
    the 100-species workload (one warm-up call, two timed calls from the same input,
    CUDA events on the stream, median); per form the Rosenbrock steps, rejections and
    the per-result error against the FP64 oracle on a stratified sample (the same
    cells for every form)."""
    import torch

    import paper_2112_05834_gb300 as pkg

    wl = "c100_262k" if args.workload == "c54_65k" else args.workload
    m, st, dt = synth.workload(wl, n_cells=args.cells)
    n = st.T.shape[0]
    dev = torch.device("cuda", 0)
    T0, p, Y0 = (torch.tensor(a, device=dev) for a in (st.T, st.p, st.Y))
    stream = torch.cuda.current_stream()
    forms = [("plain_fp64", dict(precision=0, scheduler=0)),
             ("mixed_ir1", dict(precision=1, scheduler=2, ir_sweeps=1)),
             ("mixed_ir2", dict(precision=1, scheduler=2, ir_sweeps=2)),
             ("mixed_ir3", dict(precision=1, scheduler=2, ir_sweeps=3)),
             ("w_method_fp32_assembly", dict(precision=2, scheduler=2, ir_sweeps=1, method=1))]
    res = {}
    for name, opt in forms:
        integ = pkg.Integrator(m, **opt)
        times = []
        for rep in range(3):
            T, Y = T0.clone(), Y0.clone()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            integ.integrate(T, p, Y, dt, RTOL, ATOL)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep > 0:
                times.append(e0.elapsed_time(e1))
        tot = integ.totals()
        res[name] = {"T": T.cpu().numpy(), "Y": Y.cpu().numpy(), "ms": float(np.median(times)),
                     "cell_substeps": integ.stats(n)["substeps"].cpu().numpy(), "tot": tot,
                     "block": int(integ.get_option("last_block"))}
        integ.close()
    par = same_run_parity(m, st, dt, {k: v for k, v in res.items()}, args.parity_per_class // 8,
                          args.parity_costliest // 8)
    base = res["plain_fp64"]["ms"]
    for name, _ in forms:
        r = res[name]
        print(json.dumps({"precision_form": name, "workload": wl, "n_cells": n, "rtol": RTOL, "atol": ATOL,
                          "cells_per_s": n / (r["ms"] * 1e-3), "call_ms": r["ms"], "speedup_vs_plain_fp64": base / r["ms"],
                          "substeps": r["tot"]["substeps"], "rejects": r["tot"]["rejects"],
                          "failed": r["tot"]["failed"], "block": r["block"], "parity": par["forms"][name],
                          "parity_cells": par["cells"]}), flush=True)
    if not par["ok"]:
        sys.exit(1)


def run_cfd_loop(args):
    """Learned scheduling + initial step at scale: the 100-species mechanism, 1,048,576
    cells (or --cells), 20 CFD steps of dt with the seeded mixing perturbation between
    steps. Steps 1-5 run the plain heuristic in index order and log per-cell substeps
    and first accepted steps; the MLP trains on those logs (timed, reported apart);
    steps 6-20 run the learned order and initial step. Every step also runs the plain
    form on the identical input, so the gain is measured on the same states. Mixed
    precision, work queue; CUDA events around each integrate call (MLP inference and
    the cost sort included)."""
    import torch

    import paper_2112_05834_gb300 as pkg

    n = args.cells or 1048576
    m, st, dt = synth.workload("c100_1m", n_cells=n)
    dev = torch.device("cuda", 0)
    plain = pkg.Integrator(m, precision=1, scheduler=2)
    learned = pkg.Integrator(m, precision=1, scheduler=2)
    model = pkg.CostModel(m.n_species, seed=11)
    logs = []
    tot = {"plain_ms": 0.0, "learned_ms": 0.0, "plain_sub": 0, "learned_sub": 0}

    def timed(integ, T0, p, Y0):
        T, Y = T0.clone(), Y0.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        integ.integrate(T, p, Y, dt, RTOL, ATOL)
        e1.record()
        torch.cuda.synchronize()
        s = integ.stats(n)
        return T, Y, e0.elapsed_time(e1), s

    for step in range(1, 21):
        T0, p, Y0 = (torch.tensor(a, device=dev) for a in (st.T, st.p, st.Y))
        line = {"cfd_step": step, "n_cells": n}
        if step == 6:
            t0 = time.perf_counter()
            cat = [torch.cat([lg[k] for lg in logs]) for k in range(5)]
            losses = model.train(*cat, epochs=20, batch=8192, lr=1e-3, seed=12)
            torch.cuda.synchronize()
            line["train_s"] = time.perf_counter() - t0
            line["train_loss"] = [float(losses[0]), float(losses[-1])]
            model.attach(learned)
            learned.set_option("order", 0 if args.no_learned_order else 1)
            learned.set_option("h0", 1)
            learned.set_option("h0_guard", 0 if args.no_h0_guard else 1)
            learned.set_option("h0_range", args.h0_range)
            logs.clear()
        if args.retrain_every and step > 6 and (step - 6) % args.retrain_every == 0 and logs:
            t0 = time.perf_counter()
            cat = [torch.cat([lg[k] for lg in logs]) for k in range(5)]
            losses = model.train(*cat, epochs=args.retrain_epochs, batch=8192, lr=1e-3, seed=12 + step)
            torch.cuda.synchronize()
            line["train_s"] = time.perf_counter() - t0
            line["train_loss"] = [float(losses[0]), float(losses[-1])]
            tot["retrain_s"] = tot.get("retrain_s", 0.0) + line["train_s"]
            model.attach(learned)
            logs.clear()
        T, Y, ms, s = timed(plain, T0, p, Y0)
        if args.diag_h0 and step >= 6:
            # initial-step errors against the plain form's first accepted steps (same inputs)
            hf = s["h_first"].cpu().numpy()
            ok = (s["status"].cpu().numpy() == 0) & (hf > 0)
            h_heur = plain.eval_h0(T0, p, Y0, dt, RTOL, ATOL).cpu().numpy()
            lc, lh = model.predict(T0, p, Y0)
            h_pred = np.clip(np.exp(lh.cpu().numpy().astype(np.float64)), 1e-14, dt)
            prm = model.get_params()
            D = m.n_species + 2
            mu, sd = prm[:D].astype(np.float64), prm[D:2 * D].astype(np.float64)
            x = np.concatenate([(st.T / 1000.0)[:, None], np.log(st.p)[:, None], np.log(st.Y + 1e-20)], axis=1)
            ood = (np.abs((x - mu) / sd) > 5.0).any(axis=1)
            e_l = np.abs(np.log(h_pred / np.where(ok, hf, 1.0)))
            e_h = np.abs(np.log(np.clip(h_heur, 1e-300, None) / np.where(ok, hf, 1.0)))
            line["diag_h0"] = {"ood_fraction": float(ood[ok].mean()),
                               "learned_err_in": float(np.median(e_l[ok & ~ood])) if (ok & ~ood).any() else None,
                               "learned_err_ood": float(np.median(e_l[ok & ood])) if (ok & ood).any() else None,
                               "heuristic_err_in": float(np.median(e_h[ok & ~ood])) if (ok & ~ood).any() else None,
                               "heuristic_err_ood": float(np.median(e_h[ok & ood])) if (ok & ood).any() else None,
                               "learned_shorter_frac": float((h_pred[ok] < hf[ok]).mean())}
        line.update({"plain_ms": ms, "plain_substeps": int(s["substeps"].sum()),
                     "plain_rejects": int(s["rejects"].sum()), "plain_failed": int((s["status"] != 0).sum())})
        if step <= 5:
            logs.append((T0, p, Y0, s["substeps"].clone(), s["h_first"].clone()))
        else:
            _, _, ms2, s2 = timed(learned, T0, p, Y0)
            if args.retrain_every:
                logs.append((T0, p, Y0, s2["substeps"].clone(), s2["h_first"].clone()))
            line.update({"learned_ms": ms2, "learned_substeps": int(s2["substeps"].sum()),
                         "learned_rejects": int(s2["rejects"].sum()),
                         "learned_failed": int((s2["status"] != 0).sum()), "speedup": ms / ms2})
            tot["plain_ms"] += ms
            tot["learned_ms"] += ms2
            tot["plain_sub"] += line["plain_substeps"]
            tot["learned_sub"] += line["learned_substeps"]
        print(json.dumps(line), flush=True)
        st = synth.perturb_states(synth.CellStates(T=T.cpu().numpy(), p=st.p, Y=Y.cpu().numpy(), kind=st.kind),
                                  seed=100 + step)
    print(json.dumps({"cfd_loop_summary": "steps 6-20", "n_cells": n, "retrain_every": args.retrain_every,
                      "retrain_epochs": args.retrain_epochs if args.retrain_every else None,
                      "retrain_s_total": tot.get("retrain_s", 0.0),
                      "learned_order": not args.no_learned_order, "h0_guard": not args.no_h0_guard,
                      "h0_range": args.h0_range,
                      "plain_cells_step_per_s": 15 * n / (tot["plain_ms"] / 1e3),
                      "learned_cells_step_per_s": 15 * n / (tot["learned_ms"] / 1e3),
                      "speedup": tot["plain_ms"] / tot["learned_ms"],
                      "speedup_incl_retraining": tot["plain_ms"] / (tot["learned_ms"] + 1e3 * tot.get("retrain_s", 0.0)),
                      "substeps_ratio": tot["learned_sub"] / tot["plain_sub"]}), flush=True)


def run_reference(args):
    """The reference arm: the CPU oracle (plain FP64 C++, OpenMP over cells, all host
    cores) on the same workload. Each step integrates a fresh uniform sample of
    --ref-step-cells cells of the batch (a bounded sample: the whole batch takes minutes
    on the host); ms_per_step is that step's measured wall time and the value is the
    timed steps' cells over their time."""
    import oracle

    oracle.build()
    m, st, dt = synth.workload(args.workload, n_cells=args.cells)
    n = st.T.shape[0]
    threads = host_threads()
    rng = np.random.default_rng(0)
    order = rng.permutation(n)
    k = min(args.ref_step_cells, n)
    times, pos = [], 0
    for it in range(args.warmup + args.steps):
        if pos + k > n:
            pos = 0
        idx = order[pos:pos + k]
        pos += k
        t0 = time.perf_counter()
        oracle.integrate(m, st.T[idx], st.p[idx], st.Y[idx], dt, RTOL, ATOL, n_threads=threads)
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
    total = float(sum(times))
    v = k * len(times) / total
    sample = (f"{k} uniformly sampled cells of the {n}-cell batch per step, {len(times)} timed steps, "
              f"{total:.1f} s on {threads} threads")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "cells*step/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "n_cells": n, "step_cells": k,
                       "mechanism": f"{m.n_species} species / {m.n_reactions} reactions (seeded synthetic)",
                       "pressure_bar": float(st.p[0] / 1e6), "dt_s": dt, "rtol": RTOL, "atol": ATOL,
                       "form": "CPU oracle, FP64 (RODAS4, analytic Jacobian, partial-pivot LU)"},
            "cpu_baseline": {"value": v, "unit": "cells*step/s", "cores": threads, "kind": "oracle",
                             "sample": sample, "cpu_model": cpu_model()},
            "e2e": {"value": v, "unit": "cells*step/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.sweep:
        run_sweep(args)
        return
    if args.cfd_loop:
        run_cfd_loop(args)
        return
    if args.refmap:
        run_refmap(args)
        return
    if args.batching:
        run_batching(args)
        return
    if args.precision_forms:
        run_precision_forms(args)
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if world > 1:
        import torch

        torch.distributed.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    m, st, dt, n, res, clk, e2e_s, learned, head, mlp_ms = run_ours(args, rank, world)
    if rank != 0:
        return
    hd = res["headline"]
    value = world * n * args.steps / (hd["ms_total"] / 1e3)
    ms_per_step = hd["ms_total"] / args.steps
    # roofline of the integration kernel (FP64 pipe): algorithmic FP64 flops of one
    # launch (per-step work x the Rosenbrock steps the launch took) / its event-timed
    # duration averaged over the timed steps
    w_step = algorithmic_fp64_flops_per_step(m, 1, 1)
    ff_share = float_float_flops_per_step(m, 1) / w_step
    substeps_per_launch = hd["substeps"]  # totals of the last launch
    achieved = w_step * substeps_per_launch / (hd["kernel_ms"] / 1e3) / 1e12
    line = {
        "metric": METRIC,
        "value": value, "unit": "cells*step/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": args.workload, "n_cells": n,
                   "mechanism": f"{m.n_species} species / {m.n_reactions} reactions (seeded synthetic)",
                   "pressure_bar": float(st.p[0] / 1e6), "dt_s": dt, "rtol": RTOL, "atol": ATOL,
                   "form": "mixed precision + queue" + (" + learned order/h0" if learned else ""),
                   "l2": "flushed (256 MB write) before every step", "parallelism": "replicas" if world > 1 else "1 GPU"},
        "plain_fp64": None,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS, "traffic": kernel_traffic(n),
                     "kernel": "chem::k_integrate<4, mixed>", "kernel_ms": hd["kernel_ms"],
                     "float_float_share": ff_share,
                     "fp64_executed_frac": achieved * (1.0 - ff_share) / FP64_PEAK_TFLOPS,
                     "note": "FP64 pipe; algorithmic FP64-precision flops per launch / CUDA-event launch time; "
                             "float_float_share of them (third-body sums, Jacobian assembly, refinement "
                             "residuals) run as float-float arithmetic on the FP32 pipe, fp64_executed_frac "
                             "counts the rest only; peak derived: 2 DFMA/clk/SM x 152 SMs x 2 flop x 2070 MHz"},
        "clocks": clk,
        "e2e": {"value": world * n * args.steps / e2e_s, "unit": "cells*step/s",
                "h2d_bytes_per_step": int(n * (m.n_species + 2) * 8), "d2h_bytes_per_step": int(n * (m.n_species + 1) * 8)},
        "gpu_launches": None,
        "substeps_per_step": hd["substeps"], "failed_cells": hd["failed"],
    }
    if "plain_fp64" in res:
        pl = res["plain_fp64"]
        pv = n * pl["steps"] / (pl["ms_total"] / 1e3)
        w0 = algorithmic_fp64_flops_per_step(m, 0, 0)
        a0 = w0 * pl["substeps"] / (pl["kernel_ms"] / 1e3) / 1e12
        line["plain_fp64"] = {"value": pv, "ms_per_step": pl["ms_total"] / pl["steps"], "kernel_ms": pl["kernel_ms"],
                              "substeps_per_step": pl["substeps"],
                              "roofline_fp64_frac": a0 / FP64_PEAK_TFLOPS, "achieved_tflops": a0}
        if "phases" in pl:
            line["plain_fp64"]["phase_share"] = pl["phases"]
        line["speedup_vs_plain_fp64"] = value / pv
    if "mixed" in res:
        mx = res["mixed"]
        mv = n * mx["steps"] / (mx["ms_total"] / 1e3)
        line["mixed_without_learned"] = {"value": mv, "ms_per_step": mx["ms_total"] / mx["steps"],
                                         "kernel_ms": mx["kernel_ms"], "substeps_per_step": mx["substeps"]}
        if "phases" in mx:
            line["mixed_without_learned"]["phase_share"] = mx["phases"]
        line["learned_gain"] = value / mv
    if "w_method" in res:
        wm = res["w_method"]
        wv = n * wm["steps"] / (wm["ms_total"] / 1e3)
        line["w_method_fp32_assembly"] = {
            "value": wv, "ms_per_step": wm["ms_total"] / wm["steps"], "kernel_ms": wm["kernel_ms"],
            "substeps_per_step": wm["substeps"], "rejects_per_step": wm["rejects"], "failed_cells": wm["failed"],
            "headline_substeps_per_step": hd["substeps"], "headline_rejects_per_step": hd["rejects"],
            "speed_vs_headline": wv / value,
            "form": "ROS34PW2 W-method, Jacobian assembled in FP32, FP32 Gauss-Jordan, refinement "
                    "against the FP32 matrix, queue"}
        if "phases" in wm:
            line["w_method_fp32_assembly"]["phase_share"] = wm["phases"]
    if "phases" in hd:
        line["phase_share"] = hd["phases"]
        line["phase_roofline"] = phase_rooflines(m, hd, n, mlp_ms)
    # per step: the integration kernel, plus (learned form) per 65,536-cell chunk the
    # feature, two GEMM and head kernels of the MLP, and 3 counting-sort kernels
    chunks = (n + 65535) // 65536
    line["gpu_launches"] = args.steps * (1 + ((4 * chunks + 3) if learned else 0))
    extra = []
    if world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(m, st, dt, args.cpu_seconds)
        extra = cb.pop("_results")
        line["cpu_baseline"] = cb
    # parity in the same run: the timed forms' outputs against the oracle on a sample
    line["parity"] = same_run_parity(m, st, dt, res, args.parity_per_class, args.parity_costliest, extra)
    print(json.dumps(line))
    if not line["parity"]["ok"]:
        print("parity bound exceeded: " + json.dumps(line["parity"]), file=sys.stderr)
        sys.exit(1)


if __name__ == "__main__":
    main()
