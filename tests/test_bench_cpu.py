"""bench.py's reference arm (the CPU oracle timed on the host cores), alone and under
torchrun with two gloo ranks: rank 0 prints the one JSON line, the other rank exits 0
without work (the multi-rank launch path of the benchmark, on the CPU)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
ARGS = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0", "--cpu-seconds", "2",
        "--workload", "h2_10_1k"]


@pytest.fixture(scope="module")
def built_oracle():
    import oracle

    oracle.build()


def _json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.strip().startswith("{")]


def _check_line(d):
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["unit"] == "cells*step/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "h2_10_1k"
    # the same metric string as the GPU arm, and per-step times actually measured:
    # each step integrates step_cells cells, so value x ms_per_step = step_cells
    import bench

    assert d["metric"] == bench.METRIC
    k = d["config"]["step_cells"]
    assert abs(d["value"] * d["ms_per_step"] / 1e3 - k) <= 1e-6 * k


def test_same_run_parity_host_logic(built_oracle):
    """The bench's same-run parity check on the host: the oracle's own results pass; one
    sampled cell moved by 2e-6 T, or one mass fraction moved past its bound, fails."""
    import numpy as np

    import bench
    import oracle
    from paper_2112_05834_gb300 import synth

    m, st, dt = synth.workload("c54_65k", n_cells=96, state_seed=3)
    r = oracle.integrate(m, st.T, st.p, st.Y, dt, bench.RTOL, bench.ATOL)
    res = {"headline": {"T": r["T"].copy(), "Y": r["Y"].copy(), "cell_substeps": r["substeps"]}}
    out = bench.same_run_parity(m, st, dt, res, per_class=6, costliest=4)
    assert out["ok"] and out["cells"] >= 16 and out["forms"]["headline"]["cells_outside"] == 0
    costly = int(np.argmax(r["substeps"]))  # always in the sample
    bad = {"headline": dict(res["headline"], T=res["headline"]["T"].copy())}
    bad["headline"]["T"][costly] *= 1 + 2e-6
    out = bench.same_run_parity(m, st, dt, bad, per_class=6, costliest=4)
    assert not out["ok"] and out["forms"]["headline"]["cells_outside"] == 1
    bad = {"headline": dict(res["headline"], Y=res["headline"]["Y"].copy())}
    bad["headline"]["Y"][costly, 3] += 2e-8 + 2e-5 * abs(bad["headline"]["Y"][costly, 3])
    assert not bench.same_run_parity(m, st, dt, bad, per_class=6, costliest=4)["ok"]


def test_reference_arm_single(built_oracle):
    r = subprocess.run([sys.executable] + ARGS, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_line(lines[0])


def test_reference_arm_two_gloo_ranks(built_oracle):
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port)] + ARGS + ["--gpus", "2"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1  # rank 0 only
    _check_line(lines[0])
    assert lines[0]["n_gpus"] == 2


def test_flop_model_split():
    """The roofline's flop model: the float-float part (third-body sums of the 7 RHS
    evaluations, assembly 6 n^2, residuals 12 n^2 per sweep) is a part of the mixed
    form's count, counted term by term here for the 54-species workload."""
    import bench
    from paper_2112_05834_gb300 import synth

    m, _, _ = synth.workload("c54_65k", n_cells=4)
    K, I = m.n_species, m.n_reactions
    n = K + 1
    n_tb = int((m.rxn_type >= 1).sum())
    n_fo = int((m.rxn_type >= 2).sum())
    total = bench.algorithmic_fp64_flops_per_step(m, 1, 1)
    assert total == 7 * (41 * K + 22 * I + 2 * n_tb * K + 30 * n_fo) + 24 * I + 6 * n * n + 12 * n * n
    ff = bench.float_float_flops_per_step(m, 1)
    assert ff == 7 * 2 * n_tb * K + 6 * n * n + 12 * n * n
    assert 0.0 < ff < total
    # more refinement sweeps add residual flops to both counts alike
    assert bench.float_float_flops_per_step(m, 3) - ff == bench.algorithmic_fp64_flops_per_step(m, 1, 3) - total
