"""Learned cost / initial-step model on the GPU: BF16 gradients against the FP64
reference, training, and what the trained model gains over the method without it.
The integrator's error control judges every step, so the learned form must meet
the same parity bound against the oracle."""
import time

import numpy as np
import pytest

from oracle import mlp_ref
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


def _logged(pkg, name, n, seed):
    m, st, dt = synth.workload(name, n_cells=n, state_seed=seed)
    integ = pkg.Integrator(m)
    T, p, Y = _dev(st.T), _dev(st.p), _dev(st.Y)
    sub, hf = pkg.log_cells(integ, T, p, Y, dt)
    return m, st, dt, integ, (T, p, Y, sub, hf)


# Element-wise bounds of the BF16 model against the FP64 reference, as multiples of
# (|ref| + rms(ref)) over each output column or gradient tensor. The kernels round
# every matrix-product operand to BF16 (unit roundoff u = 2^-8) and accumulate in
# FP32; a CPU emulation of those rounding points over five seeded problems of this
# shape gave at most 0.013 (outputs) and 0.032 (gradients, W1 the largest), so the
# bounds below (about 10 u and 25 u) keep a 3x margin while a wrong unit, a swapped
# block, a missing factor or a sign error moves an entry by O(|ref| + rms).
FWD_BOUND = 0.04
GRAD_BOUND = 0.1


def _mlp_problem(n, seed):
    """Seeded cells of the 54-species workload, synthetic targets (substeps log-uniform
    in [1, 400], first steps log-uniform in [1e-12, 1e-6] s), normalisation from the
    oracle's features and targets, seeded weights: all rounded to FP32, the model's
    storage type, so both sides start from identical parameters."""
    m, st, _ = synth.workload("c54_65k", n_cells=n, state_seed=seed)
    D = m.n_species + 2
    rng = np.random.default_rng(seed)
    sub = np.exp(rng.uniform(0.0, np.log(400.0), n)).astype(np.int32)
    hf = np.exp(rng.uniform(np.log(1e-12), np.log(1e-6), n))
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    x = mlp_ref.features(st.T, st.p, st.Y)
    t = mlp_ref.targets(sub, hf)
    norm = [f32(x.mean(0)), f32(np.maximum(x.std(0), 1e-3)), f32(t.mean(0)), f32(t.std(0))]
    params = {k: f32(v) for k, v in mlp_ref.init_params(D, seed=seed).items()}
    buf = np.concatenate(norm + [params[k].ravel() for k in mlp_ref.ORDER]).astype(np.float32)
    xs = (x - norm[0]) / norm[1]
    ts = (t - norm[2]) / norm[3]
    return m, st, sub, hf, norm, params, buf, xs, ts


def _scaled_err(got, ref, axis=None):
    rms = np.sqrt(np.mean(ref * ref, axis=axis, keepdims=axis is not None))
    return np.abs(got - ref) / (np.abs(ref) + rms)


def test_predict_matches_fp64_reference(pkg):
    """chem_mlp_predict against the FP64 forward pass, entry by entry, on fixed
    parameters loaded with chem_mlp_set_params (4,096 cells: 64 full 64-row tiles)."""
    m, st, sub, hf, norm, params, buf, xs, ts = _mlp_problem(4096, 51)
    model = pkg.CostModel(m.n_species, seed=0)
    model.set_params(buf)
    lc, lh = model.predict(_dev(st.T), _dev(st.p), _dev(st.Y))
    out, _ = mlp_ref.forward(params, xs)
    got = np.stack([lc.cpu().numpy(), lh.cpu().numpy()], axis=1).astype(np.float64)
    got = (got - norm[2]) / norm[3]  # back to the standardised outputs
    e = _scaled_err(got, out, axis=0)
    print("max |out - ref| / (|ref| + rms) =", e.max(), "(bound", FWD_BOUND, ")")
    assert np.all(np.isfinite(got))
    assert e.max() <= FWD_BOUND


def test_gradient_matches_fp64_reference(pkg):
    """chem_mlp_gradient (BF16 operands, FP32 accumulation) against the FP64 chain
    rule, every entry of every tensor, on 2,048 cells (a ragged last K chunk: D = 56);
    the loss within 1 %."""
    m, st, sub, hf, norm, params, buf, xs, ts = _mlp_problem(2048, 41)
    D = m.n_species + 2
    model = pkg.CostModel(m.n_species, seed=3)
    model.set_params(buf)
    sub_d = torch.tensor(sub, device="cuda", dtype=torch.int32)
    loss_g, g_gpu = model.gradient(_dev(st.T), _dev(st.p), _dev(st.Y), sub_d, _dev(hf))
    L, g = mlp_ref.loss_and_grad(params, xs, ts)
    assert abs(loss_g - L) <= 1e-2 * L, (loss_g, L)
    gg = mlp_ref.unflatten(g_gpu.astype(np.float64), D)
    for k in mlp_ref.ORDER:
        e = _scaled_err(gg[k], g[k])
        print(k, "max |g - ref| / (|ref| + rms) =", e.max())
        assert e.max() <= GRAD_BOUND, (k, e.max())


def test_adam_matches_fp64_reference(pkg):
    """Two chem_mlp_apply_gradient updates of a fresh model (its first two Adam steps)
    with seeded gradients against the FP64 Adam of the oracle: the FP32 update is
    within 2^-21 of each weight plus 1e-5 of the step size."""
    m, st, sub, hf, norm, params, buf, xs, ts = _mlp_problem(64, 52)
    D = m.n_species + 2
    model = pkg.CostModel(m.n_species, seed=5)
    model.set_params(buf)
    nn = 2 * D + 4
    w = buf[nn:].astype(np.float64)
    rng = np.random.default_rng(53)
    lr = 1e-3
    mo, vo, t = np.zeros_like(w), np.zeros_like(w), 0
    for step in range(2):
        g = rng.standard_normal(w.size) * np.exp(rng.uniform(-6.0, 2.0, w.size))
        g[rng.choice(w.size, 50, replace=False)] = 0.0
        g32 = g.astype(np.float32)
        model.apply_gradient(g32, lr=lr)
        w, mo, vo, t = mlp_ref.adam_step(w, g32.astype(np.float64), mo, vo, t, lr)
        got = model.get_params()[nn:].astype(np.float64)
        err = np.abs(got - w)
        tol = 2.0 ** -21 * np.abs(w) + 1e-5 * lr
        print("Adam step", step + 1, "max |w - ref| =", err.max(), "max err / tol =", (err / tol).max())
        assert np.all(err <= tol), step
    # the normalisation is untouched by the update
    np.testing.assert_array_equal(model.get_params()[:nn], buf[:nn])


def test_training_learns_cost(pkg):
    m, st, dt, integ, (T, p, Y, sub, hf) = _logged(pkg, "c54_65k", 16384, 42)
    model = pkg.CostModel(m.n_species, seed=4)
    losses = model.train(T, p, Y, sub, hf, epochs=20, batch=2048, lr=1e-3, seed=5)
    print("loss per epoch:", losses)
    assert losses[-1] < 0.5 * losses[0]
    # held-out cells: predicted cost ranks the actual cost
    m2, st2, dt2, integ2, (T2, p2, Y2, sub2, hf2) = _logged(pkg, "c54_65k", 4096, 43)
    lc, lh = model.predict(T2, p2, Y2)
    a = np.log(np.maximum(sub2.cpu().numpy(), 1))
    b = lc.cpu().numpy()
    ra, rb = np.argsort(np.argsort(a)), np.argsort(np.argsort(b))
    rho = np.corrcoef(ra, rb)[0, 1]
    print("Spearman(predicted, actual substeps) =", rho)
    assert rho >= 0.8
    err_h = np.abs(lh.cpu().numpy() - np.log(hf2.cpu().numpy()))
    print("median |ln h0 error| =", np.median(err_h))


def _timed_integrate(integ, st, dt, reps=3):
    """Median CUDA-event time (ms) of `reps` calls from the same input (one warm-up call
    first), the outputs of the last call and its per-cell statistics."""
    stream = torch.cuda.current_stream()
    p = _dev(st.p)
    T, Y = _dev(st.T), _dev(st.Y)
    integ.integrate(T, p, Y, dt, RTOL, ATOL)
    ms = []
    for _ in range(reps):
        T, Y = _dev(st.T), _dev(st.Y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        integ.integrate(T, p, Y, dt, RTOL, ATOL)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    s = integ.stats(st.T.shape[0])
    return float(np.median(ms)), {"T": T.cpu().numpy(), "Y": Y.cpu().numpy(),
                                  "substeps": s["substeps"].cpu().numpy(), "rejects": s["rejects"].cpu().numpy(),
                                  "status": s["status"].cpu().numpy()}


def test_learned_form_gain_and_parity(pkg):
    """What the trained network gains, held out: trained on the logs of one seeded
    65,536-cell batch of the 54-species workload, evaluated on another, against the same
    form without it (mixed precision, work queue, index order, heuristic initial step).
    Device time of the whole call (CUDA events, MLP inference and cost sort included),
    substeps and rejections are reported; the learned form must keep every sampled cell
    within the parity bound, fail no cell, and not run slower than the plain form by more
    than 3 % (its initial step is kept inside the heuristic's envelope, so a wrong
    prediction costs at most the heuristic's own range)."""
    import oracle

    oracle.build()
    n = 65536
    m, st_tr, dt = synth.workload("c54_65k", n_cells=n, state_seed=44)
    _, st, _ = synth.workload("c54_65k", n_cells=n, state_seed=45)
    plain = pkg.Integrator(m, precision=1, scheduler=2)
    learned = pkg.Integrator(m, precision=1, scheduler=2)
    Ttr, ptr, Ytr = _dev(st_tr.T), _dev(st_tr.p), _dev(st_tr.Y)
    sub, hf = pkg.log_cells(plain, Ttr, ptr, Ytr, dt)
    model = pkg.CostModel(m.n_species, seed=6)
    model.train(Ttr, ptr, Ytr, sub, hf, epochs=20, batch=8192, lr=1e-3, seed=7)
    model.attach(learned)
    learned.set_option("order", 1)
    learned.set_option("h0", 1)
    out = {}
    for name, integ in (("plain", plain), ("learned", learned)):
        ms, o = _timed_integrate(integ, st, dt)
        o["ms"] = ms
        out[name] = o
        print(name, "%.1f ms" % ms, "substeps", int(o["substeps"].sum()), "rejects", int(o["rejects"].sum()))
        assert np.all(o["status"] == 0)
    gain = out["plain"]["ms"] / out["learned"]["ms"]
    ratio = out["learned"]["substeps"].sum() / out["plain"]["substeps"].sum()
    print("learned part, held out on %d cells: speed-up %.3f, substeps ratio %.4f" % (n, gain, ratio))
    # parity of both forms on sampled cells, the costliest included
    rng = np.random.default_rng(1)
    pick = np.unique(np.concatenate([rng.choice(n, 24, replace=False),
                                     np.argsort(out["learned"]["substeps"])[-8:]]))
    ref = oracle.integrate(m, st.T[pick], st.p[pick], st.Y[pick], dt, RTOL, ATOL)
    for name, o in out.items():
        assert np.all(np.abs(o["T"][pick] - ref["T"]) <= 1e-6 * ref["T"]), name
        assert np.all(np.abs(o["Y"][pick] - ref["Y"]) <= 1e-8 + 1e-5 * np.abs(ref["Y"])), name
    assert gain >= 0.97
    assert ratio <= 1.02


def test_cfd_loop_learned(pkg):
    """The learned-scheduling configuration at 65,536 cells of the 100-species
    mechanism: between CFD steps T += U[-50, 50] K and Y mixes with a random partner
    cell. Steps 1-3 run the plain heuristic and log; the model trains on those logs;
    steps 4-6 use the learned order and initial step. Every step's outputs match the
    oracle on sampled cells of that step's inputs (random cells and the step's
    costliest), and no cell fails."""
    import oracle

    oracle.build()
    n = 65536
    m, st, dt = synth.workload("c100_1m", n_cells=n, state_seed=46)
    integ = pkg.Integrator(m, precision=1, scheduler=2)
    model = pkg.CostModel(m.n_species, seed=8)
    logs = []
    rng = np.random.default_rng(2)
    for step in range(6):
        T, p, Y = _dev(st.T), _dev(st.p), _dev(st.Y)
        if step == 3:
            cat = [torch.cat([l[k] for l in logs]) for k in range(5)]
            losses = model.train(*cat, epochs=20, batch=8192, lr=1e-3, seed=9)
            assert losses[-1] < losses[0]
            model.attach(integ)
            integ.set_option("order", 1)
            integ.set_option("h0", 1)
        T_in, Y_in = T.clone(), Y.clone()
        integ.integrate(T, p, Y, dt, RTOL, ATOL)
        s = integ.stats(n)
        assert int((s["status"] != 0).sum()) == 0
        if step < 3:
            logs.append((T_in, p, Y_in, s["substeps"].clone(), s["h_first"].clone()))
        sub = s["substeps"].cpu().numpy()
        pick = np.unique(np.concatenate([rng.choice(n, 8, replace=False), np.argsort(sub)[-2:]]))
        ref = oracle.integrate(m, st.T[pick], st.p[pick], st.Y[pick], dt, RTOL, ATOL)
        Tg, Yg = T.cpu().numpy(), Y.cpu().numpy()
        assert np.all(np.abs(Tg[pick] - ref["T"]) <= 1e-6 * ref["T"]), step
        assert np.all(np.abs(Yg[pick] - ref["Y"]) <= 1e-8 + 1e-5 * np.abs(ref["Y"])), step
        print("step", step + 1, "substeps", int(sub.sum()))
        st = synth.perturb_states(synth.CellStates(T=Tg, p=st.p, Y=Yg, kind=st.kind), seed=100 + step)


def test_carry_over_h0(pkg):
    """Option h0 = 2 (the OpenFOAM-style stored step, a baseline for the learned h0):
    with no history the call equals the heuristic bitwise; on the next CFD step
    (perturbed states of the same cells) every cell starts from the step its controller
    proposed last time and stays within the parity bound. Its cost against the
    heuristic is reported: the perturbation re-excites fast transients, so the
    carried-over step may cost rejections; it must not cost more than 25 % steps."""
    import oracle

    oracle.build()
    n = 4096
    m, st, dt = synth.workload("c54_65k", n_cells=n, state_seed=47)
    heur = pkg.Integrator(m, precision=1, scheduler=2)
    carry = pkg.Integrator(m, precision=1, scheduler=2, h0=2)
    first = {}
    for name, integ in (("heur", heur), ("carry", carry)):
        T, p, Y = _dev(st.T), _dev(st.p), _dev(st.Y)
        integ.integrate(T, p, Y, dt, RTOL, ATOL)
        first[name] = (T.cpu().numpy(), Y.cpu().numpy())
    np.testing.assert_array_equal(first["heur"][0], first["carry"][0])
    np.testing.assert_array_equal(first["heur"][1], first["carry"][1])
    st2 = synth.perturb_states(synth.CellStates(T=first["heur"][0], p=st.p, Y=first["heur"][1], kind=st.kind),
                               seed=48)
    out = {}
    for name, integ in (("heur", heur), ("carry", carry)):
        T, p, Y = _dev(st2.T), _dev(st2.p), _dev(st2.Y)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        integ.integrate(T, p, Y, dt, RTOL, ATOL)
        torch.cuda.synchronize()
        s = integ.stats(n)
        out[name] = {"T": T.cpu().numpy(), "Y": Y.cpu().numpy(), "time": time.perf_counter() - t0,
                     "substeps": s["substeps"].cpu().numpy(), "status": s["status"].cpu().numpy()}
        assert np.all(out[name]["status"] == 0)
    rng = np.random.default_rng(3)
    pick = np.unique(np.concatenate([rng.choice(n, 24, replace=False), np.argsort(out["carry"]["substeps"])[-8:]]))
    ref = oracle.integrate(m, st2.T[pick], st2.p[pick], st2.Y[pick], dt, RTOL, ATOL)
    for name, o in out.items():
        assert np.all(np.abs(o["T"][pick] - ref["T"]) <= 1e-6 * ref["T"]), name
        assert np.all(np.abs(o["Y"][pick] - ref["Y"]) <= 1e-8 + 1e-5 * np.abs(ref["Y"])), name
    sh, sc = int(out["heur"]["substeps"].sum()), int(out["carry"]["substeps"].sum())
    print("step 2 substeps heuristic", sh, "carried", sc, "RHS evaluations", 7 * sh + 2 * n, "vs", 7 * sc,
          "time %.4f vs %.4f s" % (out["heur"]["time"], out["carry"]["time"]))
    assert sc <= 1.25 * sh


def test_h0_range_falls_back_to_heuristic(pkg):
    """Option h0_range = z: a cell whose standardised model input has a feature beyond
    +-z training standard deviations starts from the heuristic, the others from the
    prediction. Per cell, the first step and the result then equal bitwise those of
    the heuristic run (flagged cells) or of the learned run without the range check
    (the others): each cell is integrated by one CTA, independently of the rest. The
    flags are recomputed here from the model's normalisation; cells within 1e-4 of the
    threshold in some feature are left out (the device takes ln in its own rounding)."""
    n = 8192
    m, st_tr, dt = synth.workload("c54_65k", n_cells=n, state_seed=44)
    _, st, _ = synth.workload("c54_65k", n_cells=n, state_seed=45)
    st = synth.perturb_states(st, seed=3)
    heur = pkg.Integrator(m, precision=1, scheduler=2)
    Ttr, ptr, Ytr = _dev(st_tr.T), _dev(st_tr.p), _dev(st_tr.Y)
    sub, hf = pkg.log_cells(heur, Ttr, ptr, Ytr, dt)
    model = pkg.CostModel(m.n_species, seed=6)
    model.train(Ttr, ptr, Ytr, sub, hf, epochs=4, batch=8192, lr=1e-3, seed=7)
    z = 2
    D = m.n_species + 2
    prm = model.get_params()
    mu, sd = prm[:D].astype(np.float64), prm[D:2 * D].astype(np.float64)
    x = np.concatenate([(st.T / 1000.0)[:, None], np.log(st.p)[:, None], np.log(st.Y + 1e-20)], axis=1)
    za = np.abs(((x - mu) / sd).astype(np.float32))
    far = (za > z).any(axis=1)
    clear = ~(np.abs(za - z) < 1e-4).any(axis=1)
    print("cells beyond %d sd: %d of %d (%d near the threshold)" % (z, far.sum(), n, (~clear).sum()))
    assert 0 < far.sum() < n
    runs = {}
    for name, opts in (("heur", {}), ("learned", {"h0": 1, "h0_range": 0}), ("ranged", {"h0": 1, "h0_range": z})):
        integ = pkg.Integrator(m, precision=1, scheduler=2, **opts)
        if opts:
            model.attach(integ)
        T, p, Y = _dev(st.T), _dev(st.p), _dev(st.Y)
        integ.integrate(T, p, Y, dt, RTOL, ATOL)
        s = integ.stats(n)
        assert int((s["status"] != 0).sum()) == 0, name
        runs[name] = (s["h_first"].cpu().numpy(), T.cpu().numpy(), Y.cpu().numpy())
    for i, name in ((0, "h_first"), (1, "T"), (2, "Y")):
        r = runs["ranged"][i]
        np.testing.assert_array_equal(r[far & clear], runs["heur"][i][far & clear], err_msg=name)
        np.testing.assert_array_equal(r[~far & clear], runs["learned"][i][~far & clear], err_msg=name)
    # the learned prediction does differ from the heuristic (the test would be vacuous otherwise)
    assert np.any(runs["learned"][0][far & clear] != runs["heur"][0][far & clear])
