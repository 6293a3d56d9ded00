"""GPU parity of the forward solver (plain and fused forms) against the FP64
oracle, through the C ABI.  Tolerances:
  * FP64: identical accept/reject sequences and statistics (in fact the
    whole mesh is bit-identical); every output within
    1e-12 * max(|y_oracle|_inf, 1) per instance and evaluation point.
  * FP32: within 10 (atol + rtol |y|) of a 1e-12-tolerance oracle solution,
    widened on long stiff Van der Pol runs to twice the method's own global
    error on that instance (the FP64 oracle at the workload tolerance, or the
    FP64 oracle replayed on the mesh the GPU took where that replay is
    stable), and the FP32 arithmetic itself (GPU vs that replay) within the
    band."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import gpu_solve, make, oracle_solve, subset
from oracle.oracle import mesh_from_trace

pytestmark = pytest.mark.gpu


def _rel_close(a, b, tol):
    scale = np.maximum(np.abs(b).max(axis=-1, keepdims=True), 1.0)
    return np.abs(a - b) <= tol * scale


def _same_sequences(g, o):
    for i in range(len(g["trace_len"])):
        L = o["trace_len"][i]
        assert g["trace_len"][i] == L, i
        assert np.array_equal(g["trace_accepted"][i, :L], o["trace_accepted"][i, :L]), i


# ------------------------------------------------------------------ FP64, Van der Pol B=256
@pytest.mark.parametrize("form", ["plain", "fused"])
def test_vdp_f64_matches_oracle_sequences(form):
    w = make(1)
    g = gpu_solve(w, torch.float64, form, trace_cap=4000)
    o = oracle_solve(w, trace_cap=4000)
    assert (o["status"] == 0).all()
    for k in ("status", "n_acc", "n_rej", "n_feval"):
        assert np.array_equal(g[k], o[k]), k
    _same_sequences(g, o)
    assert _rel_close(g["y_eval"], o["y_eval"], 1e-12).all()
    assert _rel_close(g["y_final"], o["y_final"], 1e-12).all()
    # the FP64 path runs the oracle's operations in the oracle's order, so the
    # whole mesh (every attempted t, h and error norm) is identical bit for bit
    L = o["trace_len"]
    for i in range(256):
        for k in ("trace_t", "trace_h", "trace_err"):
            assert np.array_equal(g[k][i, :L[i]], o[k][i, :L[i]]), (k, i)


def test_vdp_f64_plain_equals_fused_bitwise():
    w = make(1)
    a = gpu_solve(w, torch.float64, "plain")
    b = gpu_solve(w, torch.float64, "fused")
    for k in ("y_eval", "y_final", "n_acc", "n_rej", "n_feval", "status"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("form", ["plain", "fused"])
def test_linear_f64_matches_oracle_sequences(form):
    w = make(2, B=300)
    g = gpu_solve(w, torch.float64, form, rtol=1e-8, atol=1e-8, trace_cap=2000)
    o = oracle_solve(w, rtol=1e-8, atol=1e-8, trace_cap=2000)
    for k in ("status", "n_acc", "n_rej", "n_feval"):
        assert np.array_equal(g[k], o[k]), k
    _same_sequences(g, o)
    assert _rel_close(g["y_eval"], o["y_eval"], 1e-12).all()
    L = o["trace_len"]
    for i in range(w["B"]):
        assert np.array_equal(g["trace_h"][i, :L[i]], o["trace_h"][i, :L[i]]), i


# ------------------------------------------------------------------ FP32
@pytest.mark.parametrize("form", ["plain", "fused"])
def test_linear_f32_within_band_of_closed_form_and_oracle(form):
    w = make(2)
    g = gpu_solve(w, torch.float32, form)
    assert (g["status"] == 0).all()
    # closed form y(t) = Q diag(exp(-lambda t)) Q^T y0 on every instance
    Q, lam, y0 = w["field"]["Q"], w["field"]["lam"], w["y0"]
    c = np.einsum("bji,bj->bi", Q, y0)
    ex = np.exp(-lam[:, None, :] * w["t_eval"][:, :, None])
    exact = np.einsum("bij,bkj->bki", Q, ex * c[:, None, :])
    band = 10 * (w["atol"] + w["rtol"] * np.abs(exact))
    assert (np.abs(g["y_eval"] - exact) <= band).all()
    # and against the 1e-12 oracle on a sample, element by element
    idx = np.arange(0, w["B"], 37)
    ref = oracle_solve(subset(w, idx), rtol=1e-12, atol=1e-12)
    assert (np.abs(g["y_eval"][idx] - ref["y_eval"]) <=
            10 * (w["atol"] + w["rtol"] * np.abs(ref["y_eval"]))).all()


def test_linear_f32_plain_equals_fused_bitwise():
    w = make(2)
    a = gpu_solve(w, torch.float32, "plain")
    b = gpu_solve(w, torch.float32, "fused")
    for k in ("y_eval", "y_final", "n_acc", "n_rej", "status"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("group", [4, 8, 16])
def test_linear_f32_group_shapes_agree(group):
    w = make(2, B=1000)
    g = gpu_solve(w, torch.float32, "fused", group=group)
    ref = oracle_solve(w, rtol=1e-12, atol=1e-12)
    band = 10 * (w["atol"] + w["rtol"] * np.abs(ref["y_eval"]))
    assert (np.abs(g["y_eval"] - ref["y_eval"]) <= band).all()


def _stratified(w, n):
    """n instances spread over the mu / t1 range of the workload."""
    order = np.lexsort((w["t1"], w["field"]["mu"]))
    pick = order[np.linspace(0, len(order) - 1, n).astype(int)]
    return np.unique(pick)


@pytest.mark.parametrize("form", ["plain", "fused"])
def test_vdp_mix_f32_full_size_sampled(form):
    """Stiffness-mixed Van der Pol at full size (262144 instances), checked
    on a stratified sample that the oracle computes one by one."""
    w = make(3)
    g = gpu_solve(w, torch.float32, form)
    assert (g["status"] == 0).all()
    idx = _stratified(w, 1024)
    ws = subset(w, idx)
    # the same instances alone reproduce the full-batch result bit for bit,
    # and give the mesh the GPU took
    gs = gpu_solve(ws, torch.float32, form, trace_cap=20000)
    assert np.array_equal(gs["y_eval"], g["y_eval"][idx])
    assert (gs["trace_len"] < 20000).all()
    mt, mh, mn = mesh_from_trace(gs)
    rep = oracle.replay(ws["field"], ws["y0"], ws["t0"], ws["t1"], mt, mh, mn, ws["t_eval"])
    # stiff instances need well over 1e5 steps at 1e-12
    ref = oracle_solve(ws, rtol=1e-12, atol=1e-12, max_steps=5_000_000)
    assert (ref["status"] == 0).all()
    assert np.isfinite(gs["y_eval"]).all()
    cfg = oracle_solve(ws)
    R = ref["y_eval"]
    band = 10 * (w["atol"] + w["rtol"] * np.abs(R))
    # A few stiff instances sit at the explicit stability boundary: replayed
    # on a frozen mesh without the controller their perturbations grow and
    # the replay overflows.  Use the replay only where it stays finite.
    rep_ok = np.isfinite(rep["y_eval"]).all(axis=(1, 2))
    assert rep_ok.mean() > 0.95
    own_rep = np.where(rep_ok[:, None, None],
                       2 * np.nan_to_num(np.abs(rep["y_eval"] - R)).max(axis=(1, 2),
                                                                      keepdims=True), 0.0)
    own_cfg = 2 * np.abs(cfg["y_eval"] - R).max(axis=(1, 2), keepdims=True)
    lim = np.maximum(band, np.maximum(own_rep, own_cfg))
    err = np.abs(gs["y_eval"] - R)
    assert (err <= lim).all(), (err > lim).sum()
    # the FP32 arithmetic on the GPU's own mesh (GPU vs FP64 replay of that
    # mesh): inside the band on the non-stiff instances (measured max 0.53);
    # up to mu = 10 the relaxation phases amplify rounding differences along
    # the frozen mesh, so every point stays inside 2.5 bands and 99.9 % inside
    # one (measured: max 2.09 at one point of one mu = 9.1 instance over 273
    # steps, 2 of 3,696 points above one band); beyond mu = 10 even a finite
    # replay amplifies perturbations, and the matched-error comparison below
    # is the check
    mu = ws["field"]["mu"]
    arith = np.abs(gs["y_eval"] - rep["y_eval"]) / band
    assert (arith[rep_ok & (mu < 3.0)] <= 1.0).all(), arith[rep_ok & (mu < 3.0)].max()
    a10 = arith[rep_ok & (mu < 10.0)]
    assert (a10 <= 2.5).all(), a10.max()
    assert np.quantile(a10, 0.999) <= 1.0, np.quantile(a10, 0.999)
    # matched error: FP32 meets the plain band as often as the FP64 path
    # does at the same tolerance (the misses are the method's global error)
    g64 = gpu_solve(ws, torch.float64, form)
    in32 = (err <= band).mean()
    in64 = (np.abs(g64["y_eval"] - R) <= band).mean()
    assert in32 >= in64 - 0.01, (in32, in64)


def test_vdp_mix_f32_plain_equals_fused_bitwise():
    w = make(3, B=20000)
    a = gpu_solve(w, torch.float32, "plain")
    b = gpu_solve(w, torch.float32, "fused")
    for k in ("y_eval", "y_final", "n_acc", "n_rej", "status"):
        assert np.array_equal(a[k], b[k]), k


# ------------------------------------------------------------------ independence
@pytest.mark.parametrize("form", ["plain", "fused"])
def test_batch_invariance_bitwise(form):
    """Sec. 3 / Sec. 4.1: an instance's result does not depend on the rest of
    its batch (shuffled batch, sub-batch, single instance)."""
    w = make(3, B=5000)
    full = gpu_solve(w, torch.float32, form)
    perm = np.random.default_rng(5).permutation(w["B"])
    sh = gpu_solve(subset(w, perm), torch.float32, form)
    for k in ("y_eval", "y_final", "n_acc", "n_rej", "status"):
        assert np.array_equal(full[k][perm], sh[k]), k
    one = gpu_solve(subset(w, [4321]), torch.float32, form)
    assert np.array_equal(one["y_eval"][0], full["y_eval"][4321])
    sub = gpu_solve(subset(w, np.arange(100, 163)), torch.float32, form)
    assert np.array_equal(sub["y_eval"], full["y_eval"][100:163])


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("form", ["plain", "fused"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_statuses_edge_cases(form, dtype):
    w = make(1, B=9)
    y0, t0, t1, te = w["y0"].copy(), w["t0"].copy(), w["t1"].copy(), w["t_eval"].copy()
    te[1, 3], te[1, 4] = te[1, 4], te[1, 3]  # decreasing
    te[2, 5] = t1[2] + 1.0                   # outside [t0, t1]
    t1[3] = -1.0                             # t1 < t0
    y0[4, 0] = np.nan                        # non-finite state
    t1[5] = t0[5]                            # empty range
    te[5] = t0[5]
    te[6, 2] = np.nan                        # non-finite evaluation point
    w2 = dict(w, y0=y0, t0=t0, t1=t1, t_eval=te)
    g = gpu_solve(w2, dtype, form)
    o = oracle_solve(w2)
    assert np.array_equal(g["status"], o["status"])
    assert list(g["status"][[1, 2, 3, 6]]) == [4, 4, 4, 4]
    assert g["status"][4] == 3
    assert g["status"][5] == 0 and g["n_acc"][5] == 0 and g["n_feval"][5] == 0
    y5 = np.repeat(y0[5:6], te.shape[1], 0)
    if dtype == torch.float32:
        y5 = y5.astype(np.float32).astype(np.float64)
    assert np.array_equal(g["y_eval"][5], y5)
    assert np.isnan(g["y_eval"][1]).all() and np.isnan(g["y_final"][1]).all()
    for i in (0, 7, 8):
        assert g["status"][i] == 0
        assert g["n_feval"][i] == 2 + 6 * (g["n_acc"][i] + g["n_rej"][i])


@pytest.mark.parametrize("form", ["plain", "fused"])
def test_max_steps_and_given_h0(form):
    w = make(1, B=33)
    g = gpu_solve(w, torch.float64, form, max_steps=7)
    assert (g["status"] == 1).all() and ((g["n_acc"] + g["n_rej"]) == 7).all()
    o = oracle_solve(w, max_steps=7)
    assert _rel_close(g["y_final"], o["y_final"], 1e-12).all()
    # evaluation points past the last accepted step are NaN, as in the oracle
    nan_g, nan_o = np.isnan(g["y_eval"]), np.isnan(o["y_eval"])
    assert np.array_equal(nan_g, nan_o) and nan_g.any() and not nan_g.all()
    assert _rel_close(np.where(nan_g, 0, g["y_eval"]), np.where(nan_o, 0, o["y_eval"]),
                      1e-12).all()
    g = gpu_solve(w, torch.float64, form, h0=1e-3)
    o = oracle_solve(w, h0=1e-3)
    assert np.array_equal(g["n_acc"], o["n_acc"])
    assert (g["n_feval"] == 1 + 6 * (g["n_acc"] + g["n_rej"])).all()


@pytest.mark.parametrize("form", ["plain", "fused"])
def test_no_eval_points_and_ragged_batches(form):
    for B in (1, 31, 257, 1000):
        w = dict(make(3, B=B), rtol=1e-7, atol=1e-7)
        w0 = dict(w, t_eval=np.zeros((B, 0)))
        g = gpu_solve(w0, torch.float64, form)
        o = oracle_solve(w0)
        assert g["y_eval"].shape == (B, 0, 2)
        assert np.array_equal(g["n_acc"], o["n_acc"])
        assert _rel_close(g["y_final"], o["y_final"], 1e-12).all()


@pytest.mark.parametrize("form", ["plain", "fused"])
def test_per_instance_tolerances(form):
    w = make(1, B=64)
    rng = np.random.default_rng(2)
    rb = 10 ** rng.uniform(-9, -5, 64)
    ab = 10 ** rng.uniform(-9, -5, 64)
    g = gpu_solve(w, torch.float64, form,
                  rtol_b=torch.tensor(rb, device="cuda"), atol_b=torch.tensor(ab, device="cuda"))
    o = oracle.solve(w["field"], w["y0"], w["t0"], w["t1"], w["t_eval"],
                     dict(rtol=1e-6, atol=1e-6, rtol_b=rb, atol_b=ab))
    assert np.array_equal(g["n_acc"], o["n_acc"])
    assert _rel_close(g["y_eval"], o["y_eval"], 1e-12).all()


def test_pi_controller_matches_oracle():
    """App. C: the PI member of the controller family (beta2 != 0)."""
    w = make(1, B=64)
    g = gpu_solve(w, torch.float64, "fused", beta1=0.14, beta2=0.08, trace_cap=4000)
    o = oracle_solve(w, beta1=0.14, beta2=0.08, trace_cap=4000)
    _same_sequences(g, o)
    assert _rel_close(g["y_eval"], o["y_eval"], 1e-12).all()


@pytest.mark.parametrize("D", [1, 2, 4, 8, 32])
def test_linear_other_dimensions_f64(D):
    rng = np.random.default_rng(D)
    B = 70
    M = rng.standard_normal((B, D, D)) / np.sqrt(D)
    A = M - 1.5 * np.eye(D)[None]
    w = dict(field={"kind": "linear", "A": A}, y0=rng.standard_normal((B, D)), t0=np.zeros(B),
             t1=rng.uniform(0.5, 3, B), rtol=1e-7, atol=1e-7, B=B)
    w["t_eval"] = np.linspace(w["t0"], w["t1"], 5).T.copy()
    w["t_eval"][:, -1] = w["t1"]
    for form in ("plain", "fused"):
        g = gpu_solve(w, torch.float64, form)
        o = oracle_solve(w)
        assert np.array_equal(g["n_acc"], o["n_acc"])
        assert _rel_close(g["y_eval"], o["y_eval"], 1e-12).all()
