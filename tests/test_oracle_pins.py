"""Pins of the FP64 oracle against what mathematics fixes: closed forms,
observed convergence order, brute force on tiny inputs, the controller's
steady state, the first-step error estimate of the linear test equation,
statuses and independence (Sec. 3, Sec. 4.1, App. A, App. C)."""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import sympy as sp

import oracle
import rk_exact as rk
from oracle.oracle import mesh_from_trace
from paper_2210_12375_b300 import workloads


# ---------------------------------------------------------------- helpers
def rk4_reference(f, y0, t_end, n):
    """Classical RK4 with n uniform steps (independent of the oracle)."""
    y = np.array(y0, dtype=np.float64)
    h = t_end / n
    for _ in range(n):
        k1 = f(y)
        k2 = f(y + 0.5 * h * k1)
        k3 = f(y + 0.5 * h * k2)
        k4 = f(y + h * k3)
        y = y + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    return y


def vdp_rhs(mu):
    def f(y):
        return np.stack([y[:, 1], mu * (1 - y[:, 0] ** 2) * y[:, 1] - y[:, 0]], axis=1)
    return f


def linear_exact(w, t):
    """Q diag(exp(-lambda t)) Q^T y0 for every instance and time."""
    Q, lam, y0 = w["field"]["Q"], w["field"]["lam"], w["y0"]
    c = np.einsum("bji,bj->bi", Q, y0)  # Q^T y0
    ex = np.exp(-lam[:, None, :] * t[:, :, None])  # [B,K,D]
    return np.einsum("bij,bkj->bki", Q, ex * c[:, None, :])


def uniform_mesh(B, t1, N):
    mt = np.zeros((B, N))
    mh = np.zeros((B, N))
    for i in range(B):
        h = t1[i] / N
        mt[i] = np.arange(N) * h
        mh[i] = h
    return mt, mh, np.full(B, N, np.int32)


# ---------------------------------------------------------------- closed forms
def test_linear_closed_form_tight_tolerance():
    w = workloads.make(2, B=24)
    r = oracle.solve(w["field"], w["y0"], w["t0"], w["t1"], w["t_eval"],
                     dict(rtol=1e-11, atol=1e-11))
    assert (r["status"] == 0).all()
    ex = linear_exact(w, w["t_eval"])
    err = np.abs(r["y_eval"] - ex).max()
    assert err < 1e-9, err
    # the last evaluation point is t1 and must equal y_final exactly
    assert np.array_equal(r["y_eval"][:, -1], r["y_final"])
    # t_eval == t0 gives y0 exactly
    assert np.array_equal(r["y_eval"][:, 0], w["y0"])


def test_linear_closed_form_config_tolerance_band():
    w = workloads.make(2, B=64)
    r = oracle.solve(w["field"], w["y0"], w["t0"], w["t1"], w["t_eval"],
                     dict(rtol=w["rtol"], atol=w["atol"]))
    ex = linear_exact(w, w["t_eval"])
    band = 10 * (w["atol"] + w["rtol"] * np.abs(ex))
    assert (np.abs(r["y_eval"] - ex) <= band).all()


def test_mlp_scalar_closed_form():
    """D=1, one hidden unit: y' = v tanh(w y) has sinh(w y(t)) = sinh(w y0)
    exp(w v t); pins the MLP wiring ([y; t] input, tanh hidden, linear out)
    and the solver on a nonlinear field."""
    w_, v_ = 0.8, -1.3
    field = {"kind": "mlp", "W": [np.array([[w_, 0.0]]), np.array([[v_]])],
             "b": [np.zeros(1), np.zeros(1)]}
    B = 5
    y0 = np.linspace(-1.5, 2.0, B)[:, None]
    t0 = np.zeros(B)
    t1 = np.full(B, 3.0)
    te = np.linspace(0, 3.0, 7)[None, :].repeat(B, 0)
    r = oracle.solve(field, y0, t0, t1, te, dict(rtol=1e-11, atol=1e-11))
    ex = np.arcsinh(np.sinh(w_ * y0) * np.exp(w_ * v_ * te)) / w_
    assert np.abs(r["y_eval"][..., 0] - ex).max() < 1e-9


def test_mlp_field_known_values():
    a = math.atanh(0.5)
    # column 0 is y, column 1 is t; bias of the hidden layer, linear output
    f_y = {"kind": "mlp", "W": [np.array([[a, 0.0]]), np.array([[3.0]])],
           "b": [np.zeros(1), np.array([0.25])]}
    assert abs(oracle.field_eval(f_y, 0, 7.0, [1.0])[0] - (1.5 + 0.25)) < 1e-15
    f_t = {"kind": "mlp", "W": [np.array([[0.0, a]]), np.array([[3.0]])],
           "b": [np.zeros(1), np.zeros(1)]}
    assert abs(oracle.field_eval(f_t, 0, 1.0, [5.0])[0] - 1.5) < 1e-15
    f_b = {"kind": "mlp", "W": [np.array([[0.0, 0.0]]), np.array([[-2.0]])],
           "b": [np.array([a]), np.zeros(1)]}
    assert abs(oracle.field_eval(f_b, 0, 0.0, [0.0])[0] + 1.0) < 1e-15
    # two hidden layers: tanh(tanh(.)) composition
    f_2 = {"kind": "mlp", "W": [np.array([[0.3, 0.0]]), np.array([[0.5]]), np.array([[1.0]])],
           "b": [np.zeros(1), np.zeros(1), np.zeros(1)]}
    assert abs(oracle.field_eval(f_2, 0, 0.0, [1.0])[0] - math.tanh(0.5 * math.tanh(0.3))) < 1e-15


def test_mlp_odd_symmetry_bitwise():
    """With zero biases and no t input the MLP is odd, so the solution from
    -y0 is exactly the negated solution from y0."""
    w = workloads.make(4, B=4)
    W = [x.copy() for x in w["field"]["W"]]
    W[0][:, -1] = 0.0
    field = {"kind": "mlp", "W": W, "b": w["field"]["b"]}
    y0 = w["y0"]
    y0s = np.concatenate([y0, -y0])
    t0 = np.zeros(8)
    t1 = np.ones(8)
    te = np.concatenate([w["t_eval"], w["t_eval"]])
    r = oracle.solve(field, y0s, t0, t1, te, dict(rtol=1e-6, atol=1e-6))
    assert np.array_equal(r["y_eval"][:4], -r["y_eval"][4:])
    assert np.array_equal(r["n_acc"][:4], r["n_acc"][4:])


# ---------------------------------------------------------------- convergence
def test_observed_order_five_fixed_step_vdp():
    B = 3
    mu = np.array([0.5, 1.0, 2.0])
    y0 = np.array([[2.0, 0.0], [1.0, -1.0], [-0.5, 1.5]])
    T = 2.0
    ref = rk4_reference(vdp_rhs(mu), y0, T, 20000)
    errs = []
    for N in (20, 40, 80):
        mt, mh, mn = uniform_mesh(B, np.full(B, T), N)
        r = oracle.replay({"kind": "vdp", "mu": mu}, y0, np.zeros(B), np.full(B, T), mt, mh, mn)
        errs.append(np.abs(r["y_final"] - ref).max(axis=1))
    errs = np.array(errs)
    # order >= 5: halving h divides the error by at least ~2^5 (dopri5's
    # small principal error constant makes the pre-asymptotic ratio larger)
    for k in range(2):
        ratio = errs[k] / errs[k + 1]
        assert (ratio > 26).all(), ratio


def test_dense_output_order_fixed_step():
    """Mid-step dense output converges with order >= 4 (HNW Sec. II.6)."""
    B = 2
    mu = np.array([1.0, 1.5])
    y0 = np.array([[2.0, 0.0], [0.5, 0.5]])
    T = 2.0
    errs = []
    for N in (16, 32, 64):
        mt, mh, mn = uniform_mesh(B, np.full(B, T), N)
        # evaluation points in the middle of steps that are common to all N
        te = np.array([[0.3 * T / 16 + j * T / 16 for j in range(16)]] * B)
        r = oracle.replay({"kind": "vdp", "mu": mu}, y0, np.zeros(B), np.full(B, T), mt, mh, mn,
                          te)
        ref = np.stack([rk4_reference(vdp_rhs(mu), y0, tj, 8000) for tj in te[0]], axis=1)
        errs.append(np.abs(r["y_eval"] - ref).max())
    assert errs[0] / errs[1] > 14 and errs[1] / errs[2] > 14, errs


def test_adaptive_vdp_vs_brute_force():
    w = workloads.make(1, B=4)
    T = 3.0
    t1 = np.full(4, T)
    r = oracle.solve(w["field"], w["y0"], w["t0"], t1, None, dict(rtol=1e-12, atol=1e-12))
    ref = rk4_reference(vdp_rhs(w["field"]["mu"]), w["y0"], T, 30000)
    assert np.abs(r["y_final"] - ref).max() < 1e-9


def test_tolerance_proportionality_vdp():
    """Global error falls roughly in proportion to the tolerance (a controller
    that does not track err <= 1 fails this)."""
    w = workloads.make(1, B=16)
    ref = oracle.solve(w["field"], w["y0"], w["t0"], w["t1"], w["t_eval"],
                       dict(rtol=1e-13, atol=1e-13))
    e = []
    for tol in (1e-5, 1e-7, 1e-9):
        r = oracle.solve(w["field"], w["y0"], w["t0"], w["t1"], w["t_eval"],
                         dict(rtol=tol, atol=tol))
        e.append(np.abs(r["y_eval"] - ref["y_eval"]).max())
    assert 10 < e[0] / e[1] < 1000 and 10 < e[1] / e[2] < 1000, e


# ---------------------------------------------------------------- controller
def test_controller_power_function_accuracy():
    """The controller's x^y (a fixed exp/log procedure, identical on every
    IEEE machine) agrees with the platform pow within the error bound of
    exp(y ln x): a few ulps plus the absolute error of y ln x."""
    import ctypes as C
    from oracle import oracle as O
    lib = C.CDLL(O.build())
    lib.orc_pow.restype = C.c_double
    lib.orc_pow.argtypes = [C.c_double, C.c_double]
    xs = np.concatenate([10.0 ** np.linspace(-300, 300, 2001), np.linspace(0.01, 3.0, 3001),
                         [5e-324, 2.2e-308, 1.0 - 2 ** -53, 1.0 + 2 ** -52]])
    worst = 0.0
    for y in (-0.2, 0.2, -0.14, 0.08, 0.5, -1.0):
        for x in xs:
            try:
                ref = math.pow(x, y)
            except OverflowError:
                continue
            if ref == 0.0 or math.isinf(ref) or ref > 1e300 or ref < 1e-300:
                continue
            v = lib.orc_pow(x, y)
            bound = 2.3e-16 * (8.0 + 2.0 * abs(y * math.log(x)))
            worst = max(worst, abs(v - ref) / ref / bound)
    assert worst < 1.0, worst
    assert lib.orc_pow(1.0, -0.2) == 1.0 and lib.orc_pow(0.0, 0.2) == 0.0
    assert math.isinf(lib.orc_pow(0.0, -0.2)) and math.isnan(lib.orc_pow(-1.0, 0.2))
    assert math.isnan(lib.orc_pow(float("nan"), 0.2))


@pytest.mark.parametrize("beta1,beta2,beta3", [(0.2, 0.0, 0.0), (0.14, 0.08, 0.0),
                                               (0.16, 0.1, 0.02)])
def test_controller_steady_state(beta1, beta2, beta3):
    """For a smooth problem in the asymptotic regime (err ~ C h^p) the
    controller factor safety*err^-b1*err_prev^b2*err_prev2^-b3 drives
    accepted errors to the fixed point err* = safety^(1/(b1-b2+b3)),
    whatever p is (App. C: the PID family over the last three error
    estimates; App. A: I controller, b2 = b3 = 0)."""
    field = {"kind": "linear", "A": np.array([[[1.0]]])}
    r = oracle.solve(field, np.ones((1, 1)), np.zeros(1), np.array([12.0]), None,
                     dict(rtol=1e-10, atol=0.0, beta1=beta1, beta2=beta2, beta3=beta3),
                     trace_cap=10000)
    L = r["trace_len"][0]
    acc = r["trace_accepted"][0, :L].astype(bool)
    errs = r["trace_err"][0, :L][acc][:-1]  # drop the clipped last step
    target = 0.9 ** (1.0 / (beta1 - beta2 + beta3))
    tail = errs[len(errs) // 2:]
    assert np.abs(tail / target - 1).max() < 0.03, (tail.min(), tail.max(), target)


def test_pid_step_sequence_from_its_own_errors():
    """Every step after an accepted one is h * clamp(0.9 err_n^-b1
    err_{n-1}^b2 err_{n-2}^-b3) with the errors of the last three accepted
    steps (floored at 1e-4, 1 before the first), recomputed here with the
    platform pow from the trace: catches a wrong index or sign in the
    controller's history."""
    w = workloads.make(1, B=4)
    b1, b2, b3 = 0.16, 0.1, 0.02
    r = oracle.solve(w["field"], w["y0"], w["t0"], w["t1"], None,
                     dict(rtol=1e-7, atol=1e-7, beta1=b1, beta2=b2, beta3=b3), trace_cap=5000)
    checked = 0
    for i in range(4):
        L = r["trace_len"][i]
        h, e, a = r["trace_h"][i, :L], r["trace_err"][i, :L], r["trace_accepted"][i, :L]
        hist = [1.0, 1.0]  # err_{n-2}, err_{n-1}
        prev_rej = False
        for n in range(L - 2):  # the last attempt's successor is clipped or absent
            if a[n]:
                fac = 0.9 * math.pow(e[n], -b1) * math.pow(hist[1], b2) * math.pow(hist[0], -b3)
                fac = min(max(fac, 0.2), 10.0)
                if prev_rej:
                    fac = min(fac, 1.0)
                hist = [hist[1], max(e[n], 1e-4)]
                clipped = r["trace_t"][i, n + 1] + h[n + 1] == w["t1"][i]
                if not clipped:
                    assert abs(h[n + 1] / (h[n] * fac) - 1) < 1e-13, (i, n)
                    checked += 1
            prev_rej = not a[n]
    assert checked > 400


def _vdp_cycle(mu):
    """A rough limit-cycle period of Van der Pol's oscillator (relaxation
    form for large mu, 2 pi for small)."""
    if mu <= 1.0:
        return 2 * math.pi
    return (3 - 2 * math.log(2)) * mu + 2 * math.pi / (1 + mu) + 4.676 * mu ** (-1 / 3)


PID_BETAS = ((0.3 + 0.3 + 0.1) / 5, (0.3 + 2 * 0.1) / 5, 0.1 / 5)  # gains (p, i, d) / order 5


@pytest.mark.parametrize("mu,pid_better", [(5.0, False), (10.0, False), (25.0, True),
                                           (50.0, True)])
def test_pid_trade_off_over_one_vdp_cycle(mu, pid_better):
    """App. C: over one cycle of Van der Pol, PID control costs steps while
    the step size varies little (mu < 15) and saves steps once it varies by
    orders of magnitude (mu > 25).  Gains (p, i, d) = (0.3, 0.3, 0.1) are a
    choice of this test (the paper's come from external documentation)."""
    f = dict(kind="vdp", mu=np.array([mu]))
    T = _vdp_cycle(mu)

    def attempts(b1, b2, b3):
        r = oracle.solve(f, np.array([[2.0, 0.0]]), [0.0], [T], None,
                         dict(rtol=1e-6, atol=1e-6, beta1=b1, beta2=b2, beta3=b3))
        assert r["status"][0] == 0
        return int(r["n_acc"][0] + r["n_rej"][0])
    i_ctl, pid = attempts(0.2, 0.0, 0.0), attempts(*PID_BETAS)
    if pid_better:
        assert pid < 0.97 * i_ctl, (pid, i_ctl)
    else:
        assert pid > i_ctl, (pid, i_ctl)


def test_controller_clamps_and_no_growth_after_reject():
    w = workloads.make(1, B=8)
    # tiny first step: err ~ 0 -> factor clamped to fac_max exactly
    r = oracle.solve(w["field"], w["y0"], w["t0"], w["t1"], None,
                     dict(rtol=1e-7, atol=1e-7, h0=1e-9), trace_cap=5000)
    assert np.allclose(r["trace_h"][:, 1], 1e-8, rtol=0, atol=0)
    # huge first step: rejected; every step right after a rejection does not grow
    r = oracle.solve(w["field"], w["y0"], w["t0"], w["t1"], None,
                     dict(rtol=1e-7, atol=1e-7, h0=2.0), trace_cap=5000)
    seen = 0
    for i in range(8):
        L = r["trace_len"][i]
        acc = r["trace_accepted"][i, :L]
        h = r["trace_h"][i, :L]
        assert acc[0] == 0
        for n in range(1, L - 1):
            if acc[n - 1] == 0:
                assert h[n] <= h[n - 1] * (1 + 1e-15)  # reject shrinks
                if acc[n] == 1 and n + 1 < L:
                    assert h[n + 1] <= h[n] * (1 + 1e-15) or n + 1 == L - 1
                    seen += 1
    assert seen > 0


def test_first_step_error_estimate_matches_exact_polynomial():
    """y' = diag(l1, l2) y: the first attempt's error estimate is
    e_j = E(h l_j) y0_j with E the embedded error polynomial, exact from the
    tableau; the norm is the per-instance weighted RMS."""
    z, Rz, Ez = rk.linear_step_polys()
    lams = (-3.0, 0.7)
    A = np.array([[[lams[0], 0.0], [0.0, lams[1]]]])
    y0 = np.array([[1.3, -0.4]])
    h = 0.05
    rtol, atol = 1e-6, 1e-9
    r = oracle.solve({"kind": "linear", "A": A}, y0, np.zeros(1), np.array([1.0]), None,
                     dict(rtol=rtol, atol=atol, h0=h), trace_cap=4)
    q = []
    for j in range(2):
        zz = sp.Float(h * lams[j], 30)
        e = float(Ez.subs(z, zz)) * y0[0, j]
        y1 = float(Rz.subs(z, zz)) * y0[0, j]
        sc = atol + rtol * max(abs(y0[0, j]), abs(y1))
        q.append(e / sc)
    expect = math.sqrt((q[0] ** 2 + q[1] ** 2) / 2)
    assert abs(r["trace_err"][0, 0] / expect - 1) < 1e-9
    # and with D = 1 the norm reduces to |e|/sc
    r1 = oracle.solve({"kind": "linear", "A": A[:, :1, :1]}, y0[:, :1], np.zeros(1),
                      np.array([1.0]), None, dict(rtol=rtol, atol=atol, h0=h), trace_cap=4)
    assert abs(r1["trace_err"][0, 0] / abs(q[0]) - 1) < 1e-9


# ---------------------------------------------------------------- statuses
def test_statuses_and_counters():
    w = workloads.make(1, B=8)
    f, y0, t0, t1, te = w["field"], w["y0"].copy(), w["t0"].copy(), w["t1"].copy(), \
        w["t_eval"].copy()
    te[1, 3], te[1, 4] = te[1, 4], te[1, 3]  # decreasing
    te[2, 5] = t1[2] + 1.0                   # outside [t0, t1]
    t1[3] = -1.0                             # t1 < t0
    y0[4, 0] = np.nan                        # non-finite state
    t1[5] = t0[5]                            # empty range
    te[5] = t0[5]
    r = oracle.solve(f, y0, t0, t1, te, dict(rtol=1e-7, atol=1e-7))
    st = r["status"]
    assert list(st[[1, 2, 3]]) == [4, 4, 4]
    assert st[4] == 3
    assert st[5] == 0 and r["n_acc"][5] == 0 and r["n_feval"][5] == 0
    assert np.array_equal(r["y_eval"][5], np.repeat(y0[5:6], te.shape[1], 0))
    for i in (0, 6, 7):
        assert st[i] == 0
        assert r["n_feval"][i] == 2 + 6 * (r["n_acc"][i] + r["n_rej"][i])
    assert np.isnan(r["y_eval"][1]).all() and np.isnan(r["y_final"][1]).all()
    # max_steps
    r = oracle.solve(f, w["y0"], w["t0"], w["t1"], None, dict(rtol=1e-7, atol=1e-7,
                                                               max_steps=5))
    assert (r["status"] == 1).all() and ((r["n_acc"] + r["n_rej"]) == 5).all()
    # given first step: one evaluation for k1, none for the heuristic
    r = oracle.solve(f, w["y0"], w["t0"], w["t1"], None, dict(rtol=1e-7, atol=1e-7, h0=1e-3))
    assert (r["n_feval"] == 1 + 6 * (r["n_acc"] + r["n_rej"])).all()


def test_instances_are_independent_bitwise():
    """Sec. 3 / Sec. 4.1: an instance's result does not depend on its batch."""
    w = workloads.make(1, B=12)
    full = oracle.solve(w["field"], w["y0"], w["t0"], w["t1"], w["t_eval"],
                        dict(rtol=1e-7, atol=1e-7))
    perm = np.random.default_rng(3).permutation(12)
    fp = {"kind": "vdp", "mu": w["field"]["mu"][perm]}
    sh = oracle.solve(fp, w["y0"][perm], w["t0"][perm], w["t1"][perm], w["t_eval"][perm],
                      dict(rtol=1e-7, atol=1e-7), nthreads=3)
    for k in ("y_eval", "y_final", "n_acc", "n_rej", "status"):
        assert np.array_equal(full[k][perm], sh[k])
    one = oracle.solve({"kind": "vdp", "mu": w["field"]["mu"][5:6]}, w["y0"][5:6],
                       w["t0"][5:6], w["t1"][5:6], w["t_eval"][5:6], dict(rtol=1e-7, atol=1e-7))
    assert np.array_equal(one["y_eval"][0], full["y_eval"][5])


# ---------------------------------------------------------------- adjoint
def _loss_replay(field, w, mt, mh, mn, gy_eval):
    r = oracle.replay(field, w["y0"], w["t0"], w["t1"], mt, mh, mn, w["t_eval"])
    return float((gy_eval * r["y_eval"]).sum())


@pytest.mark.parametrize("cfg", [1, 2])
def test_adjoint_vs_central_fd_frozen_mesh(cfg):
    w = workloads.make(cfg, B=3)
    tol = 1e-6
    r = oracle.solve(w["field"], w["y0"], w["t0"], w["t1"], w["t_eval"],
                     dict(rtol=tol, atol=tol), trace_cap=20000)
    mt, mh, mn = mesh_from_trace(r)
    rng = np.random.default_rng(11)
    gye = rng.standard_normal(r["y_eval"].shape)
    adj = oracle.adjoint(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, w["t_eval"], gye)
    D = w["y0"].shape[1]
    num = np.zeros_like(w["y0"])
    for i in range(3):
        for j in range(D):
            eps = 1e-6 * max(1.0, abs(w["y0"][i, j]))
            wp = dict(w, y0=w["y0"].copy())
            wp["y0"][i, j] += eps
            lp = _loss_replay(w["field"], wp, mt, mh, mn, gye)
            wp["y0"][i, j] -= 2 * eps
            lm = _loss_replay(w["field"], wp, mt, mh, mn, gye)
            num[i, j] = (lp - lm) / (2 * eps)
    rel = np.linalg.norm(num - adj["gy0"]) / np.linalg.norm(adj["gy0"])
    assert rel < 1e-6, rel
    # parameter cotangent
    if cfg == 1:
        mu = w["field"]["mu"]
        for i in range(3):
            eps = 1e-6 * max(1, abs(mu[i]))
            fp = {"kind": "vdp", "mu": mu.copy()}
            fp["mu"][i] += eps
            lp = _loss_replay(fp, w, mt, mh, mn, gye)
            fp["mu"][i] -= 2 * eps
            lm = _loss_replay(fp, w, mt, mh, mn, gye)
            g = (lp - lm) / (2 * eps)
            assert abs(g - adj["gmu"][i]) <= 1e-6 * max(1.0, abs(g))
    else:
        A = w["field"]["A"]
        for (i, a, b) in [(0, 0, 0), (1, 3, 7), (2, 15, 2)]:
            eps = 1e-6
            fp = {"kind": "linear", "A": A.copy()}
            fp["A"][i, a, b] += eps
            lp = _loss_replay(fp, w, mt, mh, mn, gye)
            fp["A"][i, a, b] -= 2 * eps
            lm = _loss_replay(fp, w, mt, mh, mn, gye)
            g = (lp - lm) / (2 * eps)
            assert abs(g - adj["gA"][i, a, b]) <= 1e-6 * max(1.0, abs(g))


def test_adjoint_mlp_vs_fd():
    w = workloads.make(4, B=2)
    tol = 1e-5
    r = oracle.solve(w["field"], w["y0"], w["t0"], w["t1"], w["t_eval"],
                     dict(rtol=tol, atol=tol), trace_cap=5000)
    mt, mh, mn = mesh_from_trace(r)
    gye = 2.0 * r["y_eval"]  # L = sum y(t_eval)^2
    adj = oracle.adjoint(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, w["t_eval"], gye)

    def loss(field, y0):
        rr = oracle.replay(field, y0, w["t0"], w["t1"], mt, mh, mn, w["t_eval"])
        return float((rr["y_eval"] ** 2).sum())

    for (i, j) in [(0, 0), (1, 17), (1, 31)]:
        eps = 1e-6
        y = w["y0"].copy()
        y[i, j] += eps
        lp = loss(w["field"], y)
        y[i, j] -= 2 * eps
        lm = loss(w["field"], y)
        g = (lp - lm) / (2 * eps)
        assert abs(g - adj["gy0"][i, j]) <= 1e-6 * max(1.0, abs(g))
    for (l, a, b) in [(0, 5, 32), (1, 100, 7), (2, 31, 127), (0, 0, 0)]:
        eps = 1e-6
        Wp = [x.copy() for x in w["field"]["W"]]
        Wp[l][a, b] += eps
        lp = loss({"kind": "mlp", "W": Wp, "b": w["field"]["b"]}, w["y0"])
        Wp[l][a, b] -= 2 * eps
        lm = loss({"kind": "mlp", "W": Wp, "b": w["field"]["b"]}, w["y0"])
        g = (lp - lm) / (2 * eps)
        assert abs(g - adj["gW"][l][a, b]) <= 1e-6 * max(1.0, abs(g)), (l, a, b)
    for (l, a) in [(0, 3), (2, 9)]:
        eps = 1e-6
        bp = [x.copy() for x in w["field"]["b"]]
        bp[l][a] += eps
        lp = loss({"kind": "mlp", "W": w["field"]["W"], "b": bp}, w["y0"])
        bp[l][a] -= 2 * eps
        lm = loss({"kind": "mlp", "W": w["field"]["W"], "b": bp}, w["y0"])
        g = (lp - lm) / (2 * eps)
        assert abs(g - adj["gb"][l][a]) <= 1e-6 * max(1.0, abs(g))


def test_adjoint_linear_closed_form_jacobian():
    """For y' = A y, d y(T) / d y0 = expm(A T) (up to discretisation error)."""
    w = workloads.make(2, B=2)
    r = oracle.solve(w["field"], w["y0"], w["t0"], w["t1"], None,
                     dict(rtol=1e-11, atol=1e-11), trace_cap=50000)
    mt, mh, mn = mesh_from_trace(r)
    D = 16
    for i in range(2):
        M = sla.expm(w["field"]["A"][i] * w["t1"][i])
        for col in (0, 9):
            gyf = np.zeros((2, D))
            gyf[i, col] = 1.0
            adj = oracle.adjoint(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, None, None,
                                 gyf)
            # row `col` of M: d y_col(T) / d y0
            assert np.abs(adj["gy0"][i] - M[col]).max() < 1e-8


def test_backward_in_time_is_forward_with_the_negated_field():
    """Integration from t0 down to t1 < t0 (the method with negative steps)
    equals, bit for bit, forward integration of the negated field in s = -t:
    y'(t) = A y backward is z'(s) = -A z forward (IEEE rounding is symmetric
    under negation, so every step, point and decision coincides)."""
    rng = np.random.default_rng(7)
    B, D = 6, 4
    A = rng.standard_normal((B, D, D)) * 0.8
    y0 = rng.standard_normal((B, D))
    t0, t1 = np.full(B, 2.0), rng.uniform(-3.0, 0.5, B)
    te = np.stack([np.linspace(2.0, t, 9) for t in t1])
    back = oracle.solve({"kind": "linear", "A": A}, y0, t0, t1, te, dict(rtol=1e-7, atol=1e-7),
                        trace_cap=2000)
    fwd = oracle.solve({"kind": "linear", "A": -A}, y0, -t0, -t1, -te,
                       dict(rtol=1e-7, atol=1e-7), trace_cap=2000)
    assert (back["status"] == 0).all()
    for k in ("y_eval", "y_final", "n_acc", "n_rej", "n_feval", "trace_len", "trace_accepted",
              "trace_err"):
        assert np.array_equal(back[k], fwd[k]), k
    assert np.array_equal(back["trace_t"], -fwd["trace_t"])
    assert np.array_equal(back["trace_h"], -fwd["trace_h"])
    L = back["trace_len"][0]
    assert (back["trace_h"][0, :L] < 0).all()


def test_backward_in_time_closed_form_and_round_trip():
    """Linear: y(t) = Q exp(-Lambda t) Q^T y0 for t < t0 = 0 within the
    tolerance's band; Van der Pol: forward to t1 and back to t0 returns y0
    to the accuracy of the two solves."""
    w = workloads.make(2, B=16)
    Q, lam = w["field"]["Q"], w["field"]["lam"]
    t1 = -np.full(16, 0.4)
    te = np.stack([np.linspace(0.0, -0.4, 5)] * 16)
    r = oracle.solve(w["field"], w["y0"], np.zeros(16), t1, te, dict(rtol=1e-10, atol=1e-10))
    c = np.einsum("bji,bj->bi", Q, w["y0"])
    exact = np.einsum("bij,bkj->bki", Q, np.exp(-lam[:, None, :] * te[:, :, None]) * c[:, None, :])
    assert (r["status"] == 0).all()
    assert np.abs(r["y_eval"] - exact).max() <= 1e-7 * max(1.0, np.abs(exact).max())
    # (Van der Pol's limit cycle repels backward in time: a short horizon)
    v = workloads.make(1, B=8)
    v1 = np.full(8, 1.5)
    f = oracle.solve(v["field"], v["y0"], v["t0"], v1, None, dict(rtol=1e-11, atol=1e-11))
    b = oracle.solve(v["field"], f["y_final"], v1, v["t0"], None, dict(rtol=1e-11, atol=1e-11))
    assert (b["status"] == 0).all() and (b["n_acc"] > 10).all()
    assert np.abs(b["y_final"] - v["y0"]).max() < 1e-6


def test_dense_output_derivative_pins():
    """dy/dt at the evaluation points (the derivative of the dense-output
    interpolant): central differences of the interpolant itself on the same
    mesh (a replay with shifted t_eval), f(t1, y(t1)) at the end point (the
    interpolant is C1 with the FSAL stage), f(t0, y0) at t0, and the linear
    closed form's A y(t)."""
    w = workloads.make(1, B=6)
    B = 6
    K = w["t_eval"].shape[1]
    r = oracle.solve(w["field"], w["y0"], w["t0"], w["t1"], w["t_eval"],
                     dict(rtol=1e-7, atol=1e-7), trace_cap=4000, want_yp=True)
    yp = r["yp_eval"]
    mt, mh, mn = mesh_from_trace(r)
    d = 1e-5
    inner = w["t_eval"].copy()
    inner[:, 0], inner[:, -1] = inner[:, 1], inner[:, -2]  # keep t0 and t1 out
    lo = oracle.replay(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, inner - d)
    hi = oracle.replay(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, inner + d)
    fd = (hi["y_eval"] - lo["y_eval"]) / (2 * d)
    for i in range(B):
        # a step end within +-d of a point makes the difference one-sided: skip it
        ends = np.concatenate([mt[i, :mn[i]], [w["t1"][i]]])
        for q in range(1, K - 1):
            if np.min(np.abs(ends - inner[i, q])) > 2 * d:
                assert np.allclose(yp[i, q], fd[i, q], rtol=1e-6, atol=1e-6), (i, q)
        f1 = oracle.field_eval(w["field"], i, w["t1"][i], r["y_final"][i], B)
        assert np.allclose(yp[i, -1], f1, rtol=1e-12, atol=1e-12)
        f0 = oracle.field_eval(w["field"], i, w["t0"][i], w["y0"][i], B)
        assert np.array_equal(yp[i, 0], f0)
    L = workloads.make(2, B=8)
    Q, lam = L["field"]["Q"], L["field"]["lam"]
    rl = oracle.solve(L["field"], L["y0"], L["t0"], L["t1"], L["t_eval"],
                      dict(rtol=1e-11, atol=1e-11), want_yp=True)
    c = np.einsum("bji,bj->bi", Q, L["y0"])
    ex = np.einsum("bij,bkj->bki", Q, np.exp(-lam[:, None, :] * L["t_eval"][:, :, None])
                   * c[:, None, :])
    dex = np.einsum("bij,bkj->bki", L["field"]["A"], ex)
    assert np.abs(rl["yp_eval"] - dex).max() <= 1e-6 * max(1.0, np.abs(dex).max())


def test_replay_dense_derivative_equals_the_solve_on_its_own_mesh():
    """The replay's dy/dt at the points (o9 with the interpolant's derivative)
    on the mesh a solve recorded is the solve's own dy/dt, bit for bit: the
    same steps from the same states (Van der Pol with instances in both
    directions, and the MLP field, non-autonomous, with points at t0)."""
    v = workloads.make(1, B=6)
    t0, t1, te = v["t0"].copy(), v["t1"].copy(), v["t_eval"].copy()
    t0[::2], t1[::2] = v["t1"][::2], v["t0"][::2]
    te[::2] = te[::2, ::-1]
    m = workloads.make(4, B=5)
    for w in (dict(v, t0=t0, t1=t1, t_eval=te), m):
        r = oracle.solve(w["field"], w["y0"], w["t0"], w["t1"], w["t_eval"],
                         dict(rtol=w["rtol"], atol=w["atol"]), trace_cap=4000, want_yp=True)
        assert (r["status"] == 0).all()
        mt, mh, mn = mesh_from_trace(r)
        p = oracle.replay(w["field"], w["y0"], w["t0"], w["t1"], mt, mh, mn, w["t_eval"],
                          want_yp=True)
        assert np.array_equal(p["y_eval"], r["y_eval"])
        assert np.array_equal(p["yp_eval"], r["yp_eval"])
        assert (w["t_eval"][:, 0] == w["t0"]).any()


# ---------------------------------------------------------------- starting step
def _hnw_starting_step(lams, y0, rtol, atol, span):
    """The starting-step heuristic of Hairer-Norsett-Wanner Sec. II.4 for
    y' = diag(lams) y, every quantity written out from its definition:
    d0 = ||y0||, d1 = ||f0||, h0 = 0.01 d0 / d1 (1e-6 when either norm is
    below 1e-5), d2 = ||f(t0 + h0, y0 + h0 f0) - f0|| / h0 which for this
    field is ||diag(lams)^2 y0|| exactly, h1 = (0.01 / max(d1, d2))^(1/5)
    (max(1e-6, 1e-3 h0) when max(d1, d2) <= 1e-15), and the first step
    min(100 h0, h1, |t1 - t0|).  The norm is the RMS weighted by
    atol + rtol |y0|.  Returns the step and which of the three terms set it."""
    lams = np.asarray(lams, dtype=np.float64)
    y0 = np.asarray(y0, dtype=np.float64)
    sc = atol + rtol * np.abs(y0)

    def norm(v):
        return math.sqrt(float(np.mean((v / sc) ** 2)))

    d0 = norm(y0)
    d1 = norm(lams * y0)
    h0 = 1e-6 if (d0 < 1e-5 or d1 < 1e-5) else 0.01 * d0 / d1
    d2 = norm(lams * lams * y0)
    m = max(d1, d2)
    h1 = max(1e-6, h0 * 1e-3) if m <= 1e-15 else (0.01 / m) ** 0.2
    terms = {"100*h0": 100.0 * h0, "h1": h1, "span": span}
    which = min(terms, key=terms.get)
    return terms[which], which, h0


@pytest.mark.parametrize("direction", [1.0, -1.0])
def test_starting_step_matches_hnw_closed_form(direction):
    """The oracle's first attempted step on diagonal linear systems equals
    the HNW Sec. II.4 heuristic worked out in closed form, in both
    directions of integration (a backward instance attempts -h first).  The
    cases are chosen so that each term of min(100 h0, h1, t1 - t0) and each
    fallback (h0 = 1e-6 for a tiny norm, h1 = max(1e-6, 1e-3 h0) for a
    vanishing derivative) decides at least once: a wrong exponent, a missing
    cap, a dropped fallback or a wrong sign fails one of them."""
    cases = [  # lams, y0, rtol, atol, |t1 - t0|
        ((-2.0,), (1.0,), 1e-6, 1e-6, 10.0),             # h1 decides (d2 > d1)
        ((-0.3,), (1.5,), 1e-7, 1e-9, 10.0),             # h1 decides (d1 > d2)
        ((-1000.0,), (1.0,), 1e-2, 1e-2, 10.0),          # 100 h0 decides
        ((-0.5,), (2.0,), 1e-3, 1e-3, 1e-3),             # the interval decides
        ((-1.0,), (1e-12,), 1e-6, 1e-6, 10.0),           # d0 < 1e-5: h0 = 1e-6
        ((0.0,), (0.0,), 1e-6, 1e-6, 10.0),              # f = 0: both fallbacks
        ((-3.0, 0.7), (1.3, -0.4), 1e-6, 1e-9, 10.0),    # two components, mixed signs
        ((-40.0, -0.05), (0.2, 5.0), 1e-5, 1e-5, 10.0),  # two components, stiff and slow
    ]
    seen = set()
    for lams, y0, rtol, atol, span in cases:
        D = len(lams)
        A = np.diag(lams).reshape(1, D, D)
        t0 = 2.0
        t1 = t0 + direction * span
        expect, which, h0 = _hnw_starting_step(lams, y0, rtol, atol, span)
        seen.add(which)
        if which != "span":  # the decision is not a tie
            others = sorted(v for v in (100.0 * h0, span) if v != expect)
            assert not others or others[0] > expect * (1 + 1e-6)
        r = oracle.solve({"kind": "linear", "A": A}, np.array([y0]), np.array([t0]),
                         np.array([t1]), None, dict(rtol=rtol, atol=atol), trace_cap=2)
        got = r["trace_h"][0, 0]
        assert math.copysign(1.0, got) == direction, (lams, y0, got)
        assert abs(abs(got) / expect - 1.0) < 1e-12, (lams, y0, which, got, expect)
        assert r["trace_t"][0, 0] == t0
    assert seen == {"100*h0", "h1", "span"}
    # the fallbacks: h0 = 1e-6 from the tiny norm, then 100 h0 = 1e-4 decides
    assert _hnw_starting_step((-1.0,), (1e-12,), 1e-6, 1e-6, 10.0)[0] == pytest.approx(1e-4)
    # f = 0: h0 = 1e-6 and h1 = max(1e-6, 1e-9) = 1e-6
    assert _hnw_starting_step((0.0,), (0.0,), 1e-6, 1e-6, 10.0)[0] == 1e-6


@pytest.mark.parametrize("direction", [1.0, -1.0])
def test_starting_step_van_der_pol_exact(direction):
    """The same heuristic on the nonlinear Van der Pol field (Eq. 1), with
    the probe evaluation f(t0 + h0, y0 + h0 f0) taken in the direction of
    integration: d2 is computed in exact rational arithmetic from the
    definition (for a linear field the direction of the probe cannot show,
    here it moves d2 by ~1e-3).  The square roots and the 1/5 power are
    taken at the end in FP64."""
    from fractions import Fraction as Fr

    mu, y0 = Fr(8), (Fr(7, 4), Fr(-1, 2))
    rtol, atol = 1e-6, 1e-7
    sc = [Fr(atol) + Fr(rtol) * abs(v) for v in y0]

    def f(y):
        return (y[1], mu * (1 - y[0] * y[0]) * y[1] - y[0])

    def norm2(v):  # mean of squares, exact
        return sum((x / s) ** 2 for x, s in zip(v, sc)) / len(v)

    f0 = f(y0)
    d0 = math.sqrt(norm2(y0))
    d1 = math.sqrt(norm2(f0))
    h0 = 0.01 * (d0 / d1)
    assert d0 >= 1e-5 and d1 >= 1e-5
    hs = Fr(direction * h0)  # the FP64 probe step, exactly
    yp = tuple(a + hs * b for a, b in zip(y0, f0))
    diff = tuple(a - b for a, b in zip(f(yp), f0))
    d2 = math.sqrt(norm2(diff)) / h0
    h1 = (0.01 / max(d1, d2)) ** 0.2
    expect = min(100.0 * h0, h1, 20.0)
    assert expect == h1 and d2 > d1
    # the probe in the other direction would give a visibly different step
    yq = tuple(a - hs * b for a, b in zip(y0, f0))
    d2q = math.sqrt(norm2(tuple(a - b for a, b in zip(f(yq), f0)))) / h0
    assert abs((0.01 / max(d1, d2q)) ** 0.2 / h1 - 1.0) > 1e-5
    t0 = 1.0
    r = oracle.solve({"kind": "vdp", "mu": np.array([float(mu)])},
                     np.array([[float(y0[0]), float(y0[1])]]), np.array([t0]),
                     np.array([t0 + direction * 20.0]), None, dict(rtol=rtol, atol=atol),
                     trace_cap=2)
    got = r["trace_h"][0, 0]
    assert math.copysign(1.0, got) == direction
    assert abs(abs(got) / expect - 1.0) < 1e-11, (got, expect)


# ---------------------------------------------------------------- t0, t1 gradients
def _interior_t_eval(mt, mn, t0, t1, K, rng):
    """K evaluation points per instance strictly inside (t0, t1), none within
    1e-3 of the interval's length of a mesh point (so a small move of the
    mesh leaves every point in its step)."""
    B = len(t0)
    te = np.zeros((B, K))
    for i in range(B):
        pts = np.concatenate([mt[i, :mn[i]], [t1[i]]])
        span = abs(t1[i] - t0[i])
        got = []
        while len(got) < K:
            x = t0[i] + (t1[i] - t0[i]) * rng.uniform(0.02, 0.98)
            if np.min(np.abs(pts - x)) > 1e-3 * span:
                got.append(x)
        got = np.array(sorted(got, key=lambda v: (v - t0[i]) * np.sign(t1[i] - t0[i])))
        te[i] = got
    return te


def _loss_replay_t(field, y0, t0, t1, mt, mh, mn, te, gye, gyf):
    r = oracle.replay(field, y0, t0, t1, mt, mh, mn, te)
    return (gye * r["y_eval"]).sum(axis=(1, 2)) + (gyf * r["y_final"]).sum(axis=1)


@pytest.mark.parametrize("case", ["vdp", "vdp_backward", "linear", "mlp"])
def test_t_bounds_gradient_matches_frozen_mesh_differences(case):
    """dL/dt0 and dL/dt1 of the frozen map (every step size but the last and
    every point's step held; t0 moves every mesh point before t1, the last
    step absorbs the change) against central differences of the fixed-mesh
    replay moved that way; for the autonomous fields also the time-translation
    identity dL/dt0 + dL/dt1 = -sum_tau <ybar_tau, dy/dt(tau)>.  The MLP field
    takes t as an input, so its stage times enter too."""
    rng = np.random.default_rng(7)
    cfg = {"vdp": 1, "vdp_backward": 1, "linear": 2, "mlp": 4}[case]
    B = 3 if case == "mlp" else 5
    w = workloads.make(cfg, B=B)
    t0, t1 = w["t0"].copy(), w["t1"].copy()
    if case == "vdp_backward":
        t0, t1 = t1.copy(), t0.copy() + 2.0  # integrate from t1 down to below 0
        t1 = np.full(B, -1.0)
    rt = dict(rtol=1e-6, atol=1e-6)
    K = 5
    te0 = np.linspace(0, 1, K)[None, :] * (t1 - t0)[:, None] + t0[:, None]
    r = oracle.solve(w["field"], w["y0"], t0, t1, te0, rt, trace_cap=4000)
    assert (r["status"] == 0).all()
    mt, mh, mn = mesh_from_trace(r)
    te = _interior_t_eval(mt, mn, t0, t1, K, rng)
    D = w["y0"].shape[1]
    gye = rng.standard_normal((B, K, D))
    gyf = rng.standard_normal((B, D))
    adj = oracle.adjoint(w["field"], w["y0"], t0, t1, mt, mh, mn, te, gye, gyf,
                         want_t_bounds=True)
    fd0, fd1 = np.zeros(B), np.zeros(B)
    for i in range(B):
        eps = 1e-6 * max(1.0, abs(t1[i]), abs(t0[i]))
        N = mn[i]
        sl = slice(i, i + 1)
        for which in (0, 1):
            vals = []
            for sgn in (1.0, -1.0):
                a0, a1 = t0[sl].copy(), t1[sl].copy()
                m_t, m_h = mt[sl].copy(), mh[sl].copy()
                if which == 1:
                    a1 += sgn * eps
                    m_h[0, N - 1] += sgn * eps
                else:
                    a0 += sgn * eps
                    m_t[0, :N] += sgn * eps
                    m_h[0, N - 1] -= sgn * eps
                f = dict(w["field"])
                for k in ("mu", "A", "Q", "lam"):
                    if k in f:
                        f[k] = f[k][sl]
                vals.append(_loss_replay_t(f, w["y0"][sl], a0, a1, m_t, m_h, mn[sl], te[sl],
                                         gye[sl], gyf[sl])[0])
            (fd1 if which == 1 else fd0)[i] = (vals[0] - vals[1]) / (2 * eps)
    for g, fd in ((adj["gt0"], fd0), (adj["gt1"], fd1)):
        scale = np.maximum(np.abs(fd), 1e-3)
        assert (np.abs(g - fd) <= 1e-5 * scale).all(), (case, g, fd)
    if case != "mlp":
        # with interior points, and with points at t0 and t1 themselves (the
        # first counts as theta = 0 of the first step, the last as theta = 1
        # of the last; finite differences cannot move them, the identity can)
        for pts in (te, te0):
            yp = oracle.solve(w["field"], w["y0"], t0, t1, pts, rt, want_yp=True)["yp_eval"]
            a = oracle.adjoint(w["field"], w["y0"], t0, t1, mt, mh, mn, pts, gye, gyf,
                               want_t_bounds=True)
            ident = -(gye * yp).sum(axis=(1, 2))
            assert np.allclose(a["gt0"] + a["gt1"], ident, rtol=1e-9, atol=1e-9)


def _negated_mlp(field):
    """g(s, y) = -f(-s, y) as an MLP: the time column of the first layer and
    the output layer (weights and bias) negated; IEEE negation is exact."""
    W = [w.copy() for w in field["W"]]
    b = [x.copy() for x in field["b"]]
    D = W[-1].shape[0]
    W[0][:, D] = -W[0][:, D]
    W[-1] = -W[-1]
    b[-1] = -b[-1]
    return dict(field, W=W, b=b)


def test_mlp_backward_in_time_is_forward_with_the_negated_network():
    """The MLP field integrated backward (t1 < t0) is, bit for bit, the
    negated network integrated forward in s = -t (the same method with
    negative steps): outputs, statistics and the mesh; the adjoint on that
    mesh likewise (the weight gradients of the negated layers negated)."""
    w = workloads.make(4, B=4)
    B = w["y0"].shape[0]
    t0, t1 = w["t1"].copy(), w["t0"].copy()  # from 1 down to 0
    te = np.ascontiguousarray(w["t_eval"][:, ::-1])
    opts = dict(rtol=1e-6, atol=1e-6)
    b = oracle.solve(w["field"], w["y0"], t0, t1, te, opts, trace_cap=2000)
    g = _negated_mlp(w["field"])
    f = oracle.solve(g, w["y0"], -t0, -t1, np.ascontiguousarray(-te), opts, trace_cap=2000)
    assert (b["status"] == 0).all()
    for k in ("y_eval", "y_final", "n_acc", "n_rej", "n_feval"):
        assert np.array_equal(b[k], f[k]), k
    L = b["trace_len"]
    for i in range(B):
        assert np.array_equal(b["trace_h"][i, :L[i]], -f["trace_h"][i, :L[i]])
        assert np.array_equal(b["trace_t"][i, :L[i]], -f["trace_t"][i, :L[i]])
    mt, mh, mn = mesh_from_trace(b)
    rng = np.random.default_rng(3)
    gye = rng.standard_normal(b["y_eval"].shape)
    ab = oracle.adjoint(w["field"], w["y0"], t0, t1, mt, mh, mn, te, gye)
    mt2, mh2, mn2 = mesh_from_trace(f)
    af = oracle.adjoint(g, w["y0"], -t0, -t1, mt2, mh2, mn2, np.ascontiguousarray(-te), gye)
    assert np.array_equal(ab["gy0"], af["gy0"])
    D = w["y0"].shape[1]
    assert np.array_equal(ab["gW"][1], af["gW"][1])
    assert np.array_equal(ab["gW"][2], -af["gW"][2]) and np.array_equal(ab["gb"][2], -af["gb"][2])
    assert np.array_equal(ab["gW"][0][:, :D], af["gW"][0][:, :D])
    assert np.array_equal(ab["gW"][0][:, D], -af["gW"][0][:, D])
