"""Pins of the oracle's joint ("stacked") solving, Sec. 4.1: a mini-batch
of n problems of size p solved as one problem of size np, sharing the step
size, the error norm and every accept/reject decision.

Each pin checks the stacked solve against a route that does not go through
the stacking code, or against what Sec. 4.1 states about its effect.
"""
import numpy as np
import pytest

import oracle

OPTS = dict(rtol=1e-6, atol=1e-6)


def _vdp(B, mu, seed):
    rng = np.random.default_rng(seed)
    return dict(kind="vdp", mu=np.full(B, mu)), rng.uniform(-2.0, 2.0, (B, 2))


def test_joint_of_one_instance_is_the_independent_solve():
    f, y0 = _vdp(1, 3.0, 1)
    te = np.linspace(0.0, 12.0, 7)
    ind = oracle.solve(f, y0, [0.0], [12.0], te[None, :], OPTS)
    j = oracle.solve_joint(f, y0, 0.0, 12.0, te, OPTS)
    assert j["status"] == 0
    assert (j["n_acc"], j["n_rej"], j["n_feval"]) == (ind["n_acc"][0], ind["n_rej"][0],
                                                     ind["n_feval"][0])
    assert np.array_equal(j["y_eval"], ind["y_eval"])
    assert np.array_equal(j["y_final"], ind["y_final"])


def test_joint_linear_batch_is_one_block_diagonal_system():
    # B linear instances stacked = one linear instance whose matrix is the
    # block diagonal of the A_i (solved through the plain linear field: the
    # off-diagonal zeros add exact zeros, so the two runs agree bit for bit)
    rng = np.random.default_rng(2)
    B, D = 5, 3
    A = rng.standard_normal((B, D, D)) * 0.7 - 0.3 * np.eye(D)
    y0 = rng.standard_normal((B, D))
    te = np.array([0.0, 0.4, 1.1, 2.0])
    j = oracle.solve_joint(dict(kind="linear", A=A), y0, 0.0, 2.0, te, OPTS, trace_cap=500)
    big = np.zeros((1, B * D, B * D))
    for b in range(B):
        big[0, b * D:(b + 1) * D, b * D:(b + 1) * D] = A[b]
    ref = oracle.solve(dict(kind="linear", A=big), y0.reshape(1, B * D), [0.0], [2.0],
                       te[None, :], OPTS, trace_cap=500)
    assert j["status"] == 0 and j["n_acc"] == ref["n_acc"][0] and j["n_rej"] == ref["n_rej"][0]
    assert np.array_equal(j["y_eval"], ref["y_eval"][0].reshape(len(te), B, D).transpose(1, 0, 2))
    assert np.array_equal(j["trace_h"], ref["trace_h"][0, :j["trace_len"]])


def test_joint_of_identical_copies_steps_like_one_instance():
    # n copies of one problem: the stacked RMS norm equals the single
    # instance's (up to the rounding of the longer sum), so the mesh does too
    f1, y1 = _vdp(1, 5.0, 3)
    n = 6
    fn = dict(kind="vdp", mu=np.full(n, 5.0))
    te = np.linspace(0.0, 15.0, 11)
    one = oracle.solve(f1, y1, [0.0], [15.0], te[None, :], OPTS)
    j = oracle.solve_joint(fn, np.repeat(y1, n, axis=0), 0.0, 15.0, te, OPTS)
    assert (j["n_acc"], j["n_rej"]) == (one["n_acc"][0], one["n_rej"][0])
    np.testing.assert_allclose(j["y_eval"], np.repeat(one["y_eval"], n, axis=0),
                               rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("mu", [1.0, 10.0])
def test_joint_vdp_batch_needs_more_steps(mu):
    # Sec. 4.1: stacked oscillators share the smallest step of the batch at
    # every moment, so the joint solve takes at least as many steps as the
    # slowest instance and, for strong damping, several times the typical one
    B = 16
    f, y0 = _vdp(B, mu, 4)
    T = 3.0 * mu + 10.0
    te = np.linspace(0.0, T, 9)
    ind = oracle.solve(f, y0, np.zeros(B), np.full(B, T), np.tile(te, (B, 1)), OPTS)
    j = oracle.solve_joint(f, y0, 0.0, T, te, OPTS)
    assert j["status"] == 0 and (ind["status"] == 0).all()
    assert j["n_acc"] >= ind["n_acc"].max()
    ratio = j["n_acc"] / ind["n_acc"].mean()
    if mu >= 10.0:
        assert ratio > 2.5, ratio
    else:
        assert ratio < 2.0, ratio


def test_joint_dense_output_stays_accurate():
    # the shared mesh still resolves every instance: at a tight tolerance the
    # joint solution agrees with the independent one to about the tolerance
    B = 8
    f, y0 = _vdp(B, 2.0, 5)
    te = np.linspace(0.0, 8.0, 5)
    o = dict(rtol=1e-9, atol=1e-9)
    ind = oracle.solve(f, y0, np.zeros(B), np.full(B, 8.0), np.tile(te, (B, 1)), o)
    j = oracle.solve_joint(f, y0, 0.0, 8.0, te, o)
    np.testing.assert_allclose(j["y_eval"], ind["y_eval"], atol=1e-6)


def test_joint_adjoint_of_a_stacked_field_is_refused():
    # the oracle adjoint runs per instance on the shared mesh instead
    f, y0 = _vdp(2, 1.0, 6)
    lib = oracle.oracle._load()
    inner = oracle.oracle._FieldHolder(f, 2)
    st = oracle.oracle._Field()
    st.kind, st.D, st.n_inner = 4, 4, 2
    import ctypes as C
    st.inner = C.cast(C.pointer(inner.f), C.c_void_p)
    z = np.zeros(8)
    n = np.zeros(1, np.int32)
    rc = lib.orc_adjoint(C.byref(st), 1, oracle.oracle._ptr(z), oracle.oracle._ptr(z),
                         oracle.oracle._ptr(z), oracle.oracle._ptr(z), oracle.oracle._ptr(z),
                         oracle.oracle._iptr(n), 1, None, 0, None, oracle.oracle._ptr(z),
                         oracle.oracle._ptr(z), oracle.oracle._ptr(z), None, None, 1)
    assert rc == -1
