"""FP64 CPU oracle for batched adaptive explicit Runge-Kutta 5(4) solving:
Dormand-Prince (dopri5) and Tsitouras (tsit5) pairs.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg use it.  The product path never imports it.
"""
from .oracle import (  # noqa: F401
    build,
    default_opts,
    field_eval,
    dense_weights,
    solve,
    solve_joint,
    replay,
    adjoint,
    joint_adjoint,
    tableau_doubles,
    tableau_m,
    dense_weights_m,
    METHODS,
    STATUS,
)
