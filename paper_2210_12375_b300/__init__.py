"""B300-native batched adaptive Dormand-Prince 5(4) (torchode's method).

Every instance of a batch is solved independently with its own step size,
accept/reject decisions and evaluation points (torchode, Sec. 3).  The
solver is the C-ABI library ``libtode.so`` (hand-written CUDA for sm_103a);
this package only marshals torch tensors into it.
"""
from . import _abi  # noqa: F401
from .api import (MLP, Linear, Solution, TapeBuffers, VdP, adjoint, make_options,  # noqa: F401
                  solve, t_bounds_grad, t_eval_grad, joint_adjoint, joint_adjoint_workspace,
                  mlp_resolve)
from .autograd import odeint_adjoint  # noqa: F401
from .tuning import autotune, set_cache_path  # noqa: F401

__all__ = ["VdP", "Linear", "MLP", "solve", "adjoint", "TapeBuffers", "Solution",
           "make_options", "odeint_adjoint", "autotune", "set_cache_path", "t_bounds_grad",
           "joint_adjoint", "joint_adjoint_workspace",
           "t_eval_grad", "mlp_resolve"]
