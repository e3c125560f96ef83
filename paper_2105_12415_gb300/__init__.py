"""GB300-native multiresolution triangle-mesh contact detection (Noble &
Weinzierl, arXiv 2105.12415): surrogate trees, level-synchronous pruning with
the penalty sweep, exact comparison-based refinement, penalty forces and their
adjoint, the redundant-contact merge and the implicit time step's broad phase and
Picard update, all in CUDA kernels for sm_103a behind the C
ABI of include/mrdem.h."""
from . import _lib  # noqa: F401
from ._lib import MrdemError, default_params, load  # noqa: F401
from .api import (  # noqa: F401
    Context, Contacts, ContactEnergy, ContactProblem, Hierarchy, contact_energy, contact_forces,
    contact_grad, detect, detect_plain_fp64, merge_contacts, triangle_distance, broad_phase,
    move_poses, picard_update, implicit_euler_step, contact_hessian, newton_residual, newton_solve,
    implicit_euler_step_newton, refine_contacts, motion_bound, KeptCandidates, autotune,
    twist_grad, ActiveSets, active_sets_init, active_sets_step, surrogate_forces,
    implicit_euler_step_multires,
)
from .buildlib import build  # noqa: F401
