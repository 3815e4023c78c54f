"""GB300-native level-dependent multigrid for the indefinite Helmholtz equation.

A small C-ABI CUDA library (include/hh.h, built in-tree for sm_103a) with a
thin Python face: ``HelmholtzMG`` (setup / solve / adjoint / step API) and
``helmholtz_solve`` (a torch.autograd.Function giving d loss / d k^2 and
d loss / d f through the adjoint solve).  Method: Cools, Reps and Vanroose,
"A new level-dependent coarse grid correction scheme for indefinite Helmholtz
problems" (arXiv 1211.4752).
"""

from ._binding import HHError, lib, lib_path  # noqa: F401
from .mg import HelmholtzGroup, HelmholtzMG, HelmholtzSolve, helmholtz_solve, solve_group  # noqa: F401

__all__ = ["HelmholtzGroup", "HelmholtzMG", "HelmholtzSolve", "helmholtz_solve", "solve_group", "HHError",
           "lib", "lib_path"]
