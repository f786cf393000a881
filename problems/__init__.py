"""Seeded synthetic inputs (assembled CSR matrices, cell -> DOF maps, right-hand
sides) shared by the CPU oracle and the CUDA path.  Holds no patch-relaxation
arithmetic."""
from .configs import (Problem, poisson2d_q2, stokes2d_q2q1, nedelec3d, diffusion3d_q2, smooth2d_qp,
                      graded_sizes, gaussian_random_field, BUILDERS)

__all__ = ["Problem", "poisson2d_q2", "stokes2d_q2q1", "nedelec3d", "diffusion3d_q2", "smooth2d_qp",
           "graded_sizes", "gaussian_random_field", "BUILDERS"]
from .stokes3d import stokes3d_q2q1

BUILDERS["stokes3d_q2q1"] = stokes3d_q2q1
__all__.append("stokes3d_q2q1")
