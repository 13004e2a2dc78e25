"""FP64 CPU oracle for the pseudospectral Taylor-Couette time step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_1908_00587_gb300``) and never imports it.

The oracle is slow and plain: dense matrices for the radial operators, LAPACK
(``numpy.linalg.solve``, partial pivoting) for every radial solve, explicit
matrix DFTs for the (theta, z) transforms (an FFT mode via ``scipy.fft`` is
kept for timing and larger cases), and the predictor-corrector steps written
out in the order the scheme takes them.

The paper (arXiv:1908.00587, Sec. 2.1) fixes the ingredients -- a
Fourier-Galerkin ansatz in theta and z, 9-point finite differences in r on a
selectable radial grid, a predictor-corrector time integrator with dynamic time
step, Boussinesq buoyancy with a radial temperature drop and gravity along z,
divergence-free initial conditions, the analytic basic state and the Nusselt
number of Sec. 4 -- but prints no equations.  Every reading taken where the
paper is silent is stated in the docstring of the function that takes it.
"""
from .grid import Grid, fornberg_weights, fd_matrices, cgl_radii, cc_weights  # noqa: F401
from .spectral import Spectral  # noqa: F401
from .model import Model  # noqa: F401
