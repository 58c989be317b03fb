"""FP64 CPU oracle for the spacetime finite-element Dirac solver.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
restatement of what the method computes, used to check the CUDA path.  Only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The product library
(``paper_2103_14588_gb300``) never imports, links or calls anything here, and
this package imports nothing from the product library: the two share no code.

Everything is complex128 / float64 numpy, and float64 torch CPU ops for the
U-Net.  Library primitives used as single steps: Gauss-Legendre nodes
(numpy), dense LU (LAPACK via scipy), sparse LU (SuperLU via scipy), FFT
(numpy), Hermitian eigendecomposition (LAPACK), an adaptive ODE integrator
(scipy), 2D / 3D convolutions and automatic differentiation (torch).

Modules and the passages they follow (section / equation of the paper):

* ``dirac``       gamma, alpha, beta matrices          Sec. 2.1 Eq. 1, Appendix A
* ``element``     Q1 basis + element matrices          Sec. 2.2 Eqs. 13-16, Appendix A
* ``mesh``        structured spacetime mesh, indexing   Sec. 2.1 Eqs. 8-11, Algorithm 1
* ``operator``    D_w assembly, split, apply, RHS       Sec. 2.1 Eqs. 6-12, Sec. 2.2, Algorithm 1
* ``solvers``     restarted GMRES(m), flexible GMRES,   Sec. 2.2 (GMRES), Algorithm 1 step 6;
                  BiCGSTAB, dense/sparse LU             Sec. 4.1 tables (BiCGSTAB)
* ``precond``     block Jacobi, time-slab Schwarz,      Sec. 5 (the conclusion's call for a
                  Crank-Nicolson sweep                  preconditioner)
* ``unet``        convolutional U-Net preconditioner    no counterpart in the paper
* ``exact``       plane wave / packet / Klein formulas  Appendix B, Sec. 4.2 Eq. 18, Sec. 4.3 Eq. 24
* ``observables`` charge, <x>, T/R by trapezoid         Sec. 4.1, Sec. 4.2 Eq. 20, Sec. 4.3 Eq. 25

Parity status of each function is stated in its module docstring; every
function is pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py``
except where a module says "parity unpinned".
"""

from . import dirac, element, mesh, operator, solvers, exact, observables, precond  # noqa: F401
