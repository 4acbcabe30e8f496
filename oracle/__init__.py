"""Plain FP64 CPU oracle for the plane-wave Kohn-Sham Hamiltonian and its lowest eigenpairs.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import or run anything in this package.  The CUDA library
and its Python binding never import it, link it or fall back to it; the two implementations
share no code apart from the seeded input generators in ``workloads``.

Every function here follows the statement of the problem in the paper (arXiv 2507.08578):
the Kohn-Sham eigenproblem in a plane-wave basis in Hartree atomic units (§1), with
H = kinetic + local potential applied through Fourier transforms + the separable nonlocal
operator of the nonlocal-Hamiltonian equation (Eq. ham-nl, §5.2), solved for its lowest
bands (§5.1).  The oracle computes the plain definition: the finite Hermitian matrix H and
its dense eigendecomposition, plus a naive-DFT H-apply as a second, independent form.
"""
from .kss_oracle import *  # noqa: F401,F403
