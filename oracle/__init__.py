"""FP64 CPU oracle for the iterative Poisson solvers of arXiv 2605.03563.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the method in numpy float64, written from the paper (Sec. 2,
Eqs. 1-5, the MG error operator of Sec. 2.1.3, Eqs. outer_expansion and
outer_multipole of Sec. 2.2).  Only tests/, __graft_entry__.smoke() and the
CPU-baseline / reference legs of bench.py may import it.  It shares no code
with the CUDA library and must never be used as a fallback for it.

Modules
-------
grid        grid conventions and the MG level hierarchy
operators   7-point / 13-point Cartesian Laplacians, residuals
spherical   variable-coefficient spherical Laplacian (Eq. 2), red-black SOR with
            position-dependent weights (Eq. omega_n with Eq. local_rjac)
smoothers   multicolour Gauss-Seidel / SOR sweeps (Sec. 2.1.1), omega (Eqs. 3-5,
            the Chebyshev sequence of Eq. omega_n)
transfer    full-weighting restriction and P = 8 R^T prolongation (Sec. 2.1.3)
krylov      CG (Sec. 2.1.2) and right-Jacobi-preconditioned BiCGSTAB
multigrid   V-cycle, MG solve, FP64 iterative-refinement driver, PCG
compact     compact 2nd/4th/6th-order stencils, SPAI smoothers (Table 1), Galerkin
            coarse operators and their multigrid (Sec. 2.1.3)
multipole   real spherical harmonics, moments and boundary potential (Sec. 2.2)
solve       the whole-solve drivers that mirror the C ABI's poisson_solve
"""
