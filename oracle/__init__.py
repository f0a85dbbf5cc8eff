"""CPU oracle for the generalized shifted COCG hot path (TEST INFRASTRUCTURE).

This package is the plain, slow, obviously-correct reference that the CUDA
path is checked against.  It is test infrastructure: only the tests, the
smoke check in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py``
may import it.  The library under ``paper_1002_1202_gb300`` never imports it,
and it imports nothing from there; the only code the two sides share is the
seeded input generator ``tbinputs`` (geometry, STO overlaps, energy grids),
which holds none of the method's arithmetic.

Modules
-------
dense   The exact definitions, in complex float64: the ASED Hamiltonian
        (Eq. Hap-1), x_j(z) = (zS - H)^-1 e_j by Gaussian elimination with
        partial pivoting (Eq. base-2 / Eq. GreensFunc), the Mulliken
        populations, a Gauss-Jordan inverse for brute-force checks, Cholesky
        and a cyclic Jacobi eigensolver for the sum-rule closed form, and the
        adjoint quantities: dG/dz = -G S G, the band energy Tr(rho H) and its
        gradients with respect to the entries of H and S.
method  The method in the paper's order and notation: the generalized
        shifted COCG with a seed system, the shift equation for pi, the
        collinear residuals and seed switching (Section 3.3, Eqs. CGp:p,
        CGp:x, CGp:r, shift:pi, collinear), the inner CG for S^-1 r, and the
        generalized Lanczos process (Section 3.2, Eqs. 1.13, 1.18).
        With derivative=True it also carries d/dz_k of every shift's iterates
        through the same recurrences (forward-differentiated shift equation).
csc     Charge self-consistency (Section 2.2, Eq. Hap-CSC): the potential
        V = gamma dq, the correction 1/2 S (V_i + V_j), the second-order
        energy it derives from, and a linear-mixing loop over dense
        Mulliken populations.
"""
