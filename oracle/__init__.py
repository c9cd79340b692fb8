"""CPU oracle for the Hubbard exact-diagonalization hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call,
link or execute anything in this package: only the tests, the smoke check
and the CPU-baseline leg of the benchmark use it.  It shares no code with
the CUDA library (its basis, signs, tables and Lanczos are written here
from the paper's definitions); the only common dependency is the seeded
input package `workload`, which holds none of the method's arithmetic.

Modules
  basis        basis enumeration and ranking (Sec. 2.1, Eq. J-formula),
               generic Jordan-Wigner signs over all 2*Ns modes, the
               explicit sparse H of Eq. (1), sampled rows of H*v, and the
               per-spin hopping tables used for bit-exact comparison.
  lanczos      Algorithm 1, its two-vector form (Eqs. split1), a fully
               reorthogonalised variant and the tridiagonal eigensolve.
  closed_forms dimer, t = 0 and U = 0 ground-state energies.
  kron         plain-C Kronecker-sum H*v (Eq. H-Kroneckersum, the CPU
               scheme of Sec. 5) for sectors too large for explicit H.
  propagate    exp(-iHt) v (the time propagation Sec. 6 names as the other
               use of H*v) by the eigendecomposition of the dense H, by
               expm_multiply on the sparse H, and the closed forms and
               series that pin them.
"""
