"""FP64 CPU oracle for GP-FVM -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never calls it, and it
shares no code, table or helper with the GPU path: the only common input is the
seeded problem statement from ``gpfvm_workloads``.

Contents (see ``gpfvm_oracle`` for citations per function):
  * 1D Matern-5/2 covariance, its derivatives and single/double antiderivatives
    (Sec. 3.1, Eq. linop-simplified) and covariances of 1D test functionals;
  * dense Gram assembly entry by entry from Eq. (LkL) and the exact posterior
    (Eqs. lin-cond-mean / lin-cond-cov) by Cholesky;
  * an independent Kronecker matvec (Eq. kronecker-structure), the Cholesky
    (IC/BC) deflation of Sec. 4.2 and CG with the IterGP combined posterior
    (Sec. 4.1) for problems too large to assemble densely.
"""
from .gpfvm_oracle import *  # noqa: F401,F403
