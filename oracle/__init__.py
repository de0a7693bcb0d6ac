"""FP64 CPU oracle for the randomized sketching, rsvd and sketch-and-solve least squares of
arXiv:1505.07570 (Wang, "A Practical Guide to Randomized Matrix Computations with MATLAB Implementations").

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it.  The library (``paper_1505_07570_gb300``) never imports it, and it shares no
code with the library: its Philox generator, transforms, QR, SVD and solvers are independent NumPy
restatements of the published definitions, in FP64, with no blocking or fusion beyond what those
definitions state.

Modules
  philox  Philox4x32-10 (Salmon et al., SC'11) and the draws derived from it (Gaussian, signs, hashes,
          SRHT sample).
  sketch  Gaussian projection, SRHT, count sketch (Sec. 3.2), plus their explicit S for tiny inputs.
  linalg  Householder QR, one-sided Jacobi SVD, QR and normal-equation least squares.
  rsvd    randomized k-SVD with q power iterations (Sec. 5.1-5.2).
  lsr     exact and sketch-and-solve least squares (Sec. 4.1-4.2).

Parity status of each function (what pins it) is listed in the module tests under tests/test_oracle_*.py;
every function here has at least one pin that does not rely on the oracle itself.
"""
from . import linalg, lsr, philox, rsvd, sketch  # noqa: F401
