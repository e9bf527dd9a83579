"""CPU oracle for block-tridiagonal selected inversion (test infrastructure).

This package is test infrastructure only: the test-suite, the smoke check and the
benchmark's CPU-baseline leg may import it; the library path never does, and it shares no
code with the CUDA kernels.  Everything is plain numpy / scipy in float64 / complex128.

What it computes (the plain definitions the recursive Green's function method reaches):
  * Sec. 3, Eq. 1 and Table 2: for each energy the quadratic system
        (M - B^R) X^<> (M - B^R)^H = B^<>,   X^R = (M - B^R)^{-1},
    solved by *dense* inversion of the full N_B*N_BS matrix and one dense triple product.
  * Sec. 4.2 (retarded OBC, Eq. 4): the lead surface function x = (m - n x n')^{-1}, by
    Sancho-Rubio decimation (the paper cites Sancho et al. 1985 and does not print it), and
    independently by the direct eigen-decomposition route (Eq. 6, polynomial eigenproblem).
  * Sec. 4.2 (lesser/greater OBC): fluctuation-dissipation from the retarded boundary block.
  * Sec. 5.2: the symmetrisation X_ij <- (X_ij - X_ji^*)/2.
  * Table 2, right column: the W system M = I, B^R = V P^R, B^<> = V P^<> V^H, W^R = X^R V;
    with contacts (Sec. 4.2, Eq. 4 and 7), the leads folded into the edge cells by the retarded
    recursion and a Stein (discrete Lyapunov) equation for the lesser / greater boundary.
  * Sec. 4.4, Eq. 3: the element-wise energy convolution, as its explicit sum (energy_conv.py).

Pins (tests/test_oracle_pins.py) tie every function to something other than itself: closed
forms of the 1D chain, integer transmission, the eigen-route surface function, algebraic
identities, brute force on tiny cases.
"""
from .negf import *  # noqa: F401,F403
from .energy_conv import *  # noqa: F401,F403
