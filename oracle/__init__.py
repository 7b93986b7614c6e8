"""Plain FP64 CPU oracle of the FEAST interval eigensolver (arXiv 1605.08771).

This package is test infrastructure: it is imported only by the tests, by the
package smoke check and by the CPU-baseline leg of the benchmark.  The product
path (the CUDA library and its Python binding) never imports or runs it, and
the oracle shares no code with that path.

Modules:
  quadrature  Gauss-Legendre nodes, contour nodes/weights, scalar filter (Eqs. 2-3)
  dense       LU with partial pivoting, triangular solves, Cholesky-QR, Gram
              orthogonalisation, Jacobi eigensolver
  feast       filter application, Rayleigh-Ritz, selection, FEAST / XFEAST /
              RFEAST drivers (Appendix algorithms)
  exact       correctly rounded FP64 dot products (TwoProduct + exact
              summation): reference of the FP64-accurate refinement products
  general     FEAST for a general (non-Hermitian) matrix on a circle contour
  density     stochastic-trace Chebyshev moments and the count they estimate
  mlp         the proposer's MLP (forward, backward, Adam)

Parity pins: every function is checked in tests/test_oracle_*.py against
closed forms, brute force or independent library routines.  Plain FEAST's
iterates are pinned round by round: every round's in-I Ritz values, its
residual history and its round count follow from subspace iteration on
rho(A) computed in the planted eigenbasis.  The XFEAST and RFEAST drivers are
pinned by the end result on planted spectra, by their first rounds in closed
form (Rayleigh-Ritz on the Krylov windows of rho(A) of XFEAST's rounds 1 and
2, and on [Y, A Y] for RFEAST's round 1 with s = 2), by one-round
convergence where the mathematics fixes it (an invariant start; an expanded
subspace that spans the whole space, s m0 = n), and by the Rayleigh-Ritz
dimensions the literal RFEAST expansion must produce; with s = 1 both reduce
to subspace iteration on rho(A) and are pinned at every round.  Their later
rounds with s >= 2 (XFEAST from round 3, RFEAST from round 2: which pairs
are selected, the residual histories) have no independent pin: "parity
unpinned" there.
"""
from .quadrature import gauss_legendre, contour_nodes, rational_filter, circle_nodes, circle_filter  # noqa: F401
from .dense import (lu_factor, lu_solve, lu_solve_adjoint, lu_unpack,  # noqa: F401
                    cholesky_upper, cholqr, cholqr2, jacobi_eigh, gram_eig_orth,
                    round_robin_pairs, solve_right_upper, CholeskyBreakdown)
from .feast import (factor_shifts, filter_apply, rayleigh_ritz, select_pairs,  # noqa: F401
                    feast_solve, norm_estimate, orthonormalize, FeastResult,
                    PLAIN, XFEAST, RFEAST, EXPAND_ALL, EXPAND_UNCONVERGED)
from .exact import two_prod, dot_exact, matmul_entries  # noqa: F401
from .general import feast_solve_general, filter_apply_general, factor_circle  # noqa: F401
