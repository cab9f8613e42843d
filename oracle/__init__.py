"""CPU FP64 oracle for the pipelined flexible Krylov methods (arXiv 1511.07226).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import anything from here.
The GPU library never calls it, and it never calls the GPU library: the two
share no code, only the seeded input arrays of the ``workloads`` module.

It is plain NumPy in float64, written to be read against the paper:

* ``operators``        -- the cell-centred finite-volume operators (stencil,
                          CSR, dense, diagonal) written from their definition.
* ``preconditioners``  -- Jacobi, inner Jacobi-PCG (Alg. 3), Chebyshev-Jacobi,
                          the noisy preconditioner of Fig. FCGtoy, dense.
* ``krylov``           -- every method of the paper, step by step in the
                          paper's order and notation: CD-family FCG (Alg. 2),
                          PCG (Alg. 3), CGFCG (Alg. 6), naive PIPEFCG (Alg. 7),
                          PIPEFCG (Alg. 8), GCR (Alg. 9), PIPEGCR (Alg. 11),
                          PIPEGCR_w (Alg. 12), FGMRES (Alg. 13), CGFGMRES
                          (Alg. 14) and PIPEFGMRES (Alg. 15).

Pins (tests/test_oracle_*.py) tie every function to something other than
itself: dense LU, Krylov-subspace minimisation by brute force, closed-form
Chebyshev error polynomials, finite termination, orthogonality invariants and
the toy experiment of Fig. FCGtoy.  The mixed-precision (FP32 / BF16
coefficient) preconditioner emulations follow a stated rounding model (the
paper fixes no reduced-precision arithmetic) and are pinned by its
properties: representability and unit-roundoff bounds of the coefficient
copies, the error bound of the reduced-precision operator, the closed-form
Chebyshev error polynomial with the rounded D^-1, and the one-cell inner
PCG.
"""
from . import operators, preconditioners, krylov  # noqa: F401
