"""CPU oracle for the τ-preconditioned GMRES solver of the quasi-compact
Crank-Nicolson scheme for variable-coefficient Riesz fractional diffusion
(She, Zhang, Gu, Serra-Capizzano, arXiv:2404.10221).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import or run anything in this
package.  The product path (the CUDA library and its Python binding) never
calls it, and it shares no code with that path: the only common module is
the seeded input generator ``paper_2404_10221_gb300.workloads``, which holds
none of the method's arithmetic.

Everything is plain NumPy in FP64, written from the paper's equations in the
paper's order; library primitives (matmul, dense solve, eigvalsh) serve as
single steps.  Two tiers:
  * dense tier: explicit Kronecker assembly of A, B, S, tau(S), M for small n;
  * structured tier: the same operators applied as per-dimension mode
    products with explicit N_i x N_i matrices (O(N^{d+1}) per application).

Pins: every function is checked in tests/test_oracle_*.py against closed
forms, invariants, special cases or values printed in the paper (Tables 2-4).
"""

from .tau_oracle import *  # noqa: F401,F403
