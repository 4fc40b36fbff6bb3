"""Plain FP64 CPU oracle of the sparsifying-preconditioned GMRES solve (Ying, arXiv 1409.0297).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check of the
package entry file and the CPU-baseline leg of the benchmark may import this
package.  The product path (the CUDA library and its Python binding) never
imports, calls or links it, and this package never imports the product.

The oracle follows the paper step by step in plain numpy/scipy, in float64 /
complex128, with no blocking, fusion or reordering beyond what the paper
states:

  spectral.py   Section 2.1-2.2: shift/potential split (s, q), the
                pseudospectral grid, the unitary DFT, the Laplacian symbol,
                G = (L - s)^{-1} (Eq. G) and the integral operator I + G q.
  stencil.py    Section 2.3: the cell/face/edge/vertex sets, gamma/beta
                neighbourhoods, T_S = G(S, gamma^c) G(beta, gamma^c)^+,
                Q(S, gamma) = [I, -T_S] and C(S, gamma) = Q(S, gamma) G(gamma, gamma).
  precond.py    Section 2.2: sparse Q, C and P = Q + C q, an exact sparse LU of
                P (SuperLU or dense LU; any exact LU gives the same P^{-1}) and the
                preconditioner M r = P^{-1} Q r.
  gmres.py      right-preconditioned GMRES (Saad-Schultz), classical Gram-Schmidt
                applied twice, Givens rotations, explicit true residual.
  fno.py        the Fourier-layer network that supplies the solve's starting vector
                (not part of the paper: Li et al.'s Fourier neural operator and the
                Adam optimiser), forward pass, hand-derived gradient, Adam step.

Every function cites the passage it follows.  Readings where the paper is
silent are stated where they are used.
"""
from .spectral import (wavenumber_grid, laplacian_symbol, green_symbol, green_kernel,
                       apply_green, apply_operator, helmholtz_shift, schrodinger_shift,
                       resonance_gap, dft_matrix)
from .stencil import (set_types, canonical_set, canonical_gamma, canonical_beta, green_block,
                      stencil_tables, tables_from_T, pointwise_stencil_tables, matlab_pinv,
                      annihilation_ratio)
from .precond import SparsifyingPreconditioner, assemble_sparse, sampled_rows, sampled_apply_residual
from .gmres import gmres_right

__all__ = [
    "wavenumber_grid", "laplacian_symbol", "green_symbol", "green_kernel", "apply_green",
    "apply_operator", "helmholtz_shift", "schrodinger_shift", "resonance_gap", "dft_matrix",
    "set_types", "canonical_set", "canonical_gamma", "canonical_beta", "green_block",
    "stencil_tables", "tables_from_T", "pointwise_stencil_tables", "matlab_pinv", "annihilation_ratio",
    "SparsifyingPreconditioner", "assemble_sparse", "sampled_rows", "sampled_apply_residual",
    "gmres_right",
]
