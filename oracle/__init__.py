"""FP64 CPU oracle for the three-phonon scattering path of the kALDo 2.0 paper.

TEST INFRASTRUCTURE ONLY.  This package exists to check the CUDA library.  Only the
test suite, the smoke check and the bench's CPU-baseline leg may import it; the product
path (the C-ABI library and its Python binding) never does, and shares no code with it.

Every function follows the paper's equations in the paper's order, written plainly in
NumPy float64 (library primitives: matmul/einsum, eigh).  Where the paper is garbled or
silent, the reading taken is stated in the docstring of the function that applies it.

Modules
  constants  -- CODATA values and unit conversions (the paper gives none)
  grid       -- q-mesh indexing, q'' = -(q+q') mod G, irreducible set (Sec. Overview: IBZ)
  harmonic   -- Eqs. (dynmat_reciprocal), (eigenvalue_crystal), (groupvel)
  occupation -- Eqs. (bose), (heatcap)
  anharmonic -- Eqs. (phi3_proj), (gamma), (broadening), (lifetime)
  transport  -- Eq. (rta)
  bte        -- Eqs. (gamma1), (sc_iter), (inverse): iterative and direct linearised BTE
  supercell  -- Gamma-only brute force of Eq. (phi3_proj) on a supercell (folding pin)
  gammapoint -- Gamma-only linewidths of a large cell mode by mode, sparse Phi3 (1000-atom cell)
  isotope    -- Eq. (isotope): Tamura mass-variance scattering
  qhgk       -- Eqs. (qhgk), (qhgk_crystal): quasi-harmonic Green-Kubo conductivity
  surrogate  -- FP64 reference of the linewidth surrogate network (checks the GPU training)

Parity status: every function here is pinned by tests under tests/ (closed forms,
invariants, brute force); none is "parity unpinned" except the absolute value of the
LJ-argon conductivity, for which the paper prints no number.
"""
from . import constants, grid, harmonic, occupation, anharmonic, transport, supercell, surrogate, gammapoint, isotope, qhgk, bte  # noqa: F401
