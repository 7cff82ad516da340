"""GB300-native Strang splitting for the TDSE on rank-1 / rank-r lattices.

Implements the time-stepping hot path of Suzuki, Suryanarayana and Nuyens,
"Strang splitting in combination with rank-1 and rank-r lattices for the
time-dependent Schroedinger equation" (arXiv:1808.06357): the pseudo-spectral
lattice discretisation (Sec. 2.2, Thm 1) with Strang splitting in time
(Sec. 2.3-2.5, eq. StrangTDSE, Algorithm 1), as hand-written sm_103a CUDA
kernels behind a C ABI (include/lsp.h).  This package is the thin Python
binding of that ABI.
"""

from ._binding import (  # noqa: F401
    AA_EXPLICIT, AA_MINL2, C64, C128, PATH_MIXED, PATH_MULTIPASS, PATH_RANK1_4SWEEP, PATH_RANK1_TMA, PATH_RANK2, PATH_SMALL, PHYSICAL, SPECTRAL,
    Batch, LspError, Plan, adjoint, autotune_cache, cbc_reconstructing, fma_rate, library_path, load_library, strerror, strang_steps_noalloc,
    yoshida4,
)
