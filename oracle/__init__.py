"""FP64 CPU oracle for randomized block Krylov tensor-train approximation.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the paper's algorithms in float64 numpy.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg and reference
arm may import it.  It shares no code, tables, constants or helpers with the CUDA library in
``paper_2308_01480_gb300/``; neither imports the other.

Modules
-------
tt_oracle   TT-SVD (Alg. 1), TT-rBKI (Alg. 3, left block Krylov reading with
            Rayleigh-Ritz truncation; q = 0 is TT-rSVD, Alg. 2), TT-rSI
            (Alg. 4, subspace iteration), both also with the paper's steps
            taken literally (right-side Krylov matrix, first-r truncation),
            Krylov-basis helper, tail energies (Def. 3), TT contraction, the
            relative error and the PSNR of Sec. 4.
philox      Philox4x32-10 counter-based generator (Salmon et al., SC'11) and the
            Box-Muller transform that expand an Omega seed into the Gaussian
            test matrices of Alg. 3 step 3.

Parity status: every function here is pinned by tests in
``tests/test_oracle_*.py`` against closed forms, library routines on special
cases, published known-answer vectors or brute force; none is "parity
unpinned".
"""
from .tt_oracle import (  # noqa: F401
    unfold,
    clamp_ranks,
    orth_top,
    krylov_basis,
    rbki_mode,
    tt_rbki,
    subspace_basis,
    rsi_mode,
    tt_rsi,
    literal_rbki_mode,
    literal_rsi_mode,
    tt_rbki_literal,
    tt_rsi_literal,
    tt_svd,
    tt_full,
    tt_error,
    psnr,
    tt_distance,
    tail_energy,
    left_orthogonality_defect,
)
from .philox import philox4x32_10, omega_from_seed  # noqa: F401
