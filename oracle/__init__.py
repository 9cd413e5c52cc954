"""FP64 / complex128 CPU oracle for the sparse radio-interferometric imaging hot path.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
reference that the CUDA path is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  The product path (the C-ABI library and its Python binding) never imports,
calls or links anything here, and shares no code, tables or constant
generators with it.

Modules (each function cites the passage of the paper it follows):

* ``kb``          -- Kaiser-Bessel gridding kernel, its Fourier transform, the
                     pre-sampled table (Sec. 7.3, Sec. 8.1).
* ``measurement`` -- the measurement operator Phi = W G F Z S and its adjoint
                     (Sec. 2, Eq. 2), plus the brute-force non-uniform DFT of
                     the measurement equation (Sec. 2, Eq. 1).
* ``wavelets``    -- Daubechies filters by spectral factorisation and the SARA
                     analysis/synthesis operators Psi^dagger / Psi
                     (Sec. 3.1, Sec. 6.4, Sec. 7.1).
* ``prox``        -- proximal operators: positivity projection, soft
                     thresholding, l2-ball projection (Sec. 4).
* ``solvers``     -- power iteration for ||Phi||^2, the primal-dual solver
                     (Appendix A.4, Algorithm 7) and Dual Forward-Backward ADMM
                     (Sec. 5, Algorithm 1).
* ``wstack``      -- the non-coplanar measurement equation (brute force) and its
                     w-stacking operator (the wide-field method Sec. 7.1 names;
                     reading R14).

Parity status: every function here is pinned by a ``-m "not gpu"`` test to
something other than itself (closed forms, a brute-force DFT, quadrature,
orthonormality, a special case with a closed-form solution).  No function is
"parity unpinned".
"""

from . import kb, measurement, wavelets, prox, solvers, wstack  # noqa: F401
