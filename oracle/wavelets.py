"""SARA wavelet dictionary: Daubechies filters and Psi / Psi^dagger (oracle, FP64).  Test infrastructure only.

The paper represents the sky with an over-complete frame of wavelet bases
(Sec. 3.1): a Dirac basis plus 2-D separable Daubechies wavelets Db1..Db8
(Sec. 7.5), implemented as separable 2-D discrete Daubechies transforms
(Sec. 7.1).  The frame is the concatenation Psi = [Psi_1 ... Psi_nw]; the
synthesis Psi alpha sums the inverse transforms of every basis and the analysis
Psi^dagger x applies each forward transform to the same image (Sec. 6.4).

Readings:

* dbN has N vanishing moments and 2N taps (Db1 = Haar).  Its low-pass filter is
  the minimum-phase spectral factor of the Daubechies polynomial
  |m0(w)|^2 = cos^{2N}(w/2) P(sin^2(w/2)), P(y) = sum_k C(N-1+k, k) y^k, with
  sum(h) = sqrt(2); the high-pass filter is g[m] = (-1)^m h[2N-1-m].
* R6 boundaries: periodic.  One level of the 1-D analysis maps a length-n signal
  to a[k] = sum_m h[m] x[(2k+m) mod n] (first half) and
  d[k] = sum_m g[m] x[(2k+m) mod n] (second half); the 2-D level transforms the
  rows, then the columns, of the top-left (LL) block, which is recursed on
  (Mallat layout).  Each basis is orthonormal; the stack is scaled by
  1/sqrt(n_w) so that Psi Psi^dagger = I.
* Basis order 0 means the Dirac basis.

The filters are derived here from their definition (roots of P, factor
selection) and never copied from a table or library.
"""

from functools import lru_cache
from math import comb, sqrt

import numpy as np
import scipy.sparse as sp


@lru_cache(maxsize=None)
def daubechies_lowpass(N):
    """Low-pass filter h[0..2N-1] of dbN by spectral factorisation (FP64, Newton-polished roots)."""
    if N < 1:
        raise ValueError("dbN needs N >= 1")
    # P(y) = sum_{k<N} C(N-1+k, k) y^k
    p = np.array([comb(N - 1 + k, k) for k in range(N)], dtype=np.float64)
    factors = np.array([1.0 + 0j])
    if N > 1:
        roots = np.roots(p[::-1]).astype(np.complex128)
        # Newton polish on P(y) to remove the eigen-solver's rounding.
        dp = np.array([k * p[k] for k in range(1, N)])
        for _ in range(8):
            val = np.polyval(p[::-1], roots)
            der = np.polyval(dp[::-1], roots)
            roots = roots - val / der
        for y in roots:
            # y = (2 - z - 1/z) / 4  <=>  z^2 - (2 - 4y) z + 1 = 0 ; keep the root inside |z| < 1
            b = 2.0 - 4.0 * y
            disc = np.sqrt(b * b - 4.0)
            z1, z2 = (b + disc) / 2.0, (b - disc) / 2.0
            r = z1 if abs(z1) < abs(z2) else z2
            # factor (1 - r w) in the filter polynomial H(w) = sum h_n w^n
            factors = np.convolve(factors, np.array([1.0, -r]))
    binom = np.array([comb(N, k) for k in range(N + 1)], dtype=np.float64)
    h = np.convolve(binom, factors).real
    return h * (sqrt(2.0) / h.sum())


def highpass(h):
    """g[m] = (-1)^m h[L-1-m] (quadrature mirror)."""
    L = len(h)
    return np.array([(-1.0) ** m * h[L - 1 - m] for m in range(L)])


@lru_cache(maxsize=None)
def analysis_matrix(n, N):
    """n x n periodic one-level analysis matrix of dbN: rows [h shifted by 2k ; g shifted by 2k]."""
    if n % 2:
        raise ValueError("periodic DWT needs an even length")
    h = daubechies_lowpass(N)
    g = highpass(h)
    A = np.zeros((n, n))
    for k in range(n // 2):
        for m in range(len(h)):
            A[k, (2 * k + m) % n] += h[m]
            A[n // 2 + k, (2 * k + m) % n] += g[m]
    return sp.csr_matrix(A)


def dwt2(x, N, levels):
    """Forward (analysis) 2-D periodic DWT of one dbN basis, Mallat layout."""
    a = np.array(x, dtype=np.float64, copy=True)
    n = a.shape[0]
    for lev in range(levels):
        m = n >> lev
        A = analysis_matrix(m, N)
        blk = a[:m, :m]
        a[:m, :m] = (A @ (A @ blk.T).T)  # rows then columns: A blk A^T
    return a


def idwt2(alpha, N, levels):
    """Inverse (synthesis) 2-D periodic DWT, the transpose of ``dwt2``."""
    a = np.array(alpha, dtype=np.float64, copy=True)
    n = a.shape[0]
    for lev in reversed(range(levels)):
        m = n >> lev
        A = analysis_matrix(m, N)
        blk = a[:m, :m]
        a[:m, :m] = (A.T @ (A.T @ blk).T).T  # A^T blk A
    return a


def psi_adjoint(x, db_orders, levels):
    """Psi^dagger x: stack of per-basis analysis coefficients / sqrt(n_w) (Sec. 6.4)."""
    nw = len(db_orders)
    s = 1.0 / sqrt(nw)
    out = np.empty((nw,) + np.shape(x))
    for b, N in enumerate(db_orders):
        out[b] = s * (np.array(x, dtype=np.float64) if N == 0 else dwt2(x, N, levels))
    return out


def psi(alpha, db_orders, levels):
    """Psi alpha: sum over bases of per-basis synthesis / sqrt(n_w) (Sec. 6.4)."""
    nw = len(db_orders)
    s = 1.0 / sqrt(nw)
    x = np.zeros(alpha.shape[1:])
    for b, N in enumerate(db_orders):
        x += s * (alpha[b] if N == 0 else idwt2(alpha[b], N, levels))
    return x
