"""Kaiser-Bessel gridding kernel (oracle, FP64).  Test infrastructure only.

The paper interpolates visibilities off the oversampled FFT grid with a
Kaiser-Bessel kernel of support J = 4 (Sec. 7.3) and pre-samples it on a fine
1-D grid over 0 <= |u_pix| <= J/2, using its symmetry g(u) = g(-u), with
zeroth-order (nearest-sample) interpolation (Sec. 8.1).  The paper does not
print the kernel's formula; the readings used here are:

* R3 kernel: g(t) = I0(beta*sqrt(1 - (2t/J)^2)) / I0(beta) for |t| < J/2, and 0
  otherwise (open support: the edge sample at exactly J/2 is 0).  The default
  beta = 2.34 J is Fessler's choice for oversampling 2.
* Correction: the continuous Fourier transform of g,
  ghat(nu) = J sinh(sqrt(beta^2 - (pi J nu)^2)) / (I0(beta) sqrt(beta^2 - (pi J nu)^2)),
  with sin / sqrt of the magnitude when the square root's argument is negative.
* R4 table: table[i] = g(i/S) for i = 0 .. (J/2) S, with S samples per grid
  cell.
"""

import numpy as np
from scipy import special


def default_beta(J):
    """beta = 2.34 J (reading R3)."""
    return 2.34 * float(J)


def kernel(t, J, beta):
    """g(t) of reading R3, vectorised, FP64.  Open support |t| < J/2."""
    t = np.asarray(t, dtype=np.float64)
    r = 2.0 * t / float(J)
    inside = np.abs(r) < 1.0
    arg = np.sqrt(np.where(inside, 1.0 - r * r, 0.0))
    val = special.i0(beta * arg) / special.i0(beta)
    return np.where(inside, val, 0.0)


def kernel_ft(nu, J, beta):
    """ghat(nu): continuous Fourier transform of g (sign convention irrelevant: g is even)."""
    nu = np.asarray(nu, dtype=np.float64)
    s = beta * beta - (np.pi * J * nu) ** 2
    a = np.sqrt(np.abs(s))
    with np.errstate(invalid="ignore", divide="ignore"):
        pos = np.sinh(a) / a
        neg = np.sin(a) / a
    ratio = np.where(s > 0, pos, np.where(s < 0, neg, 1.0))
    ratio = np.where(a == 0.0, 1.0, ratio)
    return J * ratio / special.i0(beta)


def table(J, S, beta):
    """Pre-sampled kernel table[i] = g(i/S), i = 0 .. (J/2) S (Sec. 8.1, reading R4)."""
    n = (J // 2) * S + 1
    return kernel(np.arange(n, dtype=np.float64) / float(S), J, beta)


def correction_1d(n_side, K, J, beta):
    """S of Eq. 2 along one axis: 1 / ghat(p'/K) for centred pixel p' = p - n_side/2."""
    p = np.arange(n_side, dtype=np.float64) - n_side // 2
    return 1.0 / kernel_ft(p / float(K), J, beta)
