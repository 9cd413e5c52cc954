"""Proximal operators (oracle, FP64).  Test infrastructure only.

Sec. 4 of the paper: the projection onto the positive orthant (Sec. 4.1,
indicator function of C = R_+^N), the l2-ball projection centred at a point
(Sec. 4.2, the ball prox and its translated form), and soft thresholding as the
prox of the l1 norm (Sec. 4.3).  The Moreau decomposition (Sec. 4, proximal
calculus) turns these into the dual steps of the primal-dual solver.

Readings:
* R7: the ball is centred at the data y, the argument is the point projected
  (Algorithm 1 applies the projection to v + s with centre y).
* Ties: |x| = lambda thresholds to 0; ||x - z|| = eps returns x unchanged (the
  paper's "<=" branches).
"""

import numpy as np


def proj_positive(x):
    """P_C(x) for C = R_+^N: elementwise max(x, 0); complex input keeps max(Re x, 0)."""
    x = np.asarray(x)
    return np.maximum(np.real(x), 0.0)


def soft_threshold(x, lam):
    """soft_lambda(x)_i = 0 if |x_i| <= lambda else x_i (|x_i| - lambda) / |x_i| (real or complex)."""
    x = np.asarray(x)
    mag = np.abs(x)
    with np.errstate(invalid="ignore", divide="ignore"):
        scale = np.where(mag > lam, (mag - lam) / np.where(mag > 0, mag, 1.0), 0.0)
    return x * scale


def clip_linf(x, lam):
    """(I - soft_lambda)(x): the prox of the conjugate of lambda ||.||_1, i.e. projection onto
    the l-infinity ball of radius lambda (real: clip to [-lambda, lambda]; complex: radial)."""
    x = np.asarray(x)
    return x - soft_threshold(x, lam)


def proj_l2ball(x, center, eps):
    """Projection of x onto {v : ||v - center||_2 <= eps} (Sec. 4.2); the norm is taken in FP64."""
    x = np.asarray(x)
    d = x - center
    nrm = float(np.sqrt(np.sum(np.abs(d) ** 2)))
    if nrm <= eps:
        return x.copy(), nrm
    return center + d * (eps / nrm), nrm
