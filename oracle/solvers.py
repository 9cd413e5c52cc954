"""Proximal solvers for the constrained analysis problem (oracle, FP64).  Test infrastructure only.

Problem (Sec. 3.1, analysis form; Sec. 5):
    min_x ||Psi^dagger x||_1  s.t.  ||y - Phi x||_2 <= eps,  x >= 0.

* ``power_iteration``: the power method for the largest eigenvalue of
  Phi^dagger Phi, used to normalise the operator (Sec. 6.3.1).
* ``primal_dual``: Algorithm 7 (Appendix A.4) with L = [Psi^dagger; Phi],
  f(a, b) = gamma ||a||_1 + iota_{B(y, eps)}(b) and g = iota_{R_+^N}.  By the
  Moreau decomposition prox_{sigma f*}(z) = z - sigma prox_{f/sigma}(z/sigma)
  (Appendix A.4), the dual step splits into (reading R8):
      z1 <- clip(z1 + sigma1 Psi^dagger xhat, [-gamma, gamma])
      t  <- z2 + sigma2 Phi xhat
      z2 <- t - sigma2 P_B(y,eps)(t / sigma2)
      x+ <- max(x - tau (Psi z1 + Re Phi^dagger z2), 0)
      xhat <- x+ + theta (x+ - x)
* ``admm``: Dual Forward-Backward ADMM, Algorithm 1 (Sec. 5), with the DualFB
  inner loop reading its argument z (reading R9) and the dual d warm-started
  across outer iterations.
* ``fista``: the unconstrained analysis problem (Sec. 3.1 analysis form, the
  MAP estimate) min_x 1/2 ||y - Phi x||^2 + gamma ||Psi^dagger x||_1, x >= 0, by
  FISTA (Algorithm 4, Sec. 9 / Appendix) with f the data term and g the prior
  plus the positivity indicator; prox_{lambda g} is evaluated by the Dual
  Forward-Backward function of Algorithm 1 with threshold lambda * gamma (reading
  R11: the paper's 1 / (2 sigma^2) data weight is folded into gamma).

Local fidelity constraints (Sec. 6.9, local l2 balls): with ``balls`` = [(idx_j, eps_j)]
(a partition of the visibilities) the single constraint ||y - Phi x|| <= eps becomes
||y_j - Phi_j x|| <= eps_j for every block j, and every projection onto the l2 ball is
the product of the per-block projections (``proj_balls``).  ``balls`` = None is the
global ball.

Weighted l1 (the reweighted analysis of SARA, Sec. 3.1; reading R12): with ``weights``
w (one per coefficient of Psi^dagger x) the prior is gamma sum_i w_i |(Psi^dagger x)_i|,
so every l1 bound gamma becomes gamma w_i.  ``sara_weights`` gives the reweighting
w_i = delta / (delta + |(Psi^dagger x)_i|) for a caller-chosen delta.

Convergence (Sec. 6.6): relative iterate change ||x+ - x|| / ||x+|| < delta.
Every norm is FP64.
"""

from dataclasses import dataclass, replace

import numpy as np

from . import prox


def splitmix64(n, seed):
    """Raw 64-bit outputs of SplitMix64 (Steele, Lea & Flood 2014) at counters seed + k*golden, k = 1..n."""
    mask = (1 << 64) - 1
    out = []
    for i in range(n):
        z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & mask
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        out.append(z ^ (z >> 31))
    return out


def splitmix64_uniform(n, seed):
    """n uniforms in [0, 1): the top 53 bits of ``splitmix64`` times 2^-53.

    This is the counter-based generator both sides implement for the power method's start vector.
    """
    return np.array([(z >> 11) * (1.0 / (1 << 53)) for z in splitmix64(n, seed)], dtype=np.float64)


def power_iteration(phi, phi_adj, shape, seed=0, max_iter=200, tol=1e-8, b0=None):
    """Largest eigenvalue of Phi^dagger Phi (= ||Phi||^2) by the power method (Sec. 6.3.1).

    Start vector: 0.5 + U[0,1) from ``splitmix64_uniform`` unless ``b0`` is given.
    Returns (op_norm_sq, iterations).
    """
    n = int(np.prod(shape))
    b = (0.5 + splitmix64_uniform(n, seed)).reshape(shape) if b0 is None else np.array(b0, dtype=np.float64)
    b = b / np.sqrt(np.sum(b * b))
    prev = 0.0
    val = 0.0
    it = 0
    for it in range(1, max_iter + 1):
        c = phi_adj(phi(b))
        val = float(np.sqrt(np.sum(np.abs(c) ** 2)))
        b = c / val
        if it > 1 and abs(val - prev) <= tol * val:
            break
        prev = val
    return val, it


def proj_balls(z, y, eps, balls):
    """Projection onto the global l2 ball of radius eps around y (balls None) or onto the
    product of the local balls {||z_j - y_j|| <= eps_j} (Sec. 6.9)."""
    if balls is None:
        return prox.proj_l2ball(z, y, eps)[0]
    out = np.array(z, dtype=np.complex128, copy=True)
    for idx, e in balls:
        out[idx] = prox.proj_l2ball(z[idx], y[idx], e)[0]
    return out


@dataclass
class PDParams:
    """Primal-dual parameters (reading R8): sigma1 = 1, sigma2 = 1/||Phi||^2, tau = 0.49, theta = 1."""
    gamma: float
    op_norm_sq: float
    eps: float
    max_iter: int = 200
    rel_tol: float = 0.0
    tau: float = 0.49
    sigma1: float = 1.0
    sigma2: float = 0.0  # <= 0 means 1 / op_norm_sq
    theta: float = 1.0
    balls: object = None  # local l2 balls [(idx_j, eps_j)]; None: the global ball
    weights: object = None  # per-coefficient l1 weights (shape of Psi^dagger x); None: all 1
    reweight: object = None  # (k, delta): after iteration k, weights <- sara_weights(x, delta); duals kept


def _bound(gamma, weights):
    return gamma if weights is None else gamma * np.asarray(weights)


def sara_weights(x, psi_adj, delta):
    """w_i = delta / (delta + |(Psi^dagger x)_i|) (reading R12)."""
    return delta / (delta + np.abs(psi_adj(x)))


def primal_dual(y, phi, phi_adj, psi, psi_adj, p, x0=None):
    """Algorithm 7 instantiated for the constrained analysis problem (reading R8).

    Returns (x, info) with info = {'iters', 'rel_change', 'residual_norm', 'history'}.
    """
    sigma2 = p.sigma2 if p.sigma2 > 0 else 1.0 / p.op_norm_sq
    x = np.zeros_like(np.real(phi_adj(y))) if x0 is None else np.array(x0, dtype=np.float64)
    xhat = x.copy()
    z1 = np.zeros_like(psi_adj(x))
    z2 = np.zeros_like(np.asarray(y, dtype=np.complex128))
    rel = np.inf
    hist = []
    it = 0
    for it in range(1, p.max_iter + 1):
        z1 = prox.clip_linf(z1 + p.sigma1 * psi_adj(xhat), _bound(p.gamma, p.weights))
        t = z2 + sigma2 * phi(xhat)
        proj = proj_balls(t / sigma2, y, p.eps, p.balls)
        z2 = t - sigma2 * proj
        x_new = prox.proj_positive(x - p.tau * (psi(z1) + np.real(phi_adj(z2))))
        xhat = x_new + p.theta * (x_new - x)
        if p.reweight is not None and it == p.reweight[0]:
            p = replace(p, weights=sara_weights(x_new, psi_adj, p.reweight[1]))
        dn = float(np.sqrt(np.sum((x_new - x) ** 2)))
        xn = float(np.sqrt(np.sum(x_new ** 2)))
        rel = dn / xn if xn > 0 else (0.0 if dn == 0 else np.inf)
        hist.append(rel)
        x = x_new
        if p.rel_tol > 0 and rel < p.rel_tol:
            break
    res = float(np.sqrt(np.sum(np.abs(y - phi(x)) ** 2)))
    return x, {"iters": it, "rel_change": rel, "residual_norm": res, "history": hist}


@dataclass
class ADMMParams:
    """Dual Forward-Backward ADMM parameters (Algorithm 1; reading R9)."""
    gamma: float
    eps: float
    rho: float
    varrho: float = 1.0
    eta: float = 1.0
    dualfb_iters: int = 1
    max_iter: int = 200
    rel_tol: float = 0.0
    balls: object = None  # local l2 balls [(idx_j, eps_j)]; None: the global ball
    weights: object = None  # per-coefficient l1 weights; None: all 1
    reweight: object = None  # (k, delta): after iteration k, weights <- sara_weights(x, delta)


def admm(y, phi, phi_adj, psi, psi_adj, p, x0=None):
    """Algorithm 1: v = Phi x; r = P_B(v + s); s += varrho (v - r); xt = x - rho Phi^dagger(v - r + s);
    x = DualFB(xt, gamma) with DualFB: zbar = P_C(z); repeat { d = (1/eta)(I - soft_gamma)(eta d + Psi^dagger zbar);
    zbar = P_C(z - Psi d) }."""
    y = np.asarray(y, dtype=np.complex128)
    x = np.zeros_like(np.real(phi_adj(y))) if x0 is None else np.array(x0, dtype=np.float64)
    s = np.zeros_like(y)
    d = np.zeros_like(psi_adj(x))
    rel = np.inf
    hist = []
    it = 0
    for it in range(1, p.max_iter + 1):
        v = phi(x)
        r = proj_balls(v + s, y, p.eps, p.balls)
        s = s + p.varrho * (v - r)
        xt = x - p.rho * np.real(phi_adj(v - r + s))
        zbar = prox.proj_positive(xt)
        for _ in range(p.dualfb_iters):
            d = (1.0 / p.eta) * prox.clip_linf(p.eta * d + psi_adj(zbar), _bound(p.gamma, p.weights))
            zbar = prox.proj_positive(xt - psi(d))
        if p.reweight is not None and it == p.reweight[0]:
            p = replace(p, weights=sara_weights(zbar, psi_adj, p.reweight[1]))
        dn = float(np.sqrt(np.sum((zbar - x) ** 2)))
        xn = float(np.sqrt(np.sum(zbar ** 2)))
        rel = dn / xn if xn > 0 else (0.0 if dn == 0 else np.inf)
        hist.append(rel)
        x = zbar
        if p.rel_tol > 0 and rel < p.rel_tol:
            break
    res = float(np.sqrt(np.sum(np.abs(y - phi(x)) ** 2)))
    return x, {"iters": it, "rel_change": rel, "residual_norm": res, "history": hist}


@dataclass
class FISTAParams:
    """FISTA parameters (Algorithm 4; reading R11): prior weight gamma, gradient step lam
    (<= 1 / ||Phi||^2 for convergence), DualFB step eta and inner iterations."""
    gamma: float
    lam: float
    eta: float = 1.0
    dualfb_iters: int = 1
    max_iter: int = 200
    rel_tol: float = 0.0
    weights: object = None  # per-coefficient l1 weights; None: all 1
    reweight: object = None  # (k, delta): after iteration k, weights <- sara_weights(x, delta)


def dual_fb(z, thr, d, psi, psi_adj, eta, iters):
    """The DualFB function of Algorithm 1: prox of thr ||Psi^dagger .||_1 + iota_{R+} at z.
    zbar = P_C(z); repeat { d = (1/eta)(I - soft_thr)(eta d + Psi^dagger zbar); zbar = P_C(z - Psi d) }.
    Returns (zbar, d); d is the warm start of the next call."""
    zbar = prox.proj_positive(z)
    for _ in range(iters):
        d = (1.0 / eta) * prox.clip_linf(eta * d + psi_adj(zbar), thr)
        zbar = prox.proj_positive(z - psi(d))
    return zbar, d


def fista(y, phi, phi_adj, psi, psi_adj, p, x0=None):
    """Algorithm 4 on f(x) = 1/2 ||y - Phi x||^2, g = gamma ||Psi^dagger x||_1 + iota_{R+}:
    x+ = prox_{lam g}(xhat - lam Phi^dagger(Phi xhat - y)); theta+ = (1 + sqrt(1 + 4 theta^2)) / 2;
    xhat = x+ + (theta - 1) / theta+ (x+ - x), from x = xhat = x0 (0) and theta = 1."""
    y = np.asarray(y, dtype=np.complex128)
    x = np.zeros_like(np.real(phi_adj(y))) if x0 is None else np.array(x0, dtype=np.float64)
    xhat = x.copy()
    d = np.zeros_like(psi_adj(x))
    theta = 1.0
    rel = np.inf
    hist = []
    it = 0
    for it in range(1, p.max_iter + 1):
        z = xhat - p.lam * np.real(phi_adj(phi(xhat) - y))
        xn, d = dual_fb(z, p.lam * _bound(p.gamma, p.weights), d, psi, psi_adj, p.eta, p.dualfb_iters)
        theta_n = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * theta * theta))
        xhat = xn + ((theta - 1.0) / theta_n) * (xn - x)
        if p.reweight is not None and it == p.reweight[0]:
            p = replace(p, weights=sara_weights(xn, psi_adj, p.reweight[1]))
        dn = float(np.sqrt(np.sum((xn - x) ** 2)))
        nn = float(np.sqrt(np.sum(xn ** 2)))
        rel = dn / nn if nn > 0 else (0.0 if dn == 0 else np.inf)
        hist.append(rel)
        x, theta = xn, theta_n
        if p.rel_tol > 0 and rel < p.rel_tol:
            break
    res = float(np.sqrt(np.sum(np.abs(y - phi(x)) ** 2)))
    return x, {"iters": it, "rel_change": rel, "residual_norm": res, "history": hist}


def fista_objective(x, y, phi, psi_adj, gamma):
    """1/2 ||y - Phi x||^2 + gamma ||Psi^dagger x||_1 (x >= 0 assumed)."""
    return 0.5 * float(np.sum(np.abs(np.asarray(y) - phi(x)) ** 2)) + gamma * float(np.sum(np.abs(psi_adj(x))))


def default_gamma(y, phi_adj, psi_adj, op_norm_sq, factor=1e-3):
    """gamma = factor * max|Psi^dagger Phi^dagger y| / ||Phi||^2 (proposed; gamma does not move the
    constrained minimiser, only the speed of convergence)."""
    return factor * float(np.max(np.abs(psi_adj(np.real(phi_adj(y)))))) / op_norm_sq


def epsilon_from_sigma(sigma, M):
    """eps = sigma sqrt(M + 2 sqrt(M)): mean plus two standard deviations of ||W n||^2 / sigma^2."""
    return float(sigma * np.sqrt(M + 2.0 * np.sqrt(M)))
