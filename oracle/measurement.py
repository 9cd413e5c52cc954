"""Measurement operator Phi = W G F Z S and its adjoint (oracle, FP64).  Test infrastructure only.

Follows Sec. 2: Eq. 2 factorises the non-uniform FFT as y = W G F Z S x and the
adjoint applies the factors in reverse, Phi^dagger = S^dagger Z^dagger F^dagger
G^dagger W^dagger.  The measurement equation itself (Eq. 1) is written out as a
brute-force non-uniform DFT in ``nudft`` and pins this module.

Readings (the paper is silent on these details):

* R1 centring / axes: image pixel (row q, column p) sits at centred coordinates
  (p', q') = (p - n_side/2, q - n_side/2).  u pairs with columns (p'), v with
  rows (q').  The DFT sign is negative, as in Eq. 1.
* R2 normalisation: F is the unnormalised forward DFT on the K x K grid
  (K = oversample * n_side); F^dagger is the unnormalised inverse.  Then Phi
  approximates y_i = w_i sum x[q,p] exp(-i (u_i p' + v_i q')) with no hidden
  constant.
* u, v are in radians per image pixel, |u|, |v| <= pi (Sec. 7.3).  The grid
  coordinate is k = u K / (2 pi).
* R4 quantisation (table mode): k~ = round_half_away(u * (K S) / (2 pi)) is
  computed once in FP64 as ``float64(u) * (float64(K*S) / (2*pi))``; taps are the
  J cells j = floor(k~/S) - J/2 + 1 .. floor(k~/S) + J/2 and each takes
  table[|k~ - j S|] (exact nearest-sample zeroth-order interpolation, Sec. 8.1).
  Grid cell j lives at column (or row) j mod K.
* R5 weights: W is a real diagonal; x is real (Sec. 2) so the real adjoint takes
  Re(.) after S^dagger Z^dagger F^dagger.
* R13 first-order table mode ("linear"; Sec. 8.1 names zeroth- and first-order
  interpolation of the pre-sampled kernel and uses zeroth order): the coordinate is
  quantised F times finer than the table step, q = round_half_away(u K S F / 2 pi)
  (FP64, as in R4 with S F in place of S); the taps are the J cells around
  floor(q / (S F)), and a tap at table position d = |q - j S F| / F takes
  table[floor d] + frac(d) (table[floor d + 1] - table[floor d]) (0 beyond the support).
"""

import os

import numpy as np
import scipy.fft

from . import kb


def _workers():
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# Coordinates and interpolation weights (G)
# ---------------------------------------------------------------------------

def quantise(u, K, S):
    """Fixed-point grid coordinate k~ = round_half_away(u K S / 2pi) as int64 (reading R4)."""
    scale = np.float64(K * S) / (2.0 * np.pi)
    prod = np.asarray(u, dtype=np.float64) * scale
    return (np.sign(prod) * np.floor(np.abs(prod) + 0.5)).astype(np.int64)


def tap_weights_table(u, K, J, S, tab):
    """Cells (M, J) and weights (M, J) of G along one axis, table mode (Sec. 8.1, R4)."""
    kq = quantise(u, K, S)
    base = np.floor_divide(kq, S)
    t = np.arange(J, dtype=np.int64)
    cells = base[:, None] - (J // 2) + 1 + t[None, :]
    dist = np.abs(kq[:, None] - cells * S)
    w = np.where(dist <= (J // 2) * S, tab[np.minimum(dist, len(tab) - 1)], 0.0)
    return np.mod(cells, K), w


def tap_weights_linear(u, K, J, S, tab, F):
    """Cells and weights of G along one axis, first-order table mode (reading R13)."""
    SF = int(S) * int(F)
    kq = quantise(u, K, SF)
    base = np.floor_divide(kq, SF)
    t = np.arange(J, dtype=np.int64)
    cells = base[:, None] - (J // 2) + 1 + t[None, :]
    dist = np.abs(kq[:, None] - cells * SF)  # table position times F
    i = dist // F
    phi = (dist - i * F) / float(F)
    n = len(tab)
    t0 = np.where(i < n, tab[np.minimum(i, n - 1)], 0.0)
    t1 = np.where(i + 1 < n, tab[np.minimum(i + 1, n - 1)], 0.0)
    return np.mod(cells, K), t0 + phi * (t1 - t0)


def tap_weights_exact(u, K, J, beta):
    """Cells and weights of G along one axis with the kernel evaluated exactly (no table)."""
    k = np.asarray(u, dtype=np.float64) * K / (2.0 * np.pi)
    base = np.floor(k).astype(np.int64)
    t = np.arange(J, dtype=np.int64)
    cells = base[:, None] - (J // 2) + 1 + t[None, :]
    w = kb.kernel(k[:, None] - cells, J, beta)
    return np.mod(cells, K), w


class Geometry:
    """Everything Phi needs besides the image: grid size, kernel, coordinates, weights."""

    def __init__(self, uvw, n_side, oversample=2, J=4, S=4096, beta=None, mode="table", F=256):
        uvw = np.asarray(uvw)
        self.n_side = int(n_side)
        self.K = int(oversample) * self.n_side
        self.J = int(J)
        self.S = int(S)
        self.beta = kb.default_beta(J) if beta is None or beta <= 0 else float(beta)
        self.mode = mode
        self.u = uvw[:, 0]
        self.v = uvw[:, 1]
        self.weight = np.asarray(uvw[:, 3], dtype=np.float64)
        self.M = uvw.shape[0]
        self.corr = kb.correction_1d(self.n_side, self.K, self.J, self.beta)
        if mode == "table":
            tab = kb.table(self.J, self.S, self.beta)
            self.cols, self.gx = tap_weights_table(self.u, self.K, self.J, self.S, tab)
            self.rows, self.gy = tap_weights_table(self.v, self.K, self.J, self.S, tab)
        elif mode == "linear":
            tab = kb.table(self.J, self.S, self.beta)
            self.cols, self.gx = tap_weights_linear(self.u, self.K, self.J, self.S, tab, F)
            self.rows, self.gy = tap_weights_linear(self.v, self.K, self.J, self.S, tab, F)
        elif mode == "exact":
            self.cols, self.gx = tap_weights_exact(self.u, self.K, self.J, self.beta)
            self.rows, self.gy = tap_weights_exact(self.v, self.K, self.J, self.beta)
        else:
            raise ValueError(mode)

    def subset(self, idx):
        """Geometry restricted to visibilities ``idx`` (same grid and kernel)."""
        g = object.__new__(Geometry)
        g.__dict__.update(self.__dict__)
        for name in ("u", "v", "weight", "cols", "gx", "rows", "gy"):
            setattr(g, name, getattr(self, name)[idx])
        g.M = len(g.weight)
        return g


# ---------------------------------------------------------------------------
# The factors of Eq. 2
# ---------------------------------------------------------------------------

def _wrapped_index(n_side, K):
    return np.mod(np.arange(n_side) - n_side // 2, K)


def apply_ZS(x, geo):
    """Z S x: divide by ghat along both axes and embed into the K x K grid at (q' mod K, p' mod K)."""
    x = np.asarray(x)
    P = np.zeros((geo.K, geo.K), dtype=np.complex128)
    idx = _wrapped_index(geo.n_side, geo.K)
    P[np.ix_(idx, idx)] = x * geo.corr[:, None] * geo.corr[None, :]
    return P


def apply_F(P):
    """Unnormalised forward 2-D DFT, sign exp(-2 pi i (b p' + a q') / K) (R2)."""
    return scipy.fft.fft2(P, workers=_workers())


def apply_WG(Xhat, geo, chunk=1 << 20):
    """y_i = w_i sum_{t,t'} gx[i,t] gy[i,t'] Xhat[rows[i,t'], cols[i,t]]."""
    y = np.empty(geo.M, dtype=np.complex128)
    for s in range(0, geo.M, chunk):
        e = min(geo.M, s + chunk)
        acc = np.zeros(e - s, dtype=np.complex128)
        for tp in range(geo.J):
            rowvals = Xhat[geo.rows[s:e, tp][:, None], geo.cols[s:e]]  # (m, J)
            acc += geo.gy[s:e, tp] * np.sum(geo.gx[s:e] * rowvals, axis=1)
        y[s:e] = geo.weight[s:e] * acc
    return y


def apply_GtWt(y, geo, chunk=1 << 19):
    """H = G^dagger W^dagger y: each visibility adds w_i g g y_i to its J x J cells."""
    K = geo.K
    re = np.zeros(K * K, dtype=np.float64)
    im = np.zeros(K * K, dtype=np.float64)
    y = np.asarray(y, dtype=np.complex128)
    for s in range(0, geo.M, chunk):
        e = min(geo.M, s + chunk)
        wy = geo.weight[s:e] * y[s:e]
        for tp in range(geo.J):
            for t in range(geo.J):
                flat = geo.rows[s:e, tp] * K + geo.cols[s:e, t]
                c = wy * geo.gx[s:e, t] * geo.gy[s:e, tp]
                re += np.bincount(flat, weights=c.real, minlength=K * K)
                im += np.bincount(flat, weights=c.imag, minlength=K * K)
    return (re + 1j * im).reshape(K, K)


def apply_Ft(H):
    """Unnormalised inverse 2-D DFT (the adjoint of ``apply_F``)."""
    return scipy.fft.ifft2(H, norm="forward", workers=_workers())


def apply_StZt(G, geo, real=True):
    """S^dagger Z^dagger: crop the centred n_side x n_side block and multiply by the correction."""
    idx = _wrapped_index(geo.n_side, geo.K)
    img = G[np.ix_(idx, idx)] * geo.corr[:, None] * geo.corr[None, :]
    return img.real.copy() if real else img


def phi(x, geo):
    """Phi x = W G F Z S x (Eq. 2)."""
    return apply_WG(apply_F(apply_ZS(x, geo)), geo)


def phi_adjoint(y, geo, real=True):
    """Phi^dagger y = S^dagger Z^dagger F^dagger G^dagger W^dagger y; real part for a real image (R5)."""
    return apply_StZt(apply_Ft(apply_GtWt(y, geo)), geo, real=real)


def phi_at(x, geo, idx):
    """(Phi x)_i for a sample of visibilities ``idx``, computed one by one after one FFT."""
    return apply_WG(apply_F(apply_ZS(x, geo)), geo.subset(idx))


def nudft(x, uvw):
    """Brute-force discretised measurement equation (Eq. 1, no primary beam):
    y_i = w_i sum_{q,p} x[q,p] exp(-i (u_i p' + v_i q'))."""
    x = np.asarray(x)
    n = x.shape[0]
    c = np.arange(n, dtype=np.float64) - n // 2
    u = np.asarray(uvw[:, 0], dtype=np.float64)
    v = np.asarray(uvw[:, 1], dtype=np.float64)
    w = np.asarray(uvw[:, 3], dtype=np.float64)
    eu = np.exp(-1j * u[:, None] * c[None, :])  # (M, n) over p'
    ev = np.exp(-1j * v[:, None] * c[None, :])  # (M, n) over q'
    return w * np.einsum("mq,qp,mp->m", ev, x, eu)
