"""Non-coplanar measurement operator by w-stacking (oracle, FP64).  Test infrastructure only.

The paper's measurement equation (Eq. 1) is the coplanar one; it names w-projection and
w-stacking as the wide-field methods of its software and defers their description to the
wide-field paper it cites (Sec. 7.1, Sec. 6.7).  Reading R14, the standard non-coplanar
discretisation written out here:

    y_i = w_i sum_{q,p} x[q,p] exp(-i (u_i p' + v_i q')) exp(-2 pi i w_i (n(p', q') - 1)),
    n(p', q') = sqrt(1 - l^2 - m^2),  l = p' delta,  m = q' delta,

with u, v in radians per pixel as for Eq. 1 (u = 2 pi u_lambda delta), w in wavelengths,
delta the pixel size in direction cosines, and the primary-beam / 1/n factor of the sky
absorbed into x.

w-stacking: the w range [w_lo, w_hi] is cut into n_planes equal bins, plane k centred at
w_k = w_lo + (k + 1/2) dw, dw = (w_hi - w_lo) / n_planes; visibility i goes to plane
k(i) = min(n_planes - 1, floor((w_i - w_lo) / dw)) (one plane when w_hi = w_lo) and its w is
replaced by w_k.  With C_k = exp(-2 pi i w_k (n - 1)) the operator is

    (Phi x)_{i in plane k} = (Phi_k (C_k x))_i,   Phi^dagger y = Re sum_k conj(C_k) Phi_k^{dagger} y_k,

Phi_k the coplanar operator of Eq. 2 over plane k's visibilities (``measurement.phi`` on a
complex image, and its adjoint before the real part).  The w quantisation changes the phase
of visibility i by at most 2 pi (dw / 2) max|n - 1|.
"""

import numpy as np

from . import measurement as me


def n_minus_1(n_side, delta):
    """n(l, m) - 1 on the image grid, l = p' delta (columns), m = q' delta (rows)."""
    c = (np.arange(n_side, dtype=np.float64) - n_side // 2) * float(delta)
    l2 = c[None, :] ** 2
    m2 = c[:, None] ** 2
    r2 = l2 + m2
    if np.any(r2 >= 1.0):
        raise ValueError("field of view beyond the horizon: (n_side / 2 delta)^2 * 2 must be < 1")
    return np.sqrt(1.0 - r2) - 1.0


def screen(n_side, delta, w):
    """C = exp(-2 pi i w (n - 1)) on the image grid."""
    return np.exp(-2j * np.pi * float(w) * n_minus_1(n_side, delta))


def nudft_w(x, uvw, delta):
    """Brute-force non-coplanar measurement equation (reading R14)."""
    x = np.asarray(x)
    n = x.shape[0]
    c = np.arange(n, dtype=np.float64) - n // 2
    u, v, w, wt = (np.asarray(uvw[:, k], dtype=np.float64) for k in range(4))
    nm1 = n_minus_1(n, delta)
    eu = np.exp(-1j * u[:, None] * c[None, :])
    ev = np.exp(-1j * v[:, None] * c[None, :])
    out = np.empty(len(u), dtype=np.complex128)
    for i in range(len(u)):
        out[i] = np.sum(ev[i][:, None] * eu[i][None, :] * x * np.exp(-2j * np.pi * w[i] * nm1))
    return wt * out


def plane_index(w, n_planes, w_lo=None, w_hi=None):
    """Plane of every visibility and the plane centres (see the module text)."""
    w = np.asarray(w, dtype=np.float64)
    lo = float(np.min(w)) if w_lo is None else float(w_lo)
    hi = float(np.max(w)) if w_hi is None else float(w_hi)
    n_planes = int(n_planes)
    if len(w) == 0 or hi <= lo:
        return np.zeros(len(w), dtype=np.int64), np.full(n_planes, lo)
    dw = (hi - lo) / n_planes
    k = np.minimum(n_planes - 1, np.floor((w - lo) / dw).astype(np.int64))
    centres = lo + (np.arange(n_planes) + 0.5) * dw
    return k, centres


class WStack:
    """Per-plane coplanar geometries and screens of a non-coplanar problem."""

    def __init__(self, uvw, n_side, delta, n_planes, oversample=2, J=4, S=4096, mode="table", w_lo=None,
                 w_hi=None):
        uvw = np.asarray(uvw)
        self.n_side, self.delta, self.n_planes = int(n_side), float(delta), int(n_planes)
        self.M = uvw.shape[0]
        self.plane, self.centres = plane_index(uvw[:, 2], self.n_planes, w_lo, w_hi)
        self.idx = [np.nonzero(self.plane == k)[0] for k in range(self.n_planes)]
        self.geo = [me.Geometry(uvw[ix], n_side, oversample, J, S, mode=mode) for ix in self.idx]
        self.screens = [screen(self.n_side, self.delta, wk) for wk in self.centres]


def phi(x, ws):
    """Phi x by w-stacking."""
    y = np.zeros(ws.M, dtype=np.complex128)
    for ix, geo, C in zip(ws.idx, ws.geo, ws.screens):
        if len(ix):
            y[ix] = me.phi(C * x, geo)
    return y


def phi_adjoint(y, ws):
    """Phi^dagger y by w-stacking (real image)."""
    y = np.asarray(y, dtype=np.complex128)
    x = np.zeros((ws.n_side, ws.n_side))
    for ix, geo, C in zip(ws.idx, ws.geo, ws.screens):
        if len(ix):
            x += np.real(np.conj(C) * me.phi_adjoint(y[ix], geo, real=False))
    return x
