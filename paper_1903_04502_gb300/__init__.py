"""GB300-native sparse radio-interferometric imaging (the hot path of arXiv:1903.04502).

A thin Python binding over the C ABI of ``include/gbri.h``: the functions here
only marshal torch tensors (device memory, streams) into the C calls; every
step of the computation runs in the library's CUDA kernels.  The binding
refuses to work when the library is missing: there is no CPU fallback.

Calls (same names as the C entry points without the ``gbri_`` prefix):
``Plan`` (gbri_plan_create), ``phi``, ``phi_adjoint``, ``op_norm``, ``Wavelet``
(gbri_wavelet_create), ``psi``, ``psi_adjoint``, ``prox_l1``, ``proj_l2ball``,
``Solver`` (gbri_solver_*), ``solve``.
"""

import ctypes as C

import torch

from . import _lib
from ._lib import (ALGO_ADMM, ALGO_FISTA, ALGO_PD, F32, F64, PLAN_ORDER, GbriError, SolveParams, SolveReport,  # noqa: F401
                   K_NAMES)

__all__ = ["Plan", "Wavelet", "Solver", "Batch", "phi", "phi_adjoint", "op_norm", "psi", "psi_adjoint", "prox_l1",
           "proj_l2ball", "solve", "vis_reorder", "profile_enable", "profile_read", "launch_count",
           "GbriError", "library"]


def library():
    return _lib.load()


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else C.c_void_p(0)


_REAL = {F32: torch.float32, F64: torch.float64}
_CPLX = {F32: torch.complex64, F64: torch.complex128}


def _precision(p):
    """Precision code from F32 / F64, "f32" / "f64" or a torch dtype."""
    if p in (F32, F64):
        return p
    if p in ("f32", "fp32", torch.float32, torch.complex64):
        return F32
    if p in ("f64", "fp64", torch.float64, torch.complex128):
        return F64
    raise ValueError("precision must be F32 or F64, got %r" % (p,))


def _need(t, dtype, shape=None, name="tensor"):
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))


class Plan:
    """Measurement-operator plan for one problem (gbri_plan_create).

    uvw: float32 CUDA tensor [M, 4] of {u, v, w, weight}.  precision: F32 (float images,
    complex64 visibilities, FP64 global norms) or F64 (double / complex128, FP64 throughout).
    interp_order: 0 takes each tap from the nearest table sample (zeroth order), 1 interpolates
    linearly between the two samples around it with coordinates quantised 256 times finer.
    deterministic: gridding bitwise reproducible from run to run (fixed-order sums of the cells
    that tiles share instead of float atomics; costs a second pass and a slot buffer).
    layout: 0 automatic (the step layout of the fused primal-dual pass for FP32 polynomial-tap
    plans with J = 4, else the run layout), 1 the run layout (faster Phi / Phi^dagger alone).
    """

    def __init__(self, uvw, n_side, oversample=2, J=4, S=4096, beta=0.0, vis_per_run=0, autotune=False,
                 precision=F32, interp_order=0, deterministic=False, layout=0, stream=None):
        lib = _lib.load()
        _need(uvw, torch.float32, name="uvw")
        if uvw.dim() != 2 or uvw.shape[1] != 4:
            raise ValueError("uvw must be [M, 4]")
        self.n_side, self.J, self.S = int(n_side), int(J), int(S)
        self.M = int(uvw.shape[0])
        self.device = uvw.device
        self.precision = _precision(precision)
        self.real_dtype, self.complex_dtype = _REAL[self.precision], _CPLX[self.precision]
        self.interp_order = int(interp_order)
        d = _lib.PlanDesc(self.n_side, int(oversample), self.J, self.S, float(beta), self.M, self.precision,
                          int(vis_per_run), 1 if autotune else 0, self.interp_order, 1 if deterministic else 0,
                          int(layout))
        h = C.c_void_p()
        _lib.check(lib.gbri_plan_create(C.byref(h), C.byref(d), _ptr(uvw), _stream(stream)))
        self._h = h
        K, M, nc, nb = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        _lib.check(lib.gbri_plan_info(h, C.byref(K), C.byref(M), C.byref(nc), C.byref(nb)))
        self.K, self.n_tiles, self.device_bytes = K.value, nc.value, nb.value

    @property
    def handle(self):
        return self._h

    def launch_config(self):
        """(visibilities per run, degridding blocks, gridding blocks) in use (gbri_plan_launch_config)."""
        r, d, g_ = C.c_int32(), C.c_int32(), C.c_int32()
        _lib.check(_lib.load().gbri_plan_launch_config(self._h, C.byref(r), C.byref(d), C.byref(g_)))
        return r.value, d.value, g_.value

    def debug_word(self, reset=True, stream=None):
        """(error bits, first bad index) of a GBRI_DEBUG library build (gbri_plan_debug_word)."""
        b, i = C.c_uint32(), C.c_int64()
        _lib.check(_lib.load().gbri_plan_debug_word(self._h, C.byref(b), C.byref(i), 1 if reset else 0,
                                                    _stream(stream)))
        return b.value, i.value

    def tap_mode(self):
        """0: shared-memory table, 1: first-order table, 2: polynomial taps (gbri_plan_tap_mode)."""
        m = C.c_int32()
        _lib.check(_lib.load().gbri_plan_tap_mode(self._h, C.byref(m)))
        return m.value

    def permutation(self, stream=None):
        out = torch.empty(self.M, dtype=torch.int32, device=self.device)
        _lib.check(_lib.load().gbri_plan_permutation(self._h, _ptr(out), _stream(stream)))
        return out

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().gbri_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def phi(plan, x, y=None, plan_order=False, stream=None):
    """y = Phi x (gbri_phi).  x: real [n_side, n_side]; returns complex [M] (plan precision)."""
    _need(x, plan.real_dtype, (plan.n_side, plan.n_side), "x")
    if y is None:
        y = torch.empty(plan.M, dtype=plan.complex_dtype, device=x.device)
    _need(y, plan.complex_dtype, (plan.M,), "y")
    _lib.check(_lib.load().gbri_phi(plan.handle, _ptr(x), _ptr(y), PLAN_ORDER if plan_order else 0, _stream(stream)))
    return y


def phi_adjoint(plan, y, x=None, plan_order=False, stream=None):
    """x = Phi^dagger y (gbri_phi_adjoint).  y: complex [M]; returns real [n_side, n_side] (plan precision)."""
    _need(y, plan.complex_dtype, (plan.M,), "y")
    if x is None:
        x = torch.empty((plan.n_side, plan.n_side), dtype=plan.real_dtype, device=y.device)
    _need(x, plan.real_dtype, (plan.n_side, plan.n_side), "x")
    _lib.check(_lib.load().gbri_phi_adjoint(plan.handle, _ptr(y), _ptr(x), PLAN_ORDER if plan_order else 0,
                                            _stream(stream)))
    return x


def vis_reorder(plan, vis, to_plan=True, out=None, stream=None):
    """Reorder a complex [M] vector between caller order and plan order (gbri_vis_reorder)."""
    _need(vis, plan.complex_dtype, (plan.M,), "vis")
    if out is None:
        out = torch.empty_like(vis)
    _lib.check(_lib.load().gbri_vis_reorder(plan.handle, _ptr(vis), _ptr(out), 1 if to_plan else 0, _stream(stream)))
    return out


def op_norm(plan, max_iter=200, tol=1e-8, seed=0, stream=None):
    """||Phi||^2 by the power method (gbri_op_norm); returns (value, iterations)."""
    v, it = C.c_double(), C.c_int32()
    _lib.check(_lib.load().gbri_op_norm(plan.handle, int(max_iter), float(tol), int(seed), C.byref(v), C.byref(it),
                                        _stream(stream)))
    return v.value, it.value


class WStack:
    """Non-coplanar measurement operator by w-stacking (gbri_wstack_create): uvw [M, 4] float32
    CUDA tensor with w in wavelengths (third column), pixel_size in direction cosines, n_planes
    equal w bins, each a coplanar plan with the given options."""

    def __init__(self, uvw, n_side, n_planes, pixel_size, oversample=2, J=4, S=4096, beta=0.0,
                 precision=F32, stream=None):
        _need(uvw, torch.float32, name="uvw")
        if uvw.dim() != 2 or uvw.shape[1] != 4:
            raise ValueError("uvw must be [M, 4]")
        self.n_side, self.M = int(n_side), int(uvw.shape[0])
        self.precision = _precision(precision)
        self.real_dtype, self.complex_dtype = _REAL[self.precision], _CPLX[self.precision]
        d = _lib.PlanDesc(self.n_side, int(oversample), int(J), int(S), float(beta), self.M, self.precision, 0, 0, 0, 0)
        h = C.c_void_p()
        _lib.check(_lib.load().gbri_wstack_create(C.byref(h), C.byref(d), _ptr(uvw), int(n_planes), float(pixel_size),
                                                  _stream(stream)))
        self._h = h
        self.n_planes = int(n_planes)

    def info(self):
        """(visibilities per plane, plane centres w_k) as numpy arrays."""
        import numpy as np
        n = C.c_int32()
        counts = np.zeros(self.n_planes, dtype=np.int64)
        centres = np.zeros(self.n_planes, dtype=np.float64)
        _lib.check(_lib.load().gbri_wstack_info(self._h, C.byref(n), C.c_void_p(counts.ctypes.data),
                                                C.c_void_p(centres.ctypes.data)))
        return counts, centres

    def phi(self, x, y=None, stream=None):
        _need(x, self.real_dtype, (self.n_side, self.n_side), "x")
        if y is None:
            y = torch.empty(self.M, dtype=self.complex_dtype, device=x.device)
        _need(y, self.complex_dtype, (self.M,), "y")
        _lib.check(_lib.load().gbri_wstack_phi(self._h, _ptr(x), _ptr(y), _stream(stream)))
        return y

    def phi_adjoint(self, y, x=None, stream=None):
        _need(y, self.complex_dtype, (self.M,), "y")
        if x is None:
            x = torch.empty((self.n_side, self.n_side), dtype=self.real_dtype, device=y.device)
        _need(x, self.real_dtype, (self.n_side, self.n_side), "x")
        _lib.check(_lib.load().gbri_wstack_phi_adjoint(self._h, _ptr(y), _ptr(x), _stream(stream)))
        return x

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().gbri_wstack_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Wavelet:
    """SARA dictionary (gbri_wavelet_create): db_orders with 0 = Dirac, N = dbN; precision F32 or F64."""

    def __init__(self, n_side, levels, db_orders, precision=F32):
        lib = _lib.load()
        self.n_side, self.levels = int(n_side), int(levels)
        self.db_orders = tuple(int(o) for o in db_orders)
        self.n_w = len(self.db_orders)
        self.precision = _precision(precision)
        self.real_dtype = _REAL[self.precision]
        arr = (C.c_int32 * self.n_w)(*self.db_orders)
        h = C.c_void_p()
        _lib.check(lib.gbri_wavelet_create(C.byref(h), self.n_side, self.levels, arr, self.n_w, self.precision))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().gbri_wavelet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def psi(wav, alpha, x=None, stream=None):
    """x = Psi alpha (gbri_psi).  alpha: real [n_w, n, n] (wavelet precision)."""
    _need(alpha, wav.real_dtype, (wav.n_w, wav.n_side, wav.n_side), "alpha")
    if x is None:
        x = torch.empty((wav.n_side, wav.n_side), dtype=wav.real_dtype, device=alpha.device)
    _need(x, wav.real_dtype, (wav.n_side, wav.n_side), "x")
    _lib.check(_lib.load().gbri_psi(wav.handle, _ptr(alpha), _ptr(x), _stream(stream)))
    return x


def psi_adjoint(wav, x, alpha=None, stream=None):
    """alpha = Psi^dagger x (gbri_psi_adjoint)."""
    _need(x, wav.real_dtype, (wav.n_side, wav.n_side), "x")
    if alpha is None:
        alpha = torch.empty((wav.n_w, wav.n_side, wav.n_side), dtype=wav.real_dtype, device=x.device)
    _need(alpha, wav.real_dtype, (wav.n_w, wav.n_side, wav.n_side), "alpha")
    _lib.check(_lib.load().gbri_psi_adjoint(wav.handle, _ptr(x), _ptr(alpha), _stream(stream)))
    return alpha


def prox_l1(x, lam, out=None, stream=None):
    """Soft thresholding (gbri_prox_l1) of a float32 / float64 / complex64 / complex128 CUDA tensor."""
    if x.dtype not in (torch.float32, torch.float64, torch.complex64, torch.complex128):
        raise ValueError("prox_l1 takes float32, float64, complex64 or complex128")
    _need(x, x.dtype, name="x")
    if out is None:
        out = torch.empty_like(x)
    _need(out, x.dtype, tuple(x.shape), "out")
    _lib.check(_lib.load().gbri_prox_l1(_ptr(x), _ptr(out), x.numel(), float(lam), 1 if x.is_complex() else 0,
                                        _precision(x.dtype), _stream(stream)))
    return out


def prox_l1_weighted(x, w, lam, out=None, stream=None):
    """Weighted soft thresholding (gbri_prox_l1_weighted): threshold lam * w elementwise.
    w: real CUDA tensor of x's real precision and x's number of elements."""
    if x.dtype not in (torch.float32, torch.float64, torch.complex64, torch.complex128):
        raise ValueError("prox_l1_weighted takes float32, float64, complex64 or complex128")
    prec = _precision(x.dtype)
    _need(x, x.dtype, name="x")
    _need(w, _REAL[prec], name="w")
    if w.numel() != x.numel():
        raise ValueError("w must have one weight per element of x")
    if out is None:
        out = torch.empty_like(x)
    _need(out, x.dtype, tuple(x.shape), "out")
    _lib.check(_lib.load().gbri_prox_l1_weighted(_ptr(x), _ptr(w), _ptr(out), x.numel(), float(lam),
                                                 1 if x.is_complex() else 0, prec, _stream(stream)))
    return out


def proj_l2ball(z, center, eps, out=None, norm_out=None, stream=None):
    """Projection of complex64 / complex128 z onto the l2 ball of radius eps around center
    (gbri_proj_l2ball).  norm_out: optional float64 CUDA tensor of one element receiving ||z - center||."""
    if z.dtype not in (torch.complex64, torch.complex128):
        raise ValueError("proj_l2ball takes complex64 or complex128")
    _need(z, z.dtype, name="z")
    _need(center, z.dtype, tuple(z.shape), "center")
    if out is None:
        out = torch.empty_like(z)
    _need(out, z.dtype, tuple(z.shape), "out")
    if norm_out is not None:
        _need(norm_out, torch.float64, (1,), "norm_out")
    _lib.check(_lib.load().gbri_proj_l2ball(_ptr(z), _ptr(center), _ptr(out), z.numel(), float(eps),
                                            _ptr(norm_out), _precision(z.dtype), _stream(stream)))
    return out


def proj_l2ball_noalloc(z, center, eps, out, norm_out=None, stream=None):
    """Allocation-free projection onto the l2 ball (gbri_proj_l2ball_noalloc): same result as
    ``proj_l2ball``, with the reduction scratch in a fixed device array inside the library, for
    callers that cannot allocate device memory at that point.  ``out`` is required (it may be
    ``z`` itself): this wrapper allocates nothing, so the caller provides every buffer.
    Concurrent calls race."""
    _need(z, torch.complex64, name="z")
    _need(center, torch.complex64, tuple(z.shape), "center")
    _need(out, torch.complex64, tuple(z.shape), "out")
    if norm_out is not None:
        _need(norm_out, torch.float64, (1,), "norm_out")
    _lib.check(_lib.load().gbri_proj_l2ball_noalloc(_ptr(z), _ptr(center), _ptr(out), z.numel(), float(eps),
                                                    _ptr(norm_out), _stream(stream)))
    return out


def _params(**kw):
    p = SolveParams()
    p.algo = ALGO_PD
    p.max_iter = 200
    p.theta = -1.0
    for k, v in kw.items():
        if not hasattr(p, k):
            raise ValueError("unknown solver parameter %s" % k)
        setattr(p, k, v)
    return p


class Solver:
    """Resident solver state (gbri_solver_create / step / get_x / report)."""

    def __init__(self, plan, wav, y, plan_order=False, stream=None, **params):
        _need(y, plan.complex_dtype, (plan.M,), "y")
        self.plan, self.wav = plan, wav
        self.params = _params(**params)
        h = C.c_void_p()
        _lib.check(_lib.load().gbri_solver_create(C.byref(h), plan.handle, wav.handle, _ptr(y),
                                                  C.byref(self.params), PLAN_ORDER if plan_order else 0,
                                                  _stream(stream)))
        self._h = h

    def step(self, n_iter=1, stream=None):
        _lib.check(_lib.load().gbri_solver_step(self._h, int(n_iter), _stream(stream)))

    def capture(self):
        """Capture the iteration graph now, on this thread (gbri_solver_capture)."""
        _lib.check(_lib.load().gbri_solver_capture(self._h))

    def reweight(self, delta, stream=None):
        """Reweighted l1: w_i = delta / (delta + |(Psi^dagger x)_i|) from the current iterate
        (gbri_solver_reweight)."""
        _lib.check(_lib.load().gbri_solver_reweight(self._h, float(delta), _stream(stream)))

    def x(self, out=None, stream=None):
        if out is None:
            out = torch.empty((self.plan.n_side, self.plan.n_side), dtype=self.plan.real_dtype,
                              device=self.plan.device)
        _need(out, self.plan.real_dtype, (self.plan.n_side, self.plan.n_side), "out")
        _lib.check(_lib.load().gbri_solver_get_x(self._h, _ptr(out), _stream(stream)))
        return out

    def status(self, stream=None):
        """(iterations run, last relative iterate change) -- one scalar read (gbri_solver_status)."""
        it, rel = C.c_int32(), C.c_double()
        _lib.check(_lib.load().gbri_solver_status(self._h, C.byref(it), C.byref(rel), _stream(stream)))
        return it.value, rel.value

    def report(self, stream=None):
        r = SolveReport()
        _lib.check(_lib.load().gbri_solver_report(self._h, C.byref(r), _stream(stream)))
        return {f: getattr(r, f) for f, _ in SolveReport._fields_}

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().gbri_solver_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Resident solvers of independent problems stepped together (gbri_batch_*): every
    iteration of every member is one CUDA-graph launch; members may join and leave
    between steps."""

    def __init__(self):
        h = C.c_void_p()
        _lib.check(_lib.load().gbri_batch_create(C.byref(h)))
        self._h = h
        self.members = []

    def add(self, solver):
        _lib.check(_lib.load().gbri_batch_add(self._h, solver._h))
        self.members.append(solver)

    def remove(self, solver):
        _lib.check(_lib.load().gbri_batch_remove(self._h, solver._h))
        self.members.remove(solver)

    def __len__(self):
        return int(_lib.load().gbri_batch_size(self._h))

    def step(self, n_iter=1, stream=None):
        _lib.check(_lib.load().gbri_batch_step(self._h, int(n_iter), _stream(stream)))

    def set_shared_pass(self, enable):
        """Primal-dual members on FP32 step-layout plans share one fused degridding + gridding
        launch per iteration (default on; gbri_batch_set_shared_pass)."""
        _lib.check(_lib.load().gbri_batch_set_shared_pass(self._h, 1 if enable else 0))

    def shared_members(self):
        """Members in the shared pass at the last step (gbri_batch_shared_members)."""
        return int(_lib.load().gbri_batch_shared_members(self._h))

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().gbri_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(plan, wav, y, x_out=None, plan_order=False, stream=None, **params):
    """One-shot solve (gbri_solve); returns (x, report dict)."""
    _need(y, plan.complex_dtype, (plan.M,), "y")
    if x_out is None:
        x_out = torch.empty((plan.n_side, plan.n_side), dtype=plan.real_dtype, device=y.device)
    p = _params(**params)
    r = SolveReport()
    _lib.check(_lib.load().gbri_solve(plan.handle, wav.handle, _ptr(y), C.byref(p), _ptr(x_out), C.byref(r),
                                      PLAN_ORDER if plan_order else 0, _stream(stream)))
    return x_out, {f: getattr(r, f) for f, _ in SolveReport._fields_}


def profile_enable(capacity):
    _lib.check(_lib.load().gbri_profile_enable(int(capacity)))


def profile_read(kind):
    t, n = C.c_double(), C.c_int64()
    _lib.check(_lib.load().gbri_profile_read(int(kind), C.byref(t), C.byref(n)))
    return t.value, n.value


def inject_alloc_failure(after_n):
    """Make the after_n-th device allocation of the library from now on fail with GBRI_ENOMEM
    (test hook for out-of-memory handling; 0 disarms)."""
    _lib.check(_lib.load().gbri_debug_inject_alloc_failure(int(after_n)))


def launch_count():
    return int(_lib.load().gbri_launch_count())
