"""Thin ctypes binding of libvdwnl.so (C ABI in include/vdwnl.h).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  Device buffers are torch CUDA tensors (FP32,
contiguous, shape (N3, N2, N1) for scalars and (3, N3, N2, N1) for vectors);
work is enqueued on torch's current CUDA stream unless a stream is given.
If the library cannot be loaded every entry point raises: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvdwnl.so")

VDW_OK = 0
ERRORS = {-1: "VDW_ERR_ARG", -2: "VDW_ERR_SIZE", -3: "VDW_ERR_CUDA", -4: "VDW_ERR_OOM",
          -5: "VDW_ERR_STATE", -6: "VDW_ERR_UNSUPPORTED"}


class VdwError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = "%s failed: %s (%d)" % (where, ERRORS.get(code, "?"), code)
        try:
            detail = lib().vdw_last_error().decode()
            if detail:
                msg += ": " + detail
        except Exception:  # pragma: no cover
            pass
        super().__init__(msg)


class _Params(ctypes.Structure):
    _fields_ = [("Nq", ctypes.c_int), ("q_1", ctypes.c_double), ("q_c", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("m_c", ctypes.c_int), ("d_s", ctypes.c_double),
                ("na", ctypes.c_int), ("a_max", ctypes.c_double), ("d_asym", ctypes.c_double),
                ("r_c", ctypes.c_double), ("Nr", ctypes.c_int), ("k_max", ctypes.c_double),
                ("Nk", ctypes.c_int), ("n_cs", ctypes.c_int), ("n_min", ctypes.c_double)]


@dataclass
class Params:
    """Method parameters (same meaning and defaults as vdw_params)."""
    Nq: int = 20
    q_1: float = 1e-5
    q_c: float = 5.0
    lam: float = 1.2
    m_c: int = 12
    d_s: float = 1.0
    na: int = 256
    a_max: float = 64.0
    d_asym: float = 8.0
    r_c: float = 100.0
    Nr: int = 4096
    k_max: float = 40.0
    Nk: int = 1024
    n_cs: int = 64
    n_min: float = 1e-12

    def to_c(self):
        p = _Params()
        for f in fields(self):
            setattr(p, "lambda_" if f.name == "lam" else f.name, getattr(self, f.name))
        return p


EXPORTS = ["vdw_params_default", "vdw_kernel_table", "vdw_create", "vdw_plan", "vdw_energy_potential",
           "vdw_plan_batch", "vdw_plan_cell", "vdw_energy_potential_batched",
           "vdw_energy_potential_fd", "vdw_xc_energy_potential",
           "vdw_energy_potential_host", "vdw_last_invalid_points", "vdw_profile_enable", "vdw_profile_read",
           "vdw_delta_energy_noalloc", "vdw_spectral_gradient", "vdw_learned_param_count", "vdw_learned_load",
           "vdw_learned_energy_potential", "vdw_learned_param_grad", "vdw_learned_fit_grad",
           "vdw_learned_channels", "vdw_learned_status", "vdw_learned_tabulate", "vdw_basis_weights", "vdw_adam_step", "vdw_wait_status",
           "vdw_workspace_bytes", "vdw_destroy", "vdw_error_string", "vdw_last_error"]

LEARNED_M = 8
LEARNED_H = 64

_LIB = None


def lib():
    """Load libvdwnl.so (raises if it is missing: no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libvdwnl.so not built (run paper_0812_0244_gb300.build.build())")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    dp, fp, vp = P(ctypes.c_double), P(ctypes.c_float), ctypes.c_void_p
    L.vdw_params_default.argtypes = [P(_Params)]
    L.vdw_kernel_table.argtypes = [P(_Params), dp, dp, dp, dp]
    L.vdw_create.argtypes = [P(vp), P(_Params), dp, ctypes.c_double]
    L.vdw_plan.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
    L.vdw_energy_potential.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.vdw_energy_potential_host.argtypes = [vp, fp, fp, dp, fp, vp]
    L.vdw_plan_batch.argtypes = [vp, ctypes.c_int]
    L.vdw_plan_cell.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
    L.vdw_energy_potential_batched.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, vp]
    L.vdw_energy_potential_fd.argtypes = [vp, vp, vp, vp, vp, vp]
    L.vdw_xc_energy_potential.argtypes = [vp, vp, vp, vp, vp, ctypes.c_int, vp]
    L.vdw_last_invalid_points.argtypes = [vp, P(ctypes.c_longlong)]
    L.vdw_profile_enable.argtypes = [vp, ctypes.c_int]
    L.vdw_profile_read.argtypes = [vp, fp]
    L.vdw_delta_energy_noalloc.argtypes = [vp, vp, vp, ctypes.c_longlong, ctypes.c_double, vp, vp]
    L.vdw_spectral_gradient.argtypes = [vp, vp, vp, vp]
    L.vdw_learned_param_count.argtypes = [ctypes.c_int]
    L.vdw_learned_load.argtypes = [vp, ctypes.c_int, ctypes.c_double, dp, ctypes.c_double, ctypes.c_double, vp, vp]
    L.vdw_learned_energy_potential.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.vdw_learned_param_grad.argtypes = [vp, vp, vp, ctypes.c_double, vp, vp, vp]
    L.vdw_learned_fit_grad.argtypes = [vp, vp, vp, vp, vp, ctypes.c_double, vp, vp]
    L.vdw_learned_channels.argtypes = [vp, vp, vp, vp, vp]
    L.vdw_learned_status.argtypes = [vp, P(ctypes.c_int)]
    L.vdw_learned_tabulate.argtypes = [vp, ctypes.c_int, ctypes.c_double, vp]
    L.vdw_basis_weights.argtypes = [vp, vp, vp, vp, vp]
    L.vdw_adam_step.argtypes = [vp, vp, vp, vp, ctypes.c_longlong, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_int, vp]
    L.vdw_wait_status.argtypes = [vp, P(ctypes.c_int)]
    L.vdw_workspace_bytes.argtypes = [vp, P(ctypes.c_size_t)]
    L.vdw_destroy.argtypes = [vp]
    L.vdw_error_string.argtypes = [ctypes.c_int]
    L.vdw_error_string.restype = ctypes.c_char_p
    L.vdw_last_error.argtypes = []
    L.vdw_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("vdw_error_string", "vdw_last_error"):
            getattr(L, name).restype = ctypes.c_int
    L.vdw_learned_param_count.restype = ctypes.c_longlong
    _LIB = L
    return L


def _check(rc, where):
    if rc != VDW_OK:
        raise VdwError(rc, where)


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def kernel_table(params: Params | None = None):
    """vdw_kernel_table: q mesh, phi_ab(k) (Nq, Nq, Nk), phi0 and C_s in FP64."""
    params = params or Params()
    qm = np.zeros(params.Nq)
    phik = np.zeros((params.Nq, params.Nq, params.Nk))
    phi0 = np.zeros(1)
    cs = np.zeros(1)
    p = params.to_c()
    _check(lib().vdw_kernel_table(ctypes.byref(p), _dptr(qm), _dptr(phik), _dptr(phi0), _dptr(cs)),
           "vdw_kernel_table")
    return dict(q_mesh=qm, phi_k=phik, phi0=float(phi0[0]), C_s=float(cs[0]))


def learned_param_count(J):
    """Length of the learned model's flat parameter vector for J knots."""
    return int(lib().vdw_learned_param_count(int(J)))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _cuda_f32(t, shape=None):
    import torch
    assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
    if shape is not None:
        assert tuple(t.shape) == tuple(shape), (tuple(t.shape), shape)


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """vdw_adam_step on device tensors: p, m, v FP32, g FP64 (same length)."""
    import torch
    assert p.numel() == g.numel() == m.numel() == v.numel()
    assert g.dtype == torch.float64 and p.dtype == m.dtype == v.dtype == torch.float32
    _check(lib().vdw_adam_step(_ptr(p), _ptr(g), _ptr(m), _ptr(v), p.numel(), float(lr), float(beta1),
                               float(beta2), float(eps), int(step), _stream_handle(stream)), "vdw_adam_step")


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class VdwNL:
    """A vdwnl context: kernel tables, and after plan() a grid and its workspace."""

    def __init__(self, params: Params | None = None, phi_k: np.ndarray | None = None, C_s: float = 0.0):
        self.params = params or Params()
        self._h = ctypes.c_void_p()
        p = self.params.to_c()
        tab = None
        if phi_k is not None:
            tab = np.ascontiguousarray(phi_k, dtype=np.float64)
            assert tab.shape == (self.params.Nq, self.params.Nq, self.params.Nk)
        _check(lib().vdw_create(ctypes.byref(self._h), ctypes.byref(p), _dptr(tab) if tab is not None else None,
                                float(C_s)), "vdw_create")
        self.shape = None

    def plan(self, shape, L):
        """shape = (N3, N2, N1) of the arrays, L = (L1, L2, L3) edge lengths in bohr."""
        N3, N2, N1 = (int(s) for s in shape)
        Lc = np.ascontiguousarray(np.asarray(L, dtype=np.float64).reshape(3))
        _check(lib().vdw_plan(self._h, N1, N2, N3, _dptr(Lc)), "vdw_plan")
        self.shape = (N3, N2, N1)
        self.L = Lc.copy()
        return self

    def plan_cell(self, shape, cell):
        """vdw_plan_cell: shape = (N3, N2, N1), cell = 3 x 3 lattice vectors
        (rows, bohr) along the grid axes N1, N2, N3; orthorhombic only."""
        N3, N2, N1 = (int(s) for s in shape)
        cc = np.ascontiguousarray(np.asarray(cell, dtype=np.float64).reshape(9))
        _check(lib().vdw_plan_cell(self._h, N1, N2, N3, _dptr(cc)), "vdw_plan_cell")
        self.shape = (N3, N2, N1)
        self.L = np.array([cc[0], cc[4], cc[8]])
        return self

    @property
    def dOmega(self):
        return float(np.prod(self.L)) / float(np.prod(self.shape))

    def energy_potential(self, n, grad, E=None, v=None, w=None, stream=None):
        """Enqueue vdw_energy_potential on device tensors; returns (E, v, w)."""
        import torch
        assert n.is_cuda and n.dtype == torch.float32 and n.is_contiguous() and tuple(n.shape) == self.shape
        if grad is not None:  # None: the library computes the spectral gradient
            assert grad.is_cuda and grad.dtype == torch.float32 and grad.is_contiguous()
            assert tuple(grad.shape) == (3,) + self.shape
        for t, shp in ((v, self.shape), (w, (3,) + self.shape)):
            if t is not None:
                assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and tuple(t.shape) == shp
        if E is not None:
            assert E.is_cuda and E.dtype == torch.float64 and E.numel() >= 3
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        _check(lib().vdw_energy_potential(self._h, ptr(n), ptr(grad), ptr(E), ptr(v), ptr(w),
                                          _stream_handle(stream)), "vdw_energy_potential")
        return E, v, w

    def plan_batch(self, Bmax):
        """vdw_plan_batch: workspaces for Bmax densities per call (after plan())."""
        _check(lib().vdw_plan_batch(self._h, int(Bmax)), "vdw_plan_batch")
        self.batch_max = int(Bmax)
        return self

    def energy_potential_batched(self, n, grad, E=None, v=None, stream=None):
        """vdw_energy_potential_batched on device tensors n (B, N3, N2, N1),
        grad (B, 3, N3, N2, N1); returns (E (B, 3) float64, v (B, ...) or None)."""
        import torch
        B = int(n.shape[0])
        _cuda_f32(n, (B,) + self.shape)
        _cuda_f32(grad, (B, 3) + self.shape)
        if E is None:
            E = torch.empty((B, 3), dtype=torch.float64, device=n.device)
        assert E.is_cuda and E.dtype == torch.float64 and E.is_contiguous() and E.numel() >= 3 * B
        if v is not None:
            _cuda_f32(v, (B,) + self.shape)
        _check(lib().vdw_energy_potential_batched(self._h, B, _ptr(n), _ptr(grad), _ptr(E), _ptr(v),
                                                  _stream_handle(stream)), "vdw_energy_potential_batched")
        return E, v

    def energy_potential_fd(self, n, grad=None, E=None, v=None, stream=None):
        """vdw_energy_potential_fd: central-difference gradient (given, or
        computed by the library when grad is None); returns (E, v)."""
        import torch
        _cuda_f32(n, self.shape)
        if grad is not None:
            _cuda_f32(grad, (3,) + self.shape)
        if E is None:
            E = torch.empty(3, dtype=torch.float64, device=n.device)
        if v is not None:
            _cuda_f32(v, self.shape)
        _check(lib().vdw_energy_potential_fd(self._h, _ptr(n), _ptr(grad), _ptr(E), _ptr(v), _stream_handle(stream)),
               "vdw_energy_potential_fd")
        return E, v

    def xc_energy_potential(self, n, grad=None, v=None, fd=False, stream=None):
        """vdw_xc_energy_potential: E_xc of Eq. (Exc) and its potential;
        returns (E[4] = {E_xc, E_c^nl, E_x, E_c^LDA}, v)."""
        import torch
        _cuda_f32(n, self.shape)
        if grad is not None:
            _cuda_f32(grad, (3,) + self.shape)
        if v is not None:
            _cuda_f32(v, self.shape)
        E = torch.empty(4, dtype=torch.float64, device=n.device)
        _check(lib().vdw_xc_energy_potential(self._h, _ptr(n), _ptr(grad), _ptr(E), _ptr(v), 1 if fd else 0,
                                             _stream_handle(stream)), "vdw_xc_energy_potential")
        return E, v

    def compute(self, n, grad, want_v=True, want_w=False, stream=None):
        """Allocate outputs and run; returns (E[3] float64 device tensor, v, w)."""
        import torch
        E = torch.empty(3, dtype=torch.float64, device=n.device)
        v = torch.empty_like(n) if want_v else None
        w = torch.empty((3,) + tuple(n.shape), dtype=torch.float32, device=n.device) if want_w else None
        return self.energy_potential(n, grad, E, v, w, stream)

    # ---- spectral gradient and the learned reduced basis -----------------
    def spectral_gradient(self, f, out=None, stream=None):
        """grad f = D f (spectral, Nyquist removed) into out (3, N3, N2, N1)."""
        import torch
        _cuda_f32(f, self.shape)
        if out is None:
            out = torch.empty((3,) + self.shape, dtype=torch.float32, device=f.device)
        _cuda_f32(out, (3,) + self.shape)
        _check(lib().vdw_spectral_gradient(self._h, _ptr(f), _ptr(out), _stream_handle(stream)),
               "vdw_spectral_gradient")
        return out

    def learned_load(self, params, J, k_max, feat, base=(0.0, 0.0), stream=None):
        """vdw_learned_load: params a device FP32 tensor of learned_param_count(J)
        values, feat = (mu1, sig1, mu2, sig2, eps), base = (q_1, lambda) of the
        optional spline base mesh ((0, 0): none)."""
        _cuda_f32(params)
        assert params.numel() == learned_param_count(J)
        f = np.ascontiguousarray(np.asarray(feat, dtype=np.float64).reshape(5))
        self._lrn_params = params  # keep alive until the prepare kernel ran
        _check(lib().vdw_learned_load(self._h, int(J), float(k_max), _dptr(f), float(base[0]), float(base[1]),
                                      _ptr(params), _stream_handle(stream)), "vdw_learned_load")

    def learned_tabulate(self, T, D, stream=None):
        """vdw_learned_tabulate: the loaded network on (T+2)^2 feature nodes over
        [-D, D]^2 for inference (T = 0: evaluate the network at every point)."""
        _check(lib().vdw_learned_tabulate(self._h, int(T), float(D), _stream_handle(stream)),
               "vdw_learned_tabulate")

    def learned_energy_potential(self, n, grad, E=None, v=None, w=None, stream=None):
        _cuda_f32(n, self.shape)
        _cuda_f32(grad, (3,) + self.shape)
        _check(lib().vdw_learned_energy_potential(self._h, _ptr(n), _ptr(grad), _ptr(E), _ptr(v), _ptr(w),
                                                  _stream_handle(stream)), "vdw_learned_energy_potential")
        return E, v, w

    def learned_compute(self, n, grad, want_v=True, want_w=False, stream=None):
        import torch
        E = torch.empty(3, dtype=torch.float64, device=n.device)
        v = torch.empty_like(n) if want_v else None
        w = torch.empty_like(grad) if want_w else None
        return self.learned_energy_potential(n, grad, E, v, w, stream)

    def learned_param_grad(self, n, grad, g_params, coef=1.0, E=None, stream=None):
        """g_params (FP64 device) += coef dE/dparams; E (FP64 [3]) optional."""
        import torch
        _cuda_f32(n, self.shape)
        _cuda_f32(grad, (3,) + self.shape)
        assert g_params.is_cuda and g_params.dtype == torch.float64
        _check(lib().vdw_learned_param_grad(self._h, _ptr(n), _ptr(grad), float(coef), _ptr(g_params), _ptr(E),
                                            _stream_handle(stream)), "vdw_learned_param_grad")
        return g_params

    def learned_fit_grad(self, n, grad, target, weight, g_params, coef=1.0, stream=None):
        import torch
        _cuda_f32(n, self.shape)
        _cuda_f32(grad, (3,) + self.shape)
        _cuda_f32(target, (LEARNED_M,) + self.shape)
        _cuda_f32(weight, self.shape)
        assert g_params.is_cuda and g_params.dtype == torch.float64
        _check(lib().vdw_learned_fit_grad(self._h, _ptr(n), _ptr(grad), _ptr(target), _ptr(weight), float(coef),
                                          _ptr(g_params), _stream_handle(stream)), "vdw_learned_fit_grad")
        return g_params

    def learned_channels(self, n, grad, out=None, stream=None):
        import torch
        _cuda_f32(n, self.shape)
        _cuda_f32(grad, (3,) + self.shape)
        if out is None:
            out = torch.empty((LEARNED_M,) + self.shape, dtype=torch.float32, device=n.device)
        _check(lib().vdw_learned_channels(self._h, _ptr(n), _ptr(grad), _ptr(out), _stream_handle(stream)),
               "vdw_learned_channels")
        return out

    def learned_status(self):
        e = ctypes.c_int()
        _check(lib().vdw_learned_status(self._h, ctypes.byref(e)), "vdw_learned_status")
        return e.value

    def basis_weights(self, n, grad, out=None, stream=None):
        """Plain cardinal weights p_a(q) (Nq, N3, N2, N1) for this context's mesh."""
        import torch
        _cuda_f32(n, self.shape)
        _cuda_f32(grad, (3,) + self.shape)
        if out is None:
            out = torch.empty((self.params.Nq,) + self.shape, dtype=torch.float32, device=n.device)
        _check(lib().vdw_basis_weights(self._h, _ptr(n), _ptr(grad), _ptr(out), _stream_handle(stream)),
               "vdw_basis_weights")
        return out

    def energy_potential_host(self, n, grad, E=None, v=None, stream=None):
        """vdw_energy_potential_host on numpy float32 arrays (pinned or pageable)."""
        n = np.ascontiguousarray(n, dtype=np.float32)
        grad = np.ascontiguousarray(grad, dtype=np.float32)
        if E is None:
            E = np.zeros(3)
        if v is None:
            v = np.empty(self.shape, dtype=np.float32)
        fp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        _check(lib().vdw_energy_potential_host(self._h, fp(n), fp(grad), _dptr(E), fp(v), _stream_handle(stream)),
               "vdw_energy_potential_host")
        return E, v

    def invalid_points(self):
        c = ctypes.c_longlong()
        _check(lib().vdw_last_invalid_points(self._h, ctypes.byref(c)), "vdw_last_invalid_points")
        return c.value

    def delta_energy_noalloc(self, n, grad, dE, dOmega=None, stream=None):
        """vdw_delta_energy_noalloc: Delta E into the FP64 device tensor dE[0]
        with no device allocation (for callers that must not allocate)."""
        import torch
        assert n.is_cuda and n.dtype == torch.float32 and n.is_contiguous()
        assert grad.is_cuda and grad.dtype == torch.float32 and grad.is_contiguous()
        assert grad.numel() == 3 * n.numel()
        assert dE.is_cuda and dE.dtype == torch.float64 and dE.numel() >= 1
        if dOmega is None:
            dOmega = self.dOmega
        _check(lib().vdw_delta_energy_noalloc(self._h, ctypes.c_void_p(n.data_ptr()), ctypes.c_void_p(grad.data_ptr()),
                                              n.numel(), float(dOmega), ctypes.c_void_p(dE.data_ptr()),
                                              _stream_handle(stream)), "vdw_delta_energy_noalloc")
        return dE

    STAGES = ("pointwise", "planes_fwd", "pencils_fwd", "contract", "energy_final", "pencils_inv", "planes_inv",
              "usum", "w_planes", "pencil_div", "div_final")

    def profile(self, enable=True):
        _check(lib().vdw_profile_enable(self._h, 1 if enable else 0), "vdw_profile_enable")

    def profile_read(self):
        """Stage durations (ms) of the last call, as a dict (skipped stages omitted)."""
        ms = (ctypes.c_float * len(self.STAGES))()
        _check(lib().vdw_profile_read(self._h, ms), "vdw_profile_read")
        return {name: float(t) for name, t in zip(self.STAGES, ms) if t >= 0}

    def wait_status(self):
        """1 if a bounded wait inside a kernel gave up since plan(), else 0."""
        e = ctypes.c_int()
        _check(lib().vdw_wait_status(self._h, ctypes.byref(e)), "vdw_wait_status")
        return e.value

    def workspace_bytes(self):
        b = ctypes.c_size_t()
        _check(lib().vdw_workspace_bytes(self._h, ctypes.byref(b)), "vdw_workspace_bytes")
        return b.value

    def close(self):
        if self._h:
            lib().vdw_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
