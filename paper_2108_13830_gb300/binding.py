"""ctypes binding of libvmc (include/vmc.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; this module turns
torch tensors into device pointers and the caller's current CUDA stream,
allocates outputs with torch, and raises VMCError on a negative status.
There is no fallback: if libvmc.so is missing, loading raises.
"""
from __future__ import annotations

import ctypes as ct
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvmc.so")

VMC_OK, VMC_ERR_ARG, VMC_ERR_CUDA, VMC_ERR_NONFINITE, VMC_ERR_TIMEOUT, VMC_ERR_STATE, VMC_ERR_UNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6
VMC_FP64, VMC_FP32, VMC_BF16, VMC_FP16 = 0, 1, 2, 3
PRECISIONS = {"fp64": VMC_FP64, "fp32": VMC_FP32, "bf16": VMC_BF16, "fp16": VMC_FP16}
ERR_NAMES = {-1: "VMC_ERR_ARG", -2: "VMC_ERR_CUDA", -3: "VMC_ERR_NONFINITE", -4: "VMC_ERR_TIMEOUT",
             -5: "VMC_ERR_STATE", -6: "VMC_ERR_UNSUPPORTED"}


class VMCError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class vmc_arch(ct.Structure):
    _fields_ = [("n_layers_cc", ct.c_int), ("channels", ct.c_int), ("precision", ct.c_int),
                ("marshall_sign", ct.c_int)]


class vmc_tiles(ct.Structure):
    _fields_ = [("slab_configs", ct.c_int), ("slabs", ct.c_int), ("ctas_per_sm", ct.c_int), ("lane_cells", ct.c_int)]


_lib = None
_P, _I, _I64, _D = ct.c_void_p, ct.c_int, ct.c_int64, ct.c_double

_SIGS = {
    "vmc_create": (_I, [_I, _D, _D, ct.POINTER(vmc_arch), ct.POINTER(_P)]),
    "vmc_destroy": (None, [_P]),
    "vmc_num_params": (_I, [_P, ct.POINTER(_I64)]),
    "vmc_set_params": (_I, [_P, _P, _I, _P]),
    "vmc_get_params": (_I, [_P, _P, _P]),
    "vmc_logpsi": (_I, [_P, _P, _I64, _P, _P, _P]),
    "vmc_local_energy": (_I, [_P, _P, _I64, _P, _P, _P]),
    "vmc_local_energy_ragged": (_I, [_P, _P, _P, _P, _I64, _I, _P, _P, _P]),
    "vmc_log_derivs": (_I, [_P, _P, _I64, _P, _I, _P]),
    "vmc_metropolis": (_I, [_P, _P, _P, _I64, _P, _I, _I, _P, _P]),
    "vmc_logpsi_sym": (_I, [_P, _P, _I64, _P, _P, _P]),
    "vmc_local_energy_sym": (_I, [_P, _P, _I64, _P, _P, _P]),
    "vmc_log_derivs_sym": (_I, [_P, _P, _I64, _P, _I, _P]),
    "vmc_sr_moments": (_I, [_P, _P, _P, _I64, _P, _P, _P, _P]),
    "vmc_sr_matvec": (_I, [_P, _P, _I64, _P, _P, _D, _P, _P]),
    "vmc_ot_vec": (_I, [_P, _P, _I64, _P, _P, _P]),
    "vmc_ot_vec_noalloc": (_I, [_P, _I64, _I64, _P, _P, _P]),
    "vmc_sr_solve": (_I, [_P, _P, _P, _I64, _D, _I, _P, ct.POINTER(_D), _P]),
    "vmc_sr_update": (_I, [_P, _P, _D, _P]),
    "vmc_sync_status": (_I, [_P, _P, ct.POINTER(_I64)]),
    "vmc_set_wait_budget": (_I, [_P, _I64]),
    "vmc_set_light_cone": (_I, [_P, _I]),
    "vmc_set_sr_fused": (_I, [_P, _I]),
    "vmc_sr_solve_dense": (_I, [_P, _P, _P, _I64, _D, _P, _P, _P]),
    "vmc_set_cone_tiles": (_I, [_P, _P]),
    "vmc_get_cone_tiles": (_I, [_P, _P]),
    "vmc_set_launch_timing": (_I, [_P, _I]),
    "vmc_launch_timings": (_I, [_P, _I, _P, _P]),
    "vmc_launch_timing_name": (ct.c_char_p, [_P, _I]),
    "vmc_light_cone_active": (_I, [_P, _P]),
    "vmc_debug_wait_timeout": (_I, [_P, _I64, _P]),
    "vmc_set_tiles": (_I, [_P, _I, ct.POINTER(vmc_tiles)]),
    "vmc_get_tiles": (_I, [_P, _I, ct.POINTER(vmc_tiles)]),
    "vmc_autotune": (_I, [_P, _I, _I64, _P]),
    "vmc_last_launch_count": (_I64, [_P]),
    "vmc_last_error": (ct.c_char_p, [_P]),
    "vmc_debug_umma_selftest": (_I, [_P, _P, _P, _I, _I, _I, _I, _P]),
    "vmc_debug_umma_rate": (_I, [_I, _I, _I, ct.POINTER(_D), ct.POINTER(_D)]),
}


def lib():
    """Load libvmc.so (built by paper_2108_13830_gb300/build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run paper_2108_13830_gb300/build.py "
                               "(or __graft_entry__.build()); there is no fallback path")
        L = ct.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(t):
    return ct.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    return ct.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return t.contiguous()


class VMC:
    """One libvmc context: lattice side L, couplings, network (C, D), precision."""

    def __init__(self, L, J1=1.0, J2=0.5, C=32, D=8, precision="bf16", marshall=True):
        self._h = None
        self.L, self.J1, self.J2, self.C, self.D = L, J1, J2, C, D
        self.precision = precision
        arch = vmc_arch(D, C, PRECISIONS[precision], int(bool(marshall)))
        h = ct.c_void_p()
        rc = lib().vmc_create(L, J1, J2, ct.byref(arch), ct.byref(h))
        if rc != VMC_OK:
            raise VMCError(rc, f"vmc_create(L={L}, C={C}, D={D}, {precision}) failed")
        self._h = h
        n = ct.c_int64()
        lib().vmc_num_params(h, ct.byref(n))
        self.n = n.value

    def close(self):
        if self._h is not None and _lib is not None:
            _lib.vmc_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != VMC_OK:
            raise VMCError(rc, lib().vmc_last_error(self._h).decode())

    @property
    def last_launch_count(self):
        return int(lib().vmc_last_launch_count(self._h))

    def set_params(self, theta):
        if theta.dtype not in (torch.float64, torch.float32) or not theta.is_cuda:
            raise TypeError("theta must be a CUDA float64/float32 tensor")
        theta = theta.contiguous()
        if theta.numel() != self.n:
            raise ValueError(f"theta has {theta.numel()} values, expected {self.n}")
        self._theta_keep = theta
        self._check(lib().vmc_set_params(self._h, _ptr(theta),
                                         VMC_FP64 if theta.dtype == torch.float64 else VMC_FP32, _stream()))

    def get_params(self):
        out = torch.empty(self.n, dtype=torch.float64, device="cuda")
        self._check(lib().vmc_get_params(self._h, _ptr(out), _stream()))
        return out

    def logpsi(self, sigma):
        s = _dev(sigma, torch.int8, "sigma")
        B = s.shape[0]
        la = torch.empty(B, dtype=torch.float64, device=s.device)
        sg = torch.empty(B, dtype=torch.int8, device=s.device)
        self._check(lib().vmc_logpsi(self._h, _ptr(s), B, _ptr(la), _ptr(sg), _stream()))
        return la, sg

    def local_energy(self, sigma, out=None, n_nbr=True):
        s = _dev(sigma, torch.int8, "sigma")
        B = s.shape[0]
        e = out if out is not None else torch.empty(B, dtype=torch.float64, device=s.device)
        nn = torch.empty(B, dtype=torch.int32, device=s.device) if n_nbr else None
        self._check(lib().vmc_local_energy(self._h, _ptr(s), B, _ptr(e), _ptr(nn), _stream()))
        return e, nn

    def local_energy_ragged(self, packed, offs, Ls, L_max, out=None, n_nbr=True):
        pk = _dev(packed, torch.int8, "packed")
        of = _dev(offs, torch.int64, "offs")
        Lt = _dev(Ls, torch.int32, "Ls")
        B = of.shape[0]
        e = out if out is not None else torch.empty(B, dtype=torch.float64, device=pk.device)
        nn = torch.empty(B, dtype=torch.int32, device=pk.device) if n_nbr else None
        self._check(lib().vmc_local_energy_ragged(self._h, _ptr(pk), _ptr(of), _ptr(Lt), B, int(L_max),
                                                  _ptr(e), _ptr(nn), _stream()))
        return e, nn

    def logpsi_sym(self, sigma):
        """(log|W~|, sgn W~) of the rotationally symmetrised amplitude."""
        s = _dev(sigma, torch.int8, "sigma")
        B = s.shape[0]
        la = torch.empty(B, dtype=torch.float64, device=s.device)
        sg = torch.empty(B, dtype=torch.int8, device=s.device)
        self._check(lib().vmc_logpsi_sym(self._h, _ptr(s), B, _ptr(la), _ptr(sg), _stream()))
        return la, sg

    def local_energy_sym(self, sigma, n_nbr=True):
        s = _dev(sigma, torch.int8, "sigma")
        B = s.shape[0]
        e = torch.empty(B, dtype=torch.float64, device=s.device)
        nn = torch.empty(B, dtype=torch.int32, device=s.device) if n_nbr else None
        self._check(lib().vmc_local_energy_sym(self._h, _ptr(s), B, _ptr(e), _ptr(nn), _stream()))
        return e, nn

    def log_derivs_sym(self, sigma, dtype=torch.float32):
        s = _dev(sigma, torch.int8, "sigma")
        B = s.shape[0]
        O = torch.empty(B, self.n, dtype=dtype, device=s.device)
        code = VMC_FP64 if O.dtype == torch.float64 else VMC_FP32
        self._check(lib().vmc_log_derivs_sym(self._h, _ptr(s), B, _ptr(O), code, _stream()))
        return O

    def metropolis(self, sigma, logabs, u, hastings=False, accepted=None):
        """Advance the chains sigma [B, L, L] (int8, in place) and their
        log|psi| (float64 [B], in place) by u.shape[0] transitions drawn
        from u [steps, B, 2] (float64 in [0, 1)); accepted (int32 [B]) is
        incremented by the accepted moves."""
        if not (sigma.is_cuda and sigma.dtype == torch.int8 and sigma.is_contiguous()):
            raise TypeError("sigma must be a contiguous CUDA int8 tensor (updated in place)")
        if not (logabs.is_cuda and logabs.dtype == torch.float64 and logabs.is_contiguous()):
            raise TypeError("logabs must be a contiguous CUDA float64 tensor (updated in place)")
        uu = _dev(u, torch.float64, "u")
        B = sigma.shape[0]
        if uu.dim() != 3 or uu.shape[1] != B or uu.shape[2] != 2 or logabs.numel() != B:
            raise ValueError("u must be [steps, B, 2] and logabs [B]")
        if accepted is not None and not (accepted.is_cuda and accepted.dtype == torch.int32 and accepted.is_contiguous()):
            raise TypeError("accepted must be a contiguous CUDA int32 tensor")
        self._check(lib().vmc_metropolis(self._h, _ptr(sigma), _ptr(logabs), B, _ptr(uu), uu.shape[0],
                                         int(bool(hastings)), _ptr(accepted), _stream()))

    def log_derivs(self, sigma, dtype=torch.float32, out=None):
        s = _dev(sigma, torch.int8, "sigma")
        B = s.shape[0]
        O = out if out is not None else torch.empty(B, self.n, dtype=dtype, device=s.device)
        code = VMC_FP64 if O.dtype == torch.float64 else VMC_FP32
        self._check(lib().vmc_log_derivs(self._h, _ptr(s), B, _ptr(O), code, _stream()))
        return O

    def sr_moments(self, O, E):
        O = _dev(O, torch.float32, "O")
        E = _dev(E, torch.float64, "E")
        m = O.shape[0]
        ob = torch.empty(self.n, dtype=torch.float64, device=O.device)
        g = torch.empty(self.n, dtype=torch.float64, device=O.device)
        eb = torch.empty(1, dtype=torch.float64, device=O.device)
        self._check(lib().vmc_sr_moments(self._h, _ptr(O), _ptr(E), m, _ptr(ob), _ptr(eb), _ptr(g), _stream()))
        return ob, eb, g

    def sr_matvec(self, O, Obar, v, shift):
        O = _dev(O, torch.float32, "O")
        v = _dev(v, torch.float64, "v")
        out = torch.empty(self.n, dtype=torch.float64, device=O.device)
        self._check(lib().vmc_sr_matvec(self._h, _ptr(O), O.shape[0], _ptr(Obar), _ptr(v), float(shift),
                                        _ptr(out), _stream()))
        return out

    def ot_vec(self, O, w):
        O = _dev(O, torch.float32, "O")
        w = _dev(w, torch.float64, "w")
        out = torch.empty(self.n, dtype=torch.float64, device=O.device)
        self._check(lib().vmc_ot_vec(self._h, _ptr(O), O.shape[0], _ptr(w), _ptr(out), _stream()))
        return out

    def sr_solve_dense(self, O, E, shift=1e-4, out=None, resid=True):
        """x = (S + shift I)^{-1} G solved exactly in sample space (Woodbury)."""
        O = _dev(O, torch.float32, "O")
        E = _dev(E, torch.float64, "E")
        x = out if out is not None else torch.empty(self.n, dtype=torch.float64, device=O.device)
        r = ct.c_double(0.0)
        self._check(lib().vmc_sr_solve_dense(self._h, _ptr(O), _ptr(E), O.shape[0], float(shift), _ptr(x),
                                             ct.byref(r) if resid else None, _stream()))
        return x, (r.value if resid else None)

    def sr_solve(self, O, E, shift=1e-4, iters=50, out=None, resid=True):
        O = _dev(O, torch.float32, "O")
        E = _dev(E, torch.float64, "E")
        x = out if out is not None else torch.empty(self.n, dtype=torch.float64, device=O.device)
        r = ct.c_double(0.0)
        self._check(lib().vmc_sr_solve(self._h, _ptr(O), _ptr(E), O.shape[0], float(shift), int(iters),
                                       _ptr(x), ct.byref(r) if resid else None, _stream()))
        return x, (r.value if resid else None)

    def sr_update(self, x, eta):
        """theta <- theta - eta x on the context's parameters (Eq. 6)."""
        x = _dev(x, torch.float64, "x")
        if x.numel() != self.n:
            raise ValueError(f"x has {x.numel()} values, expected {self.n}")
        self._check(lib().vmc_sr_update(self._h, _ptr(x), float(eta), _stream()))

    def sync_status(self):
        """(code, nonfinite count) after synchronising the current stream."""
        nf = ct.c_int64(0)
        rc = lib().vmc_sync_status(self._h, _stream(), ct.byref(nf))
        return rc, nf.value

    def set_wait_budget(self, ns):
        self._check(lib().vmc_set_wait_budget(self._h, int(ns)))

    def set_sr_fused(self, enable):
        self._check(lib().vmc_set_sr_fused(self._h, 1 if enable else 0))

    def set_light_cone(self, enable):
        self._check(lib().vmc_set_light_cone(self._h, 1 if enable else 0))

    @property
    def light_cone_active(self):
        a = ct.c_int(0)
        self._check(lib().vmc_light_cone_active(self._h, ct.byref(a)))
        return bool(a.value)

    def set_launch_timing(self, enable):
        self._check(lib().vmc_set_launch_timing(self._h, 1 if enable else 0))

    def launch_timings(self):
        """[(kernel name, ms)] of the tensor-core launches recorded since
        set_launch_timing(True)."""
        cnt = ct.c_int(0)
        self._check(lib().vmc_launch_timings(self._h, 0, None, ct.byref(cnt)))
        n = cnt.value
        ms = (ct.c_double * max(n, 1))()
        self._check(lib().vmc_launch_timings(self._h, n, ms, ct.byref(cnt)))
        return [(lib().vmc_launch_timing_name(self._h, i).decode(), ms[i]) for i in range(n)]

    def debug_wait_timeout(self, budget_ns):
        self._check(lib().vmc_debug_wait_timeout(self._h, int(budget_ns), _stream()))

    def set_tiles(self, L, slab_configs=0, slabs=0, ctas_per_sm=0, lane_cells=0):
        t = vmc_tiles(slab_configs, slabs, ctas_per_sm, lane_cells)
        self._check(lib().vmc_set_tiles(self._h, L, ct.byref(t)))

    def get_tiles(self, L):
        t = vmc_tiles()
        self._check(lib().vmc_get_tiles(self._h, L, ct.byref(t)))
        return {"slab_configs": t.slab_configs, "slabs": t.slabs, "ctas_per_sm": t.ctas_per_sm,
                "lane_cells": t.lane_cells}

    def set_cone_tiles(self, slab_configs=0, slabs=0, lane_cells=0):
        t = vmc_tiles(slab_configs, slabs, 0, lane_cells)
        self._check(lib().vmc_set_cone_tiles(self._h, ct.byref(t)))

    def get_cone_tiles(self):
        t = vmc_tiles()
        self._check(lib().vmc_get_cone_tiles(self._h, ct.byref(t)))
        return {"slab_configs": t.slab_configs, "slabs": t.slabs, "lane_cells": t.lane_cells}

    def autotune(self, L, probe_B=512):
        self._check(lib().vmc_autotune(self._h, L, int(probe_B), _stream()))
        return self.get_tiles(L)


def ot_vec_noalloc(O, w, out=None):
    """O^T w through the allocation-free entry point (no context; see vmc.h).

    Returns (out, status) without raising, so callers can inspect the code."""
    m, n = O.shape
    out = out if out is not None else torch.empty(n, dtype=torch.float64, device=O.device)
    rc = lib().vmc_ot_vec_noalloc(_ptr(O), m, n, _ptr(w), _ptr(out), _stream())
    return out, rc


def umma_selftest(A, B, N, K, shift=0, variant=0):
    """One tcgen05 tile D = A[shift:shift+128] @ B^T (BF16 in, FP32 out)."""
    D = torch.empty(128, N, dtype=torch.float32, device="cuda")
    rc = lib().vmc_debug_umma_selftest(_ptr(A), _ptr(B), _ptr(D), N, K, shift, variant, _stream())
    if rc != VMC_OK:
        raise VMCError(rc, "umma selftest launch")
    return D


def umma_rate(N, count=4096, ctas=1):
    """(cycles per 128 x N x 16 UMMA, launch ms) of back-to-back issue."""
    c, ms = ct.c_double(), ct.c_double()
    rc = lib().vmc_debug_umma_rate(N, count, ctas, ct.byref(c), ct.byref(ms))
    if rc != VMC_OK:
        raise VMCError(rc, "umma rate probe")
    return c.value, ms.value


class LogPsi(torch.autograd.Function):
    """log|psi(sigma; theta)| with a backward through the library's O_k kernel.

    forward: loads theta into the context and evaluates vmc_logpsi.
    backward: recomputes the activations per sample (vmc_log_derivs) and
    returns O^T grad (vmc_ot_vec) as the gradient of theta.
    """

    @staticmethod
    def forward(ctx, theta, sigma, vmc):
        vmc.set_params(theta)
        la, _ = vmc.logpsi(sigma)
        ctx.save_for_backward(sigma)
        ctx.vmc = vmc
        ctx.theta_dtype = theta.dtype
        return la

    @staticmethod
    def backward(ctx, grad):
        (sigma,) = ctx.saved_tensors
        vmc = ctx.vmc
        O = vmc.log_derivs(sigma, dtype=torch.float32)
        g = vmc.ot_vec(O, grad.to(torch.float64).contiguous())
        return g.to(ctx.theta_dtype), None, None


def logpsi(theta, sigma, vmc):
    return LogPsi.apply(theta, sigma, vmc)
