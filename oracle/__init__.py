"""FP64 CPU oracle: plain, slow, obviously correct (test infrastructure).

Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  It shares no code with the CUDA
library: the C part (oracle.c) is compiled by oracle/build.py with gcc and
loaded through ctypes; exact diagonalisation (ed.py), the Metropolis chain
(metropolis.py) and the rotational symmetrisation (symmetry.py) sit on top of
numpy/scipy.

Functions follow the paper (arXiv:2108.13830): Hamiltonian Eq. 3, local
energy Eq. 4-5, Marshall sign Eq. 9, O_k Eq. 5, covariance Eq. 7 with the
diagonal shift of Sec. 3.2.2.
"""
from __future__ import annotations

import ctypes as _ct
import numpy as _np

from . import build as _build

_lib = None
_dp = _np.ctypeslib.ndpointer(_np.float64, flags="C_CONTIGUOUS")
_i8p = _np.ctypeslib.ndpointer(_np.int8, flags="C_CONTIGUOUS")
_i32p = _np.ctypeslib.ndpointer(_np.int32, flags="C_CONTIGUOUS")
_I, _D, _I64 = _ct.c_int, _ct.c_double, _ct.c_int64


def lib():
    global _lib
    if _lib is None:
        L = _ct.CDLL(_build.build())
        L.orc_num_params.restype = _I64
        L.orc_num_params.argtypes = [_I, _I]
        L.orc_forward_z.argtypes = [_I, _I, _I, _dp, _i8p, _dp]
        L.orc_logpsi_batch.argtypes = [_I, _I, _I, _dp, _I, _i8p, _I64, _dp, _i32p, _I]
        L.orc_local_energy_batch.argtypes = [_I, _D, _D, _I, _I, _dp, _I, _i8p, _I64, _dp,
                                             _ct.c_void_p, _I]
        L.orc_local_energy_cnn_par.restype = _D
        L.orc_local_energy_cnn_par.argtypes = [_I, _D, _D, _I, _I, _dp, _I, _i8p, _ct.c_void_p, _I]
        L.orc_local_energy_table.restype = _D
        L.orc_local_energy_table.argtypes = [_I, _D, _D, _dp, _i8p]
        L.orc_log_derivs_batch.argtypes = [_I, _I, _I, _dp, _i8p, _I64, _dp, _I]
        L.orc_sr_moments.argtypes = [_dp, _dp, _I64, _I64, _dp, _dp, _dp]
        L.orc_sr_matvec.argtypes = [_dp, _I64, _I64, _dp, _dp, _D, _dp]
        L.orc_sr_matvec_centered.argtypes = [_dp, _I64, _I64, _dp, _D, _dp]
        L.orc_sr_cg.restype = _D
        L.orc_sr_cg.argtypes = [_dp, _I64, _I64, _dp, _dp, _D, _I, _dp]
        L.orc_max_threads.restype = _I
        _lib = L
    return _lib


def _f64(a):
    return _np.ascontiguousarray(a, dtype=_np.float64)


def _cfg(sigma, L):
    s = _np.ascontiguousarray(sigma, dtype=_np.int8).reshape(-1, L * L)
    return s, s.shape[0]


def num_params(C: int, D: int) -> int:
    return int(lib().orc_num_params(C, D))


def max_threads() -> int:
    return int(lib().orc_max_threads())


def forward_z(L, C, D, theta, sigma):
    """Pre-activations of every layer for one configuration: [D+1, C, L, L]."""
    s = _np.ascontiguousarray(sigma, dtype=_np.int8).reshape(L * L)
    z = _np.zeros((D + 1) * C * L * L)
    lib().orc_forward_z(L, C, D, _f64(theta), s, z)
    return z.reshape(D + 1, C, L, L)


def logpsi(L, C, D, theta, sigma, marshall=True, nthreads=0):
    """(log|psi| [B], sign [B]) with sign = 0 where psi == 0."""
    s, B = _cfg(sigma, L)
    la = _np.zeros(B)
    sg = _np.zeros(B, _np.int32)
    lib().orc_logpsi_batch(L, C, D, _f64(theta), int(marshall), s, B, la, sg, nthreads)
    return la, sg


def local_energy(L, J1, J2, C, D, theta, sigma, marshall=True, nthreads=0):
    """(E_loc [B], number of exchange neighbours [B]) for the CNN wavefunction."""
    s, B = _cfg(sigma, L)
    e = _np.zeros(B)
    nn = _np.zeros(B, _np.int32)
    lib().orc_local_energy_batch(L, J1, J2, C, D, _f64(theta), int(marshall), s, B, e,
                                 nn.ctypes.data, nthreads)
    return e, nn


def local_energy_par(L, J1, J2, C, D, theta, sigma, marshall=True, nthreads=0):
    """Same as local_energy, one sample at a time with its neighbours spread
    over threads (for large lattices)."""
    s, B = _cfg(sigma, L)
    e = _np.zeros(B)
    nn = _np.zeros(B, _np.int32)
    th = _f64(theta)
    for b in range(B):
        row = _np.ascontiguousarray(s[b])
        e[b] = lib().orc_local_energy_cnn_par(L, J1, J2, C, D, th, int(marshall), row,
                                              nn[b:].ctypes.data, nthreads)
    return e, nn


def local_energy_table(L, J1, J2, table, sigma):
    """E_loc for a wavefunction given as a 2^(L*L) lookup table (L = 4)."""
    t = _f64(table)
    s, B = _cfg(sigma, L)
    return _np.array([lib().orc_local_energy_table(L, J1, J2, t, s[b].copy()) for b in range(B)])


def log_derivs(L, C, D, theta, sigma, nthreads=0):
    """O [B, n] = d log|psi| / d theta, FP64."""
    s, B = _cfg(sigma, L)
    n = num_params(C, D)
    O = _np.zeros((B, n))
    lib().orc_log_derivs_batch(L, C, D, _f64(theta), s, B, O, nthreads)
    return O


def sr_moments(O, E):
    """(<O> [n], <E>, G [n]) with <.> the sample mean."""
    O = _f64(O)
    m, n = O.shape
    ob = _np.zeros(n)
    g = _np.zeros(n)
    eb = _np.zeros(1)
    lib().orc_sr_moments(O, _f64(E), m, n, ob, eb, g)
    return ob, float(eb[0]), g


def sr_matvec(O, Obar, v, shift):
    """(M + shift I) v with M v = (1/m) O^T (O v) - <O>(<O>.v)."""
    O = _f64(O)
    m, n = O.shape
    out = _np.zeros(n)
    lib().orc_sr_matvec(O, m, n, _f64(Obar), _f64(v), float(shift), out)
    return out


def sr_matvec_centered(O, v, shift):
    """(M + shift I) v with M the covariance in its centred form,
    (1/m) sum_b (O_b - <O>) ((O_b - <O>) . v): equal to sr_matvec in exact
    arithmetic, without its cancellation when |<O>| >> std(O)."""
    O = _f64(O)
    m, n = O.shape
    out = _np.zeros(n)
    lib().orc_sr_matvec_centered(O, m, n, _f64(v), float(shift), out)
    return out


def sr_cg(O, E, shift, iters):
    """CG solution x of (M + shift I) x = G from x = 0; returns (x, ||r||/||G||)."""
    O = _f64(O)
    m, n = O.shape
    ob, _, g = sr_moments(O, E)
    x = _np.zeros(n)
    res = lib().orc_sr_cg(O, m, n, ob, g, float(shift), int(iters), x)
    return x, float(res)


def sr_solve_dense(O, E, shift):
    """x = (M + shift I)^{-1} G with M the covariance of Eq. 7 formed as an
    n x n matrix and factored by Cholesky (LAPACK potrf/potrs through
    scipy), the dense route of Sec. 3.2.2.  Small n only (n^2 doubles)."""
    import scipy.linalg as sla
    O = _f64(O)
    m, n = O.shape
    ob, _, g = sr_moments(O, E)
    Oc = O - ob
    M = (Oc.T @ Oc) / m + float(shift) * _np.eye(n)
    return sla.cho_solve(sla.cho_factor(M, lower=True), g)


def sr_update(theta, x, eta):
    """theta - eta x: the parameter step of Eq. 6 (Delta = eta x)."""
    return _f64(theta) - float(eta) * _f64(x)
