"""Parity of the rotationally symmetrised amplitude W~(S) = sum_i W(T^i S)
(vmc_logpsi_sym, vmc_local_energy_sym, vmc_log_derivs_sym; Sec. 2.2 and
Sec. 3.3) with the oracle and with its own definition.

FP64, L = 4 (C = 4, D = 2): log|W~|, sgn W~, E_loc and O_k against the
oracle to FP64 rounding.
BF16 / FP16: each output equals, to FP64 rounding of the combination, the
same combination formed on the host from the library's plain log|psi| of the
explicitly rotated configurations (and, for E_loc, of the rotated exchange
neighbours).  This checks the expansion, the ordering and the FP64 combine
exactly.  L = 24 with 512 samples spans two workspace chunks.  The BF16
numerics are checked against the oracle at L = 16, with the tolerances of
the plain tensor-core path.
"""
import numpy as np
import pytest
import torch

from oracle import symmetry as sym
from paper_2108_13830_gb300 import inputs
from paper_2108_13830_gb300.binding import VMC_OK
from gpu_util import make_ctx, to_dev

pytestmark = pytest.mark.gpu


def test_fp64_matches_oracle():
    w = inputs.WORKLOADS["L4_fp64"]
    sig, theta = inputs.workload_inputs(w, batch=32)
    v = make_ctx(w, theta=theta)
    s = to_dev(sig)
    la, sg = v.logpsi_sym(s)
    ra, rs = sym.logpsi_sym(w.L, w.C, w.D, theta, sig)
    np.testing.assert_allclose(la.cpu().numpy(), ra, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(sg.cpu().numpy().astype(np.int32), rs)
    e, nn = v.local_energy_sym(s)
    re, rn = sym.local_energy_sym(w.L, w.J1, w.J2, w.C, w.D, theta, sig)
    np.testing.assert_allclose(e.cpu().numpy(), re, rtol=1e-11, atol=1e-11)
    np.testing.assert_array_equal(nn.cpu().numpy(), rn)
    O = v.log_derivs_sym(s[:8], dtype=torch.float64).cpu().numpy()
    R = sym.log_derivs_sym(w.L, w.C, w.D, theta, sig[:8])
    np.testing.assert_allclose(O, R, rtol=1e-10, atol=1e-12)
    O32 = v.log_derivs_sym(s[:8]).cpu().numpy()
    rel = np.abs(O32 - R).max(axis=1) / np.abs(R).max(axis=1)
    assert rel.max() <= 1e-6
    assert v.sync_status()[0] == VMC_OK


def _host_combine(v, cfgs, L):
    """log|W~|, sgn W~ of configurations [M, L, L] from the library's plain
    log|psi| of their four rotations (combined in FP64 by the oracle's rule)."""
    R = sym.rotations(cfgs, L).reshape(-1, L, L)
    la, sg = v.logpsi(to_dev(R))
    return sym.combine(la.cpu().numpy().reshape(-1, 4), sg.cpu().numpy().astype(np.float64).reshape(-1, 4))


def _host_eloc(v, s, w):
    d, nbrs, el = sym.exchange_neighbours(s, w.L, w.J1, w.J2)
    la, sg = _host_combine(v, np.stack([s] + nbrs).reshape(-1, w.L, w.L), w.L)
    acc = 0.0
    for q, c in enumerate(el):
        acc += c * float(sg[1 + q] * sg[0]) * np.exp(la[1 + q] - la[0])
    return d + acc


@pytest.mark.parametrize("name,prec", [("L16_bf16", "bf16"), ("L16_bf16", "fp16"), ("L24_bf16_sr", "bf16")])
def test_tensor_core_equals_host_combination(name, prec):
    w = inputs.WORKLOADS[name]
    B = 512 if w.L == 24 else 64
    sig, theta = inputs.workload_inputs(w, batch=B)
    v = make_ctx(w, precision=prec, theta=theta)
    s = to_dev(sig)
    la, sg = v.logpsi_sym(s)
    ha, hs = _host_combine(v, sig, w.L)
    np.testing.assert_allclose(la.cpu().numpy(), ha, rtol=1e-14, atol=1e-12)
    np.testing.assert_array_equal(sg.cpu().numpy().astype(np.int32), hs)
    e, nn = v.local_energy_sym(s)
    assert v.sync_status()[0] == VMC_OK
    e = e.cpu().numpy()
    for b in (0, 1, B // 2, B - 1):        # L = 24: the first and the last chunk
        ref = _host_eloc(v, sig[b].reshape(-1), w)
        assert abs(e[b] - ref) <= 1e-11 * max(1.0, abs(ref)), (b, e[b], ref)
    if w.L == 16:
        O = v.log_derivs_sym(s[:4]).cpu().numpy()
        R = sym.rotations(sig[:4], w.L).reshape(-1, w.L, w.L)
        Or = v.log_derivs(to_dev(R)).cpu().numpy().reshape(4, 4, -1).astype(np.float64)
        lr, sr = v.logpsi(to_dev(R))
        lr = lr.cpu().numpy().reshape(4, 4)
        sr = sr.cpu().numpy().astype(np.float64).reshape(4, 4)
        lt, st = sym.combine(lr, sr)
        wgt = sr * st[:, None] * np.exp(lr - lt[:, None])
        ref = np.einsum("bi,bik->bk", wgt, Or)
        np.testing.assert_allclose(O, ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max())


def test_bf16_numerics_against_oracle():
    w = inputs.WORKLOADS["L16_bf16"]
    sig, theta = inputs.workload_inputs(w, batch=2)
    v = make_ctx(w, theta=theta)
    s = to_dev(sig)
    la, _ = v.logpsi_sym(s)
    ra, _ = sym.logpsi_sym(w.L, w.C, w.D, theta, sig)
    assert np.abs(la.cpu().numpy() - ra).max() <= 0.05
    e, _ = v.local_energy_sym(s[:1])
    re, _ = sym.local_energy_sym(w.L, w.J1, w.J2, w.C, w.D, theta, sig[:1])
    assert abs(float(e[0]) - re[0]) / (w.L * w.L) <= 1e-3
