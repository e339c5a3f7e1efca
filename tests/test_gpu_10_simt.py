"""Parity of the plain (SIMT) FP64 / FP32 paths with the FP64 oracle.

FP64, L = 4 (4x4, C = 4, D = 2, 256 configurations): log|psi|, E_loc,
neighbour counts and O_k against the oracle to FP64 rounding, and O_k
against central finite differences of the GPU's own log|psi|.
FP32, L = 10 (C = 16, D = 6): E_loc per site within 1e-6 of the oracle,
O_k normwise within 1e-6 per sample, on seeded subsets of the batch.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2108_13830_gb300 import inputs
from paper_2108_13830_gb300.binding import LogPsi, VMC_OK
from gpu_util import bond_counts, make_ctx, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[1.0, 3.0], ids=["std", "stressed"])
def l4(request):
    w = inputs.WORKLOADS["L4_fp64"]
    sig, theta = inputs.workload_inputs(w, scale=request.param)
    return w, sig, theta, make_ctx(w, theta=theta)


def test_fp64_logpsi(l4):
    w, sig, theta, v = l4
    la, sg = v.logpsi(to_dev(sig))
    ra, rs = oracle.logpsi(w.L, w.C, w.D, theta, sig)
    np.testing.assert_allclose(la.cpu().numpy(), ra, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(sg.cpu().numpy().astype(np.int32), rs)


def test_fp64_local_energy(l4):
    w, sig, theta, v = l4
    e, nn = v.local_energy(to_dev(sig))
    re, rn = oracle.local_energy(w.L, w.J1, w.J2, w.C, w.D, theta, sig)
    np.testing.assert_allclose(e.cpu().numpy(), re, rtol=1e-11, atol=1e-11)
    np.testing.assert_array_equal(nn.cpu().numpy(), rn)
    a1, a2 = bond_counts(sig)
    np.testing.assert_array_equal(nn.cpu().numpy(), a1 + a2)
    assert v.sync_status()[0] == VMC_OK


def test_fp64_log_derivs_vs_oracle(l4):
    w, sig, theta, v = l4
    O = v.log_derivs(to_dev(sig[:16]), dtype=torch.float64).cpu().numpy()
    R = oracle.log_derivs(w.L, w.C, w.D, theta, sig[:16])
    np.testing.assert_allclose(O, R, rtol=1e-10, atol=1e-12)


def test_fp64_log_derivs_vs_finite_differences(l4):
    """O_k against Richardson-extrapolated central differences of the GPU
    log|psi| (FP64): D(h) = (f(x+h) - f(x-h)) / 2h, (4 D(h/2) - D(h)) / 3
    has an O(h^4) truncation error.  h = 1e-6 max(1, |theta|): the stressed
    network has outputs near zero (|O| up to ~1e3), where larger steps leave
    truncation errors of 1e-4 relative; the FP64 round-off at this step is
    ~eps |log psi| / h ~ 1e-8."""
    w, sig, theta, v = l4
    s = to_dev(sig[:2])
    O = v.log_derivs(s, dtype=torch.float64).cpu().numpy()

    def central(k, h):
        tp = theta.copy(); tp[k] += h
        tm = theta.copy(); tm[k] -= h
        v.set_params(to_dev(tp))
        lp, _ = v.logpsi(s)
        v.set_params(to_dev(tm))
        lm, _ = v.logpsi(s)
        return ((lp - lm) / (2 * h)).cpu().numpy()

    fd = np.zeros_like(O)
    for k in range(theta.size):
        h = 1e-6 * max(1.0, abs(theta[k]))
        fd[:, k] = (4 * central(k, h / 2) - central(k, h)) / 3
    v.set_params(to_dev(theta))
    np.testing.assert_allclose(O, fd, rtol=1e-6, atol=1e-7 * np.abs(O).max())


def test_autograd_backward(l4):
    """LogPsi.backward = O^T grad, checked against the oracle O."""
    w, sig, theta, v = l4
    th = to_dev(theta).requires_grad_(True)
    s = to_dev(sig[:32])
    la = LogPsi.apply(th, s, v)
    gw = torch.linspace(-1.0, 1.0, 32, dtype=torch.float64, device="cuda")
    (la * gw).sum().backward()
    R = oracle.log_derivs(w.L, w.C, w.D, theta, sig[:32])
    g = gw.cpu().numpy()
    ref = R.T @ g
    # the backward stores O in FP32 (unit roundoff 2^-24) before O^T grad
    bound = 2.0 ** -23 * (np.abs(R).T @ np.abs(g))
    assert np.all(np.abs(th.grad.cpu().numpy() - ref) <= bound + 1e-15)


@pytest.fixture(scope="module")
def l10():
    w = inputs.WORKLOADS["L10_fp32"]
    sig, theta = inputs.workload_inputs(w)
    return w, sig, theta, make_ctx(w, theta=theta)


def test_fp32_local_energy_full_batch_sampled(l10):
    w, sig, theta, v = l10
    e, nn = v.local_energy(to_dev(sig))
    assert v.sync_status()[0] == VMC_OK
    e = e.cpu().numpy()
    a1, a2 = bond_counts(sig)
    np.testing.assert_array_equal(nn.cpu().numpy(), a1 + a2)
    pick = np.random.default_rng(0).choice(w.batch, 24, replace=False)
    re, _ = oracle.local_energy(w.L, w.J1, w.J2, w.C, w.D, theta, sig[pick])
    err = np.abs(e[pick] - re) / (w.L * w.L)
    assert err.max() <= 1e-6, err.max()


def test_fp32_logpsi(l10):
    w, sig, theta, v = l10
    la, sg = v.logpsi(to_dev(sig[:64]))
    ra, rs = oracle.logpsi(w.L, w.C, w.D, theta, sig[:64])
    np.testing.assert_array_equal(sg.cpu().numpy().astype(np.int32), rs)
    np.testing.assert_allclose(la.cpu().numpy(), ra, rtol=1e-6, atol=1e-5)


def test_fp32_log_derivs_normwise(l10):
    w, sig, theta, v = l10
    O = v.log_derivs(to_dev(sig[:8])).cpu().numpy().astype(np.float64)
    R = oracle.log_derivs(w.L, w.C, w.D, theta, sig[:8])
    rel = np.abs(O - R).max(axis=1) / np.abs(R).max(axis=1)
    assert rel.max() <= 1e-6, rel


def test_fp32_ragged_simt_matches_oracle():
    w = inputs.WORKLOADS["ragged_8_16"]
    packed, offs, Ls, theta = inputs.ragged_inputs(w, per_L=2)
    v = make_ctx(w, precision="fp32", theta=theta, L=16)
    e, nn = v.local_energy_ragged(to_dev(packed), to_dev(offs), to_dev(Ls), 16)
    e = e.cpu().numpy()
    for b in range(len(offs)):
        L = int(Ls[b])
        cfg = packed[offs[b]:offs[b] + L * L].reshape(1, L, L)
        re, rn = oracle.local_energy(L, w.J1, w.J2, w.C, w.D, theta, cfg)
        assert abs(e[b] - re[0]) / (L * L) <= 1e-6
        assert nn[b].item() == rn[0]


def test_empty_batch_and_bad_args(l10):
    w, sig, theta, v = l10
    e, _ = v.local_energy(to_dev(sig[:0]))
    assert e.numel() == 0
    with pytest.raises(TypeError):
        v.local_energy(torch.zeros(4, 10, 10, dtype=torch.int32, device="cuda"))


def test_ragged_bad_lattice_size_reports_arg(l10):
    w, sig, theta, v = l10
    cfg = sig[:2].reshape(-1)
    offs = np.array([0, 100], np.int64)
    Ls = np.array([10, 9], np.int32)      # odd L is invalid
    e, _ = v.local_energy_ragged(to_dev(cfg), to_dev(offs), to_dev(Ls), 10)
    rc, _ = v.sync_status()
    assert rc == -1
    e = e.cpu().numpy()
    assert np.isfinite(e[0]) and np.isnan(e[1])
