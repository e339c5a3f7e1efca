"""Parity of the batched Metropolis sampler (vmc_metropolis, Sec. 3.1,
Fig. 2b-c) with the oracle chain, driven by the same random numbers.

FP64, L = 4 (C = 4, D = 2): the chains, their log|psi| and the accepted
counts equal the oracle's after 50 transitions, for the paper's rule and
with the Hastings factor (the decision P >= r is taken in FP64 on both
sides; the test checks that no decision of these seeds lies within 1e-9 of
its threshold).
BF16, L = 16 (C = 32, D = 8), 256 chains, one transition at a time: every
proposal equals the oracle's bit for bit; every decision equals the one the
host takes from the GPU's own log|psi| of chain and proposal, and the
oracle's FP64 decision wherever its margin exceeds four times the largest
difference between GPU and oracle log-ratios; the carried log|psi| equals a
fresh evaluation of the chain bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import metropolis as mh
from paper_2108_13830_gb300 import inputs
from paper_2108_13830_gb300.binding import VMCError, VMC_OK
from gpu_util import make_ctx, to_dev

pytestmark = pytest.mark.gpu


def _log_margin(P, r):
    with np.errstate(divide="ignore"):
        return np.abs(np.log(P) - np.log(r))


@pytest.mark.parametrize("hastings", [False, True], ids=["paper", "hastings"])
def test_fp64_chains_match_oracle(hastings):
    w = inputs.WORKLOADS["L4_fp64"]
    sig, theta = inputs.workload_inputs(w, batch=64)
    u = inputs.chain_uniforms(50, 64, inputs.rng_for(w.index, 7))
    v = make_ctx(w, theta=theta)
    s = to_dev(sig)
    la, _ = v.logpsi(s)
    acc = torch.zeros(64, dtype=torch.int32, device="cuda")
    v.metropolis(s, la, to_dev(u), hastings=hastings, accepted=acc)
    assert v.sync_status()[0] == VMC_OK

    def lp(c):
        return oracle.logpsi(w.L, w.C, w.D, theta, c)[0]
    ref_s, ref_la, ref_acc, trace = mh.metropolis(sig.reshape(64, -1), lp(sig), u, lp, w.L,
                                                  hastings=hastings, trace=True)
    margins = np.concatenate([_log_margin(P, r) for P, r, _ in trace])
    assert margins.min() > 1e-9
    np.testing.assert_array_equal(s.cpu().numpy().reshape(64, -1), ref_s)
    np.testing.assert_array_equal(acc.cpu().numpy(), ref_acc)
    np.testing.assert_allclose(la.cpu().numpy(), ref_la, rtol=1e-12, atol=1e-12)
    assert 0 < ref_acc.sum() < 64 * 50


@pytest.fixture(scope="module")
def l16():
    w = inputs.WORKLOADS["L16_bf16"]
    sig, theta = inputs.workload_inputs(w, batch=256)
    return w, sig, theta, make_ctx(w, theta=theta)


def test_bf16_transitions_match_oracle(l16):
    w, sig, theta, v = l16
    B, L = sig.shape[0], w.L
    u = inputs.chain_uniforms(3, B, inputs.rng_for(w.index, 7))
    s = to_dev(sig)
    la, _ = v.logpsi(s)
    acc = torch.zeros(B, dtype=torch.int32, device="cuda")
    err_max, n_checked, n_moves = 0.0, 0, 0
    for t in range(u.shape[0]):
        prev = s.cpu().numpy().reshape(B, -1)
        la_prev = la.cpu().numpy().copy()
        v.metropolis(s, la, to_dev(u[t:t + 1]), accepted=acc)
        assert v.sync_status()[0] == VMC_OK
        now = s.cpu().numpy().reshape(B, -1)
        prop, n_pairs, bond = mh.propose(prev, L, u[t, :, 0])
        assert (bond >= 0).all()
        moved = (now != prev).any(axis=1)
        # a chain that moved took the oracle's proposal; one that stayed is unchanged
        np.testing.assert_array_equal(now[moved], prop[moved])
        # the GPU's decision from its own log|psi| of the proposals
        la_prop_g = v.logpsi(to_dev(prop.reshape(B, L, L)))[0].cpu().numpy()
        P_g = mh.accept_prob(la_prev, la_prop_g, n_pairs, n_pairs, False)
        tie = _log_margin(P_g, u[t, :, 1]) < 1e-12
        np.testing.assert_array_equal(moved[~tie], (P_g >= u[t, :, 1])[~tie])
        # the oracle's FP64 decision where its margin exceeds the measured error
        la_prev_o = oracle.logpsi(L, w.C, w.D, theta, prev)[0]
        la_prop_o = oracle.logpsi(L, w.C, w.D, theta, prop)[0]
        err = np.abs((la_prop_g - la_prev) - (la_prop_o - la_prev_o))
        err_max = max(err_max, float(err.max()))
        P_o = mh.accept_prob(la_prev_o, la_prop_o, n_pairs, n_pairs, False)
        sure = _log_margin(P_o, u[t, :, 1]) > 4 * 2 * err.max()
        np.testing.assert_array_equal(moved[sure], (P_o >= u[t, :, 1])[sure])
        n_checked += int(sure.sum())
        n_moves += int(moved.sum())
        # carried log|psi| is the forward of the current chain, bit for bit
        np.testing.assert_array_equal(la.cpu().numpy(), v.logpsi(s)[0].cpu().numpy())
    assert n_checked > 0.5 * B * u.shape[0]
    assert 0 < n_moves < B * u.shape[0]
    assert int(acc.sum()) == n_moves
    assert err_max < 0.1


def test_bf16_many_transitions_invariants(l16):
    w, sig, theta, v = l16
    B = sig.shape[0]
    u = inputs.chain_uniforms(24, B, inputs.rng_for(w.index, 8))
    s = to_dev(sig)
    la, _ = v.logpsi(s)
    acc = torch.zeros(B, dtype=torch.int32, device="cuda")
    v.metropolis(s, la, to_dev(u), hastings=True, accepted=acc)
    assert v.sync_status()[0] == VMC_OK
    now = s.cpu().numpy().reshape(B, -1).astype(np.int64)
    assert (now.sum(axis=1) == 0).all() and set(np.unique(now)) == {-1, 1}
    np.testing.assert_array_equal(la.cpu().numpy(), v.logpsi(s)[0].cpu().numpy())
    a = acc.cpu().numpy()
    assert a.max() <= 24 and a.sum() > 0
    # chains that never accepted are unchanged
    still = a == 0
    np.testing.assert_array_equal(now[still], sig.reshape(B, -1)[still])


def test_edge_cases():
    w = inputs.WORKLOADS["L4_fp64"]
    sig, theta = inputs.workload_inputs(w, batch=8)
    v = make_ctx(w, theta=theta)
    s = to_dev(sig)
    s[3] = 1                       # no antiparallel pair: no move
    la, _ = v.logpsi(s)
    before = s.clone()
    la0 = la.clone()
    acc = torch.zeros(8, dtype=torch.int32, device="cuda")
    v.metropolis(s, la, torch.zeros(0, 8, 2, dtype=torch.float64, device="cuda"), accepted=acc)
    assert torch.equal(s, before) and torch.equal(la, la0) and int(acc.sum()) == 0
    u = inputs.chain_uniforms(20, 8, inputs.rng_for(w.index, 9))
    v.metropolis(s, la, to_dev(u), accepted=acc)
    assert v.sync_status()[0] == VMC_OK
    assert torch.equal(s[3], before[3]) and int(acc[3]) == 0
    v.metropolis(s[:0], la[:0], torch.zeros(5, 0, 2, dtype=torch.float64, device="cuda"))
    with pytest.raises(VMCError):
        from paper_2108_13830_gb300.binding import lib, _ptr, _stream
        v._check(lib().vmc_metropolis(v._h, _ptr(s), _ptr(la), 8, _ptr(to_dev(u)), 20, 2, None, _stream()))
