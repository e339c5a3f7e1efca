"""Pins for the oracle's Metropolis chain (Sec. 3.1, Fig. 2b-c of
arXiv:2108.13830) against facts fixed by the paper and by mathematics.

Nothing here uses the CUDA library.  The log-amplitude is a closed-form
function of the configuration, so the stationary law of the chain can be
enumerated exactly over the 12,870 states of the 4 x 4 S^z = 0 sector.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import ed
from oracle import metropolis as mh


def _spins(states, L):
    N = L * L
    bits = (states[:, None] >> np.arange(N)[None, :]) & 1
    return np.where(bits == 1, 1, -1).astype(np.int8)


def _random_sector(rng, B, L):
    N = L * L
    s = np.full((B, N), -1, np.int8)
    for b in range(B):
        s[b, rng.permutation(N)[: N // 2]] = 1
    return s


# a log-amplitude with strong structure: beta times the number of
# antiparallel J1 bonds plus a site-dependent field, so that |psi|^2 and
# |psi|^2 n(S) are well apart
def _logpsi_fn(L, beta=0.2):
    N = L * L
    h = 0.15 * np.cos(np.arange(N) * 1.3)

    def f(cfg):
        c = np.asarray(cfg, np.int8).reshape(-1, N)
        return beta * mh.j1_pair_flags(c, L).sum(axis=1) + (c * h[None, :]).sum(axis=1)
    return f


def test_j1_propose_batch_matches_bond_list():
    """Sec. 3.1 / Fig. 2c: the J1 propose batch is the set of antiparallel
    right and lower neighbour pairs, in site order.  Checked against the
    bond list of the exact-diagonalisation module (separate code)."""
    rng = np.random.default_rng(7)
    for L in (4, 6, 8):
        pairs_ref_all = [(i, j) for (i, j, kind) in ed.bonds(L) if kind == 1]
        for s in _random_sector(rng, 5, L):
            flags = mh.j1_pair_flags(s[None], L)[0]
            got = [mh.bond_sites(L, k) for k in np.flatnonzero(flags)]
            ref = [(i, j) for (i, j) in pairs_ref_all if s[i] != s[j]]
            assert got == ref


def test_proposals_enumerate_j1_exchanges_once():
    """Scanning the selector over its n bins proposes every J1 exchange
    of S exactly once; each proposal moves two antiparallel nearest
    neighbours and keeps S^z."""
    L = 6
    rng = np.random.default_rng(3)
    s = _random_sector(rng, 1, L)[0]
    n = int(mh.j1_pair_flags(s[None], L).sum())
    seen = set()
    for k in range(n):
        sp_, nn, bond = mh.propose(s[None], L, np.array([(k + 0.5) / n]))
        assert nn[0] == n
        d = np.flatnonzero(sp_[0] != s)
        assert len(d) == 2 and s[d[0]] == -s[d[1]]
        i, j = mh.bond_sites(L, bond[0])
        assert set(d) == {i, j}
        assert sp_[0].sum() == s.sum()
        seen.add(sp_[0].tobytes())
    assert len(seen) == n
    # u just below 1 takes the last pair, u = 0 the first
    assert mh.propose(s[None], L, np.array([np.nextafter(1.0, 0.0)]))[2][0] == np.flatnonzero(
        mh.j1_pair_flags(s[None], L)[0])[-1]
    assert mh.propose(s[None], L, np.array([0.0]))[2][0] == np.flatnonzero(mh.j1_pair_flags(s[None], L)[0])[0]


@pytest.fixture(scope="module")
def sector4():
    L = 4
    states = ed.sector_states(L * L)
    return L, states, _spins(states, L)


def _transition_matrix(L, states, S, logpsi, hastings):
    """T[a, b] = probability that one transition moves S_a to S_b, built from
    the oracle's proposal and acceptance functions: pair k has probability
    1/n, acceptance probability min(1, P) (r uniform)."""
    M = len(states)
    index = {st: a for a, st in enumerate(states)}
    la = logpsi(S)
    n = mh.j1_pair_flags(S, L).sum(axis=1)
    rows, cols, vals = [], [], []
    for k in range(int(n.max())):
        act = np.flatnonzero(n > k)
        u0 = (k + 0.5) / n[act]
        sp_, nn, bond = mh.propose(S[act], L, u0)
        la_new = logpsi(sp_)
        n_new = mh.j1_pair_flags(sp_, L).sum(axis=1)
        P = mh.accept_prob(la[act], la_new, nn, n_new, hastings)
        bits = ((sp_ == 1).astype(np.int64) << np.arange(L * L)[None, :]).sum(axis=1)
        for a, st_b, p, na in zip(act, bits, P, nn):
            rows.append(a)
            cols.append(index[int(st_b)])
            vals.append(min(1.0, p) / na)
    T = sp.csr_matrix((vals, (rows, cols)), shape=(M, M))
    stay = 1.0 - np.asarray(T.sum(axis=1)).ravel()
    return T + sp.diags(stay), n


@pytest.mark.parametrize("hastings", [False, True])
def test_stationary_law_exact(sector4, hastings):
    """Detailed balance of the chain's rule, exactly over the 4 x 4 sector:
    the paper's rule (hastings=False) leaves |psi|^2 n(S) invariant, the
    Hastings-corrected one |psi|^2; the other law is not invariant."""
    L, states, S = sector4
    logpsi = _logpsi_fn(L)
    T, n = _transition_matrix(L, states, S, logpsi, hastings)
    w2 = np.exp(2.0 * (logpsi(S) - logpsi(S).max()))
    pi_paper = w2 * n / (w2 * n).sum()
    pi_h = w2 / w2.sum()
    want, other = (pi_h, pi_paper) if hastings else (pi_paper, pi_h)
    assert np.abs(T.T @ want - want).max() < 1e-14
    assert np.abs(T.T @ other - other).max() > 1e-6
    # detailed balance, not only stationarity
    F = sp.diags(want) @ T
    assert abs(F - F.T).max() < 1e-15


@pytest.mark.parametrize("hastings", [False, True])
def test_chain_samples_stationary_law(sector4, hastings):
    """The chain itself (state update, carried log|psi|, decision P >= r)
    samples the law fixed above: the mean number of antiparallel J1 bonds
    of 4000 chains after 100 transitions (from uniform S^z = 0 starts; the
    chains relax within ~40) matches its exact expectation within 4
    standard errors and is at least 5 away from the other law's (~10 apart)."""
    L, states, S = sector4
    logpsi = _logpsi_fn(L)
    rng = np.random.default_rng(2108)
    B, steps = 4000, 100
    s0 = _random_sector(rng, B, L)
    u = rng.random((steps, B, 2))
    s1, la1, acc = mh.metropolis(s0, logpsi(s0), u, logpsi, L, hastings=hastings)
    assert np.array_equal(la1, logpsi(s1))
    assert np.array_equal(s1.sum(axis=1), np.zeros(B))
    assert acc.mean() > 0.1 * steps and acc.max() <= steps
    f = mh.j1_pair_flags(s1, L).sum(axis=1).astype(np.float64)
    w2 = np.exp(2.0 * (logpsi(S) - logpsi(S).max()))
    n = mh.j1_pair_flags(S, L).sum(axis=1).astype(np.float64)
    mean_paper = (w2 * n * n).sum() / (w2 * n).sum()
    mean_h = (w2 * n).sum() / w2.sum()
    want, other = (mean_h, mean_paper) if hastings else (mean_paper, mean_h)
    se = f.std() / np.sqrt(B)
    assert abs(f.mean() - want) < 4 * se
    assert abs(f.mean() - other) > 5 * se


def test_chain_without_moves_stays():
    """A configuration with no antiparallel J1 pair has no move."""
    L = 4
    s = np.ones((2, L * L), np.int8)
    u = np.full((3, 2, 2), 0.25)
    s1, la1, acc = mh.metropolis(s, np.zeros(2), u, _logpsi_fn(L), L)
    assert np.array_equal(s1, s) and np.array_equal(acc, [0, 0]) and np.array_equal(la1, [0.0, 0.0])


def test_decision_is_p_at_least_r():
    """Acceptance exactly when (W'/W)^2 >= r: P = 0.25 for
    log|psi'| - log|psi| = -log 2."""
    P = mh.accept_prob(np.array([0.0, 0.0]), np.array([-np.log(2.0)] * 2), [4, 4], [2, 2], False)
    assert np.allclose(P, 0.25, rtol=0, atol=1e-16)
    Ph = mh.accept_prob(np.array([0.0]), np.array([-np.log(2.0)]), [4], [2], True)
    assert abs(Ph[0] - 0.5) < 1e-16
