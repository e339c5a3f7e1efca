"""Batched Metropolis sampling of |W(S)|^2 (test infrastructure).

Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this module; it shares no code with the CUDA library.

The chain follows Sec. 3.1 of arXiv:2108.13830 (Fig. 2b-c):
 - The J1 propose batch of a configuration is its list of antiparallel
   nearest-neighbour pairs, each bond once: for every site in order
   i = y L + x, the pair with its right neighbour (x + 1) and then the pair
   with its lower neighbour (y + 1), periodic.
 - A transition picks one pair of that batch uniformly at random and
   exchanges its two spins (S' keeps S^z).
 - S' is accepted when P = (W(S') / W(S))^2 >= r, r uniform in (0, 1).
 - Many independent chains advance together; one transition of every chain
   evaluates all proposals as one batch (Sec. 3.2.1, Fig. 3).
 - The paper takes L^2 transitions between recorded samples.

Readings where the paper is silent:
 - Random numbers are inputs.  u[s, b, 0] selects pair k = floor(u n)
   (clamped to 0 .. n - 1) of the n pairs; u[s, b, 1] is r.
 - P = exp(2 (log|psi(S')| - log|psi(S)|)) in FP64.
 - With hastings=True, P is multiplied by n(S) / n(S').  The proposal
   probability 1/n(S) is not symmetric, so without this factor the chain's
   stationary law is |psi|^2 n(S) / Z rather than |psi|^2 / Z.  With it,
   detailed balance holds for |psi|^2.  The paper states no such factor;
   hastings=False is its rule.
 - A configuration with no antiparallel J1 pair stays (it has no move).
"""
from __future__ import annotations

import numpy as np


def j1_pair_flags(sigma, L):
    """Antiparallel flags of the 2 N nearest-neighbour bonds, [B, 2 N].

    Bond 2 i + d joins site i to its right (d = 0) or lower (d = 1)
    neighbour on the torus.
    """
    s = np.asarray(sigma, dtype=np.int8).reshape(-1, L, L)
    right = s != np.roll(s, -1, axis=2)      # (y, x) vs (y, x + 1)
    below = s != np.roll(s, -1, axis=1)      # (y, x) vs (y + 1, x)
    return np.stack([right.reshape(-1, L * L), below.reshape(-1, L * L)], axis=2).reshape(s.shape[0], 2 * L * L)


def bond_sites(L, bond):
    """(i, j) of bond 2 i + d."""
    i, d = divmod(int(bond), 2)
    y, x = divmod(i, L)
    j = y * L + (x + 1) % L if d == 0 else ((y + 1) % L) * L + x
    return i, j


def propose(sigma, L, u0):
    """Proposals of one transition for every chain.

    Returns (sigma' [B, N], n [B], bond [B]); bond is -1 and sigma' = sigma
    where a chain has no antiparallel J1 pair.
    """
    s = np.array(sigma, dtype=np.int8).reshape(-1, L * L)
    flags = j1_pair_flags(s, L)
    n = flags.sum(axis=1)
    out = s.copy()
    bond = np.full(s.shape[0], -1, dtype=np.int64)
    for b in range(s.shape[0]):
        if n[b] == 0:
            continue
        k = min(max(int(np.floor(u0[b] * n[b])), 0), int(n[b]) - 1)
        bond[b] = int(np.flatnonzero(flags[b])[k])
        i, j = bond_sites(L, bond[b])
        out[b, i], out[b, j] = s[b, j], s[b, i]
    return out, n.astype(np.int64), bond


def accept_prob(la_old, la_new, n_old, n_new, hastings):
    """P = (W'/W)^2 (times n / n' with the Hastings factor), FP64."""
    with np.errstate(over="ignore", invalid="ignore"):
        P = np.exp(2.0 * (np.asarray(la_new, np.float64) - np.asarray(la_old, np.float64)))
        if hastings:
            P = P * (np.asarray(n_old, np.float64) / np.asarray(n_new, np.float64))
    return P


def metropolis(sigma, logabs, u, logpsi_fn, L, hastings=False, trace=False):
    """Advance B chains by u.shape[0] transitions.

    sigma [B, N] int8, logabs [B] = log|psi(sigma)|, u [steps, B, 2] in [0, 1).
    logpsi_fn(configs [M, N] int8) -> log|psi| [M] evaluates a batch.
    Returns (sigma, logabs, accepted [B]) and, with trace=True, a list of
    per-step (P [B], r [B], moved [B]) for margin checks.
    """
    s = np.array(sigma, dtype=np.int8).reshape(-1, L * L)
    la = np.array(logabs, dtype=np.float64).copy()
    u = np.asarray(u, dtype=np.float64)
    acc = np.zeros(s.shape[0], dtype=np.int64)
    steps = []
    for t in range(u.shape[0]):
        sp, n_old, bond = propose(s, L, u[t, :, 0])
        movable = bond >= 0
        la_new = np.full(s.shape[0], -np.inf)
        if movable.any():
            la_new[movable] = logpsi_fn(sp[movable])
        n_new = j1_pair_flags(sp, L).sum(axis=1)
        P = accept_prob(la, la_new, n_old, np.maximum(n_new, 1), hastings)
        r = u[t, :, 1]
        take = movable & (P >= r)
        s[take] = sp[take]
        la[take] = la_new[take]
        acc += take
        if trace:
            steps.append((P, r.copy(), take.copy()))
    if trace:
        return s, la, acc, steps
    return s, la, acc
