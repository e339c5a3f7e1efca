"""Rotationally symmetrised amplitude (test infrastructure).

Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this module; it shares no code with the CUDA library.

Sec. 2.2 of arXiv:2108.13830 (Eq. 10) enforces the
rotational symmetry of the ground state by summing the amplitude over the
four 90-degree rotations T of the L x L lattice:

    W~(S) = sum_{i=0..3} W(T^i S),   W(S) = (-1)^{M_A} W_CNN(S).

Sec. 3.3 applies it in the last fine-tuning stage at four times the cost.
Here:
 - log|W~| and sgn W~ come from the four signed amplitudes, summed in FP64
   after factoring out the largest |W(T^i S)|;
 - the local energy of Eq. 4-5 uses W~ for S and for every exchange
   neighbour S', with the full signs;
 - O_k = d log|W~| / d theta_k = sum_i (W(T^i S) / W~(S)) O_k(T^i S),
   since dW/dtheta = W dlog|W|/dtheta for a real amplitude.
The sum runs over the set {T^i S}, so the direction of T does not matter;
T^1 here is numpy's rot90 (counter-clockwise).
"""
from __future__ import annotations

import numpy as np

import oracle
from oracle import ed


def rotations(sigma, L):
    """[B, 4, L, L]: T^i S for i = 0..3."""
    s = np.asarray(sigma, dtype=np.int8).reshape(-1, L, L)
    return np.stack([np.rot90(s, i, axes=(1, 2)) for i in range(4)], axis=1)


def combine(la, sg):
    """(log|W~|, sgn W~) from the four (log|W|, sgn W) of each row of [B, 4]."""
    la = np.asarray(la, dtype=np.float64)
    sg = np.asarray(sg, dtype=np.float64)
    m = np.max(np.where(sg != 0, la, -np.inf), axis=1)
    with np.errstate(invalid="ignore", divide="ignore"):
        t = np.where(sg != 0, sg * np.exp(la - m[:, None]), 0.0).sum(axis=1)
        out_la = m + np.log(np.abs(t))
    out_sg = np.sign(t).astype(np.int32)
    out_la[out_sg == 0] = -np.inf
    return out_la, out_sg


def logpsi_sym(L, C, D, theta, sigma, marshall=True):
    """(log|W~| [B], sgn W~ [B])."""
    R = rotations(sigma, L)
    B = R.shape[0]
    la, sg = oracle.logpsi(L, C, D, theta, R.reshape(4 * B, L, L), marshall=marshall)
    return combine(la.reshape(B, 4), sg.reshape(B, 4))


def exchange_neighbours(s, L, J1, J2):
    """Diagonal energy and the (S', matrix element) pairs of one configuration.

    Bonds per site as in Sec. 3.1 / Fig. 2c (the exact-diagonalisation
    module's list); diagonal (J/4) s_i s_j; an antiparallel pair's exchange
    has element J/2 (Eq. 2-3).
    """
    s = np.asarray(s, dtype=np.int8).reshape(L * L)
    diag = 0.0
    nbrs, elems = [], []
    for i, j, kind in ed.bonds(L):
        J = J1 if kind == 1 else J2
        diag += 0.25 * J * float(s[i]) * float(s[j])
        if s[i] != s[j]:
            t = s.copy()
            t[i], t[j] = s[j], s[i]
            nbrs.append(t)
            elems.append(0.5 * J)
    return diag, nbrs, elems


def local_energy_sym(L, J1, J2, C, D, theta, sigma, marshall=True):
    """(E_loc [B], exchange-neighbour counts [B]) with the symmetrised amplitude."""
    sig = np.asarray(sigma, dtype=np.int8).reshape(-1, L * L)
    B = sig.shape[0]
    diags, counts, allc, alle = np.zeros(B), np.zeros(B, np.int32), [], []
    for b in range(B):
        d, nb, el = exchange_neighbours(sig[b], L, J1, J2)
        diags[b] = d
        counts[b] = len(nb)
        allc.append(sig[b])
        allc.extend(nb)
        alle.append(el)
    la, sg = logpsi_sym(L, C, D, theta, np.stack(allc), marshall=marshall)
    e = np.zeros(B)
    k = 0
    for b in range(B):
        la0, sg0 = la[k], sg[k]
        acc = 0.0
        for q, el in enumerate(alle[b]):
            r = k + 1 + q
            acc += el * float(sg[r] * sg0) * np.exp(la[r] - la0)
        e[b] = diags[b] + acc if sg0 != 0 else np.nan
        k += 1 + counts[b]
    return e, counts


def log_derivs_sym(L, C, D, theta, sigma, marshall=True):
    """O [B, n] = d log|W~| / d theta, FP64."""
    R = rotations(sigma, L)
    B = R.shape[0]
    flat = R.reshape(4 * B, L, L)
    la, sg = oracle.logpsi(L, C, D, theta, flat, marshall=marshall)
    la, sg = la.reshape(B, 4), sg.reshape(B, 4).astype(np.float64)
    lt, st = combine(la, sg)
    Ol = oracle.log_derivs(L, C, D, theta, flat).reshape(B, 4, -1)
    w = sg * st[:, None] * np.exp(la - lt[:, None])      # W(T^i S) / W~(S)
    return np.einsum("bi,bik->bk", w, Ol)
