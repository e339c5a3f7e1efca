"""Exact diagonalisation of the 4 x 4 J1-J2 model in the S^z = 0 sector.

Test infrastructure (pins the oracle's Hamiltonian and local energy).  The
Hamiltonian of Eq. 3 is assembled here directly from the Pauli matrices of
Eq. 2, acting on each basis state one operator at a time:
sigma^x flips a spin, sigma^y flips it with a factor +i (up -> down) or
-i (down -> up), sigma^z multiplies by s.  None of the oracle's local-energy
code is used.  The ground state is found by a plain Lanczos iteration with
full reorthogonalisation, written from the textbook recurrence.
"""
from __future__ import annotations

import itertools
import numpy as np
import scipy.sparse as sp

# basis bit i set  <=>  spin i up (s_i = +1); spin i sits at (y, x) = divmod(i, L)


def bonds(L):
    """[(i, j, kind)] with kind 1 (nearest) or 2 (next-nearest), each once.

    Per site: right and below neighbour (J1), down-right and down-left (J2),
    following Sec. 3.1 / Fig. 2c.
    """
    out = []
    for y in range(L):
        for x in range(L):
            i = y * L + x
            out.append((i, y * L + (x + 1) % L, 1))
            out.append((i, ((y + 1) % L) * L + x, 1))
            out.append((i, ((y + 1) % L) * L + (x + 1) % L, 2))
            out.append((i, ((y + 1) % L) * L + (x - 1) % L, 2))
    return out


def sector_states(N):
    """Basis states with N/2 up spins, as sorted integers."""
    states = []
    for ups in itertools.combinations(range(N), N // 2):
        st = 0
        for u in ups:
            st |= 1 << u
        states.append(st)
    return np.array(sorted(states), dtype=np.int64)


def _pauli_apply(op, i, state):
    """sigma^op_i |state> = amp |state'>; returns (amp, state')."""
    up = (state >> i) & 1
    if op == "z":
        return (1.0 if up else -1.0), state
    flipped = state ^ (1 << i)
    if op == "x":
        return 1.0, flipped
    # sigma^y |up> = i |down>,  sigma^y |down> = -i |up>
    return (1j if up else -1j), flipped


def hamiltonian(L, J1, J2, states=None):
    """Sparse H (Eq. 3) on the S^z = 0 sector; returns (H, states)."""
    N = L * L
    if states is None:
        states = sector_states(N)
    index = {int(s): k for k, s in enumerate(states)}
    rows, cols, vals = [], [], []
    for k, st in enumerate(states):
        st = int(st)
        acc = {}
        for (i, j, kind) in bonds(L):
            J = J1 if kind == 1 else J2
            for op in ("x", "y", "z"):
                a1, s1 = _pauli_apply(op, j, st)
                a2, s2 = _pauli_apply(op, i, s1)
                acc[s2] = acc.get(s2, 0.0) + (J / 4.0) * a1 * a2
        for s2, v in acc.items():
            if abs(v) > 0:
                assert abs(v.imag) < 1e-12
                rows.append(index[s2])
                cols.append(k)
                vals.append(v.real)
    n = len(states)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n)), states


def lanczos_ground(H, iters=400, seed=0, tol=1e-13):
    """Lowest eigenpair of symmetric H by Lanczos with full reorthogonalisation.

    Stops when the Ritz residual ||H x - theta x|| = beta_k |e_k . y| of the
    lowest Ritz pair falls below tol (the eigenvector, not just the
    eigenvalue, is converged).
    """
    n = H.shape[0]
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n)
    v /= np.linalg.norm(v)
    V = [v]
    alphas, betas = [], []
    for k in range(min(iters, n)):
        w = H @ V[-1]
        a = float(V[-1] @ w)
        alphas.append(a)
        w = w - a * V[-1] - (betas[-1] * V[-2] if betas else 0.0)
        for _ in range(2):                # full reorthogonalisation, twice
            for u in V:
                w -= (u @ w) * u
        b = float(np.linalg.norm(w))
        T = np.diag(alphas) + np.diag(betas, 1) + np.diag(betas, -1)
        ev, evec = np.linalg.eigh(T)
        if b * abs(evec[-1, 0]) < tol or b < 1e-14:
            break
        betas.append(b)
        V.append(w / b)
    T = np.diag(alphas) + np.diag(betas[:len(alphas) - 1], 1) + np.diag(betas[:len(alphas) - 1], -1)
    ev, evec = np.linalg.eigh(T)
    x = np.zeros(n)
    for c, u in zip(evec[:, 0], V):
        x += c * u
    x /= np.linalg.norm(x)
    return float(ev[0]), x


def ground_state(L=4, J1=1.0, J2=0.5):
    """(E0, psi0 over sector states, states, H) for the L x L lattice."""
    H, states = hamiltonian(L, J1, J2)
    e0, psi = lanczos_ground(H)
    return e0, psi, states, H


def table_from_sector(psi, states, N):
    """Full 2^N lookup table (zeros outside the sector) for table wavefunctions."""
    t = np.zeros(1 << N)
    t[states] = psi
    return t


def config_of_state(st, L):
    N = L * L
    return np.array([1 if (st >> i) & 1 else -1 for i in range(N)], np.int8).reshape(L, L)
