"""Pin of one full SR iteration (Eq. 5-7 and the update of Eq. 6) by exact
enumeration of the 4 x 4 S^z = 0 sector (12,870 states), no sampling.

With p(S) = |psi(S)|^2 / Z the exact moments are E = <E_loc>,
G_k = <O_k (E_loc - E)>, S = <O O^T> - <O><O>^T.  For a real wavefunction
the gradient of the variational energy is dE/dtheta = 2 G, so the step
theta - eta x with x = (S + shift I)^{-1} G changes the energy by
-2 eta G.x + O(eta^2) < 0: the update lowers the energy, at the first-order
rate fixed by G and x (shift 1e-4 as in the SR solve).  This pins the sign of G, of the step and of its
direction together with the oracle's E_loc and O_k.
"""
import numpy as np

import oracle
from oracle import ed
from paper_2108_13830_gb300 import inputs


def _sector_configs(L):
    states = ed.sector_states(L * L)
    bits = (states[:, None] >> np.arange(L * L)[None, :]) & 1
    return np.where(bits == 1, 1, -1).astype(np.int8)


def _energy(w, theta, S):
    la, _ = oracle.logpsi(w.L, w.C, w.D, theta, S)
    p = np.exp(2.0 * (la - la.max()))
    p /= p.sum()
    e, _ = oracle.local_energy(w.L, w.J1, w.J2, w.C, w.D, theta, S)
    return p, e, float(p @ e)


def test_exact_sr_step_lowers_energy_at_first_order_rate():
    w = inputs.WORKLOADS["L4_fp64"]
    _, theta = inputs.workload_inputs(w, batch=1)
    S = _sector_configs(w.L)
    p, e, E0 = _energy(w, theta, S)
    O = oracle.log_derivs(w.L, w.C, w.D, theta, S)
    Ob = p @ O
    G = (p * (e - E0)) @ O
    Oc = O - Ob
    Smat = (Oc * p[:, None]).T @ Oc
    shift = 1e-4
    x = np.linalg.solve(Smat + shift * np.eye(len(G)), G)
    slope = -2.0 * float(G @ x)
    assert slope < 0
    for eta in (1e-4, 1e-5):
        E1 = _energy(w, oracle.sr_update(theta, x, eta), S)[2]
        assert E1 < E0
        # the O(eta^2) term leaves a relative deviation ~2.5 eta here
        assert abs((E1 - E0) / eta / slope - 1.0) < 5 * eta
