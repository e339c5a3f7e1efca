"""The whole method on the oracle, pinned by exact diagonalisation: 40 SR
iterations on the 4 x 4 lattice at J2 = 0.5 (Sec. 2-3: Metropolis samples of
512 chains, L^2 transitions apart (Sec. 3.1), E_loc, O_k, the CG solve of
(S + shift I) x = G and the update theta - eta x of Eq. 6) take the exact
variational energy of the CNN from its random-initialisation value to
within 0.02 per site of the ground-state energy E0 = -8.457923 (the
exact-diagonalisation value of the golden file), never below it.  The
chains use the Hastings factor so that they sample |psi|^2.
"""
import os

import numpy as np

import oracle
from oracle import ed
from oracle import metropolis as mh
from paper_2108_13830_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "ed_4x4.txt")


def e0_4x4(J2):
    for line in open(GOLD):
        line = line.strip()
        if line and not line.startswith("#"):
            _, j2, e0 = (float(v) for v in line.split()[:3])   # columns J1 J2 E0 tolerance
            if abs(j2 - J2) < 1e-12:
                return e0
    raise KeyError(J2)


def exact_energy(w, theta):
    """<psi|H|psi> / <psi|psi> per site by enumerating the S^z = 0 sector."""
    states = ed.sector_states(w.L * w.L)
    bits = (states[:, None] >> np.arange(w.L * w.L)[None, :]) & 1
    S = np.where(bits == 1, 1, -1).astype(np.int8)
    la, _ = oracle.logpsi(w.L, w.C, w.D, theta, S)
    p = np.exp(2.0 * (la - la.max()))
    e, _ = oracle.local_energy(w.L, w.J1, w.J2, w.C, w.D, theta, S)
    return float(p @ e / p.sum()) / (w.L * w.L)


ITERS, CHAINS, SHIFT, ETA = 40, 512, 1e-3, 0.05


def test_oracle_vmc_reaches_ground_state():
    w = inputs.WORKLOADS["L4_fp64"]
    L, C, D = w.L, w.C, w.D
    _, theta = inputs.workload_inputs(w, batch=1)
    rng = inputs.rng_for(w.index, 20)
    s = inputs.neel_order_configs(L, CHAINS, rng).reshape(CHAINS, -1)
    e_start = exact_energy(w, theta)

    def lp_of(th):
        return lambda c: oracle.logpsi(L, C, D, th, c)[0]
    lp = lp_of(theta)
    s, _, _ = mh.metropolis(s, lp(s), inputs.chain_uniforms(4 * L * L, CHAINS, rng), lp, L, hastings=True)
    for _ in range(ITERS):
        lp = lp_of(theta)
        s, _, _ = mh.metropolis(s, lp(s), inputs.chain_uniforms(L * L, CHAINS, rng), lp, L, hastings=True)
        e, _ = oracle.local_energy(L, w.J1, w.J2, C, D, theta, s)
        O = oracle.log_derivs(L, C, D, theta, s)
        x, _ = oracle.sr_cg(O, e, SHIFT, 50)
        theta = oracle.sr_update(theta, x, ETA)
    e_end = exact_energy(w, theta)
    e0 = e0_4x4(w.J2) / (L * L)
    assert e_end >= e0 - 1e-12
    assert e_end < e0 + 0.02
    assert e_start - e_end > 0.2
