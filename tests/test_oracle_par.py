"""Pins for the oracle's thread-parallel local energy (Eq. 4-5).

`oracle.local_energy_par` (C: orc_local_energy_cnn_par) is the checker the
GPU tests use at L >= 16, so it must equal the serial definition-order
`oracle.local_energy`, which the exact-diagonalisation pins fix, and meet
the constant-psi closed form on its own.  It lists the bonds of Sec. 3.1
(Fig. 2c) in a different loop (k = 4 i + t, neighbours spread over threads,
terms summed in bond order afterwards); a slip in that decode, in its
diagonal count or in its term array would move every large-lattice parity
verdict, and fails here.
"""
import numpy as np
import pytest

import oracle
from paper_2108_13830_gb300 import inputs


def _bond_counts(sig):
    """(P1, A1, P2, A2): parallel / antiparallel J1 and J2 bond counts by np.roll."""
    s = sig.astype(np.int64)

    def cnt(nb):
        prod = s * nb
        return np.sum(prod == 1, axis=(-2, -1)), np.sum(prod == -1, axis=(-2, -1))

    right = np.roll(s, -1, axis=-1)
    down = np.roll(s, -1, axis=-2)
    p1a, a1a = cnt(right)
    p1b, a1b = cnt(down)
    p2a, a2a = cnt(np.roll(down, -1, axis=-1))
    p2b, a2b = cnt(np.roll(down, 1, axis=-1))
    return p1a + p1b, a1a + a1b, p2a + p2b, a2a + a2b


@pytest.mark.parametrize("nthreads", [1, 8])
@pytest.mark.parametrize("marshall", [True, False])
@pytest.mark.parametrize("L", [4, 6, 8, 10])
def test_parallel_equals_serial(L, marshall, nthreads):
    """Same E_loc and neighbour count as the serial oracle, stressed weights
    (std x 3, amplitude ratios far from 1), uniform and Neel-order inputs."""
    C, D = 4, 2
    theta = inputs.random_params(C, D, inputs.rng_for(40 + L), scale=3.0)
    sig = np.concatenate([inputs.uniform_configs(L, 3, inputs.rng_for(41 + L)),
                          inputs.neel_order_configs(L, 3, inputs.rng_for(42 + L))])
    J1, J2 = 1.0, 0.5
    es, ns = oracle.local_energy(L, J1, J2, C, D, theta, sig, marshall=marshall, nthreads=1)
    ep, npar = oracle.local_energy_par(L, J1, J2, C, D, theta, sig, marshall=marshall, nthreads=nthreads)
    np.testing.assert_array_equal(npar, ns)
    _, a1, _, a2 = _bond_counts(sig)
    np.testing.assert_array_equal(npar, a1 + a2)
    # the two sum the same terms in different orders
    np.testing.assert_allclose(ep, es, rtol=1e-13, atol=1e-13 * L * L)


@pytest.mark.parametrize("marshall", [True, False])
@pytest.mark.parametrize("L", [4, 8, 10])
def test_parallel_constant_psi_closed_form(L, marshall):
    """All weights 0 and last bias 1 give psi = 1, so E_loc is the integer
    closed form of the bond counts (diagonal J/4 per bond, exchange J/2 with
    the Marshall factor -1 on J1 bonds only)."""
    C, D = 4, 2
    theta = np.zeros(inputs.num_params(C, D))
    _, ob = inputs.param_offsets(C, D)[-1]
    theta[ob:ob + C] = 1.0
    J1, J2 = 1.0, 0.5
    sig = inputs.uniform_configs(L, 4, inputs.rng_for(43 + L))
    ep, npar = oracle.local_energy_par(L, J1, J2, C, D, theta, sig, marshall=marshall, nthreads=4)
    P1, A1, P2, A2 = _bond_counts(sig)
    m = -1.0 if marshall else 1.0
    closed = J1 / 4 * (P1 - A1) + J2 / 4 * (P2 - A2) + m * J1 / 2 * A1 + J2 / 2 * A2
    np.testing.assert_allclose(ep, closed, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(npar, A1 + A2)


def test_parallel_j1_only_and_j2_only():
    """J2 = 0 and J1 = 0 separate the two bond families: each run must equal
    the serial oracle, so a J1 / J2 mix-up in the k -> (site, type) decode
    shows even where the totals would agree."""
    L, C, D = 6, 4, 2
    theta = inputs.random_params(C, D, inputs.rng_for(47), scale=3.0)
    sig = inputs.uniform_configs(L, 3, inputs.rng_for(48))
    for J1, J2 in ((1.0, 0.0), (0.0, 1.0), (0.3, -0.7)):
        es, _ = oracle.local_energy(L, J1, J2, C, D, theta, sig)
        ep, _ = oracle.local_energy_par(L, J1, J2, C, D, theta, sig, nthreads=3)
        np.testing.assert_allclose(ep, es, rtol=1e-13, atol=1e-13 * L * L)
