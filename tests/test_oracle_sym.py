"""Pins for the oracle's rotationally symmetrised amplitude
W~(S) = sum_{i=0..3} W(T^i S) (Sec. 2.2, Eq. 10; Sec. 3.3) against facts
fixed by mathematics.  Nothing here uses the CUDA
library.
"""
import numpy as np
import pytest

import oracle
from oracle import ed
from oracle import symmetry as sym
from paper_2108_13830_gb300 import inputs


@pytest.mark.parametrize("L,scale", [(4, 1.0), (4, 3.0), (6, 2.0)])
def test_symmetrised_amplitude_is_rotation_invariant(L, scale):
    """W~(T S) = W~(S) for the 90 and 180 degree rotations (either
    direction), while the plain amplitude is not invariant."""
    C, D = 4, 2
    rng = inputs.rng_for(40 + L)
    theta = inputs.random_params(C, D, rng, scale=scale)
    sig = inputs.uniform_configs(L, 6, rng)
    la, sg = sym.logpsi_sym(L, C, D, theta, sig)
    for k in (1, 2, -1):
        r = np.rot90(sig, k, axes=(1, 2))
        la_r, sg_r = sym.logpsi_sym(L, C, D, theta, r)
        np.testing.assert_allclose(la_r, la, rtol=1e-12, atol=1e-12)
        np.testing.assert_array_equal(sg_r, sg)
    la_plain, _ = oracle.logpsi(L, C, D, theta, np.rot90(sig, 1, axes=(1, 2)))
    assert np.abs(la_plain - oracle.logpsi(L, C, D, theta, sig)[0]).max() > 1e-3


def _c4_symmetric_params(C, D, rng, scale=2.0):
    """Parameters whose every 3x3 kernel is invariant under 90-degree
    rotation (one value for the centre, one for the four edges, one for the
    four corners): the convolutions commute with the lattice rotation."""
    theta = inputs.random_params(C, D, rng, scale=scale)
    offs = inputs.param_offsets(C, D)
    for l in range(D + 1):
        wo = offs[l][0]
        cin = 1 if l == 0 else C
        W = theta[wo:wo + C * cin * 9].reshape(C, cin, 3, 3)
        edge = W[:, :, 0, 1].copy()
        corner = W[:, :, 0, 0].copy()
        for ky, kx in ((0, 1), (1, 0), (1, 2), (2, 1)):
            W[:, :, ky, kx] = edge
        for ky, kx in ((0, 0), (0, 2), (2, 0), (2, 2)):
            W[:, :, ky, kx] = corner
        theta[wo:wo + C * cin * 9] = W.reshape(-1)
    return theta


def test_rotation_invariant_network_gives_four_times_the_amplitude():
    """With C4-symmetric kernels W(T S) = W(S): the CNN commutes with T,
    product pooling is invariant, and for even L at S^z = 0 the Marshall
    factor is too (T exchanges the sublattices and N/2 is even).  Then
    W~ = 4 W exactly: log|W~| = log|W| + log 4, same sign."""
    L, C, D = 6, 4, 3
    rng = inputs.rng_for(47)
    theta = _c4_symmetric_params(C, D, rng)
    sig = inputs.uniform_configs(L, 8, rng)
    la, sg = oracle.logpsi(L, C, D, theta, sig)
    ls, ss = sym.logpsi_sym(L, C, D, theta, sig)
    np.testing.assert_allclose(ls, la + np.log(4.0), rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(ss, sg)


def test_symmetrised_energy_matches_hamiltonian():
    """Eq. 4 with W~: sum |W~|^2 E_loc / sum |W~|^2 = <W~|H|W~>/<W~|W~>
    over the 12,870 states of the 4 x 4 sector (H assembled from Pauli
    actions by the exact-diagonalisation module), and >= E0."""
    L, C, D, J1, J2 = 4, 4, 2, 1.0, 0.5
    theta = inputs.random_params(C, D, inputs.rng_for(48), scale=2.0)
    H, states = ed.hamiltonian(L, J1, J2)
    cfgs = np.stack([ed.config_of_state(int(s), L) for s in states])
    la, sg = sym.logpsi_sym(L, C, D, theta, cfgs)
    psi = sg * np.exp(la - la.max())
    el, nn = sym.local_energy_sym(L, J1, J2, C, D, theta, cfgs)
    w = psi ** 2
    e_mc = np.sum(w * el) / np.sum(w)
    e_h = (psi @ (H @ psi)) / (psi @ psi)
    assert abs(e_mc - e_h) < 1e-10 * abs(e_h)
    e0 = spla_e0(H)
    assert e_h >= e0 - 1e-12


def spla_e0(H):
    import scipy.sparse.linalg as spla
    return float(spla.eigsh(H, k=1, which="SA", tol=1e-12)[0][0])


def test_symmetrised_log_derivatives_match_finite_differences():
    """O_k = d log|W~| / d theta_k against Richardson-extrapolated central
    differences of the oracle's log|W~| (FP64, L = 4)."""
    L, C, D = 4, 4, 2
    rng = inputs.rng_for(49)
    theta = inputs.random_params(C, D, rng, scale=1.0)
    sig = inputs.uniform_configs(L, 3, rng)
    O = sym.log_derivs_sym(L, C, D, theta, sig)
    ks = np.concatenate([rng.choice(len(theta), 40, replace=False), np.arange(len(theta) - 4, len(theta))])
    for k in ks:
        h = 1e-4 * max(1.0, abs(theta[k]))

        def f(hh):
            t = theta.copy()
            t[k] += hh
            return sym.logpsi_sym(L, C, D, t, sig)[0]
        d1 = (f(h) - f(-h)) / (2 * h)
        d2 = (f(h / 2) - f(-h / 2)) / h
        fd = (4 * d2 - d1) / 3
        np.testing.assert_allclose(O[:, k], fd, rtol=1e-6, atol=1e-8)
