"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here uses the CUDA library.  Each test names the passage of
arXiv:2108.13830 (or the mathematical fact) it pins.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import scipy.linalg as sla
import torch
import torch.nn.functional as F

import oracle
from oracle import ed
from paper_2108_13830_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([float(v) for v in line.split()])
    return rows


@pytest.fixture(scope="module")
def ed4():
    return ed.ground_state(4, 1.0, 0.5)


# ---------------------------------------------------------------- Hamiltonian

def _full_space_h(L, J1, J2):
    """H of Eq. 3 on the full 2^N space from Kronecker products of Pauli matrices.

    Built independently of oracle/ed.py (different basis, different code):
    bit i of the basis index is spin i, with |up> = bit 1 as the first basis
    vector of Eq. 1 mapped through the little-endian ordering below.
    """
    N = L * L
    sx = sp.csr_matrix(np.array([[0, 1], [1, 0]], complex))
    sy = sp.csr_matrix(np.array([[0, -1j], [1j, 0]], complex))
    sz = sp.csr_matrix(np.array([[1, 0], [0, -1]], complex))
    eye = sp.identity(2, format="csr", dtype=complex)

    def op(i, o):
        # site i is tensor factor N-1-i (so that bit i of the index is site i);
        # basis order per factor: index bit 0 -> |down>, 1 -> |up>, so flip the
        # Pauli basis (|up>, |down>) with P = sigma^x.
        P = sx
        mats = [eye] * N
        mats[N - 1 - i] = P @ o @ P
        out = mats[0]
        for m in mats[1:]:
            out = sp.kron(out, m, format="csr")
        return out

    H = sp.csr_matrix((1 << N, 1 << N), dtype=complex)
    for y in range(L):
        for x in range(L):
            i = y * L + x
            for (dy, dx, J) in ((0, 1, J1), (1, 0, J1), (1, 1, J2), (1, -1, J2)):
                j = ((y + dy) % L) * L + (x + dx) % L
                for o in (sx, sy, sz):
                    H = H + (J / 4.0) * (op(i, o) @ op(j, o))
    return H


@pytest.mark.slow
def test_ed_two_independent_hamiltonians_agree():
    """Sector H (ed.py, Pauli action) and full-space Kronecker H share E0."""
    Hf = _full_space_h(4, 1.0, 0.5)
    assert abs(Hf - Hf.getH()).max() < 1e-14
    ef = spla.eigsh(Hf.real.tocsr(), k=1, which="SA", tol=1e-12)[0][0]
    Hs, _ = ed.hamiltonian(4, 1.0, 0.5)
    es = spla.eigsh(Hs, k=1, which="SA", tol=1e-12)[0][0]
    e_lanczos, _ = ed.lanczos_ground(Hs)
    assert abs(ef - es) < 1e-9
    assert abs(e_lanczos - es) < 1e-9


def test_ed_literature_values():
    for J1, J2, e0, tol in _golden("ed_4x4.txt"):
        e, _, _, _ = ed.ground_state(4, J1, J2)
        assert abs(e - e0) < tol, (J2, e, e0)


def test_neel_diagonal_matches_paper():
    """Sec. 4.3: the Neel start sits at about -0.25 per site (J2 = 0.5)."""
    for L, J1, J2, eps in _golden("neel_diagonal.txt"):
        L = int(L)
        N = L * L
        neel = inputs.neel_state(L)
        idx = sum(1 << i for i, s in enumerate(neel.reshape(-1)) if s == 1)
        table = np.zeros(1 << N)
        table[idx] = 1.0          # psi = delta_Neel: only the diagonal survives
        e = oracle.local_energy_table(L, J1, J2, table, neel[None])[0]
        assert abs(e / N - eps) < 1e-14


def test_zero_variance_with_exact_ground_state(ed4):
    """psi = exact eigenvector => E_loc(sigma) = E0 for every sigma (Eq. 4)."""
    e0, psi, states, _ = ed4
    table = ed.table_from_sector(psi, states, 16)
    rng = np.random.default_rng(5)
    pick = rng.choice(len(states), 400, replace=False)
    cfgs = np.stack([ed.config_of_state(int(states[k]), 4) for k in pick])
    el = oracle.local_energy_table(4, 1.0, 0.5, table, cfgs)
    assert np.max(np.abs(el - e0)) < 1e-9


def test_marshall_sign_rule_at_j2_zero():
    """Eq. 9: at J2 = 0 the ground state times (-1)^{M_A} has a single sign."""
    e0, psi, states, _ = ed.ground_state(4, 1.0, 0.0)
    signs = []
    for st, v in zip(states, psi):
        if abs(v) < 1e-12:
            continue
        c = ed.config_of_state(int(st), 4)
        ma = sum(1 for y in range(4) for x in range(4) if (x + y) % 2 == 0 and c[y, x] == 1)
        signs.append(np.sign(v) * (-1) ** ma)
    assert len(set(signs)) == 1


# ---------------------------------------------------------------- CNN

def _torch_forward(L, C, D, theta, sigma):
    """Reference CNN built from torch.nn.functional (circular pad + conv2d)."""
    th = torch.tensor(theta, dtype=torch.float64)
    offs = inputs.param_offsets(C, D)
    x = torch.tensor(sigma.reshape(-1, 1, L, L), dtype=torch.float64)
    zs = []
    for l, ((co, ci), (ow, ob)) in enumerate(zip(inputs.layer_shapes(C, D), offs)):
        W = th[ow:ob].reshape(co, ci, 3, 3)
        b = th[ob:ob + co]
        z = F.conv2d(F.pad(x, (1, 1, 1, 1), mode="circular"), W, b)
        zs.append(z)
        x = F.silu(z) if l < D else z
    return zs


def _torch_logpsi(L, C, D, theta, sigma):
    z = _torch_forward(L, C, D, theta, sigma)[-1]
    return torch.log(torch.abs(z)).sum(dim=(1, 2, 3))


@pytest.mark.parametrize("L,C,D", [(4, 4, 2), (6, 8, 3), (8, 4, 1)])
def test_forward_matches_torch_conv2d(L, C, D):
    rng = inputs.rng_for(100 + L)
    theta = inputs.random_params(C, D, rng, scale=2.0)
    sig = inputs.uniform_configs(L, 3, rng)
    zt = _torch_forward(L, C, D, theta, sig)
    for b in range(3):
        zo = oracle.forward_z(L, C, D, theta, sig[b])
        for l in range(D + 1):
            np.testing.assert_allclose(zo[l], zt[l][b].numpy(), rtol=1e-12, atol=1e-12)
    la, sg = oracle.logpsi(L, C, D, theta, sig, marshall=False)
    lt = _torch_logpsi(L, C, D, theta, sig).numpy()
    np.testing.assert_allclose(la, lt, rtol=1e-12, atol=1e-10)
    zlast = zt[-1].numpy().reshape(3, -1)
    np.testing.assert_array_equal(sg, np.prod(np.sign(zlast), axis=1).astype(np.int32))


def _marshall(sig):
    L = sig.shape[-1]
    y, x = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    ma = np.sum((sig == 1) & ((x + y) % 2 == 0), axis=(-2, -1))
    return np.where(ma % 2 == 1, -1, 1)


def test_marshall_factor_in_logpsi():
    L, C, D = 4, 4, 2
    rng = inputs.rng_for(7)
    theta = inputs.random_params(C, D, rng)
    sig = inputs.uniform_configs(L, 20, rng)
    _, s0 = oracle.logpsi(L, C, D, theta, sig, marshall=False)
    _, s1 = oracle.logpsi(L, C, D, theta, sig, marshall=True)
    np.testing.assert_array_equal(s1, s0 * _marshall(sig))


def _bond_counts(sig):
    """(P1, A1, P2, A2): parallel / antiparallel J1 and J2 bonds, via np.roll."""
    s = sig.astype(np.int64)
    def cnt(sh):
        prod = s * sh
        return np.sum(prod == 1, axis=(-2, -1)), np.sum(prod == -1, axis=(-2, -1))
    right = np.roll(s, -1, axis=-1)
    down = np.roll(s, -1, axis=-2)
    dr = np.roll(down, -1, axis=-1)
    dl = np.roll(down, 1, axis=-1)
    p1a, a1a = cnt(right)
    p1b, a1b = cnt(down)
    p2a, a2a = cnt(dr)
    p2b, a2b = cnt(dl)
    return p1a + p1b, a1a + a1b, p2a + p2b, a2a + a2b


@pytest.mark.parametrize("marshall", [True, False])
@pytest.mark.parametrize("L", [4, 6, 8])
def test_constant_psi_closed_form(L, marshall):
    """All weights 0, last bias 1 => psi = 1: E_loc is an integer closed form."""
    C, D = 4, 2
    theta = np.zeros(inputs.num_params(C, D))
    ow, ob = inputs.param_offsets(C, D)[-1]
    theta[ob:ob + C] = 1.0
    J1, J2 = 1.0, 0.5
    sig = inputs.uniform_configs(L, 10, inputs.rng_for(11))
    el, nn = oracle.local_energy(L, J1, J2, C, D, theta, sig, marshall=marshall)
    P1, A1, P2, A2 = _bond_counts(sig)
    m = -1.0 if marshall else 1.0
    closed = J1 / 4 * (P1 - A1) + J2 / 4 * (P2 - A2) + m * J1 / 2 * A1 + J2 / 2 * A2
    np.testing.assert_allclose(el, closed, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(nn, A1 + A2)


def test_exact_expectation_matches_hamiltonian(ed4):
    """Eq. 4: sum |psi|^2 E_loc / sum |psi|^2 = <psi|H|psi>/<psi|psi> >= E0."""
    e0, _, states, H = ed4
    L, C, D = 4, 4, 2
    theta = inputs.random_params(C, D, inputs.rng_for(3), scale=2.0)
    cfgs = np.stack([ed.config_of_state(int(s), 4) for s in states])
    la, sg = oracle.logpsi(L, C, D, theta, cfgs)
    psi = sg * np.exp(la - la.max())
    el, _ = oracle.local_energy(L, 1.0, 0.5, C, D, theta, cfgs)
    w = psi ** 2
    e_mc = np.sum(w * el) / np.sum(w)
    e_h = (psi @ (H @ psi)) / (psi @ psi)
    assert abs(e_mc - e_h) < 1e-10 * abs(e_h)
    assert e_h >= e0 - 1e-12


def test_translation_invariance():
    L, C, D = 6, 4, 2
    rng = inputs.rng_for(13)
    theta = inputs.random_params(C, D, rng, scale=2.0)
    sig = inputs.uniform_configs(L, 2, rng)
    la, _ = oracle.logpsi(L, C, D, theta, sig, marshall=False)
    el, _ = oracle.local_energy(L, 1.0, 0.5, C, D, theta, sig)
    for dy, dx in [(1, 0), (0, 1), (2, 3)]:
        sh = np.roll(np.roll(sig, dy, axis=1), dx, axis=2)
        la2, _ = oracle.logpsi(L, C, D, theta, sh, marshall=False)
        el2, _ = oracle.local_energy(L, 1.0, 0.5, C, D, theta, sh)
        np.testing.assert_allclose(la2, la, rtol=1e-12)
        np.testing.assert_allclose(el2, el, rtol=1e-11)


def test_spin_flip_symmetry():
    """H commutes with the global flip; flipping sigma = negating W_0."""
    L, C, D = 4, 4, 2
    rng = inputs.rng_for(17)
    theta = inputs.random_params(C, D, rng, scale=2.0)
    sig = inputs.uniform_configs(L, 5, rng)
    th2 = theta.copy()
    ow, ob = inputs.param_offsets(C, D)[0]
    th2[ow:ob] *= -1
    e1, _ = oracle.local_energy(L, 1.0, 0.5, C, D, theta, -sig)
    e2, _ = oracle.local_energy(L, 1.0, 0.5, C, D, th2, sig)
    np.testing.assert_allclose(e1, e2, rtol=1e-12)


def test_last_layer_scaling():
    """Scaling the linear last layer by 2 adds C*N*log 2 to log|psi|, keeps E_loc."""
    L, C, D = 4, 4, 2
    rng = inputs.rng_for(19)
    theta = inputs.random_params(C, D, rng)
    sig = inputs.uniform_configs(L, 5, rng)
    th2 = theta.copy()
    ow, ob = inputs.param_offsets(C, D)[-1]
    th2[ow:ob + C] *= 2.0
    la, _ = oracle.logpsi(L, C, D, theta, sig)
    lb, _ = oracle.logpsi(L, C, D, th2, sig)
    np.testing.assert_allclose(lb - la, C * L * L * np.log(2.0), rtol=1e-13)
    e1, _ = oracle.local_energy(L, 1.0, 0.5, C, D, theta, sig)
    e2, _ = oracle.local_energy(L, 1.0, 0.5, C, D, th2, sig)
    np.testing.assert_allclose(e1, e2, rtol=1e-12)


# ---------------------------------------------------------------- O_k

def test_log_derivs_vs_finite_differences():
    """Eq. 5: O_k = d log|w| / d a_k, central differences in FP64 (all params)."""
    L, C, D = 4, 4, 2
    rng = inputs.rng_for(23)
    theta = inputs.random_params(C, D, rng, scale=1.5)
    sig = inputs.uniform_configs(L, 2, rng)
    O = oracle.log_derivs(L, C, D, theta, sig)
    n = theta.size
    for b in range(2):
        fd = np.zeros(n)
        for k in range(n):
            h = 1e-5 * max(1.0, abs(theta[k]))
            tp = theta.copy(); tp[k] += h
            tm = theta.copy(); tm[k] -= h
            lp, _ = oracle.logpsi(L, C, D, tp, sig[b:b + 1])
            lm, _ = oracle.logpsi(L, C, D, tm, sig[b:b + 1])
            fd[k] = (lp[0] - lm[0]) / (2 * h)
        np.testing.assert_allclose(O[b], fd, rtol=1e-6, atol=1e-8)


def test_log_derivs_vs_torch_autograd():
    L, C, D = 6, 8, 3
    rng = inputs.rng_for(29)
    theta = inputs.random_params(C, D, rng, scale=1.5)
    sig = inputs.uniform_configs(L, 3, rng)
    O = oracle.log_derivs(L, C, D, theta, sig)
    for b in range(3):
        th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
        offs = inputs.param_offsets(C, D)
        x = torch.tensor(sig[b].reshape(1, 1, L, L), dtype=torch.float64)
        for l, ((co, ci), (ow, ob)) in enumerate(zip(inputs.layer_shapes(C, D), offs)):
            z = F.conv2d(F.pad(x, (1, 1, 1, 1), mode="circular"),
                         th[ow:ob].reshape(co, ci, 3, 3), th[ob:ob + co])
            x = F.silu(z) if l < D else z
        torch.log(torch.abs(x)).sum().backward()
        np.testing.assert_allclose(O[b], th.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_log_derivs_euler_and_bias_identities():
    """z_D is linear in (W_D, b_D): sum theta_k O_k over them = C*N;
    O for b_D[c] = sum_p 1 / z_D[c, p]."""
    L, C, D = 6, 4, 2
    rng = inputs.rng_for(31)
    theta = inputs.random_params(C, D, rng, scale=2.0)
    sig = inputs.uniform_configs(L, 3, rng)
    O = oracle.log_derivs(L, C, D, theta, sig)
    ow, ob = inputs.param_offsets(C, D)[-1]
    for b in range(3):
        s = np.dot(theta[ow:ob + C], O[b, ow:ob + C])
        assert abs(s - C * L * L) < 1e-9 * C * L * L
        z = oracle.forward_z(L, C, D, theta, sig[b])[-1]
        np.testing.assert_allclose(O[b, ob:ob + C], np.sum(1.0 / z, axis=(1, 2)), rtol=1e-12)


# ---------------------------------------------------------------- SR

def _sr_case(m=64, n=40, seed=37):
    rng = np.random.default_rng(seed)
    O = rng.standard_normal((m, n)) * rng.uniform(0.1, 2.0, n) + rng.standard_normal(n)
    E = rng.standard_normal(m) + 0.3 * O[:, 0]
    return O, E


def test_sr_moments_definition():
    O, E = _sr_case()
    ob, eb, g = oracle.sr_moments(O, E)
    np.testing.assert_allclose(ob, O.mean(axis=0), rtol=1e-13)
    assert abs(eb - E.mean()) < 1e-14
    Oc = O - O.mean(axis=0)
    np.testing.assert_allclose(g, Oc.T @ (E - E.mean()) / O.shape[0], rtol=1e-11, atol=1e-13)


def test_sr_matvec_equals_explicit_covariance():
    """Eq. 7 with <.> = sample mean: M = cov(O) (biased), plus shift I."""
    O, E = _sr_case()
    m, n = O.shape
    ob, _, _ = oracle.sr_moments(O, E)
    S = np.cov(O, rowvar=False, bias=True)
    rng = np.random.default_rng(1)
    for k in range(3):
        v = rng.standard_normal(n)
        np.testing.assert_allclose(oracle.sr_matvec(O, ob, v, 1e-3), S @ v + 1e-3 * v,
                                   rtol=1e-11, atol=1e-12)
    e3 = np.zeros(n); e3[3] = 1.0
    np.testing.assert_allclose(oracle.sr_matvec(O, ob, e3, 0.0), S[:, 3], rtol=1e-11, atol=1e-13)
    # symmetric and positive semi-definite
    M = np.stack([oracle.sr_matvec(O, ob, np.eye(n)[k], 0.0) for k in range(n)], axis=1)
    np.testing.assert_allclose(M, M.T, atol=1e-12)
    assert np.linalg.eigvalsh(M).min() > -1e-10


def test_sr_matvec_centered_form():
    """The centred covariance product equals cov(O) v + shift v (textbook
    sample covariance, biased) and the uncentred form of Eq. 7 on a
    well-conditioned O; on columns whose means dwarf their spread it keeps
    its accuracy where the uncentred form cancels."""
    O, E = _sr_case()
    m, n = O.shape
    ob, _, _ = oracle.sr_moments(O, E)
    S = np.cov(O, rowvar=False, bias=True)
    rng = np.random.default_rng(2)
    for _ in range(3):
        v = rng.standard_normal(n)
        c = oracle.sr_matvec_centered(O, v, 1e-3)
        np.testing.assert_allclose(c, S @ v + 1e-3 * v, rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(c, oracle.sr_matvec(O, ob, v, 1e-3), rtol=1e-10, atol=1e-12)
    # means 1e4 x the spread: exact result known by construction (shifting
    # every column by a constant leaves the covariance unchanged)
    base = rng.standard_normal((m, n))
    big = base + 1e4 * rng.standard_normal(n)
    v = rng.standard_normal(n)
    want = oracle.sr_matvec_centered(base, v, 0.0)
    np.testing.assert_allclose(oracle.sr_matvec_centered(big, v, 0.0), want, rtol=1e-7,
                               atol=1e-9 * np.abs(want).max())


def test_cg_matches_dense_cholesky():
    """Sec. 3.2.2 solves (M + shift I) Delta = G by Cholesky; CG reaches the same x."""
    O, E = _sr_case(m=64, n=40)
    shift = 1e-2
    ob, _, g = oracle.sr_moments(O, E)
    S = np.cov(O, rowvar=False, bias=True) + shift * np.eye(O.shape[1])
    x_ref = sla.cho_solve(sla.cho_factor(S), g)
    x, res = oracle.sr_cg(O, E, shift, 200)
    np.testing.assert_allclose(x, x_ref, rtol=1e-8, atol=1e-10 * np.abs(x_ref).max())
    assert res < 1e-9


def test_dense_solve_pins():
    """The dense Cholesky solve (Sec. 3.2.2): its x satisfies
    (M + shift I) x = G through the oracle's own covariance product, equals
    the converged CG, and equals the sample-space (Woodbury) form
    x = (G - Oc^T (m shift I + Oc Oc^T)^{-1} Oc G) / shift written out with
    numpy, for m < n and m > n."""
    for m, n in ((64, 40), (30, 80)):
        O, E = _sr_case(m=m, n=n, seed=41 + m)
        shift = 1e-2
        x = oracle.sr_solve_dense(O, E, shift)
        ob, _, g = oracle.sr_moments(O, E)
        np.testing.assert_allclose(oracle.sr_matvec(O, ob, x, shift), g, rtol=1e-9, atol=1e-11 * np.abs(g).max())
        xc, res = oracle.sr_cg(O, E, shift, 400)
        np.testing.assert_allclose(x, xc, rtol=1e-7, atol=1e-9 * np.abs(x).max())
        Oc = O - O.mean(axis=0)
        K = Oc @ Oc.T
        y = np.linalg.solve(m * shift * np.eye(m) + K, Oc @ g)
        xw = (g - Oc.T @ y) / shift
        np.testing.assert_allclose(x, xw, rtol=1e-8, atol=1e-10 * np.abs(x).max())


def test_cg_single_sample_is_zero():
    """m = 1: M = 0 and G = 0, so the solve returns x = 0."""
    O, E = _sr_case(m=1, n=10)
    x, res = oracle.sr_cg(O, E, 1e-4, 50)
    assert np.all(x == 0.0) and res == 0.0
