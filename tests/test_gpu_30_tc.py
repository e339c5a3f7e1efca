"""Parity of the tensor-core (tcgen05) path with the FP64 oracle at small
sizes, plus checks that hold exactly: the constant-psi closed form,
translation invariance, ragged vs uniform launches, and the bounded-wait
timeout path.

Tolerances.  Rounding activations and weights to a 16-bit format perturbs
each log|z| by ~2^-9 (BF16) or ~2^-12 (FP16) relative; E_loc sums ~2N
neighbour ratios whose errors are nearly independent, so the per-site error
falls with L.  For the 16-channel / 6-layer and 32-channel / 6-8-layer nets
used here, a CPU emulation of the rounding gives E_loc/site errors of
1e-4 .. 2.3e-3 in BF16 at L = 6..12 and <= 1.5e-4 in FP16.  Hence: FP16
parity at 5e-4 per site for small lattices, BF16 at 3e-3; BF16 at 5e-4 is
checked at the L = 16 and L = 24 workloads (test_gpu_40_full.py).
Networks with only 2-3 layers produce last-layer outputs near zero, where
any 16-bit rounding moves log|psi| by O(1); they are used only for checks
that hold exactly (translation, tile choices)."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2108_13830_gb300 import inputs
from paper_2108_13830_gb300.binding import VMC, VMC_OK, VMC_ERR_TIMEOUT
from gpu_util import bond_counts, make_ctx, to_dev

pytestmark = pytest.mark.gpu

FP16_TOL = 5e-4         # |E_gpu - E_oracle| / N per sample
BF16_SMALL_TOL = 3e-3   # BF16 on small lattices (see the module docstring)


def _small(L, C, D, B, seed, kind="uniform", scale=1.0, prec="bf16"):
    w = inputs.Workload(f"t{L}", L, C, D, prec, B, kind=kind, index=50 + seed)
    sig, theta = inputs.workload_inputs(w, scale=scale)
    return w, sig, theta


@pytest.mark.parametrize("L,C,D,B,prec", [(8, 32, 8, 48, "bf16"), (12, 32, 8, 24, "bf16"), (6, 32, 6, 48, "bf16"),
                                          (10, 16, 6, 48, "fp16"), (8, 16, 6, 48, "fp16"), (4, 16, 6, 64, "fp16"),
                                          (8, 32, 8, 48, "fp16")])
def test_tc_local_energy_small(L, C, D, B, prec):
    w, sig, theta = _small(L, C, D, B, L + C + D, prec=prec)
    tol = FP16_TOL if prec == "fp16" else BF16_SMALL_TOL
    v = make_ctx(w, theta=theta)
    e, nn = v.local_energy(to_dev(sig))
    assert v.sync_status()[0] == VMC_OK
    e = e.cpu().numpy()
    a1, a2 = bond_counts(sig)
    np.testing.assert_array_equal(nn.cpu().numpy(), a1 + a2)
    re, _ = oracle.local_energy(L, w.J1, w.J2, C, D, theta, sig)
    err = np.abs(e - re) / (L * L)
    assert err.max() <= tol, err.max()


@pytest.mark.parametrize("prec,tol", [("bf16", 0.05), ("fp16", 0.01)])
def test_tc_logpsi_small(prec, tol):
    """log|psi| sums C N = 2048 log terms; each carries ~2^-9 (BF16) or ~2^-12
    (FP16) relative rounding of its inputs, so the sum is off by a few 1e-2
    (BF16) or a few 1e-3 (FP16).  Signs must match exactly."""
    w, sig, theta = _small(8, 32, 8, 64, 7, prec=prec)
    v = make_ctx(w, theta=theta)
    la, sg = v.logpsi(to_dev(sig))
    ra, rs = oracle.logpsi(w.L, w.C, w.D, theta, sig)
    np.testing.assert_array_equal(sg.cpu().numpy().astype(np.int32), rs)
    assert np.abs(la.cpu().numpy() - ra).max() <= tol


@pytest.fixture(scope="module")
def l32_reference():
    """Inputs of the L = 32 check (the same for both precisions) and the
    oracle's log|psi| of all samples and E_loc of the first, computed once."""
    w, sig, theta = _small(32, 32, 6, 6, 32)
    ra, rs = oracle.logpsi(w.L, w.C, w.D, theta, sig)
    re, rn = oracle.local_energy_par(w.L, w.J1, w.J2, w.C, w.D, theta, sig[:1], nthreads=os.cpu_count() or 4)
    return sig, theta, ra, rs, re, rn


@pytest.mark.parametrize("prec,la_tol,e_tol", [("bf16", 0.25, BF16_SMALL_TOL), ("fp16", 0.05, FP16_TOL)])
def test_tc_largest_lattice_L32(prec, la_tol, e_tol, l32_reference):
    """L = 32 is the largest lattice of the tensor-core path; with C = 32
    only the one-slab geometries fit shared memory.  log|psi| and sign
    against the FP64 oracle: C N = 32768 log terms, 16 times those of the
    L = 8 check, so the random rounding error is ~4 times larger (bounds
    0.25 BF16, 0.05 FP16).  E_loc of one sample (~2000 neighbour
    configurations; the plain FP32 path does not fit L = 32 with C = 32)
    against the oracle, with the small-lattice tolerances."""
    sig, theta, ra, rs, re, rn = l32_reference
    w = inputs.Workload("t32", 32, 32, 6, prec, 6, kind="uniform", index=50 + 32)
    v = make_ctx(w, theta=theta)
    assert v.get_tiles(32)["slabs"] == 1
    la, sg = v.logpsi(to_dev(sig))
    np.testing.assert_array_equal(sg.cpu().numpy().astype(np.int32), rs)
    assert np.abs(la.cpu().numpy() - ra).max() <= la_tol
    e, nn = v.local_energy(to_dev(sig[:1]))
    np.testing.assert_array_equal(nn.cpu().numpy(), rn)
    assert (np.abs(e.cpu().numpy() - re) / (w.L * w.L)).max() <= e_tol
    assert v.sync_status()[0] == VMC_OK


@pytest.mark.parametrize("L", [6, 8, 16])
def test_bf16_constant_psi_closed_form(L):
    """All weights zero and last bias 1: psi = 1 exactly in BF16, so E_loc is
    the integer closed form (J1/4)(P1-A1) + (J2/4)(P2-A2) - (J1/2)A1 + (J2/2)A2."""
    C, D = 32, 2
    w = inputs.Workload("c", L, C, D, "bf16", 32)
    theta = np.zeros(inputs.num_params(C, D))
    ow, ob = inputs.param_offsets(C, D)[-1]
    theta[ob:ob + C] = 1.0
    sig = inputs.uniform_configs(L, 32, inputs.rng_for(60 + L))
    v = make_ctx(w, theta=theta)
    e, nn = v.local_energy(to_dev(sig))
    a1, a2 = bond_counts(sig)
    N2 = 2 * L * L
    closed = 0.25 * (N2 - 2 * a1) + 0.125 * (N2 - 2 * a2) - 0.5 * a1 + 0.25 * a2
    np.testing.assert_array_equal(e.cpu().numpy(), closed)


def test_bf16_translation_invariance():
    w, sig, theta = _small(10, 16, 4, 16, 9)
    v = make_ctx(w, theta=theta)
    la, _ = v.logpsi(to_dev(sig))
    e, _ = v.local_energy(to_dev(sig))
    sh = np.ascontiguousarray(np.roll(np.roll(sig, 3, axis=1), -2, axis=2))
    la2, _ = v.logpsi(to_dev(sh))
    e2, _ = v.local_energy(to_dev(sh))
    # every z is bitwise the same per cell; only the order of the FP64 sums moves
    np.testing.assert_allclose(la2.cpu().numpy(), la.cpu().numpy(), rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(e2.cpu().numpy(), e.cpu().numpy(), rtol=1e-9, atol=1e-9)


def test_ragged_equals_uniform_and_oracle():
    """The mixed-size workload (16 channels, 6 layers) runs with FP16 operands."""
    w = inputs.WORKLOADS["ragged_8_16"]
    packed, offs, Ls, theta = inputs.ragged_inputs(w, per_L=6)
    v = make_ctx(w, theta=theta, L=16)
    e, nn = v.local_energy_ragged(to_dev(packed), to_dev(offs), to_dev(Ls), 16)
    assert v.sync_status()[0] == VMC_OK
    e = e.cpu().numpy()
    for L in w.Ls:
        idx = np.where(Ls == L)[0]
        cfg = np.stack([packed[offs[b]:offs[b] + L * L].reshape(L, L) for b in idx])
        vu = make_ctx(w, theta=theta, L=L)
        eu, _ = vu.local_energy(to_dev(cfg))
        np.testing.assert_allclose(e[idx], eu.cpu().numpy(), rtol=1e-12, atol=1e-10)
        re, rn = oracle.local_energy(L, w.J1, w.J2, w.C, w.D, theta, cfg[:2])
        assert (np.abs(e[idx[:2]] - re) / (L * L)).max() <= FP16_TOL
        np.testing.assert_array_equal(nn.cpu().numpy()[idx[:2]], rn)


def test_ragged_launch_replays_from_a_cuda_graph():
    """The mixed-size persistent launch captured once in a CUDA graph and
    replayed gives the eager result bit for bit (the counter reset is part
    of the captured work)."""
    w = inputs.WORKLOADS["ragged_8_16"]
    packed, offs, Ls, theta = inputs.ragged_inputs(w, per_L=8)
    v = make_ctx(w, theta=theta, L=16)
    pk, of, Lt = to_dev(packed), to_dev(offs), to_dev(Ls)
    ref, _ = v.local_energy_ragged(pk, of, Lt, 16)
    torch.cuda.synchronize()
    out = torch.empty_like(ref)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        v.local_energy_ragged(pk, of, Lt, 16, out=out, n_nbr=False)
    for _ in range(2):
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    assert v.sync_status()[0] == VMC_OK


@pytest.mark.parametrize("G,S,P", [(1, 1, 1), (1, 2, 2), (3, 2, 3), (2, 1, 4), (5, 2, 1), (4, 1, 3)])
def test_bf16_tile_choices_agree(G, S, P):
    """Every slab geometry and lane packing gives bitwise the same energies:
    each output cell sums its nine taps in the same order whatever its
    position in a TMEM lane."""
    w, sig, theta = _small(8, 32, 3, 40, 11)
    v = make_ctx(w, theta=theta)
    ref, _ = v.local_energy(to_dev(sig))
    v.set_tiles(8, slab_configs=G, slabs=S, lane_cells=P)
    got, _ = v.local_energy(to_dev(sig))
    assert v.get_tiles(8)["lane_cells"] == P
    assert torch.equal(ref, got)


@pytest.mark.parametrize("P", [2, 4, 6, 8])
def test_bf16_c16_lane_packings_agree(P):
    """C = 16 packs an even number of cells per lane; all give the same bits."""
    w, sig, theta = _small(8, 16, 2, 24, 17)
    v = make_ctx(w, theta=theta)
    ref, _ = v.local_energy(to_dev(sig))
    v.set_tiles(8, lane_cells=P)
    got, _ = v.local_energy(to_dev(sig))
    assert torch.equal(ref, got)


def test_bf16_autotune_keeps_results():
    w, sig, theta = _small(8, 32, 3, 40, 12)
    v = make_ctx(w, theta=theta)
    ref, _ = v.local_energy(to_dev(sig))
    tiles = v.autotune(8, probe_B=64)
    assert tiles["slab_configs"] >= 1
    got, _ = v.local_energy(to_dev(sig))
    assert torch.equal(ref, got)


def test_wait_timeout_reports_status():
    w, sig, theta = _small(8, 32, 3, 8, 13)
    v = make_ctx(w, theta=theta)
    v.debug_wait_timeout(2_000_000)          # 2 ms on a barrier nothing arrives on
    rc, _ = v.sync_status()
    assert rc == VMC_ERR_TIMEOUT
    e, _ = v.local_energy(to_dev(sig))       # the context stays usable
    assert v.sync_status()[0] == VMC_OK
    assert np.all(np.isfinite(e.cpu().numpy()))


def test_nonfinite_parameters_are_flagged():
    w, sig, theta = _small(8, 32, 3, 8, 14)
    th = theta.copy()
    th[5] = np.nan
    v = make_ctx(w, theta=th)
    e, _ = v.local_energy(to_dev(sig))
    rc, nf = v.sync_status()
    assert rc == -3 and nf == 8
    assert np.all(np.isnan(e.cpu().numpy()))
