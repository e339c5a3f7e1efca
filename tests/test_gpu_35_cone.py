"""Light-cone evaluation of the exchange neighbours (vmc_set_light_cone).

The filters are 3 x 3 (Sec. 2.2), so after layer l a neighbour sigma' of
sigma differs from sigma's activations only within l + 1 cells of the
exchanged pair; the library recomputes that window and copies the rest of
each layer from the parent.  Every evaluated cell sums the same taps in the
same order as the plain forward and the pooling adds the last layer in
lattice order, so E_loc must equal the plain evaluation bit for bit; it is
also checked against the FP64 oracle (Eq. 4-5) at the 16-bit tolerances.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2108_13830_gb300 import inputs
from paper_2108_13830_gb300.binding import VMC_ERR_NONFINITE, VMC_OK
from gpu_util import bond_counts, make_ctx, to_dev

pytestmark = pytest.mark.gpu

FP16_TOL = 5e-4
BF16_SMALL_TOL = 3e-3


def _both(v, s):
    """(E_loc, n_nbr) with the light cone on, then with the plain evaluation."""
    v.set_light_cone(True)
    assert v.light_cone_active
    e1, n1 = v.local_energy(s)
    r1 = v.sync_status()
    v.set_light_cone(False)
    assert not v.light_cone_active
    e0, n0 = v.local_energy(s)
    r0 = v.sync_status()
    v.set_light_cone(True)
    return (e1.cpu().numpy(), n1.cpu().numpy(), r1), (e0.cpu().numpy(), n0.cpu().numpy(), r0)


@pytest.mark.parametrize("L,C,D,prec,kind,scale,marshall", [
    (6, 16, 1, "bf16", "uniform", 1.0, True),
    (6, 32, 6, "fp16", "neel", 1.0, True),
    (8, 32, 2, "bf16", "uniform", 3.0, False),
    (8, 16, 2, "fp16", "neel", 1.0, True),
    (10, 16, 6, "fp16", "uniform", 1.0, True),
    (10, 32, 3, "bf16", "neel", 3.0, True),
    (12, 32, 4, "bf16", "uniform", 1.0, True),
    (12, 16, 8, "fp16", "neel", 1.0, False),
    (14, 32, 5, "fp16", "uniform", 1.0, True),
    (16, 32, 8, "bf16", "uniform", 1.0, True),
    (20, 16, 8, "bf16", "neel", 1.0, True),
])
def test_cone_bitwise_equals_plain(L, C, D, prec, kind, scale, marshall):
    w = inputs.Workload(f"cone{L}", L, C, D, prec, 96, kind=kind, index=60 + L + D)
    sig, theta = inputs.workload_inputs(w, scale=scale)
    v = make_ctx(w, theta=theta, marshall=marshall)
    (e1, n1, r1), (e0, n0, r0) = _both(v, to_dev(sig))
    assert r1 == r0
    np.testing.assert_array_equal(n1, n0)
    a1, a2 = bond_counts(sig)
    np.testing.assert_array_equal(n1, a1 + a2)
    np.testing.assert_array_equal(e1, e0)


@pytest.mark.parametrize("L,C,D,prec", [(10, 16, 6, "fp16"), (12, 32, 8, "bf16"), (8, 32, 8, "fp16")])
def test_cone_vs_oracle(L, C, D, prec):
    w = inputs.Workload(f"coneo{L}", L, C, D, prec, 8, index=70 + L)
    sig, theta = inputs.workload_inputs(w)
    v = make_ctx(w, theta=theta)
    assert v.light_cone_active
    e, nn = v.local_energy(to_dev(sig))
    assert v.sync_status()[0] == VMC_OK
    re, rn = oracle.local_energy(L, w.J1, w.J2, C, D, theta, sig)
    np.testing.assert_array_equal(nn.cpu().numpy(), rn)
    tol = FP16_TOL if prec == "fp16" else BF16_SMALL_TOL
    assert (np.abs(e.cpu().numpy() - re) / (L * L)).max() <= tol


def test_cone_inactive_when_window_stays_small():
    """L = 16 with D = 4: the window (2D + 4 = 12) never covers the lattice,
    so the plain evaluation runs, enabled or not.  (A 5-layer net leaves
    last-layer outputs near zero, where 16-bit rounding moves log|psi| most:
    the oracle check takes the small-lattice BF16 bound.)"""
    w = inputs.Workload("cone_off", 16, 32, 4, "fp16", 4, index=75)
    sig, theta = inputs.workload_inputs(w)
    v = make_ctx(w, theta=theta)
    assert not v.light_cone_active
    e, _ = v.local_energy(to_dev(sig))
    assert v.sync_status()[0] == VMC_OK
    v.set_light_cone(False)
    e0, _ = v.local_energy(to_dev(sig))
    np.testing.assert_array_equal(e.cpu().numpy(), e0.cpu().numpy())
    re, _ = oracle.local_energy_par(16, 1.0, 0.5, 32, 4, theta, sig, nthreads=8)
    assert (np.abs(e.cpu().numpy() - re) / 256).max() <= BF16_SMALL_TOL


def test_cone_degenerate_samples():
    """A configuration without antiparallel bonds (E_loc = the diagonal
    term, no neighbour) and psi = 0 (NaN, counted) next to ordinary ones:
    the same results and status as the plain evaluation."""
    L, C, D = 8, 32, 3
    rng = inputs.rng_for(79)
    theta = inputs.random_params(C, D, rng)
    sig = inputs.uniform_configs(L, 5, rng)
    sig = np.concatenate([sig, np.ones((1, L, L), np.int8), -np.ones((1, L, L), np.int8)])
    w = inputs.Workload("cone_deg", L, C, D, "bf16", len(sig), index=79)
    v = make_ctx(w, theta=theta)
    (e1, n1, r1), (e0, n0, r0) = _both(v, to_dev(sig))
    assert r1 == r0 == (VMC_OK, 0)
    np.testing.assert_array_equal(e1, e0)
    assert n1[5] == 0 and n1[6] == 0
    assert e1[5] == 0.25 * 2 * L * L * (1.0 + 0.5)
    # psi = 0: one channel of the last layer identically zero
    wo, bo = inputs.param_offsets(C, D)[D]
    th0 = theta.copy()
    th0[wo:bo] = 0.0
    th0[bo:bo + C] = 1.0
    th0[bo] = 0.0
    v0 = make_ctx(w, theta=th0)
    (e1, n1, r1), (e0, n0, r0) = _both(v0, to_dev(sig))
    assert r1 == r0 == (VMC_ERR_NONFINITE, len(sig))
    assert np.all(np.isnan(e1)) and np.all(np.isnan(e0))
    np.testing.assert_array_equal(n1, n0)


def test_cone_full_size_L24_and_L16():
    """The bench workloads: every sample bit for bit the plain evaluation."""
    for name in ("L24_bf16_sr", "L16_bf16"):
        w = inputs.WORKLOADS[name]
        sig, theta = inputs.workload_inputs(w)
        v = make_ctx(w, theta=theta)
        (e1, n1, r1), (e0, n0, r0) = _both(v, to_dev(sig))
        assert r1 == r0 == (VMC_OK, 0)
        np.testing.assert_array_equal(n1, n0)
        np.testing.assert_array_equal(e1, e0)
        v.close()
        torch.cuda.empty_cache()


def test_cone_parent_chunks():
    """L = 32, D = 14 keeps 0.92 MB of activations per parent, so 2400
    samples run as two parent chunks (2 GiB workspace cap)."""
    w = inputs.Workload("cone32", 32, 32, 14, "bf16", 2400, index=77)
    sig, theta = inputs.workload_inputs(w)
    v = make_ctx(w, theta=theta)
    (e1, n1, r1), (e0, n0, r0) = _both(v, to_dev(sig))
    assert r1 == r0 == (VMC_OK, 0)
    np.testing.assert_array_equal(n1, n0)
    np.testing.assert_array_equal(e1, e0)


@pytest.mark.parametrize("L,C,D,prec", [(16, 32, 8, "bf16"), (10, 16, 6, "fp16")])
def test_cone_tile_choices_and_autotune(L, C, D, prec):
    """Every explicit light-cone tile choice that fits, and the autotuned
    one, give the plain evaluation's results bit for bit."""
    w = inputs.Workload(f"conet{L}", L, C, D, prec, 64, index=80 + L)
    sig, theta = inputs.workload_inputs(w)
    v = make_ctx(w, theta=theta)
    s = to_dev(sig)
    v.set_light_cone(False)
    e0, _ = v.local_energy(s)
    v.set_light_cone(True)
    e0 = e0.cpu().numpy()
    tried = 0
    for S in (1, 2):
        for P in (2, 3, 4):
            for G in (1, 2, 3):
                try:
                    v.set_cone_tiles(slab_configs=G, slabs=S, lane_cells=P)
                except Exception:
                    continue
                got = v.get_cone_tiles()
                assert (got["slabs"], got["lane_cells"], got["slab_configs"]) == (S, P, G)
                e1, _ = v.local_energy(s)
                assert v.sync_status()[0] == VMC_OK
                np.testing.assert_array_equal(e1.cpu().numpy(), e0)
                tried += 1
    assert tried >= 4
    v.set_cone_tiles()
    v.autotune(L, probe_B=256)
    e2, _ = v.local_energy(s)
    assert v.sync_status()[0] == VMC_OK
    np.testing.assert_array_equal(e2.cpu().numpy(), e0)


def test_cone_ragged_batch_bitwise():
    """A mixed batch of sides 4 .. 16 (one persistent launch walking the
    samples largest side first): the light cone gives the plain ragged
    evaluation's results bit for bit, and sides beyond L_max stay NaN with
    VMC_ERR_ARG."""
    w = inputs.Workload("cone_rag", 16, 16, 6, "fp16", 96, kind="ragged", Ls=(4, 6, 8, 12, 16), index=83)
    packed, offs, Ls, theta = inputs.ragged_inputs(w)
    v = make_ctx(w, theta=theta, L=16)
    pk, of, Lt = to_dev(packed), to_dev(offs), to_dev(Ls)
    v.set_light_cone(True)
    e1, n1 = v.local_energy_ragged(pk, of, Lt, 16)
    r1 = v.sync_status()
    v.set_light_cone(False)
    e0, n0 = v.local_energy_ragged(pk, of, Lt, 16)
    r0 = v.sync_status()
    v.set_light_cone(True)
    assert r1 == r0 == (VMC_OK, 0)
    np.testing.assert_array_equal(n1.cpu().numpy(), n0.cpu().numpy())
    np.testing.assert_array_equal(e1.cpu().numpy(), e0.cpu().numpy())
    # the same launch with L_max = 12: the side-16 samples are refused
    e2, _ = v.local_energy_ragged(pk, of, Lt, 12)
    r2 = v.sync_status()
    from paper_2108_13830_gb300.binding import VMC_ERR_ARG
    assert r2[0] == VMC_ERR_ARG
    e2 = e2.cpu().numpy()
    big = Ls == 16
    assert np.all(np.isnan(e2[big]))
    np.testing.assert_array_equal(e2[~big], e0.cpu().numpy()[~big])


def test_launch_timing_records_the_light_cone_launches():
    """vmc_set_launch_timing: one record per tensor-core launch of the calls
    made while it is on (here the parent pass and the light-cone pass of one
    local-energy call), each with a positive duration, in launch order."""
    w = inputs.Workload("cone_timing", 12, 32, 4, "bf16", 64, index=84)
    sig, theta = inputs.workload_inputs(w)
    v = make_ctx(w, theta=theta)
    s = to_dev(sig)
    v.local_energy(s)
    v.set_launch_timing(True)
    v.local_energy(s)
    t = v.launch_timings()
    v.set_launch_timing(False)
    assert [name for name, _ in t] == ["tc_eloc_kernel<parent pass>", "tc_eloc_kernel<light cone>"]
    assert all(ms > 0 for _, ms in t)
    v.set_light_cone(False)
    v.set_launch_timing(True)
    v.local_energy(s)
    t = v.launch_timings()
    assert [name for name, _ in t] == ["tc_eloc_kernel"]


@pytest.mark.parametrize("S,P", [(1, 4), (2, 2), (1, 8)])
def test_cone_ragged_explicit_tiles(S, P):
    """vmc_set_cone_tiles applies to the ragged light-cone launch (slabs and
    P for the launch, each side's windows per slab from the cost model):
    every choice gives the plain ragged evaluation's results bit for bit."""
    w = inputs.Workload("cone_ragt", 16, 16, 6, "fp16", 64, kind="ragged", Ls=(6, 8, 12, 16), index=85)
    packed, offs, Ls, theta = inputs.ragged_inputs(w)
    v = make_ctx(w, theta=theta, L=16)
    pk, of, Lt = to_dev(packed), to_dev(offs), to_dev(Ls)
    v.set_light_cone(False)
    e0, n0 = v.local_energy_ragged(pk, of, Lt, 16)
    v.set_light_cone(True)
    v.set_cone_tiles(slabs=S, lane_cells=P)
    e1, n1 = v.local_energy_ragged(pk, of, Lt, 16)
    assert v.sync_status() == (VMC_OK, 0)
    np.testing.assert_array_equal(n1.cpu().numpy(), n0.cpu().numpy())
    np.testing.assert_array_equal(e1.cpu().numpy(), e0.cpu().numpy())
