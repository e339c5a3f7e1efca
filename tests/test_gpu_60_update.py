"""Parity of the SR parameter update (vmc_sr_update, Eq. 6) with the
oracle's theta - eta x: the context's FP64 parameters bit for bit, and
every later forward equal, bit for bit, to that of a context given the
updated vector through vmc_set_params (FP64 L = 4 and BF16 L = 16).
Also one complete SR iteration on the device at L = 4: E_loc, O_k, the CG
solve (shift 0.1, where CG parity is tight) and the update, against the
oracle's solve of the same O and E.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2108_13830_gb300 import inputs
from paper_2108_13830_gb300.binding import VMCError, VMC_OK
from gpu_util import make_ctx, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["L4_fp64", "L16_bf16"])
def test_update_matches_oracle_and_fresh_context(name):
    w = inputs.WORKLOADS[name]
    sig, theta = inputs.workload_inputs(w, batch=64)
    rng = inputs.rng_for(w.index, 12)
    x = rng.standard_normal(len(theta)) * 0.1
    eta = 0.0123
    v = make_ctx(w, theta=theta)
    v.sr_update(to_dev(x), eta)
    got = v.get_params().cpu().numpy()
    want = oracle.sr_update(theta, x, eta)
    np.testing.assert_array_equal(got, want)
    fresh = make_ctx(w, theta=want)
    s = to_dev(sig)
    np.testing.assert_array_equal(v.logpsi(s)[0].cpu().numpy(), fresh.logpsi(s)[0].cpu().numpy())
    np.testing.assert_array_equal(v.local_energy(s)[0].cpu().numpy(), fresh.local_energy(s)[0].cpu().numpy())
    with pytest.raises(VMCError):
        v.sr_update(to_dev(x), float("nan"))


def test_one_sr_iteration_on_device():
    w = inputs.WORKLOADS["L4_fp64"]
    sig, theta = inputs.workload_inputs(w)
    v = make_ctx(w, theta=theta)
    s = to_dev(sig)
    e, _ = v.local_energy(s)
    O = v.log_derivs(s, dtype=torch.float32)
    shift = 0.1                    # well conditioned: two FP64-accurate CGs agree tightly
    x, res = v.sr_solve(O, e, shift=shift, iters=w.cg_iters)
    eta = 0.05
    v.sr_update(x, eta)
    assert v.sync_status()[0] == VMC_OK
    np.testing.assert_array_equal(v.get_params().cpu().numpy(), oracle.sr_update(theta, x.cpu().numpy(), eta))
    # the device direction is the oracle's CG solve on the same O (FP32) and E
    xr, _ = oracle.sr_cg(O.cpu().numpy().astype(np.float64), e.cpu().numpy(), shift, w.cg_iters)
    np.testing.assert_allclose(x.cpu().numpy(), xr, rtol=1e-8, atol=1e-8 * np.abs(xr).max())
