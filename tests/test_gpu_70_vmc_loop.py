"""The whole method through the library: 40 SR iterations on the 4 x 4
lattice at J2 = 0.5 with every step on the GPU (vmc_metropolis with the
Hastings factor, vmc_local_energy, vmc_log_derivs, vmc_sr_solve,
vmc_sr_update), the same schedule as the oracle's run in
test_oracle_vmc_loop.py.  The exact variational energy of the final
parameters (oracle enumeration of the 12,870-state sector) must lie within
0.02 per site above the exact ground-state energy, never below it, and
0.2 per site below that of the initial parameters.
"""
import pytest
import torch

from paper_2108_13830_gb300 import inputs
from paper_2108_13830_gb300.binding import VMC_OK
from gpu_util import make_ctx, to_dev
from test_oracle_vmc_loop import CHAINS, ETA, ITERS, SHIFT, e0_4x4, exact_energy

pytestmark = pytest.mark.gpu


def test_device_vmc_reaches_ground_state():
    w = inputs.WORKLOADS["L4_fp64"]
    L = w.L
    _, theta = inputs.workload_inputs(w, batch=1)
    rng = inputs.rng_for(w.index, 20)
    s = to_dev(inputs.neel_order_configs(L, CHAINS, rng))
    v = make_ctx(w, theta=theta)
    e_start = exact_energy(w, theta)
    la, _ = v.logpsi(s)
    v.metropolis(s, la, to_dev(inputs.chain_uniforms(4 * L * L, CHAINS, rng)), hastings=True)
    for _ in range(ITERS):
        la, _ = v.logpsi(s)
        v.metropolis(s, la, to_dev(inputs.chain_uniforms(L * L, CHAINS, rng)), hastings=True)
        e, _ = v.local_energy(s)
        O = v.log_derivs(s, dtype=torch.float32)
        x, _ = v.sr_solve(O, e, shift=SHIFT, iters=50, resid=False)
        v.sr_update(x, ETA)
    assert v.sync_status()[0] == VMC_OK
    e_end = exact_energy(w, v.get_params().cpu().numpy())
    e0 = e0_4x4(w.J2) / (L * L)
    assert e_end >= e0 - 1e-12
    assert e_end < e0 + 0.02
    assert e_start - e_end > 0.2
