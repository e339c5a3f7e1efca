"""The degenerate amplitude psi = 0 (one channel of the last layer
identically zero, so the product pooling of Eq. 8 vanishes): log|psi| is
-inf with sign 0, as the oracle gives it, and is not an error; the local
energy W(S')/W(S) is undefined, so every sample is NaN and counted by
VMC_ERR_NONFINITE.  Checked on the FP64 SIMT path (L = 4) and the BF16 and
FP16 tensor-core paths (L = 8, C = 32)."""
import numpy as np
import pytest

import oracle
from paper_2108_13830_gb300 import inputs
from paper_2108_13830_gb300.binding import VMC_ERR_NONFINITE, VMC_OK
from gpu_util import make_ctx, to_dev

pytestmark = pytest.mark.gpu


def _zero_channel_params(C, D, rng):
    theta = inputs.random_params(C, D, rng)
    wo, bo = inputs.param_offsets(C, D)[D]
    theta[wo:bo] = 0.0
    theta[bo:bo + C] = 1.0
    theta[bo] = 0.0
    return theta


@pytest.mark.parametrize("L,C,D,prec", [(4, 4, 2, "fp64"), (8, 32, 3, "bf16"), (8, 32, 3, "fp16")])
def test_zero_amplitude(L, C, D, prec):
    rng = inputs.rng_for(78)
    theta = _zero_channel_params(C, D, rng)
    sig = inputs.uniform_configs(L, 6, rng)
    w = inputs.Workload("zero_psi", L, C, D, prec, 6, index=78)
    v = make_ctx(w, theta=theta)
    s = to_dev(sig)
    la, sg = v.logpsi(s)
    assert v.sync_status()[0] == VMC_OK
    ra, rs = oracle.logpsi(L, C, D, theta, sig)
    assert np.all(np.isneginf(ra)) and np.all(rs == 0)
    assert np.all(np.isneginf(la.cpu().numpy())) and np.all(sg.cpu().numpy() == 0)
    e, nn = v.local_energy(s)
    rc, nf = v.sync_status()
    assert rc == VMC_ERR_NONFINITE and nf == 6
    assert np.all(np.isnan(e.cpu().numpy()))
    re, rn = oracle.local_energy(L, 1.0, 0.5, C, D, theta, sig)
    assert np.all(np.isnan(re))
    np.testing.assert_array_equal(nn.cpu().numpy(), rn)
