"""The allocation-free O^T w entry point (vmc_ot_vec_noalloc).

It serves callers that may not allocate device memory (allocator or
memory-pool callbacks, runtimes that forbid cudaMalloc after start-up), so it
keeps its scratch in a fixed array inside the library's device image.
Checked through the C ABI against the allocating entry point vmc_ot_vec and
against an FP64 O^T w on two calls in a row (different inputs, so the
second call runs on the first call's leftovers), at the tolerance the SR
tests use for vmc_ot_vec; at the largest accepted size (m = 1, which fills
the array up to its last partial); and at the first refused sizes.
Collected last so that a run stopping at the first failure has run every
other test first.
"""
import numpy as np
import pytest
import torch

from paper_2108_13830_gb300 import inputs
from paper_2108_13830_gb300.binding import VMC, VMC_OK, VMC_ERR_ARG, VMC_ERR_UNSUPPORTED, ot_vec_noalloc
from gpu_util import to_dev

pytestmark = pytest.mark.gpu

SCRATCH = 16 << 20


def _fp64_otw(O, w):
    return O.double().cpu().numpy().T @ w.cpu().numpy()


@pytest.mark.parametrize("m,C,D", [(4096, 16, 6), (300, 4, 2), (40, 4, 2)])
def test_noalloc_matches_ot_vec_twice(m, C, D):
    v = VMC(10, 1.0, 0.5, C, D, "fp32")        # only for the reference entry point
    n = v.n
    for call in range(2):
        rng = inputs.rng_for(70 + call, m)
        O = to_dev(inputs.synthetic_O(m, n, rng))
        w = to_dev(rng.standard_normal(m))
        got, rc = ot_vec_noalloc(O, w)
        ref = v.ot_vec(O, w)
        torch.cuda.synchronize()
        assert rc == VMC_OK
        g, r = got.cpu().numpy(), ref.cpu().numpy()
        np.testing.assert_allclose(g, r, rtol=1e-11, atol=1e-12 * np.abs(r).max())
        exact = _fp64_otw(O, w)
        np.testing.assert_allclose(g, exact, rtol=1e-11, atol=1e-12 * np.abs(exact).max())
    v.close()


def test_noalloc_largest_accepted_size():
    """m = 1 uses one row chunk: 256 bytes of split w, then n partials up to
    the array's last byte."""
    n = (SCRATCH - 256) // 8
    rng = inputs.rng_for(73)
    O = to_dev(rng.standard_normal((1, n)).astype(np.float32))
    w = to_dev(np.array([rng.standard_normal()]))
    for _ in range(2):
        got, rc = ot_vec_noalloc(O, w)
        torch.cuda.synchronize()
        assert rc == VMC_OK
        exact = _fp64_otw(O, w)
        np.testing.assert_allclose(got.cpu().numpy(), exact, rtol=1e-13, atol=0)
    out = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    Obig = torch.zeros(1, n + 1, dtype=torch.float32, device="cuda")
    _, rc = ot_vec_noalloc(Obig, w, out)
    assert rc == VMC_ERR_UNSUPPORTED
    assert out.abs().max().item() == 0.0      # refused before any device work


def test_noalloc_rejects_sizes_beyond_its_scratch():
    O = torch.zeros(1, dtype=torch.float32, device="cuda")
    w = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    from paper_2108_13830_gb300.binding import lib, _ptr, _stream
    # 4096 x 200000 needs 16 * 200000 * 8 bytes of partials: refused, no work launched
    assert lib().vmc_ot_vec_noalloc(_ptr(O), 4096, 200000, _ptr(w), _ptr(out), _stream()) == VMC_ERR_UNSUPPORTED
    # sizes whose byte counts would wrap 64-bit arithmetic are refused too
    assert lib().vmc_ot_vec_noalloc(_ptr(O), 1 << 61, 1, _ptr(w), _ptr(out), _stream()) == VMC_ERR_UNSUPPORTED
    assert lib().vmc_ot_vec_noalloc(_ptr(O), 1, 1 << 61, _ptr(w), _ptr(out), _stream()) == VMC_ERR_UNSUPPORTED
    assert lib().vmc_ot_vec_noalloc(None, 4096, 10, _ptr(w), _ptr(out), _stream()) == VMC_ERR_ARG
    assert lib().vmc_ot_vec_noalloc(_ptr(O), 0, 10, _ptr(w), _ptr(out), _stream()) == VMC_ERR_ARG
