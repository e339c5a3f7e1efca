"""Host-side checks that need no GPU: the C-ABI library builds, loads and
exports every entry point declared in include/vmc.h; argument validation
that returns before any CUDA call; the seeded input generators."""
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2108_13830_gb300 import build as vbuild
from paper_2108_13830_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "vmc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(vmc_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    return vbuild.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["vmc_create", "vmc_destroy", "vmc_logpsi", "vmc_local_energy",
                     "vmc_local_energy_ragged", "vmc_log_derivs", "vmc_sr_solve",
                     "vmc_sr_matvec", "vmc_sr_moments", "vmc_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (vmc_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_validates_without_gpu(libpath):
    import ctypes as ct
    from paper_2108_13830_gb300 import binding as b
    L = b.lib()
    h = ct.c_void_p(123)
    arch = b.vmc_arch(2, 4, b.VMC_FP64, 1)
    # invalid L is rejected before any CUDA call, and *out is cleared
    assert L.vmc_create(3, 1.0, 0.5, ct.byref(arch), ct.byref(h)) == b.VMC_ERR_ARG
    assert h.value is None
    assert L.vmc_create(4, 1.0, 0.5, None, ct.byref(h)) == b.VMC_ERR_ARG
    bad = b.vmc_arch(2, 5, b.VMC_FP64, 1)   # channels not a multiple of 4
    assert L.vmc_create(4, 1.0, 0.5, ct.byref(bad), ct.byref(h)) == b.VMC_ERR_ARG
    bf = b.vmc_arch(2, 8, b.VMC_BF16, 1)    # BF16 needs C in {16, 32}
    assert L.vmc_create(8, 1.0, 0.5, ct.byref(bf), ct.byref(h)) == b.VMC_ERR_ARG
    n = ct.c_int64()
    assert L.vmc_num_params(None, ct.byref(n)) == b.VMC_ERR_ARG
    assert L.vmc_logpsi(None, None, 0, None, None, None) == b.VMC_ERR_ARG
    assert L.vmc_last_error(None) == b"null context"


def test_uniform_configs_are_sz_zero():
    rng = inputs.rng_for(0)
    s = inputs.uniform_configs(10, 50, rng)
    assert s.dtype == np.int8 and s.shape == (50, 10, 10)
    assert np.all(s.reshape(50, -1).sum(axis=1) == 0)
    assert set(np.unique(s)) == {-1, 1}


def test_neel_order_configs():
    rng = inputs.rng_for(1)
    L = 16
    s = inputs.neel_order_configs(L, 200, rng).astype(np.int64)
    assert np.all(s.reshape(200, -1).sum(axis=1) == 0)
    stag = np.abs((s * inputs.neel_state(L)).reshape(200, -1).mean(axis=1))
    assert 0.0 <= stag.min() and stag.max() <= 0.75
    assert 0.15 < stag.mean() < 0.45      # f ~ U[0, 0.6] keeps about f of the order


def test_param_layout_matches_count():
    for C, D in [(4, 2), (16, 6), (32, 8), (32, 10)]:
        offs = inputs.param_offsets(C, D)
        assert offs[-1][1] + C == inputs.num_params(C, D)
    assert inputs.num_params(16, 6) == 14080
    assert inputs.num_params(32, 10) == 92800


def test_ragged_inputs_shapes():
    w = inputs.WORKLOADS["ragged_8_16"]
    packed, offs, Ls, theta = inputs.ragged_inputs(w, per_L=5)
    assert len(offs) == len(Ls) == 20
    assert sorted(set(Ls.tolist())) == [8, 10, 12, 16]
    ends = offs + Ls.astype(np.int64) ** 2
    assert ends.max() == packed.size
    for o, L in zip(offs, Ls):
        assert packed[o:o + L * L].astype(int).sum() == 0
