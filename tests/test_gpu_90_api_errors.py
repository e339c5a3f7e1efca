"""Argument checks of the entry points beyond the hot path (vmc_metropolis,
vmc_sr_update, the symmetrised calls): each returns VMC_ERR_ARG (or
VMC_ERR_STATE before parameters are set) without device work, and empty
batches are no-ops."""
import ctypes as ct

import pytest
import torch

from paper_2108_13830_gb300 import inputs
from paper_2108_13830_gb300.binding import (VMC, VMC_ERR_ARG, VMC_ERR_STATE, VMC_FP32, VMC_FP64, VMC_OK,
                                            _ptr, _stream, lib)
from gpu_util import make_ctx, to_dev

pytestmark = pytest.mark.gpu


def test_calls_before_parameters_are_set():
    v = VMC(4, 1.0, 0.5, 4, 2, "fp64")
    s = torch.ones(2, 4, 4, dtype=torch.int8, device="cuda")
    la = torch.zeros(2, dtype=torch.float64, device="cuda")
    sg = torch.zeros(2, dtype=torch.int8, device="cuda")
    u = torch.zeros(1, 2, 2, dtype=torch.float64, device="cuda")
    x = torch.zeros(v.n, dtype=torch.float64, device="cuda")
    L_ = lib()
    assert L_.vmc_metropolis(v._h, _ptr(s), _ptr(la), 2, _ptr(u), 1, 0, None, _stream()) == VMC_ERR_STATE
    assert L_.vmc_sr_update(v._h, _ptr(x), ct.c_double(0.1), _stream()) == VMC_ERR_STATE
    assert L_.vmc_logpsi_sym(v._h, _ptr(s), 2, _ptr(la), _ptr(sg), _stream()) == VMC_ERR_STATE


def test_invalid_arguments():
    w = inputs.WORKLOADS["L4_fp64"]
    sig, theta = inputs.workload_inputs(w, batch=4)
    v = make_ctx(w, theta=theta)
    s = to_dev(sig)
    la = torch.zeros(4, dtype=torch.float64, device="cuda")
    sg = torch.zeros(4, dtype=torch.int8, device="cuda")
    u = torch.zeros(3, 4, 2, dtype=torch.float64, device="cuda")
    O = torch.zeros(4, v.n, dtype=torch.float32, device="cuda")
    L_, h, st = lib(), v._h, _stream()
    assert L_.vmc_metropolis(h, _ptr(s), _ptr(la), -1, _ptr(u), 3, 0, None, st) == VMC_ERR_ARG
    assert L_.vmc_metropolis(h, _ptr(s), _ptr(la), 4, _ptr(u), -2, 0, None, st) == VMC_ERR_ARG
    assert L_.vmc_metropolis(h, None, _ptr(la), 4, _ptr(u), 3, 0, None, st) == VMC_ERR_ARG
    assert L_.vmc_metropolis(h, _ptr(s), _ptr(la), 4, None, 3, 0, None, st) == VMC_ERR_ARG
    assert L_.vmc_metropolis(h, _ptr(s), _ptr(la), 4, _ptr(u), 3, 7, None, st) == VMC_ERR_ARG
    assert L_.vmc_metropolis(h, _ptr(s), _ptr(la), 0, None, 3, 0, None, st) == VMC_OK
    assert L_.vmc_sr_update(h, None, ct.c_double(0.1), st) == VMC_ERR_ARG
    assert L_.vmc_sr_update(h, _ptr(la), ct.c_double(float("inf")), st) == VMC_ERR_ARG
    assert L_.vmc_logpsi_sym(h, _ptr(s), -3, _ptr(la), _ptr(sg), st) == VMC_ERR_ARG
    assert L_.vmc_logpsi_sym(h, _ptr(s), 4, None, _ptr(sg), st) == VMC_ERR_ARG
    assert L_.vmc_local_energy_sym(h, None, 4, _ptr(la), None, st) == VMC_ERR_ARG
    assert L_.vmc_local_energy_sym(h, _ptr(s), 0, None, None, st) == VMC_OK
    assert L_.vmc_log_derivs_sym(h, _ptr(s), 4, _ptr(O), 9, st) == VMC_ERR_ARG
    assert L_.vmc_log_derivs_sym(h, _ptr(s), 4, None, VMC_FP32, st) == VMC_ERR_ARG
    # FP64 O rows need an FP64 context
    wb = inputs.WORKLOADS["L16_bf16"]
    sb, tb = inputs.workload_inputs(wb, batch=2)
    vb = make_ctx(wb, theta=tb)
    Ob = torch.zeros(2, vb.n, dtype=torch.float64, device="cuda")
    assert L_.vmc_log_derivs_sym(vb._h, _ptr(to_dev(sb)), 2, _ptr(Ob), VMC_FP64, st) == VMC_ERR_ARG
    assert v.sync_status()[0] == VMC_OK
    assert vb.sync_status()[0] == VMC_OK
