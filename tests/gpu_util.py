"""Shared helpers of the GPU tests (seeded inputs, contexts)."""
import numpy as np
import torch

from paper_2108_13830_gb300 import inputs
from paper_2108_13830_gb300.binding import VMC


def make_ctx(w, precision=None, theta=None, L=None, marshall=True):
    v = VMC(L or w.L, w.J1, w.J2, w.C, w.D, precision or w.precision, marshall=marshall)
    if theta is not None:
        v.set_params(torch.as_tensor(theta, dtype=torch.float64).cuda())
    return v


def to_dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def bond_counts(sig):
    """(A1, A2) antiparallel J1 / J2 bond counts by np.roll (independent of both sides)."""
    s = sig.astype(np.int64)
    right = np.roll(s, -1, axis=-1)
    down = np.roll(s, -1, axis=-2)
    dr = np.roll(down, -1, axis=-1)
    dl = np.roll(down, 1, axis=-1)
    a1 = np.sum(s * right == -1, axis=(-2, -1)) + np.sum(s * down == -1, axis=(-2, -1))
    a2 = np.sum(s * dr == -1, axis=(-2, -1)) + np.sum(s * dl == -1, axis=(-2, -1))
    return a1, a2
