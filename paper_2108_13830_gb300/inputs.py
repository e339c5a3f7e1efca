"""Seeded synthetic inputs: spin configurations and CNN parameter vectors.

This module holds no arithmetic of the method itself: it draws random spin
configurations in the S^z = 0 sector and random network parameters, and it
knows the flat parameter layout shared by the library and the oracle.  Both
the GPU path and the CPU oracle are fed from here, never from each other.

Workload recipe (stand-in for the paper's Monte Carlo samples, Sec. 3.1 and
Table 2): periodic L x L lattices, J1 = 1, J2 = 0.5, spins s_i = +-1 with
sum_i s_i = 0; "uniform" configurations are a random permutation of N/2 up
and N/2 down spins; "neel" configurations start from the Neel state (the
chain start named in Sec. 3.1) and permute the spins of a random (1 - f)
fraction of the sites among themselves, f ~ U[0, 0.6].
"""
from __future__ import annotations

import dataclasses
import numpy as np

BASE_SEED = 2108_13830


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    L: int                 # lattice side (L even, >= 4)
    C: int                 # channels
    D: int                 # number of C -> C conv layers after the 1 -> C embedding
    precision: str         # "fp64" | "fp32" | "bf16"
    batch: int             # number of sampled configurations
    kind: str = "uniform"  # "uniform" | "neel" | "ragged"
    Ls: tuple = ()         # ragged: lattice sides, `batch` configurations each
    J1: float = 1.0
    J2: float = 0.5
    shift: float = 1e-4    # SR diagonal shift
    cg_iters: int = 50
    index: int = 0         # seed offset


# The five seeded workloads: a 4x4 FP64 case checked against exact
# diagonalisation, a 10x10 FP32 case, a 16x16 BF16-vs-FP32 case, a ragged
# mixed-size batch and the 24x24 case that also runs the SR solve.
WORKLOADS = {
    "L4_fp64": Workload("L4_fp64", 4, 4, 2, "fp64", 256, index=0),
    "L10_fp32": Workload("L10_fp32", 10, 16, 6, "fp32", 4096, index=1),
    "L16_bf16": Workload("L16_bf16", 16, 32, 8, "bf16", 8192, index=2),
    "ragged_8_16": Workload("ragged_8_16", 16, 16, 6, "fp16", 2048, kind="ragged",
                            Ls=(8, 10, 12, 16), index=3),
    "L24_bf16_sr": Workload("L24_bf16_sr", 24, 32, 10, "bf16", 4096, index=4),
}


def num_params(C: int, D: int) -> int:
    """Length of the flat parameter vector: 1->C embedding then D C->C layers."""
    return (9 * C + C) + D * (9 * C * C + C)


def layer_shapes(C: int, D: int):
    """[(c_out, c_in)] for the D + 1 conv layers, in flat-vector order."""
    return [(C, 1)] + [(C, C)] * D


def param_offsets(C: int, D: int):
    """Offsets of (W_l, b_l) in the flat vector.

    Layout per layer l: W_l as [c_out][c_in][3][3] (row ky, column kx) then
    b_l as [c_out]; layers in order 0..D.
    """
    offs = []
    o = 0
    for co, ci in layer_shapes(C, D):
        offs.append((o, o + 9 * co * ci))
        o += 9 * co * ci + co
    return offs


def rng_for(seed_offset: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([BASE_SEED + seed_offset, stream]))


def uniform_configs(L: int, B: int, rng: np.random.Generator) -> np.ndarray:
    """B configurations, int8 [B, L, L], exactly N/2 spins +1 and N/2 spins -1."""
    N = L * L
    base = np.concatenate([np.ones(N // 2, np.int8), -np.ones(N // 2, np.int8)])
    out = np.empty((B, N), np.int8)
    for b in range(B):
        out[b] = rng.permutation(base)
    return out.reshape(B, L, L)


def neel_state(L: int) -> np.ndarray:
    y, x = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    return np.where((x + y) % 2 == 0, 1, -1).astype(np.int8)


def neel_order_configs(L: int, B: int, rng: np.random.Generator,
                       fmax: float = 0.6) -> np.ndarray:
    """Neel state with the spins of a random (1 - f) fraction of sites permuted.

    f ~ U[0, fmax]; the permutation keeps sum s_i = 0 and leaves the
    staggered magnetisation near f.
    """
    N = L * L
    neel = neel_state(L).reshape(N)
    out = np.empty((B, N), np.int8)
    for b in range(B):
        f = rng.uniform(0.0, fmax)
        k = int(round((1.0 - f) * N))
        sites = rng.choice(N, size=k, replace=False)
        s = neel.copy()
        s[sites] = s[rng.permutation(sites)]
        out[b] = s
    return out.reshape(B, L, L)


def random_params(C: int, D: int, rng: np.random.Generator, scale: float = 1.0,
                  last_bias: float = 1.0) -> np.ndarray:
    """Flat float64 parameter vector.

    Weights ~ N(0, (scale / sqrt(9 c_in))^2); biases 0 except the last
    layer's, which are `last_bias`.  scale = 3 gives a "stressed" network
    whose amplitude ratios stray far from 1.
    """
    theta = np.zeros(num_params(C, D), np.float64)
    for l, ((co, ci), (ow, ob)) in enumerate(zip(layer_shapes(C, D), param_offsets(C, D))):
        std = scale / np.sqrt(9.0 * ci)
        theta[ow:ob] = rng.normal(0.0, std, ob - ow)
        theta[ob:ob + co] = last_bias if l == D else 0.0
    return theta


def workload_inputs(w: Workload, batch: int | None = None, scale: float = 1.0, sample_stream: int = 0):
    """(sigma, theta) for a uniform-L workload; sigma int8 [B, L, L].

    The parameters depend only on the workload; `sample_stream` selects an
    independent stream of configurations (one per replica)."""
    B = w.batch if batch is None else batch
    rng = rng_for(w.index, 0)
    theta = random_params(w.C, w.D, rng, scale=scale)
    rs = rng_for(w.index, 1 + sample_stream)
    if w.kind == "neel":
        sigma = neel_order_configs(w.L, B, rs)
    else:
        sigma = uniform_configs(w.L, B, rs)
    return sigma, theta


def ragged_inputs(w: Workload, per_L: int | None = None, scale: float = 1.0):
    """Mixed-size batch: `per_L` Neel-order configurations for each L in w.Ls.

    Returns (packed int8 [sum L^2], offsets int64 [B], Ls int32 [B], theta).
    Samples are interleaved across sizes so the batch is genuinely mixed.
    """
    n = w.batch if per_L is None else per_L
    rng = rng_for(w.index, 0)
    theta = random_params(w.C, w.D, rng, scale=scale)
    groups = []
    for j, L in enumerate(w.Ls):
        groups.append(neel_order_configs(L, n, rng_for(w.index, 10 + j)))
    order = []
    for b in range(n):
        for j in range(len(w.Ls)):
            order.append((j, b))
    perm = rng_for(w.index, 2).permutation(len(order))
    order = [order[i] for i in perm]
    packed, offs, Ls = [], [], []
    o = 0
    for j, b in order:
        c = groups[j][b].reshape(-1)
        packed.append(c)
        offs.append(o)
        Ls.append(w.Ls[j])
        o += c.size
    return (np.concatenate(packed).astype(np.int8), np.asarray(offs, np.int64),
            np.asarray(Ls, np.int32), theta)


def synthetic_O(m: int, n: int, rng: np.random.Generator, dtype=np.float32) -> np.ndarray:
    """Seeded stand-in for a log-derivative matrix: columns with nonzero means
    and scales spread over two decades, plus a shared low-rank component
    (samples are correlated), stored in FP32 like the library's O."""
    scale = np.exp(rng.uniform(np.log(0.05), np.log(5.0), n))
    mean = rng.normal(0.0, 1.0, n)
    lowrank = rng.normal(0.0, 1.0, (m, 4)) @ rng.normal(0.0, 0.3, (4, n))
    O = mean + scale * rng.standard_normal((m, n)) + lowrank
    return O.astype(dtype)


def synthetic_E(m: int, rng: np.random.Generator) -> np.ndarray:
    """Stand-in local energies around -0.5 per site of a 10x10 lattice."""
    return -50.0 + 3.0 * rng.standard_normal(m)


def chain_uniforms(steps: int, B: int, rng: np.random.Generator) -> np.ndarray:
    """Random numbers of `steps` Metropolis transitions of B chains:
    float64 [steps, B, 2] in [0, 1) (pair selector, acceptance threshold)."""
    return rng.random((steps, B, 2))
