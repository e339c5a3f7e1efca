"""Host logic of the light-cone pass: every plan the library's planner can
build (all uniform candidates the autotuner may time, and ragged plans with
the cost model's or explicit tiles) is checked against a brute-force model
of the kernel's shared-memory accesses (`csrc/tc_kern.cuh`):

* bounds: within each of the buffer's P (C/8) channel planes, every lane an
  MMA reads (the tile's 128 lanes, one grid row and one lane either side)
  and every lane the epilogue, the border (ring) copies or the embedding
  im2col write lies inside the plane; the last layer's pooling partials fit
  one buffer; the shared memory fits the limit;
* tile-level hand-off: for a layer whose window grows, the rule by which
  tile t of layer l + 1 waits for the drain of layer-l tiles 0 .. dep_tile
  (a mirror of the device function) covers every lane the tile reads that a
  layer-l tile writes (tiles drain in order).

The plans come from tests/plan_dump_main.cu, which includes the planner
(csrc/tc_fwd.cu) and prints them; it is compiled here with nvcc (host code
only runs).  The light-cone geometry follows Sec. 2.2 (3 x 3 filters: after
layer l a neighbour differs from its parent within l + 1 cells of the pair).
"""
import os
import re
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def plans(tmp_path_factory):
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    if not (os.path.exists(nvcc) or shutil.which("nvcc")):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("plans") / "plan_dump")
    cmd = [nvcc if os.path.exists(nvcc) else "nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17",
           "-O1", "-I", os.path.join(ROOT, "include"), "-o", exe, os.path.join(HERE, "plan_dump_main.cu"),
           "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.splitlines()
    res, i = [], 0
    head = re.compile(r"(uniform|ragged) L (\d+) C (\d+) D (\d+) S (\d+) P (\d+) G (\d+) BUF (\d+) smem (\d+) limit (\d+)")
    lay = re.compile(r"\s+l (\d+) w (\d+) T (\d+) PW (\d+) RW (\d+) NRm (\d+)")
    while i < len(out):
        m = head.match(out[i])
        assert m, out[i]
        kind = m.group(1)
        L, C, D, S, P, G, BUF, smem, limit = map(int, m.groups()[1:])
        layers = []
        for l in range(D + 1):
            mm = lay.match(out[i + 1 + l])
            layers.append(dict(zip(("l", "w", "T", "PW", "RW", "NRm"), map(int, mm.groups()))))
        res.append(dict(kind=kind, L=L, C=C, D=D, S=S, P=P, G=G, BUF=BUF, smem=smem, limit=limit, layers=layers))
        i += D + 2
    return res


def tile_row(g, t):
    return g["RW"] + min(128 * t, g["NRm"])


def dep_tile(g0, g1, t):
    """Mirror of the kernel's dep_tile: the last layer-l tile whose drain
    tile t of layer l + 1 waits for."""
    ymax = (tile_row(g1, t) + 128 + g1["RW"]) // g1["RW"]
    yn = min(ymax - 1, g0["w"])
    x = (yn + 1) * g0["RW"] - 1 - g0["RW"] - 127
    return min(0 if x <= 0 else (x + 127) // 128, g0["T"] - 1)


def grows(layers, l):
    return l + 1 < len(layers) and layers[l + 1]["w"] > layers[l]["w"]


def test_plans_cover_the_cases(plans):
    kinds = {p["kind"] for p in plans}
    assert kinds == {"uniform", "ragged"}
    # the bench's L = 24 choice is among them
    assert any(p["kind"] == "uniform" and (p["L"], p["C"], p["S"], p["P"], p["G"]) == (24, 32, 1, 2, 2) for p in plans)
    assert len(plans) > 500


def test_shared_memory_bounds(plans):
    bad = []
    for p in plans:
        L, C, D, P, G = p["L"], p["C"], p["D"], p["P"], p["G"]
        cp8 = C // 8
        lanes = (p["BUF"] // (P * cp8 * 16) * 16) // 16      # 16-byte lanes per channel plane
        worst = 0
        for l, g in enumerate(p["layers"]):
            w, RW, PW = g["w"], g["RW"], g["PW"]
            for t in range(g["T"]):
                r0 = tile_row(g, t)
                # MMA A rows: lanes r0 + 1 + row, shifted by -/+ one grid row
                # (C -> C layers) and one lane (the neighbouring lanes' cells)
                worst = max(worst, r0 + 128 if l == 0 else r0 + RW + 129)
            if l == len(p["layers"]) - 1:
                nq = (w + 2) * PW
                assert 2 * cp8 * nq * 4 <= p["BUF"], ("pooling partials", p)
                continue
            if grows(p["layers"], l):
                # outputs to cell (x + 2, Y + 1) of the next window's grid and
                # its ring (rows 0, 1, w + 2, w + 3, columns 0, 1, w + 2, w + 3)
                RWn = p["layers"][l + 1]["RW"]
                xg_max = G * (w + 4) - 1
                worst = max(worst, (w + 3) * RWn + xg_max // P + 1)
            else:
                # the same grid with its circular halo rows 0 and w + 1
                worst = max(worst, (w + 1) * RW + (PW - 1) // P + 1)
        g0 = p["layers"][0]
        w0 = g0["w"]
        for j in range(G):   # embedding im2col, cells 1 .. w0 of each window
            q = w0 * g0["PW"] + j * (w0 + 2) + w0
            worst = max(worst, q // P + 1)
        if worst >= lanes:
            bad.append((p["kind"], L, C, D, p["S"], P, G, worst, lanes))
        assert p["smem"] <= p["limit"], p
    assert not bad, bad[:5]


def test_tile_dependencies_cover_every_read(plans):
    checked = 0
    for p in plans:
        P, G = p["P"], p["G"]
        layers = p["layers"]
        for l in range(len(layers) - 1):
            if not grows(layers, l):
                continue
            g0, g1 = layers[l], layers[l + 1]
            w, RW, RWn = g0["w"], g0["RW"], g1["RW"]
            # the layer-l tile that writes each lane of the next grid (fresh
            # lanes only: the last tile skips the ones the tile before drained)
            writer = {}
            for t in range(g0["T"]):
                r0 = tile_row(g0, t)
                ov = 128 * t - g0["NRm"] if t == g0["T"] - 1 else 0
                for q in range(max(ov, 0), 128):
                    Y, rX = divmod(r0 + q, RW)
                    if not 1 <= Y <= w:
                        continue
                    for c in range(P):
                        j, xx = divmod(P * rX + c, w + 2)
                        x = xx - 1
                        if j >= G or not 0 <= x < w:
                            continue
                        ln = (Y + 1) * RWn + (j * (w + 4) + x + 2) // P
                        writer[ln] = max(writer.get(ln, -1), t)
            for tp in range(g1["T"]):
                r0p = tile_row(g1, tp)
                need = max([writer.get(ln, -1) for ln in range(r0p - RWn - 1, r0p + 128 + RWn + 1)] + [-1])
                assert need <= dep_tile(g0, g1, tp), (p["kind"], p["L"], p["C"], p["D"], P, G, l, tp)
                checked += 1
    assert checked > 1000
