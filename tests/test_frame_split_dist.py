"""The host side of one frame split across ranks, on CPU: gloo processes set up as torchrun
sets up one rank per GPU.  Each rank takes its range of a synthetic frame's hit list (hits in
pixel order, ranges from the library's nis_part_range), the ranges are gathered to rank 0
by frame_split.gather_parts, and rank 0 assembles them.  Checks: the ranges cover every hit
exactly once and in order, nothing but hits is named, the radiance bits survive the
exchange, and the assembled image equals the single-rank assembly of the same hit list.
The device half (render_frame_part against render_frame, scatter_part) is a GPU test."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_PROGRAM = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch, torch.distributed as dist
from paper_2401_14051_gb300 import nis, frame_split
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
# (width, height, hit density, seed): ragged sizes, an empty frame, one hit, all hits
cases = [(37, 23, 0.4, 1), (64, 64, 0.05, 2), (5, 3, 0.0, 3), (1, 1, 1.0, 4), (17, 9, 1.0, 5),
         (2, 1, 0.0, 6), (1, 2, 1.0, 7)]
out = []
for (w, h, density, seed) in cases:
    rng = np.random.default_rng(seed)
    hits = np.nonzero(rng.random(w * h) < density)[0].astype(np.int32)   # pixel order
    rgb = rng.standard_normal((len(hits), 3)).astype(np.float32)
    if len(hits) >= 3:                    # bit patterns that an arithmetic copy could change
        rgb[0] = [np.float32(1e-42), -0.0, np.inf]
    first, count = nis.part_range(len(hits), rank, world)
    part_rgb = torch.from_numpy(rgb[first:first + count].copy())
    part_pix = torch.from_numpy(hits[first:first + count].copy())
    rows = max(nis.part_capacity(len(hits), world), 1)
    parts = frame_split.gather_parts(part_rgb, part_pix, rows, dst=0)
    if rank != 0:
        assert parts is None
        continue
    all_pix = torch.cat([p for _, p in parts]).numpy()
    all_rgb = torch.cat([c for c, _ in parts]).numpy()
    counts = [int(p.shape[0]) for _, p in parts]
    image = np.zeros((h * w, 3), np.float32)
    image[all_pix] = all_rgb
    single = np.zeros((h * w, 3), np.float32)
    single[hits] = rgb
    covered = np.bincount(all_pix, minlength=w * h) if len(all_pix) else np.zeros(w * h, int)
    out.append({"case": [w, h, density, seed], "counts": counts, "n_hits": int(len(hits)),
                "in_order": bool(np.array_equal(all_pix, hits)),
                "each_once": bool(np.array_equal(covered, np.isin(np.arange(w * h), hits).astype(int))),
                "bits_equal": bool(np.array_equal(image.view(np.int32), single.view(np.int32))),
                "rgb_bits_equal": bool(np.array_equal(all_rgb.view(np.int32), rgb.view(np.int32)))})
dist.barrier()
if rank == 0:
    print("RESULT " + json.dumps(out), flush=True)
dist.destroy_process_group()
"""


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_env(rank: int, world: int, port: int) -> dict:
    env = dict(os.environ)
    env.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                "OMP_NUM_THREADS": "1", "CUDA_VISIBLE_DEVICES": ""})
    return env


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_split_and_assemble_a_frame(world):
    port = _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", RANK_PROGRAM, ROOT], cwd=ROOT,
                              env=_rank_env(r, world, port), stdout=subprocess.PIPE,
                              stderr=subprocess.STDOUT, text=True)
             for r in range(world)]
    outs = []
    for p in procs:
        out, _ = p.communicate(timeout=240)
        assert p.returncode == 0, out
        outs.append(out)
    line = [l for l in outs[0].splitlines() if l.startswith("RESULT ")]
    assert len(line) == 1, outs[0]
    results = json.loads(line[0][len("RESULT "):])
    assert len(results) == 7
    for r in results:
        n = r["n_hits"]
        assert sum(r["counts"]) == n, r
        # equal contiguous ranges: sizes differ by at most one, the larger ones last
        assert max(r["counts"]) - min(r["counts"]) <= 1, r
        assert r["counts"] == sorted(r["counts"]), r
        assert r["in_order"] and r["each_once"], r
        assert r["bits_equal"] and r["rgb_bits_equal"], r


def test_part_range_is_floor_of_equal_shares():
    """nis_part_range (host only) against its definition, including sizes whose products
    overflow 64 bits if computed naively."""
    sys.path.insert(0, ROOT)
    from paper_2401_14051_gb300 import nis
    for n in (0, 1, 2, 7, 100, 215053, 2 ** 40 + 3, 2 ** 62 + 11):
        for parts in (1, 2, 3, 8, 1000):
            got = [nis.part_range(n, p, parts) for p in range(min(parts, 4))] + \
                  [nis.part_range(n, parts - 1, parts)]
            for p, (first, count) in zip(list(range(min(parts, 4))) + [parts - 1], got):
                assert first == p * n // parts
                assert count == (p + 1) * n // parts - p * n // parts
    assert nis.part_capacity(10, 3) == 4 and nis.part_capacity(9, 3) == 3
    for bad in ((-1, 0, 1), (5, 0, 0), (5, 2, 2), (5, -1, 2)):
        with pytest.raises(nis.NisError):
            nis.part_range(*bad)
