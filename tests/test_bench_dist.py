"""The multi-rank host logic of bench.py on CPU: two processes with the gloo backend, set up
the way torchrun sets up one rank per GPU (RANK, LOCAL_RANK, WORLD_SIZE, MASTER_ADDR,
MASTER_PORT).  Each rank renders its own copy of the workload with no collective on the
data path, so what is shared is the rendezvous, the barriers around the timed region and
the reduction of the timings: whole-job throughput is the units all ranks processed over
the slowest rank's time."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_PROGRAM = r"""
import json, sys, time
sys.path.insert(0, sys.argv[1])
import bench
rank, local, world = bench.dist_init("gloo")
bench.barrier(world)
seconds = 1.0 + 0.5 * rank           # rank 1 is the slow one
units = 1000.0 * (rank + 1)          # ranks may shade different point counts
rate, slowest = bench.whole_job_rate(units, seconds, world)
out = {"rank": rank, "local": local, "world": world,
       "max": bench.max_over_ranks(float(rank) - 7.0, world),
       "sum": bench.sum_over_ranks(float(rank + 1), world),
       "rate": rate, "slowest": slowest}
bench.barrier(world)
print("RESULT " + json.dumps(out), flush=True)
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


def test_gloo_two_ranks_reduce_timings():
    world, port = 2, _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", RANK_PROGRAM, ROOT], cwd=ROOT,
                              env=_rank_env(r, world, port), stdout=subprocess.PIPE,
                              stderr=subprocess.STDOUT, text=True)
             for r in range(world)]
    results = {}
    for p in procs:
        out, _ = p.communicate(timeout=240)
        assert p.returncode == 0, out
        line = [l for l in out.splitlines() if l.startswith("RESULT ")]
        assert len(line) == 1, out
        r = json.loads(line[0][len("RESULT "):])
        results[r["rank"]] = r
    assert sorted(results) == [0, 1]
    for rank, r in results.items():
        assert r["local"] == rank and r["world"] == world
        assert r["max"] == 1.0 - 7.0                 # max of -7 and -6
        assert r["sum"] == 3.0                       # 1 + 2
        assert r["slowest"] == 1.5
        assert r["rate"] == pytest.approx((1000.0 + 2000.0) / 1.5, rel=0, abs=1e-9)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    saved = {k: os.environ.pop(k) for k in ("RANK", "LOCAL_RANK", "WORLD_SIZE") if k in os.environ}
    try:
        assert bench.dist_init("gloo") == (0, 0, 1)
        bench.barrier(1)
        assert bench.max_over_ranks(2.5, 1) == 2.5
        assert bench.whole_job_rate(300.0, 1.5, 1) == (200.0, 1.5)
    finally:
        os.environ.update(saved)


def test_reference_arm_under_torchrun_prints_once_from_rank_zero():
    """The launch the multi-GPU bench uses, with the oracle arm on the small 64^3 case: rank 0
    alone times the oracle and prints one JSON line, the other rank exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--workload", "1", "--steps", "1",
           "--warmup", "0"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stdout + p.stderr
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["value"] == line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_dense_layer_bytes_per_point_hand_count():
    # Counted by hand, w = 200.  A chain of n blocks over features of width d moves
    # op (n (d + 2w) + w) + st w (4n - 2) + 24 n bytes:
    #   FC-1 reads x (op d) and 24 B of row constants, and h_prev from the second block
    #   on; it writes e (st w) and s (op w).
    #   FC-2 reads s and e, and writes h (st w, op w at the chain's end).
    # Per type the chains have 8 and 4 blocks, and the merge reads 2w and writes w at op:
    #   op (12 d + 29 w) + 44 st w + 288.
    # Summed over d = 225, 225, 80: 23,760 op + 26,400 st + 864.
    # The head 600 -> 200 -> 200 -> 3 adds op (4w + 2w + w) plus 12 B of RGB:
    #   25,160 op + 26,400 st + 876 in all.
    import bench
    for op, st in ((6, 4), (2, 2), (1, 2)):
        assert bench.mlp_bytes_per_point(op, st) == 25160 * op + 26400 * st + 876


def test_compact_summary_fits_the_end_of_a_log():
    # the bench line ends with a summary of its figures; a log that keeps only the last
    # ~1.5 KB of the output must still hold it whole
    import json
    import bench
    fam = {f: 1.0 for f in ("pyramid", "march", "phase", "hits", "gather", "cnn", "mlp", "other")}
    sub = {"value": 1e7, "frame_ms": 20.0, "mean_rel_err_vs_fp32": 0.006,
           "step_breakdown_ms": fam, "roofline": {"frac": 0.3}}
    serv = {"throughput_req_s": 30.0, "p50_ms": 50.0, "p99_ms": 250.0, "mean_batch_requests": 1.5,
            "load_sweep": [{"load": 1.0, "throughput_req_s": 40.0, "p50_ms": 60.0, "p99_ms": 300.0,
                            "mean_batch_requests": 2.0}] * 2}
    line = {"frame_ms": 36.0, "value": 5.9e6, "step_breakdown_ms": fam,
            "roofline": {"bound": "tensor", "frac": 0.3}, "gather_roofline": {"frac": 0.2},
            "e2e": {"value": 5.8e6}, "bf16": sub, "fp8": sub,
            "paper_template_model": {"frame_ms": 27.0}, "shear_warp": {"frame_ms": 33.0},
            "serving": serv, "serving_shear_warp": serv,
            "plume1024_60f": {"shear_warp": {"frames": 60, "frame_ms_median": 80.0, "frame_ms_p99": 90.0},
                              "march": {"frames": 8, "frame_ms_median": 1200.0, "frame_ms_p99": 1210.0}},
            "cpu_baseline": {"value": 9.0, "single_thread": {"value": 3.0}}}
    s = json.dumps({"summary": bench.compact_summary(line)})
    assert len(s) < 1400, len(s)
    assert '"bf16"' in s and '"plume_60f"' in s and '"sweep"' in s
