"""Host-side logic of bench.py that needs no GPU: the max-over-ranks timing
of the multi-process run (world size 2 on the gloo backend), the CPU
oracle reference arm (rank 0 prints the JSON line, other ranks do no work)
and the summary of the clock samples taken during the timed region."""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    local = [0.75, 1.25][rank]  # each rank's timed seconds
    total = bench.max_over_ranks(local, world)
    out.put((rank, total, world * 4 / total))  # value = all ranks' steps / the slowest rank's time
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world_2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [1.25, 1.25]
    assert all(abs(g[2] - 2 * 4 / 1.25) < 1e-12 for g in got)


def test_max_over_ranks_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.5, 1) == 0.5


def test_reference_arm_rank_nonzero_does_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


@pytest.mark.slow
def test_reference_arm_prints_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--ref-iters", "1"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "cpu_baseline",
              "e2e", "config"):
        assert k in line
    assert line["impl"] == "reference" and line["unit"] == "solves/s" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_clock_summary_of_nvidia_smi_rows():
    sys.path.insert(0, ROOT)
    import bench
    idle = "345, 2070, 150.1, 0x0000000000000001, Not Active, Not Active, Not Active, Not Active"
    busy = "2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    capped = "1980, 2070, 1400.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
    rows = [idle, busy, busy, capped, busy, "garbage line", "[N/A], 2070, 1, 0, a, b, c, d", ""]
    out = bench.summarize_clocks(rows)
    # the idle sample (below half the peak) is left out of the median
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 5}
    hot = "1500, 2070, 1200.0, 0x0000000000000048, Active, Active, Not Active, Not Active"
    out = bench.summarize_clocks([busy, hot, hot])
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"] and out["sm_mhz"] == 1500.0
    assert bench.summarize_clocks(["", "x, y"]) is None


def test_metric_summaries_are_short_and_last():
    """The mixed-vs-FP64, serving and batching summaries that end the JSON
    line keep the numbers a reader of the line's tail needs, in a few hundred
    characters."""
    sys.path.insert(0, ROOT)
    import bench
    mixed = {"24^3x8 Wilson k=0.155": {"fp64_solves_s": 59.71, "mixed_f16_solves_s": 165.3, "ratio": 2.768,
                                       "mixed_true_rel_residual": 9.1e-11, "fp64_true_rel_residual": 8.7e-11},
             "48^3x12 twisted mass k=0.16 mu=0.01": {"fp64_solves_s": 6.07, "mixed_f16_solves_s": 17.2,
                                                     "ratio": 2.834, "mixed_true_rel_residual": 9.9e-11,
                                                     "fp64_true_rel_residual": 9.2e-11}}
    m = bench.mixed_summary(mixed)
    assert m["24^3x8"] == {"fp64": 59.71, "f16_mixed": 165.3, "ratio": 2.77, "max_res": 9.1e-11}
    assert m["48^3x12 tm"]["ratio"] == 2.83
    sv = {"requests": 2000, "arrival_rate_per_s": 30.0, "solves_s": 29.81, "latency_p50_ms": 40.12,
          "latency_p99_ms": 490.4, "failed": 0, "max_true_rel_residual": 9.96e-11}
    s = bench.serving_summary(sv)
    assert s["failed"] == 0 and s["p99_ms"] == 490.0 and s["p50_ms"] == 40.1
    b = {"solve": {"speedup": 0.981, "batched_solves_s": 76.2, "max_true_rel_residual": 9e-11},
         "kappa_batch": {"speedup": 0.731, "max_true_rel_residual": 9.5e-11},
         "dslash_f32_r12": {"rhs_per_s_16rhs": 92700.0, "rhs_per_s_1rhs": 43000.0}}
    bb = bench.batched_summary(b)
    assert bb["dslash_f32_r12_rhs_speedup"] == 2.16 and bb["max_res"] == 9.5e-11
    assert len(json.dumps({"batched_multi_rhs": bb, "serving": s, "mixed_vs_fp64": m})) < 700


def test_both_arms_share_the_config():
    sys.path.insert(0, ROOT)
    import bench
    c = bench.workload_config()
    assert c == bench.workload_config() and c["lattice"] == [24, 24, 24, 8] and c["tol"] == 1e-10
