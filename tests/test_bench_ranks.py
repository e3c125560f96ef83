"""The benchmark's multi-rank logic on the CPU (gloo, two ranks): the timing
reduction takes the slowest rank, the whole-job rate counts every rank's
units, and the reference arm prints exactly one line under torchrun."""
import importlib.util
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    b = _bench()
    r, w, _ = b._dist_init(world)
    assert (r, w) == (rank, world)
    b._barrier(w)
    ms = 10.0 + 5.0 * rank          # the slower rank decides
    m = b._max_over_ranks(ms, w, torch.device("cpu"))
    out.put((rank, m, b._whole_job_rate(4, 100, w, m)))
    dist.destroy_process_group()


def test_max_over_ranks_and_rate_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    for rank, m, rate in res:
        assert m == 15.0
        assert rate == pytest.approx(4 * 100 * 2 / 15e-3)


def test_reference_arm_two_ranks_prints_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--cpu-budget-s", "0.3"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_traffic_rows_follow_the_source(tmp_path):
    """roofline.traffic comes from the committed ncu table only while the
    row's source hash matches the detection kernels' source: comment edits
    and other files keep it, a code edit drops it."""
    b = _bench()
    csrc = tmp_path / "paper_2105_12415_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "mrdem_detect.cu").write_text("// a kernel\n__global__ void k() {}\n")
    (csrc / "mrdem_step.cu").write_text("__global__ void other() {}\n")
    b.ROOT = str(tmp_path)
    h = b._source_hash()
    table = f"| kernel | bytes | hash |\n|---|---|---|\n| k_tile | 1234 | {h} |\n| k_old | 99 | 0000 |\n"
    (tmp_path / "profiles" / "dram_traffic_c2_batched.md").write_text(table)
    assert b._traffic_per_launch() == {"k_tile": 1234.0}
    (csrc / "mrdem_detect.cu").write_text("/* reworded\n comment */\n__global__ void k() {}  // same code\n\n")
    assert b._source_hash() == h and b._traffic_per_launch() == {"k_tile": 1234.0}
    # a file the detection kernels are not built from does not count
    (csrc / "mrdem_step.cu").write_text("__global__ void other() { int y = 1; }\n")
    assert b._source_hash() == h
    (csrc / "mrdem_detect.cu").write_text("__global__ void k() { int x = 0; }\n")
    assert b._source_hash() != h and b._traffic_per_launch() == {}


def test_merge_oracle_baseline_reports_partition_parity():
    """The bench's timed oracle merge compares its partition with the GPU's
    member counts (here a hand-made list and the counts it must give)."""
    import numpy as np
    b = _bench()
    pa = np.array([[0.0, 0, 0], [0.001, 0, 0], [5.0, 0, 0]])
    c = dict(pair=np.array([0, 0, 0]), ta=np.array([1, 2, 3]), tb=np.zeros(3, int), pa=pa,
             pb=pa + [0, 0, 0.01], d=np.full(3, 0.01))
    r = b.merge_oracle_baseline(c, np.array([0.01]), np.array([2, 1]))
    assert r["partition_equal"] and r["contacts_out"] == 2 and r["kind"] == "oracle"
    assert not b.merge_oracle_baseline(c, np.array([0.01]), np.array([1, 1, 1]))["partition_equal"]


def test_cpu_baseline_single_thread_and_model():
    """The oracle baseline runs on a bounded sample with one thread as well as
    all cores, and names the host CPU."""
    from gen import scene_tiny
    b = _bench()
    s = scene_tiny(n_pairs=16)
    one = b.cpu_oracle_baseline(s, 0.5, n_threads=1)
    assert one["cores"] == 1 and one["value"] > 0 and one["kind"] == "oracle"
    assert isinstance(b._cpu_model(), str) and b._cpu_model()


def test_clock_summary_reads_samples():
    """The clock record taken during the timed region: median SM clock, the
    maximum, and the throttle reasons that were active."""
    b = _bench()
    c = b.Clocks(0)
    c.lines = ["0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 2040, 2070, 950.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 910.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    r = c.summary()
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert b.Clocks(0).summary()["samples"] == 0
