"""Host-side logic of bench.py: the multi-rank replicas (max of times and sum of
units over ranks) on two gloo ranks on the CPU, the reference arm's rank
rule, first-come-first-served finish times, the process pool of the CPU
baseline, the traffic gate, the peak lookup and the clock samples."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    r, w, _ = bench.dist_setup(False)
    assert (r, w) == (rank, world)
    local_ms = 100.0 + 50.0 * rank          # rank 1 is slower
    local_units = 1000.0 * (rank + 1)
    total_ms = bench.reduce_max(local_ms, w, torch.device("cpu"))
    units = bench.reduce_sum(local_units, w, torch.device("cpu"))
    bench.barrier(w)
    results[rank] = (total_ms, units)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_the_total_units():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        results = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, results)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert results[0] == results[1] == (150.0, 3000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), dict(steps=1, warmup=0, gpus=2))()
    assert bench.run_reference(args, bench.WORKLOADS["eu"], 1) == 0
    assert capsys.readouterr().out == ""


def test_fifo_finish_times():
    """One server, arrival order: a job waits for the previous one."""
    import numpy as np
    import bench
    fin = bench.fifo_finish(np.array([0.0, 0.5, 0.6, 5.0]), np.array([1.0, 1.0, 0.5, 0.25]))
    assert np.allclose(fin, [1.0, 2.0, 2.5, 5.25])


def test_oracle_sample_runs_one_process_per_core():
    """The CPU baseline of the batched workload: independent graphs through the
    oracle in a 'spawn' pool; every graph is run once and the CPU seconds add up."""
    import bench
    from paper_2210_03211_gb300 import workloads as W
    graphs = [W.planted_er(n=120, num_comms=4, size_lo=10, size_hi=30, seed=s) for s in range(5)]
    gps, cpu_s = bench.oracle_graphs_per_s(graphs, 4, 0.01, 50, 2)
    assert gps > 0 and cpu_s > 0
    # the wall time of the sample cannot be below its CPU time spread over two processes
    assert len(graphs) / gps >= cpu_s / 2 * 0.9
    assert bench.host_cores() >= 1


def test_traffic_is_reported_only_for_the_captured_source(tmp_path, monkeypatch):
    """The committed ncu traffic counts are reported only for the source,
    workload and queue size they were captured for (else None)."""
    import hashlib
    import bench
    src_dir = tmp_path / "paper_2210_03211_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = src_dir / "lf_run.cu"
    src.write_text("// kernel source\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles" / "k_eval_traffic.txt").write_text(
        "# comment: with a colon\nsource: lf_run.cu\n"
        f"source_sha256_16: {sha}\ndram_bytes_per_launch_scaled: 2977331\ncaptured_on: test\n"
        "bench_workload: large\nbench_queue_size: 65536\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("k_eval", "large", 65536) == {"bytes_per_launch": 2977331.0, "workload": "test"}
    assert bench.ncu_traffic("k_eval", "large", 1024) is None
    assert bench.ncu_traffic("k_eval", "dblp", 65536) is None
    src.write_text("// kernel source, changed\n")
    assert bench.ncu_traffic("k_eval", "large", 65536) is None
    assert bench.ncu_traffic("k_other", "large", 65536) is None


def test_measured_peak_and_its_fallback(tmp_path, monkeypatch):
    import json
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_hbm() == (bench.FALLBACK_HBM_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6813.8, "bf16_tflops": 1900}))
    assert bench.measured_hbm() == (6813.8, "measured")


def test_clock_samples_give_median_max_and_reasons(tmp_path):
    import bench
    s = bench.ClockSampler("GPU-0")
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as f:
        f.write("2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n")
        f.write("1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n")
        f.write("2055, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n")
        f.write("[N/A]\n")
    out = s.stop()
    assert out == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_host_info_names_the_cpu():
    import bench
    h = bench.host_info()
    assert h["nproc"] == bench.host_cores() >= 1 and h["machine"]
    assert h["cpu_model"] is None or isinstance(h["cpu_model"], str)
