"""Multi-GPU form = replicas: one process per GPU, each solving its own batch
with no exchange on the data path; the job's time is the slowest rank's and
its work the sum over ranks.  The host-side logic (rank aggregation, the
reference arm's rank filter) runs here as world-size-2 gloo groups on CPU."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _combine_worker(rank, world, port, q):
    import time

    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        # rank r: a replica that took 10 + 5 r ms for 100 (r + 1) units
        dist.barrier()
        t0 = time.perf_counter()
        time.sleep(0.02 * rank)  # uneven ranks: the barrier below waits for the slowest
        dist.barrier()
        waited = time.perf_counter() - t0
        T, U = bench.combine_ranks(10.0 + 5.0 * rank, 100.0 * (rank + 1), dist)
        q.put((rank, T, U, waited))
    finally:
        dist.destroy_process_group()


def test_combine_ranks_gloo_world2():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_combine_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, T, U, waited in out:
        assert T == 15.0          # MAX over ranks
        assert U == 300.0         # SUM over ranks
        assert waited >= 0.015    # both ranks left the barrier after the slow one arrived
    # one rank: its own numbers
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(7.0, 11.0, None) == (7.0, 11.0)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_json_contract():
    """Rank 0 of the reference arm (the FP64 oracle on a bounded sample of
    the throughput workload, host cores only) prints one JSON line with the
    keys of the benchmark contract."""
    import json
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.strip().splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "Mpixel*iter/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


@pytest.mark.gpu
def test_bench_json_contract_gpu():
    """A short run of the GPU arm prints one JSON line with the contract's
    keys: roofline of the trial kernel, e2e through the C ABI with host
    buffers, the clock record of the timed region, launch count."""
    import json
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "1", "--warmup", "3",
                        "--n512", "1", "--n256", "1", "--iters", "5", "--no-cpu-baseline", "--no-forms"],
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.strip().splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert key in d, key
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["dtype"] == "f32" and d["gpu_launches"] > 0
    rf = d["roofline"]
    assert rf["bound"] == "alu" and rf["unit"] == "TFLOP/s" and 0 < rf["frac"] < 1.5
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-3
    # the FP32 peak is the measured FMA rate; the SM count comes from the device
    pk = d["peaks"]
    assert pk["sms"] > 0 and pk["ffma"] > 0 and rf["peak"] == pytest.approx(pk["ffma"], rel=1e-3)
    # derived peak = SMs x 128 lanes x 2 flop x a clock between 1 and 2.1 GHz
    assert 1.0e3 <= rf["peak_derived"] * 1e6 / (pk["sms"] * 256) <= 2.1e3
    assert 0.5 < pk["ffma"] / rf["peak_derived"] < 1.05
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    # a timed region this short may end before the 200 ms clock sampler sees
    # the GPU under load: null, else the median clock and the throttle reasons
    assert d["clocks"] is None or ("sm_mhz" in d["clocks"] and "reasons" in d["clocks"])
