"""Host-side checks of the benchmark driver: the multi-process path (replicas, barrier and the
max over ranks) with two gloo ranks on the CPU, and the CPU reference arm's JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    assert bench.dist_env() == (rank, world, rank)
    bench.barrier(world)
    v = bench.reduce_max(float(10 * (rank + 1)), world)   # per-rank step times: the job takes the slowest
    out.put((rank, v))
    bench.barrier(world)
    dist.destroy_process_group()


def test_replicas_barrier_and_max_over_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 20.0), (1, 20.0)]


def test_reference_arm_json_line():
    """`bench.py --impl reference` times the CPU oracle and prints one JSON line."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "c1",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "unknowns/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["higher_is_better"] is True and line["config"]["name"] == "c1"


def test_recorded_traffic_is_keyed_on_kernel_source(tmp_path, monkeypatch):
    """Recorded DRAM traffic is reported only while the kernels' source is the one captured: an
    edit to the factor section or the substitution kernels drops it to None, an edit to the
    host-side handle struct does not."""
    sys.path.insert(0, ROOT)
    import json
    import shutil

    import bench

    root = tmp_path / "tree"
    csrc = root / "paper_2504_07269_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = os.path.join(ROOT, "paper_2504_07269_gb300", "csrc")
    for name in ("k_band.cu", "k_subst.cu", "async.cuh", "device.cuh", "k_mf.cu"):
        shutil.copy(os.path.join(src, name), csrc / name)
    (root / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(root))
    rec = {"band_factor_fp32_c3": {"k_band_sha": bench.kernel_source_sha(), "dram_bytes_per_launch": 1.0e12},
           "mf_subst_fp32_c3": {"src_sha": bench.kernel_source_sha("mf"), "dram_bytes_per_launch": 2.0e11}}
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.profiled_traffic("band_factor_fp32_c3") == 1.0e12
    assert bench.profiled_traffic("band_factor_fp32_c2") is None      # no capture of that workload
    assert bench.profiled_traffic("mf_subst_fp32_c3", "mf") == 2.0e11
    assert bench.profiled_traffic("mf_subst_fp32_c3") is None         # recorded against the multifrontal source
    mf = (csrc / "k_mf.cu").read_text()
    (csrc / "k_mf.cu").write_text(mf + "\n// edited\n")
    assert bench.profiled_traffic("mf_subst_fp32_c3", "mf") is None   # multifrontal source changed
    assert bench.profiled_traffic("band_factor_fp32_c3") == 1.0e12    # the banded record is unaffected
    (csrc / "k_mf.cu").write_text(mf)
    dev = (csrc / "device.cuh").read_text()
    (csrc / "device.cuh").write_text(dev.replace("struct st_fdm {", "struct st_fdm {\n    int host_only_field = 0;", 1))
    assert bench.profiled_traffic("band_factor_fp32_c3") == 1.0e12             # host bookkeeping only
    dev = (csrc / "device.cuh").read_text()
    (csrc / "device.cuh").write_text(dev.replace("struct BandArgs {", "struct BandArgs {\n    int extra;", 1))
    assert bench.profiled_traffic("band_factor_fp32_c3") is None               # the banded kernels' arguments changed
    (csrc / "device.cuh").write_text(dev)
    sub = (csrc / "k_subst.cu").read_text()
    (csrc / "k_subst.cu").write_text(sub + "\n// edited\n")
    assert bench.profiled_traffic("band_factor_fp32_c3") is None               # kernel source changed
