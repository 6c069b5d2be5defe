"""Host-side logic of bench.py without a GPU: the reference-arm line, the
max-over-ranks timing of replicas with two gloo ranks, rank > 0 of the
reference arm doing no work."""
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


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True,
                         check=True, cwd=ROOT, timeout=600).stdout.strip().splitlines()
    assert len(out) == 1
    d = json.loads(out[0])
    assert d["impl"] == "reference" and d["metric"] == "MLUPS" and d["unit"] == "MLUPS"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["nx"] == 2048 and d["config"]["ny"] == 8192


def test_reference_arm_other_ranks_do_no_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "1", "--gpus", "2"], capture_output=True,
                       text=True, cwd=ROOT, env=env, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def _rank(rank, port, secs, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=2)
    q.put((rank, bench.max_over_ranks(secs[rank], dist)))
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    secs = [0.25, 0.75]
    ps = [ctx.Process(target=_rank, args=(r, port, secs, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
    assert res == {0: 0.75, 1: 0.75}


def test_max_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.5, None) == 1.5


def test_kernel_hash_ignores_comments_not_code(tmp_path):
    """The recorded ncu traffic is tied to the step kernels' code: a comment
    edit keeps the hash, a code edit changes it (bench.py then reports the
    traffic as unknown until the kernel is profiled again)."""
    import shutil
    sys.path.insert(0, ROOT)
    import bench
    src = os.path.join(ROOT, "paper_2103_02119_gb300", "csrc")
    for f in bench.STEP_KERNEL_SOURCES:
        shutil.copy(os.path.join(src, f), tmp_path / f)
    base = bench.step_kernel_hash(str(tmp_path))
    assert base == bench.step_kernel_hash()
    p = tmp_path / "step_block.cuh"
    text = p.read_text()
    p.write_text(text.replace("namespace lbm {", "namespace lbm {  // a remark\n/* a block\n remark */", 1))
    assert bench.step_kernel_hash(str(tmp_path)) == base
    p.write_text(text.replace("constexpr int kHalo = 4;", "constexpr int kHalo = 8;", 1))
    assert bench.step_kernel_hash(str(tmp_path)) != base


def test_recorded_traffic_per_variant():
    """The committed ncu traffic record holds the FP32 step with and without
    a link mask and the FP64 step, each tied to the current kernels' code;
    bench.py scales the per-cell bytes to its grid and reads the masked
    entry only for a masked line."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    with open(os.path.join(ROOT, "profiles", "rc_step_traffic.json")) as fh:
        rec = json.load(fh)
    cells = 2048 * 8192
    for key, prec, mask, algo in (("fp32", 32, False, 72), ("fp32_mask", 32, True, 73),
                                  ("fp64", 64, False, 144)):
        e = rec[key]
        assert e["kernel_sha"] == bench.step_kernel_hash(), key
        assert abs(e["dram_bytes_per_cell"] - algo) <= 0.03 * algo, key
        assert bench.profiled_traffic(prec, cells, mask) == e["dram_bytes_per_cell"] * cells
