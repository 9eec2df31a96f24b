"""Host-side logic of bench.py: the multi-rank timing path on gloo ranks
(world size 2, CPU), the throughput formula and the oracle-arm sizing."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import bench
dist = bench.dist_setup(int(os.environ["WORLD_SIZE"]))
rank = int(os.environ["RANK"])
bench.barrier(dist)
t = bench.max_over_ranks(10.0 + 5.0 * rank, dist)      # ranks report 10 ms and 15 ms
v = bench.job_throughput(int(os.environ["WORLD_SIZE"]), 1000, 4, t)
print(json.dumps({{"rank": rank, "max_ms": t, "value": v, "backend": dist.get_backend()}}))
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_gloo_ranks_take_the_max_time():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["backend"] == "gloo"
        assert o["max_ms"] == 15.0
        # 2 ranks x 1000 voxels x 4 steps in the slowest rank's 15 ms
        assert o["value"] == pytest.approx(2 * 1000 * 4 / 0.015)


def test_single_rank_needs_no_process_group():
    assert bench.dist_setup(1) is None
    assert bench.max_over_ranks(3.5, None) == 3.5


def test_reference_crop_is_bounded():
    for steps, warm in ((1, 3), (10, 3), (200, 10), (5000, 10)):
        n1, n2, n3 = bench.reference_crop(steps, warm)
        assert n1 == n2 and 16 <= n1 <= 512 and n1 % 16 == 0 and n3 == 224
        est = (steps + warm) * n1 * n2 * n3 / 1.5e6
        assert est <= 130 or n1 == 16


def test_reference_crop_fits_the_memory():
    """The crop is cut so that one oracle process per core fits in 60 % of
    the available memory (8 processes of a 352x352x224 crop would need about
    110 GB)."""
    for procs, avail in ((8, 62e9), (16, 62e9), (16, 400e9), (1, 4e9)):
        n1, n2, n3 = bench.reference_crop(3, 3, procs=procs, avail=avail)
        assert n1 == n2 and 16 <= n1 <= 512 and n1 % 16 == 0 and n3 == 224
        assert procs * n1 * n2 * n3 * bench.ORACLE_BYTES_PER_VOXEL <= 0.6 * avail or n1 == 16
    # enough memory: the time budget alone decides
    assert bench.reference_crop(3, 3, procs=1, avail=1e15) == bench.reference_crop(3, 3, procs=1, avail=0)


def test_oracle_timing_runs_on_a_small_crop():
    value, dt = bench.time_oracle(1, 0, shape=(16, 16, 8))
    assert value > 0 and dt > 0


def test_k1_traffic_record_is_keyed_on_the_translation_unit(tmp_path, monkeypatch):
    """The recorded DRAM bytes of K1 are valid for one translation unit: its
    source and the package headers it includes.  A change to an included
    header (as a change to the source) invalidates the record, so the bench
    line reports no traffic for a kernel the counters were not taken on."""
    import shutil
    from paper_2510_00562_gb300 import build
    csrc = tmp_path / "csrc"
    shutil.copytree(build.CSRC, csrc, ignore=shutil.ignore_patterns("*.o", "*.so"))
    monkeypatch.setattr(build, "CSRC", str(csrc))
    sha0 = bench.k1_source_sha("tma")
    assert sha0 == bench.k1_source_sha("tma")
    # the committed record matches the tree as it stands
    rec = json.load(open(os.path.join(ROOT, "profiles", "k1_traffic.json")))
    assert rec["tma"]["sha256"] == sha0
    assert bench.k1_traffic_record("fp32", "tma") == rec["tma"]["fp32"]["bytes_per_voxel"]
    # a header two includes deep (k_stencil_tma.cu -> gsstv_l1.cuh -> gsstv_internal.cuh)
    hdr = csrc / "gsstv_internal.cuh"
    hdr.write_bytes(hdr.read_bytes() + b"\n// edited\n")
    assert bench.k1_source_sha("tma") != sha0
    assert bench.k1_traffic_record("fp32", "tma") is None
