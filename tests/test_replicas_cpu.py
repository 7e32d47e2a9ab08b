"""The multi-GPU path of bench.py on the CPU: replicas only (the solve has no
exchange step), timed by the slowest rank; world size 2 over gloo."""

import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 3.0 + rank                    # rank 1 is the slower replica
    ms_max = bench.rank_max(torch, dist, ms, "cpu")
    out[rank] = (ms_max, bench.replica_value(1000, world, ms_max))
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_sets_the_time():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms_max, value = res[r]
        assert ms_max == 4.0
        # both replicas' interactions over the slowest time
        assert value == pytest.approx(1000 * world / 4.0e-3)


def test_single_process_needs_no_group():
    assert bench.rank_max(torch, None, 2.5, "cpu") == 2.5
    assert bench.replica_value(10, 1, 2.0) == pytest.approx(5000.0)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_line_on_rank_0():
    """The oracle arm (no GPU needed) prints one JSON line with the keys the
    contract asks for: the same metric, unit and direction as the GPU arm,
    impl = reference, a cpu_baseline describing the run and an e2e object
    with no host-device traffic."""
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["warmup"] == 3 and d["value"] > 0 and d["vs_baseline"] is None
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("cfg5")


def test_m2l_rates_by_kernel():
    """Each same-level kernel's rate is its own interactions over its own
    time; a kernel that did not run (no time or no work) is left out."""
    per_kernel = {"multipole": {"ms_per_step": 2.0}, "monopole": {"ms_per_step": 0.5},
                  "root": {"ms_per_step": 0.0}, "pack": {"ms_per_step": 9.0}}
    rates = bench.m2l_rates_by_kernel(per_kernel, [1000, 3000, 40, 7])
    assert rates == {"mp<-mp and mp<-mono (multipole kernel)": 1000 / 0.002,
                     "mono<-mono (monopole kernel)": 3000 / 0.0005}
    assert bench.m2l_rates_by_kernel({}, [1, 2, 3, 4]) == {}


def test_per_cell_force_errors():
    """Per-cell relative errors use vector norms, skip cells whose reference
    field is below the floor, and take nearest-rank quantiles."""
    import torch
    g_ref = torch.zeros(1, 3, 512, dtype=torch.float64)
    g_ref[0, 0, :] = 1.0                      # |g_ref| = 1 in every cell ...
    g_ref[0, 0, 500:] = 1e-6                  # ... but 12 cells below the floor
    g = g_ref.clone()
    rel = torch.arange(500, dtype=torch.float64) * 1e-8   # 0, 1e-8, ..., 4.99e-6
    g[0, 1, :500] = rel                       # an orthogonal error of that size
    g[0, 2, 500:] = 1.0                       # huge errors where the floor excludes
    out = bench.per_cell_force_errors(g, g_ref)
    assert out["cells"] == 500
    assert out["median"] == rel[249].item()
    assert out["p99"] == rel[int(0.99 * 499)].item()


def test_direct_field_of_two_masses():
    """The bench's O(N^2) reference field (order sweep): two point masses
    attract each other with G m / r^2, self term excluded, in blocks."""
    import numpy as np
    pos = np.array([[0.0, 0.0, 0.0], [3.0, 0.0, 4.0]] + [[10.0 + i, 0.0, 0.0] for i in range(300)])
    m = np.zeros(len(pos))
    m[0], m[1] = 2.0, 5.0
    g = bench._direct_field(pos, m, G=1.5)
    np.testing.assert_allclose(g[0], 1.5 * 5.0 / 125.0 * np.array([3.0, 0.0, 4.0]), rtol=1e-14)
    np.testing.assert_allclose(g[1], -1.5 * 2.0 / 125.0 * np.array([3.0, 0.0, 4.0]), rtol=1e-14)
