"""bench.py host logic on the CPU: the multi-rank path (gloo, world size 2,
127.0.0.1 rendezvous) reduces the slowest rank's time and aggregates the
whole-job real-time factor; the per-workload flop and sample counts follow
the definitions (8 flop per complex MAC over the baseline triangle)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    t = 100.0 + 50.0 * rank                       # rank 1 is slower
    bench.barrier(ws)
    mx = bench.max_over_ranks(t, ws)
    out[rank] = (mx, bench.aggregate_value(1.00663 * 5, ws, mx / 1e3))
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        mx, val = out[rank]
        assert mx == 150.0                        # slowest rank's time on every rank
        assert val == pytest.approx(1.00663 * 5 * 2 / 0.150)


def test_workload_counts():
    w = bench.WORKLOADS["lofar16_fp32"]
    assert bench.sky_seconds(w) == pytest.approx(1.00663, rel=1e-5)
    # 8 * 2080 baselines * 4 products * 64 channels * 3072 spectra * 244 subbands
    assert bench.useful_xflops(w) == pytest.approx(3.1930e12, rel=1e-4)
    assert bench.samples(w) == 128 * 3072 * 64 * 244
    assert bench.fp32_alu_peak_tflops(152) == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    # both arms print the same config dict
    assert bench.config_of(w, 1) == bench.config_of(w, 1) and bench.config_of(w, 1)["x_stage"] == "tf32_split"
    # executed tensor work of the TF32 split at 64 stations, per 16 spectra per channel: 4 TF32 MMAs of
    # 128 x 256 x 8 and 4 BF16 MMAs of 128 x 256 x 16
    class _C:
        I_pad, S_pad = 128, 3072
    ex_t, ex_b = bench.executed_xflops_split(_C, w)
    assert ex_t == pytest.approx(4 * 2 * 128 * 256 * 8 * 192 * 64 * 244)
    assert ex_b == pytest.approx(4 * 2 * 128 * 256 * 16 * 192 * 64 * 244)
    # the mixed roofline: at equal peaks the floor is the total flops over the peak
    r = bench.split_roofline(1e12, (2e12, 4e12), 10.0, 1000.0, 1000.0)
    assert r["floor_ms"] == pytest.approx(3.0) and r["frac"] == pytest.approx(0.3)
    assert r["executed_floor_ms"] == pytest.approx(6.0)
    assert bench.aggregate_value(10.0, 1, 2.0) == 5.0


def test_recorded_traffic_requires_matching_source():
    assert bench.recorded_traffic("no_such_kernel", "lofar16_fp32") is None
    assert bench.recorded_traffic("xcorr_f32_kernel", "other_workload") is None
