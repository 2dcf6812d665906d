"""The bench's whole-job aggregation over independent replicas (2 gloo ranks
on CPU): the value is the work of all ranks over the slowest rank's time."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    total_ms = 100.0 * (rank + 1)              # rank 1 is the slowest replica
    value, t_max = bench.aggregate(total_ms, units_per_step=1000.0, steps=5)
    out[rank] = (value, t_max)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_replicas():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        value, t_max = out[r]
        assert t_max == pytest.approx(200.0)
        assert value == pytest.approx(1000.0 * 5 * 2 / 0.2)


def test_aggregate_single_process():
    import bench

    value, t_max = bench.aggregate(50.0, units_per_step=10.0, steps=4)
    assert t_max == 50.0 and value == pytest.approx(10.0 * 4 / 0.05)


def test_clock_summary_reports_median_clock_and_active_reasons():
    """The timing rules reject runs that saw thermal or hardware slowdown:
    the sampler must report every reason that was active in any sample and
    the median SM clock under load."""
    import bench

    s = bench.ClockSampler(0)
    s.lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2050, 2070, 1399.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1400.2, 0x0000000000000008, Active, Not Active, Not Active, Active",
        "garbage line",
    ]
    out = s.summary()
    assert out["sm_mhz"] == 2050 and out["sm_max_mhz"] == 2070 and out["samples"] == 3
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]
    s.lines = []
    assert s.summary()["reasons"] == ["unsampled"]


def test_pcg_bytes_model_counts_the_tridiagonal_extras():
    import bench

    jac = bench.pcg_bytes_per_row_lane(True, 0.13, 6.9, 64)
    tri = bench.pcg_bytes_per_row_lane(True, 0.13, 6.9, 64, tri=True)
    assert 60 < jac < 90 and tri > jac
    assert bench.pcg_bytes_per_row_lane(False, 0.13, 6.9, 64) > jac      # FP64 vectors


def test_fine_byte_model_plain_cg_part_is_the_scope_model():
    """The plain CG part of the bench's per-(row, lane, iteration) byte model
    is 7 s phi + 7 (s (1 - phi) + 4) / N + 13 s: 56.5 B in FP32 for the medium
    workload (phi = 2600 / 19801 special rows, N = 64).  The V-cycle adds 11
    fine-level vector passes, the special rows' Jacobian twice with their l1
    norms, and 10 passes per coarse level scaled by its length."""
    import bench

    b = bench.fine_bytes_per_row_lane_round(True, 2600 / 19801, 64, [])
    assert abs(b["pcg"] - 56.49) < 0.01 and b["vcycle"] == 0.0
    rows = [19801, 4488, 739, 148]
    b = bench.fine_bytes_per_row_lane_round(True, 2600 / 19801, 64, rows)
    coarse = sum(rows[1:]) / rows[0]
    assert abs(b["vcycle"] - (44 + 64 * 2600 / 19801 + 40 * coarse)) < 1e-9
    assert b["total"] == b["pcg"] + b["vcycle"]
