"""The multi-process side of bench.py on CPU (world size 2, gloo): the job's time is the
slowest rank's, the ranks share one build per step (the auxiliary index sharded over them),
and a single process needs no group."""
import os
import socket

import pytest
import torch
import torch.distributed as tdist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms = [12.5, 20.0][rank]
        m = bench.max_over_ranks(ms, ws, torch.device("cpu"))
        out[rank] = (m, bench.job_rate(m))
    finally:
        tdist.destroy_process_group()


def test_two_ranks_take_the_slowest_clock():
    ws, port = 2, _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
    for r in range(ws):
        m, rate = out[r]
        assert m == 20.0
        assert rate == pytest.approx(1e3 / 20.0)


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(7.0, 1, torch.device("cpu")) == 7.0
    assert bench.job_rate(8.0) == pytest.approx(125.0)
    assert bench.job_rate(8.0, 64) == pytest.approx(8000.0)


def test_roofline_peak_follows_the_timed_region():
    """Burst peak for a short region at full clocks; sustained for a long region, for
    clocks well below their maximum, and as the fallback when the file lacks a figure."""
    pk = {"bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
    full = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0}
    assert bench.tensor_peak(pk, 0.1, full) == ("burst", 1900.0)
    assert bench.tensor_peak(pk, 3.0, full) == ("sustained", 1700.0)
    assert bench.tensor_peak(pk, 0.1, {"sm_mhz": 1500.0, "sm_max_mhz": 2070.0}) == \
        ("sustained", 1700.0)
    assert bench.tensor_peak(pk, 0.1, None) == ("burst", 1900.0)
    kind, peak = bench.tensor_peak({}, 0.1, full)
    assert kind == "burst" and peak == bench.FALLBACK_PEAKS["bf16_tflops"]
