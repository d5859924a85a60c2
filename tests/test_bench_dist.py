"""Host logic of the N > 1 benchmark path on CPU ranks (gloo, world size 2):
every rank solves its own replica, the reported time is the maximum over
ranks, and only rank 0 of the reference arm does any work."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, l = bench.dist_setup()
        assert (w, r, l) == (world, rank, rank)
        elapsed = 10.0 + 5.0 * rank
        out[rank] = bench.max_over_ranks(elapsed, world)
        p = bench.replica_problem(rank)
        out[world + rank] = p.seed
        args = type("A", (), {"steps": 1, "warmup": 0, "gpus": world, "reference_particles": 8,
                              "workload": "c3"})()
        if rank != 0:
            assert bench.run_reference(args, world, rank) == 0   # returns at once
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks_take_max_time_and_distinct_replicas():
    world = 2
    port = _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    assert out[0] == out[1] == 15.0
    assert out[2] != out[3]


def test_units_and_flops_per_unit():
    import scenarios as S
    p = S.config2()
    assert bench.units_per_solve(p) == 65536 * 32 * 8 * 60 * 30
    f = bench.flops_per_unit(p)
    assert 150 < f < 400
    assert bench.flops_per_unit(S.config3()) > f          # more pairs, soft form, noise
    assert bench.flops_per_unit_tally(S.config3()) > bench.flops_per_unit_tally(p)
    assert bench.fp32_peak_tflops(152, 2070) == pytest.approx(80.54, rel=1e-3)


def test_oracle_sample_charges_the_wind_generation_at_its_share(monkeypatch):
    """The CPU baseline's solve runs on the workload's wind field, generated
    once; the generation time enters each sample at the share L_sample / L."""
    import time

    import oracle as O
    seen = []
    monkeypatch.setattr(O, "wind_field", lambda p: (time.sleep(0.25), "field")[1])
    monkeypatch.setattr(O, "smc_solve", lambda p, W=None, nthreads=1: seen.append((p.L, W, nthreads)))
    bench._ORACLE_WIND.clear()
    try:
        for wl, full in (("c2", 65536), ("c3", 262144)):
            seen.clear()
            v, dt, units = bench.oracle_sample(wl, 512, 3)
            _, dt2, _ = bench.oracle_sample(wl, 512, 3)          # the field is not generated again
            t_wind = bench.oracle_wind(wl)[1]
            assert seen == [(512, "field", 3), (512, "field", 3)]
            p = bench.workload_problem(wl)
            assert units == 512 * p.M * p.N * p.H * p.J_max
            assert t_wind >= 0.25
            share = t_wind * 512 / full
            assert share <= dt < share + 0.05 and share <= dt2 < share + 0.05
            assert v == pytest.approx(units / dt)
    finally:
        bench._ORACLE_WIND.clear()


def test_workloads_name_their_problem():
    for wl, spec in bench.WORKLOADS.items():
        p = bench.workload_problem(wl)
        assert f"{p.N}ac-L{p.L}-M{p.M}-H{p.H}-grid{'x'.join(str(g) for g in p.grid)}-J{p.J_max}" in spec["name"]
    p = bench.workload_problem("c3")
    assert (p.N, p.L, p.M, p.H, p.w_noise, p.sep_mode) == (24, 262144, 64, 120, 0.1, 2)
