"""Host-side logic of bench.py on CPU: the max-over-ranks timing with a
world_size-2 gloo group, the clock-record parser, the ALU peak."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    def reduce_max(v):
        t = torch.tensor([v], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    got = bench.aggregate(1.0 + rank, world, reduce_max)
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == 2.0 and out[1] == 2.0


def test_clock_parser_and_peaks():
    import bench
    c = bench.ClockSampler(0)
    c.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout=None: 0,
                            "kill": lambda self: None})()
    c.lines = ["0, 1500, 2070, 900.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
               "0, 1700, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage"]
    r = c.stop()
    assert r["sm_mhz"] == 1600.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]
    assert abs(bench.alu_peak_tflops(False, 2070.0) - 152 * 128 * 2 * 2.07e-3) < 1e-9
    assert bench.alu_peak_tflops(True, 2070.0) == 1.25


def test_batch_generator_mix():
    import math
    from synthetic import circuits as sc
    insts = sc.batch_instances(64, seed=0)
    ns = {b.rows * b.cols for b in insts}
    assert ns <= set(sc.BATCH_GRIDS) and len(ns) >= 5
    assert all(8 <= b.cycles <= 20 and b.chi in sc.BATCH_CHIS for b in insts)
    assert all(len(b.circuit.layers) == math.ceil(b.cycles / 2) for b in insts)
    again = sc.batch_instances(64, seed=0)
    assert [(b.rows, b.cycles, b.chi, b.seed) for b in insts] == [(b.rows, b.cycles, b.chi, b.seed) for b in again]


def test_sequence_two_pattern_order():
    """Sequence II uses the patterns in the order CDBA-BACD; every cycle is a
    matching (no qubit twice) and eight cycles cover every grid edge twice."""
    import collections
    from synthetic import circuits as sc
    c2 = sc.random_circuit(4, 5, 8, cycles_per_layer=1, seed=3, pattern_order=sc.PATTERN_ORDER_II)
    pats = sc.grid_edges(4, 5)
    count = collections.Counter()
    for cyc, layer in enumerate(c2.layers):
        pairs = [(a, b) for (a, b, u) in layer if b >= 0]
        assert sorted(pairs) == sorted(pats[sc.PATTERN_ORDER_II[cyc]])
        qs = [q for p in pairs for q in p]
        assert len(qs) == len(set(qs))
        count.update(tuple(sorted(p)) for p in pairs)
    assert set(count.values()) == {2} and len(count) == len(sc.all_edges(4, 5))


def test_reference_step_visits_every_cost_stratum():
    """A step of the reference arm times one oracle update at the middle bond
    of each of four equal-frequency cost strata, so the mean of its updates
    estimates the layer's mean update (a 3 x 4 grid at chi = 8 keeps it fast)."""
    import bench
    from synthetic import circuits as sc
    circ = sc.random_circuit(3, 4, 4, seed=0)
    shapes = bench.workload_shapes(3, 4, 8, circ.layers[1])
    strata = bench.stratified_bonds(shapes, 4)
    flops = sorted(bench.update_flops(s) for s in shapes)
    assert [bench.update_flops(shapes[i]) for i in strata] == sorted(bench.update_flops(shapes[i]) for i in strata)
    assert len(set(strata)) == 4
    done, secs, threads, bonds = bench.reference_step(shapes)
    assert done == 4 and secs > 0 and threads >= 1
    assert sorted(bonds) == sorted(strata)
    # the middle of each quarter of the cost order
    for k, i in enumerate(strata):
        assert bench.update_flops(shapes[i]) == flops[min(len(flops) - 1, int((k + 0.5) * len(flops) / 4))]
