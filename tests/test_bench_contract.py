"""bench.py's JSON line on the CPU: the host-side bookkeeping of the timed
loop run against stand-ins for the CUDA events and the library context (no
GPU), checked for every key of the benchmark contract and for the arithmetic
that turns event times into the reported rates."""
import itertools
import json

import numpy as np
import pytest

STAT_KEYS = ["gemm_ms", "gemm_flops", "gemm_launches", "svd_ms", "svd_flops", "svd_launches", "jacobi_sweeps",
             "mpo_ms", "other_ms", "updates", "kernel_launches", "rsvd_attempts", "rsvd_accepted", "eig_svds",
             "eig_fallbacks", "eig_skipped"]


class _Event:
    ticks = itertools.count()

    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        self.t = next(_Event.ticks)

    def elapsed_time(self, other):   # 10 ms per recorded event in between
        return 10.0 * (other.t - self.t)


class _Stream:
    cuda_stream = 0


class _Ctx:
    def __init__(self, rows, cols, chi, precision=0, timing=False, stream=None, order="V", groups=None, **opts):
        self.n, self.chi, self.h = rows * cols, chi, 1
        self.st = {k: 0 for k in STAT_KEYS}

    def _bump(self):
        for k in self.st:
            self.st[k] += 1

    def sweep(self, n):
        self._bump()
        return 0.5

    def stats(self):
        return dict(self.st)

    def reset_stats(self):
        self.st = {k: 0 for k in STAT_KEYS}

    def fidelity(self):
        return -1.0, 0.5

    def history(self):
        return [0.5] * (2 * (self.n - 1))

    def amplitude(self, bits):
        self._bump()
        return np.zeros(len(bits), dtype=np.complex128)

    def bond_dims(self):
        return [self.chi] * (self.n - 1), [4] * (self.n - 1)

    def get_mps(self):
        return [], 0

    def close(self):
        pass


class _Lib:
    def dmrgc_apply_layer(self, h, gates, n):
        return 0


def test_bench_line_has_every_contract_key(monkeypatch, capsys):
    import torch

    import bench
    import paper_2207_05612_gb300 as pkg
    from paper_2207_05612_gb300 import binding
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "set_device", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a, **k: _Stream())
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(pkg, "Context", _Ctx)
    monkeypatch.setattr(binding, "lib", lambda: _Lib())
    monkeypatch.setattr(binding, "dmrgc_set_jacobi_kernel", lambda v: None)
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.main(["--steps", "2", "--warmup", "3", "--no-cpu-baseline", "--fp64-updates", "0"]) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "e2e", "roofline", "cpu_baseline",
                "clocks", "gpu_launches"):
        assert key in line, key
    assert line["metric"] == "two-site updates/s" and line["unit"] == "updates/s"
    assert line["n_gpus"] == 1 and line["steps"] == 2 and line["warmup"] == 3
    assert line["higher_is_better"] is True and line["scaling"] == "weak" and line["vs_baseline"] is None
    assert "workload" in line["config"] and line["config"]["chi"] == 512
    for key in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert key in line["e2e"]
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in line["roofline"]
    assert line["roofline"]["frac"] == pytest.approx(line["roofline"]["achieved"] / line["roofline"]["peak"])
    # each step records start, split and end events 10 ms apart: apply_layer and
    # the sweep take 10 ms each, a step 20 ms; 106 updates per step
    assert line["ms_per_step"] == pytest.approx(20.0)
    assert line["value"] == pytest.approx(2 * 106 / 0.040)
    assert line["excluding_mpo_and_guess"]["value"] == pytest.approx(2 * 106 / 0.020)
    assert line["excluding_mpo_and_guess"]["apply_layer_ms_per_step"] == pytest.approx(10.0)
    assert line["gpu_launches"] > 0


def test_reference_arm_line(monkeypatch, capsys):
    """--impl reference (the oracle on the host cores) on a small grid: the
    same metric and config keys, impl = reference, its own cpu_baseline and an
    e2e without host-device traffic; value = the four stratum updates of each
    step over their time."""
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    argv = ["--impl", "reference", "--steps", "2", "--warmup", "1", "--rows", "3", "--cols", "4", "--chi", "8"]
    assert bench.main(argv) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == "two-site updates/s"
    assert line["unit"] == "updates/s" and line["higher_is_better"] is True and line["steps"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "updates/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["value"] == pytest.approx(2 * 4 / (2e-3 * line["ms_per_step"]))


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"]) == 0
    assert capsys.readouterr().out.strip() == ""
