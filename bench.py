"""Benchmark: two-site updates/s of the circuit-DMRG compression sweep.

Workload (N=1): 54 qubits on a 6x9 grid, Sycamore-like random circuit
(sqrt(X/Y/W) + fSim(pi/2, pi/6), staggered ABCD-CDAB pattern), K = 2 cycles per
compression step, chi = 512, 2 sweeps per step (2(N-1) = 106 two-site updates).
One benchmark step = one compression step of the whole hot path: layer-MPO
build and lossless compression, zip-up guess, 106 updates (theta, truncated
SVD, environments).  The
first --warmup steps grow the bond dimension to chi; the next --steps are timed.

value: updates/s from CUDA events on the library's stream (gate records already
packed); e2e: the same metric by wall clock through the C ABI with host
buffers, including per step the gate upload, the fidelity read-back and the
amplitudes of 1024 bit strings (host bits in, host amplitudes out).
Inputs are far larger than L2 (environment caches of several GB), so no L2 flush.

--impl reference times the CPU oracle on the host cores instead (one oracle
update per step at a bulk bond of the same workload).

Multi-GPU: one independent circuit instance per rank (the sweep of one circuit
is sequential), weak scaling; timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PRECISIONS = {"fp64": 0, "bf16x3": 1, "tf32x3": 2, "fp32": 3}
DTYPE_NAME = {"fp64": "c128-f64", "bf16x3": "c64-bf16x3", "tf32x3": "c64-tf32x3", "fp32": "c64-f32"}
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of each kernel at the shape that dominates the bench (summaries
# in profiles/).  Only reported while the bench runs that kernel variant.
NCU_TRAFFIC = {
    "jacobi_wp4": {"bytes": 10.91e6, "launch": "1024 x 1024 complex64 (saturated bond, chi = 512)",
                   "profile": "profiles/jacobi_wp4_1024x1024_fp32.md"},
    "tc_gemm_bf16x3": {"bytes": 761.73e6, "launch": "M 65536, N 1024, K 512",
                       "profile": "profiles/tc_gemm_65536x1024x512_bf16x3.md"},
}
FP32_LANES_PER_SM = 128
FP64_PEAK_TFLOPS = 1.25   # nominal GB300 FP64 (CUDA cores and tensor cores alike)
N_SMS = 152


# ------------------------------------------------------------------ helpers

T_START = time.perf_counter()


def note(msg: str) -> None:
    """Progress line on stderr (the JSON result is the only stdout line)."""
    print(f"[bench {time.perf_counter() - T_START:7.1f}s] {msg}", file=sys.stderr, flush=True)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(value_local: float, group_world: int, reduce_max):
    """Max over ranks of a local time (reduce_max: callable or None for N=1)."""
    if group_world <= 1 or reduce_max is None:
        return value_local
    return reduce_max(value_local)


def alu_peak_tflops(fp64: bool, sm_mhz: float | None) -> float:
    """CUDA-core FMA peak at the sampled SM clock: 152 SMs x 128 FP32 lanes x 2
    flops x clock; FP64 uses the nominal 1.25 TFLOP/s scaled by the clock."""
    mhz = sm_mhz or 2070.0
    if fp64:
        return FP64_PEAK_TFLOPS * mhz / 2070.0
    return N_SMS * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


# --------------------------------------------------------------- CPU oracle


def workload_shapes(rows: int, cols: int, chi: int, layer, compress: bool = True):
    """Per bond (i, i+1) of a saturated step of the workload, the operand
    shapes of one two-site update: MPS bonds min(2^i, 2^(N-i), chi) (old and
    new state alike) and the layer MPO's bonds (the oracle's MPO of the given
    layer, compressed like the bench's).  Returns [(chi_l, D_l, chi_m, D_m,
    chi_r, D_r)] for bonds 0..N-2."""
    from oracle import mpo as om
    n = rows * cols
    order = om.snake_order(rows, cols)
    dmpo = [1] + om.bond_dims(om.layer_mpo(layer, order, compress=compress)) + [1]
    chib = [min(2 ** min(i, n - i), chi) for i in range(n + 1)]
    return [(chib[i], dmpo[i], chib[i + 1], dmpo[i + 1], chib[i + 2], dmpo[i + 2]) for i in range(n - 1)]


def update_flops(shape) -> float:
    """Complex MACs of one oracle update at a bond (X, Y, theta, environment)."""
    cl, dl, cm, dm, cr, dr = shape
    x = cl * dl * cl * 2 * cm + cl * 2 * cm * dl * 2 * dm      # L B, then W
    y = cr * dr * cr * 2 * cm + cr * 2 * cm * dr * 2 * dm
    th = 2 * cl * 2 * cr * dm * cm
    env = cm * 2 * cl * dm * cm
    return float(x + y + th + env)


def stratified_bonds(shapes, count: int):
    """count bonds of the layer spread evenly over the cost order of one
    update (the middle of each of count equal-frequency strata), so that their
    mean time estimates the mean update of the layer."""
    order = sorted(range(len(shapes)), key=lambda i: update_flops(shapes[i]))
    return [order[min(len(order) - 1, int((k + 0.5) * len(order) / count))] for k in range(count)]


def reference_step(shapes):
    """One step of the reference arm: an oracle update at each of the four
    stratum bonds (their mean time estimates the layer's mean update).
    Returns (updates, seconds, threads, bonds)."""
    return oracle_updates(shapes, float("inf"), seed=0, max_updates=4)


def _oracle_worker(shapes, budget_s, seed, max_updates, whole_rounds, q):
    q.put(oracle_updates(shapes, budget_s, seed, max_updates, whole_rounds))


def oracle_updates_bounded(shapes, budget_s: float, timeout_s: float, seed: int = 0, max_updates: int = 1 << 30,
                           whole_rounds: bool = False):
    """oracle_updates in a spawned process that is stopped after timeout_s
    (one oracle update cannot be interrupted from inside).  Returns the
    result, or None on timeout."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_oracle_worker, args=(shapes, budget_s, seed, max_updates, whole_rounds, q))
    p.start()
    try:
        return q.get(timeout=timeout_s)
    except Exception:
        return None
    finally:
        p.join(5)
        if p.is_alive():
            p.kill()
            p.join(5)


def oracle_updates(shapes, budget_s: float, seed: int = 0, max_updates: int = 1 << 30,
                   whole_rounds: bool = False):
    """Oracle two-site updates (Sec. IV.B: X, Y, theta, truncated SVD, left
    environment) on random tensors of the given shapes (the cost does not
    depend on the values), at four bonds spread over the layer's cost order
    taken in turn, until budget_s of CPU time or max_updates; whole_rounds
    also finishes the round of four bonds it is in, so that every stratum
    counts equally.  Returns (updates, seconds, threads, bonds)."""
    from oracle import dmrg as od
    rng = np.random.default_rng(seed)

    def rnd(*shape):
        return rng.normal(size=shape) + 1j * rng.normal(size=shape)

    done, spent, picked = 0, 0.0, []
    strata = stratified_bonds(shapes, 4)
    while done < max_updates and (done == 0 or spent < budget_s or (whole_rounds and done % len(strata))):
        i = strata[(done + seed) % len(strata)]
        cl, dl, cm, dm, cr, dr = shapes[i]
        lenv, renv = rnd(cl, dl, cl), rnd(cr, dr, cr)
        b1, b2 = rnd(cl, 2, cm), rnd(cm, 2, cr)
        w1, w2 = rnd(dl, 2, 2, dm), rnd(dm, 2, 2, dr)
        t0 = time.perf_counter()
        x = od.make_x(lenv, b1, w1)
        y = od.make_y(renv, b2, w2)
        th = od.theta_of(x, y)
        u, s, vh, _ = od.svd_truncate(th, cm, 1e-12)
        od.env_left(u.reshape(cl, 2, -1), x)
        spent += time.perf_counter() - t0
        done += 1
        picked.append(i)
    threads = os.cpu_count() or 1
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            threads = max(int(i.get("num_threads", 1)) for i in info)
    except Exception:
        pass
    return done, spent, threads, picked


# ------------------------------------------------------------------- main


STAT_KEYS = ("gemm_ms", "gemm_flops", "svd_ms", "svd_flops", "mpo_ms", "other_ms", "kernel_launches",
             "jacobi_sweeps", "svd_launches", "updates", "eig_svds", "eig_fallbacks", "eig_skipped")


def stats_delta(a: dict, b: dict) -> dict:
    return {k: b[k] - a[k] for k in STAT_KEYS}


def run_ours(args, world, rank, local):
    import torch
    torch.cuda.set_device(local)
    from paper_2207_05612_gb300 import Context, binding
    from synthetic import circuits as sc

    reduce_max = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

        def reduce_max(v):
            t = torch.tensor([v], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            return float(t.item())

    rows, cols = args.rows, args.cols
    n = rows * cols
    layers_needed = args.warmup + args.steps
    cycles = max(20, 2 * layers_needed)
    circ = sc.random_circuit(rows, cols, cycles, seed=args.seed + rank)
    stream = torch.cuda.current_stream()
    prec = PRECISIONS[args.precision]
    ctx = Context(rows, cols, args.chi, precision=prec, timing=True, stream=stream.cuda_stream,
                  mpo_compress=args.mpo_compress, svd_path=args.svd_path)
    packed = [binding.pack_gates(l) for l in circ.layers[:args.warmup]]
    bits = sc.random_bitstrings(n, 1024, seed=7)
    upd_per_step = 2 * (n - 1)
    lf_20 = None

    # warm-up steps: grow the bonds to chi
    for li in range(args.warmup):
        binding._check(binding.lib().dmrgc_apply_layer(ctx.h, packed[li], len(circ.layers[li])), ctx.h)
        ctx.sweep(2)
        if li == 9:
            lf_20 = ctx.fidelity()[0]
        st_w = ctx.stats()
        note(f"warm-up layer {li}: max bond {max(ctx.bond_dims()[0])}, svd {st_w['svd_ms']:.0f} ms, "
             f"gemm {st_w['gemm_ms']:.0f} ms, eigensolver {st_w['eig_svds']} / fallbacks {st_w['eig_fallbacks']}"
             f" / skipped {st_w['eig_skipped']}")
    # the warmed state, for the FP64 comparison on the first timed layer
    warm = None
    if args.fp64_updates > 0 and world == 1 and args.precision != "fp64":
        mps, _ = ctx.get_mps()
        lf_w, fd_w = ctx.fidelity()
        warm = (mps, lf_w)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    ctx.reset_stats()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
    mid = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]   # apply_layer | sweep
    h2d = d2h = 0
    dev_stats = None
    readout = None
    hist0 = None
    t_region0 = time.perf_counter()
    for k in range(args.steps):
        li = args.warmup + k
        layer = circ.layers[li]
        # one step through the public API from host data: gate records packed on
        # the host and copied in by apply_layer; the device part (apply_layer +
        # two sweeps) is bracketed by CUDA events; fidelity and 1024 amplitudes
        # come back to the host
        gates = binding.pack_gates(layer)
        ev[2 * k].record(stream)
        binding._check(binding.lib().dmrgc_apply_layer(ctx.h, gates, len(layer)), ctx.h)
        mid[k].record(stream)
        ctx.sweep(2)
        ev[2 * k + 1].record(stream)
        s_dev = ctx.stats()            # the sweep synchronised: its kernels are counted
        if k == 0:
            hist0 = ctx.history()
        lf_k, _ = ctx.fidelity()
        if li == 9:
            lf_20 = lf_k
        amps = ctx.amplitude(bits)
        s_out = ctx.stats()
        d = stats_delta(s_dev, s_out)
        readout = d if readout is None else {key: readout[key] + d[key] for key in STAT_KEYS}
        h2d += len(layer) * 264 + bits.nbytes
        d2h += amps.size * 16 + 16
        note(f"timed step {k}: svd {s_dev['svd_ms']:.0f} ms, gemm {s_dev['gemm_ms']:.0f} ms, eigensolver "
             f"{s_dev['eig_svds']} / fallbacks {s_dev['eig_fallbacks']} / skipped {s_dev['eig_skipped']} (cumulative)")
    torch.cuda.synchronize()
    t_region = time.perf_counter() - t_region0
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clk = clocks.stop()
    dev_ms = sum(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(args.steps))
    sweep_ms = sum(mid[k].elapsed_time(ev[2 * k + 1]) for k in range(args.steps))
    st_all = ctx.stats()
    st = {key: st_all[key] - readout[key] for key in STAT_KEYS}   # the device-timed part only
    dev_s = aggregate(dev_ms / 1e3, world, reduce_max)
    sweep_s = aggregate(sweep_ms / 1e3, world, reduce_max)
    region_s = aggregate(t_region, world, reduce_max)
    total_updates = upd_per_step * args.steps * world
    lf, fd = ctx.fidelity()
    bonds, dmpo = ctx.bond_dims()
    out = {
        "ctx": ctx, "dev_s": dev_s, "sweep_s": sweep_s, "region_s": region_s, "updates": total_updates, "stats": st,
        "readout": readout, "clocks": clk, "h2d": h2d // args.steps, "d2h": d2h // args.steps, "log_ft": lf,
        "log_ft_20_cycles": lf_20, "f_delta": fd, "max_chi": max(bonds), "max_D": max(dmpo), "rank": rank,
        "n2g": sum(1 for l in circ.layers[:args.warmup + args.steps] for g in l if g[1] >= 0),
        "first_layer": circ.layers[args.warmup], "vs_fp64": None,
    }
    if warm is not None:
        note("FP64 comparison")
        out["vs_fp64"] = fp64_comparison(args, warm, circ.layers[args.warmup], hist0, stream, upd_per_step)
        note(f"FP64 comparison done: {out['vs_fp64']}")
    return out


def fp64_comparison(args, warm, layer, hist_mixed, stream, upd_per_step):
    """The plain FP64 GPU path on the first timed layer from the same warmed
    state (loaded with set_mps): apply_layer (MPO build and zip-up guess) and
    the first --fp64-updates updates of its sweep, each timed with CUDA events;
    the partial fidelities of those updates against the mixed run's."""
    import torch
    from paper_2207_05612_gb300 import Context
    mps, lf_w = warm
    # the complex64 modes' cutoffs, so that both runs apply the same truncation rules
    ctx = Context(args.rows, args.cols, args.chi, precision=PRECISIONS["fp64"], timing=True,
                  stream=stream.cuda_stream, mpo_compress=args.mpo_compress,
                  sweep_rel_cutoff=2e-5, zip_rel_cutoff=4e-3)
    ctx.set_mps(mps, lf_w)
    note("FP64: state loaded")
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record(stream)
    ctx.apply_layer(layer)
    e[1].record(stream)
    ctx.sweep_updates(args.fp64_updates)
    e[2].record(stream)
    torch.cuda.synchronize()
    apply_ms = e[0].elapsed_time(e[1])
    upd_ms = e[1].elapsed_time(e[2])
    h64 = np.array(ctx.history())
    hm = np.array(hist_mixed[:len(h64)])
    ctx.close()
    per_update = upd_ms / 1e3 / max(1, args.fp64_updates)
    step_s = apply_ms / 1e3 + per_update * upd_per_step
    return {"updates_per_s": 1.0 / per_update,
            "step_updates_per_s_estimate": upd_per_step / step_s,
            "apply_layer_s": apply_ms / 1e3, "updates_timed": int(args.fp64_updates), "updates_s": upd_ms / 1e3,
            "max_rel_diff_partial_fidelity": float(np.max(np.abs(h64 - hm) / hm)) if len(hm) else None,
            "sample": f"FP64 context (complex128, the complex64 modes' cutoffs) loaded with the warmed state "
                      f"(set_mps), the first timed layer: apply_layer and the first {args.fp64_updates} updates "
                      "of its sweep, CUDA events; step estimate = apply_layer + 106 x the mean update time; "
                      "max_rel_diff_partial_fidelity: those updates' f against the timed run's"}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=list(PRECISIONS))
    ap.add_argument("--rows", type=int, default=6)
    ap.add_argument("--cols", type=int, default=9)
    ap.add_argument("--chi", type=int, default=512)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--jacobi", default="wp4", choices=["wp4", "gram"],
                    help="complex64 Jacobi kernel for m <= 1024")
    ap.add_argument("--svd-path", type=int, default=0, choices=[0, 1],
                    help="0 (default): Gram eigensolver where it resolves the kept spectrum, else Jacobi; "
                         "1: Jacobi only")
    ap.add_argument("--fp64-updates", type=int, default=6,
                    help="updates of the FP64 comparison on the first timed layer (0: skip)")
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle CPU time for cpu_baseline")
    ap.add_argument("--mpo-compress", type=int, default=1, choices=[0, 1],
                    help="1 (default): lossless compression of each layer MPO before the guess; "
                         "0: the bond is the product of the straddling gates' Schmidt ranks")
    ap.add_argument("--records", type=int, default=20000, help="learned: training records to log")
    ap.add_argument("--eval-layers", type=int, default=4, help="learned: layers of the random circuit to run")
    ap.add_argument("--workload", default="random", choices=["random", "qaoa", "batch", "learned", "grouping"],
                    help="qaoa: grid-graph QAOA (p = --layers), reports the sampled cut value; "
                         "batch: independent instances of uneven N, depth and chi on concurrent streams")
    ap.add_argument("--batch-count", type=int, default=32, help="batch: number of instances")
    ap.add_argument("--workers", default="auto",
                    help="batch: worker streams, or 'auto' to pick the best of 1, 2, 4, 8, 16 on a calibration subset")
    ap.add_argument("--batch-serial", type=int, default=1,
                    help="batch: 1 also runs the instances one at a time (twice) for the speedup and the "
                         "run-to-run spread; 0 runs the batched pass only")
    ap.add_argument("--layers", type=int, default=4, help="QAOA levels")
    ap.add_argument("--samples", type=int, default=10000)
    ap.add_argument("--chi-oracle", type=int, default=64)
    ap.add_argument("--fidelity-report", action="store_true",
                    help="report F_tilde of every precision on the 24-qubit version and the oracle")
    args = ap.parse_args(argv)
    if args.impl == "ours":
        from paper_2207_05612_gb300 import binding
        binding.dmrgc_set_jacobi_kernel(0 if args.jacobi == "wp4" else 1)
    if args.fidelity_report:
        return fidelity_report(args)
    if args.workload == "qaoa":
        return qaoa_report(args)
    if args.workload == "batch":
        return batch_report(args)
    if args.workload == "grouping":
        return grouping_report(args)
    if args.workload == "learned":
        return learned_report(args)
    world, rank, local = dist_setup()
    workload = f"random circuit {args.rows}x{args.cols} ({args.rows * args.cols}q), K=2 cycles/step, chi={args.chi}, 2 sweeps"
    config = {"workload": workload, "grid": f"{args.rows}x{args.cols}", "chi": args.chi,
              "cycles_per_step": 2, "sweeps_per_step": 2,
              "updates_per_step": 2 * (args.rows * args.cols - 1),
              "jacobi_kernel": args.jacobi, "svd_path": "gram eigensolver + jacobi fallback" if args.svd_path == 0
              else "jacobi",
              "mpo": "compressed (operator Schmidt ranks)" if args.mpo_compress else "product of gate Schmidt ranks",
              "l2": "inputs larger than L2 (environment caches of GBs), no flush"}

    if args.impl == "reference":
        if rank != 0:
            return 0
        from synthetic import circuits as sc
        circ = sc.random_circuit(args.rows, args.cols, max(20, 2 * (args.warmup + args.steps)), seed=args.seed)
        shapes = workload_shapes(args.rows, args.cols, args.chi, circ.layers[args.warmup],
                                 compress=bool(args.mpo_compress))
        for _ in range(args.warmup):   # untimed: one update at the cheapest stratum warms the BLAS threads
            oracle_updates(shapes, 0.0, seed=0, max_updates=1)
        tot, ups, threads = 0.0, 0, 1
        for _ in range(args.steps):
            done, dt, threads, _ = reference_step(shapes)
            tot += dt
            ups += done
        value = ups / tot
        sample = (f"per step four oracle two-site updates, one at the middle bond of each of four equal-frequency "
                  f"cost strata of the first timed layer's bonds, so that their mean is the layer's mean update "
                  f"(the workload's operand shapes: saturated MPS bonds <= {args.chi}, the layer's compressed MPO "
                  f"bonds; random values)")
        line = {"impl": "reference", "metric": "two-site updates/s", "value": value,
                "unit": "updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "c128-f64", "data": "synthetic", "config": config,
                "cpu_baseline": {"value": value, "unit": "updates/s", "cores": threads,
                                 "kind": "oracle", "sample": sample},
                "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    r = run_ours(args, world, rank, local)
    if rank != 0:
        return 0
    st = r["stats"]
    peaks, peak_src = measured_peaks()
    value = r["updates"] / r["dev_s"]
    e2e = r["updates"] / r["region_s"]
    fp64 = args.precision == "fp64"
    gemm_s, svd_s = st["gemm_ms"] / 1e3, st["svd_ms"] / 1e3
    clk = r["clocks"]
    gemm_ach = st["gemm_flops"] / max(gemm_s, 1e-12) / 1e12
    svd_ach = st["svd_flops"] / max(svd_s, 1e-12) / 1e12
    tensor = args.precision in ("bf16x3", "tf32x3")
    if tensor:
        ratio = 1.0 if args.precision == "bf16x3" else 0.5
        gpeak = peaks.get("bf16_tflops_sustained", 1700.0) * ratio / 3.0
        roof_gemm = {"bound": "tensor", "kernel": "tc_gemm_kernel (complex GEMM, tcgen05)",
                     "achieved": gemm_ach, "peak": gpeak, "unit": "TFLOP/s", "frac": gemm_ach / gpeak,
                     "traffic": None,
                     "peak_note": f"{peak_src} sustained bf16 TFLOP/s x {ratio} (dtype) / 3 split products, "
                                  "algorithmic complex flops (8 per complex MAC)"}
    else:
        gpeak = alu_peak_tflops(fp64, clk.get("sm_mhz"))
        roof_gemm = {"bound": "alu", "kernel": "gemm_kernel (complex GEMM, CUDA cores)", "achieved": gemm_ach,
                     "peak": gpeak, "unit": "TFLOP/s", "frac": gemm_ach / gpeak, "traffic": None,
                     "peak_note": "CUDA-core FMA peak at the sampled SM clock"}
    spk = alu_peak_tflops(fp64, clk.get("sm_mhz"))
    roof_svd = {"bound": "alu", "kernel": "truncated SVD (Gram eigensolver: he_tridiag, tri_*, he_backtrans; "
                                          "Jacobi where it falls back)",
                "achieved": svd_ach, "peak": spk, "unit": "TFLOP/s", "frac": svd_ach / spk, "traffic": None,
                "peak_note": "CUDA-core FMA peak: 152 SMs x 128 FP32 lanes x 2 x sampled SM clock"
                             if not fp64 else "nominal FP64 1.25 TFLOP/s x sampled/max SM clock",
                "work_note": "algorithmic flops: 16/3 n^3 + 8 n^2 k per Gram eigensolver SVD, "
                             "Jacobi 16 m per pair visited + 14 m per rotation",
                "traffic_note": "null: the class is several kernels per SVD; ncu of its largest, he_tridiag_kernel "
                                "at n = 1024, read 8.4 MB (the 8 MB Gram once) and wrote 31 KB "
                                "(profiles/eig_gram_1024x1024_tf32x3.md): latency-bound, not DRAM-bound"}
    if args.precision == "bf16x3":
        t = NCU_TRAFFIC["tc_gemm_bf16x3"]
        roof_gemm["traffic"] = t["bytes"]
        roof_gemm["traffic_note"] = f"ncu, one launch of {t['launch']} ({t['profile']})"
    roof = roof_gemm if st["gemm_ms"] >= st["svd_ms"] else roof_svd
    roof_other = roof_svd if roof is roof_gemm else roof_gemm
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        note("CPU baseline")
        shapes = workload_shapes(args.rows, args.cols, args.chi, r["first_layer"], compress=bool(args.mpo_compress))
        got = oracle_updates_bounded(shapes, args.cpu_budget, 6 * args.cpu_budget + 120, seed=0, whole_rounds=True)
        if got is None:
            cpu = {"value": None, "unit": "updates/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"no oracle update finished within {6 * args.cpu_budget + 120:.0f} s"}
            note("CPU baseline timed out")
        else:
            done, spent, threads, picked = got
            note(f"CPU baseline: {done} updates in {spent:.1f} s")
            cpu = {"value": done / spent, "unit": "updates/s", "cores": threads, "kind": "oracle",
                   "sample": f"{done} oracle two-site updates, whole rounds over the middle bonds of four "
                             f"equal-frequency cost strata of the timed layer's {len(shapes)} bonds, so that their "
                             f"mean is the layer's mean update (operand shapes of the workload: saturated "
                             f"MPS bonds <= {args.chi}, the layer's compressed MPO bonds; random values), "
                             f"{spent:.1f} s of CPU time, bonds {picked}"}
    line = {
        "metric": "two-site updates/s", "value": value, "unit": "updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * r["dev_s"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE_NAME[args.precision], "data": "synthetic", "config": config,
        "e2e": {"value": e2e, "unit": "updates/s", "h2d_bytes_per_step": r["h2d"],
                "d2h_bytes_per_step": r["d2h"]},
        "excluding_mpo_and_guess": {"value": r["updates"] / r["sweep_s"], "unit": "updates/s",
                                    "apply_layer_ms_per_step": 1e3 * (r["dev_s"] - r["sweep_s"]) / args.steps,
                                    "note": "the same updates over the sweeps' CUDA-event time alone: apply_layer "
                                            "(layer MPO build and compression, zip-up guess) left out"},
        "roofline": roof,
        "roofline_secondary": roof_other,
        "cpu_baseline": cpu,
        "vs_fp64": r["vs_fp64"],
        "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"),
                   "reasons": clk.get("reasons")},
        "gpu_launches": int(st["kernel_launches"] + r["readout"]["kernel_launches"]),
        "fidelity": {"log_F_tilde": r["log_ft"], "f_delta_last": r["f_delta"],
                     "eps_tilde": float(1 - np.exp(r["log_ft"] / max(1, r["n2g"]))),
                     "n_2q_gates": r["n2g"], "cycles": 2 * (args.warmup + args.steps),
                     "log_F_tilde_after_20_cycles": r["log_ft_20_cycles"]},
        "breakdown_ms": {"gemm": st["gemm_ms"], "svd": st["svd_ms"], "mpo": st["mpo_ms"],
                         "other": st["other_ms"],
                         "gemm_tflops": st["gemm_flops"] / max(gemm_s, 1e-12) / 1e12,
                         "svd_tflops": st["svd_flops"] / max(svd_s, 1e-12) / 1e12,
                         "eig_svds": st["eig_svds"], "eig_fallbacks": st["eig_fallbacks"],
                         "eig_skipped": st["eig_skipped"],
                         "jacobi_sweeps": st["jacobi_sweeps"],
                         "note": "device-timed part only (apply_layer + sweeps)"},
        "readout_ms": {"amplitudes_1024": r["readout"]["gemm_ms"] + r["readout"]["other_ms"],
                       "note": "per run, outside value, inside e2e"},
        "state": {"max_chi": r["max_chi"], "max_D": r["max_D"]},
    }
    print(json.dumps(line))
    return 0


def fidelity_report(args):
    """Config-2 error table: the 4x6 (24-qubit) version of the random circuit,
    10 steps, every precision of the library against its FP64 run, and at a
    bond dimension the CPU oracle finishes in minutes, against the oracle."""
    import math
    from paper_2207_05612_gb300 import Context
    from synthetic import circuits as sc
    rows, cols = 4, 6
    circ = sc.random_circuit(rows, cols, 20, seed=args.seed)
    out = {"report": "fidelity", "workload": "random circuit 4x6 (24q), 20 cycles, K=2, 2 sweeps",
           "note": "rel_err = |delta log F_tilde| = relative error of F_tilde; "
                   "fp64_gates_perturbed_1e-7 gives the spread of the method itself under a "
                   "rounding-sized change of its input"}
    for chi in (512, args.chi_oracle):
        res = {}
        for name in ("fp64", "fp32", "tf32x3", "bf16x3"):
            ctx = Context(rows, cols, chi, precision=PRECISIONS[name])
            t0 = time.perf_counter()
            for layer in circ.layers:
                ctx.apply_layer(layer)
                ctx.sweep(2)
            lf, _ = ctx.fidelity()
            res[name] = {"log_F_tilde": lf, "seconds": time.perf_counter() - t0}
            ctx.close()
        # the method's own sensitivity: FP64 on the circuit with every gate
        # perturbed by a unitary of size 1e-7 (about one complex64 rounding)
        pc = sc.perturb_circuit(circ, 1e-7, seed=args.seed + 1)
        ctx = Context(rows, cols, chi, precision=PRECISIONS["fp64"])
        t0 = time.perf_counter()
        for layer in pc.layers:
            ctx.apply_layer(layer)
            ctx.sweep(2)
        lf, _ = ctx.fidelity()
        ctx.close()
        res["fp64_gates_perturbed_1e-7"] = {"log_F_tilde": lf, "seconds": time.perf_counter() - t0}
        for name in res:
            res[name]["rel_err_vs_fp64"] = abs(res[name]["log_F_tilde"] - res["fp64"]["log_F_tilde"])
        if chi == args.chi_oracle:
            from oracle import dmrg as od
            from oracle import mpo as om
            order = om.snake_order(rows, cols)
            t0 = time.perf_counter()
            mps = od.product_state(rows * cols)
            lo = 0.0
            for layer in circ.layers:
                mps, r = od.compress_layer(mps, om.layer_mpo(layer, order, compress=False), chi)
                lo += math.log(r.f_delta)
            res["oracle"] = {"log_F_tilde": lo, "seconds": time.perf_counter() - t0}
            for name in ("fp64", "fp32", "tf32x3", "bf16x3"):
                res[name]["rel_err_vs_oracle"] = abs(res[name]["log_F_tilde"] - lo)
        out[f"chi={chi}"] = res
    print(json.dumps(out))
    return 0


GROUPINGS_4x7 = {   # Sec. V.C on the 4 x 7 grid (the paper's 28-qubit n_b = 4, n_c = 8 size): (kind, widths, K)
    "V(1^7)": ("V", [1] * 7, 2),          # one column (4 qubits) per tensor
    "V(2,1,1,1,2)": ("V", [2, 1, 1, 1, 2], 2),
    "H(1^4)": ("H", [1] * 4, 2),          # one row (7 qubits) per tensor
    "D(2^5)": ("D", [2] * 5, 1),          # pairs of anti-diagonals; K = 1 as in the paper for D
}


def grouping_report(args):
    """Error per gate of the random circuits on the 4 x 7 grid for the
    two-site variant and the single-site variant under several qubit
    groupings (Sec. V.C, Sec. V.D.2 "role of the qubit grouping"), Sequence I
    and Sequence II (Sec. V.A): eps = 1 - F~^(1 / N_2g) against chi at the
    final depth, and against depth at one chi.  BF16x3 (the error per gate
    needs no more than 1e-4 relative); single-site runs start every step
    from the seeded random guess and sweep n_s = 4 times, the two-site runs
    use the zip-up guess and 2 one-direction sweeps.  K = 2 cycles per step,
    except K = 1 for the diagonal grouping (its two-cycle layer operator has
    bond 4^7 at some cuts; the paper also runs D with K = 1)."""
    import math
    from paper_2207_05612_gb300 import Context
    from synthetic import circuits as sc
    rows, cols, cycles = 4, 7, 20
    chis = (8, 16, 32, 64)
    chi_depth = 32
    prec = PRECISIONS["bf16x3"]
    out = {"report": "grouping", "grid": f"{rows}x{cols}", "cycles": cycles, "precision": "bf16x3",
           "eps": "1 - F_tilde^(1/N_2g), N_2g the two-qubit gates applied so far", "curves": {}}
    t_all = time.perf_counter()
    for seq_name, order in (("I", sc.PATTERN_ORDER), ("II", sc.PATTERN_ORDER_II)):
        variants = {"two-site": None}
        variants.update(GROUPINGS_4x7)
        curves = {}
        for name, grp in variants.items():
            k_cyc = 2 if grp is None else grp[2]
            circ = sc.random_circuit(rows, cols, cycles, cycles_per_layer=k_cyc, seed=args.seed,
                                     pattern_order=order)
            n2g = [sum(1 for g in layer if g[1] >= 0) for layer in circ.layers]
            res = {"K": k_cyc, "eps_vs_chi": {}, "eps_vs_depth": None, "seconds": 0.0}
            for chi in chis:
                t0 = time.perf_counter()
                if grp is None:
                    ctx = Context(rows, cols, chi, precision=prec)
                    sweeps = 2
                else:
                    kind, widths, _ = grp
                    ctx = Context(rows, cols, chi, precision=prec, order=kind,
                                  groups=sc.grouping(rows, cols, kind, widths), seed=args.seed + 17, mpo_compress=1)
                    sweeps = 4
                lf_depth, total2 = [], 0
                for layer, ng in zip(circ.layers, n2g):
                    ctx.apply_layer(layer)
                    ctx.sweep(sweeps)
                    total2 += ng
                    lf, _ = ctx.fidelity()
                    lf_depth.append(1.0 - math.exp(lf / total2))
                ctx.close()
                res["eps_vs_chi"][chi] = lf_depth[-1]
                if chi == chi_depth:
                    res["eps_vs_depth"] = lf_depth
                res["seconds"] += time.perf_counter() - t0
            curves[name] = res
            note(f"grouping: sequence {seq_name} {name}: eps(chi) {res['eps_vs_chi']} ({res['seconds']:.0f} s)")
        out["curves"][f"sequence {seq_name}"] = curves
    out["seconds"] = time.perf_counter() - t_all
    print(json.dumps(out))
    return 0


def qaoa_report(args):
    """Config 3: QAOA MaxCut on the rows x cols grid graph, p levels, from
    |+>^N, chi = --chi, precision --precision (TF32x3 by default in the
    configuration); samples --samples bit strings and reports the mean cut."""
    import torch
    from paper_2207_05612_gb300 import Context
    from synthetic import circuits as sc
    circ, gam, bet, edges = sc.qaoa_circuit(args.rows, args.cols, args.layers, seed=args.seed)
    n = args.rows * args.cols
    ctx = Context(args.rows, args.cols, args.chi, precision=PRECISIONS[args.precision], timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for layer in circ.layers:
        ctx.apply_layer(layer)
        ctx.sweep(2)
    t1 = time.perf_counter()
    bits = ctx.sample(args.samples, seed=args.seed + 1)
    t2 = time.perf_counter()
    e = np.array(edges)
    cut = np.sum(bits[:, e[:, 0]] != bits[:, e[:, 1]], axis=1).astype(float)
    lf, fd = ctx.fidelity()
    st = ctx.stats()
    print(json.dumps({"report": "qaoa", "grid": f"{args.rows}x{args.cols}", "p": args.layers, "chi": args.chi,
                      "precision": args.precision, "edges": len(edges),
                      "updates_per_s": st["updates"] / max(t1 - t0, 1e-9), "sweep_seconds": t1 - t0,
                      "samples": args.samples, "sample_seconds": t2 - t1,
                      "cut_mean": float(cut.mean()), "cut_stderr": float(cut.std(ddof=1) / np.sqrt(len(cut))),
                      "log_F_tilde": lf, "eps_tilde": float(1 - np.exp(lf / max(1, len(edges) * args.layers))),
                      "gammas": [float(g) for g in gam], "betas": [float(b) for b in bet]}))
    return 0


def learned_report(args):
    """Learned truncated SVD.  (1) Log rank-model records with the full Jacobi
    SVD on small random and QAOA circuits (4x6, 6x9; chi 64-128) until
    --records; (2) train the model on the GPU; (3) run the same workloads with
    svd_mode 0 (Jacobi), 1 (sketch rank = bond dimension) and 2 (learned):
    QAOA 6x9 p=4 at chi=256 (the structured configuration) and the first
    --eval-layers layers of the 6x9 random circuit at --chi (1024 in the
    learned configuration), each against the Jacobi run."""
    import torch
    from paper_2207_05612_gb300 import Context, binding
    from synthetic import circuits as sc
    prec = PRECISIONS[args.precision]
    t0 = time.perf_counter()
    xs, ys, n, seed = [], [], 0, 0
    sources = {}
    while n < args.records and time.perf_counter() - t0 < 600:
        if seed % 3 == 2:
            circ, _, _, _ = sc.qaoa_circuit(6, 9, 4, seed=1000 + seed)
            chi, name = 64, "qaoa 6x9 chi=64"
        else:
            circ = sc.random_circuit(4, 6, 20, seed=1000 + seed)
            chi, name = (64 if seed % 3 == 0 else 128), "random 4x6 chi=64/128"
        ctx = Context(circ.rows, circ.cols, chi, precision=prec, log_rank_records=1)
        for layer in circ.layers:
            ctx.apply_layer(layer)
            ctx.sweep(2)
        x, y = ctx.rank_records()
        ctx.close()
        xs.append(x)
        ys.append(y)
        n += len(y)
        sources[name] = sources.get(name, 0) + len(y)
        seed += 1
    x = np.concatenate(xs)
    y = np.concatenate(ys)
    t_log = time.perf_counter() - t0
    t1 = time.perf_counter()
    params, loss = binding.dmrgc_mlp_train(x, y, epochs=40, batch=256, lr=2e-3, seed=args.seed)
    t_train = time.perf_counter() - t1

    def run(circ, chi, mode, layers):
        ctx = Context(circ.rows, circ.cols, chi, precision=prec, timing=True, svd_mode=mode,
                      mpo_compress=args.mpo_compress)
        if mode == 2:
            ctx.set_rank_model(params)
        torch.cuda.synchronize()
        ts = time.perf_counter()
        for layer in circ.layers[:layers]:
            ctx.apply_layer(layer)
            ctx.sweep(2)
        torch.cuda.synchronize()
        dt = time.perf_counter() - ts
        lf, _ = ctx.fidelity()
        st = ctx.stats()
        ctx.close()
        return {"updates_per_s": st["updates"] / dt, "seconds": dt, "log_F_tilde": lf,
                "svd_ms": st["svd_ms"], "gemm_ms": st["gemm_ms"], "jacobi_sweeps": st["jacobi_sweeps"],
                "sketches_accepted": st["rsvd_accepted"], "sketches_tried": st["rsvd_attempts"]}

    out = {"report": "learned", "precision": args.precision,
           "training": {"records": int(len(y)), "sources": sources, "log_seconds": t_log,
                        "train_seconds": t_train, "epochs": 40, "loss_first": float(loss[0]),
                        "loss_last": float(loss[-1]), "label": "log2 r, r = rank holding 1-1e-6 of the kept weight"}}
    qc, _, _, _ = sc.qaoa_circuit(6, 9, 4, seed=args.seed + 7)
    rc = sc.random_circuit(6, 9, 20, seed=args.seed)
    for name, circ, chi, layers in (("qaoa 6x9 p=4 chi=256", qc, 256, len(qc.layers)),
                                    (f"random 6x9 chi={args.chi} first {args.eval_layers} layers", rc, args.chi,
                                     args.eval_layers)):
        res = {}
        for mode, label in ((0, "jacobi"), (1, "sketch_rank_rule"), (2, "learned")):
            res[label] = run(circ, chi, mode, layers)
        for label in res:
            res[label]["speedup_vs_jacobi"] = res["jacobi"]["seconds"] / res[label]["seconds"]
            res[label]["abs_dlog_F_tilde_vs_jacobi"] = abs(res[label]["log_F_tilde"] - res["jacobi"]["log_F_tilde"])
        out[name] = res
    print(json.dumps(out))
    return 0


def batch_report(args):
    """Batched workload: --batch-count independent random-circuit instances,
    N uniform in {16, 20, 24, 30, 36, 42, 54} (near-rectangular grids), depth
    uniform in 8..20 cycles, chi uniform in {32, 64, 128, 256}, K = 2, two
    sweeps per step.  The worker count is tuned on a calibration subset; the
    whole batch then runs on the tuned count and on one worker (the instances
    one at a time), and the aggregate updates/s of both are reported."""
    from paper_2207_05612_gb300 import binding
    from synthetic import circuits as sc
    prec = PRECISIONS[args.precision]
    insts = sc.batch_instances(args.batch_count, seed=args.seed)
    opt = binding.dmrgc_default_options()
    opt.precision = prec
    opt.mpo_compress = args.mpo_compress

    def run(subset, workers):
        items, keep = binding.pack_batch([(b.rows, b.cols, b.chi, b.circuit.layers, 2) for b in subset])
        wall = binding.dmrgc_batch_run(items, len(subset), workers, opt)
        res = [items[i] for i in range(len(subset))]
        bad = [(i, r.status) for i, r in enumerate(res) if r.status != 0]
        if bad:
            raise RuntimeError(f"batch instances failed: {bad[:5]}")
        ups = sum(r.updates for r in res)
        return wall, ups, res

    run(insts[:2], 2)   # warm-up: module load, tensor-map encoder, kernel attributes
    tune = {}
    if args.workers == "auto":
        calib = insts[:min(len(insts), 12)]
        for w in (1, 2, 4, 8, 16):
            wall, ups, _ = run(calib, w)
            tune[w] = ups / wall
        workers = max(tune, key=tune.get)
    else:
        workers = int(args.workers)
    wall_b, ups_b, res_b = run(insts, workers)
    wall_s = ups_s = dlog = dlog_rep = None
    if args.batch_serial:
        wall_s, ups_s, res_s = run(insts, 1)
        dlog = max(abs(a.log_F_tilde - b.log_F_tilde) for a, b in zip(res_b, res_s))
        # run-to-run spread of the serial runs alone (0 when every reduction
        # order is fixed)
        _, _, res_s2 = run(insts, 1)
        dlog_rep = max(abs(a.log_F_tilde - b.log_F_tilde) for a, b in zip(res_s, res_s2))
    print(json.dumps({
        "report": "batch", "precision": args.precision, "instances": len(insts),
        "workload": "random circuits, N in {16,20,24,30,36,42,54}, 8-20 cycles, chi in {32,64,128,256}, "
                    "K=2, 2 sweeps per step",
        "mix": {"n": [b.rows * b.cols for b in insts], "cycles": [b.cycles for b in insts],
                "chi": [b.chi for b in insts]},
        "updates": ups_b,
        "workers": workers, "autotune_updates_per_s": {str(k): v for k, v in tune.items()},
        "batched_updates_per_s": ups_b / wall_b, "batched_seconds": wall_b,
        "serial_updates_per_s": ups_s / wall_s if wall_s else None, "serial_seconds": wall_s,
        "speedup": wall_s / wall_b if wall_s else None,
        "max_abs_dlog_F_tilde_batched_vs_serial": dlog,
        "max_abs_dlog_F_tilde_serial_vs_serial": dlog_rep,
        "log_F_tilde": [r.log_F_tilde for r in res_b]}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
