"""Throughput of the per-sweep SCO hot path on GB300.

One step = one MC step of the whole path at n_sw = 1: switch every dipolar pair (step (A)),
compact the survivors into the CSR graph, Kuhn-Wattenhofer colouring and colour classes,
and one colour-class Metropolis sweep (every site updated once).  Metric: spin updates/s
= N * steps / time.  Workload: L = 2304 (N = 5,308,416) open lattice, J = 0, D = 1,
T = 0.6 D, seed 0, spins uniform on the sphere (synthetic, like the paper's lattices).

Prints one JSON line.  Under torchrun every rank runs its own replica (seed + rank, no
collective on the data path; weak scaling); rank 0 reports the max time over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "spin updates/s (switch+colour+sweep) at L=2304; FP32-guarded vs FP64; % HBM"
UNIT = "spin updates/s"
FALLBACK_HBM_GBS = 6800.0
# switching candidates per site (half plane) for independent uniform spins, from the closed
# form of the survival statistics (planning values of the work per site)
CANDIDATES_PER_SITE = {0.2: 30.5, 0.3: 23.1, 0.4: 19.0, 0.5: 16.3, 0.6: 14.4, 0.8: 11.8,
                       1.2: 9.0, 1.5: 7.7}
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--L", type=int, default=2304)
    ap.add_argument("--T", type=float, default=0.6)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32-guarded arm")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline")
    ap.add_argument("--cpu-L", type=int, default=2304, help="lattice of the oracle sample")
    ap.add_argument("--ref-L", type=int, default=384, help="lattice of one reference-arm step")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-replicas arm")
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--seq-steps", type=int, default=2,
                    help="steps per replica of the sequential single-lattice comparison")
    ap.add_argument("--batch-sizes", default="64,128,256,512",
                    help="lattice sizes of the batched arm (16 temperatures each by default)")
    ap.add_argument("--batch-temps", type=int, default=16)
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched arm: keep the default launch tuning")
    ap.add_argument("--only-batch", action="store_true",
                    help="run only the batched arm and print its object (profiling)")
    ap.add_argument("--long-steps", type=int, default=500,
                    help="MC steps of the long L=2304 FP64 run (all-step and last-half rates); "
                         "0 skips it")
    ap.add_argument("--prec-steps", type=int, default=1000,
                    help="MC steps per run of the L=1024 FP32-guarded vs FP64 comparison at "
                         "T = 0.4 D and 0.8 D; 0 skips it")
    ap.add_argument("--prec-L", type=int, default=1024)
    ap.add_argument("--nsw100-steps", type=int, default=100,
                    help="MC steps of the FP64 run with switch + colour every 100 steps (the "
                         "paper's n_sw, Eq. (8)'s t_ave); 0 skips it")
    ap.add_argument("--no-kw-bound", action="store_true",
                    help="skip t_R of both colour-reduction variants against Eq. (5)'s bound")
    ap.add_argument("--protocol", action="store_true",
                    help="run the paper's cooling protocol instead (Table 1 at L=2304, M_phi(T) "
                         "at L=128) and print its JSON line")
    ap.add_argument("--proto-L", type=int, default=2304)
    ap.add_argument("--proto-eq", type=int, default=1000,
                    help="MC steps at every temperature of the L=2304 cooling")
    ap.add_argument("--proto-graphs", type=int, default=35,
                    help="graphs (epochs of n_sw steps) averaged at each Table 1 temperature")
    ap.add_argument("--mphi-L", type=int, default=128)
    ap.add_argument("--mphi-runs", type=int, default=10)
    ap.add_argument("--mphi-eq", type=int, default=2000)
    ap.add_argument("--mphi-meas", type=int, default=2000)
    return ap.parse_args()


def rank_seed(seed, rank):
    """Seed of rank r's lattice: every rank runs an independent replica (no collective on
    the data path)."""
    return seed + rank


def batch_seed_offset(rank):
    """Added to every replica seed of the batched arm on rank r."""
    return 1000 * rank


def max_over_ranks(x, world, device=None):
    """Max of a per-rank time over all ranks (the job's time); identity at world size 1."""
    if world == 1:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(sites_per_rank, steps, world, ms):
    """Spin updates per second of the whole job: every rank's sites, over the max time."""
    return sites_per_rank * steps * world / (ms / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if r[3 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


FP64_NOMINAL_GFLOPS = 1250.0  # GB300 FP64 (vector and tensor), nominal: context only
# FP64 sweep kernels, per pair of the switched graph and per spin update, from one ncu capture
# of the current kernels on a smaller lattice at T = 0.6 D (DRAM bytes and executed FP64
# thread-instructions scale with the updates and pairs, not with L): see the named profile
SWEEP64_EXECUTED_FP64_PER_PAIR = 28.0  # k_propose + k_sweep + k_resolve, thread-instructions
SWEEP64_DRAM_BYTES_PER_UPDATE = 2352.0  # dram__bytes_read.sum + dram__bytes_write.sum
SWEEP64_TRAFFIC_T = 0.6
SWEEP64_EXECUTED_SOURCE = "profiles/k_sweep_fp64_L1024_T0.6.md"


def fp64_peak(local):
    """Measured FP64 throughput of this GPU (sco_probe_fp64: independent FMA chains filling
    every SM), with the SM clock sampled while it ran."""
    import paper_1503_03295_gb300 as sco

    with ClockSampler(local) as clk:
        r = sco.probe_fp64(8192)
    r["gflops"] = r["flops"] / 1e9
    r["clocks"] = clk.summary()
    return r


def low_levels(g, M):
    """KW levels taken block-locally (groups of g 2^p <= 4096 vertices, palettes <= 64)."""
    p = 0
    if g <= 64:
        while p < M and (g << (p + 1)) <= 4096:
            p += 1
    return p


def algorithmic_bytes(k, M, p0, cache=False):
    """Bytes per spin update that each phase must move at least once, k the mean degree, M the
    KW levels and p0 the block-local ones: switch + CSR 40 + 16k; colouring + classes: the
    first p0 levels read the rows once and write the colours (4 + 4k + 9), every later level
    half the rows and colours (4 + 2k), classes 12; sweep 60 + 8k.  With the FP64 form's pair
    cache (cache=True) the switch also writes a 16-byte record per kept pair and the fill a
    4-byte id per CSR entry (+12k), and the sweep reads per pair endpoint the id and one
    16-byte record half and writes 16 bytes for one of the two endpoints (+28k)."""
    colour = (4 + 4 * k + 9 if p0 else 0) + (M - p0) * (4 + 2 * k) + 12
    if cache:
        return {"switch": 40 + 28 * k, "colour": colour, "sweep": 60 + 36 * k}
    return {"switch": 40 + 16 * k, "colour": colour, "sweep": 60 + 8 * k}


def algorithmic_flops(k, cand):
    """FP64 operations per spin update of the FP64 form, planning figures: 51 per switching
    candidate (the pair energy 30, one expm1 20, and one multiply for the candidate search on
    the table of decay values, which takes the place of a logarithm) and, per pair endpoint of
    the sweep, two pair energies (20) and the pseudointeraction term of the proposed spin (50, a
    log1mexp counted as two transcendentals): the old spin's term is read from the pair cache,
    which the switch filled, so 70 (120 without the cache); the colouring has none.  The kernels
    issue fewer (about 23 per candidate, 28.0 per pair endpoint: see
    SWEEP64_EXECUTED_FP64_PER_PAIR), so these fractions measure work done against the plan."""
    return {"switch": 51.0 * cand, "colour": 0.0, "sweep": 70.0 * k}


def phase_ms(ph):
    return {"switch": ph["switch_ms"] / max(ph["switch_calls"], 1),
            "colour": ph["colour_ms"] / max(ph["colour_calls"], 1),
            "sweep": ph["sweep_ms"] / max(ph["sweep_calls"], 1)}


def rooflines(per_step, N, k, M, p0, cand, hbm, how, fp64_gflops=None):
    """HBM roofline of every phase and, for the FP64 form (fp64_gflops: the measured FP64
    peak; its bytes include the pair cache), the FP64-ALU roofline against the planning
    operation counts."""
    ab = algorithmic_bytes(k, M, p0, cache=bool(fp64_gflops))
    af = algorithmic_flops(k, cand)
    out = {}
    for ph, ms in per_step.items():
        gbs = ab[ph] * N / (ms / 1e3) / 1e9
        r = {"hbm_achieved_GBs": gbs, "hbm_frac": gbs / hbm, "algorithmic_bytes_per_update": ab[ph]}
        if fp64_gflops and af[ph] > 0:
            gf = af[ph] * N / (ms / 1e3) / 1e9
            r.update({"fp64_achieved_GFLOPs": gf, "fp64_frac": gf / fp64_gflops,
                      "algorithmic_fp64_ops_per_update": af[ph]})
        out[ph] = r
    return out


def run_ours(args, rank, world, local):
    import torch
    import paper_1503_03295_gb300 as sco

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    sh = stream.cuda_stream
    L = args.L
    N = L * L

    def lattice(prec):
        return sco.Lattice(sco.make_params(L, T=args.T, seed=rank_seed(args.seed, rank),
                                           precision=prec), stream=sh)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(lat, K, W, timing=False):
        lat.sweep(W)
        lat.sync()
        barrier()
        l0 = lat.observables()["kernel_launches"]
        if timing:
            lat.set_timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(stream):
            e0.record(stream)
            lat.sweep(K)
            e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        ms = e0.elapsed_time(e1)
        ph = lat.timing() if timing else None
        if timing:
            lat.set_timing(False)
        launches = lat.observables()["kernel_launches"] - l0
        return ms, ph, launches

    out = {"fp64_peak": fp64_peak(local)}
    lat = lattice(sco.FP64)
    with ClockSampler(local) as clk:
        ms, ph, launches = timed(lat, args.steps, args.warmup, timing=True)
    ms = max_over_ranks(ms, world, dev)
    obs = lat.observables()
    out["fp64"] = dict(ms=ms, phases=ph, launches=launches, obs=obs, clocks=clk.summary())
    if not args.no_e2e:
        # end to end through the public API with host buffers: every step copies the spins
        # in from pinned host memory and the spins out to pinned host memory
        hin = torch.empty(3 * N, dtype=torch.float64, pin_memory=True)
        hout = torch.empty(3 * N, dtype=torch.float64, pin_memory=True)
        import ctypes as C
        Lb = sco.load()
        st = Lb.sco_get_spins(lat.handle, C.c_void_p(hin.data_ptr()), 0)
        assert st == 0
        K = max(1, args.steps // 2)
        torch.cuda.synchronize(dev)
        barrier()
        t0 = time.perf_counter()
        for _ in range(K):
            assert Lb.sco_set_spins(lat.handle, C.c_void_p(hin.data_ptr()), 0) == 0
            lat.sweep(1)
            assert Lb.sco_get_spins(lat.handle, C.c_void_p(hout.data_ptr()), 0) == 0
            hin, hout = hout, hin
        torch.cuda.synchronize(dev)
        t_e2e = max_over_ranks(time.perf_counter() - t0, world, dev)
        out["e2e"] = dict(value=N * K * world / t_e2e, unit=UNIT, h2d_bytes_per_step=3 * N * 8,
                          d2h_bytes_per_step=3 * N * 8, steps=K)
    if rank == 0:
        out["graph_stats"] = graph_stats_report(lat)
    lat.close()
    del lat
    if not args.no_fp32:
        lat32 = lattice(sco.FP32_GUARDED)
        ms32, ph32, l32 = timed(lat32, args.steps, args.warmup, timing=True)
        ms32 = max_over_ranks(ms32, world, dev)
        out["fp32"] = dict(ms=ms32, phases=ph32, launches=l32, obs=lat32.observables())
        lat32.close()
        del lat32
    if args.long_steps > 0:
        out["long"] = run_long(args, rank, world, dev, stream)
    if args.nsw100_steps > 0:
        out["n_sw_100"] = run_nsw100(args, rank, world, dev, stream)
    if args.prec_steps > 0:
        out["precision"] = run_precision(args, rank, world, dev, stream)
    if not args.no_kw_bound:
        out["kw_bound"] = [kw_bound(L, args.T, rank_seed(args.seed, rank), stream)
                           for L in sorted({256, args.L})]
    if not args.no_batch:
        out["batch"] = run_batch(args, rank, local)
    return out


def _timed_steps(lat, K, dev, stream):
    """Device time (ms) of K MC steps of a lattice, CUDA events on its stream."""
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        e0.record(stream)
        lat.sweep(K)
        e1.record(stream)
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1)


def graph_stats_report(lat, n_rbins=32):
    """Diagnostics of the lattice's current graph: P_survive per distance shell (Fig. 5), P_IPC
    and the mean colour-count imbalance Delta R (Eq. (9)) of the Fig. 6 processor counts."""
    out = {"p_ipc": {}, "delta_r_mean": {}, "delta_r_max": {}, "delta_r_weighted": {}}
    for nproc, (cx, cy) in CELL_SPLITS.items():
        if cx > lat.params.Lx or cy > lat.params.Ly:
            continue
        st = lat.graph_stats(cx, cy, n_rbins)
        out["p_ipc"][str(nproc)] = st["p_ipc"]
        out["delta_r_mean"][str(nproc)] = st["delta_r_mean"]
        out["delta_r_max"][str(nproc)] = st["delta_r_max"]
        out["delta_r_weighted"][str(nproc)] = st["delta_r_weighted"]
    out["p_survive_r1_to_r%d" % n_rbins] = [float(x) for x in st["p_survive"]]
    out["cell_splits"] = {str(k): v for k, v in CELL_SPLITS.items()}
    return out


def run_long(args, rank, world, dev, stream):
    """The long FP64 run at the benchmark lattice from the random start: rate over all steps
    and over the second half (spins order as the run goes on, so the graph's mean degree
    grows), with the mean degree at the end."""
    import paper_1503_03295_gb300 as sco

    K = args.long_steps
    lat = sco.Lattice(sco.make_params(args.L, T=args.T, seed=rank_seed(args.seed, rank)),
                      stream=stream.cuda_stream)
    k0 = None
    lat.sweep(1)
    k0 = 2.0 * lat.observables()["n_edges"] / lat.N
    first = K // 2
    ms_a = max_over_ranks(_timed_steps(lat, first - 1, dev, stream), world, dev)
    ms_b = max_over_ranks(_timed_steps(lat, K - first, dev, stream), world, dev)
    o = lat.observables()
    lat.close()
    N = args.L * args.L
    # the first step (untimed, before the events) is counted at the first half's rate
    ms_all = (ms_a + ms_b) * K / (K - 1)
    return {"steps": K, "precision": "fp64",
            "value_all_steps": whole_job_rate(N, K, world, ms_all),
            "value_last_half": whole_job_rate(N, K - first, world, ms_b),
            "ms_per_step_all": ms_all / K, "ms_per_step_last_half": ms_b / (K - first),
            "mean_degree_first_step": k0, "mean_degree_end": 2.0 * o["n_edges"] / N,
            "max_degree_end": o["max_degree"], "n_colours_end": o["n_colours"],
            "e_switched_per_spin_end": o["e_switched"] / N,
            "workload": "L=%d, J=0, D=1, T=%gD, seed %d, n_sw=1, FP64, %d MC steps from the "
                        "random start" % (args.L, args.T, args.seed, K)}


def run_nsw100(args, rank, world, dev, stream):
    """The paper's schedule on the benchmark lattice: switch and colour every n_sw = 100 MC
    steps (Sec. 3.1), FP64.  Eq. (8)'s t_ave = t_switch / 100 + t_color / 100 + t_MC, from the
    phase times of K steps (K / 100 switches); the graph of each epoch carries the pair cache
    from one step to the next."""
    import paper_1503_03295_gb300 as sco

    K = args.nsw100_steps
    lat = sco.Lattice(sco.make_params(args.L, T=args.T, seed=rank_seed(args.seed, rank),
                                      n_sw=100), stream=stream.cuda_stream)
    lat.sweep(100)  # one whole epoch untimed (warm-up)
    lat.sync()
    lat.set_timing(True)
    ms = max_over_ranks(_timed_steps(lat, K, dev, stream), world, dev)
    ph = lat.timing()
    lat.set_timing(False)
    lat.close()
    N = args.L * args.L
    t_sw = ph["switch_ms"] / max(ph["switch_calls"], 1)
    t_col = ph["colour_ms"] / max(ph["colour_calls"], 1)
    t_mc = ph["sweep_ms"] / max(ph["sweep_calls"], 1)
    return {"steps": K, "n_sw": 100, "precision": "fp64",
            "value": whole_job_rate(N, K, world, ms), "ms_per_step": ms / K,
            "t_switch_ms": t_sw, "t_color_ms": t_col, "t_mc_ms": t_mc,
            "t_ave_ms": t_sw / 100 + t_col / 100 + t_mc,
            "switches": ph["switch_calls"],
            "workload": "L=%d, J=0, D=1, T=%gD, seed %d, n_sw=100, FP64, %d MC steps after one "
                        "epoch" % (args.L, args.T, args.seed, K)}


def run_precision(args, rank, world, dev, stream):
    """The precision workload: FP32-guarded against FP64 on the same seeds at T = 0.4 D and
    0.8 D, each run the same number of MC steps; the two forms take identical decisions, so
    their spins must end bit-identical (energy then equal to summation order)."""
    import numpy as np
    import paper_1503_03295_gb300 as sco

    L, K = args.prec_L, args.prec_steps
    N = L * L
    res = {"L": L, "steps": K, "runs": []}
    for T in (0.4, 0.8):
        row = {"T": T}
        spins = {}
        for name, prec in (("fp64", sco.FP64), ("fp32_guarded", sco.FP32_GUARDED)):
            lat = sco.Lattice(sco.make_params(L, T=T, seed=1 + rank, precision=prec),
                              stream=stream.cuda_stream)
            lat.sweep(1)
            ms = max_over_ranks(_timed_steps(lat, K - 1, dev, stream), world, dev)
            o = lat.observables()
            spins[name] = lat.spins()
            lat.close()
            row[name] = {"value": whole_job_rate(N, K - 1, world, ms),
                         "ms_per_step": ms / (K - 1), "e_switched": o["e_switched"],
                         "guard_hits_fp32": o["guard_hits_fp32"],
                         "guard_hits_fp64": o["guard_hits_fp64"],
                         "mean_degree_end": 2.0 * o["n_edges"] / N}
        row["identical_spins"] = bool(np.array_equal(spins["fp64"], spins["fp32_guarded"]))
        e64, e32 = row["fp64"]["e_switched"], row["fp32_guarded"]["e_switched"]
        row["energy_rel_diff"] = abs(e32 - e64) / max(abs(e64), 1e-300)
        row["speedup_fp32_guarded"] = row["fp32_guarded"]["value"] / row["fp64"]["value"]
        res["runs"].append(row)
    res["workload"] = ("L=%d, J=0, D=1, T in {0.4, 0.8} D, seed 1, n_sw=1, %d MC steps per "
                       "form from the random start (the first untimed)" % (L, K))
    return res


def kw_bound(L, T, seed, stream):
    """t_R of the colouring for both colour reductions on the same switched graph (the first
    graph of the run), against Eq. (5)'s (Delta + 1) log2(N / (Delta + 1)) and the level
    count M = ceil(log2 ceil(N / (Delta + 1)))."""
    import math
    import paper_1503_03295_gb300 as sco

    out = {"L": L, "T": T}
    for variant, name in ((0, "modified_bcr"), (1, "plain_bcr")):
        lat = sco.Lattice(sco.make_params(L, T=T, seed=seed, colour_variant=variant),
                          stream=stream.cuda_stream)
        lat.colour()
        o = lat.observables()
        lat.close()
        g = o["max_degree"] + 1
        N = L * L
        G = -(-N // g)
        M = 0
        while (1 << M) < G:
            M += 1
        out[name] = {"t_R": o["kw_rounds"], "n_colours": o["n_colours"]}
        out.update({"max_degree": o["max_degree"], "levels_M": M, "g_times_M": g * M,
                    "eq5_bound": g * math.log2(N / g) if N > g else 0.0})
    out["plain_over_modified"] = out["plain_bcr"]["t_R"] / max(out["modified_bcr"]["t_R"], 1)
    return out


def run_batch(args, rank, local):
    """64 replicas (L in {64, 128, 256, 512} x 16 temperatures in [0.2, 1.5] D, seed r,
    FP32-guarded) advanced together, against the same replicas run one after another as
    single lattices."""
    import torch
    import paper_1503_03295_gb300 as sco

    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    sizes = tuple(int(x) for x in args.batch_sizes.split(","))
    ps = sco.replica_params(L_list=sizes, n_T=args.batch_temps, precision=sco.FP32_GUARDED)
    for p in ps:
        p.seed += batch_seed_offset(rank)
    ntot = sum(p.Lx * p.Ly for p in ps)
    b = sco.Batch(ps, stream=stream.cuda_stream)
    tuning = b.tuning() if args.no_autotune else b.autotune(trial_steps=2)
    b.run(args.warmup)
    i0 = b.info()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        e0.record(stream)
        b.run(args.batch_steps)
        e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    i1 = b.info()
    picks = sorted({0, args.batch_temps - 1, len(ps) - args.batch_temps, len(ps) - 1})
    obs = [b.observables(r) for r in picks]
    b.close()
    del b
    # the same replicas as single lattices, one after another
    seq_ms = 0.0
    seq_launches = 0
    for p in ps:
        lat = sco.Lattice(p, stream=stream.cuda_stream)
        lat.sweep(1)
        lat.sync()
        l0 = lat.observables()["kernel_launches"]
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(stream):
            e0.record(stream)
            lat.sweep(args.seq_steps)
            e1.record(stream)
        torch.cuda.synchronize(dev)
        seq_ms += e0.elapsed_time(e1)
        seq_launches += lat.observables()["kernel_launches"] - l0
        lat.close()
    value = ntot * args.batch_steps / (ms / 1e3)
    seq_value = ntot * args.seq_steps / (seq_ms / 1e3)
    return {
        "value": value, "unit": UNIT, "ms_per_step": ms / args.batch_steps,
        "steps": args.batch_steps, "replicas": len(ps), "sites": ntot, "precision": "fp32_guarded",
        "workload": "%d replicas: L in {%s} x %d, T = (0.2 + b 1.3/%d) D, seed r, J=0, D=1, "
                    "n_sw=1" % (len(ps), args.batch_sizes, args.batch_temps,
                                max(args.batch_temps - 1, 1)),
        "tuning": tuning, "gpu_launches": i1["launches"] - i0["launches"],
        "graph_launches": i1["graph_launches"] - i0["graph_launches"], "replans": i1["replans"],
        "sample_max_degree": {str(r): o["max_degree"] for r, o in zip(picks, obs)},
        "sequential": {"value": seq_value, "ms_per_step_all_replicas": seq_ms / args.seq_steps,
                       "steps": args.seq_steps, "gpu_launches": seq_launches},
        "speedup_vs_sequential": value / seq_value,
    }


# Table 1 of the paper: T / J, <k>, <Delta> at L = 2304 over 35 graphs
TABLE1 = {1.25: (1.40, 8.54), 0.45: (3.36, 12.9), 0.05: (22.7, 41.6)}
# virtual cell splits of the L = 2304 lattice for the processor counts of Fig. 6: the factor
# pair of N_proc closest to square (the paper's cells are squares where N_proc allows)
CELL_SPLITS = {48: (6, 8), 144: (12, 12), 288: (16, 18)}


def cooling_schedule(T_hi=1.25, T_lo=0.05, dT=0.05):
    """Temperatures of Sec. 3.1's cooling, T_hi down to T_lo in steps of dT (in units of J)."""
    n = int(round((T_hi - T_lo) / dT))
    return [round(T_hi - k * dT, 10) for k in range(n + 1)]


def _mean_sem(x):
    import numpy as np

    x = np.asarray(x, float)
    return float(x.mean()), float(x.std(ddof=1) / np.sqrt(len(x))) if len(x) > 1 else 0.0


def run_protocol(args, local):
    """Sec. 3.1's protocol on the paper's model (J = 1, D = 0.1, n_sw = 100): cooling from 1.25 J
    to 0.05 J in steps of 0.05 J with the spins carried over.  (1) L = 2304 (FP32-guarded, whose
    decisions equal the FP64 form's): at the three temperatures of Table 1, <k> and <Delta> over
    35 graphs, and the graph diagnostics of Figs. 5, 6 and Eq. (9); (2) L = 128, several
    independent runs advanced together as a batch: |M_phi| of Eq. (7) against T."""
    import numpy as np
    import torch
    import paper_1503_03295_gb300 as sco

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    n_sw = 100
    sched = cooling_schedule()
    t0 = time.perf_counter()
    L = args.proto_L
    N = L * L
    lat = sco.Lattice(sco.make_params(L, T=sched[0], J=1.0, D=0.1, seed=args.seed, n_sw=n_sw,
                                      precision=sco.FP32_GUARDED), stream=stream.cuda_stream)
    rows = []
    ms_mc = []
    for T in sched:
        lat.set_temperature(T)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            lat.sweep(args.proto_eq)
            e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_mc.append(e0.elapsed_time(e1) / args.proto_eq)
        key = min(TABLE1, key=lambda a: abs(a - T))
        if abs(key - T) > 1e-9:
            continue
        ks, ds, dr, drw, pipc, ps = [], [], [], [], {n: [] for n in CELL_SPLITS}, []
        for _ in range(args.proto_graphs):
            lat.sweep(n_sw)  # the epoch's graph is switched at its first step
            o = lat.observables()
            ks.append(2.0 * o["n_edges"] / N)
            ds.append(o["max_degree_dipolar"])
            for nproc, (cx, cy) in CELL_SPLITS.items():
                st = lat.graph_stats(cx, cy, 64)
                pipc[nproc].append(st["p_ipc"])
                if nproc == 288:
                    dr.append(st["delta_r_mean"])
                    drw.append(st["delta_r_weighted"])
                    ps.append(st["p_survive"])
        o = lat.observables()
        k_m, k_s = _mean_sem(ks)
        d_m, d_s = _mean_sem(ds)
        pmean = np.mean(np.asarray(ps), axis=0)
        rows.append({"T_J": T, "k_mean": k_m, "k_sem": k_s, "delta_mean": d_m, "delta_sem": d_s,
                     "graphs": len(ks), "paper_k": TABLE1[key][0], "paper_delta": TABLE1[key][1],
                     "m_phi": o["m_phi"], "m_abs": o["m_abs"],
                     "e_switched_per_spin": o["e_switched"] / N,
                     "p_survive_r1_to_r16": [float(x) for x in pmean[:16]],
                     "p_ipc": {str(n): _mean_sem(v)[0] for n, v in pipc.items()},
                     "delta_r_mean_288_cells": _mean_sem(dr)[0],
                     "delta_r_weighted_288_cells": _mean_sem(drw)[0]})
    lat.close()
    t1 = time.perf_counter()
    # (2) M_phi(T): independent runs (seeds 0..R-1) as one batch
    R = args.mphi_runs
    ps_ = [sco.make_params(args.mphi_L, T=sched[0], J=1.0, D=0.1, seed=s, n_sw=n_sw,
                           precision=sco.FP32_GUARDED) for s in range(R)]
    b = sco.Batch(ps_, stream=stream.cuda_stream)
    curve = []
    every = 10
    for T in sched:
        for r in range(R):
            b.set_temperature(r, T)
        b.run(args.mphi_eq)
        acc = np.zeros(R)
        nm = 0
        for _ in range(args.mphi_meas // every):
            b.run(every)
            acc += [abs(b.observables(r)["m_phi"]) for r in range(R)]
            nm += 1
        m, sem = _mean_sem(acc / nm)
        curve.append({"T_J": T, "m_phi_abs": m, "sem": sem})
    b.close()
    t2 = time.perf_counter()
    return {
        "protocol": "Sec. 3.1: J=1, D=0.1, n_sw=100, cooling 1.25J -> 0.05J in 0.05J steps",
        "table1": {"L": L, "precision": "fp32_guarded", "steps_per_T": args.proto_eq,
                   "graphs_per_T": args.proto_graphs, "rows": rows,
                   "ms_per_mc_step_by_T": dict(zip([str(t) for t in sched], ms_mc)),
                   "cell_splits": {str(k): v for k, v in CELL_SPLITS.items()},
                   "wall_s": t1 - t0},
        "m_phi": {"L": args.mphi_L, "runs": R, "eq_steps": args.mphi_eq,
                  "meas_steps": args.mphi_meas, "every": every, "curve": curve,
                  "wall_s": t2 - t1},
    }


def cpu_baseline(L, T, seed):
    import oracle as O

    ncores = os.cpu_count() or 1
    O.set_threads(ncores)
    ch = O.Chain(O.make_params(L, T=T, seed=seed))
    t0 = time.perf_counter()
    ch.sweep(1)
    dt = time.perf_counter() - t0
    return {"value": L * L / dt, "unit": UNIT, "cores": ncores, "kind": "oracle",
            "sample": "1 MC step (switch+colour+sweep, n_sw=1) of the L=%d lattice at T=%gD "
                      "from the seed-%d start, %d OpenMP threads, %.1f s" % (L, T, seed, ncores, dt)}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    if args.protocol:
        if rank == 0:
            print(json.dumps(run_protocol(args, local)), flush=True)
        return
    if args.only_batch:
        import torch
        torch.cuda.set_device(local)
        b = run_batch(args, rank, local)
        if rank == 0:
            print(json.dumps({"batched": b}), flush=True)
        return
    res = run_ours(args, rank, world, local)
    if rank != 0:
        return
    N = args.L * args.L
    K = args.steps
    f64 = res["fp64"]
    value = whole_job_rate(N, K, world, f64["ms"])
    obs = f64["obs"]
    k = 2.0 * obs["n_edges"] / N
    levels = 0
    g = obs["max_degree"] + 1
    G = -(-N // g)
    while (1 << levels) < G:
        levels += 1
    cand = CANDIDATES_PER_SITE.get(round(args.T, 3), 14.4)
    hbm, how = peaks()
    fpk = res["fp64_peak"]
    per_step = phase_ms(f64["phases"])
    p0 = low_levels(g, levels)
    roof = rooflines(per_step, N, k, levels, p0, cand, hbm, how, fpk["gflops"])
    # the dominant kernel: k_sweep of the sweep phase is the longest kernel of the step in the
    # ncu launch list; the colour phase, about as long in all, is spread over the block-local
    # kernel and three launches per grid-wide level
    dom = "sweep" if "sweep" in per_step else max(per_step, key=per_step.get)
    if roof[dom].get("fp64_achieved_GFLOPs"):
        primary = {"bound": "alu", "kernel": dom, "achieved": roof[dom]["fp64_achieved_GFLOPs"],
                   "peak": fpk["gflops"], "unit": "GFLOP/s",
                   "frac": roof[dom]["fp64_frac"], "traffic": None,
                   "peak_source": "measured in this run: sco_probe_fp64, independent FP64 FMA "
                                  "chains filling every SM (2 flops per FMA), SM clock %s MHz" % (
                                      fpk["clocks"]["sm_mhz"],),
                   "algorithmic_fp64_ops_per_update": roof[dom]["algorithmic_fp64_ops_per_update"]}
        if dom == "sweep" and SWEEP64_EXECUTED_FP64_PER_PAIR:
            # the same phase against the FP64 instructions its kernels execute (ncu count of a
            # class launch per pair of the switched graph), at the measured FMA issue rate
            ex = SWEEP64_EXECUTED_FP64_PER_PAIR * k
            rate = ex * N / (per_step["sweep"] / 1e3)
            primary["executed"] = {
                "fp64_lane_inst_per_update": ex, "achieved_inst_per_s": rate,
                "peak_inst_per_s": fpk["dfma_per_s"], "frac": rate / fpk["dfma_per_s"],
                "source": SWEEP64_EXECUTED_SOURCE}
            if abs(args.T - SWEEP64_TRAFFIC_T) < 1e-9 and SWEEP64_DRAM_BYTES_PER_UPDATE:
                primary["traffic"] = SWEEP64_DRAM_BYTES_PER_UPDATE * N
                primary["traffic_unit"] = ("DRAM bytes per step of the sweep phase: ncu bytes "
                                           "per spin update of the same kernels on a smaller "
                                           "lattice at this T, times N")
                primary["traffic_source"] = SWEEP64_EXECUTED_SOURCE
    else:
        primary = {"bound": "hbm", "kernel": dom, "achieved": roof[dom]["hbm_achieved_GBs"],
                   "peak": hbm, "unit": "GB/s", "frac": roof[dom]["hbm_frac"], "traffic": None,
                   "peak_source": how,
                   "algorithmic_bytes_per_update": roof[dom]["algorithmic_bytes_per_update"]}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": f64["ms"] / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "L=%d open lattice, J=0, D=1, T=%gD, seed %d, n_sw=1, FP64" % (
            args.L, args.T, args.seed), "L": args.L, "N": N, "T": args.T,
            "precision": "fp64", "parallelism": "replicas" if world > 1 else "single",
            "l2": "working set > L2 (spins %.0f MB + CSR %.0f MB + tables)" % (
                3 * N * 8 / 1e6, 2 * obs["n_edges"] * 4 / 1e6)},
        "gpu_launches": f64["launches"],
        "clocks": f64["clocks"],
        "phases_ms_per_step": per_step,
        "graph": {"mean_degree": k, "max_degree": obs["max_degree"],
                  "n_colours": obs["n_colours"], "kw_rounds": obs["kw_rounds"],
                  "kw_levels": levels, "kw_block_local_levels": p0},
        "roofline": primary,
        "roofline_phases": roof,
    }
    if "e2e" in res:
        line["e2e"] = res["e2e"]
    if "fp32" in res:
        f32 = res["fp32"]
        p32 = phase_ms(f32["phases"])
        line["fp32_guarded"] = {
            "value": whole_job_rate(N, K, world, f32["ms"]), "ms_per_step": f32["ms"] / K,
            "gpu_launches": f32["launches"], "phases_ms_per_step": p32,
            "roofline_phases": rooflines(p32, N, k, levels, p0, cand, hbm, how, None),
            "guard_hits_fp32": f32["obs"]["guard_hits_fp32"],
            "guard_hits_fp64": f32["obs"]["guard_hits_fp64"]}
    line["fp64_peak"] = {"gflops": fpk["gflops"], "dfma_per_s": fpk["dfma_per_s"],
                         "expm1_per_s": fpk["expm1_per_s"], "log_per_s": fpk["log_per_s"],
                         "clocks": fpk["clocks"], "nominal_gflops": FP64_NOMINAL_GFLOPS}
    for key in ("long", "n_sw_100", "precision", "kw_bound", "graph_stats"):
        if key in res:
            line[key] = res[key]
    if "batch" in res:
        line["batched"] = res["batch"]
    if not args.no_cpu and world == 1:
        line["cpu_baseline"] = cpu_baseline(args.cpu_L, args.T, args.seed)
    print(json.dumps(line), flush=True)


def reference_arm(args, rank, world):
    """The oracle (plain C, all host cores) timed on a bounded sample of the workload."""
    if rank != 0:
        return
    import oracle as O

    ncores = os.cpu_count() or 1
    O.set_threads(ncores)
    L = args.ref_L
    ch = O.Chain(O.make_params(L, T=args.T, seed=args.seed))
    ch.sweep(args.warmup)
    t0 = time.perf_counter()
    ch.sweep(args.steps)
    dt = time.perf_counter() - t0
    value = L * L * args.steps / dt
    sample = ("%d MC steps (switch+colour+sweep, n_sw=1) of an L=%d lattice at T=%gD, %d OpenMP "
              "threads, %.1f s; per-site work matches the L=%d workload" % (
                  args.steps, L, args.T, ncores, dt, args.L))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": "L=%d open lattice, J=0, D=1, T=%gD, seed %d, n_sw=1, FP64 (a "
                               "bounded sample of the L=%d workload: same per-site work)" % (
                                   L, args.T, args.seed, args.L),
                   "L": L, "N": L * L, "T": args.T, "precision": "fp64",
                   "sample_of": {"L": args.L, "N": args.L * args.L}},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
