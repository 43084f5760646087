"""Throughput of the truncated-solver loop pipeline on one GB300 (or N replicas).

One step = one pass of the whole hot path over one batch of Z4 sources:
  nrhs low-precision bulk sources (multi-RHS CG on M^dag M, 16-bit sloppy)
  + n_hp correction sources (FP32/FP64-reliable CG and the same LP map)
  + the one-end contraction of all of them over 160 insertions and the
    p^2 <= 9 momenta, FP64 accumulation and the TSM combination.
metric: TSM sources/s (all sources of the step, LP and HP) at 24^3 x 48.

  value  -- device-timed (CUDA events) tsm_solve_tsm_dev: result stays in HBM
  e2e    -- wall time of tsm_solve_tsm with the result read back to pinned host
            memory and the momentum list sent every step
Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {
    "workload": "tsm_loops_24x24x24x48",
    "dims": [24, 24, 24, 48],
    "eps": 0.25, "gauge_seed": 3, "kappa": 0.125, "mu": 0.005, "t_bc": -1,
    "rho_lp": 1e-2, "rho_hp": 1e-8, "p2max": 9, "n_insertions": 160,
}
METRIC = "TSM sources/s incl. 160-insertion loops, 24^3x48"
UNIT = "sources/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nrhs", type=int, default=32)
    ap.add_argument("--n-hp", type=int, default=2)
    ap.add_argument("--lp", default="f16", choices=["f16", "bf16"])
    ap.add_argument("--precond", default="eo", choices=["none", "eo"],
                    help="eo: even-odd (Schur complement) preconditioned CG for both maps")
    ap.add_argument("--dims", default=None, help="Lx,Ly,Lz,T (default 24,24,24,48)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-equal-accuracy", action="store_true")
    ap.add_argument("--no-tdil", action="store_true", help="skip the time-dilution measurement")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 16^3x32 TSM-vs-FP64 and 32^3x64 1000+50 source workloads")
    ap.add_argument("--probe", default=None, choices=["dslash", "tsm"],
                    help="run a few launches of one kernel family for an ncu capture and exit")
    ap.add_argument("--probe-time", action="store_true", help="with --probe dslash: print event-timed GB/s")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []  # (perf_counter time, line)
        self.reader = None

    def start(self):
        """Start sampling every 50 ms and wait (at most 3 s) for the first
        sample, so that the timed region is covered from its start."""
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return

        def read():
            for line in self.proc.stdout:
                self.lines.append((time.perf_counter(), line))
        self.reader = threading.Thread(target=read, daemon=True)
        self.reader.start()
        t_end = time.perf_counter() + 3.0
        while not self.lines and time.perf_counter() < t_end:
            time.sleep(0.01)

    def stop(self, t0=None, t1=None):
        """Samples taken between perf_counter times t0 and t1 (all samples if
        none fall inside)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        if self.reader is not None:
            self.reader.join(timeout=5)
        lines = [ln for t, ln in self.lines if t0 is None or (t0 <= t <= t1)]
        if not lines:
            lines = [ln for _, ln in self.lines]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak_gbs():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------- oracle timing
# The oracle (plain numpy FP64) is timed on every host core through a pool of
# processes started with "spawn" (never forked from a process that has touched
# the GPU).  Each worker loads the same links, the Z4 source 0 and g5 A of it
# once; a timed "oracle step" is one source's worth of oracle work spread over
# the workers as tasks: `iters` applications of M^dag M (the CG's operator
# work; the vector updates are a few percent of it and are not timed), one
# application of A (g5 A s for the loops), and the densities and direct
# p^2 <= 9 projection of all 160 insertions in chunks.
_W = {}


def _oracle_init(path, dims, kappa, mu):
    import numpy as np
    from oracle import dirac, lattice, momenta, philox
    links = np.load(path, mmap_mode="r")
    _W["u"] = lattice.effective_links(links, -1)
    _W["dims"], _W["kappa"], _W["mu"] = tuple(dims), kappa, mu
    _W["eta"] = philox.z4_source(tuple(dims), 1003, 0)
    _W["v"] = dirac.gamma5(dirac.apply_A(_W["u"], _W["eta"], kappa))
    _W["moms"] = momenta.momentum_list(9)


def _oracle_task(task):
    from oracle import contract, dirac, solver
    kind = task[0]
    t0 = time.perf_counter()
    if kind == "mdm":
        dirac.apply_MdagM(_W["u"], _W["eta"], _W["kappa"], _W["mu"])
        extra = None
    elif kind == "A":
        dirac.apply_A(_W["u"], _W["eta"], _W["kappa"])
        extra = None
    elif kind == "ins":
        ins = list(task[1])
        dens = contract.loop_densities_pair(_W["u"], _W["eta"], _W["eta"], _W["kappa"], _W["mu"], only=set(ins),
                                            chi1=_W["v"])
        contract.project(dens[ins], _W["dims"], _W["moms"])
        extra = len(ins)
    else:  # "cg": the oracle's own CG to rho (iteration count)
        _, iters, res = solver.solve(_W["u"], _W["eta"], _W["kappa"], _W["mu"], task[1])
        extra = iters
    return kind, time.perf_counter() - t0, extra


class OraclePool:
    """Spawned worker processes holding the oracle's inputs at full size."""

    def __init__(self, dims, kappa, mu, workers=None):
        import multiprocessing as mp
        import tempfile
        import numpy as np
        from paper_1401_6750_gb300 import synth
        avail = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
        v = 1
        for d in dims:
            v *= d
        # about 12 site-sized complex fields plus the 160-insertion density array per worker
        per_worker = v * (160 * 16 + 12 * 192 + 2 * 576)
        try:
            mem = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
        except (ValueError, OSError):
            mem = 64 << 30
        self.workers = max(1, min(workers or avail, avail, int(0.6 * mem // per_worker)))
        self.cores_available = avail
        self.tmp = tempfile.NamedTemporaryFile(suffix=".npy", delete=False)
        self.tmp.close()
        np.save(self.tmp.name, synth.gauge_links(dims, 0.25, 3))
        t0 = time.perf_counter()
        self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_oracle_init,
                                                 initargs=(self.tmp.name, list(dims), kappa, mu))
        # wait until every worker has run its initializer
        self.pool.map(time.sleep, [0.2] * self.workers)
        self.setup_s = time.perf_counter() - t0

    def step(self, iters):
        """One source's worth of oracle work over all workers; wall seconds and task times."""
        chunks = max(1, self.workers)
        ins_chunks = [list(range(k, 160, chunks)) for k in range(chunks)]
        tasks = [("mdm",)] * int(round(iters)) + [("A",)] + [("ins", c) for c in ins_chunks]
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_task, tasks, chunksize=1)
        wall = time.perf_counter() - t0
        cpu = {"mdm": [], "A": [], "ins": []}
        for kind, t, _ in res:
            cpu[kind].append(t)
        return wall, cpu

    def cg_iterations(self, rho):
        kind, t, iters = self.pool.apply(_oracle_task, (("cg", rho),))
        return iters, t

    def close(self):
        self.pool.terminate()
        self.pool.join()
        try:
            os.unlink(self.tmp.name)
        except OSError:
            pass


def oracle_step_model(wall, cpu, iters_lp, iters_hp, n_lp, n_hp):
    """Oracle seconds for the 32 + 2 source TSM step from one timed oracle
    step (a source solved with iters_lp CG iterations and contracted, on all
    workers): every source gets an LP solve and a contraction, the correction
    sources also an HP solve (iters_hp iterations) and a second contraction."""
    import statistics
    t_mdm = statistics.median(cpu["mdm"])
    t_contract = sum(cpu["A"]) + sum(cpu["ins"])
    t_source_cpu = iters_lp * t_mdm + t_contract           # one core, under full load
    step_cpu = (n_lp + n_hp) * t_source_cpu + n_hp * (iters_hp * t_mdm + t_contract)
    return step_cpu, t_mdm, t_contract, t_source_cpu


def cpu_baseline(dims, kappa, mu, iters_lp, iters_hp, n_lp, n_hp, iters_how):
    """The oracle as it stands on all host cores: one timed oracle step (see
    OraclePool), scaled to the bench's TSM step of n_lp + n_hp sources."""
    pool = OraclePool(dims, kappa, mu)
    try:
        wall, cpu = pool.step(iters_lp)
    finally:
        pool.close()
    step_cpu, t_mdm, t_contract, t_src = oracle_step_model(wall, cpu, iters_lp, iters_hp, n_lp, n_hp)
    # the step's sources are independent: the workers process them in parallel
    step_wall = step_cpu / pool.workers
    return {
        "value": (n_lp + n_hp) / step_wall, "unit": UNIT, "cores": pool.workers,
        "cores_available": pool.cores_available, "kind": "oracle",
        "single_core_value": (n_lp + n_hp) / step_cpu,
        "sample": ("oracle numpy FP64 at %s on %d spawned worker processes: one source's oracle work (%d M^dag M "
                   "applications, %.2f s each; g5 A s and the densities with direct p^2<=9 projection of all 160 "
                   "insertions, %.1f s in all) took %.1f s of wall time; the %d + %d source TSM step (every source "
                   "an LP solve of %d iterations and a contraction, the %d correction sources also an HP solve of "
                   "%d iterations and a second contraction) is that per-source work scaled, spread over the "
                   "workers; iteration counts %s" % (
                       "x".join(map(str, dims)), pool.workers, int(round(iters_lp)), t_mdm, t_contract, wall, n_lp,
                       n_hp, int(round(iters_lp)), n_hp, int(round(iters_hp)), iters_how)),
        "extrapolated": True,
    }


def gpu_cg_iterations(dims, kappa, mu, rhos, device=0, gauge=None):
    """Iterations of the library's FP64 full-lattice CG on M^dag M (the same
    textbook CG and stopping rule as the oracle's: the parity tests check the
    counts agree within one) for Z4 source 0 of noise seed 1003, at each rho."""
    from paper_1401_6750_gb300 import abi, api, synth
    ctx = None
    g = gauge
    if g is None:
        ctx = api.Context(device)
        g = api.Gauge(ctx, synth.gauge_links(dims, 0.25, 3), dims, -1, precisions=(abi.TSM_F64,))
    out = []
    for rho in rhos:
        _, st = g.solve_sources(kappa, mu, abi.TSM_SOLVER_F64, rho, 1003, 0, 1)
        out.append(float(st[0]["iterations"]))
    if ctx is not None:
        g.close()
        ctx.close()
    return out


def run_reference(args):
    """Reference arm: the FP64 oracle, timed on all host cores.  Each step is
    one timed oracle step (one source solved with the oracle CG's own LP
    iteration count and contracted over all 160 insertions, spread over the
    spawned workers), scaled to the bench's 32 + 2 source TSM step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    dims = [int(v) for v in args.dims.split(",")] if args.dims else WORKLOAD["dims"]
    kappa, mu = WORKLOAD["kappa"], WORKLOAD["mu"]
    n_lp, n_hp = args.nrhs, args.n_hp
    # the HP count from the library's FP64 CG (an oracle CG to 1e-8 at this size runs for many minutes);
    # the LP count from the oracle's own CG, measured below
    iters_hp, how_hp = None, ""
    try:
        import torch
        if torch.cuda.is_available():
            iters_hp = gpu_cg_iterations(dims, kappa, mu, [WORKLOAD["rho_hp"]])[0]
            how_hp = "HP %d from the library's FP64 CG (same algorithm)" % iters_hp
    except Exception as e:  # no GPU: LP-only model
        how_hp = "no GPU for the HP count (%s): HP solves counted as LP" % type(e).__name__
    pool = OraclePool(dims, kappa, mu)
    try:
        iters_lp, t_cg = pool.cg_iterations(WORKLOAD["rho_lp"])
        if iters_hp is None:
            iters_hp = iters_lp
        how = "LP %d measured by the oracle's own CG (%.0f s); %s" % (iters_lp, t_cg, how_hp)
        vals = []
        for k in range(args.warmup + args.steps):
            wall, cpu = pool.step(iters_lp)
            if k >= args.warmup:
                step_cpu, t_mdm, t_contract, _ = oracle_step_model(wall, cpu, iters_lp, iters_hp, n_lp, n_hp)
                vals.append(((n_lp + n_hp) * pool.workers / step_cpu, wall, t_mdm, t_contract))
    finally:
        pool.close()
    vals.sort()
    v, wall, t_mdm, t_contract = vals[len(vals) // 2]
    sample = ("each step: one source's oracle work (%d M^dag M applications, %.2f s each; g5 A s and the 160 "
              "insertion densities with direct p^2<=9 projection, %.1f s in all) on %d spawned worker processes, "
              "%.1f s of wall time, scaled to the %d + %d source TSM step (every source an LP solve and a "
              "contraction, the correction sources also an HP solve and a second contraction): the value is "
              "extrapolated from the timed pieces; iteration counts %s" % (
                  int(round(iters_lp)), t_mdm, t_contract, pool.workers, wall, n_lp, n_hp, how))
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * (n_lp + n_hp) / v, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(WORKLOAD, dims=dims, sources_per_step={"lp_bulk": n_lp, "hp_correction": n_hp}),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": pool.workers, "cores_available": pool.cores_available,
                         "kind": "oracle", "sample": sample, "extrapolated": True},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _dslash_roofline(g, abi, torch, peak, prec, nrhs, reps=10):
    """Stand-alone operator M (tsm_dslash_tm) with an L2 flush before each
    launch; each launch is bracketed by CUDA events on the launching stream.
    The flush READS a 512 MB buffer (a sum), so that L2 holds clean lines when
    the operator starts: a flush by writing would leave the cache full of
    dirty lines whose write-back the timed kernel would pay for."""
    import ctypes
    dims = g.dims
    v = g.volume
    stream = torch.cuda.current_stream()
    src = g.sources(77, 0, nrhs, prec)
    out = g.empty_native(prec, nrhs)
    flush = torch.ones(128 * 1024 * 1024, dtype=torch.float32, device="cuda")
    link_b = {abi.TSM_F16: 96, abi.TSM_BF16: 96, abi.TSM_F32: 192, abi.TSM_F64: 576}[prec]
    spin_b = 16 * abi.CHUNKS[prec]
    times = []
    for k in range(reps + 2):
        flush.sum()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        abi.check(abi.lib().tsm_dslash_tm(g.handle, 0.125, 0.005, abi.TSM_OP_M, prec, ctypes.c_void_p(src.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), nrhs,
                                          ctypes.c_void_p(stream.cuda_stream)), "tsm_dslash_tm")
        e1.record(stream)
        e1.synchronize()
        if k >= 2:
            times.append(e0.elapsed_time(e1) * 1e-3)
    t = sorted(times)[len(times) // 2]
    bytes_ = v * (link_b + nrhs * 2 * spin_b)
    return {"kernel": "dslash_tm M %s r12, %d rhs, %s" % ({2: "f16", 3: "bf16", 1: "f32", 0: "f64"}[prec], nrhs,
                                                          "x".join(map(str, dims))),
            "achieved": bytes_ / t / 1e9, "peak": peak, "unit": "GB/s", "frac": bytes_ / t / 1e9 / peak,
            "bytes_per_launch": bytes_, "us_per_launch": t * 1e6, "l2": "flushed (512 MB read) before each launch"}


def measured_traffic(kernel_class):
    """DRAM bytes per launch of `kernel_class` from the committed ncu capture
    (profiles/roofline_traffic.txt), or None when that capture was taken for
    another kernel or on other sources of the kernel's translation unit (the
    record's source_files; all CUDA sources when it lists none)."""
    from paper_1401_6750_gb300 import build
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", "roofline_traffic.txt")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_class") != kernel_class or rec.get("source_digest") != build.source_digest(rec.get("source_files")):
        return None
    return rec.get("dram_bytes_per_launch")


def probe(args):
    """Small, self-contained workloads for profiler captures (no timing output).
    `--probe tsm` runs a first TSM step (workspaces, autotuner, graphs) and a
    steady-state one inside the NVTX range "tsm_step".  The correction solves
    run on the calling thread (TSM_STREAMS=1): a profiler serialises the
    kernels anyway, and one stream keeps the launch order readable."""
    import ctypes

    os.environ.setdefault("TSM_STREAMS", "1")

    import torch
    from paper_1401_6750_gb300 import abi, api, build, synth
    build.build()
    torch.cuda.set_stream(torch.cuda.Stream())  # launches and events on one non-default stream
    dims = [int(v) for v in args.dims.split(",")] if args.dims else WORKLOAD["dims"]
    links = synth.gauge_links(dims, WORKLOAD["eps"], WORKLOAD["gauge_seed"])
    ctx = api.Context(0)
    g = api.Gauge(ctx, links, dims, WORKLOAD["t_bc"], precisions=(abi.TSM_F64, abi.TSM_F32, abi.TSM_F16,
                                                                   abi.TSM_BF16))
    if args.probe == "dslash":
        prec = abi.TSM_F16 if args.lp == "f16" else abi.TSM_BF16
        src = g.sources(5, 0, args.nrhs, prec)
        for _ in range(3):
            g.dslash(abi.TSM_OP_M, WORKLOAD["kappa"], WORKLOAD["mu"], prec, src, args.nrhs)
        if args.probe_time:
            peak, _ = measured_peak_gbs()
            for p in (abi.TSM_F16, abi.TSM_BF16, abi.TSM_F32, abi.TSM_F64):
                print(json.dumps(_dslash_roofline(g, abi, torch, peak, p, args.nrhs)), flush=True)
    else:
        flag = abi.TSM_SOLVER_EO if args.precond == "eo" else 0
        lp = (abi.TSM_SOLVER_LP_F16 if args.lp == "f16" else abi.TSM_SOLVER_LP_BF16) | flag

        def step(seed):
            g.tsm(WORKLOAD["kappa"], WORKLOAD["mu"], args.nrhs, args.n_hp, WORKLOAD["rho_lp"], WORKLOAD["rho_hp"], lp,
                  abi.TSM_SOLVER_F32_RELIABLE | flag, seed, api.momentum_table(9), nrhs_per_launch=args.nrhs)
        step(10)  # first step: workspaces, autotuner timings, graph captures
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("tsm_step")  # a steady-state step (ncu --nvtx --nvtx-include tsm_step/)
        step(11)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    g.close()
    ctx.close()


def lp_variants(g, abi, torch, w, flag, hp_solver, moms, n_lp, n_hp, steps=2):
    """The same TSM step (n_lp bulk + n_hp correction sources) with the bulk
    LP solves at 12 right-hand sides per launch (FP16) and at 32 with BF16
    storage: the other two launch shapes of the 24^3x48 batched workload.
    One warm-up step, then `steps` steps timed with CUDA events."""
    import ctypes
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    n_out = 160 * moms.shape[0] * w["dims"][3] * 2
    out = torch.empty(n_out, dtype=torch.float64, device="cuda")
    res = []
    for nrhs, lp_name in ((12, "f16"), (32, "bf16")):
        lp = (abi.TSM_SOLVER_LP_F16 if lp_name == "f16" else abi.TSM_SOLVER_LP_BF16) | flag

        def step(k):
            p = abi.tsm_params(w["kappa"], w["mu"], n_lp, n_hp, w["rho_lp"], w["rho_hp"], lp, hp_solver,
                               77003 + 7919 * k, 20000, nrhs, moms.shape[0],
                               moms.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
            st = abi.tsm_stats()
            abi.check(abi.lib().tsm_solve_tsm_dev(g.handle, ctypes.byref(p), ctypes.c_void_p(out.data_ptr()), None,
                                                  ctypes.byref(st), sp), "tsm_solve_tsm_dev")
            return st
        step(0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        its = []
        for k in range(steps):
            st = step(1 + k)
            its.append(st.lp_iterations_total / (n_lp + n_hp))
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) * 1e-3
        res.append({"nrhs_per_launch": nrhs, "lp_storage": lp_name, "sources_per_step": n_lp + n_hp,
                    "sources_per_s": (n_lp + n_hp) * steps / t, "ms_per_step": t / steps * 1e3,
                    "lp_iterations_mean": round(sum(its) / len(its), 1)})
    return res


def equal_accuracy(g, abi, torch, w, lp_solver, hp_solver, moms, n_lp=64, n_hp=8, nrhs=32):
    """TSM against the plain high-precision path at equal final loop accuracy.

    Per-source samples (the scalar and gamma_5 loops of both flavour
    structures at p = 0, summed over timeslices) give the variances of
    the LP estimate, the correction L_HP - L_LP and the plain HP estimate;
    with the measured per-source times the cost to reach a given error is
      plain: sigma_HP^2 / eps^2 x t_HP
      TSM:   N_LP t_LP + N_HP (t_HP + t_LP), with sigma_LP^2/N_LP + sigma_corr^2/N_HP = eps^2
    and the TSM optimum N_LP/N_HP = sqrt(sigma_LP^2 (t_HP + t_LP) / (sigma_corr^2 t_LP)).
    """
    import ctypes

    import numpy as np
    seed = 424242
    sel = [0, 15, 80, 95]
    mom = [(0, 0, 0)]
    all_moms = np.ascontiguousarray(np.asarray(moms, dtype=np.int32))
    scratch_out = torch.zeros((abi.TSM_N_INSERTIONS, all_moms.shape[0], g.dims[3], 2), dtype=torch.float64,
                              device="cuda")

    def per_source(solver, first, n):
        # timed per batch: the solve and the 160-insertion contraction over all
        # p^2 <= 9 momenta, as in the TSM step; the per-source p = 0 samples
        # for the variances are taken afterwards, outside the timed region
        stream = torch.cuda.current_stream()
        kind = solver & ~abi.TSM_SOLVER_EO
        prec = abi.TSM_F64 if kind in (abi.TSM_SOLVER_F64, abi.TSM_SOLVER_F32_RELIABLE) else abi.TSM_F32
        t = 0.0
        vals = []
        for k0 in range(0, n, nrhs):
            m = min(nrhs, n - k0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sol, _ = g.solve_sources(w["kappa"], w["mu"], solver, w["rho_lp"] if solver == lp_solver else w["rho_hp"],
                                     seed, first + k0, m, nrhs_per_launch=m)
            if prec == abi.TSM_F64:  # contract in FP32 like the TSM driver
                sol = g.pack(g.unpack(sol, abi.TSM_F64, m), abi.TSM_F32)
            g.contract(w["kappa"], w["mu"], abi.TSM_F32, sol, m, all_moms, out=scratch_out)
            e1.record(stream)
            e1.synchronize()
            t += e0.elapsed_time(e1) * 1e-3
            field = g.native_bytes(abi.TSM_F32, 1)
            for j in range(m):
                out = g.contract(w["kappa"], w["mu"], abi.TSM_F32, sol[j * field:(j + 1) * field], 1, mom)
                a = out.cpu().numpy()
                vals.append((a[sel, 0, :, 0] + 1j * a[sel, 0, :, 1]).sum(axis=1))
        return np.array(vals), t / n

    lp_bulk, t_lp = per_source(lp_solver, 0, n_lp)
    hp, t_hp = per_source(hp_solver, n_lp, n_hp)
    lp_corr, _ = per_source(lp_solver, n_lp, n_hp)

    def var(a):  # real and imaginary parts, per observable
        return a.real.var(axis=0, ddof=1) + a.imag.var(axis=0, ddof=1)

    s_lp, s_corr, s_hp = var(lp_bulk), var(hp - lp_corr), var(hp)
    out = []
    for k, name in enumerate(["scalar tau3", "gamma5 tau3", "scalar", "gamma5"]):
        if s_hp[k] <= 0:
            continue
        ratio = np.sqrt(s_lp[k] * (t_hp + t_lp) / max(s_corr[k] * t_lp, 1e-300))
        # cost per unit inverse variance: plain s_hp t_hp; TSM (s_lp + s_corr/r)(t_lp + (t_hp+t_lp)/r)
        cost_plain = s_hp[k] * t_hp
        cost_tsm = (s_lp[k] + s_corr[k] / ratio) * (t_lp + (t_hp + t_lp) / ratio)
        out.append({"observable": name, "var_lp": float(s_lp[k]), "var_corr": float(s_corr[k]),
                    "var_hp": float(s_hp[k]), "opt_lp_per_hp": float(ratio),
                    "speedup_at_equal_error": float(cost_plain / cost_tsm)})
    return {"samples": {"lp": n_lp, "hp": n_hp}, "t_lp_s_per_source": t_lp, "t_hp_s_per_source": t_hp,
            "plain_hp_sources_per_s": 1.0 / t_hp, "observables": out,
            "note": "per-source times are solve + 160-insertion contraction over all p^2 <= 9 momenta, in batches "
                    "of %d; p = 0 loops summed over timeslices; variances from per-source samples" % nrhs}


def time_dilution(g, abi, torch, w, lp_solver, moms, reps=3):
    """The time-dilution workload (Sec. 2.2) on the same lattice: the T
    diluted sources of one noise vector, solved together by the LP map and
    contracted with the standard estimator on their own timeslices.  Timed
    with CUDA events on the current stream, after one warm-up pass."""
    import ctypes
    T = g.dims[3]
    stream = torch.cuda.current_stream()
    kind = lp_solver & ~abi.TSM_SOLVER_EO
    prec = abi.TSM_F64 if kind in (abi.TSM_SOLVER_F64, abi.TSM_SOLVER_F32_RELIABLE) else abi.TSM_F32
    t0 = list(range(T))
    out = torch.zeros((abi.TSM_N_INSERTIONS, len(moms), T, 2), dtype=torch.float64, device="cuda")
    times, t_solve, iters = [], [], []
    for rep in range(reps + 1):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        eta = g.diluted_sources(1017, rep, 0, T, prec)
        sol, st = g.invert(abi.TSM_OP_M, w["kappa"], w["mu"], lp_solver, w["rho_lp"], eta, T)
        e1.record(stream)
        g.contract_tdil(prec, sol, eta, T, t0, moms, out=out, accumulate=rep > 0)
        e2.record(stream)
        e2.synchronize()
        if rep > 0:
            times.append(e0.elapsed_time(e2) * 1e-3)
            t_solve.append(e0.elapsed_time(e1) * 1e-3)
            iters.append(sum(x["iterations"] for x in st) / T)
    t = sorted(times)[len(times) // 2]
    return {"workload": "one Z4 noise vector diluted over all %d timeslices (%d sources), LP map, standard "
                        "estimator on each source's timeslice" % (T, T),
            "diluted_sources_per_s": T / t, "noise_vectors_per_s": 1.0 / t, "ms_per_noise_vector": t * 1e3,
            "solve_share": sorted(t_solve)[len(t_solve) // 2] / t, "lp_iterations_mean": sum(iters) / len(iters),
            "reps": reps}


def hpe_variance(g, abi, torch, w, lp_solver, n=16):
    """Hopping parameter expansion against the plain standard estimator:
    n volume Z4 sources solved by the LP map; per source, the p = 0 scalar
    and g5 loops (summed over timeslices) of both flavour combinations, with
    and without the expansion; their variances over the sources and the
    event-timed cost of each contraction."""
    import numpy as np
    kind = lp_solver & ~abi.TSM_SOLVER_EO
    prec = abi.TSM_F64 if kind in (abi.TSM_SOLVER_F64, abi.TSM_SOLVER_F32_RELIABLE) else abi.TSM_F32
    stream = torch.cuda.current_stream()
    eta = g.sources(2017, 0, n, prec)
    sol, _ = g.invert(abi.TSM_OP_M, w["kappa"], w["mu"], lp_solver, w["rho_lp"], eta, n)
    field = g.native_bytes(prec, 1)
    sel = {"scalar (tau3)": 0, "g5 (tau3)": 15, "scalar": 80, "g5": 95}
    vals = {"plain": [], "hpe": []}
    times = {"plain": [], "hpe": []}
    mom = [(0, 0, 0)]
    for j in range(n):
        ej, sj = eta[j * field:(j + 1) * field], sol[j * field:(j + 1) * field]
        for kind_, fn in (("plain", lambda: g.contract_tdil(prec, sj, ej, 1, None, mom)),
                          ("hpe", lambda: g.contract_hpe(w["kappa"], w["mu"], prec, sj, ej, 1, None, mom))):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            e1.synchronize()
            times[kind_].append(e0.elapsed_time(e1))
            a = out.cpu().numpy()
            vals[kind_].append([(a[i, 0, :, 0] + 1j * a[i, 0, :, 1]).sum() for i in sel.values()])
    obs = []
    for k, name in enumerate(sel):
        vp = np.array([v[k] for v in vals["plain"]])
        vh = np.array([v[k] for v in vals["hpe"]])
        var_p = float(vp.real.var(ddof=1) + vp.imag.var(ddof=1))
        var_h = float(vh.real.var(ddof=1) + vh.imag.var(ddof=1))
        obs.append({"observable": name, "mean_plain": [float(vp.mean().real), float(vp.mean().imag)],
                    "mean_hpe": [float(vh.mean().real), float(vh.mean().imag)], "var_plain": var_p,
                    "var_hpe": var_h, "variance_ratio": var_p / var_h if var_h > 0 else None})
    med = lambda x: sorted(x[1:])[len(x[1:]) // 2]
    return {"sources": n, "estimator": "standard, volume Z4 sources, LP map", "observables": obs,
            "ms_contract_plain": med(times["plain"]), "ms_contract_hpe": med(times["hpe"]),
            "note": "variances per source of the p = 0 loops summed over timeslices"}


def binary_storage(g, abi, torch, w, lp_solver, moms, nrhs, k_end=5):
    """Binary-weight accumulation (Sec. 2.1.1, Fig. 2) of the bulk LP loops of
    2^k_end - 1 sources into block files in a temporary directory: wall time,
    files and bytes against one file per source, and the any-N read back."""
    import shutil
    import tempfile
    from paper_1401_6750_gb300 import api
    T = g.dims[3]
    n_values = 160 * len(moms) * T * 2
    d = tempfile.mkdtemp(prefix="tsm_blocks_")
    try:
        st = api.BinStore(os.path.join(d, "bulk"), n_values)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stats = st.accumulate(g, w["kappa"], w["mu"], lp_solver, w["rho_lp"], 2025, moms, k_end,
                              nrhs_per_launch=nrhs)
        t_acc = time.perf_counter() - t0
        n = st.sources
        t0 = time.perf_counter()
        for m in (n, n // 2 + 1):
            st.mean(m)
        t_read = (time.perf_counter() - t0) / 2
        files = sorted(f for f in os.listdir(d) if f.endswith(".bin"))
        size = sum(os.path.getsize(os.path.join(d, f)) for f in files)
        st.close()
    finally:
        shutil.rmtree(d, ignore_errors=True)
    per_source = n_values * 8
    return {"sources": n, "files": len(files), "bytes": size, "bytes_one_file_per_source": n * per_source,
            "storage_reduction": 1.0 - size / (n * per_source), "seconds_accumulate": t_acc,
            "sources_per_s": n / t_acc, "seconds_mean_any_n": t_read,
            "lp_iterations_mean": stats["lp_iterations_total"] / n}


def _tsm_dev_call(g, abi, torch, kappa, mu, n_lp, n_hp, rho_lp, rho_hp, lp, hp, seed, moms, nrhs, parts=False):
    """One tsm_solve_tsm_dev call, CUDA-event timed on the current stream."""
    import ctypes
    stream = torch.cuda.current_stream()
    n_out = 160 * moms.shape[0] * g.dims[3] * 2
    out = torch.empty(n_out, dtype=torch.float64, device="cuda")
    pt = torch.empty(3 * n_out, dtype=torch.float64, device="cuda") if parts else None
    p = abi.tsm_params(kappa, mu, n_lp, n_hp, rho_lp, rho_hp, lp, hp, seed, 20000, nrhs, moms.shape[0],
                       moms.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    st = abi.tsm_stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    abi.check(abi.lib().tsm_solve_tsm_dev(g.handle, ctypes.byref(p), ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(pt.data_ptr()) if parts else None, ctypes.byref(st),
                                          ctypes.c_void_p(stream.cuda_stream)), "tsm_solve_tsm_dev")
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) * 1e-3, out, pt, {f: getattr(st, f) for f, _ in st._fields_}


def tsm_vs_plain_16x16x16x32(ctx, abi, api, torch, synth, nrhs=32):
    """The 16^3 x 32 configuration (eps 0.3, gauge seed 2, kappa 0.125,
    mu 0.01, noise seed 1002): a TSM of 200 FP16 LP sources (rho 1e-2) and
    10 HP sources (FP32 CG, float-float reliable updates, rho 1e-8), all 160
    insertions over the p^2 <= 9 momenta, against the plain FP64 GPU path
    (every one of the 210 sources solved by the FP64 CG to 1e-8 and
    contracted in FP64).  Both timed with CUDA events after a warm-up; the two
    estimates of the p = 0 scalar and g5 loops (summed over timeslices) are
    compared in units of the plain path's standard error."""
    import numpy as np
    dims, kappa, mu, seed = (16, 16, 16, 32), 0.125, 0.01, 1002
    n_lp, n_hp = 200, 10
    eo = abi.TSM_SOLVER_EO
    lp, hp = abi.TSM_SOLVER_LP_F16 | eo, abi.TSM_SOLVER_F32_RELIABLE | eo
    g = api.Gauge(ctx, synth.gauge_links(dims, 0.3, 2), dims, -1,
                  precisions=(abi.TSM_F64, abi.TSM_F32, abi.TSM_F16))
    moms = np.ascontiguousarray(np.array(api.momentum_table(9), dtype=np.int32))
    try:
        _tsm_dev_call(g, abi, torch, kappa, mu, n_lp, n_hp, 1e-2, 1e-8, lp, hp, seed + 77, moms, nrhs)  # warm-up
        t_tsm, est, _, st = _tsm_dev_call(g, abi, torch, kappa, mu, n_lp, n_hp, 1e-2, 1e-8, lp, hp, seed, moms, nrhs)
        est = est.view(160, moms.shape[0], dims[3], 2).cpu().numpy()
        # plain FP64 path on the same 210 sources: batched solves + FP64 contraction, timed together
        stream = torch.cuda.current_stream()
        n = n_lp + n_hp
        acc = torch.zeros((160, moms.shape[0], dims[3], 2), dtype=torch.float64, device="cuda")
        g.solve_sources(kappa, mu, abi.TSM_SOLVER_F64 | eo, 1e-8, seed + 77, 0, nrhs, nrhs_per_launch=nrhs)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sols = []
        for k0 in range(0, n, nrhs):
            m = min(nrhs, n - k0)
            sol, _ = g.solve_sources(kappa, mu, abi.TSM_SOLVER_F64 | eo, 1e-8, seed, k0, m, nrhs_per_launch=m)
            g.contract(kappa, mu, abi.TSM_F64, sol, m, moms, out=acc, accumulate=k0 > 0)
            sols.append((sol, m))
        e1.record(stream)
        e1.synchronize()
        t_plain = e0.elapsed_time(e1) * 1e-3
        plain = acc.cpu().numpy() / n
        # per-source samples of the plain path (p = 0) for its standard error
        field = g.native_bytes(abi.TSM_F64, 1)
        samples = []
        for sol, m in sols:
            for j in range(m):
                o = g.contract(kappa, mu, abi.TSM_F64, sol[j * field:(j + 1) * field], 1, [(0, 0, 0)]).cpu().numpy()
                samples.append([complex(o[i, 0, :, 0].sum(), o[i, 0, :, 1].sum()) for i in (0, 15, 80, 95)])
        samples = np.array(samples)
        obs = []
        for k, (i, name) in enumerate(zip((0, 15, 80, 95), ("scalar tau3", "gamma5 tau3", "scalar", "gamma5"))):
            e_tsm = complex(est[i, 0, :, 0].sum(), est[i, 0, :, 1].sum())
            e_plain = complex(plain[i, 0, :, 0].sum(), plain[i, 0, :, 1].sum())
            se = np.sqrt((samples[:, k].real.var(ddof=1) + samples[:, k].imag.var(ddof=1)) / n)
            obs.append({"observable": name, "tsm": [e_tsm.real, e_tsm.imag], "plain_f64": [e_plain.real, e_plain.imag],
                        "diff_over_plain_stderr": abs(e_tsm - e_plain) / se if se > 0 else None})
        return {"workload": "16x16x16x32 eps 0.3 seed 2, kappa 0.125, mu 0.01: TSM 200 FP16 LP + 10 HP sources vs "
                            "the plain FP64 GPU path on the same 210 sources (even-odd CG, 160 insertions, "
                            "%d momenta)" % moms.shape[0],
                "tsm_seconds": t_tsm, "tsm_sources_per_s": n / t_tsm,
                "plain_f64_seconds": t_plain, "plain_f64_sources_per_s": n / t_plain,
                "speedup": t_plain / t_tsm,
                "lp_iterations_mean": st["lp_iterations_total"] / (n_lp + n_hp),
                "hp_iterations_mean": st["hp_iterations_total"] / n_hp,
                "lp_max_true_residual": st["lp_max_true_residual"], "hp_max_true_residual": st["hp_max_true_residual"],
                "observables": obs}
    finally:
        g.close()


def tsm_32x32x32x64(ctx, abi, api, torch, synth, nrhs=32):
    """Throughput of the differentiation configuration's volume, 32^3 x 64
    (eps 0.3, gauge seed 7, kappa 0.125, mu 0.01): one TSM of 1000 FP16 LP
    sources and 50 HP sources (FP32 CG, float-float reliable updates), all
    160 insertions and p^2 <= 9 momenta, CUDA-event timed after a warm-up
    call that builds the same launch shapes."""
    import numpy as np
    dims, kappa, mu, seed = (32, 32, 32, 64), 0.125, 0.01, 1005
    eo = abi.TSM_SOLVER_EO
    lp, hp = abi.TSM_SOLVER_LP_F16 | eo, abi.TSM_SOLVER_F32_RELIABLE | eo
    g = api.Gauge(ctx, synth.gauge_links(dims, 0.3, 7), dims, -1,
                  precisions=(abi.TSM_F64, abi.TSM_F32, abi.TSM_F16))
    moms = np.ascontiguousarray(np.array(api.momentum_table(9), dtype=np.int32))
    try:
        _tsm_dev_call(g, abi, torch, kappa, mu, 40, 50, 1e-2, 1e-8, lp, hp, seed + 77, moms, nrhs)  # warm-up
        t, _, _, st = _tsm_dev_call(g, abi, torch, kappa, mu, 1000, 50, 1e-2, 1e-8, lp, hp, seed, moms, nrhs)
        return {"workload": "32x32x32x64 eps 0.3 seed 7, kappa 0.125, mu 0.01: TSM 1000 FP16 LP + 50 HP sources "
                            "(even-odd CG, 160 insertions, %d momenta)" % moms.shape[0],
                "seconds": t, "sources_per_s": 1050 / t,
                "lp_iterations_mean": st["lp_iterations_total"] / 1050, "hp_iterations_mean": st["hp_iterations_total"] / 50,
                "lp_max_true_residual": st["lp_max_true_residual"], "hp_max_true_residual": st["hp_max_true_residual"],
                "n_not_converged": st["n_not_converged"]}
    finally:
        g.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.probe:
        probe(args)
        return
    import ctypes

    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1401_6750_gb300 import abi, api, build, synth
    build.build()
    lib = abi.lib()
    # one dedicated stream: the library launches on it and the events are recorded on it
    bench_stream = torch.cuda.Stream()
    torch.cuda.set_stream(bench_stream)

    dims = [int(v) for v in args.dims.split(",")] if args.dims else WORKLOAD["dims"]
    w = dict(WORKLOAD, dims=dims)
    links = synth.gauge_links(dims, w["eps"], w["gauge_seed"])
    ctx = api.Context(local)
    g = api.Gauge(ctx, links, dims, w["t_bc"], precisions=(abi.TSM_F64, abi.TSM_F32, abi.TSM_F16, abi.TSM_BF16))
    del links
    flag = abi.TSM_SOLVER_EO if args.precond == "eo" else 0
    lp_solver = (abi.TSM_SOLVER_LP_F16 if args.lp == "f16" else abi.TSM_SOLVER_LP_BF16) | flag
    hp_solver = abi.TSM_SOLVER_F32_RELIABLE | flag
    moms = np.ascontiguousarray(np.array(api.momentum_table(w["p2max"]), dtype=np.int32))
    n_mom = moms.shape[0]
    T = dims[3]
    n_out = 160 * n_mom * T * 2
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    out_dev = torch.empty(n_out, dtype=torch.float64, device="cuda")
    host_out = torch.empty(n_out, dtype=torch.float64, pin_memory=True)
    units_per_step = args.nrhs + args.n_hp

    def params(step):
        # distinct sources every step and on every rank (weak scaling over replicas)
        seed = 1003 + 1000003 * rank + 7919 * step
        return abi.tsm_params(w["kappa"], w["mu"], args.nrhs, args.n_hp, w["rho_lp"], w["rho_hp"], lp_solver,
                              hp_solver, seed, 20000, args.nrhs, n_mom,
                              moms.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))

    stats_log = []

    def step_dev(k):
        p = params(k)
        st = abi.tsm_stats()
        rc = lib.tsm_solve_tsm_dev(g.handle, ctypes.byref(p), ctypes.c_void_p(out_dev.data_ptr()), None,
                                   ctypes.byref(st), sp)
        abi.check(rc, "tsm_solve_tsm_dev")
        stats_log.append({f: getattr(st, f) for f, _ in st._fields_})

    def step_host(k):
        p = params(k)
        rc = lib.tsm_solve_tsm(g.handle, ctypes.byref(p), ctypes.c_void_p(host_out.data_ptr()), None, None, sp)
        abi.check(rc, "tsm_solve_tsm")

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            torch.cuda.synchronize()

    def max_over_ranks(x):
        from paper_1401_6750_gb300 import replicas
        return replicas.max_over_ranks(x, device="cuda")

    for k in range(args.warmup):
        step_dev(k)
    launches0 = lib.tsm_kernel_launches()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t_wall0 = time.perf_counter()
    e0.record(stream)
    for k in range(args.steps):
        step_dev(args.warmup + k)
    e1.record(stream)
    e1.synchronize()
    t_wall1 = time.perf_counter()
    elapsed = e0.elapsed_time(e1) * 1e-3
    clk = clocks.stop(t_wall0, t_wall1)
    launches = lib.tsm_kernel_launches() - launches0
    barrier()
    elapsed = max_over_ranks(elapsed)
    value = world * units_per_step * args.steps / elapsed
    timed_stats = stats_log[args.warmup:]
    lp_iters = sum(s["lp_iterations_total"] for s in timed_stats) / max(1, sum(
        (args.nrhs + args.n_hp) for _ in timed_stats))
    hp_iters = sum(s["hp_iterations_total"] for s in timed_stats) / max(1, args.n_hp * len(timed_stats))

    e2e = None
    if not args.no_e2e:
        barrier()
        t0 = time.perf_counter()
        for k in range(args.steps):
            step_host(args.warmup + args.steps + k)
        torch.cuda.synchronize()
        t_e2e = max_over_ranks(time.perf_counter() - t0)
        n_contract_calls = 1 + 2 * ((args.n_hp + args.nrhs - 1) // args.nrhs) if args.n_hp else 1
        e2e = {"value": world * units_per_step * args.steps / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": int(n_contract_calls * moms.nbytes + ctypes.sizeof(abi.tsm_params)),
               "d2h_bytes_per_step": int(n_out * 8)}

    # roofline: one profiled step (kernel classes event-timed), plus the stand-alone operator
    peak, peak_kind = measured_peak_gbs()
    barrier()
    lib.tsm_profile_enable(1)
    step_dev(10**6)
    torch.cuda.synchronize()
    lib.tsm_profile_enable(0)
    n = lib.tsm_profile_read(None, 0)
    buf = (abi.tsm_kernel_profile * n)()
    lib.tsm_profile_read(buf, n)
    kern = [{"name": b.name.decode(), "launches": b.launches, "seconds": b.seconds, "bytes": b.bytes,
             "flops": b.flops} for b in buf]
    kern.sort(key=lambda d: -d["seconds"])
    total_s = sum(d["seconds"] for d in kern)
    dom = kern[0]
    achieved = dom["bytes"] / dom["seconds"] / 1e9
    roofline = {"bound": "hbm", "kernel": dom["name"], "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind, "traffic": measured_traffic(dom["name"]),
                "us_per_launch": dom["seconds"] / dom["launches"] * 1e6,
                "bytes_per_launch": dom["bytes"] / dom["launches"],
                "share_of_step": dom["seconds"] / total_s}
    kernels = [{"name": d["name"], "launches": d["launches"], "share": round(d["seconds"] / total_s, 4),
                "GB/s": round(d["bytes"] / d["seconds"] / 1e9, 1),
                "TFLOP/s": round(d["flops"] / d["seconds"] / 1e12, 2)} for d in kern]
    # the FP32-pipe-bound kernels against the FP32 arithmetic peak: SMs x 128
    # FP32 lanes x 2 flops per FMA x the SM clock sampled in the timed region
    # (a measured register-only FFMA2 loop reaches 0.99 of this)
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = clk.get("sm_mhz") or 2070.0
    fp32_peak = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12
    alu = [{"kernel": d["name"], "bound": "alu", "achieved": d["flops"] / d["seconds"] / 1e12, "peak": fp32_peak,
            "unit": "TFLOP/s", "frac": d["flops"] / d["seconds"] / 1e12 / fp32_peak,
            "peak_source": "derived: %d SMs x 128 FP32 lanes x 2 x %.0f MHz" % (n_sm, sm_mhz)}
           for d in kern if d["name"] in ("contract_fields_f32", "eo_hop_to_even_f16", "eo_hop_to_odd_Mp_f16")]
    dslash = [_dslash_roofline(g, abi, torch, peak, prec, nrhs)
              for prec in (abi.TSM_F16, abi.TSM_F32) for nrhs in (1, 12)]

    eq = None
    if rank == 0 and not args.no_equal_accuracy:
        eq = equal_accuracy(g, abi, torch, w, lp_solver, hp_solver, moms)

    variants = None
    if rank == 0 and not args.no_tdil:
        variants = lp_variants(g, abi, torch, w, flag, hp_solver, moms, args.nrhs, args.n_hp)

    tdil = None
    hpe_var = None
    binstore = None
    if rank == 0 and not args.no_tdil:
        tdil = time_dilution(g, abi, torch, w, lp_solver, moms)
        hpe_var = hpe_variance(g, abi, torch, w, lp_solver)
        binstore = binary_storage(g, abi, torch, w, lp_solver, moms, args.nrhs)

    cfg16 = cfg32 = None
    if rank == 0 and not args.no_configs:
        cfg16 = tsm_vs_plain_16x16x16x32(ctx, abi, api, torch, synth)
        cfg32 = tsm_32x32x32x64(ctx, abi, api, torch, synth)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        it_lp, it_hp = gpu_cg_iterations(dims, w["kappa"], w["mu"], [w["rho_lp"], w["rho_hp"]], gauge=g)
        cpu = cpu_baseline(dims, w["kappa"], w["mu"], it_lp, it_hp, args.nrhs, args.n_hp,
                           "LP %d and HP %d from the library's FP64 full-lattice CG (the oracle's CG, the same "
                           "algorithm and stopping rule), measured in this run" % (it_lp, it_hp))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w["workload"], "dims": dims, "eps": w["eps"], "kappa": w["kappa"], "mu": w["mu"],
                       "lp_solver": "%s storage (links r12, p, Ap), f32 x/r, rho %g" % (args.lp, w["rho_lp"]),
                       "hp_solver": "f32 CG + float-float reliable updates and solution sum, rho %g" % w["rho_hp"],
                       "preconditioning": "even-odd (Schur complement on odd sites)" if flag else "none",
                       "sources_per_step": {"lp_bulk": args.nrhs, "hp_correction": args.n_hp},
                       "nrhs_per_launch": args.nrhs, "insertions": 160, "momenta": n_mom,
                       "l2": "inputs larger than L2 (CG working set %.1f GB)" % (
                           args.nrhs * g.volume * (96 * 4 + 48 * 2) / 1e9),
                       "parallelism": "replicas x%d" % world},
            "roofline": roofline,
            "kernels": kernels[:14],
            "alu_roofline": alu,
            "dslash": dslash,
            "iterations": {"lp_mean": round(lp_iters, 1), "hp_mean": round(hp_iters, 1)},
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk,
            "cpu_baseline": cpu,
            "equal_accuracy": eq,
            "launch_shapes": variants,
            "time_dilution": tdil,
            "hpe": hpe_var,
            "binary_storage": binstore,
            "tsm_vs_plain_f64_16x16x16x32": cfg16,
            "tsm_1000_50_32x32x32x64": cfg32,
        }
        print(json.dumps(line), flush=True)
    g.close()
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
