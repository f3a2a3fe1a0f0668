"""Benchmark of the MDWF propagator solve on GB300.

Workload (default, the precision configuration): 24^3 x 64 lattice, Ls = 10, Moebius
b5 = 1.5, c5 = 0.5, M5 = 1.3, m_f = 0.01, synthetic links exp(i 0.5 H) reunitarised
(Philox seed 3), one spin-colour point source at the origin.  One step = the point-source
propagator column through the library's public calls: 4D source -> 5D source
(Pauli-Villars injection), mixed-precision (F16 + norm storage, FP32 accumulation, FP64
reliable updates) even-odd CG on the normal equations to a true FP64 relative residual of
1e-10, and the 4D projection.

Reported: value = algorithmic HBM GB/s of the whole step (bytes the library's kernels must
move, counted by the library, divided by the step's device time), the mixed and the plain
FP64 solve times to 1e-10 and their ratio, the roofline of the dominant kernel (the fused
hop + M5^-1 kernel, timed alone with an L2 flush before every launch), the same step end
to end through the library's host-buffer path (MDWF_HOST pointers: the library copies
in and out), SM clocks during the timed region, and the FP64 CPU oracle timed on the host
cores (one core, and all cores on independent T-slabs of the lattice).

--impl reference runs the oracle (the FP64 numpy reference of the method) on all host
cores on a bounded sample of the same workload and prints the same JSON line.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: dims (X,Y,Z,T), Ls, mf, eps, seed
    "16^3x32_Ls12": ((16, 16, 16, 32), 12, 0.02, 0.4, 2),
    "24^3x64_Ls10": ((24, 24, 24, 64), 10, 0.01, 0.5, 3),
    "4^4_Ls8": ((4, 4, 4, 4), 8, 0.05, 0.2, 1),
    "32^3x64_Ls12": ((32, 32, 32, 64), 12, 0.01, 0.5, 4),
    "48^3x96_Ls8": ((48, 48, 48, 96), 8, 0.005, 0.6, 5),
}
# extra modes (one JSON line each, not the default benchmark line)
MODES = ("batch32", "large48", "graphbatch", "multirhs")
METRIC = "MDWF Dslash HBM GB/s (% of peak); solve time to 1e-10, mixed vs FP64"


# the files that define the device code and launch of the hop kernels (the roofline kernel)
KERNEL_FILES = ["dslash.cu", "dslash_bf16.cu", "dslash_f16.cu", "dslash_f32.cu", "dslash_f64.cu", "dslash_i16.cu",
                "dslash2_bf16.cu", "dslash2_f16.cu", "dslash2_f32.cu", "dslash2_i16.cu",
                "dslash3_bf16.cu", "dslash3_f16.cu", "dslash3_i16.cu",
                "dslash_impl.cuh", "dslash_umma.cu", "mdwf_epi.cuh", "mdwf_impl.cuh", "mdwf_kernels.h"]


def kernel_sources_hash():
    """sha256 over the sources of the hop kernels: identifies the kernels a stored ncu
    capture belongs to (host-side solver changes leave it alone)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1810_01609_gb300", "csrc")
    for name in KERNEL_FILES:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()


def stored_traffic(key, tune_value=None):
    """DRAM bytes per launch from profiles/roofline_traffic.json if it was captured on the
    current kernel sources and on the same kernel variant (the tuner value's flag bits:
    single-column, 64-register, tensor-core or paired-column kernel), else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            d = json.load(f)
        if d.get("sources_sha256") != kernel_sources_hash():
            return None
        e = d["entries"][key]
        if tune_value is not None and "tune_value" in e and (e["tune_value"] >> 16) != (tune_value >> 16):
            return None
        return e["dram_bytes_per_launch"]
    except Exception:
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, gpu_index):
        self.samples = []
        self.proc = None
        self.idx = gpu_index

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def slab_dims(dims):
    """A periodic T-slab of the lattice (the same X, Y, Z; T / 16, at least 2 and even)
    whose oracle CG iteration costs about a sixteenth of the full one (the whole lattice when
    T <= 8): the bounded sample
    of the workload that the CPU baseline times (per-site arithmetic of the oracle does not
    depend on the lattice extent)."""
    X, Y, Z, T = dims
    ts = T if T <= 8 else max(2, (T // 16) // 2 * 2)
    return (X, Y, Z, ts)


def oracle_slab_iterations(dims, Ls, mf, eps, seed, k, budget_s, max_iters=50):
    """CGNR iterations (one M_pc and one M_pc^+ apply each) of the FP64 numpy oracle on
    slab k of the workload (links and a Gaussian odd-site field drawn with seed*1000+k),
    repeated until budget_s seconds have passed.  Returns (iterations, seconds); the link
    and field generation is not timed."""
    import inputs
    from oracle import dirac
    from oracle.dirac import MobiusParams
    sd = slab_dims(dims)
    U = inputs.gauge_links(sd, eps, seed * 1000 + k)
    p = MobiusParams(Ls=Ls, mf=mf)
    Ub = dirac.boundary_links(U, -1.0)
    par = dirac.parity_mask(sd)
    x = dirac.on_parity(inputs.gaussian_spinor5d(sd, Ls, seed * 1000 + k + 100), par, 1)
    t0 = time.perf_counter()
    its = 0
    while True:
        q = dirac.mpc(Ub, x, p)
        x = dirac.mpc_dag(Ub, q, p) * 1e-1
        its += 1
        if time.perf_counter() - t0 >= budget_s or its >= max_iters:
            break
    return its, time.perf_counter() - t0


def _oracle_worker(a):
    return oracle_slab_iterations(*a)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_oracle(dims, Ls, mf, eps, seed, budget_s, workers):
    """Oracle throughput on the host cores, as GB/s of the GPU step's algorithmic bytes per
    CG iteration: workers = 1 runs one slab in this process; workers > 1 runs one slab per
    process in a spawn pool (independent slabs, together a CG iteration over the whole
    lattice when workers = 16) and divides the bytes of all slabs by the slowest worker's
    time.  Returns (GB/s, description, workers used)."""
    sd = slab_dims(dims)
    per_it = per_iteration_bytes(sd, Ls)
    if workers <= 1:
        its, dt = oracle_slab_iterations(dims, Ls, mf, eps, seed, 0, budget_s)
        gbs = its * per_it / dt / 1e9
        return gbs, "%d CGNR iteration(s) of the FP64 numpy oracle on one %s slab, Ls=%d, one process, %.1f s" % (
            its, "x".join(map(str, sd)), Ls, dt), 1
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    # memory: about 12 slab-sized complex fields per worker
    vol = sd[0] * sd[1] * sd[2] * sd[3] * Ls * 12 * 16
    try:
        mem = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
        workers = max(1, min(workers, int(mem * 0.5 // (12 * vol))))
    except Exception:
        pass
    args = [(dims, Ls, mf, eps, seed, k, budget_s, 1) for k in range(workers)]
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_worker, args))
    its = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    gbs = its * per_it / dt / 1e9
    return gbs, ("%d CGNR iterations of the FP64 numpy oracle, one per process on %d independent %s slabs "
                 "(Ls=%d) at once, %.1f s (slowest process)" % (its, workers, "x".join(map(str, sd)), Ls, dt)), workers


def oracle_smallest_solve_s():
    """Wall time of the oracle's full FP64 even-odd CG solve of the smallest configuration
    (4^4, Ls 8, m_f 0.05, links eps 0.2 seed 1, point source) to 1e-10."""
    import inputs
    from oracle import dirac, solve
    from oracle.dirac import MobiusParams
    dims, Ls = (4, 4, 4, 4), 8
    U = inputs.gauge_links(dims, 0.2, 1)
    b = np.zeros((Ls,) + tuple(reversed(dims)) + (4, 3), dtype=np.complex128)
    b[0, 0, 0, 0, 0, 0, 0] = 1.0
    t0 = time.perf_counter()
    _, its, _ = solve.solve_eo(dirac.boundary_links(U, -1.0), b, MobiusParams(Ls=Ls, mf=0.05), tol=1e-10)
    return time.perf_counter() - t0, its


def per_iteration_bytes(dims, Ls, nrhs=1):
    """Algorithmic bytes of one mixed (F16) CG iteration, the library's own count:
    K1 hop (in, out, links), K2 hop (+centre), K3 hop, K4 hop (+centre, r read+write),
    cg_update (x F32 read+write, p read+write, r read, phat write)."""
    vh = dims[0] * dims[1] * dims[2] * dims[3] // 2
    f16 = vh * Ls * nrhs * 52.0
    f32 = vh * Ls * nrhs * 96.0
    links = vh * 8 * 18 * 2.0
    return (2 * f16 + links) + (3 * f16 + links) + (2 * f16 + links) + (4 * f16 + links) + (2 * f32 + 4 * f16)


def replica_aggregate(ms_step_local, bytes_step_local, dist=None, device="cpu"):
    """Replicas: every rank runs the same independent workload.  Returns (ms_step, value):
    the slowest rank's step time and the whole-job throughput = sum over ranks of the
    bytes per step / that time (GB/s)."""
    import torch
    world = 1
    ms, nbytes = float(ms_step_local), float(bytes_step_local)
    if dist is not None and dist.is_initialized():
        world = dist.get_world_size()
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        b = torch.tensor([nbytes], dtype=torch.float64, device=device)
        dist.all_reduce(b, op=dist.ReduceOp.SUM)
        ms, nbytes = float(t.item()), float(b.item())
    return ms, nbytes / (ms * 1e-3) / 1e9


def run_reference(args, wl):
    dims, Ls, mf, eps, seed = WORKLOADS[wl]
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = min(16, host_cores())
    vals, descs, ws = [], [], []
    t_all = time.perf_counter()
    for i in range(args.warmup + args.steps):
        gbs, desc, w = cpu_oracle(dims, Ls, mf, eps, seed, args.ref_budget, cores)
        if i >= args.warmup:
            vals.append(gbs)
            descs.append(desc)
            ws.append(w)
    gbs = float(np.mean(vals))
    per_it = per_iteration_bytes(slab_dims(dims), Ls) * ws[-1]
    out = {"metric": METRIC, "value": gbs, "unit": "GB/s", "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_it / (gbs * 1e9) * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": wl, "lattice": list(dims), "Ls": Ls, "mf": mf},
           "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": ws[-1], "kind": "oracle",
                            "sample": descs[-1] + "; per step"},
           "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "wall_s": time.perf_counter() - t_all}
    print(json.dumps(out))


def kernel_only(args, m, ctx, dims, Ls, seed, stream):
    import torch
    import inputs
    prec = m.PRECS[args.sloppy]
    nr = args.nrhs
    nb = ctx.field_bytes(args.sloppy, nr)
    fin = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    fout = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    src = inputs.gaussian_spinor5d_device(dims, Ls, seed + 100, nrhs=nr)
    m.mdwf_pack(ctx.h, src, fin, prec, nr, stream)
    del src
    m.mdwf_apply(ctx.h, m.OP[args.op], prec, fin, fout, nr, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.kernel_launches):
        m.mdwf_apply(ctx.h, m.OP[args.op], prec, fin, fout, nr, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(1, args.kernel_launches)
    print(json.dumps({"kernel_only": args.op, "nrhs": nr, "launches": args.kernel_launches, "ms_per_launch": ms,
                      "tune": ctx.tune_entries()}))


def _setup_gpu():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1810_01609_gb300 as m
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    return torch, m, stream


def mode_batch32(args):
    """32^3x64, Ls 12: 12 spin-colour point sources -> multi-RHS mixed solves (groups of
    --group right-hand sides per launch), Feynman-Hellmann sequential solves, nucleon 2-pt
    and FH 3-pt (both u lines) contractions in FP64."""
    torch, m, stream = _setup_gpu()
    import inputs
    dims, Ls, mf, eps, seed = WORKLOADS["32^3x64_Ls12"]
    ctx = m.Context(dims, Ls, mf=mf)
    t0 = time.perf_counter()
    ctx.load_gauge(inputs.gauge_links(dims, eps, seed))
    t_links = time.perf_counter() - t0
    G = args.group
    b4 = torch.stack([torch.from_numpy(inputs.point_source4d(dims, k // 3, k % 3)) for k in range(12)]).cuda()

    def solve_cols(src4):
        cols, its, rus, res = [], [], [], []
        for g0 in range(0, 12, G):
            eta = ctx.make_source_4d(src4[g0:g0 + G].contiguous(), nrhs=G, stream=stream)
            y, infos = ctx.solve_multi(eta, sloppy=args.sloppy, tol=1e-10, full_residual=False, stream=stream)
            del eta
            cols.append(ctx.project_4d(y, nrhs=G, stream=stream))
            del y
            its += [i.iterations for i in infos]
            rus += [i.reliable_updates for i in infos]
            res += [i.true_residual for i in infos]
        return torch.cat(cols), its, rus, res

    torch.cuda.synchronize()
    bytes0, launches0 = ctx.algorithmic_bytes(), ctx.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    S, its, rus, res = solve_cols(b4)
    SF, its_f, rus_f, res_f = solve_cols(ctx.fh_source(S, nrhs=12, stream=stream))
    C2 = ctx.contract_nucleon(S, S, S, stream=stream)
    C3 = ctx.contract_nucleon(SF, S, S, stream=stream) + ctx.contract_nucleon(S, S, SF, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    nbytes = ctx.algorithmic_bytes() - bytes0
    c2 = C2.cpu().numpy()
    geff = m.mdwf_fh_effective_coupling(C2, C3)
    out = {"metric": METRIC, "value": nbytes / (ms * 1e-3) / 1e9, "unit": "GB/s", "n_gpus": 1, "steps": 1,
           "warmup": 0, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f16+f32 (inner), f64", "data": "synthetic",
           "config": {"workload": "batch32: 32^3x64 Ls12, 12 point sources + 12 FH sequential solves + contractions",
                      "lattice": list(dims), "Ls": Ls, "mf": mf, "link_eps": eps, "seed": seed,
                      "rhs_per_launch": G, "sloppy": args.sloppy, "tol": 1e-10},
           "solve": {"iterations": its, "iterations_fh": its_f, "reliable_updates": rus,
                     "max_true_residual": max(res + res_f)},
           "nucleon_2pt_t0_4": [[float(z.real), float(z.imag)] for z in c2[:5]],
           "fh_effective_coupling_t0_4": [float(v) for v in geff[:5]],
           "gpu_launches": int(ctx.launch_count() - launches0), "host_link_generation_s": t_links}
    print(json.dumps(out))


def mode_multirhs(args):
    """16^3x32, Ls 12: the 12 spin-colour point-source propagator solves with 1, 3, 6 and
    12 right-hand sides per mdwf_solve_multi launch (after one warm-up pass per grouping:
    tuning, graph capture); per-solve wall time, iterations and worst true residual."""
    torch, m, stream = _setup_gpu()
    import inputs
    dims, Ls, mf, eps, seed = WORKLOADS["16^3x32_Ls12"]
    ctx = m.Context(dims, Ls, mf=mf)
    ctx.load_gauge(inputs.gauge_links(dims, eps, seed))
    b4 = torch.stack([torch.from_numpy(inputs.point_source4d(dims, k // 3, k % 3)) for k in range(12)]).cuda()
    eta = ctx.make_source_4d(b4, nrhs=12, stream=stream)
    res = {}
    for G in (1, 3, 6, 12):
        def run():
            its, worst = [], 0.0
            for g0 in range(0, 12, G):
                _, infos = ctx.solve_multi(eta[g0:g0 + G].contiguous(), sloppy=args.sloppy, tol=1e-10, stream=stream)
                its += [i.iterations for i in infos]
                worst = max(worst, max(i.true_residual for i in infos))
            return its, worst
        run()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its, worst = run()
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
        res[str(G)] = {"ms_per_solve": ms / 12, "iterations": [min(its), max(its)], "max_true_residual": worst}
    out = {"metric": METRIC, "value": 12 / (min(r["ms_per_solve"] for r in res.values()) * 12e-3), "unit": "solves/s",
           "n_gpus": 1, "steps": 1, "warmup": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f16+f32 (inner), f64", "data": "synthetic",
           "config": {"workload": "multirhs: 16^3x32 Ls12, 12 point sources, 1/3/6/12 right-hand sides per launch",
                      "lattice": list(dims), "Ls": Ls, "mf": mf, "sloppy": args.sloppy, "tol": 1e-10},
           "per_launch_grouping": res}
    print(json.dumps(out))


def mode_large48(args):
    """48^3x96, Ls 8, m 0.005: one point-source mixed solve (links drawn on the device)."""
    torch, m, stream = _setup_gpu()
    import inputs
    dims, Ls, mf, eps, seed = WORKLOADS["48^3x96_Ls8"]
    ctx = m.Context(dims, Ls, mf=mf)
    U = inputs.gauge_links_device(dims, eps, seed)
    ctx.load_gauge(U, stream=stream)
    del U
    b4 = torch.from_numpy(inputs.point_source4d(dims, 0, 0)).cuda().reshape((1,) + ctx.shape4d())
    eta = ctx.make_source_4d(b4, nrhs=1, stream=stream)[0]
    ctx.solve(eta, sloppy=args.sloppy, tol=1e-10, maxiter=200, stream=stream)   # tuning, graphs
    torch.cuda.synchronize()
    bytes0 = ctx.algorithmic_bytes()
    t0 = time.perf_counter()
    x, info = ctx.solve(eta, sloppy=args.sloppy, tol=1e-10, stream=stream)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    nbytes = ctx.algorithmic_bytes() - bytes0
    out = {"metric": METRIC, "value": nbytes / (ms * 1e-3) / 1e9, "unit": "GB/s", "n_gpus": 1, "steps": 1,
           "warmup": 1, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f16+f32 (inner), f64", "data": "synthetic",
           "config": {"workload": "large48: 48^3x96 Ls8 point-source solve", "lattice": list(dims), "Ls": Ls,
                      "mf": mf, "link_eps": eps, "seed": seed, "links": "device Philox (inputs.gauge_links_device)",
                      "sloppy": args.sloppy, "tol": 1e-10},
           "solve": {"ms": ms, "iterations": info.iterations, "reliable_updates": info.reliable_updates,
                     "fp64_residuals": info.fp64_residuals,
                     "true_residual": info.true_residual, "full_residual": info.full_residual},
           "device_memory_peak_gb": torch.cuda.max_memory_allocated() / 1e9}
    print(json.dumps(out))


def mode_graphbatch(args):
    """64 solves drawn uniformly from {8^3x16, 12^3x24, 16^3x32} x Ls {8, 12}, Z2-noise
    sources, CG iterations replayed as captured graphs per shape; solves/s and p50/p99
    latency, against the plain FP64 solver on the first --fp64-solves of the same draws."""
    torch, m, stream = _setup_gpu()
    import inputs
    shapes = [(d, ls) for d in ((8, 8, 8, 16), (12, 12, 12, 24), (16, 16, 16, 32)) for ls in (8, 12)]
    mf, eps, seed = 0.005, 0.6, 5
    rng = np.random.default_rng(seed)
    draws = rng.integers(0, len(shapes), size=64)
    ctxs = {}
    for k, (d, ls) in enumerate(shapes):
        c = m.Context(d, ls, mf=mf)
        c.load_gauge(inputs.gauge_links(d, eps, seed + 10 * k))
        ctxs[k] = c

    def src(i):
        d, ls = shapes[draws[i]]
        z = torch.from_numpy(inputs.z2_source4d(d, seed + 1000 + i)).cuda().reshape((1,) + ctxs[draws[i]].shape4d())
        return ctxs[draws[i]].make_source_4d(z, nrhs=1, stream=stream)[0]

    srcs = [src(i) for i in range(64)]
    for k in ctxs:   # one warm solve per shape: tuning and graph capture
        j = int(np.nonzero(draws == k)[0][0]) if np.any(draws == k) else None
        if j is not None:
            ctxs[k].solve(srcs[j], sloppy=args.sloppy, tol=1e-10, stream=stream)
    torch.cuda.synchronize()
    lat, its = [], []
    t0 = time.perf_counter()
    for i in range(64):
        t = time.perf_counter()
        x, info = ctxs[draws[i]].solve(srcs[i], sloppy=args.sloppy, tol=1e-10, stream=stream)
        lat.append((time.perf_counter() - t) * 1e3)
        its.append(info.iterations)
    total = time.perf_counter() - t0
    lat64 = []
    for k in ctxs:   # FP64 path warmed up per shape as well (its kernels tune on first use)
        j = int(np.nonzero(draws == k)[0][0]) if np.any(draws == k) else None
        if j is not None:
            ctxs[k].solve(srcs[j], sloppy="f64", tol=1e-10, stream=stream)
    torch.cuda.synchronize()
    for i in range(min(args.fp64_solves, 64)):
        t = time.perf_counter()
        ctxs[draws[i]].solve(srcs[i], sloppy="f64", tol=1e-10, stream=stream)
        lat64.append((time.perf_counter() - t) * 1e3)
    out = {"metric": METRIC, "value": 64 / total, "unit": "solves/s", "n_gpus": 1, "steps": 64, "warmup": len(ctxs),
           "ms_per_step": total * 1e3 / 64, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f16+f32 (inner), f64", "data": "synthetic",
           "config": {"workload": "graphbatch: 64 Z2-noise solves over 3 lattices x 2 Ls", "mf": mf, "link_eps": eps,
                      "seed": seed, "sloppy": args.sloppy, "tol": 1e-10,
                      "draw_counts": {"%dx%d_Ls%d" % (shapes[k][0][0], shapes[k][0][3], shapes[k][1]): int(np.sum(draws == k)) for k in range(len(shapes))}},
           "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "mean": float(np.mean(lat))},
           "fp64_latency_ms_first_%d" % len(lat64): {"p50": float(np.percentile(lat64, 50)), "p99": float(np.percentile(lat64, 99)),
                                                     "mean": float(np.mean(lat64))},
           "mixed_latency_ms_first_%d" % len(lat64): {"mean": float(np.mean(lat[:len(lat64)]))},
           "iterations": {"min": int(min(its)), "max": int(max(its))}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="24^3x64_Ls10", choices=sorted(WORKLOADS) + list(MODES))
    ap.add_argument("--group", type=int, default=3, help="batch32: right-hand sides per multi-RHS launch")
    ap.add_argument("--fp64-solves", type=int, default=16, help="graphbatch: solves repeated with plain FP64")
    ap.add_argument("--sloppy", default="f16", choices=["f16", "bf16", "f32", "i16", "f64", "f64e"],
                    help="inner storage of the mixed solve; with --kernel-only the kernel's precision "
                         "(f64: FP64, f64e: FP64 storage with emulated-FP64 hops)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--kernel-launches", type=int, default=20)
    ap.add_argument("--ref-budget", type=float, default=8.0)
    ap.add_argument("--kernel-only", action="store_true",
                    help="only launch the fused hop + M5^-1 kernel a few times (for ncu captures)")
    ap.add_argument("--op", default="HOP_OE_M5INV")
    ap.add_argument("--nrhs", type=int, default=1, help="kernel-only: right-hand sides per launch")
    ap.add_argument("--print-hash", action="store_true", help="print the kernel-source hash and exit")
    args = ap.parse_args()
    wl = args.workload
    if args.print_hash:
        print(kernel_sources_hash())
        return
    if args.impl == "reference":
        if wl in MODES:
            wl = {"batch32": "32^3x64_Ls12", "large48": "48^3x96_Ls8", "graphbatch": "16^3x32_Ls12",
                  "multirhs": "16^3x32_Ls12"}[wl]
        return run_reference(args, wl)
    if wl in MODES:
        return {"batch32": mode_batch32, "large48": mode_large48, "graphbatch": mode_graphbatch,
                "multirhs": mode_multirhs}[wl](args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    __graft_entry__.build()
    import inputs
    import paper_1810_01609_gb300 as m

    dims, Ls, mf, eps, seed = WORKLOADS[wl]
    X, Y, Z, T = dims
    V = X * Y * Z * T
    U = inputs.gauge_links(dims, eps, seed)
    ctx = m.Context(dims, Ls, mf=mf)
    ctx.load_gauge(U)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)   # graphs cannot be captured on the legacy default stream
    if args.kernel_only:
        return kernel_only(args, m, ctx, dims, Ls, seed, stream)
    b4 = torch.from_numpy(inputs.point_source4d(dims, 0, 0)).cuda().reshape((1,) + ctx.shape4d())

    def step(b4d, sloppy):
        eta = ctx.make_source_4d(b4d, nrhs=1, stream=stream)
        x, info = ctx.solve(eta[0], sloppy=sloppy, tol=1e-10, stream=stream)
        q = ctx.project_4d(x.reshape((1,) + x.shape), nrhs=1, stream=stream)
        return q, info

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(b4, args.sloppy)
    barrier()
    # where the timed region starts in a kernel launch list (the library's own launches;
    # a profiler also counts the framework's few fills and copies)
    print("library launches before the timed region: %d" % ctx.launch_count(), file=sys.stderr)
    sampler = ClockSampler(local)
    sampler.start()
    bytes0, launches0 = ctx.algorithmic_bytes(), ctx.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        q, info = step(b4, args.sloppy)
        infos.append(info)
    e1.record(stream)
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    step_bytes = (ctx.algorithmic_bytes() - bytes0) / args.steps
    launches = ctx.launch_count() - launches0
    ms_step, value = replica_aggregate(ms / args.steps, step_bytes, dist, device="cuda")

    # plain FP64 solve of the same source (same accuracy): one untimed solve (the FP64
    # kernels tune on first use), then the timed one
    fp64 = None
    if not args.no_fp64:
        eta = ctx.make_source_4d(b4, nrhs=1, stream=stream)
        # a short FP64 solve first: the FP64 kernels tune on first use (untimed)
        ctx.solve(eta[0], sloppy="f64", tol=1e-10, maxiter=30, check_interval=10, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x64, i64 = ctx.solve(eta[0], sloppy="f64", tol=1e-10, full_residual=True, stream=stream)
        torch.cuda.synchronize()
        fp64 = {"ms": (time.perf_counter() - t0) * 1e3, "iterations": i64.iterations,
                "true_residual": i64.true_residual, "full_residual": i64.full_residual}
        del x64

    # roofline leg: the fused hop + M5^-1 kernel (F16) timed alone, L2 flushed before each launch
    prec = m.PRECS[args.sloppy]
    nb = ctx.field_bytes(args.sloppy, 1)
    fin = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    fout = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    src = torch.from_numpy(inputs.gaussian_spinor5d(dims, Ls, seed + 100)).cuda()
    m.mdwf_pack(ctx.h, src, fin, prec, 1, stream)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    op = m.OP["HOP_OE_M5INV"]
    for _ in range(3):
        m.mdwf_apply(ctx.h, op, prec, fin, fout, 1, stream)
    kt = []
    for _ in range(args.kernel_launches):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        m.mdwf_apply(ctx.h, op, prec, fin, fout, 1, stream)
        b.record(stream)
        b.synchronize()
        kt.append(a.elapsed_time(b))
    kms = float(np.mean(kt))
    # the configuration the autotuner chose for this kernel (sites per CTA; flags 65536:
    # 64-register build, 131072: tensor-core kernel, 262144: paired-column kernel, 524288:
    # bulk-staged kernel)
    rk = [(k, v) for k, v, _ in ctx.tune_entries()
          if k.startswith("hop|") and k.endswith("|p%d|epi2000" % prec) and "|n1|" in k]
    roof_cfg = {"tune_key": rk[0][0], "tune_value": rk[0][1]} if rk else None
    vh = V // 2
    site = {"f16": 52.0, "bf16": 48.0, "f32": 96.0, "i16": 52.0, "f64": 192.0, "f64e": 192.0}[args.sloppy]
    link = {"f16": 2, "bf16": 2, "f32": 4, "i16": 2, "f64": 8, "f64e": 8}[args.sloppy] * 18.0
    kbytes = vh * Ls * 2 * site + vh * 8 * link
    peak, peak_kind = peaks()
    achieved = kbytes / (kms * 1e-3) / 1e9
    del flush

    # end to end through the public API with HOST buffers: mdwf_propagator takes the pinned
    # 4D source, copies it in, injects, solves and projects on the device and copies the
    # 4D propagator column back (the 5D source and solution never leave the device)
    b4h = b4.cpu().pin_memory()
    q_h = torch.empty((1,) + ctx.shape4d(), dtype=torch.complex128).pin_memory()
    sp_e2e = ctx.solve_params(tol=1e-10, sloppy=args.sloppy)

    def step_host():
        return m.mdwf_propagator(ctx.h, 1, b4h, q_h, sp_e2e, stream)[0]

    step_host()   # the context's host-path staging buffers are allocated here
    torch.cuda.synchronize()
    ee0, ee1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_bytes0 = ctx.algorithmic_bytes()
    ee0.record(stream)
    for _ in range(args.steps):
        ih = step_host()
    ee1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = ee0.elapsed_time(ee1) / args.steps
    e2e_val = world * (ctx.algorithmic_bytes() - e2e_bytes0) / args.steps / (e2e_ms * 1e-3) / 1e9
    b4b = b4h.numel() * 16
    # the same pinned 4D buffer copied by torch alone, both ways: the link's own speed
    dtmp = torch.empty_like(q_h, device="cuda")
    c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    c0.record(stream)
    dtmp.copy_(q_h, non_blocking=True)
    c1.record(stream)
    q_h.copy_(dtmp, non_blocking=True)
    c2.record(stream)
    torch.cuda.synchronize()
    pinned_gbs = {"h2d": b4b / (c0.elapsed_time(c1) * 1e-3) / 1e9, "d2h": b4b / (c1.elapsed_time(c2) * 1e-3) / 1e9}
    del dtmp
    e2e_h2d = b4b      # the 4D source
    e2e_d2h = b4b      # the 4D propagator column

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        g1, d1, _ = cpu_oracle(dims, Ls, mf, eps, seed, args.ref_budget, 1)
        cores = min(16, host_cores())
        ga, da, wa = cpu_oracle(dims, Ls, mf, eps, seed, args.ref_budget, cores)
        ts, tits = oracle_smallest_solve_s()
        cpu = {"value": ga, "unit": "GB/s", "cores": wa, "host_cores_available": host_cores(), "kind": "oracle",
               "sample": da + "; GB/s = the GPU step's algorithmic bytes per CG iteration x iterations / time",
               "single_core": {"value": g1, "unit": "GB/s", "cores": 1, "sample": d1},
               "oracle_solve_4^4_Ls8_s": ts, "oracle_solve_4^4_Ls8_iterations": tits}

    mixed_ms = float(np.mean([i.time_ms for i in infos]))
    out = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 arithmetic on f16 storage (inner CG); f64 reliable updates and reductions",
        "data": "synthetic",
        "config": {"workload": wl, "lattice": list(dims), "Ls": Ls, "mf": mf, "b5": 1.5, "c5": 0.5, "M5": 1.3,
                   "link_eps": eps, "seed": seed, "source": "point (spin 0, colour 0, origin)",
                   "sloppy": args.sloppy, "tol": 1e-10,
                   "l2": "step working set > L2; roofline kernel launches preceded by a 512 MB L2 flush",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "solve": {"mixed_ms": mixed_ms, "iterations": infos[-1].iterations,
                  "reliable_updates": infos[-1].reliable_updates, "fp64_residuals": infos[-1].fp64_residuals,
                  "emulated_fp64_residuals": infos[-1].emulated_residuals,
                  "true_residual": infos[-1].true_residual,
                  "fp64_ms": fp64["ms"] if fp64 else None, "fp64_iterations": fp64["iterations"] if fp64 else None,
                  "fp64_true_residual": fp64["true_residual"] if fp64 else None,
                  "fp64_full_residual": fp64["full_residual"] if fp64 else None,
                  "speedup_vs_fp64": (fp64["ms"] / mixed_ms) if fp64 else None},
        "roofline": {"kernel": "fused hop + M5^-1 (HOP_OE_M5INV, %s)" % args.sloppy, "bound": "hbm",
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": stored_traffic("%s/HOP_OE_M5INV/%s" % (wl, args.sloppy),
                                                              roof_cfg["tune_value"] if roof_cfg else None),
                     "bytes_per_launch": kbytes, "ms_per_launch": kms, "launch_config": roof_cfg},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "GB/s", "ms_per_step": e2e_ms,
                "path": "mdwf_propagator (injection, solve, projection in one C-ABI call) with pinned HOST 4D source and propagator",
                "true_residual": ih.true_residual,
                "h2d_bytes_per_step": int(e2e_h2d), "d2h_bytes_per_step": int(e2e_d2h),
                "pinned_copy_gbs_torch": pinned_gbs},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
