"""Benchmark: EPRL vertex shells/s on one GB300 (and N GPUs by weak scaling).

Workload (the homogeneous scaling sweep): sixteen vertices with all ten boundary spins
j = lambda/2, lambda = 1..16, gamma = 1.2, dl = 10 (11^6 = 1,771,561 shells each), rapidity rule
r_max = 40, 40 panels x 50 Gauss-Legendre nodes. One step runs the whole path through the C ABI:
{6j} tables, d-tables and boosters of all sixteen vertices, then the shell sum over one slice of
every vertex (the same 1/S range of its group-major shell index), so S consecutive steps cover the
sweep exactly once. Ranks of a multi-GPU run take different slices (weak scaling, no collective on
the data path).

Prints one JSON line (rank 0). ``--impl reference`` times the CPU oracle on a bounded sample of
the same workload instead.
"""
import argparse
import hashlib
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

RULE = (40.0, 40, 50)
METRIC = "EPRL vertex shells/sec (mixed vs FP64 GPU path) at stated relative error"


def workload_name(slices):
    return ("homogeneous sweep: 16 vertices, all spins j=lambda/2 for lambda=1..16, gamma=1.2, dl=10 (11^6 shells "
            "each), rule r_max=40 / 40 panels x 50 nodes; one step = 6j tables + d-tables + boosters of all 16 "
            "vertices + shell sum over a 1/%d slice of every vertex's group-major shell range" % slices)
SWEEP = [(lam, 10) for lam in range(1, 17)]
GAMMA = 1.2
# FP64 FMA pipe of the GB300: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.070 GHz (max SM clock)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# FP32 pipe: 152 SMs x 128 lanes x 2.070 GHz, in lane operations (FFMA, FADD, FMUL) per second
FP32_PEAK_TOPS = 152 * 128 * 2.070e9 / 1e12
PRECISIONS = {"fp64": 0, "mixed": 1, "mixed_ff": 2}
# FP32 lane operations per multiply-add of the compensated-pair phases (SF_MIXED_FF): D is a Dot2
# step with a pair times a float (FMUL, 2 FFMA, TwoSum = 6, 2 FADD), F a pair times a pair (one
# more FFMA); the FP32 booster phases take one FFMA per multiply-add
FF_OPS = {"D": 11, "F": 12}
# DRAM bytes (read + write) of the benchmark's shell-sum launch from one ncu capture (the first timed
# launch, slice 3 of the sweep; profiles/k_shell_mixed_ff_sweep_traffic.md), valid while the kernel
# source hashes to "sha1"
NCU_TRAFFIC = {"sha1": "77e3c11e9e92", "bytes_per_launch": {"mixed_ff": 32906166784 + 118807808, "mixed": None, "fp64": None}}


def kernel_sha1():
    """sha1 prefix of the shell kernel's source: sf_shell.cu up to its host-side launchers (the
    kernel and the device helpers it uses)."""
    p = os.path.join(ROOT, "paper_2107_13952_gb300", "csrc", "sf_shell.cu")
    src = open(p, "rb").read()
    cut = src.find(b"int sf_shell_prepare(")
    return hashlib.sha1(src[:cut] if cut > 0 else src).hexdigest()[:12]


# ------------------------------------------------------------------------------------------
# executed FP64 FMA count of the shell-sum kernel (trip counts of its loops), for the roofline
# ------------------------------------------------------------------------------------------
def _pair(a, b, c, d):
    import numpy as np
    a, b, c, d = np.broadcast_arrays(a, b, c, d)
    lo = np.maximum(np.abs(a - b), np.abs(c - d))
    hi = np.minimum(a + b, c + d)
    n = np.where(((a + b + c + d) % 2 == 0) & (hi >= lo), (hi - lo) // 2 + 1, 0)
    return lo, n


def executed_fmas(tj, dl, g0, g1):
    """FMAs the shell kernel executes for groups [g0, g1) of one vertex (all tiles), per phase."""
    import numpy as np
    from paper_2107_13952_gb300 import intertwiner_ranges
    lo, dim = intertwiner_ranges(tj, GAMMA, dl)
    D = dl + 1
    j12, j13, j14, j15, j23, j24, j25, j34, j35, j45 = tj
    d = np.arange(D)
    # axes: 0 d25, 1 d35, 2 d45, 3 d24, 4 d34, 5 d23
    sh = [1] * 6

    def ax(i):
        s = list(sh)
        s[i] = D
        return d.reshape(s)
    l25, l35, l45, l24, l34, l23 = (j25 + 2 * ax(0), j35 + 2 * ax(1), j45 + 2 * ax(2), j24 + 2 * ax(3),
                                    j34 + 2 * ax(4), j23 + 2 * ax(5))
    k5lo, nk5 = _pair(j15, l25, l35, l45)
    k4lo, nk4 = _pair(l45, j14, l24, l34)
    k2lo, nk2 = _pair(l23, l24, l25, j12)
    k3lo, nk3 = _pair(l34, l35, j13, l23)
    valid = (nk2 > 0) & (nk3 > 0)
    nk3v = np.where(valid, nk3, 0)
    nk2v = np.where(valid, nk2, 0)
    k3lo_v = np.where(valid, k3lo, 10 ** 6)
    k3hi_v = np.where(valid, k3lo + 2 * (nk3 - 1), -1)
    shape5 = (D, D, D, D, D)
    k3u = np.broadcast_to((k3hi_v.max(axis=5) - k3lo_v.min(axis=5)) // 2 + 1, shape5)
    anyv = np.broadcast_to(valid.any(axis=5), shape5)
    sum_nk3 = np.broadcast_to(nk3v.sum(axis=5), shape5)
    sum_nk3nk2 = np.broadcast_to((nk3v * nk2v).sum(axis=5), shape5)
    nk5b = np.broadcast_to(nk5[..., 0], shape5)
    nk4b = np.broadcast_to(nk4[..., 0], shape5)
    k5lob = np.broadcast_to(k5lo[..., 0], shape5)
    k4lob = np.broadcast_to(k4lo[..., 0], shape5)
    l25b = np.broadcast_to(l25[..., 0], shape5)
    l35b = np.broadcast_to(l35[..., 0], shape5)
    gidx = (np.arange(D)[:, None, None] * D + np.arange(D)[None, :, None]) * D + np.arange(D)[None, None, :]
    gmask = np.broadcast_to(((gidx >= g0) & (gidx < g1))[..., None, None], shape5)
    di3, di4, di5 = dim[2], dim[3], dim[4]
    total = {k: 0 for k in "BCDFGH"}
    k5hi = k5lob + 2 * (nk5b - 1)
    k4hi = k4lob + 2 * (nk4b - 1)

    def mind(c, lo_, hi_):
        return np.where(c < lo_, lo_ - c, np.where(c > hi_, c - hi_, (c + lo_) % 2))
    xlo_b = mind(j14, k5lob, k5hi)
    xlo_c = mind(l35b, k4lob, k4hi)
    for ci1 in range(dim[0]):
        i1 = lo[0] + 2 * ci1
        xlo = np.maximum(np.abs(i1 - l25b), np.maximum(xlo_b, xlo_c))
        xhi = np.minimum(i1 + l25b, np.minimum(k5hi + j14, k4hi + l35b))
        xlo = xlo + ((xlo - np.abs(i1 - l25b)) % 2)
        nx = np.where(xhi >= xlo, (xhi - xlo) // 2 + 1, 0)
        live = gmask & anyv & (nk5b > 0) & (nk4b > 0) & (nx > 0)
        for name, per5 in (("B", sum_nk3nk2 * nx), ("C", nx * di3 * sum_nk3), ("D", nk4b * nx * di3 * k3u),
                           ("F", nk4b * nk5b * di3 * nx), ("G", di4 * nk5b * di3 * nk4b)):
            total[name] += int(np.where(live, per5, 0).sum())
    # H: once per group with a non-empty k5 range
    g_live = ((gidx >= g0) & (gidx < g1)) & (nk5[..., 0, 0, 0] > 0)
    total["H"] += int(dim[0] * np.where(g_live, di4 * di5 * di3 * nk5[..., 0, 0, 0], 0).sum())
    return {k: v * dim[1] for k, v in total.items()}


FP32_PHASES_MIXED = ("B", "C", "G")   # booster contractions the mixed paths run in FP32


def pipe_ops(phases, precision):
    """(FP64 flops, FP32 lane ops) the shell kernel executes for a phase count dict."""
    f64, f32 = 0, 0
    for name, n in phases.items():
        if precision != "fp64" and name in FP32_PHASES_MIXED:
            f32 += n
        elif precision == "mixed_ff" and name in FF_OPS:
            f32 += FF_OPS[name] * n
        else:
            f64 += 2 * n
    return f64, f32


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ------------------------------------------------------------------------------------------
def _oracle_worker(args):
    seed, deadline, lam_list = args
    import numpy as np
    from oracle import vertex as ov
    from oracle import wigner as ow
    rng = np.random.default_rng(seed)
    done = 0
    cache = {}
    six = ov.SixJCache()
    while time.time() < deadline:
        lam = int(lam_list[rng.integers(0, len(lam_list))])
        tj, dl = (lam,) * 10, 10
        if lam not in cache:
            bs = {}
            D = dl + 1
            for e in (2, 3, 4, 5):
                di = len(ow.pair_range(*ov.edge_spins(tj, tuple(tj[4:]))[e][0]))
                klo = np.zeros(D ** 3, dtype=np.int64)
                nk = np.zeros(D ** 3, dtype=np.int64)
                for t in range(D ** 3):
                    dd = (t // (D * D), (t // D) % D, t % D)
                    tl6 = dict(zip(ov.FREE, [tj[ov.FACES.index(f)] for f in ov.FREE]))
                    for f, df in zip(ov.EDGE_TRIPLES[e], dd):
                        tl6[f] += 2 * df
                    kr = ow.pair_range(*ov.edge_spins(tj, tuple(tl6[f] for f in ov.FREE))[e][1])
                    klo[t] = kr[0] if kr else 0
                    nk[t] = len(kr)
                bs[e] = {"B": rng.standard_normal((D ** 3, di, max(1, int(nk.max())))), "klo": klo}
            cache[lam] = bs
        s = int(rng.integers(0, (dl + 1) ** 6))
        ov.shell_contribution(tj, dl, s, cache[lam], six)
        done += 1
    return done


def oracle_rate(seconds, seed=0):
    """Oracle shell-sum throughput (shells/s) on all host cores for `seconds` of wall time."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    lam_list = [lam for lam, _ in SWEEP]
    ctx = mp.get_context("spawn")
    t0 = time.time()
    deadline = t0 + seconds
    with ctx.Pool(cores) as pool:
        counts = pool.map(_oracle_worker, [(seed * 1000 + i, deadline, lam_list) for i in range(cores)])
    el = time.time() - t0
    n = sum(counts)
    return n / el, cores, n, el


# ------------------------------------------------------------------------------------------
def batched_measure(shells, steps=3):
    """The batched workload: 256 irregular vertices (ten spins uniform in {1/2..6}, redrawn until all
    five intertwiner ranges are non-empty; dl uniform in 0..12; gamma from {0.1, 1.2, 5.0}; seed 0),
    the first ``shells`` shells of every vertex, as one planned launch (persistent shell kernel +
    one reduction) replayed as a CUDA graph, tiling autotuned on a sample, in both precisions."""
    import torch
    import paper_2107_13952_gb300 as sf
    from paper_2107_13952_gb300 import inputs
    batch = inputs.random_batch(256, seed=0)
    t = sf.sf_6j_table([sf.vertex(b["two_j"], b["gamma"], b["dl"]) for b in batch])
    sf.sf_boosters(t, RULE)
    n = sum(min(shells, (b["dl"] + 1) ** 6) for b in batch)
    stream = torch.cuda.current_stream()
    res, outs = {}, {}
    for name, prec in PRECISIONS.items():
        plan = sf.Plan(t, prec, 0, shells)
        tiling = plan.autotune(min(shells, 2048))
        plan.graph_launch()
        plan.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            plan.graph_launch()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        res[name] = {"value": n / (ms / 1e3), "unit": "shells/s", "ms_per_launch": ms,
                     "tiling": {"x_chunk": tiling[0], "items_per_sm": tiling[1]}}
        outs[name] = [o.clone() for o in plan.outputs]
        del plan
    den = sum(float(b.norm()) ** 2 for b in outs["fp64"]) ** 0.5
    errs = {}
    for name in ("mixed", "mixed_ff"):
        num = sum(float((a - b).norm()) ** 2 for a, b in zip(outs[name], outs["fp64"])) ** 0.5
        errs[name] = num / den if den > 0 else None
    return {"workload": "256 irregular vertices (spins 1/2..6, dl 0..12, gamma 0.1/1.2/5.0, seed 0), shells "
                        "[0, %d) of every vertex, %d shells in all; one CUDA-graph replay of a planned launch "
                        "per step, %d steps; tables and boosters built once before the replays (not flushed "
                        "between them)" % (shells, n, steps),
            "fp64": res["fp64"], "mixed": res["mixed"], "mixed_ff": res["mixed_ff"],
            "rel_err_vs_fp64": errs}


def other_workloads(large_fraction=32):
    """The two remaining workloads, timed once each after a warm-up (CUDA events):
    * spin 4, gamma 1.2, dl 20 (21^6 = 85,766,121 shells): the first 1/large_fraction of its
      group-major shell range in the pair path and the FP64 path, and the relative error between them;
    * spin 3, gamma 1.2, dl 8 (9^6 shells): the boundary-contracted amplitude and its gradients with
      respect to the five seeded boundary vectors and the four booster tensors (adjoint kernels)."""
    import torch
    import paper_2107_13952_gb300 as sf
    from paper_2107_13952_gb300 import inputs
    stream = torch.cuda.current_stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    res = {}
    w = inputs.large_shell()
    t = sf.sf_6j_table([sf.vertex(w["two_j"], w["gamma"], w["dl"])])
    sf.sf_boosters(t, RULE)
    D = w["dl"] + 1
    end = (D ** 3 // large_fraction) * D ** 3
    lg = {"workload": "all spins 4, gamma 1.2, dl 20: shells [0, %d) of 85,766,121 (group-major)" % end}
    outs = {}
    for name, p in (("mixed_ff", sf.SF_MIXED_FF), ("fp64", sf.SF_FP64)):
        ms, o = timed(lambda: sf.sf_vertex_amplitude(t, p, 0, end)[0].clone())
        lg[name] = {"value": end / (ms / 1e3), "unit": "shells/s", "ms": ms}
        outs[name] = o
    lg["mixed_ff_vs_fp64_rel_err"] = float((outs["mixed_ff"] - outs["fp64"]).norm() / outs["fp64"].norm())
    res["large_shell"] = lg
    del t
    w = inputs.boundary_contraction_vertex()
    t = sf.sf_6j_table([sf.vertex(w["two_j"], w["gamma"], w["dl"])])
    sf.sf_boosters(t, RULE)
    dims = sf.intertwiner_ranges(w["two_j"], w["gamma"], w["dl"])[1]
    psis = [torch.tensor(v, dtype=torch.complex128, device="cuda") for v in inputs.boundary_vectors(dims)]
    n = (w["dl"] + 1) ** 6
    ms, _ = timed(lambda: sf.sf_vertex_adjoint(t, psis, want_grads=True))
    res["adjoint"] = {"workload": "all spins 3, gamma 1.2, dl 8 (531,441 shells): contracted amplitude and "
                                  "gradients w.r.t. five boundary vectors and four booster tensors, FP64",
                      "value": n / (ms / 1e3), "unit": "shells/s", "ms": ms}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed_ff", choices=list(PRECISIONS),
                    help="path timed for `value`; the other paths are timed for one step beside it")
    ap.add_argument("--slices", type=int, default=16, help="steps per full pass over the sweep")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched-shells", type=int, default=16384,
                    help="shells per vertex of the 256-vertex batched measurement (0: skip)")
    ap.add_argument("--case", default=None, help="lambda:groups:precision -- one shell-sum launch (profiling)")
    ap.add_argument("--no-other-workloads", action="store_true", help="skip the spin-4 dl-20 and adjoint timings")
    args = ap.parse_args()

    if args.case:
        # one shell-sum launch on a small range of one vertex (for profiler captures)
        import torch
        import paper_2107_13952_gb300 as sf
        lam, ngroups, p = (int(v) for v in args.case.split(":"))
        t = sf.sf_6j_table([sf.vertex((lam,) * 10, GAMMA, 10)])
        sf.sf_boosters(t, RULE)
        A = sf.sf_vertex_amplitude(t, p, 0, ngroups * 11 ** 3)[0]
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "norm": float(A.norm()), "kernel_ms": sf.last_kernel_ms()}))
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    total_shells_per_vertex = 11 ** 6

    if args.impl == "reference":
        if rank != 0:
            return
        rates = []
        n_all, t_all = 0, 0.0
        for i in range(args.warmup + args.steps):
            r, cores, n, el = oracle_rate(max(2.0, args.cpu_seconds / max(1, args.steps)), seed=i)
            if i >= args.warmup:
                rates.append(r)
                n_all += n
                t_all += el
        value = n_all / t_all
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "shells/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * t_all / max(1, args.steps), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload_name(args.slices), "slices_per_pass": args.slices,
                           "sample": "the CPU oracle's shell-sum phase on %d shells drawn uniformly from the sweep "
                                     "(boosters random), on all host cores" % n_all},
                "cpu_baseline": {"value": value, "unit": "shells/s", "cores": cores, "kind": "oracle",
                                 "sample": "%d shells drawn uniformly from the sweep's %d shells, boosters "
                                           "random (shell-sum phase only)" % (n_all, 16 * total_shells_per_vertex)},
                "e2e": {"value": value, "unit": "shells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    import paper_2107_13952_gb300 as sf
    sf.load()
    prec = PRECISIONS[args.precision]
    verts = [sf.vertex((lam,) * 10, GAMMA, dl) for lam, dl in SWEEP]
    dims = [sf.intertwiner_ranges((lam,) * 10, GAMMA, dl)[1] for lam, dl in SWEEP]
    S = args.slices
    N = total_shells_per_vertex
    G = 11 ** 3
    outs = [torch.empty(d, dtype=torch.float64, device="cuda") for d in dims]
    host = [torch.empty(d, dtype=torch.float64, pin_memory=True) for d in dims]
    stream = torch.cuda.current_stream()

    def slice_bounds(k):
        g0, g1 = G * k // S, G * (k + 1) // S
        return g0 * 121 * 11, g1 * 121 * 11, g0, g1

    def step(k, to_host, p=None):
        b, e, _, _ = slice_bounds(k % S)
        t = sf.sf_6j_table(verts)
        sf.sf_boosters(t, RULE)
        sf.sf_vertex_amplitude(t, prec if p is None else p, b, e, out=outs)
        kms = sf.last_kernel_ms()
        if to_host:
            for o, h in zip(outs, host):
                h.copy_(o, non_blocking=True)
        del t
        return kms, 16 * (e - b)

    def barrier():
        if world > 1:
            dist.barrier()

    # warm-up
    for i in range(args.warmup):
        step(i * world + rank, False)
    torch.cuda.synchronize()

    def timed(to_host, first):
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        kms_all, shells, slices = [], 0, []
        launches0 = sf.kernel_launches()
        e0.record(stream)
        for i in range(args.steps):
            k = (first + i) * world + rank
            kms, n = step(k, to_host)
            kms_all.append(kms)
            shells += n
            slices.append(k % S)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        return ms, kms_all, shells, slices, sf.kernel_launches() - launches0

    clk = ClockSampler(local)
    clk.start()
    ms, kms_all, shells, slices, launches = timed(False, args.warmup)
    clocks = clk.stop()
    ms_e2e, _, shells_e2e, _, _ = timed(True, args.warmup + args.steps)

    # every path on one slice, timed the same way (one warm step each), and the relative error of
    # the mixed paths against the FP64 path on that slice
    kk = (args.warmup + 2 * args.steps) * world + rank
    others, res_slice = {}, {}
    for name, p in PRECISIONS.items():
        step(kk, False, p)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        kms_o, n_o = step(kk, False, p)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_o = e0.elapsed_time(e1)
        res_slice[name] = [o.clone() for o in outs]
        if name != args.precision:
            others[name] = {"value": n_o * world / (ms_o / 1e3), "unit": "shells/s", "ms_per_step": ms_o,
                            "kernel_ms_per_step": kms_o}
    den = sum(float(r.norm()) ** 2 for r in res_slice["fp64"]) ** 0.5
    rel_err = {}
    for name in ("mixed", "mixed_ff"):
        num = sum(float((o - r).norm()) ** 2 for o, r in zip(res_slice[name], res_slice["fp64"])) ** 0.5
        rel_err[name] = num / den if den > 0 else None
    # the same per vertex (per lambda), for both mixed paths
    rel_err_per_lambda = {}
    for name in ("mixed", "mixed_ff"):
        per = {}
        for (lam, _), o, r in zip(SWEEP, res_slice[name], res_slice["fp64"]):
            rn = float(r.norm())
            per[str(lam)] = float((o - r).norm()) / rn if rn > 0 else None
        rel_err_per_lambda[name] = per

    # max over ranks
    if world > 1:
        tm = torch.tensor([ms, ms_e2e], device="cuda")
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        ms, ms_e2e = float(tm[0]), float(tm[1])
    total_shells = shells * world
    value = total_shells / (ms / 1e3)
    e2e_value = shells_e2e * world / (ms_e2e / 1e3)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel (the shell sum): executed FP64 flops / event-timed duration
    flops, ops32 = 0, 0
    for k in slices:
        _, _, g0, g1 = slice_bounds(k)
        for lam, dl in SWEEP:
            f64, f32 = pipe_ops(executed_fmas((lam,) * 10, dl, g0, g1), args.precision)
            flops += f64
            ops32 += f32
    kern_s = sum(kms_all) / 1e3
    fp64_tflops = flops / kern_s / 1e12 if kern_s > 0 else None
    fp32_tops = ops32 / kern_s / 1e12 if kern_s > 0 else None
    if args.precision == "mixed_ff":
        # the FP32 pipe carries the kernel: lane operations (FFMA, FADD, FMUL) per second
        roof = {"bound": "alu", "achieved": fp32_tops, "peak": FP32_PEAK_TOPS, "unit": "Tops/s (FP32 lane ops)",
                "frac": (fp32_tops / FP32_PEAK_TOPS) if fp32_tops else None,
                "ops_counted": "FP32 lane operations of the loops (compensated-pair steps at 11-12 operations per "
                               "multiply-add, FP32 booster contractions at one FFMA), trip counts x operations",
                "fp64_tflops": fp64_tflops, "fp64_frac": (fp64_tflops / FP64_PEAK_TFLOPS) if fp64_tflops else None}
    else:
        roof = {"bound": "alu", "achieved": fp64_tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": (fp64_tflops / FP64_PEAK_TFLOPS) if fp64_tflops else None,
                "flops_counted": "FP64-pipe FMAs the kernel executes x 2 (loop trip counts); the FP32 phases of the "
                                 "mixed path are reported separately",
                "fp32_tops": fp32_tops}
    traffic = None
    if NCU_TRAFFIC["sha1"] == kernel_sha1():
        traffic = NCU_TRAFFIC["bytes_per_launch"].get(args.precision)

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        r, cores, n, el = oracle_rate(args.cpu_seconds)
        cpu = {"value": r, "unit": "shells/s", "cores": cores, "kind": "oracle",
               "sample": "%d shells drawn uniformly from the sweep (%.1f s on %d processes), boosters random "
                         "(shell-sum phase only)" % (n, el, cores)}

    batched = None
    if args.batched_shells > 0 and world == 1:
        batched = batched_measure(args.batched_shells)
    others_w = None
    if not args.no_other_workloads and world == 1:
        others_w = other_workloads()

    d2h = sum(h.numel() * 8 for h in host)
    h2d = len(verts) * 56
    line = {
        "metric": METRIC,
        "value": value, "unit": "shells/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "mixed": "f64+f32", "mixed_ff": "f64+f32+f32x2"}[args.precision], "data": "synthetic",
        "config": {"workload": workload_name(S),
                   "slices_per_pass": S, "precision": args.precision,
                   "cache": "inputs larger than L2: every step rebuilds the {6j} tables, d-tables and boosters of "
                            "all 16 vertices (the spin-8 S3 table alone, FP64 plus pair copy, is 384 MB, 3x the "
                            "L2), so no step starts with its working set in L2; no separate flush"},
        "roofline": dict(roof, traffic=traffic, kernel="k_shell<%d>" % PRECISIONS[args.precision],
                         kernel_ms_per_step=1e3 * kern_s / args.steps),
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "shells/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clocks,
        "path": args.precision,
        "other_paths": others,
        "batched": batched,
        "other_workloads": others_w,
        "mixed_vs_fp64": {"rel_err": rel_err, "rel_err_per_lambda": rel_err_per_lambda, "stated_bound": 1e-6,
                          "metric": "||A_mixed - A_fp64|| / ||A_fp64|| over the 16 vertices of one slice"},
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
