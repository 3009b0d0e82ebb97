"""Benchmark: EPRL vertex shells/s on one GB300 (and N GPUs by weak scaling).

Workload (the homogeneous scaling sweep): sixteen vertices with all ten boundary spins
j = lambda/2, lambda = 1..16, gamma = 1.2, dl = 10 (11^6 = 1,771,561 shells each), rapidity rule
r_max = 40, 40 panels x 50 Gauss-Legendre nodes. One step runs the whole path through the C ABI:
the shell sum over one slice of every vertex (the same 1/S range of its group-major shell index)
together with the {6j} tables, d-tables and boosters that the slice's shells read (built for the
slice, as one process of a split sum builds its own), so S consecutive steps cover the sweep
exactly once. Shells are counted when they are non-empty (all four virtual-intertwiner
ranges non-empty); the count over the whole grid is reported beside. Ranks of a multi-GPU run take
different slices (weak scaling, no collective on the data path).

``value`` is the path whose precision split keeps the {6j} values exact-then-FP64, the {15j}
auxiliary-spin sum and every sum across shells in FP64 and runs the booster contractions in
FP32-class arithmetic with the k4 contraction on the tensor cores (SF_MIXED_TC); the FP64 path and
the other mixed paths (SF_MIXED; SF_MIXED_FF and SF_MIXED_PX, faster, with the {15j} x-sum in
compensated FP32 pairs, beyond that split) are timed over the same steps beside it, with their
errors against the FP64 path per lambda. The remaining workloads (all 256 irregular vertices in full, the spin-4 dl-20
vertex in full, the boundary-contracted adjoint, the spin-1 simplex, the vertex-tensor
contractions and the Delta_3 network) are timed after it.

Prints one JSON line (rank 0). ``--impl reference`` times the CPU oracle on a bounded sample of
the same workload instead.
"""
import argparse
import ctypes
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
SWEEP = [(lam, 10) for lam in range(1, 17)]
GAMMA = 1.2
CLOCK_GHZ = 2.070
# FP64 FMA pipe of the GB300: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.070 GHz (max SM clock)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * CLOCK_GHZ / 1e3
# FP32 pipe: 152 SMs x 128 lanes x 2.070 GHz, in lane operations (FFMA, FADD, FMUL) per second
FP32_PEAK_TOPS = 152 * 128 * CLOCK_GHZ / 1e3
PRECISIONS = {"fp64": 0, "mixed": 1, "mixed_ff": 2, "mixed_tc": 3, "mixed_px": 4}
DTYPES = {"fp64": "f64", "mixed": "f64+f32", "mixed_ff": "f64+f32+f32x2", "mixed_tc": "f64+f32+bf16x3",
          "mixed_px": "f64+f32+f32x2"}
HEADLINE = "mixed_tc"
# precision split of each path: phases B (k2), C (l23 sum with B3), D (k3 with S3), F (x-sum),
# G (k4 with B4), H (k5 with B5); "64" FP64, "32" FP32 CUDA cores, "ff" compensated pairs, "tc"
# tensor cores (split BF16)
PHASE_PRECISION = {"fp64": dict(B="64", C="64", D="64", F="64", G="64", H="64"),
                   "mixed": dict(B="32", C="32", D="64", F="64", G="32", H="64"),
                   "mixed_ff": dict(B="32", C="32", D="ff", F="ff", G="32", H="64"),
                   "mixed_tc": dict(B="32", C="32", D="32", F="64", G="tc", H="64"),
                   "mixed_px": dict(B="32", C="32", D="32", F="ffd", G="32", H="64")}
# FP32 lane operations per multiply-add of the pair phases: "ff" pair x float (D) or pair x pair
# (F), "ffd" pair x float
FF_OPS = {"D": 11, "F": 12}
FFD_OPS = 11
# DRAM bytes (read + write) of the headline path's shell-sum launches of one step (the step's two
# launch classes) from one ncu capture of the benchmark's first timed step after three warm-up
# steps (slice 3 of 32), valid while the kernel source hashes to "sha1"
NCU_TRAFFIC = {"sha1": "0cf314fbb99f", "bytes_per_step": 329967360 + 90086912 + 507539200 + 30302720}


def workload_name(slices):
    return ("homogeneous sweep: 16 vertices, all spins j=lambda/2 for lambda=1..16, gamma=1.2, dl=10 (11^6 shells "
            "each), rule r_max=40 / 40 panels x 50 nodes; one step = shell sum over a 1/%d slice of every vertex's "
            "group-major shell range with the 6j tables, d-tables and boosters the slice reads, built in the step"
            % slices)


def kernel_sha1():
    """sha1 prefix of the shell kernel's source: sf_shell.cu up to its host-side launchers."""
    p = os.path.join(ROOT, "paper_2107_13952_gb300", "csrc", "sf_shell.cu")
    src = open(p, "rb").read()
    cut = src.find(b"int sf_shell_prepare(")
    return hashlib.sha1(src[:cut] if cut > 0 else src).hexdigest()[:12]


# ------------------------------------------------------------------------------------------
# shell bookkeeping on the host (numpy): non-empty shells, executed and canonical operation counts
# ------------------------------------------------------------------------------------------
from paper_2107_13952_gb300.shells import _pair, _shell_axes, canonical_flops, nonempty_shells  # noqa: E402


def executed_fmas(tj, dl, g0, g1):
    """Multiply-adds the shell kernel executes for groups [g0, g1) of one vertex (all tiles), per
    phase (trip counts of its loops)."""
    import numpy as np
    from paper_2107_13952_gb300 import intertwiner_ranges
    lo, dim = intertwiner_ranges(tj, GAMMA, dl)
    D = dl + 1
    j12, j13, j14, j15 = tj[:4]
    l25, l35, l45, l24, l34, l23 = _shell_axes(tj, dl)
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
    g_live = ((gidx >= g0) & (gidx < g1)) & (nk5[..., 0, 0, 0] > 0)
    total["H"] += int(dim[0] * np.where(g_live, di4 * di5 * di3 * nk5[..., 0, 0, 0], 0).sum())
    return {k: v * dim[1] for k, v in total.items()}


def pipe_ops(phases, precision):
    """(FP64 flops, FP32 lane ops, tensor-core multiply-adds before padding) of a phase count."""
    f64, f32, tc = 0, 0, 0
    for name, n in phases.items():
        p = PHASE_PRECISION[precision][name]
        if p == "64":
            f64 += 2 * n
        elif p == "32":
            f32 += n
        elif p == "ff":
            f32 += FF_OPS[name] * n
        elif p == "ffd":
            f32 += FFD_OPS * n
        else:
            tc += n
    return f64, f32, tc


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
        if ov.shell_contribution(tj, dl, s, cache[lam], six) is not None:   # count non-empty shells
            done += 1
    return done


def oracle_rate(seconds, seed=0):
    """Oracle shell-sum throughput (non-empty shells/s) on all host cores for `seconds` of wall time."""
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
# the other workloads
# ------------------------------------------------------------------------------------------
def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def batched_measure(precisions):
    """All 256 irregular vertices (ten spins uniform in {1/2..6}, redrawn until all five
    intertwiner ranges are non-empty; dl uniform in 0..12; gamma from {0.1, 1.2, 5.0}; seed 0), every
    shell of every vertex, as one planned launch (persistent shell kernel + one reduction) replayed
    as a CUDA graph, tiling autotuned on the first 2048 shells of every vertex."""
    import torch
    import paper_2107_13952_gb300 as sf
    from paper_2107_13952_gb300 import inputs
    batch = inputs.random_batch(256, seed=0)
    t = sf.sf_6j_table([sf.vertex(b["two_j"], b["gamma"], b["dl"]) for b in batch])
    sf.sf_boosters(t, RULE)
    n_all = sum((b["dl"] + 1) ** 6 for b in batch)
    n_ne = int(sum(int(nonempty_shells(b["two_j"], b["dl"]).sum()) for b in batch))
    stream = torch.cuda.current_stream()
    res, outs = {}, {}
    for name in precisions:
        plan = sf.Plan(t, PRECISIONS[name])
        tiling = plan.autotune(2048)
        plan.graph_launch()
        plan.sync()
        e0, e1 = _events()
        e0.record(stream)
        plan.graph_launch()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        res[name] = {"value": n_ne / (ms / 1e3), "unit": "non-empty shells/s", "all_shells_per_s": n_all / (ms / 1e3),
                     "amplitudes_per_s": len(batch) / (ms / 1e3), "ms_per_launch": ms,
                     "tiling": dict(zip(("x_chunk", "items_per_sm", "threads", "i3_split"), tiling))}
        outs[name] = [o.clone() for o in plan.outputs]
        del plan
    if "fp64" in outs:
        den = sum(float(b.norm()) ** 2 for b in outs["fp64"]) ** 0.5
        for name in outs:
            if name != "fp64":
                num = sum(float((a - b).norm()) ** 2 for a, b in zip(outs[name], outs["fp64"])) ** 0.5
                res[name]["rel_err_vs_fp64"] = num / den
    return dict(workload="256 irregular vertices (spins 1/2..6, dl 0..12, gamma 0.1/1.2/5.0, seed 0), all shells: "
                         "%d (%d non-empty); one CUDA-graph replay of a planned launch, tiling autotuned; tables "
                         "and boosters built before the replay" % (n_all, n_ne), **res)


def large_shell_measure(precisions):
    """All spins 4, gamma 1.2, dl 20: all 21^6 = 85,766,121 shells (55,341,615 non-empty) in one call
    per path, and the relative error of the mixed paths against the FP64 path."""
    import torch
    import paper_2107_13952_gb300 as sf
    from paper_2107_13952_gb300 import inputs
    w = inputs.large_shell()
    t = sf.sf_6j_table([sf.vertex(w["two_j"], w["gamma"], w["dl"])])
    sf.sf_boosters(t, RULE)
    n_ne = int(nonempty_shells(w["two_j"], w["dl"]).sum())
    stream = torch.cuda.current_stream()
    res, outs = {}, {}
    for name in precisions:
        e0, e1 = _events()
        e0.record(stream)
        A = sf.sf_vertex_amplitude(t, PRECISIONS[name])[0]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        res[name] = {"value": n_ne / (ms / 1e3), "unit": "non-empty shells/s", "ms": ms,
                     "amplitudes_per_s": 1e3 / ms, "kernel_ms": sf.last_kernel_ms()}
        outs[name] = A.clone()
    for name in outs:
        if name != "fp64" and "fp64" in outs:
            res[name]["rel_err_vs_fp64"] = float((outs[name] - outs["fp64"]).norm() / outs["fp64"].norm())
    return dict(workload="all spins 4, gamma 1.2, dl 20: all 85,766,121 shells (%d non-empty), one call per path"
                         % n_ne, **res)


def adjoint_measure():
    """All spins 3, gamma 1.2, dl 8 (531,441 shells): contracted amplitude and gradients with respect
    to the five seeded boundary vectors and the four booster tensors (adjoint kernels, FP64), and the
    amplitude alone."""
    import torch
    import paper_2107_13952_gb300 as sf
    from paper_2107_13952_gb300 import inputs
    w = inputs.boundary_contraction_vertex()
    t = sf.sf_6j_table([sf.vertex(w["two_j"], w["gamma"], w["dl"])])
    sf.sf_boosters(t, RULE)
    dims = sf.intertwiner_ranges(w["two_j"], w["gamma"], w["dl"])[1]
    psis = [torch.tensor(v, dtype=torch.complex128, device="cuda") for v in inputs.boundary_vectors(dims)]
    n_ne = int(nonempty_shells(w["two_j"], w["dl"]).sum())
    stream = torch.cuda.current_stream()
    out = {}
    for label, want in (("with_gradients", True), ("amplitude_only", False)):
        sf.sf_vertex_adjoint(t, psis, want_grads=want)
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record(stream)
        sf.sf_vertex_adjoint(t, psis, want_grads=want)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[label] = {"value": n_ne / (ms / 1e3), "unit": "non-empty shells/s", "ms": ms, "amplitudes_per_s": 1e3 / ms}
    return dict(workload="all spins 3, gamma 1.2, dl 8 (531,441 shells, %d non-empty): boundary-contracted "
                         "amplitude, FP64" % n_ne, **out)


def simplex_measure():
    """All spins 1, gamma 1.2, dl = 0..3, full rule: tables, boosters and the whole tensor per dl
    (the smallest workload; launch-bound)."""
    import torch
    import paper_2107_13952_gb300 as sf
    stream = torch.cuda.current_stream()
    out = {}
    for dl in range(4):
        def run():
            t = sf.sf_6j_table([sf.vertex((2,) * 10, 1.2, dl)])
            sf.sf_boosters(t, RULE)
            return sf.sf_vertex_amplitude(t, sf.SF_FP64)[0]
        run()
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record(stream)
        run()
        e1.record(stream)
        torch.cuda.synchronize()
        out["dl%d" % dl] = {"ms_end_to_end": e0.elapsed_time(e1), "non_empty_shells": int(nonempty_shells((2,) * 10, dl).sum())}
    return dict(workload="all spins 1, gamma 1.2, dl 0..3, FP64, tables + boosters + tensor per call", **out)


def contraction_measure(hbm_peak, reps=5):
    """The paper's GPU workload (Sec. 4, fig. contractions): complete contraction of two vertex
    tensors and of one vertex tensor with five boundary vectors, all spins J = 2, 4, ..., 24 at
    dl = 0 ((2J+1)^5 entries), seeded random FP64 tensors of those shapes (the cost depends on the
    shape only); CUDA events over `reps` back-to-back launches after a warm one."""
    import numpy as np
    import torch
    import paper_2107_13952_gb300 as sf
    stream = torch.cuda.current_stream()
    g = torch.Generator(device="cuda")
    g.manual_seed(2107)
    rng = np.random.default_rng(13952)
    rows = []
    for J in range(2, 25, 2):
        D = 2 * J + 1
        A = torch.randn((D,) * 5, dtype=torch.float64, device="cuda", generator=g)
        B = torch.randn((D,) * 5, dtype=torch.float64, device="cuda", generator=g)
        psis = [torch.tensor(rng.standard_normal(D) + 1j * rng.standard_normal(D), dtype=torch.complex128,
                             device="cuda") for _ in range(5)]
        row = {"J": J, "entries": D ** 5, "bytes": 8 * D ** 5}
        for label, fn, nbytes, fmas in (("vertex_vertex", lambda: sf.contract_vertices(A, B), 16 * D ** 5, D ** 5),
                                        ("vertex_5_vectors", lambda: sf.contract_vectors(A, psis), 8 * D ** 5,
                                         2 * D ** 5)):
            fn()
            torch.cuda.synchronize()
            e0, e1 = _events()
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            gbs = nbytes / (ms / 1e3) / 1e9
            row[label] = {"ms": ms, "GB_per_s": gbs, "hbm_frac": gbs / hbm_peak,
                          "fp64_frac": 2 * fmas / (ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS}
        rows.append(row)
        del A, B
    return {"workload": "vertex tensors (2J+1)^5, J = 2..24 step 2, seeded random FP64; %d back-to-back stream-ordered "
                        "calls per timing (each with its small stream-ordered scratch allocation); inputs above the "
                        "129 MB L2 from J = 14" % reps,
            "rows": rows}


def delta3_measure():
    """The Delta_3 network (Sec. 5) for boundary spins J = 1 and 2 at dl = 2, gamma 1.2: all
    internal spins x, vertex tensors by the shell sum (one batched launch), contractions and the sum
    over x on the GPU; end-to-end time per network."""
    import numpy as np
    import torch
    import paper_2107_13952_gb300 as sf
    from paper_2107_13952_gb300 import network as net
    out = {}
    stream = torch.cuda.current_stream()
    for two_J in (2, 4):
        D = two_J + 1
        rng = np.random.default_rng(two_J)
        psis = [v / np.linalg.norm(v) for v in (rng.standard_normal((9, D)) + 1j * rng.standard_normal((9, D)))]
        net.delta3(two_J, 2, 1.2, psis, rule=RULE)
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record(stream)
        xs, amps, tot, _ = net.delta3(two_J, 2, 1.2, psis, rule=RULE)
        e1.record(stream)
        torch.cuda.synchronize()
        out["J%d" % (two_J // 2)] = {"ms": e0.elapsed_time(e1), "internal_spins": len(xs),
                                     "amplitude": [float(complex(tot).real), float(complex(tot).imag)]}
    return dict(workload="Delta_3 graph, boundary spins J, dl 2, gamma 1.2, seeded unit boundary vectors, FP64", **out)


# ------------------------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=HEADLINE, choices=list(PRECISIONS), help="path timed for `value`")
    ap.add_argument("--slices", type=int, default=32, help="steps per full pass over the sweep")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other-workloads", action="store_true", help="time the sweep only")
    ap.add_argument("--case", default=None, help="lambda:groups:precision -- one shell-sum launch (profiling)")
    ap.add_argument("--contract-case", type=int, default=None,
                    help="J -- one vertex-vertex and one vertex-5-vectors contraction of (2J+1)^5 tensors (profiling)")
    args = ap.parse_args()

    if args.contract_case:
        import numpy as np
        import torch
        import paper_2107_13952_gb300 as sf
        D = 2 * args.contract_case + 1
        g = torch.Generator(device="cuda")
        g.manual_seed(2107)
        A = torch.randn((D,) * 5, dtype=torch.float64, device="cuda", generator=g)
        B = torch.randn((D,) * 5, dtype=torch.float64, device="cuda", generator=g)
        rng = np.random.default_rng(13952)
        psis = [rng.standard_normal(D) + 1j * rng.standard_normal(D) for _ in range(5)]
        vv = float(sf.contract_vertices(A, B))
        a = complex(sf.contract_vectors(A, psis))
        print(json.dumps({"contract_case": args.contract_case, "vertex_vertex": vv, "vertex_5_vectors": [a.real, a.imag]}))
        return

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
    S = args.slices
    G = 11 ** 3

    def slice_bounds(k):
        g0, g1 = G * k // S, G * (k + 1) // S
        return g0 * 121 * 11, g1 * 121 * 11, g0, g1

    import numpy as np
    nonempty = {lam: np.cumsum(np.concatenate([[0], nonempty_shells((lam,) * 10, dl)])) for lam, dl in SWEEP}

    def slice_shells(k):
        b, e, _, _ = slice_bounds(k % S)
        return sum(int(c[e] - c[b]) for c in nonempty.values()), 16 * (e - b)

    if args.impl == "reference":
        if rank != 0:
            return
        n_all, t_all = 0, 0.0
        for i in range(args.warmup + args.steps):
            r, cores, n, el = oracle_rate(max(2.0, args.cpu_seconds / max(1, args.steps)), seed=i)
            if i >= args.warmup:
                n_all += n
                t_all += el
        value = n_all / t_all
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "non-empty shells/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * t_all / max(1, args.steps), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload_name(S), "slices_per_pass": S,
                           "sample": "the CPU oracle's shell-sum phase on %d non-empty shells drawn uniformly from the "
                                     "sweep (boosters random), on all host cores" % n_all},
                "cpu_baseline": {"value": value, "unit": "non-empty shells/s", "cores": cores, "kind": "oracle",
                                 "sample": "%d non-empty shells drawn uniformly from the sweep's %d shells, boosters "
                                           "random (shell-sum phase only)" % (n_all, 16 * 11 ** 6)},
                "e2e": {"value": value, "unit": "non-empty shells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
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
    hbm_peak = 6791.0
    try:
        hbm_peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        pass
    verts = [sf.vertex((lam,) * 10, GAMMA, dl) for lam, dl in SWEEP]
    dims = [sf.intertwiner_ranges((lam,) * 10, GAMMA, dl)[1] for lam, dl in SWEEP]
    outs = [torch.empty(d, dtype=torch.float64, device="cuda") for d in dims]
    host = [torch.empty(d, dtype=torch.float64, pin_memory=True) for d in dims]
    stream = torch.cuda.current_stream()

    def step(k, prec, to_host):
        b, e, _, _ = slice_bounds(k % S)
        t = sf.sf_6j_table(verts, shell_range=(b, e))
        sf.sf_boosters(t, RULE)
        sf.sf_vertex_amplitude(t, prec, b, e, out=outs)
        kms = sf.last_kernel_ms()
        if to_host:
            for o, h in zip(outs, host):
                h.copy_(o, non_blocking=True)
        del t
        return kms

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(prec, first, to_host, nsteps=None):
        barrier()
        torch.cuda.synchronize()
        e0, e1 = _events()
        kms_all, ne, alls, ks = [], 0, 0, []
        launches0 = sf.kernel_launches()
        e0.record(stream)
        for i in range(nsteps or args.steps):
            k = (first + i) * world + rank
            kms_all.append(step(k, prec, to_host))
            a, b = slice_shells(k)
            ne += a
            alls += b
            ks.append(k % S)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return e0.elapsed_time(e1), kms_all, ne, alls, ks, sf.kernel_launches() - launches0

    head = PRECISIONS[args.precision]
    for i in range(args.warmup):
        step(i * world + rank, head, False)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    ms, kms_all, ne, alls, slices, launches = timed(head, args.warmup, False)
    clocks = clk.stop()
    last = {args.precision: [o.clone() for o in outs]}
    n_short = min(args.steps, 4)
    ms_e2e, _, ne_e2e, _, _, _ = timed(head, args.warmup, True, n_short)

    # the FP64 path and SF_MIXED over the same steps (same slices), the pair path over the first
    # min(steps, 4) of them (its last slice is then compared with the FP64 path's tensors of that
    # slice, recomputed), and each path's tensors of its last step
    others = {}
    for name, p in PRECISIONS.items():
        if name == args.precision:
            continue
        n = args.steps if name in ("fp64", "mixed") else n_short
        step(args.warmup * world + rank, p, False)
        ms_o, kms_o, ne_o, all_o, ks_o, _ = timed(p, args.warmup, False, n)
        others[name] = {"value": ne_o * world / (ms_o / 1e3), "unit": "non-empty shells/s",
                        "all_shells_per_s": all_o * world / (ms_o / 1e3), "ms_per_step": ms_o / n, "steps": n,
                        "kernel_ms_per_step": sum(kms_o) / n, "dtype": DTYPES[name]}
        last[name] = [o.clone() for o in outs]
        if n != args.steps:   # compare on the slice it ended on: the FP64 path on that slice
            step(ks_o[-1], PRECISIONS["fp64"], False)
            last[name + "@fp64"] = [o.clone() for o in outs]
    # errors of the mixed paths against the FP64 path on the last slice, per lambda
    rel_err_per_lambda = {}
    for name in PRECISIONS:
        if name == "fp64":
            continue
        per = {}
        ref = last.get(name + "@fp64", last["fp64"])
        for (lam, _), o, r in zip(SWEEP, last[name], ref):
            rn = float(r.norm())
            per[str(lam)] = float((o - r).norm()) / rn if rn > 0 else None
        rel_err_per_lambda[name] = per

    if world > 1:
        tm = torch.tensor([ms, ms_e2e], device="cuda")
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        ms, ms_e2e = float(tm[0]), float(tm[1])
    value = ne * world / (ms / 1e3)
    e2e_value = ne_e2e * world / (ms_e2e / 1e3)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # cancellation factor per lambda on the last slice: kappa = sum_s ||C_s|| / ||A_slice||, over
    # every shell of the slice (kappa pass of the library, FP64)
    kappa = {}
    b, e, _, _ = slice_bounds(slices[-1])
    tk = sf.sf_6j_table(verts, shell_range=(b, e))
    sf.sf_boosters(tk, RULE)
    _, ks = sf.sf_vertex_amplitude(tk, sf.SF_FP64, b, e, kappa=True)
    for (lam, dl), r, kv in zip(SWEEP, last["fp64"], ks):
        if float(r.norm()) > 0.0:
            kappa[str(lam)] = kv / float(r.norm())
    del tk
    u32 = 2.0 ** -24
    err_model = {name: {lam: (per[lam] / (kappa[lam] * u32) if lam in kappa and per[lam] is not None else None)
                        for lam in per} for name, per in rel_err_per_lambda.items()
                 if name + "@fp64" not in last}   # the paths compared on the slice kappa is taken on

    # roofline of the dominant kernel (the shell sum of the timed path)
    f64, f32, tcm, canon = 0, 0, 0, 0.0
    canon_cum = {lam: np.cumsum(np.concatenate([[0.0], canonical_flops((lam,) * 10, dl)])) for lam, dl in SWEEP}
    for k in slices:
        bb, ee, g0, g1 = slice_bounds(k)
        for lam, dl in SWEEP:
            a64, a32, atc = pipe_ops(executed_fmas((lam,) * 10, dl, g0, g1), args.precision)
            f64 += a64
            f32 += a32
            tcm += atc
            canon += float(canon_cum[lam][ee] - canon_cum[lam][bb])
    kern_s = sum(kms_all) / 1e3
    fp64_tflops = f64 / kern_s / 1e12
    fp32_tops = f32 / kern_s / 1e12
    # the bounding pipe: the one whose executed operations take the longest at its peak rate
    if f32 / FP32_PEAK_TOPS >= f64 / FP64_PEAK_TFLOPS:
        pipe = {"achieved": fp32_tops, "peak": FP32_PEAK_TOPS, "unit": "Tops/s", "frac": fp32_tops / FP32_PEAK_TOPS,
                "peak_note": "FP32 pipe, derived: 152 SMs x 128 lanes x 2.07 GHz, in lane operations (FFMA, FADD, "
                             "FMUL each one) per second (no measured FP32 figure)",
                "counted": "FP32 lane operations the kernel's loops execute in this path's FP32 and pair phases, "
                           "from the trip counts (one per FP32 multiply-add, %d per pair-by-float Dot2 step, %d per "
                           "pair-by-pair step)" % (FFD_OPS, FF_OPS["F"])}
    else:
        pipe = {"achieved": fp64_tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": fp64_tflops / FP64_PEAK_TFLOPS,
                "peak_note": "FP64 pipe, derived: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz (no measured FP64 figure)",
                "counted": "FP64 flops the kernel's loops execute in this path's FP64 phases, 2 per multiply-add, "
                           "from the trip counts"}
    roof = {"bound": "alu", **pipe,
            "fp64_tflops": fp64_tflops, "fp64_frac": fp64_tflops / FP64_PEAK_TFLOPS,
            "fp32_lane_ops_per_s": fp32_tops, "fp32_frac": fp32_tops / FP32_PEAK_TOPS,
            "tensor_mma_macs": tcm, "tensor_tflops_unpadded": 2 * tcm / kern_s / 1e12,
            "canonical_tflops": canon / kern_s / 1e12, "canonical_frac": canon / kern_s / 1e12 / FP64_PEAK_TFLOPS,
            "canonical_note": "the framed algorithm's FP64 flop count (W by the x-sum plus four mode products per "
                              "non-empty shell) over the kernel time: above 1 because the hoisted order executes a "
                              "fraction of those operations",
            "kernel": "k_shell<%d> (one launch per launch class of the step)" % head,
            "kernel_ms_per_step": 1e3 * kern_s / args.steps,
            "traffic_note": "dram__bytes_read.sum + dram__bytes_write.sum of the shell-sum launches of one step "
                            "(slice 3), from one ncu capture, per step like achieved"}
    traffic = None
    if NCU_TRAFFIC["sha1"] == kernel_sha1() and args.precision == HEADLINE:
        traffic = NCU_TRAFFIC["bytes_per_step"]
    roof["traffic"] = traffic

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        r, cores, n, el = oracle_rate(args.cpu_seconds)
        cpu = {"value": r, "unit": "non-empty shells/s", "cores": cores, "kind": "oracle",
               "sample": "%d non-empty shells drawn uniformly from the sweep (%.1f s on %d processes), boosters "
                         "random (shell-sum phase only)" % (n, el, cores)}

    extra = {}
    if not args.no_other_workloads and world == 1:
        main_paths = [HEADLINE, "mixed_px", "fp64"]
        extra["batched_256"] = batched_measure(main_paths)
        extra["large_shell_j4_dl20"] = large_shell_measure(main_paths)
        extra["adjoint_j3_dl8"] = adjoint_measure()
        extra["simplex_j1"] = simplex_measure()
        extra["contractions"] = contraction_measure(hbm_peak)
        extra["delta3"] = delta3_measure()

    d2h = sum(h.numel() * 8 for h in host)
    h2d = len(verts) * ctypes.sizeof(sf.sf_vertex) + ctypes.sizeof(sf.sf_quad_rule)
    line = {
        "metric": METRIC,
        "value": value, "unit": "non-empty shells/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[args.precision], "data": "synthetic",
        "config": {"workload": workload_name(S), "slices_per_pass": S, "precision": args.precision,
                   "counting": "non-empty shells (all four virtual-intertwiner ranges non-empty); all_shells_per_s "
                               "counts the whole (dl+1)^6 grid",
                   "cache": "inputs larger than L2: every step rebuilds the {6j} tables, d-tables and boosters its "
                            "slice reads (the spin-8 S3 table alone, FP64 plus pair copy, is 384 MB, 3x the L2; "
                            "each slice reads the groups of other l35 values than the previous one), so no step "
                            "starts with its working set in L2; no separate flush"},
        "all_shells_per_s": alls * world / (ms / 1e3),
        # whole vertex tensors of the sweep per second at this rate (16 tensors per S steps)
        "amplitudes_per_s": len(SWEEP) * world / (S * ms / args.steps / 1e3),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "non-empty shells/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clocks,
        "path": args.precision,
        "precision_split": PHASE_PRECISION[args.precision],
        "other_paths": others,
        "speedup_vs_fp64": value / others["fp64"]["value"] if "fp64" in others else None,
        "mixed_vs_fp64": {"rel_err_per_lambda": rel_err_per_lambda, "kappa_per_lambda": kappa,
                          "rel_err_over_kappa_u32": err_model, "stated_bound": 1e-6,
                          "metric": "||A_mixed - A_fp64|| / ||A_fp64|| per vertex on the last timed slice; kappa = "
                                    "sum over that slice's shells of ||C_s|| / ||A_slice||"},
        **extra,
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
