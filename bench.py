"""Benchmark: Lloyd iterations/s of accelerated spherical k-means on one GB300.

Workload (default): the RCV-1-like sparse TF-IDF set -- n = 100,000 rows,
d = 50,000 terms, nnz/row lognormal(mean 120, sigma 0.8) clipped to
[5, 2000], Zipf(1.1) terms, unit FP32 rows + int32 indices, k = 100 seeded
initial rows, run to convergence (at most 100 iterations).

One step = one complete clustering run from the seeded initial centers
(restart, then assign + update until no label changes).  value = Lloyd
iterations per second over the K timed steps of the variant given (Simplified
Elkan by default -- the paper's fastest variant on most of its data sets,
Table 3); the plain standard variant and the other bounded variants are
timed on the same workload, their label sequences are identical, and their
rates are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--variant elkan]
  python bench.py --impl reference ...   (the FP64 CPU oracle on host cores)
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "Lloyd iterations/sec and point·center sims/sec vs plain FP32 standard (same GB300, same labels)"
K_CLUSTERS = 100
MAX_ITERS = 100
INIT_SEED = 2


def workload_cfg():
    return synth.CSR_RCV1_LIKE


def config_block(cfg, variant, l2_note):
    return {"workload": f"rcv1-like sparse TF-IDF n={cfg.n} d={cfg.d} nnz/row~lognormal(120,0.8) Zipf(1.1) "
                        f"k={K_CLUSTERS} to convergence (max {MAX_ITERS})",
            "variant": variant, "n": cfg.n, "d": cfg.d, "k": K_CLUSTERS, "seed": cfg.seed,
            "step": "one full clustering run from the seeded initial rows", "l2": l2_note,
            "parallelism": "replicas"}


def whole_job_ms(ms, world, device):
    """The whole job's time: the slowest rank's (identity for one rank).  Every
    rank calls it with its own time."""
    if world > 1:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    return ms


def job_value(world, iters_per_rank, job_ms):
    """Whole-job throughput of independent replicas (weak scaling): every rank
    ran iters_per_rank iterations within job_ms."""
    return world * iters_per_rank / (job_ms / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi SM clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------ roofline helpers

# the source file of each profiled kernel (with the shared header)
KERNEL_FILES = {"k_rows_top2": "k_assign.cu", "k_rows_top2(list)": "k_assign.cu", "k_elk_bounds": "k_assign.cu",
                "k_elk_recompute": "k_assign.cu", "k_ham_bounds": "k_assign.cu", "k_center_sum": "k_update.cu",
                "k_center_sum_multi": "k_update.cu", "k_colnorm_part": "k_update.cu",
                "k_normalize_drift": "k_update.cu", "k_bf16_topk": "k_mma.cu"}


def source_hash(kernel: str | None = None) -> str:
    """sha1 over the CUDA source of `kernel` (its file and the shared header;
    all sources when unknown): a recorded ncu traffic figure only applies to
    the kernel code it was measured on."""
    import glob
    import hashlib
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2107_04074_gb300", "csrc")
    if kernel in KERNEL_FILES:
        files = [os.path.join(csrc, KERNEL_FILES[kernel]), os.path.join(csrc, "skm_internal.cuh")]
    else:
        files = sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh")))
    for f in files:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:12]


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` from profiles/dram_traffic.txt
    (lines: kernel workload source_hash bytes_per_launch), if it was taken on
    the kernel's current source; else None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    cur = source_hash(kernel)
    for ln in lines:
        f = ln.split()
        if len(f) == 4 and f[0] == kernel and f[1] == workload and f[2] == cur:
            return int(float(f[3]))
    return None


def screen_opt(args):
    """--screen 1 / 0: FP16 screening of the Elkan whole-row recomputes on /
    off; absent: the library's choice (on for k > 128)."""
    return None if args.screen is None else bool(args.screen)


def measured_peaks(skm, torch):
    """FP32 and FP64 FMA rates from the library's own microbenchmark
    (skm_measure_peak), and the FP8-E4M3 GEMM rate of cuBLAS through
    torch._scaled_mm (8192^3, best of 10; None where this PyTorch lacks it)."""
    f32, f32x2 = skm.measure_peak("fp32"), skm.measure_peak("fp32x2")
    # the FP32 roof: the higher of scalar and packed-pair FMA issue
    out = {"fp32_fma_tflops": round(max(f32, f32x2), 1), "fp32_fma_scalar_tflops": round(f32, 1),
           "fp32_fma_packed_tflops": round(f32x2, 1),
           "fp64_fma_tflops": round(skm.measure_peak("fp64"), 2),
           "l2_gather_tbps": round(skm.measure_peak("l2_gather"), 2)}
    try:
        N = 8192
        a = torch.randn(N, N, device="cuda").to(torch.float8_e4m3fn)
        b = torch.randn(N, N, device="cuda").to(torch.float8_e4m3fn).t()  # column-major operand
        one = torch.tensor(1.0, device="cuda")
        for _ in range(3):
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        best = None
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        out["fp8_gemm_tflops"] = round(2.0 * N ** 3 / (best / 1e3) / 1e12, 1)
        del a, b
    except Exception as ex:  # noqa: BLE001
        out["fp8_gemm_tflops"] = None
        out["fp8_note"] = f"{type(ex).__name__}: {ex}"[:160]
    out["how"] = ("fp32/fp64: skm_measure_peak (independent FMA chains on every SM, CUDA events; FP32 the "
                  "higher of scalar and packed fma.rn.f32x2 chains); l2_gather: 416-byte rows at random rows "
                  "of an L2-resident 20.8 MB table, 16 in flight per warp; "
                  "fp8: torch._scaled_mm E4M3 8192^3 -> BF16, best of 10")
    return out


def launch_traffic(name, avg_rows):
    """ncu DRAM bytes per launch of `name` on the RCV-1-like workload: a
    per-launch record, or a per-row record times the launch's average rows
    (whole-row launches treat a different number of rows each iteration)."""
    t = recorded_traffic(name, "rcv1-like-k100")
    if t is not None:
        return t
    per_row = recorded_traffic(name, "rcv1-like-k100-per-row")
    return int(per_row * avg_rows) if per_row is not None else None


def kernel_bytes(name, it_rows, n, d, k, nnz, variant, full_sum=True, u_width=4):
    """Compulsory (algorithmic) bytes of one launch: what any implementation
    must move between HBM and the SMs for that step, given the rows it treats.
    it_rows: rows treated by the launch (all rows, the recompute list, ...)."""
    avg = nnz / n
    elk = variant in ("elkan", "simp_elkan")
    row = 8 + 8 * avg + 4 + 4 + 4 + 4  # row_ptr, (col, val) entries, label r/w, 1/|x|, delta
    if name in ("k_rows_top2", "k_rows_top2(list)"):
        out = (u_width * k if elk else 0) + (8 if variant != "standard" else 0)
        return int(it_rows * (row + out + (4 if name.endswith("(list)") else 0)) + 4 * d * k)
    if name == "k_elk_bounds":
        return int(elk_bound_bytes(n, k, u_width))
    if name == "k_elk_recompute":
        return int(it_rows * ((u_width + (4 if variant == "elkan" else 0)) * k + row + 4))
    if name == "k_center_sum":  # only a full recomputation moves data (else the kernel returns at once)
        return int(8 * nnz + 8 * d * k + 4 * n) if full_sum else 0
    if name == "k_ham_bounds":
        return int(24 * n)
    return None


def gather_bytes(name, it_rows, n, k, nnz):
    """Center values a whole-row launch gathers (4 B per center of the padded
    slice per non-zero of the rows it treats): the traffic that binds it, served
    from L1/L2 since the term-major centers are L2-resident."""
    if name in ("k_rows_top2", "k_rows_top2(list)"):
        return int(it_rows * (nnz / n) * 4 * ((k + 7) // 8 * 8))
    return None


def run_ours(args, rank, world, local):
    import torch
    from paper_2107_04074_gb300 import skm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = workload_cfg()
    csr = synth.tfidf(cfg)
    init = synth.init_rows(csr.n, K_CLUSTERS, INIT_SEED)
    n, d, k, nnz = csr.n, csr.d, K_CLUSTERS, csr.nnz
    rp = torch.from_numpy(csr.row_ptr).to(dev)
    col = torch.from_numpy(csr.col).to(dev)
    val = torch.from_numpy(csr.val).to(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

    def make(variant):
        # every variant (the plain standard one included) replays its steady-state
        # iteration as a CUDA graph
        return skm.KMeans(n, d, rp, col, val, k, variant=variant, init_rows=init, stream=stream.cuda_stream,
                          graph=not args.no_graph, screen=screen_opt(args))

    def timed_runs(km, steps, warmup):
        for _ in range(warmup):
            km.reset(init)
            km.run(MAX_ITERS)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        total_ms, iters, sims = 0.0, 0, 0
        l0 = skm.kernel_launches()
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            km.reset(init)
            it, J = km.run(MAX_ITERS)
            e1.record(stream)
            torch.cuda.synchronize()
            total_ms += e0.elapsed_time(e1)
            iters += it
            sims += km.stats().total_sims
        launches = skm.kernel_launches() - l0
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        return total_ms, iters, sims, launches, J

    variant = args.variant
    km = make(variant)
    if args.trace:
        return trace_run(km, init, n, k)
    sampler = ClockSampler(local)
    sampler.start()
    ms, iters, sims, launches, J = timed_runs(km, args.steps, args.warmup)
    clocks = sampler.stop()
    lab_v = km.labels()
    if args.quick:
        km.close()
        return {"metric": METRIC, "value": round(world * iters / (ms / 1e3), 3), "unit": "Lloyd iterations/s",
                "quick": True, "ms_per_step": round(ms / args.steps, 4), "iterations_per_run": iters / args.steps}
    # whole-job time = max over ranks
    ms = whole_job_ms(ms, world, dev)
    it_per_step = iters / args.steps
    value = job_value(world, iters, ms)

    # the plain FP32 standard variant at identical labels
    std_steps = max(1, min(args.steps, 3))
    km_std = make("standard")
    ms_s, iters_s, sims_s, _, J_s = timed_runs(km_std, std_steps, 1)
    lab_s = km_std.labels()
    labels_identical = bool(np.array_equal(lab_v, lab_s)) and iters_s / std_steps == it_per_step
    std_rate = iters_s / (ms_s / 1e3)
    km_std.close()

    # per-kernel CUDA-event profile of one more run (not part of the timed
    # value), iteration by iteration so that each launch's rows are known
    flush.fill_(1.0)
    km.reset(init)
    prof_ms, prof_n, prof_bytes, prof_gather, prof_flops, prof_rows = {}, {}, {}, {}, {}, {}
    u_width = elk_u_width(skm, n, k)
    peaks_meas = measured_peaks(skm, torch)
    upd = {"full": [0.0, 0], "incremental": [0.0, 0]}  # center update: ms, count
    for it in range(MAX_ITERS):
        km.profile(True)
        ch = km.assign()
        st = km.stats()
        pa = km.profile_read()
        km.profile(True)
        if ch:
            km.update_centers()
        pu = km.profile_read()
        km.profile(False)
        rows_of = {"k_rows_top2": n, "k_rows_top2(list)": st.last_rechecks, "k_elk_recompute": st.last_survivors}
        full_sum = it == 0 or ch * 8 > n
        if ch:
            u = upd["full" if full_sum else "incremental"]
            u[0] += sum(v[0] for v in pu.values())
            u[1] += 1
        for nm, (ms_k, cnt_k) in list(pa.items()) + list(pu.items()):
            nm = skipped_name(nm, st)
            prof_ms[nm] = prof_ms.get(nm, 0.0) + ms_k
            prof_n[nm] = prof_n.get(nm, 0) + cnt_k
            prof_rows[nm] = prof_rows.get(nm, 0) + rows_of.get(nm, n) * cnt_k
            b = kernel_bytes(nm, rows_of.get(nm, n), n, d, k, nnz, variant, full_sum, u_width)
            if b is not None:
                prof_bytes[nm] = prof_bytes.get(nm, 0) + b * cnt_k
            gb = gather_bytes(nm, rows_of.get(nm, n), n, k, nnz)
            if gb is not None:
                prof_gather[nm] = prof_gather.get(nm, 0) + gb * cnt_k
                # the similarity FMAs of a whole-row launch: 2 per entry and center
                prof_flops[nm] = prof_flops.get(nm, 0) + 2 * rows_of.get(nm, n) * (nnz / n) * k * cnt_k
        if ch == 0:
            break
    km.close()
    center_update = {kind: {"iterations": c, "ms_per_update": round(t / c, 4) if c else None}
                     for kind, (t, c) in upd.items()}
    center_update["note"] = ("CUDA events over all kernels of one center update; incremental = only the changed "
                             "rows' contributions moved in the exact fixed-point sums (full recompute when more "
                             "than n/8 labels changed)")
    # spherical k-means++ seeding of the same data (k passes over the rows),
    # then its first assignment: a separate pass (skm_assign) or pre-initialised
    # from the seeding's own similarities (skm_seed_kmeanspp_assign)
    seed_u = np.random.Generator(np.random.PCG64(INIT_SEED + 1)).random(k)

    def host_ms(fn, reps=3):
        best = None
        for _ in range(reps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t) * 1e3
            best = dt if best is None else min(best, dt)
        return best

    seeding = {}
    for sv in (variant, "hamerly"):
        kp = make(sv)
        kp.seed_kmeanspp(seed_u)
        kp.seed_kmeanspp_assign(seed_u)
        e = {"seed_ms": round(host_ms(lambda: kp.seed_kmeanspp(seed_u)), 3),
             "seed_then_first_assignment_ms": round(host_ms(lambda: (kp.seed_kmeanspp(seed_u), kp.assign())), 3),
             "seed_with_preinitialised_first_assignment_ms": round(host_ms(lambda: kp.seed_kmeanspp_assign(seed_u)),
                                                                   3)}
        kp.seed_kmeanspp_assign(seed_u)
        kp.update_centers()
        it_pp, _ = kp.run(MAX_ITERS)
        e["run_from_seeds_iterations"] = it_pp + 1  # with the pre-initialised first assignment
        e["run_from_seeds_sims"] = kp.stats().total_sims
        seeding[sv] = e
        kp.close()
    seed_ms = seeding[variant]["seed_ms"]
    tot_prof = sum(prof_ms.values()) or 1.0
    top_name = max(prof_ms, key=prof_ms.get)
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm_peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        hbm_peak, peak_src = 6800.0, "fallback"
    roof = None
    if top_name in prof_bytes:
        avg_s = prof_ms[top_name] / 1e3 / prof_n[top_name]
        ab = prof_bytes[top_name] / prof_n[top_name]
        ach = ab / avg_s / 1e9
        roof = {"kernel": top_name, "bound": "hbm", "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(ach / hbm_peak, 4), "peak_source": peak_src,
                "traffic": launch_traffic(top_name, prof_rows.get(top_name, 0) / prof_n[top_name]),
                "avg_launch_us": round(avg_s * 1e6, 2), "launches": prof_n[top_name],
                "algorithmic_bytes_per_launch": int(ab)}
        if top_name in prof_flops and peaks_meas.get("fp32_fma_tflops"):
            fpl = prof_flops[top_name] / prof_n[top_name]
            ach_f = fpl / avg_s / 1e12
            roof["fma_view"] = {"achieved": round(ach_f, 2), "peak": peaks_meas["fp32_fma_tflops"],
                                "unit": "TFLOP/s", "frac": round(ach_f / peaks_meas["fp32_fma_tflops"], 4),
                                "peak_source": "measured (skm_measure_peak FP32 FMA)",
                                "flops_per_launch": int(fpl)}
        if top_name in prof_gather:
            gpl = prof_gather[top_name] / prof_n[top_name]
            roof["gathered_bytes_per_launch"] = int(gpl)
            roof["gather_GBps"] = round(gpl / avg_s / 1e9, 1)
            roof["note"] = ("bound by the L1/L2 gathers of center slices (ncu: L1 throughput ~78% of peak), "
                            "not by HBM")
            if peaks_meas.get("l2_gather_tbps"):
                gt = gpl / avg_s / 1e12
                roof["gather_view"] = {"achieved": round(gt, 2), "peak": peaks_meas["l2_gather_tbps"], "unit": "TB/s",
                                       "frac": round(gt / peaks_meas["l2_gather_tbps"], 4),
                                       "peak_source": "measured (skm_measure_peak L2 gather: uniform random 416-byte "
                                                      "rows; the kernel's Zipf terms also hit L1, so it can exceed it)"}
    kernel_share = {}
    for nm in sorted(prof_ms, key=lambda x: -prof_ms[x]):
        e = {"ms": round(prof_ms[nm], 3), "launches": prof_n[nm], "share": round(prof_ms[nm] / tot_prof, 4)}
        if nm in prof_bytes:
            e["GB_per_s"] = round(prof_bytes[nm] / (prof_ms[nm] / 1e3) / 1e9, 1)
        kernel_share[nm] = e

    # every variant on the same workload (same labels), for comparison
    others = {}
    for v in ("standard", "hamerly", "elkan", "simp_hamerly", "simp_elkan", "yinyang"):
        if v == variant:
            others[v] = round(value / world, 3)
            continue
        kv = make(v)
        ms_o, it_o, _, _, _ = timed_runs(kv, std_steps, 1)
        others[v] = round(it_o / (ms_o / 1e3), 3)
        kv.close()

    # end to end through the C ABI with host buffers (pinned), copies included
    pin = [torch.from_numpy(a).pin_memory() for a in (csr.row_ptr, csr.col, csr.val)]
    host = [t.numpy() for t in pin]
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_iters = 0
    for _ in range(e2e_steps):
        kh = skm.KMeans(n, d, host[0], host[1], host[2], k, variant=variant, init_rows=init,
                        stream=stream.cuda_stream, graph=not args.no_graph, screen=screen_opt(args))
        it, _ = kh.run(MAX_ITERS)
        lab_h = kh.labels()
        kh.close()
        e2e_iters += it
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    assert np.array_equal(lab_h, lab_v)
    h2d = int(csr.row_ptr.nbytes + csr.col.nbytes + csr.val.nbytes + init.nbytes)
    d2h = int(4 * n + 8 + 8 * 8)

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "Lloyd iterations/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_block(cfg, variant, "L2 flushed (256 MB write) before every step"),
        "iterations_per_run": it_per_step,
        "sims_per_s_effective": round(world * n * k * iters / (ms / 1e3), 1),
        "sims_per_s_evaluated": round(world * sims / (ms / 1e3), 1),
        "standard_iters_per_s": round(std_rate, 3),
        "speedup_vs_standard": round(value / world / std_rate, 3),
        "labels_identical_to_standard": labels_identical,
        "variants_iters_per_s": others,
        "objective": J,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "roofline": roof,
        "kernel_time_share": kernel_share,
        "measured_peaks": peaks_meas,
        "center_update": center_update,
        "kmeanspp_seeding": {"ms": seed_ms, "k": k, "rows": n, "variants": seeding,
                             "note": "host-timed, synchronised, best of 3: skm_seed_kmeanspp alone; followed by "
                                     "skm_assign (a pass over all n k similarities); skm_seed_kmeanspp_assign, "
                                     "whose seeding keeps the first assignment's labels and bounds (one more "
                                     "center's similarities instead of that pass)"},
        "e2e": {"value": round(e2e_iters / e2e_s, 3), "unit": "Lloyd iterations/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "note": "skm_init with host CSR (H2D copy, row norms, term-major copy) + run + labels to host"},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(csr, init, variant)
    if rank == 0 and not args.no_extras:
        # the other two forms of the path, summarised (their own modes:
        # --workload embed / batch); a failure there is reported, not fatal
        del km, km_std, rp, col, val, flush
        torch.cuda.empty_cache()
        for key, fn in (("precision_form", summarize_embed), ("batched_form", summarize_batch),
                        ("large_sparse", summarize_large)):
            try:
                out[key] = fn(args, rank, world, local)
            except Exception as ex:  # noqa: BLE001
                out[key] = {"error": f"{type(ex).__name__}: {ex}"}
            torch.cuda.empty_cache()
    return out


def summarize_embed(args, rank, world, local):
    r = run_embed(args, rank, world, local)
    p = r["paths"]
    keep = ("iters", "iters_per_s")
    return {"workload": r["workload"], "labels_identical_across_paths": r["labels_identical_across_paths"],
            "iters_per_s": {k: v["iters_per_s"] for k, v in p.items()},
            "ms_median_min_max": {k: [v["ms"]] + v["ms_min_max"] for k, v in p.items()},
            "repeats": p["standard/bf16"]["repeats"],
            "error_vs_fp64_oracle": r["error_vs_fp64_oracle"],
            "speedup_bf16_vs_fp32_standard": r["speedup_bf16_vs_fp32_standard"],
            "speedup_fp8_vs_fp32_standard": r["speedup_fp8_vs_fp32_standard"],
            "roofline": r["bf16_gemm_roofline"],
            "fp8_roofline": r["fp8_gemm_roofline"],
            "fp32_roofline": r["fp32_gemm_roofline"],
            "ambiguous_fraction_first_last": {kk: [v["ambiguous_fraction_per_iter"][0],
                                                   v["ambiguous_fraction_per_iter"][-1]]
                                              for kk, v in p.items() if "ambiguous_fraction_per_iter" in v},
            "rows_candidate_recheck_first_last": [p["standard/bf16"]["rows_candidate_recheck_per_iter"][0],
                                                  p["standard/bf16"]["rows_candidate_recheck_per_iter"][-1]],
            "note": "BF16 tcgen05 bulk with candidate selection, FP32 recheck; see --workload embed"} \
        if all(k in p["standard/bf16"] for k in keep) else r


def summarize_batch(args, rank, world, local):
    a = argparse.Namespace(**vars(args))
    a.steps, a.warmup = 2, 1
    r = run_batch(a, rank, world, local)
    for v in r["variants"].values():
        v.pop("kernel_time_share", None)
    r["note"] = "see --workload batch"
    return r


def trace_run(km, init, n, k):
    """One run, assign and update timed per iteration with per-kernel events."""
    km.reset(init)
    rows = []
    for it in range(MAX_ITERS):
        km.profile(True)
        ch = km.assign()
        st = km.stats()
        pa = km.profile_read()
        km.profile(True)
        if ch:
            km.update_centers()
        pu = km.profile_read()
        km.profile(False)
        rows.append({"it": it + 1, "changed": ch, "sims": st.last_sims, "survivors": st.last_survivors,
                     "rows": st.last_rechecks,
                     "assign_ms": round(sum(v[0] for v in pa.values()), 4),
                     "update_ms": round(sum(v[0] for v in pu.values()), 4),
                     "assign_kernels": {kk: round(v[0], 4) for kk, v in pa.items()},
                     "update_kernels": {kk: round(v[0], 4) for kk, v in pu.items()}})
        if ch == 0:
            break
    return {"trace": rows, "n": n, "k": k}


def oracle_assign_rows(Xs, rows, C, prev, threads=None):
    """The FP64 oracle's assignment of the dense rows Xs[rows] from centers C
    (teacher-forced: prev holds their current labels), on contiguous blocks of
    the sample in parallel host threads.  Returns (labels, top-2 gaps)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    P = threads or os.cpu_count() or 1
    cuts = np.linspace(0, len(rows), P + 1).astype(np.int64)
    C64 = np.ascontiguousarray(C, dtype=np.float64)

    def one(q):
        sub = oracle.Data.from_dense(Xs[rows[cuts[q]:cuts[q + 1]]])
        lab, _, _, _, gap = oracle.assign(sub, oracle.rinv(sub), C64, prev[cuts[q]:cuts[q + 1]])
        return lab, gap

    with ThreadPoolExecutor(max_workers=P) as pool:
        outs = list(pool.map(one, range(P)))
    return np.concatenate([o[0] for o in outs]), np.concatenate([o[1] for o in outs])


def embed_error_vs_oracle(skm, Xd, Xs, k, init, iters, precision, nsample=20000, check_at=(1, 2, 5, 10, 20)):
    """Per-result error of a dense path against the FP64 oracle, teacher-forced
    at the listed iterations: label mismatches on a seeded sample of rows (the
    oracle assigns them from the GPU's centers and previous labels; mismatches
    at FP64 top-2 gaps below 1e-6 are counted apart as near-ties), and after
    the update the largest center error |c_gpu - c_oracle| and the objective's
    relative error (the oracle updates from the GPU's labels over all rows)."""
    import oracle
    rng = np.random.Generator(np.random.PCG64(77))
    rows = np.sort(rng.choice(len(Xs), size=min(nsample, len(Xs)), replace=False))
    X = oracle.Data.from_dense(Xs)
    ri = oracle.rinv(X)
    km = skm.KMeans.dense(Xd, k, variant="standard", init_rows=init, precision=precision)
    prev = np.full(len(Xs), -1, np.int32)
    out = []
    for t in range(1, iters + 1):
        C = km.centers()
        ch = km.assign()
        lab = km.labels()
        if t in check_at:
            want, gap = oracle_assign_rows(Xs, rows, C, prev[rows])
            diff = want != lab[rows]
            e = {"iteration": t, "rows": int(len(rows)), "label_mismatches": int(np.sum(diff & (gap >= 1e-6))),
                 "near_ties": int(np.sum(diff & (gap < 1e-6)))}
        if ch == 0:
            if t in check_at:
                out.append(e)
            break
        J = km.update_centers()
        if t in check_at:
            Co, _, Jo = oracle.update(X, ri, lab, C.astype(np.float64))
            e["center_max_err"] = float(np.max(np.linalg.norm(km.centers().astype(np.float64) - Co, axis=1)))
            e["objective_rel_err"] = float(abs(J - Jo) / abs(Jo))
            out.append(e)
        prev = lab
    km.close()
    return out


def run_embed(args, rank, world, local):
    """Precision form on dense embeddings: n = 1e6 unit rows in d = 384 from a
    mixture of 1000 vMF(kappa = 40) components, k = 1000; FP32 GEMM vs the
    BF16 tensor-core bulk with FP32 recheck, standard and Hamerly.  Each path
    is timed over `embed_repeats` runs (L2 flushed before each), and the BF16
    path's results are compared with the FP64 oracle."""
    import torch
    from paper_2107_04074_gb300 import skm

    torch.cuda.set_device(local)
    n, d, k, iters = args.embed_n, 384, 1000, args.embed_iters
    Xs = synth.vmf(n, d, 1000, 40.0, seed=3)
    init = synth.init_rows(n, k, 3)
    X = torch.from_numpy(Xs).cuda()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    res, labels = {}, {}
    for variant, prec in (("standard", "fp32"), ("standard", "bf16"), ("hamerly", "fp32"), ("hamerly", "bf16"),
                          ("standard", "fp8"), ("hamerly", "fp8")):
        km = skm.KMeans.dense(X, k, variant=variant, init_rows=init, precision=prec, stream=stream.cuda_stream)
        km.reset(init)
        km.run(2)  # warm-up
        times = []
        for _ in range(max(1, args.embed_repeats)):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            km.reset(init)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            it, J = km.run(iters)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = float(np.median(times))
        labels[(variant, prec)] = km.labels()
        # per-iteration recheck counts and kernel times (separate, profiled run)
        km.reset(init)
        rech, cand, prof = [], [], {}
        for _ in range(it):
            km.profile(True)
            ch = km.assign()
            st = km.stats()
            for nm, (t, c) in km.profile_read().items():
                prof.setdefault(nm, [0.0, 0])
                prof[nm][0] += t
                prof[nm][1] += c
            km.profile(False)
            rech.append(st.last_rechecks)
            cand.append(st.last_cand_rechecks)
            if ch == 0:
                break
            km.update_centers()
        km.close()
        entry = {"iters": it, "ms": round(ms, 3), "iters_per_s": round(it / (ms / 1e3), 3), "objective": J,
                 "repeats": len(times), "ms_min_max": [round(min(times), 3), round(max(times), 3)],
                 "rows_whole_row_recheck_per_iter": rech,
                 "rows_candidate_recheck_per_iter": cand,
                 "kernels_ms": {nm: round(v[0], 3) for nm, v in sorted(prof.items(), key=lambda kv: -kv[1][0])}}
        if "k_dense_top2" in prof and prec == "fp32" and variant == "standard":
            t_ms, c = prof["k_dense_top2"]
            entry["fp32_gemm_tflops"] = round(2.0 * n * k * d / (t_ms / c / 1e3) / 1e12, 1)
        for kn, tag in (("k_bf16_topk", "bf16"), ("k_fp8_topk", "fp8")):
            if kn in prof:
                t_ms, c = prof[kn]
                flops = 2.0 * n * k * d  # the method's work; the kernel also multiplies padding centers up to 1024
                entry[f"{tag}_gemm_us_per_launch"] = round(t_ms / c * 1e3, 1)
                entry[f"{tag}_gemm_tflops"] = round(flops / (t_ms / c / 1e3) / 1e12, 1)
        if prec != "fp32":
            # rows whose reduced-precision top-2 did not decide the label (the
            # whole-row rechecks are a subset of them)
            entry["ambiguous_fraction_per_iter"] = [round(b / n, 4) for b in cand]
        res[f"{variant}/{prec}"] = entry
    ref = labels[("standard", "fp32")]
    same = all(np.array_equal(v, ref) for v in labels.values())
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        peak = 1900.0
    g = res["standard/bf16"]
    traffic = recorded_traffic("k_bf16_topk", "vmf-n1e6-d384-k1000") if n == 1_000_000 else None
    pk = measured_peaks(skm, torch)
    fp32_peak = pk["fp32_fma_tflops"]
    if pk.get("fp8_gemm_tflops"):
        fp8_peak, fp8_src = pk["fp8_gemm_tflops"], "measured (cuBLAS E4M3 GEMM via torch._scaled_mm, burst)"
    else:
        fp8_peak, fp8_src = 2 * peak, "2 x the measured BF16 burst peak (nominal FP8:BF16 ratio)"
    f32 = res["standard/fp32"].get("fp32_gemm_tflops")
    fp32_roof = {"kernel": "k_dense_top2", "bound": "alu", "achieved": f32, "peak": round(fp32_peak, 1),
                 "unit": "TFLOP/s", "frac": round(f32 / fp32_peak, 4) if f32 else None,
                 "peak_source": "measured (skm_measure_peak FP32 FMA)", "flops_per_launch": 2 * n * k * d}
    errors = {}
    if not args.no_oracle_check:
        for prec in ("bf16", "fp8", "fp32"):
            errors[prec] = embed_error_vs_oracle(skm, X, Xs, k, init, iters, prec)
    return {"workload": f"vmf-embeddings n={n} d={d} k={k} kappa=40 ({iters} iterations max)",
            "labels_identical_across_paths": same, "paths": res, "measured_peaks": pk,
            "speedup_bf16_vs_fp32_standard": round(g["iters_per_s"] / res["standard/fp32"]["iters_per_s"], 2),
            "speedup_fp8_vs_fp32_standard": round(res["standard/fp8"]["iters_per_s"] /
                                                  res["standard/fp32"]["iters_per_s"], 2),
            "error_vs_fp64_oracle": errors,
            "fp32_gemm_roofline": fp32_roof,
            "fp8_gemm_roofline": {"kernel": "k_fp8_topk", "bound": "tensor",
                                  "achieved": res["standard/fp8"].get("fp8_gemm_tflops"), "peak": fp8_peak,
                                  "unit": "TFLOP/s", "peak_source": fp8_src,
                                  "frac": round(res["standard/fp8"].get("fp8_gemm_tflops", 0) / fp8_peak, 4),
                                  "traffic": None, "flops_per_launch": 2 * n * k * d},
            "bf16_gemm_roofline": {"kernel": "k_bf16_topk", "bound": "tensor", "achieved": g.get("bf16_gemm_tflops"),
                                   "peak": peak, "unit": "TFLOP/s", "peak_source": "measured (burst)",
                                   "frac": round(g.get("bf16_gemm_tflops", 0) / peak, 4), "traffic": traffic,
                                   "flops_per_launch": 2 * n * k * d,
                                   "traffic_note": "ncu DRAM bytes of an n=2e5 launch scaled by rows"}}


def run_batch(args, rank, world, local):
    """Batched form: 64 independent runs (n_r lognormal over [5e3, 2e5],
    d = 2e4, k_r uniform over {10, 50, 100, 250, 500}, at most 50 iterations
    each) in one context -- Elkan bounds (and Simplified Elkan beside it), one
    launch per phase for all runs, the iteration replayed as a CUDA graph,
    launch shape autotuned -- against the plain FP32 standard variant run by
    run (one context each, one after the other), at identical labels."""
    import tempfile

    import torch
    from paper_2107_04074_gb300 import skm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nruns, iters = args.batch_runs, 50
    cfgs, ks = synth.batch_runs(nruns)
    parts = [synth.tfidf(c) for c in cfgs]
    X, run_rows = synth.concat(parts)
    inits = [synth.init_rows(p.n, int(k), 1000 + r) for r, (p, k) in enumerate(zip(parts, ks))]
    init_all = np.concatenate(inits)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    Xd = [torch.from_numpy(a).to(dev) for a in (X.row_ptr, X.col, X.val)]
    cache = os.path.join(tempfile.gettempdir(), "skm_autotune.txt")
    sampler = ClockSampler(local)
    sampler.start()
    per_variant, lab_b = {}, {}
    for variant in ("elkan", "simp_elkan"):
        b = skm.Batch(X.n, X.d, *Xd, run_rows, ks, variant=variant, init_rows=init_all, graph=True,
                      stream=stream.cuda_stream)
        t0 = time.perf_counter()
        from_cache = b.autotune(cache, iters=3)
        tune_s = time.perf_counter() - t0
        for _ in range(args.warmup):
            b.reset(init_all)
            b.run(iters)
        ms_b, its = 0.0, []
        l0 = skm.kernel_launches()
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.reset(init_all)
            it, J = b.run(iters)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_b += e0.elapsed_time(e1)
            its.append(it)
        launches = skm.kernel_launches() - l0
        lab_b[variant] = b.labels()
        sims = b.stats().total_sims
        # kernel shares of one eager run with per-kernel events
        b.reset(init_all)
        prof = profiled_run(b, iters)
        b.close()
        per_step = ms_b / args.steps
        tot = sum(v[0] for v in prof.values()) or 1.0
        per_variant[variant] = {
            "batch_ms_per_step": round(per_step, 3), "batch_iterations": its[-1],
            "run_iterations_per_s": round(nruns * its[-1] / (per_step / 1e3), 1),
            "sims_evaluated": sims, "gpu_launches_per_step": int(launches / args.steps),
            "autotune": {"from_cache": from_cache, "seconds": round(tune_s, 2)},
            "kernel_time_share": {nm: {"ms": round(v[0], 3), "launches": v[1], "share": round(v[0] / tot, 4)}
                                  for nm, v in sorted(prof.items(), key=lambda kv: -kv[1][0])[:12]}}
    clocks = sampler.stop()
    # the plain FP32 standard variant, run by run (contexts built outside the timing)
    ms_s, it_s, lab_s = 0.0, 0, []
    for r, p in enumerate(parts):
        pd = [torch.from_numpy(a).to(dev) for a in (p.row_ptr, p.col, p.val)]
        km = skm.KMeans(p.n, p.d, *pd, int(ks[r]), variant="standard", init_rows=inits[r],
                        stream=stream.cuda_stream)
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it, _ = km.run(iters)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_s += e0.elapsed_time(e1)
        it_s += it
        lab_s.append(km.labels())
        km.close()
    ref = np.concatenate(lab_s)
    for v, e in per_variant.items():
        e["labels_identical_to_standard"] = bool(np.array_equal(lab_b[v], ref))
        e["speedup_vs_sequential_standard"] = round(ms_s / e["batch_ms_per_step"], 2)
    head = per_variant["elkan"]
    return {"workload": f"{nruns} sparse TF-IDF runs, n_r in [5e3, 2e5] (sum {X.n}, {X.nnz} nnz), d=20000, "
                        f"k_r in {{10,50,100,250,500}} (sum {int(ks.sum())}), at most {iters} iterations each",
            "variant": "elkan", **{kk: vv for kk, vv in head.items() if kk != "kernel_time_share"},
            "sequential_standard_ms": round(ms_s, 3), "sequential_standard_run_iterations": it_s,
            "variants": per_variant, "clocks": clocks}


def sampled_parity(km, csr, sample, prev, C):
    """Teacher-forced check of the assignment just made from centers C on the
    sampled rows against the FP64 oracle (labels differ only below the 1e-6
    similarity gap).  Returns (rows checked, mismatches, near-ties)."""
    import oracle
    sub = csr.rows(sample)
    X = oracle.Data.from_csr(sub)
    want, _, _, _, gap = oracle.assign(X, oracle.rinv(X), C.astype(np.float64), prev[sample])
    lab = km.labels()[sample]
    diff = want != lab
    return int(len(sample)), int(np.sum(diff & (gap >= 1e-6))), int(np.sum(diff & (gap < 1e-6)))


def elk_bound_bytes(n, k, u_width=4):
    """Algorithmic bytes of one Elkan bound launch: the n x k upper bounds of
    u_width bytes each read and written once, plus per point l read and
    written, a(i), delta_i and the row length (16 B)."""
    return 2 * u_width * n * k + 16 * n


def elk_u_width(skm, n, k):
    """Stored bytes per Elkan upper bound, from skm_bound_bytes (4n + w n k)."""
    return (skm.bound_bytes("elkan", n, k) - 4 * n) // (n * k)


def skipped_name(nm, st):
    """A launch of the pass the library skipped in this assignment (Elkan's
    bound pass, Hamerly's tightening: the kernel only forwards every survivor
    to the whole-row list) is reported under its own name, so that the
    kernel's bytes per launch describe the passes that streamed the bounds."""
    if st.last_skipped and nm in ("k_elk_bounds", "k_ham_tighten"):
        return nm + "(skipped)"
    return nm


def profiled_run(km, iters):
    """One eager run with per-kernel CUDA events (not a timed value): per kernel
    its summed ms and launches."""
    prof = {}
    for _ in range(iters):
        km.profile(True)
        ch = km.assign()
        st = km.stats()
        if ch:
            km.update_centers()
        for nm, (t, c) in km.profile_read().items():
            nm = skipped_name(nm, st)
            prof.setdefault(nm, [0.0, 0])
            prof[nm][0] += t
            prof[nm][1] += c
        km.profile(False)
        if ch == 0:
            break
    return prof


def run_large(args, rank, world, local):
    """Large sparse workload: n = 4e6 rows, d = 2e5, nnz/row lognormal(200,
    0.9) clipped to [10, 5000] (~8e8 nnz), Zipf(1.05), FP16 values, k = 1000,
    30 iterations; Elkan, Simplified Elkan, Hamerly and standard at identical
    labels, with the first and last assignments of the Elkan run checked
    against the FP64 oracle on 2000 sampled rows, and the Elkan bound kernel's
    HBM rate (its n x k bound array, 16 GB, is far larger than L2)."""
    import torch
    from paper_2107_04074_gb300 import skm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = synth.CSR_LARGE
    if args.large_frac < 1.0:
        cfg = synth.scaled(cfg, n=int(cfg.n * args.large_frac))
    t0 = time.perf_counter()
    csr = synth.tfidf(cfg)
    gen_s = time.perf_counter() - t0
    k, iters = 1000, 30
    init = synth.init_rows(csr.n, k, cfg.seed)
    stream = torch.cuda.current_stream(dev)
    Xd = [torch.from_numpy(a).to(dev) for a in (csr.row_ptr, csr.col, csr.val)]
    rng = np.random.Generator(np.random.PCG64(55))
    sample = np.sort(rng.choice(csr.n, size=min(2000, csr.n), replace=False))
    try:
        hbm_peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
        peak_src = "measured"
    except (OSError, KeyError, ValueError):
        hbm_peak, peak_src = 6800.0, "fallback"
    res, labels, bound_roof = {}, {}, {}
    sampler = ClockSampler(local)
    sampler.start()
    for variant in ("elkan", "simp_elkan", "hamerly", "standard"):
        km = skm.KMeans(csr.n, csr.d, *Xd, k, variant=variant, init_rows=init, stream=stream.cuda_stream,
                        screen=screen_opt(args))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it, J = km.run(iters)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        labels[variant] = km.labels()
        res[variant] = {"iterations": it, "ms": round(ms, 1), "iters_per_s": round(it / (ms / 1e3), 3),
                        "sims_evaluated": km.stats().total_sims, "objective": J}
        if variant in ("elkan", "simp_elkan"):
            km.reset(init)
            prof = profiled_run(km, iters)
            tot = sum(v[0] for v in prof.values()) or 1.0
            res[variant]["kernel_time_share"] = {
                nm: {"ms": round(v[0], 2), "launches": v[1], "share": round(v[0] / tot, 4)}
                for nm, v in sorted(prof.items(), key=lambda kv: -kv[1][0])[:8]}
            if "k_elk_bounds" in prof:
                t_ms, c = prof["k_elk_bounds"]
                ab = elk_bound_bytes(csr.n, k, elk_u_width(skm, csr.n, k))
                ach = ab / (t_ms / c / 1e3) / 1e9
                bound_roof[variant] = {"kernel": "k_elk_bounds", "bound": "hbm", "achieved": round(ach, 1),
                                       "peak": hbm_peak, "unit": "GB/s", "frac": round(ach / hbm_peak, 4),
                                       "peak_source": peak_src, "avg_launch_us": round(t_ms / c * 1e3, 1),
                                       "launches": c, "algorithmic_bytes_per_launch": int(ab),
                                       "traffic": recorded_traffic("k_elk_bounds", "large-n4e6-k1000")}
        if variant == "elkan":
            # teacher-forced oracle checks of the first and the last assignment
            km.reset(init)
            prev = np.full(csr.n, -1, np.int32)
            checks = []
            for t in range(it):
                C = km.centers() if t in (0, it - 1) else None
                km.assign()
                if C is not None:
                    checks.append({"iteration": t + 1, **dict(zip(("rows", "mismatches", "near_ties"),
                                                                  sampled_parity(km, csr, sample, prev, C)))})
                if t == it - 2:
                    prev = km.labels()
                if t < it - 1:
                    km.update_centers()
            res[variant]["oracle_sample"] = checks
        km.close()
    clocks = sampler.stop()
    same = all(np.array_equal(v, labels["standard"]) for v in labels.values())
    std = res["standard"]["iters_per_s"]
    return {"workload": f"large sparse n={csr.n} d={csr.d} nnz={csr.nnz} (FP16 values) k={k} "
                        f"{iters} iterations", "generate_s": round(gen_s, 1), "labels_identical": same,
            "variants": res, "bound_kernel_roofline": bound_roof, "clocks": clocks,
            "speedup_vs_standard": {v: round(res[v]["iters_per_s"] / std, 3) for v in res if v != "standard"}}


def summarize_large(args, rank, world, local):
    a = argparse.Namespace(**vars(args))
    a.large_frac = 1.0
    return run_large(a, rank, world, local)


def csr_slice(csr, a, b):
    """Rows [a, b) of a CSR as their own CSR (views of the arrays)."""
    rp = csr.row_ptr[a:b + 1] - csr.row_ptr[a]
    return synth.CSR(b - a, csr.d, rp, csr.col[csr.row_ptr[a]:csr.row_ptr[b]],
                     csr.val[csr.row_ptr[a]:csr.row_ptr[b]])


def oracle_standard_all_cores(csr, init, iters=2, threads=None):
    """The FP64 oracle's standard iterations with one host thread per core:
    its assignment runs on contiguous row blocks in parallel (the oracle's C
    code releases the interpreter lock; its arithmetic is untouched), then its
    center update over all rows.  Returns (iterations/s, threads, seconds)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    P = threads or os.cpu_count() or 1
    X = oracle.Data.from_csr(csr)
    ri = oracle.rinv(X)
    C = oracle.unit_rows(X, init)
    cuts = np.linspace(0, csr.n, P + 1).astype(np.int64)
    parts = [oracle.Data.from_csr(csr_slice(csr, int(a), int(b))) for a, b in zip(cuts[:-1], cuts[1:])]
    ris = [ri[a:b] for a, b in zip(cuts[:-1], cuts[1:])]
    lab = np.full(csr.n, -1, np.int32)
    with ThreadPoolExecutor(max_workers=P) as pool:
        t0 = time.perf_counter()
        for _ in range(iters):
            outs = list(pool.map(lambda q: oracle.assign(parts[q], ris[q], C, lab[cuts[q]:cuts[q + 1]])[0],
                                 range(P)))
            lab = np.concatenate(outs)
            C, _, _ = oracle.update(X, ri, lab, C)
        dt = time.perf_counter() - t0
    return iters / dt, P, dt


def cpu_baseline(csr, init, variant, iters=3):
    """The FP64 oracle as it stands, single-threaded, on a bounded sample: the
    first `iters` iterations of the same run on the full data; beside it the
    oracle's standard iterations on all host cores."""
    import oracle
    X = oracle.Data.from_csr(csr)
    C0 = oracle.unit_rows(X, init)
    t0 = time.perf_counter()
    tr = oracle.run(X, C0, variant, max_iters=iters)
    dt = time.perf_counter() - t0
    v_all, P, dt_all = oracle_standard_all_cores(csr, init)
    return {"value": round(tr.iters / dt, 4), "unit": "Lloyd iterations/s", "cores": 1, "kind": "oracle",
            "sample": f"first {tr.iters} {variant} iterations of the same run on the full data "
                      f"(early iterations prune least), {dt:.1f} s",
            "host_cpu_count": os.cpu_count(),
            "all_cores": {"value": round(v_all, 4), "unit": "Lloyd iterations/s", "cores": P, "kind": "oracle",
                          "variant": "standard",
                          "sample": f"first 2 standard iterations on the full data, assignment parallel over "
                                    f"row blocks ({P} threads), {dt_all:.1f} s"}}


def run_reference(args, rank, world):
    """The oracle arm: each step = the first 2 iterations of the run (FP64, one
    host core)."""
    import oracle
    cfg = workload_cfg()
    csr = synth.tfidf(cfg)
    init = synth.init_rows(csr.n, K_CLUSTERS, INIT_SEED)
    X = oracle.Data.from_csr(csr)
    C0 = oracle.unit_rows(X, init)
    ri = oracle.rinv(X)
    per_step = 2
    for _ in range(args.warmup):
        oracle.run(X, C0, args.variant, max_iters=1, ri=ri)
    t0 = time.perf_counter()
    its = 0
    for _ in range(args.steps):
        its += oracle.run(X, C0, args.variant, max_iters=per_step, ri=ri).iters
    dt = time.perf_counter() - t0
    v = its / dt
    return {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "Lloyd iterations/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt * 1e3 / args.steps, 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_block(cfg, args.variant, "n/a (CPU)"),
            "cpu_baseline": {"value": round(v, 4), "unit": "Lloyd iterations/s", "cores": 1, "kind": "oracle",
                             "sample": f"each step = the first {per_step} {args.variant} iterations, full data"},
            "e2e": {"value": round(v, 4), "unit": "Lloyd iterations/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variant", default="simp_elkan", choices=["standard", "hamerly", "elkan", "simp_hamerly",
                                                                 "simp_elkan", "yinyang"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="eager iterations (one host sync each) instead of the "
                                                             "CUDA-graph replay")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the precision-form and batched-form summaries of the default line")
    ap.add_argument("--quick", action="store_true",
                    help="only the timed runs of the chosen variant (for profiler captures)")
    ap.add_argument("--workload", default="rcv1", choices=["rcv1", "embed", "batch", "large"],
                    help="rcv1: the bench line; embed: the dense precision-form measurement; "
                         "batch: the batched form; large: the 8e8-nonzero sparse workload")
    ap.add_argument("--batch-runs", type=int, default=64)
    ap.add_argument("--large-frac", type=float, default=1.0, help="fraction of the large workload's rows")
    ap.add_argument("--embed-n", type=int, default=1_000_000)
    ap.add_argument("--embed-iters", type=int, default=20)
    ap.add_argument("--embed-repeats", type=int, default=5)
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the precision form's per-result comparison with the FP64 oracle")
    ap.add_argument("--screen", type=int, default=None, choices=[0, 1],
                    help="Elkan variants: screen whole-row recomputes against FP16 centers (1) or not (0); "
                         "default: the library's choice (on for k > 128)")
    ap.add_argument("--trace", action="store_true",
                    help="print a per-iteration table (labels changed, similarities, survivors, kernel ms) and exit")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)), flush=True)
        return
    if args.workload == "embed":
        if rank == 0:
            print(json.dumps(run_embed(args, rank, world, local)), flush=True)
        return
    if args.workload == "batch":
        if rank == 0:
            print(json.dumps(run_batch(args, rank, world, local)), flush=True)
        return
    if args.workload == "large":
        if rank == 0:
            print(json.dumps(run_large(args, rank, world, local)), flush=True)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world, local)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
