#!/usr/bin/env python3
"""Throughput of PERMANOVA's s_W on GB300: pair-permutation evaluations/s.

A step is one permanova_sW call over one batch of label rows of the workload
(all kernels of the path: label packing/validation, the dominant s_W kernel,
the FP64 cross-tile reduction).  The default workload is n = 100,000 objects
(Gaussian points in R^16, Euclidean fp32 distances, 40 GB), K = 10 groups with
Dirichlet(2) sizes and 99,999 permutations in uint8 labels, processed in
batches of 8,192 label rows per step; D (40 GB) is far larger than L2, so no
flush is needed between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "pair-perm evals/s for s_W at n=100k"
UNIT = "pair-perm evals/s"
WORKLOADS = {
    "euclid-100k": dict(batch=8192),
    "braycurtis-50k": dict(batch=8192),
    "euclid-20k": dict(batch=4000),
    "jaccard-25k": dict(batch=4000),
    "euclid-1k": dict(batch=1000),
}
L2_BYTES = 129 << 20


def host_matrix_bytes(n: int, ld: int) -> int:
    """Bytes of D that permanova_sW_host copies with the tensor-core form: for
    each 128-row band whose trapezoid rows span at least half the width, its
    flat host range from the diagonal element to the end of its last row (the
    rows' lower-left parts come along in one flat copy); for the later bands,
    the trapezoid alone (one two-dimensional copy)."""
    total = 0
    for r0 in range(0, n, 128):
        rows, width = min(128, n - r0), n - r0
        total += (rows * width if 2 * width < n else (rows - 1) * ld + width) * 4
    return total


def peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0, "source": "fallback"}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            try:
                power.append(float(parts[2]))
            except ValueError:
                pass
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w": statistics.median(power) if power else None,
                "power_w_max": max(power) if power else None}


def gpu_query_id(torch, dev: int) -> str | None:
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        if u and u != "None":
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if vis:
        first = vis.split(",")[dev] if dev < len(vis.split(",")) else ""
        return first or None
    return None


# ---------------------------------------------------------------------------
# the oracle on a bounded sample (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_rate(cfg: dict, X: np.ndarray, label_rows: np.ndarray, target_s: float,
                extras: bool = True) -> dict:
    """Time the FP64 oracle on the leading n_s x n_s block of the workload:
    Algorithm 1 on all host threads (the reported value, one label row per
    thread, the row count sized so the run takes about ``target_s`` seconds),
    Algorithm 1 on one thread, and Algorithm 2 (tiled, 64 x 64) on all
    threads and, as the paper's CPU method, in FP32 (with ``extras``), each a
    bounded sample of label rows."""
    import oracle
    T = oracle.max_threads()
    K = cfg["K"]
    w = cfg["w"].astype(np.float64)

    ns = min(X.shape[0], 4096 if cfg["kind"] == "braycurtis" else 16384)
    D = synth.recipe_matrix_host(cfg, X[:ns])
    pairs_s = ns * (ns - 1) / 2

    def rows_for(R: int) -> np.ndarray:
        return np.ascontiguousarray(np.resize(label_rows[:, :ns], (R, ns)).astype(np.int32) % K)

    def run(R: int, threads: int, alg: int = 1) -> float:
        rows = rows_for(R)
        t0 = time.perf_counter()
        if alg == 1:
            oracle.sW_alg1(D, rows, K, w, threads=threads)
        elif alg == 2:
            oracle.sW_alg2(D, rows, K, w, 64, threads=threads)
        else:
            oracle.sW_alg2_f32(D, rows, K, w, 64, threads=threads)
        return time.perf_counter() - t0

    R = T
    t = run(R, T)
    rate = R * pairs_s / max(t, 1e-6)
    if t < target_s / 3:
        R = T * max(1, int(round(target_s * rate / pairs_s / T)))
        R = min(R, 64 * T)
        t = run(R, T)
        rate = R * pairs_s / t
    res = {"value": rate, "unit": UNIT, "cores": T, "kind": "oracle", "seconds": t,
           "sample": f"FP64 Algorithm-1 oracle on the leading {ns}x{ns} block of the workload's "
                     f"matrix with {R} label rows ({T} threads), {t:.1f} s"}
    if extras:
        # one thread, a few rows; Algorithm 2 on all threads, one row per thread
        r1 = max(1, min(8, int(round(target_s / 3 * rate / T / pairs_s))))
        t1 = run(r1, 1)
        t2 = run(T, T, alg=2)
        t3 = run(T, T, alg=3)
        res["single_thread"] = {"value": r1 * pairs_s / t1,
                                "sample": f"Algorithm 1, {r1} label rows, 1 thread, {t1:.1f} s"}
        res["alg2_tiled"] = {"value": T * pairs_s / t2, "sample": f"Algorithm 2 (64 x 64 tiles), "
                             f"{T} label rows, {T} threads, {t2:.1f} s"}
        res["alg2_tiled_fp32"] = {"value": T * pairs_s / t3,
                                  "sample": f"the paper's CPU method: Algorithm 2 (64 x 64 tiles) "
                                            f"with FP32 values, {T} label rows, {T} threads, {t3:.1f} s"}
        res["cpu_model"] = cpu_model()
    return res


# ---------------------------------------------------------------------------
def roofline(form: str, K: int, evals_per_launch: float, kernel_ms: float, pk: dict,
             traffic: float | None) -> dict:
    s = kernel_ms / 1e3
    if form == "gemm":
        flops = 4.0 * K * evals_per_launch          # two 16-bit planes (hi, lo) x 2K flops per pair-perm
        achieved = flops / s / 1e12
        peak = pk["bf16_tflops_sustained"]
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_source": pk["source"] + " (sustained bf16)"}
    if form == "permblock":
        ops = 2.0 * evals_per_launch                 # one compare + one add per pair-perm
        achieved = ops / s / 1e12
        peak = 152 * 128 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tlane-op/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_source": "152 SMs x 128 FP32 lanes x max SM clock"}
    byts = 4.0 * evals_per_launch                    # fp32 d_ij re-read per label row
    achieved = byts / s / 1e9
    peak = pk["hbm_gbs"]
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "peak_source": pk["source"] + " (copy)"}


def traffic_per_launch(form: str, evals: float, workload: str | None = None) -> float | None:
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source and (when the record names one) on this
    workload: bytes per pair-perm evaluation x evaluations.  The bytes per
    evaluation of the cached forms depend on n (L2 reuse), so a record is
    only applied to the workload it was measured on."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    src = {"gemm": "k_gemm.cu", "permblock": "k_permblock.cu", "brute": "k_brute.cu"}[form]
    with open(os.path.join(ROOT, "paper_2505_04556_gb300", "csrc", src), "rb") as f:
        sha = hashlib.sha1(f.read()).hexdigest()[:12]
    for line in open(path):
        kv = dict(tok.split("=", 1) for tok in line.split() if "=" in tok)
        if kv.get("form") == form and kv.get("src_sha") == sha and "bytes_per_eval" in kv:
            if workload is not None and kv.get("workload", workload) != workload:
                continue
            return float(kv["bytes_per_eval"]) * evals
    return None


def combine_ranks(elapsed: float, units: float) -> tuple[float, float]:
    """Across torch.distributed ranks: the max elapsed time and the summed
    units (replicas: no data is exchanged, only these two numbers)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return elapsed, units
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([elapsed], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def rank_seed(base: int, rank: int) -> int:
    """Label-row seed of a rank: ranks draw disjoint streams of label rows."""
    return base + 1000 * rank


def _guarded(fn):
    """fn() or, if it raises, {"error": its message} (after clearing the GPU's
    cached allocations), so one failed extra measurement does not lose the
    bench line."""
    try:
        return fn()
    except Exception as e:  # noqa: BLE001 - recorded in the line
        try:
            import torch
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
        except Exception:
            pass
        return {"error": f"{type(e).__name__}: {e}"[:300]}


def forms_compare(pk: dict, reps: int = 3, workload: str = "euclid-20k", cases=None,
                  idx=(0, 1, 63, 127, 255, 256, 300, 511)) -> dict:
    """Kernel forms on one workload in the same run (default euclid-20k, n =
    20,000, K = 4: every form, 4,000 label rows, 512 for the brute force,
    which re-reads D from HBM per row), the dominant kernel timed with CUDA
    events inside the library (mean of ``reps`` launches after one warm-up;
    D is larger than L2), each form's roofline fraction, and its relative
    errors against the FP64 oracle on the label rows ``idx`` every form
    computes (largest, and mean signed)."""
    import torch
    import oracle
    import paper_2505_04556_gb300 as pm
    if cases is None:
        cases = [("brute", dict(form=pm.FORM_BRUTE), 512),
                 ("permblock_pair", dict(form=pm.FORM_PERMBLOCK, permblock_variant=0), 4000),
                 ("permblock_f32", dict(form=pm.FORM_PERMBLOCK, permblock_variant=1), 4000),
                 ("gemm", dict(form=pm.FORM_GEMM), 4000)]
    cfg = synth.recipe(workload)
    n, K = cfg["n"], cfg["K"]
    X = synth.recipe_points(cfg)
    D = synth.recipe_matrix_device(cfg, X)
    n_rows = max(rows for _, _, rows in cases)
    lab = synth.device_label_rows(cfg["labels"], n_rows, cfg["seed_perms"], dtype=torch.uint8)
    w = torch.from_numpy(cfg["w"]).cuda()
    idx = np.array(idx)
    ref = oracle.sW_alg1(D.cpu().numpy(), lab[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.int32), K,
                         cfg["w"].astype(np.float64))
    pairs = n * (n - 1) / 2
    out = {"workload": workload, "n": n, "K": K, "error_rows": idx.tolist()}
    with pm.Context(0) as ctx:
        for name, plan, rows in cases:
            pm.permanova_set_plan(ctx.handle, **plan)
            res = torch.empty(rows, dtype=torch.float64, device="cuda")
            pm.permanova_sW(ctx.handle, D, n, n, lab[:rows], pm.LABEL_U8, K, rows, w, res)
            pm.permanova_sync(ctx.handle)
            pm.permanova_profile_enable(ctx.handle, True)
            for _ in range(reps):
                pm.permanova_sW(ctx.handle, D, n, n, lab[:rows], pm.LABEL_U8, K, rows, w, res)
            prof = pm.permanova_profile_read(ctx.handle)
            pm.permanova_profile_enable(ctx.handle, False)
            pm.permanova_sync(ctx.handle)
            ms = prof["main_kernel_ms"] / max(1, prof["main_kernel_launches"])
            evals = pairs * rows
            rl = roofline("gemm" if name == "gemm" else "permblock" if name.startswith("permblock")
                          else "brute", K, evals, ms, pk, None)
            rel = (res.cpu().numpy()[idx] - ref) / ref
            out[name] = {"evals_per_s": evals / (ms / 1e3), "kernel_ms": ms, "rows": rows,
                         "roofline_frac": rl["frac"], "bound": rl["bound"],
                         "max_rel_err_vs_oracle": float(np.max(np.abs(rel))),
                         "mean_rel_err_vs_oracle": float(np.mean(rel))}
        pm.permanova_set_plan(ctx.handle, pm.FORM_AUTO)
    fp32 = [out[c]["evals_per_s"] for c in ("permblock_pair", "permblock_f32") if c in out]
    out["gemm_over_best_fp32"] = out["gemm"]["evals_per_s"] / max(fp32)
    del D, lab
    torch.cuda.empty_cache()
    return out


def precision_compare(pk: dict) -> dict:
    """The precision configuration: braycurtis-50k (n = 50,000 Bray-Curtis
    distances in [0, 1], K = 8): the split-BF16 tensor-core form against the
    plain FP32 CUDA-core kernel on the same 4,000 label rows, each with its
    errors against the FP64 oracle on eight rows spread over the launch."""
    import paper_2505_04556_gb300 as pm
    cases = [("permblock_pair", dict(form=pm.FORM_PERMBLOCK, permblock_variant=0), 4000),
             ("gemm", dict(form=pm.FORM_GEMM), 4000)]
    return forms_compare(pk, reps=2, workload="braycurtis-50k", cases=cases,
                         idx=(0, 1, 127, 128, 255, 1000, 2047, 3999))


def serving_run(rate: float, duration: float, slots: int, warmup_s: float = 3.0,
                seed: int = 5005, burst_tests: int = 600, sweep: tuple = (30.0, 120.0, 160.0),
                sweep_duration: float = 6.0, sweep_warmup_s: float = 1.5) -> dict:
    """Serving workload: 64 resident matrices (n log-uniform in 500..30,000,
    Gaussian points in R^16/R^32, Euclidean fp32), each with 1-20 categorical
    factors (K uniform in 2..12, Dirichlet(2) sizes, each group >= 2), tests of
    999 or 9,999 permutations (even odds) arriving as a Poisson process at
    ``rate`` tests/s, served with prepared matrices (each matrix's operands
    made on its first request).  Arrivals during the first ``warmup_s`` seconds are
    served but not counted; tests/s and p50/p99 latency (arrival to result)
    are taken over the ``duration`` seconds after that.  The same server then
    takes the offered rates in ``sweep`` (shorter phases, each drained before
    the next) to show where p99 turns up.  Then ``burst_tests`` tests of the
    same mix are submitted at once: completed tests / time to the last result
    is the server's capacity."""
    import torch
    import paper_2505_04556_gb300 as pm
    from paper_2505_04556_gb300.serve import Request, Server
    pm.build()
    rng = np.random.default_rng(seed)
    mats, factors = {}, {}
    for m in range(64):
        n = int(round(math.exp(rng.uniform(math.log(500), math.log(30000)))))
        dim = 16 if m % 2 == 0 else 32
        X = rng.standard_normal((n, dim))
        cfg = {"kind": "euclid"}
        mats[m] = synth.recipe_matrix_device(cfg, X)
        fl = []
        for _ in range(int(rng.integers(1, 21))):
            K = int(rng.integers(2, 13))
            sizes = synth.largest_remainder_sizes(n, rng.dirichlet(2.0 * np.ones(K)), min_size=2)
            fl.append((synth.observed_labels(sizes, int(rng.integers(1 << 30))), K))
        factors[m] = fl
    torch.cuda.synchronize()
    resident = sum(int(D.numel()) * 4 for D in mats.values())
    srv = Server(mats, n_slots=slots, reserve_per_slot=8 << 30, prepare=True)
    k = 0

    def draw():
        m = int(rng.integers(64))
        lab, K = factors[m][int(rng.integers(len(factors[m])))]
        P = 999 if rng.random() < 0.5 else 9999
        return m, lab, K, P

    def phase(rate_, warm, dur):
        """Poisson arrivals at rate_ for warm + dur seconds; the arrivals after
        the warm-up are measured; waits for every result."""
        nonlocal k
        reqs, measured = [], []
        t0 = time.perf_counter()
        t_next = t0
        while True:
            t_next += rng.exponential(1.0 / rate_)
            if t_next - t0 > warm + dur:
                break
            while time.perf_counter() < t_next:
                time.sleep(min(0.002, max(0.0, t_next - time.perf_counter())))
            m, lab, K, P = draw()
            r = srv.submit(Request(m, lab, K, P, seed=10_000 + k))
            reqs.append(r)
            if t_next - t0 >= warm:
                measured.append(r)
            k += 1
        for r in reqs:
            r.done.wait(600)
        wall = max(r.t_done for r in measured) - (t0 + warm)
        return measured, wall

    measured, wall = phase(rate, warmup_s, duration)
    sweep_out = []
    for rt in sweep:
        meas_r, wall_r = phase(rt, sweep_warmup_s, sweep_duration)
        sr = Server.summarize(meas_r, wall_r)
        sweep_out.append({"offered_rate": rt, "tests_per_s": sr.get("tests_per_s"), "p50_s": sr.get("p50_s"),
                          "p99_s": sr.get("p99_s"), "tests": sr.get("tests"),
                          "mean_batch": sr.get("mean_batch")})
    # capacity: a burst of tests from the same mix submitted at once, timed
    # from the first submission to the last result (the server saturated)
    burst = []
    tb = time.perf_counter()
    for j in range(burst_tests):
        m, lab, K, P = draw()
        burst.append(srv.submit(Request(m, lab, K, P, seed=50_000 + j)))
    for r in burst:
        r.done.wait(600)
    burst_wall = max(r.t_done for r in burst) - tb
    burst_ok = sum(r.error is None for r in burst)
    srv.close()
    s = Server.summarize(measured, wall)
    evals = sum(mats[r.matrix_id].shape[0] * (mats[r.matrix_id].shape[0] - 1) / 2 * (r.n_perms + 1)
                for r in measured if r.error is None)
    out = {"metric": "served PERMANOVA tests/s (p50/p99 latency)", "value": s.get("tests_per_s"),
           "unit": "tests/s", "p50_s": s.get("p50_s"), "p99_s": s.get("p99_s"),
           "tests": s.get("tests"), "errors": s.get("errors"), "offered_rate": rate,
           "duration_s": duration, "warmup_s": warmup_s, "slots": slots,
           "mean_batch": s.get("mean_batch"), "pair_perm_evals_per_s": evals / wall,
           "sweep": sweep_out,
           "capacity_tests_per_s": burst_ok / burst_wall, "capacity_burst": burst_tests,
           "capacity_mean_batch": float(np.mean([r.batch_size for r in burst])),
           "matrices_resident": len(mats), "resident_gb": round(resident / 1e9, 1),
           "config": {"workload": "serving-64", "matrices": 64, "n_range": [500, 30000],
                      "perms": [999, 9999], "K_range": [2, 12], "factors_per_matrix": [1, 20],
                      "arrivals": "Poisson"}}
    del mats
    torch.cuda.empty_cache()
    return out


def serving_bench(args) -> None:
    """``--serving``: the serving workload alone, one JSON line."""
    import torch
    line = serving_run(args.rate, args.duration, args.slots)
    line.update({"higher_is_better": True, "n_gpus": 1, "data": "synthetic",
                 "gpu": torch.cuda.get_device_name(0),
                 "gpu_sms": torch.cuda.get_device_properties(0).multi_processor_count})
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--serving", action="store_true")
    ap.add_argument("--rate", type=float, default=60.0)
    ap.add_argument("--duration", type=float, default=12.0)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="euclid-100k", choices=sorted(WORKLOADS))
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--form", default="auto", choices=["auto", "brute", "permblock", "gemm"])
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-prepared", action="store_true")
    args = ap.parse_args()
    if args.serving:
        serving_bench(args)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    cfg = synth.recipe(args.workload)
    B = args.batch or WORKLOADS[args.workload]["batch"]
    B = min(B, cfg["P"])
    n, K, P = cfg["n"], cfg["K"], cfg["P"]
    pairs = n * (n - 1) / 2
    X = synth.recipe_points(cfg)

    if args.impl == "reference":
        if rank != 0:
            return
        # every step: the oracle on a bounded sample of the same workload
        rows = synth.shuffled_rows(cfg["labels"], 64, cfg["seed_perms"])
        per_step = max(2.0, 150.0 / max(1, args.steps + args.warmup))
        first = oracle_rate(cfg, X, rows, per_step)
        rates, secs = [], []
        for k in range(args.steps + args.warmup - 1):
            r = oracle_rate(cfg, X, rows, per_step, extras=False)
            if k >= args.warmup - 1:
                rates.append(r["value"])
                secs.append(r["seconds"])
        if not rates:
            rates, secs = [first["value"]], [first["seconds"]]
        value = statistics.median(rates)
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "n": n, "K": K, "P_total": P,
                           "label_type": cfg["label_type"],
                           "l2": "n/a (CPU)"},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": first["cores"],
                                 "kind": "oracle", "sample": first["sample"],
                                 "single_thread": first.get("single_thread"),
                                 "alg2_tiled": first.get("alg2_tiled"),
                                 "alg2_tiled_fp32": first.get("alg2_tiled_fp32"),
                                 "cpu_model": first.get("cpu_model")},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    import paper_2505_04556_gb300 as pm

    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    dev = local_rank
    torch.cuda.set_device(dev)
    pm.build()
    ctx = pm.Context(dev)
    form_id = {"auto": pm.FORM_AUTO, "brute": pm.FORM_BRUTE, "permblock": pm.FORM_PERMBLOCK,
               "gemm": pm.FORM_GEMM}[args.form]
    ctx.set_form(form_id)
    form = pm.FORM_NAMES[pm.permanova_plan_form(ctx.handle, n, K, B)]

    # ---- inputs resident in HBM before timing ----
    D = synth.recipe_matrix_device(cfg, X, device=f"cuda:{dev}")
    # label rows resident for the run: whole batches only, so every step is a
    # full batch of B rows (the ring of batches wraps when warm-up + steps
    # batches exceed the workload's permutations)
    n_rows = max(B, min(P, (args.warmup + args.steps) * B) // B * B)
    lab = synth.device_label_rows(cfg["labels"], n_rows, rank_seed(cfg["seed_perms"], rank),
                                  device=f"cuda:{dev}", dtype=torch.uint8)
    w = torch.from_numpy(cfg["w"]).to(f"cuda:{dev}")
    out = torch.empty(n_rows, dtype=torch.float64, device=f"cuda:{dev}")
    stream = torch.cuda.current_stream(dev)

    def step(k: int):
        b0 = (k * B) % n_rows
        bb = min(B, n_rows - b0)
        pm.permanova_sW(ctx.handle, D, n, D.stride(0), lab[b0:b0 + bb], pm.LABEL_U8, K, bb, w,
                        out[b0:b0 + bb], stream)
        return bb

    # the plan: the autotuner times candidate plans on a sample of the first
    # batch's label rows (outside the timed region) unless a form is forced
    if args.form == "auto" and not args.no_autotune:
        pm.permanova_autotune(ctx.handle, D, n, D.stride(0), lab[:B], pm.LABEL_U8, K, B, w, stream)
    plan = pm.permanova_plan_describe(ctx.handle, n, K, B)
    form = plan["form"]
    for k in range(args.warmup):
        step(k)
    pm.permanova_sync(ctx.handle, stream)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # D larger than L2 needs no flush; a small D is flushed from L2 between
    # steps (a write of 2 x L2), and only the steps themselves are timed
    flush = None
    if n * n * 4 < 2 * L2_BYTES:
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=f"cuda:{dev}")
    sampler = ClockSampler(gpu_query_id(torch, dev))
    pm.permanova_profile_enable(ctx.handle, True)
    torch.cuda.synchronize(dev)
    barrier()
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps if flush is not None else 1)]
    ev[0][0].record(stream)
    rows_done = 0
    for k in range(args.steps):
        if flush is not None and k > 0:
            with torch.cuda.stream(stream):
                flush.fill_(float(k))
            ev[k][0].record(stream)
        rows_done += step(args.warmup + k)
        if flush is not None:
            ev[k][1].record(stream)
    ev[-1][1].record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clocks = sampler.stop()
    prof = pm.permanova_profile_read(ctx.handle)
    pm.permanova_profile_enable(ctx.handle, False)
    pm.permanova_sync(ctx.handle, stream)
    ms, rows_total = combine_ranks(sum(a.elapsed_time(b) for a, b in ev), float(rows_done))
    value = pairs * rows_total / (ms / 1e3)

    # ---- the same steps on a prepared matrix (the operand preparation paid
    # once per job: its time is spread over the job's ceil(P / B) batches) ----
    prepared = None
    if form == "gemm" and not args.no_prepared:
        pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pe0.record(stream)
        prep = pm.permanova_prepare(ctx.handle, D, n, D.stride(0), stream)
        pe1.record(stream)
        pe1.synchronize()
        prep_ms = pe0.elapsed_time(pe1)

        def pstep(k: int):
            b0 = (k * B) % n_rows
            pm.permanova_sW_prepared(ctx.handle, prep, lab[b0:b0 + B], pm.LABEL_U8, K, B, w,
                                     out[b0:b0 + B], stream)
        pstep(0)
        pm.permanova_sync(ctx.handle, stream)
        pev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        pev[0].record(stream)
        for k in range(args.steps):
            pstep(args.warmup + k)
        pev[1].record(stream)
        torch.cuda.synchronize(dev)
        pms = pev[0].elapsed_time(pev[1])
        batches = math.ceil(P / B)
        prepared = {"value": pairs * B * args.steps / ((pms + prep_ms * args.steps / batches) / 1e3),
                    "unit": UNIT, "ms_per_step": pms / args.steps, "prepare_ms": prep_ms,
                    "job_batches": batches,
                    "api": "permanova_prepare once, then permanova_sW_prepared per batch; the "
                           "preparation time is spread over the job's batches"}
        pm.permanova_prepared_destroy(prep)

    # ---- dominant kernel roofline ----
    launches = max(1, prof["main_kernel_launches"])
    kernel_ms = prof["main_kernel_ms"] / launches
    evals_per_launch = pairs * rows_done / launches
    pk = peaks()
    rl = roofline(form, K, evals_per_launch, kernel_ms, pk,
                  traffic_per_launch(form, evals_per_launch, args.workload))
    rl["kernel_ms"] = kernel_ms

    # ---- end to end through the host entry point ----
    e2e = None
    if not args.no_e2e:
        Dh = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
        Dh.copy_(D)
        labh = torch.empty((B, n), dtype=torch.uint8, pin_memory=True)
        labh.copy_(lab[:B])
        wh = torch.from_numpy(cfg["w"].copy())
        outh = torch.empty(B, dtype=torch.float64, pin_memory=True)
        del D
        torch.cuda.empty_cache()

        def e2e_step():
            pm.permanova_sW_host(ctx.handle, Dh, n, n, labh, pm.LABEL_U8, K, B, wh, outh, stream)
            return float(outh[0])

        e2e_step()
        barrier()
        # this machine's host->device copy rate from the same pinned buffer: 1 GiB
        # copies (2 each) at five offsets across the whole buffer; the
        # end-to-end step cannot beat max(kernel time, copy time of its bytes)
        probe_n = min(Dh.numel(), (1 << 30) // 4)
        probe_dst = torch.empty(probe_n, dtype=torch.float32, device=f"cuda:{dev}")
        h2d_at = []
        for frac in (0.0, 0.25, 0.5, 0.75, 1.0):
            o = int(frac * (Dh.numel() - probe_n))
            probe_src = Dh.view(-1)[o:o + probe_n]
            probe_dst.copy_(probe_src, non_blocking=True)
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea.record()
            for _ in range(2):
                probe_dst.copy_(probe_src, non_blocking=True)
            eb.record()
            eb.synchronize()
            h2d_at.append(round(2 * probe_n * 4 / (ea.elapsed_time(eb) / 1e3) / 1e9, 1))
        h2d_gbs = min(h2d_at)
        del probe_dst
        torch.cuda.empty_cache()
        e2e_sampler = ClockSampler(gpu_query_id(torch, dev))
        pm.permanova_profile_enable(ctx.handle, True)
        e2e_sampler.start()
        t0 = time.perf_counter()
        step_ms = []
        for _ in range(args.e2e_steps):
            ts = time.perf_counter()
            e2e_step()
            step_ms.append(round(1e3 * (time.perf_counter() - ts), 2))
        barrier()
        te, rows_e2e = combine_ranks(time.perf_counter() - t0, float(B * args.e2e_steps))
        e2e_clocks = e2e_sampler.stop()
        hp = pm.permanova_profile_read(ctx.handle)
        pm.permanova_profile_enable(ctx.handle, False)
        calls = max(1, hp["host_calls"])
        # device-side timeline of one step (CUDA events, averaged over the steps)
        timeline = {"device_ms": round(hp["host_total_ms"] / calls, 2),
                    "first_segment_landed_ms": round(hp["host_first_segment_ms"] / calls, 2),
                    "last_segment_landed_ms": round(hp["host_copy_ms"] / calls, 2),
                    "h2d_gbs_in_step": round(hp["host_h2d_bytes"] / max(1e-9, hp["host_copy_ms"] / 1e3)
                                             / 1e9, 1),
                    "kernel_ms_device_resident": round(kernel_ms * B / (rows_done / launches), 2),
                    "segments_landed_ms": [round(x / calls, 1) for x in hp["host_seg_landed_ms"]],
                    "segments_kernel_done_ms": [round(x / calls, 1) for x in hp["host_seg_done_ms"]]}
        e2e = {"value": pairs * rows_e2e / te, "unit": UNIT,
               "h2d_bytes_per_step": int(host_matrix_bytes(n, n) + B * n + K * 4),
               "d2h_bytes_per_step": int(B * 8), "steps": args.e2e_steps, "step_ms": step_ms,
               "clocks": e2e_clocks, "h2d_gbs": round(h2d_gbs, 1), "h2d_gbs_at_offsets": h2d_at,
               "timeline": timeline,
               "api": "permanova_sW_host (pinned host D, labels, weights, results; "
                      "band copies of D (flat, or 2D for the later bands) in segments overlapped "
                      "with the kernels)"}

    cpu = None
    rows_h = lab[:64].cpu().numpy()
    serving = forms = precision = None
    if rank == 0 and world == 1 and not args.no_serving:
        # the serving workload on the same GPU, after the step's buffers and the
        # context's scratch are given back
        del lab, out
        Dh = labh = outh = None
        pm.permanova_release_scratch(ctx.handle)
        torch.cuda.empty_cache()
        # the extra measurements are reported, not required: a failure in one
        # is recorded in its place and the line still carries the rest
        serving = _guarded(lambda: serving_run(args.rate, args.duration, args.slots))
        forms = _guarded(lambda: forms_compare(peaks()))
        precision = _guarded(lambda: precision_compare(peaks()))
    if rank == 0 and not args.no_cpu:
        cpu = _guarded(lambda: oracle_rate(cfg, X, rows_h, 15.0))

    if rank == 0:
        dtype = "bf16 hi + fp16 lo, f32 accumulate" if form == "gemm" else "f32"
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": dtype, "data": "synthetic",
                "config": {"workload": args.workload, "n": n, "K": K, "P_total": P,
                           "batch": B, "label_type": "u8", "form": form, "plan": plan,
                           "matrix": {"euclid": f"Gaussian points in R^{cfg['dim']} (group shift "
                                                f"0.3 sd), Euclidean fp32",
                                      "braycurtis": "Dirichlet(0.5) x 200, Bray-Curtis fp32",
                                      "jaccard": "presence profiles (1,000 features), Jaccard fp32"
                                      }[cfg["kind"]],
                           "l2": (f"inputs larger than L2 (D = {n * n * 4 / 1e9:.1f} GB)"
                                  if flush is None else
                                  "L2 flushed between steps (2 x L2 write, untimed)"),
                           "parallelism": f"replicas x{world} (label rows split)"},
                "roofline": rl, "cpu_baseline": cpu, "e2e": e2e, "prepared": prepared, "serving": serving, "forms": forms,
                "precision": precision,
                "clocks": clocks,
                "gpu_launches": int(prof["kernel_launches"]),
                "gpu": torch.cuda.get_device_name(dev),
                "gpu_sms": torch.cuda.get_device_properties(dev).multi_processor_count}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
