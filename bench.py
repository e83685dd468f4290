#!/usr/bin/env python
"""Benchmark: policy-scenario reserve valuations per second on one GB300 (or N).

Workload (one "step"): the 100,000-policy four-product mix (40% single-life
annuities, 20% joint-life reversionary annuities with 3 states and reversion
50-100%, 20% term assurances 5-40 y, 20% endowments 10-30 y; ages 20-85) under
1,000 exact-step Vasicek scenarios (a=0.1, b=0.04, sigma=0.01, r0=0.03) of
1,200 monthly discount factors: 1e8 policy-scenario chains, the backward
vector reserve recurrence of every chain to t = 0, the reserves written out
and the per-scenario portfolio totals summed in FP64.

Timing: W warm-up steps, then K steps, each bracketed by CUDA events on the
launching stream, with a 256 MiB write between steps to flush L2 (the inputs
are L2-sized).  ``value`` = chains of all ranks / (sum of step times, max over
ranks).  ``e2e`` times the same step through the C ABI with host buffers: the
scenario, portfolio and table uploads and the device-to-host copy of every
reserve are inside the timed region.

``--impl reference`` times the FP64 CPU oracle instead (rank 0, host cores,
a bounded sample of the same workload per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
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

METRIC = "policy-scenario reserve valuations/s (plain vs surrogate) at stated error"
N_POL, N_SCEN, N_STEPS = 100_000, 1000, 1200
N_POL_MIX = 100_000
WORKLOAD = ("100,000-policy mix (40% SL annuities, 20% JL reversionary 3-state, 20% term 5-40y, "
            "20% endowments 10-30y, ages 20-85) x 1,000 Vasicek scenarios x 1,200 monthly steps")

# FP32 (FP64 for f64) operations per chain-step of each form and product
# (add/sub/mul/min/max = 1, FMA = 2), counted from the formulas the kernels
# evaluate: plain annuity v*p then an FMA; compensated annuity a double-float
# product (7) and the shifted update 1 + g R (9); compensated assurance two
# double-float products and an ordered sum (20); the JL product as three
# annuity chains a_x, a_y, a_xy: plain three products and three FMAs (9),
# compensated three double-float products (21) and three shifted updates
# (27): 48.
FLOPS = {"f32": {0: 3, 1: 9, 2: 3, 3: 3},
         "f32comp": {0: 16, 1: 48, 2: 20, 3: 20},
         "f64": {0: 3, 1: 9, 2: 3, 3: 3}}
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
FP32_PEAK_TFLOPS = 2 * FP32_LANES * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12   # 80.5 at 2070 MHz

FORMS = {"f64": 0, "f32": 1, "f32comp": 2}


def policy_steps(pol, n_ages=1440, horizon=0):
    """Projection length of each policy (the same rules as the library applies)."""
    prod, a1, a2, term = pol["product"], pol["age1_m"], pol["age2_m"], pol["term_m"]
    S = np.where(prod == 0, np.maximum(0, n_ages - a1),
                 np.where(prod == 1, np.maximum(0, n_ages - np.minimum(a1, a2)), term))
    S = np.where((prod <= 1) & (term > 0), np.minimum(S, term), S)
    if horizon > 0:
        S = np.minimum(S, horizon)
    return S.astype(np.int64)


def algorithmic_flops(pol, form, n_scen):
    S = policy_steps(pol)
    return float(sum(FLOPS[form][p] * S[pol["product"] == p].sum() for p in range(4)) * n_scen)


def kernel_source_hash():
    """Hash of the sources the valuation recurrence kernel is built from."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1401_1757_gb300", "csrc")
    for f in ("rsv_device.cuh", "recur_kernel.cuh", "recur_comp.cu", "recur_f32.cu", "recur_f64.cu"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(form):
    """DRAM bytes per launch of the recurrence kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "recur_traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    e = d.get(form)
    if not e or e.get("kernel_hash") != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.lines, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
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
            for n, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def reference_arm(args, rank):
    """The FP64 CPU oracle on the host cores, a bounded sample of the workload per step."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    pol = synth.portfolio_mix(N_POL, seed=0)
    tab = synth.gm_monthly_survival()
    v = synth.vasicek_paths(N_SCEN, N_STEPS, seed=0)
    n_sample = args.ref_policies
    sub = synth.take(pol, slice(0, n_sample))
    threads = os.cpu_count() or 1
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.reserves_batch(sub, tab, v, nthreads=threads)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    per = sum(times) / len(times)
    value = n_sample * N_SCEN / per
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "valuations/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"first {n_sample} policies x {N_SCEN} scenarios per step"},
            "cpu_baseline": {"value": value, "unit": "valuations/s", "cores": threads, "kind": "oracle",
                             "sample": f"first {n_sample} of {N_POL} policies x all {N_SCEN} scenarios"},
            "e2e": {"value": value, "unit": "valuations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


NESTED = dict(n_pol=2000, n_outer=100, n_nodes=40, node_step=12, n_inner=1000)
NESTED_WORKLOAD = ("nested brute force: 2,000 single-life annuities (ages 60-90) x 100 outer Vasicek paths x "
                   "40 annual nodes x 1,000 inner paths, compensated FP32")


def bench_nested(rsv, torch, tab, steps, warmup, n_outer=None, sur_epochs=10, sur_train=3_000_000):
    """The nested valuation: live (policy, outer path, node, inner path) valuations per
    second, device time of the whole pipeline (outer paths, inner-path generation,
    recurrence, node statistics), plus the closed-form inner expectation."""
    cfg = dict(NESTED)
    if n_outer:
        cfg["n_outer"] = n_outer
    pol = synth.portfolio_single_life(cfg["n_pol"], seed=0)
    S = policy_steps(pol)
    live = chain_steps = 0
    for n in range(cfg["n_nodes"]):
        rem = S - n * cfg["node_step"]
        live += int((rem > 0).sum())
        chain_steps += int(rem[rem > 0].sum())
    scale = cfg["n_outer"] * cfg["n_inner"]
    ctx = rsv.rsv_create(torch.cuda.current_device(), torch.cuda.current_stream())
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    NO, NN, NI = cfg["n_outer"], cfg["n_nodes"], cfg["n_inner"]
    mean = torch.empty((NO, NN), dtype=torch.float64, device="cuda")
    q = torch.empty((NO, NN), dtype=torch.float64, device="cuda")
    spec = dict(n_outer=NO, n_nodes=NN, node_step_m=cfg["node_step"], seed=0, on_device=True, L_mean=mean, L_q995=q)
    res = {}
    modes = [(rsv.RSV_NESTED_MC, "brute_force", NI), (rsv.RSV_NESTED_CURVE, "curve", 1)]
    if sur_epochs > 0:
        # the surrogate, trained on this portfolio's own recurrence labels up to the last node
        t0 = time.perf_counter()
        rsv.rsv_mlp_init(ctx, 0)
        rep = rsv.rsv_surrogate_train(ctx, n_train=sur_train, n_val=max(200_000, sur_train // 10), epochs=sur_epochs,
                                      batch=8192, lr=2e-3, seed=0, max_node_m=(NN - 1) * cfg["node_step"])
        res["surrogate_training"] = {"labels": sur_train, "epochs": sur_epochs, "wall_s": time.perf_counter() - t0,
                                     "held_out_median_rel": rep["val_median_rel"],
                                     "served_max_rel": rep["combined_max_rel"],
                                     "fallback_share": rep["frac_fallback"]}
        modes.append((rsv.RSV_NESTED_SURROGATE, "surrogate", 1))
    means = {}
    for mode, name, ni in modes:
        nfb = np.zeros(1, np.int64)
        for _ in range(warmup):
            rsv.rsv_compute_nested(ctx, rsv.RSV_FORM_F32_COMP, n_inner=NI, mode=mode, n_fallback=nfb, **spec)
        torch.cuda.synchronize()
        ms, walls = [], []
        for _ in range(steps):
            w0 = time.perf_counter()
            rsv.rsv_compute_nested(ctx, rsv.RSV_FORM_F32_COMP, n_inner=NI, mode=mode, n_fallback=nfb, **spec)
            ms.append(rsv.rsv_last_kernel_ms(ctx))
            torch.cuda.synchronize()
            walls.append(time.perf_counter() - w0)
        t = statistics.mean(ms) / 1e3
        vals = live * (cfg["n_outer"] * ni)
        res[name] = {"valuations_s": vals / t, "ms": t * 1e3, "wall_ms": statistics.mean(walls) * 1e3,
                     "valuations": vals, "chain_steps_s": chain_steps * cfg["n_outer"] * ni / t}
        if mode == rsv.RSV_NESTED_SURROGATE:
            res[name]["fallback_queries"] = int(nfb[0])
            res[name]["note"] = ("valuations = (policy, outer path, node) expectations, each replacing n_inner "
                                 "inner-path valuations; ms is the device time of the whole call")
        means[name] = mean.cpu().numpy().copy()
    if "surrogate" in means:
        exact = means["curve"]
        live_m = exact > 0
        res["node_liability_max_rel_vs_exact"] = {
            k: float(np.max(np.abs(means[k] - exact)[live_m] / exact[live_m])) for k in ("brute_force", "surrogate")}
        res["surrogate_speedup_vs_brute_force"] = res["brute_force"]["ms"] / res["surrogate"]["ms"]
    rsv.rsv_destroy(ctx)
    res["workload"] = NESTED_WORKLOAD if cfg["n_outer"] == NESTED["n_outer"] else \
        f"profiling case: {NESTED_WORKLOAD.replace('100 outer', str(cfg['n_outer']) + ' outer')}"
    res["live_valuations"] = live * scale
    res["chain_steps"] = chain_steps * scale
    res["paper_brute_force_estimate"] = ("the paper's cost model (Section 5.3.2) for its 500k portfolio is "
                                         "~550 h on a 2-core laptop")
    return res


def bench_cashflows(rsv, torch, ctx, fid, level_ms, steps, warmup, flush):
    """The main workload with the paper's payment mix (Section 5: about 80%
    monthly and 20% annual payments, 5% escalating at 3%, 4.25% or 5% on each
    anniversary), expanded on the device and valued by the general-cash-flow
    kernel; against the level cash flows of the timed step."""
    sch = synth.payment_schedules(N_POL, seed=0)
    rsv.rsv_load_schedules(ctx, sch, N_STEPS)
    V0 = torch.empty((N_POL, N_SCEN), dtype=torch.float32, device="cuda")
    tot = torch.empty(N_SCEN, dtype=torch.float64, device="cuda")
    outs = rsv.RSV_OUT_V0 | rsv.RSV_OUT_SCEN_TOTAL
    for _ in range(warmup):
        rsv.rsv_compute_reserves(ctx, fid, outs, on_device=True, V0=V0, scen_total=tot)
    ms = []
    for _ in range(steps):
        flush.zero_()
        rsv.rsv_compute_reserves(ctx, fid, outs, on_device=True, V0=V0, scen_total=tot)
        ms.append(rsv.rsv_last_kernel_ms(ctx))
    rsv.rsv_clear_cashflows(ctx)
    t = statistics.mean(ms)
    return {"workload": WORKLOAD + "; payment schedules: 80% monthly / 20% annual, 5% escalating",
            "kernel_ms": t, "valuations_s": N_POL * N_SCEN / (t / 1e3), "level_kernel_ms": level_ms,
            "cost_vs_level": t / level_ms,
            "variant": "general cash flows (unshifted states, c_t per policy and step)"}


# Operations per chain-step of the m-life kernel (m lives; FMA = 2): each of
# the m 2^(m-1) one-life mixes p a + q b, the scaling by v of the live states,
# and the cash flow added to the paying states.  Plain forms: mix = FMA + MUL
# (3), scale 1, add 1.  Compensated: mix = two double-float products (7 each)
# and an ordered sum (7) = 21, scale 7, add 6.
def mlife_flops(form, m, assurance, k):
    n = 1 << m
    marked = sum(1 for S in range(n) if (bin(S).count("1") >= k if assurance else m - bin(S).count("1") >= k))
    mix, sc, add = (21, 7, 6) if form == "f32comp" else (3, 1, 1)
    scaled = n - marked if assurance else n
    return m * (n // 2) * mix + scaled * sc + (0 if assurance else marked) * add


def mlife_bench_portfolio(n, seed=0):
    """m = 2..4 lives (equal shares) aged 55-85; half annuities paid while k of m
    are alive (whole life), half k-th death assurances (10-30 y); k uniform."""
    rng = np.random.default_rng(seed)
    pol = {"m": rng.integers(2, 5, n), "kind": rng.integers(0, 2, n), "k": np.zeros(n, int),
           "term_m": np.zeros(n, int), "age_m": np.zeros((n, 4), int), "table": np.zeros((n, 4), int),
           "dead0": np.zeros(n, int), "amount": rng.lognormal(np.log(1e3), 0.5, n)}
    for i in range(n):
        m = pol["m"][i]
        pol["k"][i] = rng.integers(1, m + 1)
        pol["age_m"][i, :m] = rng.integers(55 * 12, 85 * 12 + 1, m)
        if pol["kind"][i] == 1:
            pol["term_m"][i] = 12 * rng.integers(10, 31)
    return pol


def bench_mlife(rsv, torch, tab, n_pol=20_000, reps=3):
    """m-life contracts (Section 4.3) under the 1,000 scenarios of 1,200 steps."""
    pol = mlife_bench_portfolio(n_pol)
    v = synth.vasicek_paths(N_SCEN, N_STEPS, seed=0)
    ctx = rsv.rsv_create(torch.cuda.current_device(), torch.cuda.current_stream())
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_scenarios(ctx, v)
    # steps of each policy (the kernel's rule): annuity to the k-th longest-lived
    # table, assurance its term
    S = np.zeros(n_pol, int)
    for i in range(n_pol):
        m, k = pol["m"][i], pol["k"][i]
        if pol["kind"][i] == 1:
            S[i] = pol["term_m"][i]
        else:
            rem = sorted(max(0, len(tab) - a) for a in pol["age_m"][i, :m])
            S[i] = rem[m - k]
    V0 = torch.empty((n_pol, N_SCEN), dtype=torch.float32, device="cuda")
    res = {"workload": f"{n_pol:,} m-life policies (m = 2-4, half k-of-m annuities, half k-th death "
                       f"assurances 10-30y, ages 55-85) x {N_SCEN:,} Vasicek scenarios x {N_STEPS:,} steps",
           "chain_steps": int(S.sum()) * N_SCEN}
    for form in ("f32comp", "f64"):
        fid = FORMS[form]
        rsv.rsv_compute_mlife(ctx, pol, fid, rsv.RSV_OUT_V0, on_device=True, V0=V0)
        ms = []
        for _ in range(reps):
            rsv.rsv_compute_mlife(ctx, pol, fid, rsv.RSV_OUT_V0, on_device=True, V0=V0)
            ms.append(rsv.rsv_last_kernel_ms(ctx))
        t = statistics.mean(ms) / 1e3
        flops = sum(mlife_flops(form, int(pol["m"][i]), pol["kind"][i] == 1, int(pol["k"][i])) * int(S[i])
                    for i in range(n_pol)) * N_SCEN
        res[form] = {"ms": t * 1e3, "valuations_s": n_pol * N_SCEN / t, "flops_per_launch": flops,
                     "achieved_tflops": flops / t / 1e12}
    rsv.rsv_destroy(ctx)
    return res


def bench_config1(rsv, torch, tab, reps=20):
    """Config 1 (1,000 annuities, one flat 4% rate, FP64): a latency-bound run with
    one scenario.  Kernel time of the scenario-parallel FP64 kernel against the
    parallel-in-time scan (one warp per chain, lanes over blocks of steps)."""
    pol = synth.portfolio_single_life(1000, seed=0)
    v = synth.flat_scenarios(n_steps=720)
    ctx = rsv.rsv_create(torch.cuda.current_device(), torch.cuda.current_stream())
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_load_scenarios(ctx, v)
    V0 = torch.empty((1000, 1), dtype=torch.float64, device="cuda")
    res = {"workload": "1,000 single-life annuities (ages 60-90) x 1 flat 4% scenario x up to 720 steps, FP64"}
    for name, var in (("scenario_parallel", -1), ("time_scan", rsv.RSV_VARIANT_TIME_SCAN)):
        ms = []
        for i in range(reps + 3):
            rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F64, rsv.RSV_OUT_V0, on_device=True, variant=var, V0d=V0)
            if i >= 3:
                ms.append(rsv.rsv_last_kernel_ms(ctx))
        t = statistics.median(ms)
        res[name] = {"kernel_ms": t, "valuations_s": 1000 / (t / 1e3)}
    rsv.rsv_destroy(ctx)
    return res


FIG1_STEPS = (60, 120, 240, 360, 480, 600, 720)
FIG1_WORKLOAD = ("the paper's algorithm comparison (Section 5.2): single-life annuities from age 60 with a term of "
                 "S months, one flat 4% scenario, FP64, the reserve at every step; time per policy")


def bench_figure1(rsv, torch, tab, n_pol=60_000, reps=3):
    """Summation (O(S^2)) against recurrence (O(S)) as the projection length S
    grows, on the GPU: the summation-definition kernel, the time scan and the
    scenario-parallel recurrence kernel, each writing the whole trajectory."""
    v = synth.flat_scenarios(n_steps=max(FIG1_STEPS))
    ctx = rsv.rsv_create(torch.cuda.current_device(), torch.cuda.current_stream())
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_scenarios(ctx, v)
    traj = torch.empty((n_pol, v.shape[1] + 1, 1), dtype=torch.float64, device="cuda")
    res = {"workload": FIG1_WORKLOAD + f" ({n_pol} policies)", "S": list(FIG1_STEPS),
           "gpu_summation_us": [], "gpu_time_scan_us": [], "gpu_recurrence_us": []}
    for S in FIG1_STEPS:
        pol = synth.portfolio_single_life(n_pol, seed=0, age_lo_y=60, age_hi_y=60)
        pol["term_m"][:] = S
        rsv.rsv_load_portfolio(ctx, pol)
        for key, var in (("gpu_summation_us", rsv.RSV_VARIANT_SUMMATION), ("gpu_time_scan_us", rsv.RSV_VARIANT_TIME_SCAN),
                         ("gpu_recurrence_us", -1)):
            ms = []
            for i in range(reps + 1):
                rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F64, rsv.RSV_OUT_TRAJ, on_device=True, variant=var,
                                         traj=traj)
                if i > 0:
                    ms.append(rsv.rsv_last_kernel_ms(ctx))
            res[key].append(statistics.median(ms) * 1e3 / n_pol)
    rsv.rsv_destroy(ctx)
    del traj
    return res


def cpu_figure1(tab, n_pol=2000):
    """The same comparison for the FP64 CPU oracle (its summation and its
    recurrence, every step, all host cores): time per policy."""
    import oracle
    oracle.build()
    v = synth.flat_scenarios(n_steps=max(FIG1_STEPS))
    threads = os.cpu_count() or 1
    res = {"workload": FIG1_WORKLOAD + f" ({n_pol} policies)", "cores": threads, "S": list(FIG1_STEPS),
           "cpu_summation_us": [], "cpu_recurrence_us": []}
    for S in FIG1_STEPS:
        pol = synth.portfolio_single_life(n_pol, seed=0, age_lo_y=60, age_hi_y=60)
        pol["term_m"][:] = S
        for key, method in (("cpu_summation_us", "summation"), ("cpu_recurrence_us", "recurrence")):
            t0 = time.perf_counter()
            oracle.reserves_batch(pol, tab, v, nthreads=threads, method=method, totals=False)
            res[key].append((time.perf_counter() - t0) * 1e6 / n_pol)
    return res


C5 = dict(n_pol=1_000_000, n_scen=1000, n_steps=600, n_nodes=50, sample_pol=10_000, sample_outer=10)
C5_WORKLOAD = ("full scale: 1,000,000 single-life annuities (ages 60-90) x 1,000 Vasicek scenarios x 600 monthly "
               "steps (50 y); nested: 1,000 outer paths x 50 annual nodes x 1,000 inner paths")


def bench_full_scale(rsv, torch, tab, sur_epochs=10, reps=3):
    """(A) The plain batched recurrence at full scale, plain and compensated
    FP32.  (B) The nested run with the surrogate (all 1,000 outer paths, a
    policy sample, extrapolated by policies), the brute-force inner loop and
    the closed-form curve (a sample of outer paths too, extrapolated by outer
    paths and policies); node-liability errors against the curve on the
    common sample."""
    c = C5
    res = {"workload": C5_WORKLOAD}
    pol = synth.portfolio_single_life(c["n_pol"], seed=5)
    v = synth.vasicek_paths(c["n_scen"], c["n_steps"], seed=5)
    ctx = rsv.rsv_create(torch.cuda.current_device(), torch.cuda.current_stream())
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_load_scenarios(ctx, v)
    V0 = torch.empty((c["n_pol"], c["n_scen"]), dtype=torch.float32, device="cuda")
    tot = torch.empty(c["n_scen"], dtype=torch.float64, device="cuda")
    outs = rsv.RSV_OUT_V0 | rsv.RSV_OUT_SCEN_TOTAL
    for name, form in (("A_plain_f32", rsv.RSV_FORM_F32), ("A_compensated_f32", rsv.RSV_FORM_F32_COMP)):
        rsv.rsv_tune(ctx, form, horizon=c["n_steps"], reps=1)
        ms = []
        for i in range(reps + 1):
            rsv.rsv_compute_reserves(ctx, form, outs, horizon=c["n_steps"], on_device=True, V0=V0, scen_total=tot)
            if i:
                ms.append(rsv.rsv_last_kernel_ms(ctx))
        t = statistics.median(ms)
        res[name] = {"kernel_ms": t, "valuations_s": c["n_pol"] * c["n_scen"] / (t / 1e3)}
    del V0
    # (B) nested, on the first sample_pol policies
    sub = synth.take(pol, slice(0, c["sample_pol"]))
    rsv.rsv_load_portfolio(ctx, sub)
    NN = c["n_nodes"]
    t0 = time.perf_counter()
    rsv.rsv_mlp_init(ctx, 0)
    rep = rsv.rsv_surrogate_train(ctx, n_train=3_000_000, n_val=300_000, epochs=sur_epochs, batch=8192, lr=2e-3,
                                  seed=5, max_node_m=(NN - 1) * 12)
    train_s = time.perf_counter() - t0
    scale_pol = c["n_pol"] / c["sample_pol"]
    runs = {}
    for name, mode, n_outer in (("surrogate", rsv.RSV_NESTED_SURROGATE, c["n_scen"]),
                                ("surrogate_sample", rsv.RSV_NESTED_SURROGATE, c["sample_outer"]),
                                ("brute_force", rsv.RSV_NESTED_MC, c["sample_outer"]),
                                ("curve_sample", rsv.RSV_NESTED_CURVE, c["sample_outer"]),
                                ("curve", rsv.RSV_NESTED_CURVE, c["n_scen"])):
        L = torch.empty((n_outer, NN), dtype=torch.float64, device="cuda")
        q = torch.empty((n_outer, NN), dtype=torch.float64, device="cuda")
        nfb = np.zeros(1, np.int64)
        rsv.rsv_compute_nested(ctx, rsv.RSV_FORM_F32_COMP, n_outer=n_outer, n_nodes=NN, node_step_m=12, n_inner=1000,
                               seed=5, mode=mode, on_device=True, L_mean=L, L_q995=q, n_fallback=nfb)
        torch.cuda.synchronize()
        runs[name] = (rsv.rsv_last_kernel_ms(ctx), L.cpu().numpy(), int(nfb[0]))
    rsv.rsv_destroy(ctx)
    full_outer = c["n_scen"] / c["sample_outer"]
    exact = runs["curve_sample"][1]
    live = exact > 0
    res["B_surrogate"] = {"measured_ms": runs["surrogate"][0], "measured_on": f"{c['sample_pol']} policies x "
                          f"{c['n_scen']} outer x {NN} nodes", "fallback_queries": runs["surrogate"][2],
                          "extrapolated_full_s": runs["surrogate"][0] * scale_pol / 1e3,
                          "node_liability_max_rel_vs_curve":
                              float(np.max(np.abs(runs["surrogate_sample"][1] - exact)[live] / exact[live])),
                          "training_s": train_s, "held_out_median_rel": rep["val_median_rel"],
                          "served_max_rel": rep["combined_max_rel"], "fallback_share": rep["frac_fallback"]}
    res["B_brute_force"] = {"measured_ms": runs["brute_force"][0], "measured_on": f"{c['sample_pol']} policies x "
                            f"{c['sample_outer']} outer x {NN} nodes x 1000 inner",
                            "extrapolated_full_s": runs["brute_force"][0] * scale_pol * full_outer / 1e3,
                            "node_liability_max_rel_vs_curve":
                                float(np.max(np.abs(runs["brute_force"][1] - exact)[live] / exact[live]))}
    res["B_curve"] = {"measured_ms": runs["curve"][0], "measured_on": f"{c['sample_pol']} policies x "
                      f"{c['n_scen']} outer x {NN} nodes",
                      "extrapolated_full_s": runs["curve"][0] * scale_pol / 1e3,
                      "max_rel_vs_sample_run": float(np.max(np.abs(runs["curve"][1][: c["sample_outer"]] - exact)[live]
                                                            / exact[live]))}
    res["B_speedup_surrogate_vs_brute_force"] = (res["B_brute_force"]["extrapolated_full_s"] /
                                                 res["B_surrogate"]["extrapolated_full_s"])
    return res


SURROGATE_WORKLOAD = ("MLP surrogate of the inner-loop expectation: 32->4x256->1 GELU, BF16 weights and activations, "
                      "FP32 accumulation, trained on 10M recurrence labels of the 100,000-policy mix, scored on 1M "
                      "held-out queries")


def bench_surrogate(rsv, torch, tab, epochs, lr=2e-3, n_train=10_000_000, n_val=1_000_000):
    """Train the surrogate on recurrence labels of the four-product portfolio and
    score it; throughput of the network against the recurrence it replaces."""
    pol = synth.portfolio_mix(N_POL_MIX, seed=0)
    ctx = rsv.rsv_create(torch.cuda.current_device(), torch.cuda.current_stream())
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_mlp_init(ctx, 0)
    rep = rsv.rsv_surrogate_train(ctx, n_train=n_train, n_val=n_val, epochs=epochs, batch=8192, lr=lr, seed=0)
    rsv.rsv_destroy(ctx)
    flops_q = 2 * (32 * 256 + 3 * 256 * 256 + 256)
    return {
        "workload": SURROGATE_WORKLOAD if (n_train, n_val) == (10_000_000, 1_000_000) else
        f"profiling case: {n_train} labels, {n_val} held-out queries", "epochs": epochs, "lr": lr,
        "held_out": {k: rep[k] for k in ("val_max_rel", "val_p99_rel", "val_median_rel", "val_rms_rel")},
        "tol": 1e-3, "margin": 0.3, "frac_fallback": rep["frac_fallback"], "combined_max_rel": rep["combined_max_rel"],
        "buckets_flagged": f"{rep['n_flagged']} of {rep['n_buckets']}",
        "residual_target_sd": rep["y_std"],
        "network_queries_s": rep["n_infer"] / (rep["infer_ms"] / 1e3),
        "network_tflops": rep["n_infer"] * flops_q / (rep["infer_ms"] / 1e3) / 1e12,
        "recurrence_fp64_queries_s": rep["n_label"] / (rep["label_ms"] / 1e3),
        "train_s": rep["train_ms"] / 1e3,
        "train_samples_s": epochs * (n_train // 8192) * 8192 / max(rep["train_ms"] / 1e3, 1e-9),
    }


def cpu_baseline(pol, tab, v, n_sample, gpu_rows):
    """Oracle timed on the host cores on the first n_sample policies x all
    scenarios; also the max relative error of each GPU form on that sample."""
    import oracle
    oracle.build()
    sub = synth.take(pol, slice(0, n_sample))
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    ref, _ = oracle.reserves_batch(sub, tab, v, nthreads=threads)
    dt = time.perf_counter() - t0
    errs = {}
    scale = np.maximum(np.abs(ref), 1e-9 * np.abs(sub["amount"])[:, None])
    for form, rows in gpu_rows.items():
        e = np.abs(rows.astype(np.float64) - ref) / scale
        errs[form] = {"max_rel_err": float(e.max()), "p99_rel_err": float(np.quantile(e, 0.99)),
                      "median_rel_err": float(np.median(e))}
    return {"value": n_sample * v.shape[0] / dt, "unit": "valuations/s", "cores": threads, "kind": "oracle",
            "sample": f"first {n_sample} of {len(pol['product'])} policies x all {v.shape[0]} scenarios "
                      f"({dt:.1f} s wall)"}, errs


def main():
    global N_POL, N_SCEN, WORKLOAD
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--forms", default="f32comp,f32,f64")
    ap.add_argument("--cpu-sample", type=int, default=1500, help="policies in the CPU oracle sample")
    ap.add_argument("--policies", type=int, default=100_000, help="smaller portfolios for profiling runs")
    ap.add_argument("--scenarios", type=int, default=1000, help="smaller scenario sets for profiling runs")
    ap.add_argument("--ref-policies", type=int, default=1000, help="policies per reference-arm step")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-nested", action="store_true")
    ap.add_argument("--surrogate-epochs", type=int, default=0, help="train and score the surrogate (0: skip)")
    ap.add_argument("--surrogate-lr", type=float, default=2e-3)
    ap.add_argument("--surrogate-train", type=int, default=10_000_000, help="training labels (profiling runs: fewer)")
    ap.add_argument("--surrogate-val", type=int, default=1_000_000, help="held-out queries")
    ap.add_argument("--nested-outer", type=int, default=NESTED["n_outer"], help="outer paths (profiling runs: fewer)")
    ap.add_argument("--full-scale", action="store_true", help="also the 1M-policy full-scale configuration")
    ap.add_argument("--mlife-only", action="store_true",
                    help="time only the m-life contracts (--policies of them) and print their record")
    ap.add_argument("--nested-surrogate-epochs", type=int, default=10,
                    help="train the surrogate on the nested portfolio and time its mode (0: skip)")
    args = ap.parse_args()
    if (args.policies, args.scenarios) != (N_POL, N_SCEN):
        N_POL, N_SCEN = args.policies, args.scenarios
        WORKLOAD = f"profiling case: {N_POL}-policy mix x {N_SCEN} Vasicek scenarios x {N_STEPS} monthly steps"

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank)
    if args.mlife_only:   # a profiling case of the m-life kernel
        import torch
        from paper_1401_1757_gb300 import rsv
        torch.cuda.set_device(local)
        print(json.dumps({"mlife": bench_mlife(rsv, torch, synth.gm_monthly_survival(), n_pol=args.policies)}),
              flush=True)
        return

    import torch
    import torch.distributed as dist
    from paper_1401_1757_gb300 import rsv

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    # weak scaling: every rank values the full portfolio under its own scenario set
    pol = synth.portfolio_mix(N_POL, seed=0)
    tab = synth.gm_monthly_survival()
    v = synth.vasicek_paths(N_SCEN, N_STEPS, seed=rank)
    stream = torch.cuda.current_stream()
    ctx = rsv.rsv_create(local, stream)
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_load_scenarios(ctx, v)

    V0 = torch.empty((N_POL, N_SCEN), dtype=torch.float32, device="cuda")
    tot = torch.empty(N_SCEN, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    outs = rsv.RSV_OUT_V0 | rsv.RSV_OUT_SCEN_TOTAL
    forms = [f for f in args.forms.split(",") if f]
    head = forms[0]
    results, sample_rows = {}, {}
    clocks = None
    for form in forms:
        fid = FORMS[form]
        best, tune_ms = rsv.rsv_tune(ctx, fid, reps=1)
        K = args.steps if form != "f64" else min(args.steps, 3)
        for _ in range(args.warmup):
            rsv.rsv_compute_reserves(ctx, fid, outs, on_device=True, V0=V0, scen_total=tot)
        torch.cuda.synchronize()
        sampler = None
        if form == head:
            sampler = ClockSampler(local)
            sampler.start()
            time.sleep(0.5)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        evs = []
        kern_ms = []
        t_wall = time.perf_counter()
        for _ in range(K):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rsv.rsv_compute_reserves(ctx, fid, outs, on_device=True, V0=V0, scen_total=tot)
            e1.record(stream)
            evs.append((e0, e1))
            kern_ms.append(rsv.rsv_last_kernel_ms(ctx))   # waits for this step's kernel
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_wall
        if world > 1:
            dist.barrier()
        if sampler:
            clocks = sampler.stop()
        step_ms = [a.elapsed_time(b) for a, b in evs]
        total_ms = sum(step_ms)
        if world > 1:
            t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            total_ms = float(t.item())
        per_ms = total_ms / K
        chains = N_POL * N_SCEN
        results[form] = {
            "valuations_s": world * chains / (per_ms / 1e3),
            "chain_steps_s": world * float(policy_steps(pol).sum()) * N_SCEN / (per_ms / 1e3),
            "ms_per_step": per_ms, "median_ms": statistics.median(step_ms), "best_ms": min(step_ms),
            "kernel_ms": statistics.mean(kern_ms), "steps": K,
            "variant": rsv.rsv_variant_name(fid, best),
            "tune_ms": {rsv.rsv_variant_name(fid, i): round(m, 3) for i, m in enumerate(tune_ms)},
            "wall_s_incl_flush": wall,
        }
        # accuracy sample: the same launch writing FP64 reserves for the first policies
        V0d = torch.empty((N_POL, N_SCEN), dtype=torch.float64, device="cuda")
        rsv.rsv_compute_reserves(ctx, fid, rsv.RSV_OUT_V0, on_device=True, V0d=V0d)
        torch.cuda.synchronize()
        sample_rows[form] = V0d[: args.cpu_sample].cpu().numpy()
        del V0d

    # end to end through the C ABI with host buffers (head form)
    e2e = None
    if not args.no_e2e:
        fid = FORMS[head]
        v_host = torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
        recs = rsv.policy_records(pol)
        V0_host = torch.empty((N_POL, N_SCEN), dtype=torch.float32).pin_memory()
        tot_host = torch.empty(N_SCEN, dtype=torch.float64).pin_memory()
        V0n, totn = V0_host.numpy(), tot_host.numpy()

        def e2e_step():
            rsv.rsv_load_decrements(ctx, 0, tab)
            rsv.rsv_load_scenarios(ctx, v_host)
            rsv.rsv_load_portfolio(ctx, recs)
            rsv.rsv_compute_reserves(ctx, fid, outs, on_device=False, V0=V0n, scen_total=totn)

        for _ in range(max(1, args.warmup)):
            e2e_step()
        if world > 1:
            dist.barrier()
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            e2e_step()
            times.append(time.perf_counter() - t0)
        tot_s = sum(times)
        if world > 1:
            t = torch.tensor([tot_s], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            tot_s = float(t.item())
        e2e = {"value": world * N_POL * N_SCEN * args.steps / tot_s, "unit": "valuations/s",
               "h2d_bytes_per_step": int(v.nbytes + recs.nbytes + tab.nbytes),
               "d2h_bytes_per_step": int(V0_host.numel() * 4 + tot_host.numel() * 8),
               "ms_per_step": 1e3 * tot_s / args.steps}

    cashflows = None
    if not args.no_nested and rank == 0:
        cashflows = bench_cashflows(rsv, torch, ctx, FORMS[head], results[head]["kernel_ms"], args.steps,
                                    args.warmup, flush)
    rsv.rsv_destroy(ctx)
    nested = config1 = figure1 = mlife = None
    if not args.no_nested and rank == 0:
        mlife = bench_mlife(rsv, torch, tab)
        config1 = bench_config1(rsv, torch, tab)
        figure1 = bench_figure1(rsv, torch, tab)
        nested = bench_nested(rsv, torch, tab, steps=2, warmup=1, n_outer=args.nested_outer,
                              sur_epochs=args.nested_surrogate_epochs)
    full = None
    if args.full_scale and rank == 0:
        full = bench_full_scale(rsv, torch, tab)
    peaks = None
    if rank == 0:
        peaks = {"fp32_fma_tflops": rsv.rsv_probe_fma_peak(local, None, False),
                 "fp64_fma_tflops": rsv.rsv_probe_fma_peak(local, None, True),
                 "how": "independent FMA chains on every SM, best of 5 launches"}
    surrogate = None
    if args.surrogate_epochs > 0 and rank == 0:
        surrogate = bench_surrogate(rsv, torch, tab, args.surrogate_epochs, lr=args.surrogate_lr,
                                    n_train=args.surrogate_train, n_val=args.surrogate_val)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    cpu, errs = (None, {})
    if not args.no_cpu:
        cpu, errs = cpu_baseline(pol, tab, v, args.cpu_sample, sample_rows)
        if figure1 is not None:
            figure1["cpu_oracle"] = cpu_figure1(tab)
    for f in results:
        results[f].update(errs.get(f, {}))

    h = results[head]
    flops = algorithmic_flops(pol, head, N_SCEN)
    achieved = flops / (h["kernel_ms"] / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP32_PEAK_TFLOPS, "traffic": measured_traffic(head),
            "kernel": f"recur_kernel ({h['variant']})",
            "peak_note": "FP32 FMA pipe, 152 SMs x 128 lanes x 2 flop x 2070 MHz (nominal units x max clock)",
            "flops_per_launch": flops}
    if peaks:
        roof["frac_of_measured_fma_peak"] = achieved / peaks["fp32_fma_tflops"]
    for f, r in results.items():   # every form against the measured peak of its arithmetic
        fl = algorithmic_flops(pol, f, N_SCEN)
        r["achieved_tflops"] = fl / (r["kernel_ms"] / 1e3) / 1e12
        if peaks:
            pk = peaks["fp64_fma_tflops"] if f == "f64" else peaks["fp32_fma_tflops"]
            r["frac_of_measured_fma_peak"] = r["achieved_tflops"] / pk
    if mlife and peaks:
        mlife["f32comp"]["frac_of_measured_fp32_fma_peak"] = mlife["f32comp"]["achieved_tflops"] / peaks["fp32_fma_tflops"]
        mlife["f64"]["frac_of_measured_fp64_fma_peak"] = mlife["f64"]["achieved_tflops"] / peaks["fp64_fma_tflops"]
    line = {
        "metric": METRIC, "value": h["valuations_s"], "unit": "valuations/s", "n_gpus": world,
        "steps": h["steps"], "warmup": args.warmup, "ms_per_step": h["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32-compensated" if head == "f32comp" else head,
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "policies": N_POL, "scenarios": N_SCEN, "steps": N_STEPS,
                   "form": head, "variant": h["variant"], "l2": "flushed between timed steps (256 MiB write)",
                   "scenario_seed": "rank"},
        "roofline": roof,
        "measured_alu_peaks": peaks,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": 3 * h["steps"],
        "clocks": clocks,
        "forms": results,
        "config1_latency": config1,
        "summation_vs_recurrence": figure1,
        "cash_flows": cashflows,
        "mlife": mlife,
        "full_scale": full,
        "nested": nested,
        "surrogate": surrogate,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
