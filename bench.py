#!/usr/bin/env python
"""Benchmark: policy-scenario reserve valuations per second on one GB300 (or N).

Headline workload (one "step"): the full-scale configuration, part (A): 1,000,000
single-life monthly level annuities (ages 60-90, Gompertz-Makeham mortality)
under 1,000 exact-step Vasicek scenarios (a=0.1, b=0.04, sigma=0.01, r0=0.03)
of 600 monthly discount factors (50 years; projections are truncated there):
1e9 policy-scenario chains, each valued by the backward recurrence to t = 0,
the reserves written out (4 GB FP32) and the per-scenario portfolio totals
summed in FP64.  The chosen form is the recurrence in deflated units
(RSV_FORM_F32_DEFLATED, compensated FP32); the plain FP32 recurrence, the
double-float recurrence and FP64 run on the same data beside it, each with
its relative error against the FP64 oracle on sampled policies.

Also measured (rank 0): the 100,000-policy four-product mix (configuration 2)
in every form; part (B) of the full-scale configuration (the nested run with
the surrogate and recurrence fallback against the brute-force inner loop and
the closed-form curve); the surrogate trained on 10M recurrence labels and
scored on 1M held-out queries (configuration 4); the nested brute force
(configuration 3); configuration 1's latency; the paper's summation against
recurrence comparison; varying cash flows; m-life contracts.

Timing: W warm-up steps, then K steps, each bracketed by CUDA events on the
launching stream, with a 256 MiB write between steps to flush L2 (the
scenario inputs are L2-sized; the 4 GB of reserves are not).  ``value`` = the
chains of all ranks / (sum of step times, max over ranks).  With N ranks the
portfolio is partitioned by policy (balanced by projection steps), every rank
values its share under the same scenarios, and the per-scenario FP64 totals
are summed over the ranks inside each timed step (strong scaling).  ``e2e``
times the same step through the C ABI with host buffers: the scenario,
portfolio and table uploads and the device-to-host copy of every reserve are
inside the timed region.

``--impl reference`` times the FP64 CPU oracle instead (rank 0, host cores,
a bounded sample of the headline workload per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from paper_1401_1757_gb300.shard import PolicyPartition, projection_steps  # noqa: E402

METRIC = "policy-scenario reserve valuations/s (plain vs surrogate) at stated error"
C5 = dict(n_pol=1_000_000, n_scen=1000, n_steps=600, horizon=600, seed=5, n_nodes=50, sample_pol=10_000,
          sample_outer=10)
HEAD_WORKLOAD = ("full scale (A): 1,000,000 single-life monthly level annuities (ages 60-90, Gompertz-Makeham) x "
                 "1,000 Vasicek scenarios x 600 monthly steps (50 y, projections truncated there); V0 of every chain "
                 "and FP64 per-scenario totals")
C5B_WORKLOAD = ("full scale (B): the same annuities; nested run on the 1,000 outer Vasicek paths x 50 annual nodes x "
                "1,000 inner paths")
C2 = dict(n_pol=100_000, n_scen=1000, n_steps=1200, seed=0)
C2_WORKLOAD = ("100,000-policy mix (40% SL annuities, 20% JL reversionary 3-state, 20% term 5-40y, "
               "20% endowments 10-30y, ages 20-85) x 1,000 Vasicek scenarios x 1,200 monthly steps")

FORMS = {"f64": 0, "f32": 1, "f32comp": 2, "f32defl": 3}
HEAD = "f32defl"
DTYPE = {"f32defl": "f32-deflated-compensated", "f32comp": "f32-compensated", "f32": "f32", "f64": "f64"}

# Algorithmic work of the method per chain-step (the same for every form):
# 3 flop for a one-state step (v p (c + r'): one multiply and one fused
# multiply-add), 16 for the three-state reversionary step (five products of
# the 3x3 upper-triangular W, three adds, three scalings, px py shared).
ALGO_FLOPS = {0: 3, 1: 16, 2: 3, 3: 3}
# FP32 (FP64 for f64) operations each form's kernels issue per chain-step
# (FMA = 2, add/sub/mul/min/max = 1): plain v p then an FMA; the double-float
# forms' products and ordered sums; the deflated form per 16 steps two
# products and 14 FMAs (30), the join of its two partial sums (1) and the
# ordered fold (6: max, min, three adds, one more into l), plus for the
# reversionary annuity the expected cash flow (two products, one subtraction,
# one FMA: 5) per policy-step shared by the M scenarios of a lane.
ISSUED_FLOPS = {"f32": {0: 3, 1: 9, 2: 3, 3: 3},
                "f32comp": {0: 16, 1: 48, 2: 20, 3: 20},
                "f64": {0: 3, 1: 9, 2: 3, 3: 3},
                "f32defl": {0: 37 / 16, 1: 37 / 16, 2: 37 / 16, 3: 37 / 16}}
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
FP32_PEAK_TFLOPS = 2 * FP32_LANES * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12   # 80.5 at 2070 MHz


def chain_steps_by_product(pol, horizon=0):
    S = projection_steps(pol, horizon=horizon)
    return {p: int(S[pol["product"] == p].sum()) for p in range(4)}


def algorithmic_flops(pol, n_scen, horizon=0):
    cs = chain_steps_by_product(pol, horizon)
    return float(sum(ALGO_FLOPS[p] * cs[p] for p in cs) * n_scen)


def issued_flops(pol, form, n_scen, horizon=0, variant_name=""):
    cs = chain_steps_by_product(pol, horizon)
    per = dict(ISSUED_FLOPS[form])
    if form == "f32defl":
        if variant_name.endswith(" tm2"):   # one fold per 32 steps: 2 x 30 + the spans' add (2) + join and fold (7)
            per = {p: 69.0 / 32 for p in per}
        # the JL expected cash flow, amortised over the lane's M scenarios
        m = re.search(r"xM(\d+)", variant_name)
        per[1] += 5.0 / (int(m.group(1)) if m else 4)
    return float(sum(per[p] * cs[p] for p in cs) * n_scen)


def kernel_source_hash(form=HEAD):
    """Hash of the sources a form's valuation kernel is built from."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1401_1757_gb300", "csrc")
    files = (("rsv_device.cuh", "defl_kernel.cuh", "recur_defl.cu") if form == "f32defl" else
             ("rsv_device.cuh", "recur_kernel.cuh", "recur_comp.cu", "recur_f32.cu", "recur_f64.cu"))
    for f in files:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(form, workload_key):
    """DRAM bytes per launch of a form's kernel on a workload, from the
    committed ncu summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "recur_traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    e = d.get(f"{form}:{workload_key}")
    if not e or e.get("kernel_hash") != kernel_source_hash(form):
        return None
    return e.get("dram_bytes_per_launch")


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


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


NESTED = dict(n_pol=2000, n_outer=100, n_nodes=40, node_step=12, n_inner=1000)
NESTED_WORKLOAD = ("nested brute force: 2,000 single-life annuities (ages 60-90) x 100 outer Vasicek paths x "
                   "40 annual nodes x 1,000 inner paths, deflated FP32 (and the double-float recurrence)")


def bench_nested(rsv, torch, tab, steps, warmup, n_outer=None, sur_epochs=10, sur_train=3_000_000):
    """The nested valuation: live (policy, outer path, node, inner path) valuations per
    second, device time of the whole pipeline (outer paths, inner-path generation,
    recurrence, node statistics), plus the closed-form inner expectation."""
    cfg = dict(NESTED)
    if n_outer:
        cfg["n_outer"] = n_outer
    pol = synth.portfolio_single_life(cfg["n_pol"], seed=0)
    S = projection_steps(pol)
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
    # the brute force in the chosen (deflated) form and in the double-float recurrence
    modes = [(rsv.RSV_NESTED_MC, "brute_force", NI), (rsv.RSV_NESTED_MC, "brute_force_compensated", NI),
             (rsv.RSV_NESTED_CURVE, "curve", 1)]
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
        form = rsv.RSV_FORM_F32_COMP if name == "brute_force_compensated" else rsv.RSV_FORM_F32_DEFLATED
        for _ in range(warmup):
            rsv.rsv_compute_nested(ctx, form, n_inner=NI, mode=mode, n_fallback=nfb, **spec)
        torch.cuda.synchronize()
        ms, walls = [], []
        for _ in range(steps):
            w0 = time.perf_counter()
            rsv.rsv_compute_nested(ctx, form, n_inner=NI, mode=mode, n_fallback=nfb, **spec)
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
            k: float(np.max(np.abs(means[k] - exact)[live_m] / exact[live_m]))
            for k in ("brute_force", "brute_force_compensated", "surrogate")}
        res["brute_force_forms_max_rel_diff"] = float(np.max(np.abs(means["brute_force"] - means["brute_force_compensated"])
                                                             [live_m] / np.abs(means["brute_force_compensated"])[live_m]))
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
    n_pol, n_scen, n_steps = C2["n_pol"], C2["n_scen"], C2["n_steps"]
    sch = synth.payment_schedules(n_pol, seed=0)
    rsv.rsv_load_schedules(ctx, sch, n_steps)
    V0 = torch.empty((n_pol, n_scen), dtype=torch.float32, device="cuda")
    tot = torch.empty(n_scen, dtype=torch.float64, device="cuda")
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
    return {"workload": C2_WORKLOAD + "; payment schedules: 80% monthly / 20% annual, 5% escalating",
            "kernel_ms": t, "valuations_s": n_pol * n_scen / (t / 1e3), "level_kernel_ms": level_ms,
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
    v = synth.vasicek_paths(C2["n_scen"], C2["n_steps"], seed=0)
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
    V0 = torch.empty((n_pol, C2["n_scen"]), dtype=torch.float32, device="cuda")
    res = {"workload": f"{n_pol:,} m-life policies (m = 2-4, half k-of-m annuities, half k-th death "
                       f"assurances 10-30y, ages 55-85) x {C2['n_scen']:,} Vasicek scenarios x {C2['n_steps']:,} steps",
           "chain_steps": int(S.sum()) * C2["n_scen"]}
    for form in ("f32comp", "f64"):
        fid = FORMS[form]
        rsv.rsv_compute_mlife(ctx, pol, fid, rsv.RSV_OUT_V0, on_device=True, V0=V0)
        ms = []
        for _ in range(reps):
            rsv.rsv_compute_mlife(ctx, pol, fid, rsv.RSV_OUT_V0, on_device=True, V0=V0)
            ms.append(rsv.rsv_last_kernel_ms(ctx))
        t = statistics.mean(ms) / 1e3
        flops = sum(mlife_flops(form, int(pol["m"][i]), pol["kind"][i] == 1, int(pol["k"][i])) * int(S[i])
                    for i in range(n_pol)) * C2["n_scen"]
        res[form] = {"ms": t * 1e3, "valuations_s": n_pol * C2["n_scen"] / t, "flops_per_launch": flops,
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
FIG1_WORKLOAD = ("the paper's algorithm comparison (Section 5.1.2, Fig. 1): single-life annuities from age 60 with a term of "
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


SURROGATE_WORKLOAD = ("MLP surrogate of the inner-loop expectation: 32->4x256->1 GELU, BF16 weights and activations, "
                      "FP32 accumulation, trained on 10M recurrence labels of the 100,000-policy mix, scored on 1M "
                      "held-out queries")


def bench_surrogate(rsv, torch, tab, epochs, lr=2e-3, n_train=10_000_000, n_val=1_000_000):
    """Train the surrogate on recurrence labels of the four-product portfolio and
    score it; throughput of the network against the recurrence it replaces."""
    pol = synth.portfolio_mix(C2["n_pol"], seed=0)
    ctx = rsv.rsv_create(torch.cuda.current_device(), torch.cuda.current_stream())
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_mlp_init(ctx, 0)
    rep = rsv.rsv_surrogate_train(ctx, n_train=n_train, n_val=n_val, epochs=epochs, batch=8192, lr=lr, seed=0)
    flops_q = 2 * (32 * 256 + 3 * 256 * 256 + 256)
    # the tcgen05 inference kernel alone on batches of 2^19 queries (features
    # already on the device; CUDA events around the kernel, best of 5)
    Xq = np.random.default_rng(1).normal(0, 1, (1 << 19, 32)).astype(np.float32)
    Xq[:, 20:] = 0.0
    ks = []
    for _ in range(6):
        rsv.rsv_mlp_forward(ctx, Xq)
        ks.append(rsv.rsv_last_kernel_ms(ctx))
    k_ms = min(ks[1:])
    rsv.rsv_destroy(ctx)
    peaks = measured_peaks()
    return {
        "workload": SURROGATE_WORKLOAD if (n_train, n_val) == (10_000_000, 1_000_000) else
        f"profiling case: {n_train} labels, {n_val} held-out queries", "epochs": epochs, "lr": lr,
        "held_out": {k: rep[k] for k in ("val_max_rel", "val_p99_rel", "val_median_rel", "val_rms_rel")},
        "tol": 1e-3, "margin": 0.3, "frac_fallback": rep["frac_fallback"], "combined_max_rel": rep["combined_max_rel"],
        "buckets_flagged": f"{rep['n_flagged']} of {rep['n_buckets']}",
        "residual_target_sd": rep["y_std"],
        "scoring_queries_s": rep["n_infer"] / (rep["infer_ms"] / 1e3),
        "scoring_note": "held-out scoring: features, the network and the reserve, batches of 524,288",
        "network_kernel": {
            "kernel": "mlp_fwd_tc_kernel (tcgen05, TMEM accumulators)", "queries": 1 << 19, "kernel_ms": k_ms,
            "flops_per_query": flops_q, "tflops": (1 << 19) * flops_q / (k_ms / 1e3) / 1e12,
            "frac_of_measured_bf16_burst_peak": (1 << 19) * flops_q / (k_ms / 1e3) / 1e12 / peaks["bf16_tflops"]
            if peaks else None,
            "peak": peaks["bf16_tflops"] if peaks else None},
        "recurrence_fp64_queries_s": rep["n_label"] / (rep["label_ms"] / 1e3),
        "train_s": rep["train_ms"] / 1e3,
        "train_samples_s": epochs * (n_train // 8192) * 8192 / max(rep["train_ms"] / 1e3, 1e-9),
    }


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def head_inputs(n_pol=None, n_scen=None):
    c = C5
    pol = synth.portfolio_single_life(n_pol or c["n_pol"], seed=c["seed"])
    v = synth.vasicek_paths(n_scen or c["n_scen"], c["n_steps"], seed=c["seed"])
    return pol, v


def oracle_runs(pol, tab, v, horizon, runs, warm=1):
    """Time the FP64 oracle on all host cores: ``warm`` untimed runs, then ``runs`` timed ones."""
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    times = []
    for i in range(warm + runs):
        t0 = time.perf_counter()
        oracle.reserves_batch(pol, tab, v, horizon=horizon, nthreads=threads)
        if i >= warm:
            times.append(time.perf_counter() - t0)
    return times, threads


def cpu_full_configs(tab, runs, with_c2):
    """The oracle on whole configurations (the paper's timing method, Section
    5.2.1: minimum and median of ``runs`` timed runs after one warm-up, all
    host cores):
    configuration 1 always (1,000 annuities, one flat scenario, a few ms),
    configuration 2 on request (10^5 policies x 1,000 scenarios x 1,200
    steps, about 80 s a run on 16 cores)."""
    out = {}
    cases = [("config1", synth.portfolio_single_life(1000, seed=0), synth.flat_scenarios(n_steps=720),
              "1,000 single-life annuities x 1 flat 4% scenario x up to 720 steps, in full")]
    if with_c2:
        cases.append(("config2", synth.portfolio_mix(C2["n_pol"], seed=C2["seed"]),
                      synth.vasicek_paths(C2["n_scen"], C2["n_steps"], seed=C2["seed"]), C2_WORKLOAD + ", in full"))
    for name, pol, v, what in cases:
        times, threads = oracle_runs(pol, tab, v, 0, runs)
        vals = len(pol["product"]) * v.shape[0]
        out[name] = {"value": vals / min(times), "unit": "valuations/s", "median_value": vals / statistics.median(times),
                     "min_s": min(times), "median_s": statistics.median(times), "runs": runs, "cores": threads,
                     "cpu_model": cpu_model(), "kind": "oracle", "sample": what}
    return out


def reference_arm(args, rank):
    """The FP64 CPU oracle on the host cores, a bounded sample of the headline
    workload per step (the same policies, all scenarios, the same horizon)."""
    if rank != 0:
        return
    pol, v = head_inputs(args.policies, args.scenarios)
    tab = synth.gm_monthly_survival()
    n_sample = min(args.ref_policies, len(pol["product"]))
    sub = synth.take(pol, slice(0, n_sample))
    times, threads = oracle_runs(sub, tab, v, C5["horizon"], args.steps, warm=args.warmup)
    per = sum(times) / len(times)
    value = n_sample * v.shape[0] / per
    sample = (f"first {n_sample} of {len(pol['product'])} policies x all {v.shape[0]} scenarios x "
              f"{C5['horizon']} steps per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "valuations/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": HEAD_WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "valuations/s", "cores": threads, "kind": "oracle",
                             "sample": sample, "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "valuations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(pol, tab, v, horizon, n_sample, runs=7):
    """The oracle on the host cores, the paper's timing method (Section 5.2.1:
    the minimum of seven runs; the median beside it): one warm-up and
    ``runs`` timed runs of the first n_sample policies x all scenarios."""
    sub = synth.take(pol, slice(0, n_sample))
    times, threads = oracle_runs(sub, tab, v, horizon, runs)
    vals = n_sample * v.shape[0]
    return {"value": vals / min(times), "unit": "valuations/s", "cores": threads, "kind": "oracle",
            "sample": f"first {n_sample} of {len(pol['product'])} policies x all {v.shape[0]} scenarios"
                      + (f" x {horizon} steps" if horizon else "") + f", min of {runs} runs",
            "runs": runs, "min_s": min(times), "median_s": statistics.median(times),
            "median_value": vals / statistics.median(times), "cpu_model": cpu_model()}


def rel_errors(got, ref, amount):
    scale = np.maximum(np.abs(ref), 1e-9 * np.abs(amount)[:, None])
    e = np.abs(got - ref) / scale
    return {"max_rel_err": float(e.max()), "p99_rel_err": float(np.quantile(e, 0.99)),
            "median_rel_err": float(np.median(e))}


def time_form(rsv, torch, ctx, form, V0, tot, horizon, steps, warmup, flush, stream, part=None, dist=None,
              sampler=None, tune=True):
    """K timed steps of one form (tuned first), CUDA events on the launching
    stream around each step; with a partition, the FP64 sum of the totals over
    the ranks is inside the step."""
    fid = FORMS[form]
    outs = rsv.RSV_OUT_V0 | rsv.RSV_OUT_SCEN_TOTAL
    tune_ms = None
    if tune:
        best, tune_ms = rsv.rsv_tune(ctx, fid, horizon=horizon, reps=1)
    else:
        best = 0
    world = part.world if part else 1
    for _ in range(warmup):
        rsv.rsv_compute_reserves(ctx, fid, outs, horizon=horizon, on_device=True, V0=V0, scen_total=tot)
        if part:
            part.reduce_totals(tot, dist)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(0.5)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    evs, kern = [], []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rsv.rsv_compute_reserves(ctx, fid, outs, horizon=horizon, on_device=True, V0=V0, scen_total=tot)
        if part:
            part.reduce_totals(tot, dist)
        e1.record(stream)
        evs.append((e0, e1))
        kern.append(rsv.rsv_last_kernel_ms(ctx))   # waits for this step's kernel
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    r = {"ms_per_step": total_ms / steps, "median_ms": statistics.median(step_ms), "best_ms": min(step_ms),
         "kernel_ms": statistics.mean(kern), "steps": steps, "variant": rsv.rsv_variant_name(fid, best)}
    if tune_ms:
        r["tune_ms"] = {rsv.rsv_variant_name(fid, i): round(m, 3) for i, m in enumerate(tune_ms)}
    return r, clocks


def sampled_rows(rsv, torch, ctx, form, n_pol, n_scen, horizon, idx):
    """The same launch writing FP64 reserves; the rows of the sampled policies."""
    V0d = torch.empty((n_pol, n_scen), dtype=torch.float64, device="cuda")
    rsv.rsv_compute_reserves(ctx, FORMS[form], rsv.RSV_OUT_V0, horizon=horizon, on_device=True, V0d=V0d)
    torch.cuda.synchronize()
    rows = V0d[torch.as_tensor(idx, device="cuda")].cpu().numpy()
    del V0d
    return rows


def bench_forms(rsv, torch, ctx, pol, tab, v, forms, horizon, steps, warmup, flush, stream, n_sample, seed,
                part=None, dist=None, head_sampler=None):
    """Every form on one loaded workload: timing, algorithmic and issued
    throughput, and the error of each against the oracle on sampled policies."""
    import oracle
    n_pol, n_scen = len(pol["product"]), v.shape[0]
    V0 = torch.empty((n_pol, n_scen), dtype=torch.float32, device="cuda")
    tot = torch.empty(n_scen, dtype=torch.float64, device="cuda")
    world = part.world if part else 1
    cs = float(projection_steps(pol, horizon=horizon).sum()) * n_scen
    results, clocks = {}, None
    for form in forms:
        slow = form == "f64"
        r, ck = time_form(rsv, torch, ctx, form, V0, tot, horizon, min(steps, 2) if slow else steps,
                          1 if slow else warmup, flush, stream, part, dist,
                          head_sampler if form == forms[0] else None, tune=not slow)
        if ck:
            clocks = ck
        t = r["ms_per_step"] / 1e3
        r["valuations_s"] = world * n_pol * n_scen / t
        r["chain_steps_s"] = world * cs / t
        kt = r["kernel_ms"] / 1e3
        r["algorithmic_tflops"] = algorithmic_flops(pol, n_scen, horizon) / kt / 1e12
        r["issued_tflops"] = issued_flops(pol, form, n_scen, horizon, r["variant"]) / kt / 1e12
        results[form] = r
    del V0
    if n_sample > 0:
        rng = np.random.default_rng(seed)
        idx = np.sort(rng.choice(n_pol, min(n_sample, n_pol), replace=False))
        sub = synth.take(pol, idx)
        ref, _ = oracle.reserves_batch(sub, tab, v, horizon=horizon)
        for form in forms:
            rows = sampled_rows(rsv, torch, ctx, form, n_pol, n_scen, horizon, idx)
            results[form].update(rel_errors(rows, ref, sub["amount"]))
            results[form]["error_sample"] = f"{len(idx)} random policies x all {n_scen} scenarios, FP64 output"
    return results, clocks


def bench_config2(rsv, torch, tab, forms, steps, warmup, flush, stream):
    """Configuration 2 (the four-product mix) in every form."""
    c = C2
    pol = synth.portfolio_mix(c["n_pol"], seed=c["seed"])
    v = synth.vasicek_paths(c["n_scen"], c["n_steps"], seed=c["seed"])
    ctx = rsv.rsv_create(torch.cuda.current_device(), stream)
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_load_scenarios(ctx, v)
    res, _ = bench_forms(rsv, torch, ctx, pol, tab, v, forms, 0, steps, warmup, flush, stream, 300, seed=0)
    res["workload"] = C2_WORKLOAD
    return res, ctx, pol


def bench_c5_nested(rsv, torch, tab, sur_epochs=10):
    """Part (B) of the full-scale configuration: the nested run with the
    surrogate (all 1,000 outer paths, a policy sample, extrapolated by
    policies), the brute-force inner loop and the closed-form curve (a sample
    of outer paths too, extrapolated by outer paths and policies);
    node-liability errors against the curve on the common sample."""
    c = C5
    res = {"workload": C5B_WORKLOAD}
    pol = synth.take(synth.portfolio_single_life(c["n_pol"], seed=c["seed"]), slice(0, c["sample_pol"]))
    ctx = rsv.rsv_create(torch.cuda.current_device(), torch.cuda.current_stream())
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
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
        rsv.rsv_compute_nested(ctx, rsv.RSV_FORM_F32_DEFLATED, n_outer=n_outer, n_nodes=NN, node_step_m=12,
                               n_inner=1000, seed=5, mode=mode, on_device=True, L_mean=L, L_q995=q, n_fallback=nfb)
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
    res["extrapolation"] = ("times measured on the stated samples on one GB300, scaled linearly by policies (and by "
                            "outer paths for the brute force) to 1,000,000 policies x 1,000 outer paths")
    return res


def bench_e2e(rsv, torch, ctx, pol, tab, v, form, horizon, steps, warmup, world, dist):
    """The head step through the C ABI with host buffers: uploads of the table,
    scenarios and portfolio from pinned memory, the host rebuild of the layout
    after the portfolio reload, and every reserve written to page-locked host
    memory (by the kernel itself in the deflated form, else by a copy), all
    inside the timed region."""
    fid = FORMS[form]
    outs = rsv.RSV_OUT_V0 | rsv.RSV_OUT_SCEN_TOTAL
    n_pol, n_scen = len(pol["product"]), v.shape[0]
    v_host = torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
    recs = torch.from_numpy(rsv.policy_records(pol).view(np.uint8)).pin_memory()
    V0_host = torch.empty((n_pol, n_scen), dtype=torch.float32).pin_memory()
    tot_host = torch.empty(n_scen, dtype=torch.float64).pin_memory()
    V0n, totn = V0_host.numpy(), tot_host.numpy()
    recn = recs.numpy().view(rsv.POLICY_DTYPE)

    def step():
        rsv.rsv_load_decrements(ctx, 0, tab)
        rsv.rsv_load_scenarios(ctx, v_host)
        rsv.rsv_load_portfolio(ctx, recn)
        rsv.rsv_compute_reserves(ctx, fid, outs, horizon=horizon, on_device=False, V0=V0n, scen_total=totn)

    for _ in range(max(1, warmup)):
        step()
    if world > 1:
        dist.barrier()
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    tot_s = sum(times)
    if world > 1:
        t = torch.tensor([tot_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_s = float(t.item())
    return {"value": world * n_pol * n_scen * steps / tot_s, "unit": "valuations/s",
            "h2d_bytes_per_step": int(v.nbytes + recn.nbytes + tab.nbytes),
            "d2h_bytes_per_step": int(V0_host.numel() * 4 + tot_host.numel() * 8),
            "ms_per_step": 1e3 * tot_s / steps,
            "note": "per rank: uploads of its portfolio share, the scenarios and the table, and the layout "
                    "rebuilt on the host; its V0 (written to page-locked host memory) and totals back"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--forms", default="f32defl,f32comp,f32,f64", help="the first is the headline form")
    ap.add_argument("--policies", type=int, default=C5["n_pol"], help="smaller portfolios for profiling runs")
    ap.add_argument("--scenarios", type=int, default=C5["n_scen"], help="smaller scenario sets for profiling runs")
    ap.add_argument("--sample-policies", type=int, default=200, help="policies in each form's oracle error sample")
    ap.add_argument("--cpu-sample", type=int, default=2000, help="policies in each CPU oracle run")
    ap.add_argument("--cpu-runs", type=int, default=7)
    ap.add_argument("--ref-policies", type=int, default=1000, help="policies per reference-arm step")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-full", action="store_true",
                    help="also time the oracle on all of configuration 2 (about 80 s a run on 16 cores)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="only the headline workload")
    ap.add_argument("--no-nested", action="store_true")
    ap.add_argument("--surrogate-epochs", type=int, default=30, help="configuration 4 (0: skip)")
    ap.add_argument("--surrogate-lr", type=float, default=2e-3)
    ap.add_argument("--surrogate-train", type=int, default=10_000_000, help="training labels (profiling runs: fewer)")
    ap.add_argument("--surrogate-val", type=int, default=1_000_000, help="held-out queries")
    ap.add_argument("--nested-outer", type=int, default=NESTED["n_outer"], help="outer paths (profiling runs: fewer)")
    ap.add_argument("--nested-surrogate-epochs", type=int, default=10,
                    help="train the surrogate on the nested portfolio and time its mode (0: skip)")
    ap.add_argument("--mlife-only", action="store_true",
                    help="time only the m-life contracts (--policies of them) and print their record")
    ap.add_argument("--nested-only", action="store_true",
                    help="time only the nested valuation (--nested-outer paths) and print its record")
    ap.add_argument("--surrogate-only", action="store_true",
                    help="train and score only the surrogate (--surrogate-* sizes) and print its record")
    args = ap.parse_args()
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
    if args.surrogate_only:   # a profiling case of the network kernels
        import torch
        from paper_1401_1757_gb300 import rsv
        torch.cuda.set_device(local)
        print(json.dumps({"surrogate": bench_surrogate(rsv, torch, synth.gm_monthly_survival(), args.surrogate_epochs,
                                                       lr=args.surrogate_lr, n_train=args.surrogate_train,
                                                       n_val=args.surrogate_val)}), flush=True)
        return
    if args.nested_only:   # a profiling case of the nested kernels
        import torch
        from paper_1401_1757_gb300 import rsv
        torch.cuda.set_device(local)
        print(json.dumps({"nested": bench_nested(rsv, torch, synth.gm_monthly_survival(), steps=1, warmup=1,
                                                 n_outer=args.nested_outer,
                                                 sur_epochs=args.nested_surrogate_epochs)}), flush=True)
        return

    import torch
    import torch.distributed as dist
    from paper_1401_1757_gb300 import rsv

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    full = (args.policies, args.scenarios) == (C5["n_pol"], C5["n_scen"])
    workload = HEAD_WORKLOAD if full else (f"profiling case: {args.policies} single-life annuities x "
                                           f"{args.scenarios} Vasicek scenarios x 600 steps")
    pol_all, v = head_inputs(args.policies, args.scenarios)
    tab = synth.gm_monthly_survival()
    horizon = C5["horizon"]
    part = PolicyPartition(projection_steps(pol_all, horizon=horizon), world, rank)
    pol = part.take(pol_all)
    stream = torch.cuda.current_stream()
    ctx = rsv.rsv_create(local, stream)
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_load_scenarios(ctx, v)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    forms = [f for f in args.forms.split(",") if f]
    head = forms[0]
    sampler = ClockSampler(local)
    results, clocks = bench_forms(rsv, torch, ctx, pol, tab, v, forms, horizon, args.steps, args.warmup, flush,
                                  stream, args.sample_policies if rank == 0 else 0, seed=C5["seed"], part=part,
                                  dist=dist, head_sampler=sampler)
    e2e = None
    if not args.no_e2e:
        e2e = bench_e2e(rsv, torch, ctx, pol, tab, v, head, horizon, args.steps, args.warmup, world, dist)
    rsv.rsv_destroy(ctx)
    torch.cuda.empty_cache()

    extras = {}
    peaks = None
    if rank == 0:
        peaks = {"fp32_fma_tflops": rsv.rsv_probe_fma_peak(local, None, False),
                 "fp64_fma_tflops": rsv.rsv_probe_fma_peak(local, None, True),
                 "how": "independent FMA chains on every SM, best of 5 launches"}
    if rank == 0 and not args.no_extras:
        c2, c2ctx, c2pol = bench_config2(rsv, torch, tab, forms, args.steps, args.warmup, flush, stream)
        extras["config2"] = c2
        extras["cash_flows"] = bench_cashflows(rsv, torch, c2ctx, FORMS["f32comp"], c2["f32comp"]["kernel_ms"],
                                               args.steps, args.warmup, flush) if "f32comp" in c2 else None
        rsv.rsv_destroy(c2ctx)
        torch.cuda.empty_cache()
        extras["mlife"] = bench_mlife(rsv, torch, tab)
        extras["config1_latency"] = bench_config1(rsv, torch, tab)
        extras["summation_vs_recurrence"] = bench_figure1(rsv, torch, tab)
        if not args.no_nested:
            extras["nested"] = bench_nested(rsv, torch, tab, steps=2, warmup=1, n_outer=args.nested_outer,
                                            sur_epochs=args.nested_surrogate_epochs)
            extras["full_scale_nested"] = bench_c5_nested(rsv, torch, tab)
        if args.surrogate_epochs > 0:
            extras["surrogate"] = bench_surrogate(rsv, torch, tab, args.surrogate_epochs, lr=args.surrogate_lr,
                                                  n_train=args.surrogate_train, n_val=args.surrogate_val)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    cpu = None
    if not args.no_cpu:
        cpu = cpu_baseline(pol_all, tab, v, horizon, min(args.cpu_sample, len(pol_all["product"])), args.cpu_runs)
        if "summation_vs_recurrence" in extras:
            extras["summation_vs_recurrence"]["cpu_oracle"] = cpu_figure1(tab)
        extras["cpu_oracle_full"] = cpu_full_configs(tab, args.cpu_runs, args.cpu_full)
    for f, r in results.items():
        pk = peaks["fp64_fma_tflops"] if f == "f64" else peaks["fp32_fma_tflops"]
        r["algorithmic_frac_of_measured_peak"] = r["algorithmic_tflops"] / pk
        r["issued_frac_of_measured_peak"] = r["issued_tflops"] / pk
    if "mlife" in extras:
        m = extras["mlife"]
        m["f32comp"]["frac_of_measured_fp32_fma_peak"] = m["f32comp"]["achieved_tflops"] / peaks["fp32_fma_tflops"]
        m["f64"]["frac_of_measured_fp64_fma_peak"] = m["f64"]["achieved_tflops"] / peaks["fp64_fma_tflops"]
    if "config2" in extras:
        for f, r in extras["config2"].items():
            if isinstance(r, dict) and "algorithmic_tflops" in r:
                pk = peaks["fp64_fma_tflops"] if f == "f64" else peaks["fp32_fma_tflops"]
                r["algorithmic_frac_of_measured_peak"] = r["algorithmic_tflops"] / pk

    h = results[head]
    n_scen = v.shape[0]
    flops = algorithmic_flops(pol, n_scen, horizon)
    ifl = issued_flops(pol, head, n_scen, horizon, h["variant"])
    kt = h["kernel_ms"] / 1e3
    roof = {"bound": "alu", "achieved": flops / kt / 1e12, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": flops / kt / 1e12 / FP32_PEAK_TFLOPS,
            "traffic": measured_traffic(head, "c5A") if full else None,
            "kernel": f"defl_kernel ({h['variant']}) with its deflator-plane pass" if head == "f32defl" else
                      f"recur_kernel ({h['variant']})",
            "flops_per_launch": flops,
            "count": "algorithmic: 3 flop per one-state chain-step, 16 per three-state chain-step",
            "peak_note": "FP32 FMA pipe, 152 SMs x 128 lanes x 2 flop x 2070 MHz (nominal units x max clock)",
            "frac_of_measured_fma_peak": flops / kt / 1e12 / peaks["fp32_fma_tflops"],
            "issued_flops_per_launch": ifl, "issued_frac": ifl / kt / 1e12 / FP32_PEAK_TFLOPS,
            "issued_count": "FP32 operations the kernel issues per chain-step (FMA 2, others 1)"}
    line = {
        "metric": METRIC, "value": h["valuations_s"], "unit": "valuations/s", "n_gpus": world,
        "steps": h["steps"], "warmup": args.warmup, "ms_per_step": h["ms_per_step"], "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": DTYPE[head], "data": "synthetic",
        "config": {"workload": workload, "policies": len(pol_all["product"]), "scenarios": n_scen,
                   "steps": C5["n_steps"], "horizon": horizon, "form": head, "variant": h["variant"],
                   "max_rel_err_vs_oracle": h.get("max_rel_err"),
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"policy partition over {world} GPU(s), FP64 sum of per-scenario totals"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": (4 if head == "f32defl" else 3) * h["steps"],
        "clocks": clocks,
        "forms": results,
        "measured_alu_peaks": peaks,
        **extras,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
