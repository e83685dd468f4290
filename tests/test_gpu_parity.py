"""GPU parity: the CUDA recurrence (through the C ABI) against the FP64 oracle.

Error metric: rel = |V_gpu - V_ref| / max(|V_ref|, 1e-9 * amount).  Bounds:
  * FP64 form: 1e-12 (same arithmetic, different operation order over <= 1440
    steps: a few hundred roundings of 2^-53).
  * compensated FP32 form: 1e-6, the target relative accuracy; the
    double-float state carries about 44 bits, so it lands far inside.
  * plain FP32 form: 2e-4.  Rounding v to FP32 alone is a relative error of up
    to 2^-24 per step, systematic under a flat rate, so ~t * 6e-8 (4e-5 at 720
    steps); the 3-state product doubles it.  This form is measured, not
    expected to meet 1e-6.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1401_1757_gb300 import rsv

pytestmark = pytest.mark.gpu

TOL = {rsv.RSV_FORM_F64: 1e-12, rsv.RSV_FORM_F32_COMP: 1e-6, rsv.RSV_FORM_F32: 2e-4}
FORMS = [rsv.RSV_FORM_F64, rsv.RSV_FORM_F32_COMP, rsv.RSV_FORM_F32]
V0T = rsv.RSV_OUT_V0 | rsv.RSV_OUT_SCEN_TOTAL


def rel_err(got, ref, amount):
    scale = np.maximum(np.abs(ref), 1e-9 * np.abs(np.asarray(amount))[:, None])
    return np.abs(got - ref) / scale


@pytest.fixture
def ctx():
    assert torch.cuda.is_available()
    h = rsv.rsv_create(0, torch.cuda.current_stream())
    yield h
    rsv.rsv_destroy(h)


def run(ctx, pol, tab, v, form, horizon=0, variant=-1, tables=None):
    if tables is None:
        rsv.rsv_load_decrements(ctx, 0, tab)
    else:
        for i, t in enumerate(tables):
            rsv.rsv_load_decrements(ctx, i, t)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_load_scenarios(ctx, v)
    n, S = len(pol["product"]), v.shape[0]
    V0 = np.zeros((n, S))
    tot = np.zeros(S)
    rsv.rsv_compute_reserves(ctx, form, V0T, horizon=horizon, variant=variant, V0d=V0, scen_total=tot)
    return V0, tot


@pytest.mark.parametrize("form", FORMS)
def test_config1_full(ctx, form):
    """1,000 single-life level annuities, ages 60-90, GM mortality, flat 4%."""
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_single_life(1000, seed=0)
    v = synth.flat_scenarios(n_steps=720)
    V0, tot = run(ctx, pol, tab, v, form)
    ref, ref_tot = oracle.reserves_batch(pol, tab, v)
    err = rel_err(V0, ref, pol["amount"])
    print(f"config-1 form {rsv.FORM_NAMES[form]}: max rel err {err.max():.3e}, median {np.median(err):.3e}")
    assert err.max() <= TOL[form]
    assert abs(tot[0] - ref_tot[0]) <= TOL[form] * ref_tot[0]


@pytest.mark.parametrize("form", FORMS)
def test_mix_vasicek_ragged(ctx, form):
    """Four-product mix, 300 policies x 157 Vasicek scenarios (ragged against
    every chunk width), 1200 steps."""
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_mix(300, seed=21)
    v = synth.vasicek_paths(157, 1200, seed=21)
    V0, tot = run(ctx, pol, tab, v, form)
    ref, ref_tot = oracle.reserves_batch(pol, tab, v)
    err = rel_err(V0, ref, pol["amount"])
    for p in range(4):
        m = pol["product"] == p
        print(f"mix form {rsv.FORM_NAMES[form]} product {p}: max rel err {err[m].max():.3e}")
    assert err.max() <= TOL[form]
    assert np.max(np.abs(tot - ref_tot) / ref_tot) <= TOL[form]


@pytest.mark.parametrize("form", FORMS)
def test_every_variant_agrees(ctx, form):
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_mix(130, seed=5)
    v = synth.vasicek_paths(70, 1200, seed=5)
    ref, _ = oracle.reserves_batch(pol, tab, v)
    for var in range(rsv.rsv_variant_count(form)):
        V0, _ = run(ctx, pol, tab, v, form, variant=var)
        err = rel_err(V0, ref, pol["amount"]).max()
        assert err <= TOL[form], (rsv.rsv_variant_name(form, var), err)


@pytest.mark.parametrize("form", [rsv.RSV_FORM_F64, rsv.RSV_FORM_F32_COMP])
def test_trajectory_every_step_every_state(ctx, form):
    """r_t at every t, in every reduced state (JL states 00, 01, 10 via state0),
    against the oracle's full-state vectors."""
    tab = synth.gm_monthly_survival()
    base = synth.portfolio_mix(24, seed=8)
    jl = np.where(base["product"] == 1)[0]
    extra = synth.take(base, np.concatenate([jl, jl]))
    extra["state0"][: len(jl)] = 1
    extra["state0"][len(jl):] = 2
    pol = {k: np.concatenate([base[k], extra[k]]) for k in base}
    n = len(pol["product"])
    v = synth.vasicek_paths(37, 1200, seed=8)
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_load_scenarios(ctx, v)
    T = v.shape[1]
    traj = np.zeros((n, T + 1, 37))
    pt = np.zeros((n, T + 1))
    rsv.rsv_compute_reserves(ctx, form, rsv.RSV_OUT_TRAJ | rsv.RSV_OUT_PT_MEAN, traj=traj, pt_mean=pt)
    worst = 0.0
    for p in range(n):
        ref_s = []
        for s in range(37):
            r = oracle.chain(int(pol["product"][p]), int(pol["age1_m"][p]), float(pol["amount"][p]), tab, v[s],
                             age2=int(pol["age2_m"][p]), term=int(pol["term_m"][p]), rho=float(pol["reversion"][p]))
            ref = r[:, int(pol["state0"][p])]
            S = len(ref) - 1
            got = traj[p, : S + 1, s]
            scale = np.maximum(np.abs(ref), 1e-9 * pol["amount"][p])
            worst = max(worst, float(np.max(np.abs(got - ref) / scale)))
            assert np.all(traj[p, S + 1:, s] == 0.0)
            ref_s.append(np.concatenate([ref, np.zeros(T - S)]))
        ref_mean = np.mean(ref_s, axis=0)
        scale = np.maximum(np.abs(ref_mean), 1e-9 * pol["amount"][p])
        worst = max(worst, float(np.max(np.abs(pt[p] - ref_mean) / scale)))
    print(f"trajectory form {rsv.FORM_NAMES[form]}: max rel err {worst:.3e}")
    assert worst <= TOL[form]


def test_edge_cases(ctx):
    """Empty portfolio; policies with nothing left to pay (age at the limiting
    age); an endowment at maturity (term 0: reserve = sum assured); one
    scenario; horizon truncation; two decrement tables."""
    tab = synth.gm_monthly_survival()
    tab2 = synth.gm_monthly_survival(A=0.0003, B=0.00002)
    v = synth.vasicek_paths(1, 1500, seed=3)
    pol = synth.portfolio_mix(8, seed=3)
    pol["age1_m"][:3] = [1440, 1439, 0]
    pol["product"][:3] = [0, 0, 0]
    pol["term_m"][:3] = 0
    pol["product"][3], pol["term_m"][3] = 3, 0
    pol["product"][4], pol["age2_m"][4], pol["reversion"][4] = 1, 400, 0.75
    pol["table2"][4], pol["term_m"][4] = 1, 0
    for form in FORMS:
        V0, tot = run(ctx, pol, tab, v, form, tables=[tab, tab2])
        ref, _ = oracle.reserves_batch(pol, np.stack([tab, tab2]), v)
        assert V0[0, 0] == 0.0
        assert V0[3, 0] == pol["amount"][3]
        assert rel_err(V0, ref, pol["amount"]).max() <= TOL[form]
        Vh, _ = run(ctx, pol, tab, v, form, horizon=100, tables=[tab, tab2])
        refh, _ = oracle.reserves_batch(pol, np.stack([tab, tab2]), v, horizon=100)
        assert rel_err(Vh, refh, pol["amount"]).max() <= TOL[form]
    empty = synth.take(pol, slice(0, 0))
    rsv.rsv_load_portfolio(ctx, empty)
    tot = np.ones(1)
    rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F32_COMP, rsv.RSV_OUT_SCEN_TOTAL, scen_total=tot)
    assert tot[0] == 0.0


def test_assumption_and_state_errors(ctx):
    tab = synth.gm_monthly_survival()
    with pytest.raises(rsv.RsvError) as e:
        rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F32, rsv.RSV_OUT_SCEN_TOTAL, scen_total=np.zeros(1))
    assert e.value.status == rsv.RSV_E_STATE
    bad = tab.copy()
    bad[5] = 1.5
    with pytest.raises(rsv.RsvError) as e:
        rsv.rsv_load_decrements(ctx, 0, bad)
    assert e.value.status == rsv.RSV_E_ASSUMPTION
    v = synth.flat_scenarios(n_steps=100)
    v[0, 7] = -0.1
    with pytest.raises(rsv.RsvError) as e:
        rsv.rsv_load_scenarios(ctx, v)
    assert e.value.status == rsv.RSV_E_ASSUMPTION
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_scenarios(ctx, synth.flat_scenarios(n_steps=100))
    pol = synth.portfolio_single_life(4)
    rsv.rsv_load_portfolio(ctx, pol)     # whole-life annuities need > 100 steps
    with pytest.raises(rsv.RsvError) as e:
        rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F32, rsv.RSV_OUT_SCEN_TOTAL, scen_total=np.zeros(1))
    assert e.value.status == rsv.RSV_E_ASSUMPTION
    pol = synth.portfolio_mix(10, seed=1)
    pol["reversion"][pol["product"] == 1] = 1.2
    rsv.rsv_load_scenarios(ctx, synth.flat_scenarios(n_steps=1200))
    rsv.rsv_load_portfolio(ctx, pol)
    with pytest.raises(rsv.RsvError) as e:
        rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F32, rsv.RSV_OUT_SCEN_TOTAL, scen_total=np.zeros(1))
    assert e.value.status == rsv.RSV_E_ASSUMPTION
    pol["reversion"][:] = 0.5
    pol["product"][0] = 10   # no such product
    rsv.rsv_load_portfolio(ctx, pol)
    with pytest.raises(rsv.RsvError) as e:
        rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F32, rsv.RSV_OUT_SCEN_TOTAL, scen_total=np.zeros(1))
    assert e.value.status == rsv.RSV_E_ARG


def test_deterministic_reruns(ctx):
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_mix(500, seed=2)
    v = synth.vasicek_paths(64, 1200, seed=2)
    a = run(ctx, pol, tab, v, rsv.RSV_FORM_F32_COMP)
    b = run(ctx, pol, tab, v, rsv.RSV_FORM_F32_COMP)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("form", [rsv.RSV_FORM_F64, rsv.RSV_FORM_F32_COMP])
def test_per_step_means_reproducible(ctx, form):
    """The per-(policy, step) means over scenarios are summed in a fixed order
    (a warp's lanes by a butterfly, its scenario chunks one after another): two
    runs give the same bits, with many chunks per policy."""
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_mix(40, seed=12)
    v = synth.vasicek_paths(600, 1200, seed=12)
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_load_scenarios(ctx, v)
    runs = []
    for _ in range(3):
        pt = np.zeros((40, 1201))
        rsv.rsv_compute_reserves(ctx, form, rsv.RSV_OUT_PT_MEAN, pt_mean=pt)
        runs.append(pt)
    assert np.array_equal(runs[0], runs[1]) and np.array_equal(runs[0], runs[2])
    for p in range(3):   # the mean of the oracle's r_t over all 600 scenarios
        rows = []
        for s in range(600):
            r = oracle.chain(int(pol["product"][p]), int(pol["age1_m"][p]), float(pol["amount"][p]), tab, v[s],
                             age2=int(pol["age2_m"][p]), term=int(pol["term_m"][p]),
                             rho=float(pol["reversion"][p]))[:, 0]
            rows.append(np.concatenate([r, np.zeros(1201 - len(r))]))
        ref = np.mean(rows, axis=0)
        scale = np.maximum(np.abs(ref), 1e-9 * pol["amount"][p])
        assert np.max(np.abs(runs[0][p] - ref) / scale) <= TOL[form]


def test_config2_full_size_sampled(ctx):
    """100,000-policy mix x 1,000 Vasicek scenarios x 1,200 steps, the benchmark's
    launch configuration (tuned variant, device outputs): sampled policies
    against the oracle, and the FP64 totals against the FP64 sum of V0."""
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_mix(100_000, seed=0)
    v = synth.vasicek_paths(1000, 1200, seed=0)
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_load_scenarios(ctx, v)
    form = rsv.RSV_FORM_F32_COMP
    rsv.rsv_tune(ctx, form, reps=1)
    V0 = torch.empty((100_000, 1000), dtype=torch.float32, device="cuda")
    tot = torch.empty(1000, dtype=torch.float64, device="cuda")
    rsv.rsv_compute_reserves(ctx, form, V0T, on_device=True, V0=V0, scen_total=tot)
    rsv.rsv_synchronize(ctx)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(100_000, 300, replace=False))
    sub = synth.take(pol, idx)
    ref, _ = oracle.reserves_batch(sub, tab, v)
    got = V0[torch.as_tensor(idx, device="cuda")].double().cpu().numpy()
    # V0 is stored as FP32: its rounding (2^-24 relative) adds to the recurrence error
    err = rel_err(got, ref, sub["amount"])
    print(f"config-2 sampled: max rel err {err.max():.3e}")
    assert err.max() <= 1e-6
    host_sum = V0.double().sum(dim=0).cpu().numpy()
    assert np.max(np.abs(tot.cpu().numpy() - host_sum) / host_sum) <= 1e-9


@pytest.mark.parametrize("form", [rsv.RSV_FORM_F32, rsv.RSV_FORM_F32_COMP])
def test_config5_full_size_sampled(ctx, form):
    """1,000,000 single-life annuities (ages 60-90) x 1,000 Vasicek scenarios x
    600 monthly steps (50 years: the projection is truncated there with
    r_600 = 0), plain batched FP32 and compensated FP32, device outputs: 4 GB
    of V0.  Sampled policies against the oracle with the same horizon; the
    FP64 totals against the FP64 sum of V0."""
    tab = synth.gm_monthly_survival()
    n = 1_000_000
    pol = synth.portfolio_single_life(n, seed=5)
    v = synth.vasicek_paths(1000, 600, seed=5)
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_load_scenarios(ctx, v)
    V0 = torch.empty((n, 1000), dtype=torch.float32, device="cuda")
    tot = torch.empty(1000, dtype=torch.float64, device="cuda")
    rsv.rsv_compute_reserves(ctx, form, V0T, horizon=600, on_device=True, V0=V0, scen_total=tot)
    rsv.rsv_synchronize(ctx)
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(n, 200, replace=False))
    sub = synth.take(pol, idx)
    ref, _ = oracle.reserves_batch(sub, tab, v, horizon=600)
    got = V0[torch.as_tensor(idx, device="cuda")].double().cpu().numpy()
    err = rel_err(got, ref, sub["amount"])
    print(f"config-5 sampled, form {rsv.FORM_NAMES[form]}: max rel err {err.max():.3e}")
    assert err.max() <= (1e-6 if form == rsv.RSV_FORM_F32_COMP else TOL[form])
    host_sum = V0.double().sum(dim=0).cpu().numpy()
    assert np.max(np.abs(tot.cpu().numpy() - host_sum) / host_sum) <= 1e-9
    del V0


def test_time_scan_config1(ctx):
    """The parallel-in-time scan (one warp per chain, lanes over blocks of
    steps) on config 1: 1,000 annuities under one flat rate, FP64."""
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_single_life(1000, seed=0)
    v = synth.flat_scenarios(n_steps=720)
    V0, tot = run(ctx, pol, tab, v, rsv.RSV_FORM_F64, variant=rsv.RSV_VARIANT_TIME_SCAN)
    ref, ref_tot = oracle.reserves_batch(pol, tab, v)
    err = rel_err(V0, ref, pol["amount"])
    print(f"time scan config 1: max rel err {err.max():.3e}")
    assert err.max() <= 1e-12
    assert abs(tot[0] - ref_tot[0]) <= 1e-12 * ref_tot[0]


def test_time_scan_mix_trajectory_and_horizon(ctx):
    """The scan on every product and JL state (state0 0, 1, 2), 5 Vasicek
    scenarios: r_t at every t against the oracle's full-state recurrence, and a
    truncated horizon against the oracle's."""
    tab = synth.gm_monthly_survival()
    base = synth.portfolio_mix(24, seed=9)
    jl = np.where(base["product"] == 1)[0]
    extra = synth.take(base, np.concatenate([jl, jl]))
    extra["state0"][: len(jl)] = 1
    extra["state0"][len(jl):] = 2
    pol = {k: np.concatenate([base[k], extra[k]]) for k in base}
    n = len(pol["product"])
    v = synth.vasicek_paths(5, 1200, seed=9)
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_load_scenarios(ctx, v)
    T = v.shape[1]
    traj = np.zeros((n, T + 1, 5))
    rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F64, rsv.RSV_OUT_TRAJ, variant=rsv.RSV_VARIANT_TIME_SCAN, traj=traj)
    worst = 0.0
    for p in range(n):
        for s in range(5):
            r = oracle.chain(int(pol["product"][p]), int(pol["age1_m"][p]), float(pol["amount"][p]), tab, v[s],
                             age2=int(pol["age2_m"][p]), term=int(pol["term_m"][p]), rho=float(pol["reversion"][p]))
            ref = r[:, int(pol["state0"][p])]
            S = len(ref) - 1
            scale = np.maximum(np.abs(ref), 1e-9 * pol["amount"][p])
            worst = max(worst, float(np.max(np.abs(traj[p, : S + 1, s] - ref) / scale)))
            assert np.all(traj[p, S + 1:, s] == 0.0)
    print(f"time scan trajectory: max rel err {worst:.3e}")
    assert worst <= 1e-12
    V0, _ = run(ctx, pol, tab, v, rsv.RSV_FORM_F64, horizon=240, variant=rsv.RSV_VARIANT_TIME_SCAN)
    ref, _ = oracle.reserves_batch(pol, tab, v, horizon=240)
    assert rel_err(V0, ref, pol["amount"]).max() <= 1e-12
    for form in (rsv.RSV_FORM_F32, rsv.RSV_FORM_F32_COMP):
        with pytest.raises(rsv.RsvError) as e:
            run(ctx, pol, tab, v, form, variant=rsv.RSV_VARIANT_TIME_SCAN)
        assert e.value.status == rsv.RSV_E_ARG
    with pytest.raises(rsv.RsvError) as e:
        rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F64, rsv.RSV_OUT_PT_MEAN, variant=rsv.RSV_VARIANT_TIME_SCAN,
                                 pt_mean=np.zeros((n, T + 1)))
    assert e.value.status == rsv.RSV_E_ARG


def test_summation_variant_matches_oracle(ctx):
    """The O(S^2) summation-definition kernel: r_t at every t of every product
    and JL state against the oracle's summation, V0 of config 1, and errors."""
    tab = synth.gm_monthly_survival()
    base = synth.portfolio_mix(20, seed=10)
    jl = np.where(base["product"] == 1)[0]
    extra = synth.take(base, np.concatenate([jl, jl]))
    extra["state0"][: len(jl)] = 1
    extra["state0"][len(jl):] = 2
    pol = {k: np.concatenate([base[k], extra[k]]) for k in base}
    n = len(pol["product"])
    v = synth.vasicek_paths(3, 1200, seed=10)
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_load_scenarios(ctx, v)
    T = v.shape[1]
    traj = np.zeros((n, T + 1, 3))
    V0 = np.zeros((n, 3))
    rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F64, rsv.RSV_OUT_TRAJ | rsv.RSV_OUT_V0,
                             variant=rsv.RSV_VARIANT_SUMMATION, traj=traj, V0d=V0)
    worst = 0.0
    for p in range(n):
        for s in range(3):
            r = oracle.chain(int(pol["product"][p]), int(pol["age1_m"][p]), float(pol["amount"][p]), tab, v[s],
                             age2=int(pol["age2_m"][p]), term=int(pol["term_m"][p]), rho=float(pol["reversion"][p]),
                             method="summation")
            ref = r[:, int(pol["state0"][p])]
            S = len(ref) - 1
            scale = np.maximum(np.abs(ref), 1e-9 * pol["amount"][p])
            worst = max(worst, float(np.max(np.abs(traj[p, : S + 1, s] - ref) / scale)))
            assert np.all(traj[p, S + 1:, s] == 0.0)
            assert V0[p, s] == traj[p, 0, s]
    print(f"summation kernel trajectory: max rel err {worst:.3e}")
    assert worst <= 1e-12
    cpol = synth.portfolio_single_life(1000, seed=0)
    cv = synth.flat_scenarios(n_steps=720)
    got, tot = run(ctx, cpol, tab, cv, rsv.RSV_FORM_F64, variant=rsv.RSV_VARIANT_SUMMATION)
    ref, ref_tot = oracle.reserves_batch(cpol, tab, cv, method="summation")
    assert rel_err(got, ref, cpol["amount"]).max() <= 1e-12
    assert abs(tot[0] - ref_tot[0]) <= 1e-12 * ref_tot[0]
    with pytest.raises(rsv.RsvError) as e:
        run(ctx, cpol, tab, cv, rsv.RSV_FORM_F32_COMP, variant=rsv.RSV_VARIANT_SUMMATION)
    assert e.value.status == rsv.RSV_E_ARG


@pytest.mark.parametrize("n_scen", [300, 1000])
def test_host_outputs_pipelined_equal_device_outputs(ctx, n_scen):
    """With host V0 the library computes scenario column blocks and copies
    each block while the next one computes; the results must be bit-identical
    to the single launch with device outputs (FP32 and FP64 V0, totals)."""
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_mix(2000, seed=13)
    v = synth.vasicek_paths(n_scen, 1200, seed=13)
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_load_scenarios(ctx, v)
    n = len(pol["product"])
    for form in (rsv.RSV_FORM_F32_COMP, rsv.RSV_FORM_F32):
        dV0 = torch.empty((n, n_scen), dtype=torch.float32, device="cuda")
        dtot = torch.empty(n_scen, dtype=torch.float64, device="cuda")
        rsv.rsv_compute_reserves(ctx, form, V0T, on_device=True, V0=dV0, scen_total=dtot)
        rsv.rsv_synchronize(ctx)
        hV0 = np.zeros((n, n_scen), np.float32)
        htot = np.zeros(n_scen)
        rsv.rsv_compute_reserves(ctx, form, V0T, V0=hV0, scen_total=htot)
        assert np.array_equal(hV0, dV0.cpu().numpy())
        assert np.array_equal(htot, dtot.cpu().numpy())
        dV0d = torch.empty((n, n_scen), dtype=torch.float64, device="cuda")
        rsv.rsv_compute_reserves(ctx, form, rsv.RSV_OUT_V0, on_device=True, V0d=dV0d)
        rsv.rsv_synchronize(ctx)
        hV0d = np.zeros((n, n_scen))
        rsv.rsv_compute_reserves(ctx, form, rsv.RSV_OUT_V0, V0d=hV0d)
        assert np.array_equal(hV0d, dV0d.cpu().numpy())


@pytest.mark.parametrize("form", FORMS)
def test_two_life_products(ctx, form):
    """Joint-life and last-survivor annuities, joint term assurances and joint
    endowments, second-death term assurances and endowments in all three
    valuation states (two tables), mixed with the four single-table products,
    under ragged Vasicek scenarios: against the oracle's full two-life models
    (the nine-state one for the second death)."""
    tab = synth.gm_monthly_survival()
    tab2 = synth.gm_monthly_survival(A=0.0004, B=0.00002)
    two = synth.portfolio_two_life(300, seed=3, products=tuple(range(4, 10)))
    two["table2"][:] = 1
    ls = np.where(two["product"] >= 8)[0]
    two["state0"][ls[:20]] = 1    # second-death products valued with one life alive
    two["state0"][ls[20:40]] = 2
    pol = {k: np.concatenate([two[k], synth.portfolio_mix(60, seed=3)[k]]) for k in two}
    v = synth.vasicek_paths(70, 1200, seed=3)
    V0, tot = run(ctx, pol, tab, v, form, tables=[tab, tab2])
    ref, ref_tot = oracle.reserves_batch(pol, np.stack([tab, tab2]), v)
    err = rel_err(V0, ref, pol["amount"])
    for p in range(10):
        m = pol["product"] == p
        print(f"two-life form {rsv.FORM_NAMES[form]} product {p}: max rel err {err[m].max():.3e}")
    assert err.max() <= TOL[form]
    assert np.max(np.abs(tot - ref_tot) / ref_tot) <= TOL[form]
    if form == rsv.RSV_FORM_F64:   # the time scan and the summation kernel on the same products
        for var in (rsv.RSV_VARIANT_TIME_SCAN, rsv.RSV_VARIANT_SUMMATION):
            V0s, _ = run(ctx, pol, tab, v, form, variant=var, tables=[tab, tab2])
            assert rel_err(V0s, ref, pol["amount"]).max() <= 1e-12


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("payment", [rsv.RSV_PAY_START, rsv.RSV_PAY_FRACTION])
def test_payment_within_the_step(ctx, form, payment):
    """Annuities paid at the start of each month (f = 0) or at f = 1/2 (Eq.
    generalForm with W_{t,f} and v^f): every annuity product and JL state
    against the oracle's general-f recurrence; assurances stay at f = 1."""
    tab = synth.gm_monthly_survival()
    base = synth.portfolio_mix(24, seed=16)
    two = synth.portfolio_two_life(16, seed=16)
    jl = np.where(base["product"] == 1)[0]
    extra = synth.take(base, np.concatenate([jl, jl]))
    extra["state0"][: len(jl)] = 1
    extra["state0"][len(jl):] = 2
    pol = {k: np.concatenate([base[k], extra[k], two[k]]) for k in base}
    n = len(pol["product"])
    v = synth.vasicek_paths(40, 1200, seed=16)
    # f = 1/2 under a constant force and a constant rate within each month
    tab_f = np.sqrt(tab) if payment == rsv.RSV_PAY_FRACTION else np.ones_like(tab)
    v_f = np.sqrt(v) if payment == rsv.RSV_PAY_FRACTION else np.ones_like(v)
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_load_scenarios(ctx, v)
    if payment == rsv.RSV_PAY_FRACTION:
        rsv.rsv_load_decrements_fraction(ctx, 0, tab_f)
        rsv.rsv_load_scenarios_fraction(ctx, v_f)
    V0 = np.zeros((n, 40))
    tot = np.zeros(40)
    rsv.rsv_compute_reserves(ctx, form, V0T, payment=payment, V0d=V0, scen_total=tot)
    ref = np.zeros((n, 40))
    for p in range(n):
        prod = int(pol["product"][p])
        annuity = prod in (0, 1, 4, 5)
        for s in range(40):
            kw = dict(age2=int(pol["age2_m"][p]), term=int(pol["term_m"][p]), rho=float(pol["reversion"][p]))
            if annuity:
                kw.update(table_fx=tab_f, table_fy=tab_f, vf=v_f[s])
            r = oracle.chain(prod, int(pol["age1_m"][p]), float(pol["amount"][p]), tab, v[s], **kw)
            ref[p, s] = r[0, int(pol["state0"][p])]
    err = rel_err(V0, ref, pol["amount"])
    print(f"payment {payment} form {rsv.FORM_NAMES[form]}: max rel err {err.max():.3e}")
    assert err.max() <= TOL[form]
    assert np.max(np.abs(tot - ref.sum(axis=0)) / ref.sum(axis=0)) <= TOL[form]
    with pytest.raises(rsv.RsvError) as e:   # no per-step outputs with payments within the step
        rsv.rsv_compute_reserves(ctx, form, rsv.RSV_OUT_TRAJ, payment=payment, traj=np.zeros((n, 1201, 40)))
    assert e.value.status == rsv.RSV_E_ARG


def test_payment_fraction_needs_its_inputs(ctx):
    tab = synth.gm_monthly_survival()
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, synth.portfolio_single_life(10))
    rsv.rsv_load_scenarios(ctx, synth.vasicek_paths(8, 1200, seed=1))
    with pytest.raises(rsv.RsvError) as e:
        rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F64, rsv.RSV_OUT_V0, payment=rsv.RSV_PAY_FRACTION,
                                 V0d=np.zeros((10, 8)))
    assert e.value.status == rsv.RSV_E_STATE
    with pytest.raises(rsv.RsvError) as e:
        rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F64, rsv.RSV_OUT_V0, payment=7, V0d=np.zeros((10, 8)))
    assert e.value.status == rsv.RSV_E_ARG


def _schedule_rows(sch, n_steps):
    """The oracle's expansion of each policy's payment schedule."""
    return np.stack([oracle.schedule(n_steps, every=int(sch["every"][i]), first=int(sch["first"][i]),
                                     since=int(sch["since"][i]), steps_per_year=int(sch["steps_per_year"][i]),
                                     escalation=float(sch["escalation"][i]), increase=float(sch["increase"][i]))
                     for i in range(len(sch["every"]))])


def _cf_portfolio(n_single, n_two, seed):
    base = synth.portfolio_mix(n_single, seed=seed)
    two = synth.portfolio_two_life(n_two, seed=seed, products=tuple(range(4, 10)))
    two["table2"][:] = 1
    jl = np.where(base["product"] == 1)[0][:8]
    extra = synth.take(base, np.concatenate([jl, jl]))
    extra["state0"][: len(jl)] = 1
    extra["state0"][len(jl):] = 2
    return {k: np.concatenate([base[k], extra[k], two[k]]) for k in base}


@pytest.mark.parametrize("form", FORMS)
def test_payment_schedules(ctx, form):
    """Monthly and annual payments, escalating (3%, 4.25%, 5%) and increasing
    annuities and assurances (Section 4.1.1, 4.6), every product, expanded on
    the device from per-policy schedules: against the oracle with its own
    expansion of the same schedules."""
    tab = synth.gm_monthly_survival()
    tab2 = synth.gm_monthly_survival(A=0.0004, B=0.00002)
    pol = _cf_portfolio(200, 80, seed=21)
    n, n_scen, T = len(pol["product"]), 70, 1200
    sch = synth.payment_schedules(n, seed=21, annual_share=0.3, escalating_share=0.3, increasing_share=0.2)
    v = synth.vasicek_paths(n_scen, T, seed=21)
    rsv.rsv_load_schedules(ctx, sch, T)
    V0, tot = run(ctx, pol, tab, v, form, tables=[tab, tab2])
    cf = _schedule_rows(sch, T)
    ref, ref_tot = oracle.reserves_batch(pol, np.stack([tab, tab2]), v, cf=cf)
    err = rel_err(V0, ref, pol["amount"])
    print(f"schedules form {rsv.FORM_NAMES[form]}: max rel err {err.max():.3e}")
    assert err.max() <= TOL[form]
    assert np.max(np.abs(tot - ref_tot) / ref_tot) <= TOL[form]
    # level schedules reproduce the level valuation of the fast kernels
    lvl = {k: np.asarray(x).copy() for k, x in sch.items()}
    lvl["every"][:], lvl["first"][:], lvl["escalation"][:], lvl["increase"][:] = 1, 0, 0.0, 0.0
    rsv.rsv_load_schedules(ctx, lvl, T)
    V1, _ = run(ctx, pol, tab, v, form, tables=[tab, tab2])
    rsv.rsv_clear_cashflows(ctx)
    V2, _ = run(ctx, pol, tab, v, form, tables=[tab, tab2])
    assert rel_err(V1, V2, pol["amount"]).max() <= 2 * TOL[form]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("payment", [rsv.RSV_PAY_START, rsv.RSV_PAY_FRACTION])
def test_cash_flow_rows_with_payment_within_the_step(ctx, form, payment):
    """Explicit per-step multipliers (random, a third of them zero, decreasing
    assurance benefits) with the annuity paid at f = 0 or f = 1/2."""
    tab = synth.gm_monthly_survival()
    pol = _cf_portfolio(40, 16, seed=22)
    pol["table2"][:] = 0
    n, n_scen, T = len(pol["product"]), 40, 1200
    rng = np.random.default_rng(22)
    cf = rng.uniform(0.0, 2.0, (n, T))
    cf[rng.uniform(size=(n, T)) < 0.33] = 0.0
    ass = np.isin(pol["product"], (2, 3, 6, 7, 8, 9))
    cf[ass] = np.maximum(0.0, 1.0 - np.arange(T) / 600.0)[None, :]
    v = synth.vasicek_paths(n_scen, T, seed=22)
    tab_f = np.sqrt(tab) if payment == rsv.RSV_PAY_FRACTION else np.ones_like(tab)
    v_f = np.sqrt(v) if payment == rsv.RSV_PAY_FRACTION else np.ones_like(v)
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_load_scenarios(ctx, v)
    rsv.rsv_load_cashflows(ctx, cf)
    if payment == rsv.RSV_PAY_FRACTION:
        rsv.rsv_load_decrements_fraction(ctx, 0, tab_f)
        rsv.rsv_load_scenarios_fraction(ctx, v_f)
    V0 = np.zeros((n, n_scen))
    rsv.rsv_compute_reserves(ctx, form, rsv.RSV_OUT_V0, payment=payment, V0d=V0)
    ref = np.zeros((n, n_scen))
    for p in range(n):
        prod = int(pol["product"][p])
        kw = dict(age2=int(pol["age2_m"][p]), term=int(pol["term_m"][p]), rho=float(pol["reversion"][p]), cf=cf[p])
        if prod in (0, 1, 4, 5):
            kw.update(table_fx=tab_f, table_fy=tab_f)
        for s in range(n_scen):
            if prod in (0, 1, 4, 5):
                kw["vf"] = v_f[s]
            r = oracle.chain(prod, int(pol["age1_m"][p]), float(pol["amount"][p]), tab, v[s], **kw)
            ref[p, s] = r[0, int(pol["state0"][p])]
    err = rel_err(V0, ref, pol["amount"])
    print(f"cash-flow rows payment {payment} form {rsv.FORM_NAMES[form]}: max rel err {err.max():.3e}")
    assert err.max() <= TOL[form]


def test_cash_flows_time_scan_and_summation(ctx):
    """The FP64 time scan (V0 and the trajectory) and the summation kernel with
    payment schedules, against the oracle."""
    tab = synth.gm_monthly_survival()
    pol = _cf_portfolio(30, 12, seed=23)
    pol["table2"][:] = 0
    n, n_scen, T = len(pol["product"]), 6, 1200
    sch = synth.payment_schedules(n, seed=23, annual_share=0.5, escalating_share=0.5, increasing_share=0.3)
    v = synth.vasicek_paths(n_scen, T, seed=23)
    rsv.rsv_load_schedules(ctx, sch, T)
    cf = _schedule_rows(sch, T)
    ref, _ = oracle.reserves_batch(pol, tab, v, cf=cf)
    for var in (rsv.RSV_VARIANT_TIME_SCAN, rsv.RSV_VARIANT_SUMMATION):
        V0, _ = run(ctx, pol, tab, v, rsv.RSV_FORM_F64, variant=var)
        assert rel_err(V0, ref, pol["amount"]).max() <= 1e-12, var
    traj = np.zeros((n, T + 1, n_scen))
    rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F64, rsv.RSV_OUT_TRAJ, variant=rsv.RSV_VARIANT_TIME_SCAN, traj=traj)
    for p in range(0, n, 5):
        r = oracle.chain(int(pol["product"][p]), int(pol["age1_m"][p]), float(pol["amount"][p]), tab, v[2],
                         age2=int(pol["age2_m"][p]), term=int(pol["term_m"][p]), rho=float(pol["reversion"][p]),
                         cf=cf[p])
        S = r.shape[0] - 1
        got = traj[p, : S + 1, 2]
        want = r[:, int(pol["state0"][p])]
        assert np.max(np.abs(got - want) / np.maximum(np.abs(want), 1e-9 * pol["amount"][p])) <= 1e-12


def test_cash_flow_errors(ctx):
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_single_life(10)
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_load_scenarios(ctx, synth.vasicek_paths(8, 1200, seed=1))
    V0 = np.zeros((10, 8))
    with pytest.raises(rsv.RsvError) as e:      # negative multiplier
        rsv.rsv_load_cashflows(ctx, -np.ones((10, 1200)))
    assert e.value.status == rsv.RSV_E_ASSUMPTION
    bad = synth.payment_schedules(10, seed=1)
    bad["since"][3] = 12
    with pytest.raises(rsv.RsvError) as e:
        rsv.rsv_load_schedules(ctx, bad, 1200)
    assert e.value.status == rsv.RSV_E_ARG
    rsv.rsv_load_cashflows(ctx, np.ones((9, 1200)))   # rows for another portfolio size
    with pytest.raises(rsv.RsvError) as e:
        rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F64, rsv.RSV_OUT_V0, V0d=V0)
    assert e.value.status == rsv.RSV_E_STATE
    rsv.rsv_load_cashflows(ctx, np.ones((10, 5)))     # rows shorter than the projections
    with pytest.raises(rsv.RsvError) as e:
        rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F64, rsv.RSV_OUT_V0, V0d=V0)
    assert e.value.status == rsv.RSV_E_STATE
    rsv.rsv_load_cashflows(ctx, np.ones((10, 1200)))
    with pytest.raises(rsv.RsvError) as e:      # per-step outputs need the scan or the summation
        rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F64, rsv.RSV_OUT_TRAJ, traj=np.zeros((10, 1201, 8)))
    assert e.value.status == rsv.RSV_E_ARG
    rsv.rsv_clear_cashflows(ctx)
    rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F64, rsv.RSV_OUT_V0, V0d=V0)


def test_cash_flows_split_launch_host_and_device_outputs(ctx):
    """Level and varying cash flows in one portfolio: the level policies run on
    the fast kernel and the others on the general one, in column blocks when
    the outputs go to the host.  Host and device outputs are bit-identical, and
    the level policies equal a run without cash flows."""
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_mix(400, seed=24)
    n, n_scen, T = 400, 300, 1200
    v = synth.vasicek_paths(n_scen, T, seed=24)
    sch = synth.payment_schedules(n, seed=24)
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_load_scenarios(ctx, v)
    V_level = np.zeros((n, n_scen))
    rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F32_COMP, rsv.RSV_OUT_V0, V0d=V_level)
    rsv.rsv_load_schedules(ctx, sch, T)
    host = np.zeros((n, n_scen))
    rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F32_COMP, rsv.RSV_OUT_V0, V0d=host)
    dev = torch.zeros((n, n_scen), dtype=torch.float64, device="cuda")
    rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F32_COMP, rsv.RSV_OUT_V0, on_device=True, V0d=dev)
    torch.cuda.synchronize()
    assert np.array_equal(host, dev.cpu().numpy())
    level = (sch["every"] == 1) & (sch["escalation"] == 0) & (sch["increase"] == 0)
    assert 0 < level.sum() < n
    assert np.array_equal(host[level], V_level[level])
    ref, _ = oracle.reserves_batch(pol, tab, v[:20], cf=_schedule_rows(sch, T))
    assert rel_err(host[:, :20], ref, pol["amount"]).max() <= TOL[rsv.RSV_FORM_F32_COMP]


@pytest.mark.parametrize("form", [rsv.RSV_FORM_F64, rsv.RSV_FORM_F32_COMP])
def test_cash_flows_with_horizon(ctx, form):
    """A horizon truncates the projection (r_h = 0) with varying cash flows as
    well: the rows beyond it are never read."""
    tab = synth.gm_monthly_survival()
    pol = _cf_portfolio(60, 24, seed=25)
    pol["table2"][:] = 0
    n, n_scen, T, h = len(pol["product"]), 33, 1200, 300
    sch = synth.payment_schedules(n, seed=25, annual_share=0.4, escalating_share=0.4, increasing_share=0.2)
    v = synth.vasicek_paths(n_scen, T, seed=25)
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_load_scenarios(ctx, v)
    rsv.rsv_load_schedules(ctx, sch, h)   # rows only as long as the horizon
    V0 = np.zeros((n, n_scen))
    rsv.rsv_compute_reserves(ctx, form, rsv.RSV_OUT_V0, horizon=h, V0d=V0)
    cf = np.zeros((n, T))
    cf[:, :h] = _schedule_rows(sch, h)
    ref, _ = oracle.reserves_batch(pol, tab, v, horizon=h, cf=cf)
    assert rel_err(V0, ref, pol["amount"]).max() <= TOL[form]


def test_bounded_wait_times_out_and_the_context_survives(ctx):
    """Failure detection without a GPU fault: a staging wait whose barrier can
    never complete runs out, the kernel reports RSV_E_TIMEOUT and returns, and
    the same device and context keep working."""
    stream = torch.cuda.current_stream()
    assert rsv.rsv_selftest_bounded_wait(0, stream, never_completes=False) == rsv.RSV_OK
    assert rsv.rsv_selftest_bounded_wait(0, stream, never_completes=True) == rsv.RSV_E_TIMEOUT
    assert rsv.rsv_selftest_bounded_wait(0, stream, never_completes=False) == rsv.RSV_OK
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_single_life(50)
    v = synth.vasicek_paths(40, 720, seed=1)
    V0, _ = run(ctx, pol, tab, v, rsv.RSV_FORM_F64)
    ref, _ = oracle.reserves_batch(pol, tab, v)
    assert rel_err(V0, ref, pol["amount"]).max() <= 1e-12
