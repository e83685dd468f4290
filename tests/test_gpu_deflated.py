"""GPU parity of the deflated form (RSV_FORM_F32_DEFLATED) against the FP64 oracle.

The form runs the backward recurrence in deflated units, U_t = U_{t+1} +
D_{t+1} E_t (one FP32 fused multiply-add per chain-step), with the discount
products D in FP64 per scenario and the life table in FP64, and compensated
accumulation.  Its bound: every reserve within about 15 x 2^-24 = 8.9e-7 of
the value on the FP64 inputs (8 FP32 roundings per 8-term partial sum, one
for adding two spans' partial sums in the variants that fold once per
block, one for joining the two partial sums, one rounding each of D and of
the expected cash flow E, up to three for E of the reversionary annuity;
the double-float fold is exact to 2^-48).  The tests hold it to the 1e-6 target
of the compensated forms, and FP32 V0 adds its own rounding (2^-24).
Error metric: rel = |V_gpu - V_ref| / max(|V_ref|, 1e-9 * amount).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1401_1757_gb300 import rsv

pytestmark = pytest.mark.gpu

DEFL = rsv.RSV_FORM_F32_DEFLATED
TOL = 1e-6
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


def load(ctx, pol, tables, v):
    for i, t in enumerate(tables):
        rsv.rsv_load_decrements(ctx, i, t)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_load_scenarios(ctx, v)


def run(ctx, pol, tables, v, horizon=0, variant=-1):
    load(ctx, pol, tables, v)
    n, S = len(pol["product"]), v.shape[0]
    V0 = np.zeros((n, S))
    tot = np.zeros(S)
    rsv.rsv_compute_reserves(ctx, DEFL, V0T, horizon=horizon, variant=variant, V0d=V0, scen_total=tot)
    return V0, tot


def with_jl_states(base):
    """The portfolio plus its reversionary annuities valued in states 01 and 10."""
    jl = np.where(base["product"] == 1)[0]
    extra = synth.take(base, np.concatenate([jl, jl]))
    extra["state0"][: len(jl)] = 1
    extra["state0"][len(jl):] = 2
    return {k: np.concatenate([base[k], extra[k]]) for k in base}


def test_config1_full(ctx):
    """1,000 single-life annuities (ages 60-90), one flat 4% scenario: the
    systematic rounding of a constant v is what compounds in plain FP32; the
    deflated form never multiplies a rounded value by the next factor."""
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_single_life(1000, seed=0)
    v = synth.flat_scenarios(n_steps=720)
    V0, tot = run(ctx, pol, [tab], v)
    ref, ref_tot = oracle.reserves_batch(pol, tab, v)
    err = rel_err(V0, ref, pol["amount"])
    print(f"config-1 deflated: max rel err {err.max():.3e}, median {np.median(err):.3e}")
    assert err.max() <= TOL
    assert abs(tot[0] - ref_tot[0]) <= TOL * ref_tot[0]


def test_mix_every_state_ragged(ctx):
    """The four-product mix plus the reversionary annuities in states 01 and 10,
    under 157 Vasicek scenarios (ragged against every chunk width) of 1,200 steps."""
    tab = synth.gm_monthly_survival()
    pol = with_jl_states(synth.portfolio_mix(400, seed=21))
    v = synth.vasicek_paths(157, 1200, seed=21)
    V0, tot = run(ctx, pol, [tab], v)
    ref, ref_tot = oracle.reserves_batch(pol, tab, v)
    err = rel_err(V0, ref, pol["amount"])
    for p in range(4):
        for s0 in range(3):
            m = (pol["product"] == p) & (pol["state0"] == s0)
            if m.any():
                print(f"deflated product {p} state {s0}: max rel err {err[m].max():.3e}")
    assert err.max() <= TOL
    assert np.max(np.abs(tot - ref_tot) / ref_tot) <= TOL


def test_every_variant_agrees(ctx):
    tab = synth.gm_monthly_survival()
    pol = with_jl_states(synth.portfolio_mix(260, seed=5))
    v = synth.vasicek_paths(70, 1200, seed=5)
    ref, ref_tot = oracle.reserves_batch(pol, tab, v)
    assert rsv.rsv_variant_count(DEFL) >= 4
    for var in range(rsv.rsv_variant_count(DEFL)):
        V0, tot = run(ctx, pol, [tab], v, variant=var)
        err = rel_err(V0, ref, pol["amount"]).max()
        print(f"{rsv.rsv_variant_name(DEFL, var)}: max rel err {err:.3e}")
        assert err <= TOL, (rsv.rsv_variant_name(DEFL, var), err)
        assert np.max(np.abs(tot - ref_tot) / ref_tot) <= TOL


def test_packed_variants_give_the_scalar_bits(ctx):
    """The packed-pair (f32x2) variants round every operation as the scalar
    ones do, and their fold is the same ordered Fast2Sum on pairs of chains:
    their reserves are bit-identical to the scalar variant of the same shape,
    on the whole mix with every state."""
    tab = synth.gm_monthly_survival()
    pol = with_jl_states(synth.portfolio_mix(300, seed=8))
    v = synth.vasicek_paths(201, 1200, seed=8)
    names = {rsv.rsv_variant_name(DEFL, i): i for i in range(rsv.rsv_variant_count(DEFL))}
    pairs = [(names[n[:-3]], i) for n, i in names.items() if n.endswith(" x2") and n[:-3] in names]
    assert pairs
    for scalar, packed in pairs:
        a, ta = run(ctx, pol, [tab], v, variant=scalar)
        b, tb = run(ctx, pol, [tab], v, variant=packed)
        assert np.array_equal(a, b), rsv.rsv_variant_name(DEFL, packed)
        assert np.array_equal(ta, tb)


def test_tmem_variants_give_the_packed_bits(ctx):
    """The variants that keep each chain's double-float sum in tensor memory
    (16 warps at 128 registers) run the packed variants' arithmetic: their
    reserves are bit-identical to the register variant's (the per-scenario
    totals group the policies by a different super-tile width)."""
    tab = synth.gm_monthly_survival()
    pol = with_jl_states(synth.portfolio_mix(300, seed=8))
    v = synth.vasicek_paths(201, 1200, seed=8)
    names = {rsv.rsv_variant_name(DEFL, i): i for i in range(rsv.rsv_variant_count(DEFL))}
    tms = [i for n, i in names.items() if n.endswith(" tm")]
    assert tms
    a, ta = run(ctx, pol, [tab], v, variant=names["deflated P4xM4 nw11 buf8 x2"])
    for t in tms:
        b, tb = run(ctx, pol, [tab], v, variant=t)
        assert np.array_equal(a, b), rsv.rsv_variant_name(DEFL, t)
        assert np.max(np.abs(tb - ta) / np.abs(ta)) <= 1e-14


def test_negative_rates_and_steep_weights(ctx):
    """Scenarios with negative rates (discount factors above 1, so the weights
    can grow along the chain) and a steep constant-force table: the ordered
    folds and the table range stay within the bound."""
    tab = synth.gm_monthly_survival()
    steep = synth.constant_force_table(0.5)
    pol = synth.portfolio_mix(300, seed=31)
    pol["table1"][: 100] = 1
    pol["table2"][pol["product"] == 1] = 1
    v = synth.vasicek_paths(96, 1200, seed=31, b=-0.02, sigma=0.03, r0=-0.01)
    assert (v > 1.0).any()
    V0, tot = run(ctx, pol, [tab, steep], v)
    ref, ref_tot = oracle.reserves_batch(pol, np.stack([tab, steep]), v)
    err = rel_err(V0, ref, pol["amount"])
    print(f"negative rates, steep table: max rel err {err.max():.3e}")
    assert err.max() <= TOL
    assert np.max(np.abs(tot - ref_tot) / ref_tot) <= TOL


def test_edge_cases(ctx):
    """Nothing left to pay (age at the limiting age), an endowment at maturity
    (reserve = sum assured), one scenario, a horizon, two tables, an empty
    portfolio."""
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
    tabs = [tab, tab2]
    V0, _ = run(ctx, pol, tabs, v)
    ref, _ = oracle.reserves_batch(pol, np.stack(tabs), v)
    assert V0[0, 0] == 0.0
    assert abs(V0[3, 0] - pol["amount"][3]) <= 1e-7 * pol["amount"][3]
    assert rel_err(V0, ref, pol["amount"]).max() <= TOL
    for h in (1, 100, 333):
        Vh, _ = run(ctx, pol, tabs, v, horizon=h)
        refh, _ = oracle.reserves_batch(pol, np.stack(tabs), v, horizon=h)
        assert rel_err(Vh, refh, pol["amount"]).max() <= TOL, h
    rsv.rsv_load_portfolio(ctx, synth.take(pol, slice(0, 0)))
    tot = np.ones(1)
    rsv.rsv_compute_reserves(ctx, DEFL, rsv.RSV_OUT_SCEN_TOTAL, scen_total=tot)
    assert tot[0] == 0.0


def test_lives_at_and_past_the_limiting_age(ctx):
    """Term assurances that run past the limiting age (the benefit is then
    certain in the month the table ends), a life already past the table's end
    (death within the first month certain), an endowment at maturity past it,
    and reversionary annuities with one life past the limit (the other life's
    annuity, or the reversion from the first month)."""
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_mix(12, seed=6)
    spec = [(2, 1438, 0, 60), (2, 1440, 0, 12), (2, 1450, 0, 12), (3, 1450, 0, 0), (3, 1420, 0, 120),
            (1, 900, 1445, 0), (1, 1445, 700, 0), (1, 1300, 1300, 0), (0, 1440, 0, 0), (2, 30, 0, 480),
            (3, 1000, 0, 600), (1, 240, 1020, 0)]
    for i, (p, a1, a2, term) in enumerate(spec):
        pol["product"][i], pol["age1_m"][i], pol["age2_m"][i], pol["term_m"][i] = p, a1, a2, term
        pol["reversion"][i] = 0.8 if p == 1 else 0.0
    v = synth.vasicek_paths(40, 1500, seed=6)
    V0, tot = run(ctx, pol, [tab], v)
    ref, ref_tot = oracle.reserves_batch(pol, tab, v)
    err = rel_err(V0, ref, pol["amount"])
    print("limiting-age cases:", " ".join(f"{e:.1e}" for e in err.max(axis=1)))
    assert err.max() <= TOL
    assert np.max(np.abs(tot - ref_tot) / ref_tot) <= TOL
    # past the table's end: the whole sum at the end of the first month
    assert np.allclose(V0[2], pol["amount"][2] * v[:, 0], rtol=1e-7, atol=0)
    assert np.allclose(V0[3], pol["amount"][3], rtol=1e-7, atol=0)


def test_joint_and_last_survivor_annuities(ctx):
    """Joint-life and last-survivor annuities (two tables) beside the mix; the
    two-life assurances are not taken by this form (RSV_E_ARG)."""
    tab = synth.gm_monthly_survival()
    tab2 = synth.gm_monthly_survival(A=0.0004, B=0.00002)
    two = synth.portfolio_two_life(200, seed=3, products=(4, 5))
    two["table2"][:] = 1
    mix = synth.portfolio_mix(100, seed=4)
    pol = {k: np.concatenate([two[k], mix[k]]) for k in two}
    v = synth.vasicek_paths(45, 1200, seed=3)
    V0, tot = run(ctx, pol, [tab, tab2], v)
    ref, ref_tot = oracle.reserves_batch(pol, np.stack([tab, tab2]), v)
    err = rel_err(V0, ref, pol["amount"])
    print(f"joint and last-survivor annuities: max rel err {err.max():.3e}")
    assert err.max() <= TOL
    assert np.max(np.abs(tot - ref_tot) / ref_tot) <= TOL
    for prod in (6, 7, 8, 9):
        bad = synth.portfolio_two_life(4, seed=1, products=(prod,))
        rsv.rsv_load_portfolio(ctx, bad)
        with pytest.raises(rsv.RsvError) as e:
            rsv.rsv_compute_reserves(ctx, DEFL, rsv.RSV_OUT_V0, V0d=np.zeros((4, 45)))
        assert e.value.status == rsv.RSV_E_ARG


def test_requests_it_does_not_take(ctx):
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_mix(16, seed=2)
    v = synth.vasicek_paths(8, 1200, seed=2)
    load(ctx, pol, [tab], v)
    n, T = 16, 1200
    with pytest.raises(rsv.RsvError) as e:
        rsv.rsv_compute_reserves(ctx, DEFL, rsv.RSV_OUT_PT_MEAN, pt_mean=np.zeros((n, T + 1)))
    assert e.value.status == rsv.RSV_E_ARG
    with pytest.raises(rsv.RsvError) as e:
        rsv.rsv_compute_reserves(ctx, DEFL, rsv.RSV_OUT_V0, payment=rsv.RSV_PAY_START, V0d=np.zeros((n, 8)))
    assert e.value.status == rsv.RSV_E_ARG
    with pytest.raises(rsv.RsvError) as e:
        rsv.rsv_compute_reserves(ctx, DEFL, rsv.RSV_OUT_V0, variant=rsv.RSV_VARIANT_TIME_SCAN, V0d=np.zeros((n, 8)))
    assert e.value.status == rsv.RSV_E_ARG
    rsv.rsv_load_cashflows(ctx, np.ones((n, T)))
    with pytest.raises(rsv.RsvError) as e:
        rsv.rsv_compute_reserves(ctx, DEFL, rsv.RSV_OUT_V0, V0d=np.zeros((n, 8)))
    assert e.value.status == rsv.RSV_E_STATE
    rsv.rsv_clear_cashflows(ctx)
    # a table whose survival falls below 2^-220 is out of the form's range
    rsv.rsv_load_decrements(ctx, 0, synth.constant_force_table(2.0))
    with pytest.raises(rsv.RsvError) as e:
        rsv.rsv_compute_reserves(ctx, DEFL, rsv.RSV_OUT_V0, V0d=np.zeros((n, 8)))
    assert e.value.status == rsv.RSV_E_ARG


def test_deterministic_reruns(ctx):
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_mix(500, seed=2)
    v = synth.vasicek_paths(64, 1200, seed=2)
    a = run(ctx, pol, [tab], v)
    b = run(ctx, pol, [tab], v)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("n_scen", [300, 1000])
def test_host_outputs_pipelined_equal_device_outputs(ctx, n_scen):
    """Host V0 is computed in scenario column blocks, each copied while the next
    computes: bit-identical to one launch with device outputs."""
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_mix(2000, seed=13)
    v = synth.vasicek_paths(n_scen, 1200, seed=13)
    load(ctx, pol, [tab], v)
    n = len(pol["product"])
    dV0 = torch.empty((n, n_scen), dtype=torch.float32, device="cuda")
    dtot = torch.empty(n_scen, dtype=torch.float64, device="cuda")
    rsv.rsv_compute_reserves(ctx, DEFL, V0T, on_device=True, V0=dV0, scen_total=dtot)
    rsv.rsv_synchronize(ctx)
    hV0 = np.zeros((n, n_scen), np.float32)
    htot = np.zeros(n_scen)
    rsv.rsv_compute_reserves(ctx, DEFL, V0T, V0=hV0, scen_total=htot)
    assert np.array_equal(hV0, dV0.cpu().numpy())
    assert np.array_equal(htot, dtot.cpu().numpy())


def test_config2_full_size_sampled(ctx):
    """100,000-policy mix x 1,000 Vasicek scenarios x 1,200 steps in the
    benchmark's launch configuration (tuned variant, device outputs): sampled
    policies against the oracle; the FP64 totals against the FP64 sum of V0."""
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_mix(100_000, seed=0)
    v = synth.vasicek_paths(1000, 1200, seed=0)
    load(ctx, pol, [tab], v)
    rsv.rsv_tune(ctx, DEFL, reps=1)
    V0 = torch.empty((100_000, 1000), dtype=torch.float32, device="cuda")
    tot = torch.empty(1000, dtype=torch.float64, device="cuda")
    rsv.rsv_compute_reserves(ctx, DEFL, V0T, on_device=True, V0=V0, scen_total=tot)
    rsv.rsv_synchronize(ctx)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(100_000, 300, replace=False))
    sub = synth.take(pol, idx)
    ref, _ = oracle.reserves_batch(sub, tab, v)
    got = V0[torch.as_tensor(idx, device="cuda")].double().cpu().numpy()
    err = rel_err(got, ref, sub["amount"])
    print(f"config-2 sampled, deflated: max rel err {err.max():.3e}")
    assert err.max() <= TOL
    host_sum = V0.double().sum(dim=0).cpu().numpy()
    assert np.max(np.abs(tot.cpu().numpy() - host_sum) / host_sum) <= 1e-8


def test_config5_full_size_sampled(ctx):
    """1,000,000 single-life annuities x 1,000 Vasicek scenarios x 600 steps
    (the projection truncated at 50 years, r_600 = 0), device outputs: 4 GB of
    V0; sampled policies against the oracle with the same horizon."""
    tab = synth.gm_monthly_survival()
    n = 1_000_000
    pol = synth.portfolio_single_life(n, seed=5)
    v = synth.vasicek_paths(1000, 600, seed=5)
    load(ctx, pol, [tab], v)
    V0 = torch.empty((n, 1000), dtype=torch.float32, device="cuda")
    tot = torch.empty(1000, dtype=torch.float64, device="cuda")
    rsv.rsv_compute_reserves(ctx, DEFL, V0T, horizon=600, on_device=True, V0=V0, scen_total=tot)
    rsv.rsv_synchronize(ctx)
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(n, 200, replace=False))
    sub = synth.take(pol, idx)
    ref, _ = oracle.reserves_batch(sub, tab, v, horizon=600)
    got = V0[torch.as_tensor(idx, device="cuda")].double().cpu().numpy()
    err = rel_err(got, ref, sub["amount"])
    print(f"config-5 sampled, deflated: max rel err {err.max():.3e}")
    assert err.max() <= TOL
    host_sum = V0.double().sum(dim=0).cpu().numpy()
    assert np.max(np.abs(tot.cpu().numpy() - host_sum) / host_sum) <= 1e-8
    del V0


def test_pinned_host_v0_written_by_the_kernel(ctx):
    """A page-locked host V0 (FP32 or FP64) is written by the kernel itself; a
    pageable one is staged on the device and copied.  Both give the bits of
    the device-resident call."""
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_mix(700, seed=13)
    v = synth.vasicek_paths(300, 1200, seed=13)
    load(ctx, pol, [tab], v)
    n, S = len(pol["product"]), v.shape[0]
    Vd = torch.empty((n, S), device="cuda")
    Vdd = torch.empty((n, S), dtype=torch.float64, device="cuda")
    td = torch.empty(S, dtype=torch.float64, device="cuda")
    rsv.rsv_compute_reserves(ctx, DEFL, V0T, on_device=True, V0=Vd, V0d=Vdd, scen_total=td)
    ref, refd, reft = Vd.cpu().numpy(), Vdd.cpu().numpy(), td.cpu().numpy()
    for pinned in (True, False):
        Vh = torch.full((n, S), np.nan, dtype=torch.float32)
        Vhd = torch.full((n, S), np.nan, dtype=torch.float64)
        if pinned:
            Vh, Vhd = Vh.pin_memory(), Vhd.pin_memory()
        th = np.zeros(S)
        rsv.rsv_compute_reserves(ctx, DEFL, V0T, V0=Vh.numpy(), scen_total=th)
        assert np.array_equal(Vh.numpy(), ref), pinned
        assert np.array_equal(th, reft)
        rsv.rsv_compute_reserves(ctx, DEFL, rsv.RSV_OUT_V0, V0=Vh.numpy(), V0d=Vhd.numpy())
        assert np.array_equal(Vh.numpy(), ref) and np.array_equal(Vhd.numpy(), refd), pinned
