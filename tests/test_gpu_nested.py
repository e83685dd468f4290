"""GPU parity of the nested (brute-force) valuation against the FP64 oracle.

Both sides generate the same counter-based Philox4x32-10 / Box-Muller / exact
Vasicek scenarios from their own code; the paths then agree to FP64 rounding
of log, sin, cos and exp (1e-15), far below the tolerances of the forms.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1401_1757_gb300 import rsv

pytestmark = pytest.mark.gpu

TOL = {rsv.RSV_FORM_F64: 1e-11, rsv.RSV_FORM_F32_COMP: 1e-6, rsv.RSV_FORM_F32: 2e-4, rsv.RSV_FORM_F32_DEFLATED: 1e-6}


@pytest.fixture
def ctx():
    h = rsv.rsv_create(0, torch.cuda.current_stream())
    yield h
    rsv.rsv_destroy(h)


def nested(ctx, pol, tab, form, **spec):
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    NO, NN = spec["n_outer"], spec["n_nodes"]
    n_in = spec.get("n_inner", 1000) if spec.get("mode", 0) == rsv.RSV_NESTED_MC else 1
    out = dict(L_mean=np.zeros((NO, NN)), L_q995=np.zeros((NO, NN)), r_node=np.zeros((NO, NN)),
               D0=np.zeros((NO, NN)), L_all=np.zeros((NO, NN, n_in)))
    rsv.rsv_compute_nested(ctx, form, **spec, **out)
    return out


def mixed_portfolio(n=40, seed=12):
    pol = synth.portfolio_mix(n, seed=seed, age_lo_y=55, age_hi_y=85)
    jl = np.where(pol["product"] == 1)[0]
    pol["state0"][jl[:2]] = [1, 2]
    return pol


@pytest.mark.parametrize("form", [rsv.RSV_FORM_F64, rsv.RSV_FORM_F32_COMP, rsv.RSV_FORM_F32, rsv.RSV_FORM_F32_DEFLATED])
def test_nested_small_against_oracle(ctx, form):
    """3 outer paths (in batches of 2 and 1) x 5 nodes 24 months apart x 70 inner
    paths (ragged against the 32-path chunks), four-product mix with JL
    policies valued from every state."""
    tab = synth.gm_monthly_survival()
    pol = mixed_portfolio()
    spec = dict(n_outer=3, n_nodes=5, node_step_m=24, n_inner=70, seed=77, batch_outer=2)
    out = nested(ctx, pol, tab, form, **spec)
    worst = 0.0
    for o in range(3):
        for n in range(5):
            L, rn, d0 = oracle.nested_node(pol, tab, 77, o, n, np.arange(70), node_step=24)
            assert math.isclose(out["r_node"][o, n], rn, rel_tol=1e-12, abs_tol=1e-15)
            assert math.isclose(out["D0"][o, n], d0, rel_tol=1e-12)
            worst = max(worst, float(np.max(np.abs(out["L_all"][o, n] - L) / np.abs(L))))
    print(f"nested form {rsv.FORM_NAMES[form]}: max rel err {worst:.3e}")
    assert worst <= TOL[form]
    # node statistics from the same L_all
    srt = np.sort(out["L_all"], axis=2)
    assert np.allclose(out["L_mean"], out["L_all"].mean(axis=2), rtol=1e-13, atol=0)
    assert np.array_equal(out["L_q995"], srt[:, :, -1])          # ceil(0.005 * 70) = 1: the largest


def test_nested_deflated_unaligned_nodes_and_edges(ctx):
    """The deflated brute force with nodes 7 months apart (table runs start at
    every offset within a group of four), assurances that run past the
    limiting age or start past it, endowments maturing at a node, joint-life
    and last-survivor annuities (two tables), the reversionary annuity from
    every state: every (o, n, i) against the oracle; reruns bit-identical."""
    tab = synth.gm_monthly_survival()
    tab2 = synth.gm_monthly_survival(A=0.0004, B=0.00002)
    pol = mixed_portfolio(36, seed=17)
    two = synth.portfolio_two_life(8, seed=3, age_lo_y=55, age_hi_y=85, products=(4, 5))
    two["table2"][:] = 1
    pol = {k: np.concatenate([pol[k], two[k]]) for k in pol}
    spec_rows = [(2, 1430, 60), (2, 1445, 24), (3, 900, 21), (3, 1000, 7), (0, 1430, 0)]
    for i, (prod, age, term) in enumerate(spec_rows):
        pol["product"][i], pol["age1_m"][i], pol["term_m"][i] = prod, age, term
        pol["age2_m"][i], pol["reversion"][i], pol["state0"][i] = 0, 0.0, 0
    rsv.rsv_load_decrements(ctx, 1, tab2)
    spec = dict(n_outer=2, n_nodes=6, node_step_m=7, n_inner=70, seed=41)
    out = nested(ctx, pol, tab, rsv.RSV_FORM_F32_DEFLATED, **spec)
    worst = 0.0
    for o in range(2):
        for n in range(6):
            L, _, _ = oracle.nested_node(pol, np.stack([tab, tab2]), 41, o, n, np.arange(70), node_step=7)
            worst = max(worst, float(np.max(np.abs(out["L_all"][o, n] - L) / np.abs(L))))
    print(f"deflated nested, unaligned nodes: max rel err {worst:.3e}")
    assert worst <= 1e-6
    again = nested(ctx, pol, tab, rsv.RSV_FORM_F32_DEFLATED, **spec)
    assert np.array_equal(again["L_all"], out["L_all"])


def test_nested_deflated_batching_gives_the_same_bits(ctx):
    """The deflated brute force runs its generator and its valuation on two
    streams, batch i + 1's inner paths being generated into the second plane
    buffer while batch i is valued; the inner paths are counter-based, so the
    liabilities must not depend on the batching: one outer path per batch
    (nine batches, both buffers reused four times) against one batch."""
    tab = synth.gm_monthly_survival()
    pol = mixed_portfolio(60, seed=23)
    spec = dict(n_outer=9, n_nodes=7, node_step_m=12, n_inner=200, seed=29)
    one = nested(ctx, pol, tab, rsv.RSV_FORM_F32_DEFLATED, batch_outer=9, **spec)
    many = nested(ctx, pol, tab, rsv.RSV_FORM_F32_DEFLATED, batch_outer=1, **spec)
    default = nested(ctx, pol, tab, rsv.RSV_FORM_F32_DEFLATED, **spec)
    assert np.array_equal(one["L_all"], many["L_all"])
    assert np.array_equal(one["L_all"], default["L_all"])
    assert np.array_equal(one["L_q995"], many["L_q995"])


@pytest.mark.parametrize("form", [rsv.RSV_FORM_F32_COMP, rsv.RSV_FORM_F32_DEFLATED])
def test_outer_paths_split_across_calls(ctx, form):
    """Outer paths keyed by their global index: two calls on outer paths 0-2
    and 3-5 (outer_first = 3) give the rows of one call on all six, bit for
    bit, so ranks can split the outer paths with no exchange."""
    tab = synth.gm_monthly_survival()
    pol = mixed_portfolio(30, seed=31)
    spec = dict(n_nodes=5, node_step_m=12, n_inner=96, seed=37)
    whole = nested(ctx, pol, tab, form, n_outer=6, **spec)
    lo = nested(ctx, pol, tab, form, n_outer=3, **spec)
    hi = nested(ctx, pol, tab, form, n_outer=3, outer_first=3, **spec)
    for key in ("L_all", "L_mean", "L_q995", "r_node", "D0"):
        assert np.array_equal(np.concatenate([lo[key], hi[key]]), whole[key]), key
    with pytest.raises(rsv.RsvError):
        nested(ctx, pol, tab, form, n_outer=3, outer_first=(1 << 24) - 2, **spec)


def test_node_statistics_fifth_largest(ctx):
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_single_life(50, seed=4)
    out = nested(ctx, pol, tab, rsv.RSV_FORM_F32_COMP, n_outer=2, n_nodes=3, node_step_m=12, n_inner=1000, seed=3)
    srt = np.sort(out["L_all"], axis=2)
    assert np.array_equal(out["L_q995"], srt[:, :, -5])          # 5th largest of 1000
    assert np.allclose(out["L_mean"], out["L_all"].mean(axis=2), rtol=1e-13, atol=0)


def test_inner_mean_matches_curve_mode(ctx):
    """The inner Monte Carlo mean estimates the recurrence on the Vasicek forward
    curve (RSV_NESTED_CURVE) to within 4 standard errors at every node."""
    tab = synth.gm_monthly_survival()
    pol = mixed_portfolio(30, seed=5)
    spec = dict(n_outer=2, n_nodes=4, node_step_m=36, seed=9)
    mc = nested(ctx, pol, tab, rsv.RSV_FORM_F32_COMP, n_inner=1000, **spec)
    cv = nested(ctx, pol, tab, rsv.RSV_FORM_F32_COMP, n_inner=1000, mode=rsv.RSV_NESTED_CURVE, **spec)
    se = mc["L_all"].std(axis=2) / math.sqrt(1000)
    z = np.abs(mc["L_mean"] - cv["L_mean"]) / se
    print("z-scores MC mean vs curve:", np.round(z, 2).tolist())
    assert np.all(z < 4.0)
    assert np.array_equal(cv["L_mean"], cv["L_q995"])
    assert np.allclose(mc["r_node"], cv["r_node"], rtol=0, atol=0)


@pytest.mark.parametrize("form", [rsv.RSV_FORM_F32_COMP, rsv.RSV_FORM_F32_DEFLATED])
def test_config3_full_size_sampled(ctx, form):
    """2,000 single-life annuities (ages 60-90) x 100 outer paths x 40 annual
    nodes x 1,000 inner paths, compensated FP32 and deflated: sampled (o, n, i)
    against the oracle, statistics against the returned liabilities."""
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_single_life(2000, seed=0)
    NO, NN, NI = 100, 40, 1000
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    L_all = torch.empty((NO, NN, NI), dtype=torch.float64, device="cuda")
    mean = torch.empty((NO, NN), dtype=torch.float64, device="cuda")
    q = torch.empty((NO, NN), dtype=torch.float64, device="cuda")
    rsv.rsv_compute_nested(ctx, form, n_outer=NO, n_nodes=NN, node_step_m=12, n_inner=NI, seed=0,
                           on_device=True, L_mean=mean, L_q995=q, L_all=L_all)
    rsv.rsv_synchronize(ctx)
    L = L_all.cpu().numpy()
    rng = np.random.default_rng(1)
    worst = 0.0
    for o, n in [(0, 0), (37, 5), (99, 39), (12, 20), (64, 33)]:
        idx = np.sort(rng.choice(NI, 3, replace=False))
        ref, _, _ = oracle.nested_node(pol, tab, 0, o, n, idx, node_step=12)
        worst = max(worst, float(np.max(np.abs(L[o, n, idx] - ref) / np.abs(ref))))
    print(f"config-3 sampled, form {rsv.FORM_NAMES[form]}: max rel err {worst:.3e}")
    assert worst <= 1e-6
    srt = np.sort(L, axis=2)
    assert np.array_equal(q.cpu().numpy(), srt[:, :, -5])
    assert np.allclose(mean.cpu().numpy(), L.mean(axis=2), rtol=1e-13, atol=0)


def test_nested_argument_errors(ctx):
    tab = synth.gm_monthly_survival()
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, synth.portfolio_single_life(3))
    m = np.zeros((1, 1))
    for bad in [dict(n_outer=0), dict(n_inner=0), dict(node_step_m=0), dict(a=0.0), dict(sigma=-1.0),
                dict(mode=7)]:
        spec = dict(n_outer=1, n_nodes=1, node_step_m=12, n_inner=8)
        spec.update(bad)
        with pytest.raises(rsv.RsvError) as e:
            rsv.rsv_compute_nested(ctx, rsv.RSV_FORM_F32_COMP, **spec, L_mean=m, L_q995=m)
        assert e.value.status == rsv.RSV_E_ARG
    with pytest.raises(rsv.RsvError) as e:
        rsv.rsv_compute_nested(ctx, rsv.RSV_FORM_F32_COMP, n_outer=1, n_nodes=1, n_inner=8)
    assert e.value.status == rsv.RSV_E_ARG


def test_surrogate_mode_gain_over_brute_force(ctx):
    """What the trained network gains over the method without it.  The surrogate
    mode values each (policy, node) expectation with one network query -- or, in
    buckets flagged by its held-out error, one recurrence on the forward curve --
    instead of 1,000 inner paths.  Its node liabilities must match the exact
    inner expectation (RSV_NESTED_CURVE) where the network serves them to the
    tolerance it was calibrated to, and the run must be far faster than the
    brute-force inner loop, whose own Monte Carlo error at 1,000 paths is
    several 1e-3."""
    import time
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_single_life(2000, seed=0)
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_portfolio(ctx, pol)
    rsv.rsv_mlp_init(ctx, 1)
    rep = rsv.rsv_surrogate_train(ctx, n_train=3_000_000, n_val=400_000, epochs=10, batch=8192, lr=2e-3, seed=1,
                                  max_node_m=480)
    NO, NN = 8, 40
    spec = dict(n_outer=NO, n_nodes=NN, node_step_m=12, seed=4, n_inner=1000)
    res, secs = {}, {}
    for mode in (rsv.RSV_NESTED_MC, rsv.RSV_NESTED_SURROGATE, rsv.RSV_NESTED_CURVE):
        L = np.zeros((NO, NN))
        q = np.zeros((NO, NN))
        nfb = np.zeros(1, np.int64)
        rsv.rsv_compute_nested(ctx, rsv.RSV_FORM_F32_COMP, mode=mode, L_mean=L, L_q995=q, n_fallback=nfb, **spec)
        t0 = time.perf_counter()
        rsv.rsv_compute_nested(ctx, rsv.RSV_FORM_F32_COMP, mode=mode, L_mean=L, L_q995=q, n_fallback=nfb, **spec)
        secs[mode] = time.perf_counter() - t0
        res[mode] = (L.copy(), int(nfb[0]))
    exact = res[rsv.RSV_NESTED_CURVE][0]
    live = exact > 0
    sur_err = np.max(np.abs(res[rsv.RSV_NESTED_SURROGATE][0] - exact)[live] / exact[live])
    mc_err = np.max(np.abs(res[rsv.RSV_NESTED_MC][0] - exact)[live] / exact[live])
    speed = secs[rsv.RSV_NESTED_MC] / secs[rsv.RSV_NESTED_SURROGATE]
    print(f"surrogate mode: max rel err vs exact {sur_err:.2e} (fallback queries "
          f"{res[rsv.RSV_NESTED_SURROGATE][1]}), brute force {mc_err:.2e}; speed-up over brute force {speed:.1f}x; "
          f"held-out median {rep['val_median_rel']:.2e}, fallback share {rep['frac_fallback']:.2f}")
    # every query the network serves was in a bucket whose held-out error stayed
    # under 0.3 x 1e-3; the node liability is a positive combination of such
    # values and of exact ones, so it stays within the 1e-3 target
    assert sur_err <= 1e-3
    # the recurrence fallback (compacted per segment) ran for the flagged buckets
    assert res[rsv.RSV_NESTED_SURROGATE][1] > 0
    assert speed > 10


def test_nested_two_life_products_against_oracle(ctx):
    """The nested valuation of the two-life products (joint and last-survivor
    annuities, joint term assurances and endowments, second-death term
    assurances and endowments): every (o, n, i) of a small run against the
    oracle's full-state node liabilities."""
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_two_life(48, seed=14, age_lo_y=50, age_hi_y=80, products=tuple(range(4, 10)))
    ls = np.where(pol["product"] >= 8)[0]
    pol["state0"][ls[:4]] = 1     # valued with only the first life alive
    pol["state0"][ls[4:8]] = 2    # only the second
    spec = dict(n_outer=2, n_nodes=4, node_step_m=24, n_inner=40, seed=15)
    out = nested(ctx, pol, tab, rsv.RSV_FORM_F32_COMP, **spec)
    worst = 0.0
    for o in range(2):
        for n in range(4):
            L, _, _ = oracle.nested_node(pol, tab, 15, o, n, np.arange(40), node_step=24)
            worst = max(worst, float(np.max(np.abs(out["L_all"][o, n] - L) / np.abs(L))))
    print(f"nested two-life products: max rel err {worst:.3e}")
    assert worst <= 1e-6


def test_generator_math_against_libm():
    """The inner-path generator's own FP64 logarithm, sine, cosine (table-driven)
    and exponential series against NumPy's libm: random draws plus both ends of
    (0, 1), the table boundaries and the switch to log1p(u - 1) near u = 1."""
    rng = np.random.default_rng(11)
    w = np.concatenate([rng.integers(0, 2**32, 200_000, dtype=np.uint64),
                        np.arange(2**32 - 4096, 2**32), np.arange(0xFF000000 - 2048, 0xFF000000 + 2048),
                        np.arange(0, 4096), np.arange(2**22 - 8, 2**22 + 8), (np.arange(1024) << 22),
                        (np.arange(1024) << 22) + 0x3FFFFF]).astype(np.uint32)
    x = np.concatenate([rng.uniform(-0.0625, 0.0625, len(w) - 4000), rng.uniform(-3.0, 3.0, 4000)])
    out = rsv.rsv_selftest_generator_math(w, x)
    u = (w.astype(np.float64) + 0.5) / 2.0**32
    ln_ref = np.log(u)
    rel_ln = np.abs(out[:, 0] - ln_ref) / np.abs(ln_ref)
    ang = 2.0 * np.pi * u   # rounded angle: the reference itself is off by up to ~4 pi 2^-53
    err_sin = np.abs(out[:, 1] - np.sin(ang))
    err_cos = np.abs(out[:, 2] - np.cos(ang))
    rel_exp = np.abs(out[:, 3] - np.exp(x)) / np.exp(x)
    print(f"generator math: ln {rel_ln.max():.2e} rel, sin {err_sin.max():.2e}, cos {err_cos.max():.2e} abs, "
          f"exp {rel_exp.max():.2e} rel")
    assert rel_ln.max() <= 1e-15
    assert max(err_sin.max(), err_cos.max()) <= 2e-15
    assert rel_exp.max() <= 1e-15
    assert np.allclose(out[:, 1] ** 2 + out[:, 2] ** 2, 1.0, rtol=0, atol=1e-15)
    assert rsv.load_library().rsv_selftest_generator_math(0, None, None, None, 5, None) == rsv.RSV_E_ARG
    assert rsv.rsv_selftest_generator_math(np.zeros(0, np.uint32), np.zeros(0)).shape == (0, 4)
