"""GPU parity of the m-life contracts (Section 4.3) against the oracle's
full tensor-product models.

The oracle builds W^m by the Kronecker induction over the full state space
(2^m states for annuities, 3^m for assurances) and runs the plain recurrence;
the kernel carries 2^m reduced states and applies one-life passes.  Same
bounds as the other parity tests: 1e-12 (FP64), 1e-6 (compensated FP32),
2e-4 (plain FP32)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1401_1757_gb300 import rsv

pytestmark = pytest.mark.gpu

TOL = {rsv.RSV_FORM_F64: 1e-12, rsv.RSV_FORM_F32_COMP: 1e-6, rsv.RSV_FORM_F32: 2e-4}


@pytest.fixture
def ctx():
    assert torch.cuda.is_available()
    h = rsv.rsv_create(0, torch.cuda.current_stream())
    yield h
    rsv.rsv_destroy(h)


def mlife_portfolio(n, seed):
    """m = 1..4 lives aged 55-85 on three tables; annuities (k of m alive, whole
    life or 10-30 y) and k-th death assurances (5-30 y); some lives already dead."""
    rng = np.random.default_rng(seed)
    pol = {"m": rng.integers(1, 5, n), "kind": rng.integers(0, 2, n), "k": np.zeros(n, int),
           "term_m": np.zeros(n, int), "age_m": np.zeros((n, 4), int), "table": np.zeros((n, 4), int),
           "dead0": np.zeros(n, int), "amount": rng.lognormal(np.log(1e3), 0.5, n)}
    for i in range(n):
        m = pol["m"][i]
        pol["k"][i] = rng.integers(1, m + 1)
        pol["age_m"][i, :m] = rng.integers(55 * 12, 85 * 12 + 1, m)
        pol["table"][i, :m] = rng.integers(0, 3, m)
        if pol["kind"][i] == rsv.RSV_MLIFE_ASSURANCE:
            pol["term_m"][i] = 12 * rng.integers(5, 31)
            max_dead = pol["k"][i] - 1          # fewer than k dead
        else:
            pol["term_m"][i] = 0 if rng.uniform() < 0.6 else 12 * rng.integers(10, 31)
            max_dead = m - pol["k"][i]          # at least k alive
        if max_dead > 0 and rng.uniform() < 0.4:
            dead = rng.choice(m, rng.integers(1, max_dead + 1), replace=False)
            pol["dead0"][i] = int(sum(1 << int(j) for j in dead))
    return pol


def oracle_reserve(pol, i, tables, v):
    """amount x r_0 in the valuation state, from the full-state oracle model.
    Life j is digit j of the state index, life 1 the most significant."""
    m, k, kind = int(pol["m"][i]), int(pol["k"][i]), int(pol["kind"][i])
    model = 3 if kind == rsv.RSV_MLIFE_ASSURANCE else 2
    n = model ** m
    digits = [[(s // model ** (m - 1 - j)) % model for j in range(m)] for s in range(n)]
    if model == 2:
        c = np.array([1.0 if d.count(0) >= k else 0.0 for d in digits])
    else:   # the k-th death falls in the step: #dead before < k <= #dead before + #died in it
        c = np.array([1.0 if d.count(2) < k <= d.count(2) + d.count(1) else 0.0 for d in digits])
    dead_digit = 1 if model == 2 else 2
    st = sum(dead_digit * model ** (m - 1 - j) for j in range(m) if pol["dead0"][i] >> j & 1)
    S = int(pol["term_m"][i]) if pol["term_m"][i] > 0 else v.shape[1]   # survival is 0 past the tables
    tabs = np.stack([tables[pol["table"][i, j]] for j in range(m)])
    ages = [int(a) for a in pol["age_m"][i, :m]]
    return np.array([pol["amount"][i] * oracle.mlife_chain(m, model, tabs, ages, c, np.zeros(n), S, v[s])[0, st]
                     for s in range(v.shape[0])])


@pytest.mark.parametrize("form", [rsv.RSV_FORM_F64, rsv.RSV_FORM_F32_COMP, rsv.RSV_FORM_F32])
def test_mlife_against_oracle(ctx, form):
    tables = [synth.gm_monthly_survival(), synth.gm_monthly_survival(A=0.0004, B=0.00002),
              synth.gm_monthly_survival(A=0.0007, B=0.00004)]
    pol = mlife_portfolio(48, seed=5)
    n, n_scen = len(pol["m"]), 40
    v = synth.vasicek_paths(n_scen, 1200, seed=5)
    for t, tab in enumerate(tables):
        rsv.rsv_load_decrements(ctx, t, tab)
    rsv.rsv_load_scenarios(ctx, v)
    V0 = np.zeros((n, n_scen))
    tot = np.zeros(n_scen)
    rsv.rsv_compute_mlife(ctx, pol, form, rsv.RSV_OUT_V0 | rsv.RSV_OUT_SCEN_TOTAL, V0d=V0, scen_total=tot)
    ref = np.stack([oracle_reserve(pol, i, tables, v) for i in range(n)])
    err = np.abs(V0 - ref) / np.maximum(np.abs(ref), 1e-9 * pol["amount"][:, None])
    for m in range(1, 5):
        sel = pol["m"] == m
        print(f"m-life form {rsv.FORM_NAMES[form]} m={m}: max rel err {err[sel].max():.3e}")
    assert err.max() <= TOL[form]
    assert np.max(np.abs(tot - ref.sum(axis=0)) / ref.sum(axis=0)) <= TOL[form]


def test_mlife_two_lives_match_the_two_life_products(ctx):
    """m = 2: the joint-life (k = 2) and last-survivor (k = 1) annuities, and the
    first- and second-death assurances, equal the two-life products of the
    scenario-parallel kernels (FP64)."""
    tab = synth.gm_monthly_survival()
    rsv.rsv_load_decrements(ctx, 0, tab)
    v = synth.vasicek_paths(33, 1200, seed=6)
    rsv.rsv_load_scenarios(ctx, v)
    two = synth.portfolio_two_life(24, seed=6, products=(4, 5, 6, 8))
    kind = {4: (0, 2), 5: (0, 1), 6: (1, 1), 8: (1, 2)}
    ml = {"m": np.full(24, 2), "kind": [kind[p][0] for p in two["product"]], "k": [kind[p][1] for p in two["product"]],
          "term_m": two["term_m"], "age_m": np.stack([two["age1_m"], two["age2_m"], 0 * two["age1_m"],
                                                      0 * two["age1_m"]], axis=1),
          "table": np.zeros((24, 4), int), "dead0": np.zeros(24, int), "amount": two["amount"]}
    V0 = np.zeros((24, 33))
    rsv.rsv_compute_mlife(ctx, ml, rsv.RSV_FORM_F64, rsv.RSV_OUT_V0, V0d=V0)
    rsv.rsv_load_portfolio(ctx, two)
    V1 = np.zeros((24, 33))
    rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F64, rsv.RSV_OUT_V0, V0d=V1)
    assert np.max(np.abs(V0 - V1) / np.abs(V1)) <= 1e-12


def test_mlife_errors(ctx):
    tab = synth.gm_monthly_survival()
    rsv.rsv_load_decrements(ctx, 0, tab)
    rsv.rsv_load_scenarios(ctx, synth.vasicek_paths(8, 600, seed=1))
    good = {"m": [3], "kind": [0], "k": [2], "term_m": [0], "age_m": [[900, 910, 920, 0]],
            "table": [[0, 0, 0, 0]], "dead0": [0], "amount": [1.0]}
    V0 = np.zeros((1, 8))
    rsv.rsv_compute_mlife(ctx, good, rsv.RSV_FORM_F64, rsv.RSV_OUT_V0, V0d=V0)
    for key, val, status in [("m", 5, rsv.RSV_E_ARG), ("k", 4, rsv.RSV_E_ARG), ("dead0", 3, rsv.RSV_E_ARG),
                             ("table", [[0, 5, 0, 0]], rsv.RSV_E_ARG), ("amount", np.inf, rsv.RSV_E_ASSUMPTION),
                             ("age_m", [[100, 110, 920, 0]], rsv.RSV_E_ASSUMPTION)]:
        bad = dict(good)
        bad[key] = [val] if not isinstance(val, list) else val
        with pytest.raises(rsv.RsvError) as e:
            rsv.rsv_compute_mlife(ctx, bad, rsv.RSV_FORM_F64, rsv.RSV_OUT_V0, V0d=V0)
        assert e.value.status == status, key
    ass = dict(good, kind=[1], term_m=[0])           # an assurance needs a term
    with pytest.raises(rsv.RsvError) as e:
        rsv.rsv_compute_mlife(ctx, ass, rsv.RSV_FORM_F64, rsv.RSV_OUT_V0, V0d=V0)
    assert e.value.status == rsv.RSV_E_ARG


def test_mlife_empty_and_single_life(ctx):
    """No policies: the totals are zero.  m = 1 annuity and assurance against
    the single-life products of the scenario-parallel kernels."""
    tab = synth.gm_monthly_survival()
    rsv.rsv_load_decrements(ctx, 0, tab)
    v = synth.vasicek_paths(40, 1200, seed=8)
    rsv.rsv_load_scenarios(ctx, v)
    tot = np.full(40, 7.0)
    empty = {k: [] for k in ("m", "kind", "k", "term_m", "dead0", "amount")}
    empty.update(age_m=np.zeros((0, 4), int), table=np.zeros((0, 4), int))
    rsv.rsv_compute_mlife(ctx, empty, rsv.RSV_FORM_F64, rsv.RSV_OUT_SCEN_TOTAL, scen_total=tot)
    assert np.all(tot == 0.0)
    pol = synth.portfolio_mix(40, seed=8)
    sl = np.isin(pol["product"], (0, 2))
    pol = synth.take(pol, np.where(sl)[0])
    n = len(pol["product"])
    ml = {"m": np.ones(n, int), "kind": (pol["product"] == 2).astype(int), "k": np.ones(n, int),
          "term_m": pol["term_m"], "age_m": np.stack([pol["age1_m"]] + [0 * pol["age1_m"]] * 3, axis=1),
          "table": np.zeros((n, 4), int), "dead0": np.zeros(n, int), "amount": pol["amount"]}
    V0 = np.zeros((n, 40))
    rsv.rsv_compute_mlife(ctx, ml, rsv.RSV_FORM_F64, rsv.RSV_OUT_V0, V0d=V0)
    rsv.rsv_load_portfolio(ctx, pol)
    V1 = np.zeros((n, 40))
    rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F64, rsv.RSV_OUT_V0, V0d=V1)
    assert np.max(np.abs(V0 - V1) / np.abs(V1)) <= 1e-12
