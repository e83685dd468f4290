"""Pins of the oracle's varying cash-flow sequences c_t (Section 4.1.1: level,
increasing, escalating and limited-term annuities differ only in c_t;
Section 4.6: the sequence carries escalation and timing, e.g. one non-zero step
in twelve for annual payments on monthly steps).

Each check is a closed form (geometric and arithmetic-geometric series under a
flat rate and constant survival), a brute-force enumeration over death steps
with the cash flows weighted step by step (no transition matrix), or the
agreement of the oracle's two separate code paths (recurrence and summation).
"""
import itertools

import numpy as np
import pytest

import oracle

SL, JL, TERM, ENDOW = 0, 1, 2, 3
JOINT, LASTS, JTERM, JENDOW = 4, 5, 6, 7


def flat(p, n):
    return np.full(n, p)


# --------------------------------------------------------- closed forms ----

@pytest.mark.parametrize("esc", [0.0, 0.03, 0.0425, 0.05])
def test_escalating_annuity_geometric_series(esc):
    """Annual steps (steps_per_year = 1), escalation at every step from the
    second: PV = sum_{t<S} (v p)^(t+1) g^t = x (1 - (x g)^S) / (1 - x g), x = v p."""
    p, v, S = 0.97, 1.0 / 1.04, 30
    tab = flat(p, 200)
    cf = oracle.schedule(S, steps_per_year=1, escalation=esc)
    r = oracle.chain(SL, 10, 1.0, tab, np.full(S, v), term=S, cf=cf)
    x, g = v * p, 1.0 + esc
    want = x * (1 - (x * g) ** S) / (1 - x * g)
    assert abs(r[0, 0] - want) <= 1e-13 * want


@pytest.mark.parametrize("inc", [0.0, 0.1, 0.5])
def test_increasing_annuity_arithmetic_geometric_series(inc):
    """PV = sum_{t<S} x^(t+1) (1 + inc t), with sum_{t<S} t x^t =
    x (1 - S x^(S-1) + (S-1) x^S) / (1 - x)^2."""
    p, v, S = 0.98, 1.0 / 1.05, 40
    cf = oracle.schedule(S, steps_per_year=1, increase=inc)
    r = oracle.chain(SL, 0, 2.5, flat(p, 100), np.full(S, v), term=S, cf=cf)
    x = v * p
    lvl = x * (1 - x ** S) / (1 - x)
    tx = x * (1 - S * x ** (S - 1) + (S - 1) * x ** S) / (1 - x) ** 2
    want = 2.5 * (lvl + inc * x * tx)
    assert abs(r[0, 0] - want) <= 1e-13 * want


def test_increasing_annuity_monthly_steps():
    """Monthly payments, the level raised by inc at each anniversary:
    PV = x (1 - x^12) / (1 - x) sum_{k<K} (1 + inc k) y^k, y = x^12."""
    p, v, K, inc = 0.999, 1.05 ** (-1.0 / 12.0), 15, 0.25
    S = 12 * K
    cf = oracle.schedule(S, increase=inc)
    r = oracle.chain(SL, 0, 1.0, flat(p, 400), np.full(S, v), term=S, cf=cf)
    x = v * p
    y = x ** 12
    geo = (1 - y ** K) / (1 - y)
    ari = y * (1 - K * y ** (K - 1) + (K - 1) * y ** K) / (1 - y) ** 2
    want = x * (1 - x ** 12) / (1 - x) * (geo + inc * ari)
    assert abs(r[0, 0] - want) <= 1e-13 * want


@pytest.mark.parametrize("esc", [0.0, 0.05])
def test_annual_payments_on_monthly_steps(esc):
    """Paid at the end of every twelfth month (first = 11), escalating at each
    anniversary: PV = sum_k y^(k+1) g^k, y = (v p)^12, an annual annuity."""
    p, v, years = 0.998, 1.04 ** (-1.0 / 12.0), 20
    S = 12 * years
    cf = oracle.schedule(S, every=12, first=11, escalation=esc)
    assert np.count_nonzero(cf) == years
    r = oracle.chain(SL, 700, 1.0, flat(p, 2000), np.full(S, v), term=S, cf=cf)
    y, g = (v * p) ** 12, 1.0 + esc
    want = sum(y ** (k + 1) * g ** k for k in range(years))
    assert abs(r[0, 0] - want) <= 1e-13 * want


def test_anniversary_phase_moves_the_escalation():
    """since = s: the first rise comes at step 12 - s.  With a flat rate and
    p = 1 the PV is a sum of v^(t+1) g^floor((t + s)/12) over the steps."""
    v, S, g = 0.995, 36, 1.03
    for since in (0, 1, 7, 11):
        cf = oracle.schedule(S, since=since, escalation=g - 1)
        assert np.all(cf[: 12 - since] == 1.0) and cf[12 - since] == pytest.approx(g, rel=1e-15)
        r = oracle.chain(SL, 0, 1.0, flat(1.0, 100), np.full(S, v), term=S, cf=cf)
        want = 0.0
        for k in range(3):
            lo, hi = max(0, 12 * k - since), min(S, 12 * (k + 1) - since)
            want += g ** k * sum(v ** (t + 1) for t in range(lo, hi))
        want += g ** 3 * sum(v ** (t + 1) for t in range(max(0, 36 - since), S))
        assert abs(r[0, 0] - want) <= 1e-13 * want


def test_increasing_term_assurance_closed_form():
    """Death benefit 1 + inc t in year t of death (annual steps):
    PV = sum_t x^t v q (1 + inc t), x = v p."""
    p, v, S, inc = 0.95, 1.0 / 1.03, 25, 0.2
    cf = oracle.schedule(S, steps_per_year=1, increase=inc)
    r = oracle.chain(TERM, 5, 1.0, flat(p, 100), np.full(S, v), term=S, cf=cf)
    x = v * p
    want = sum(x ** t * v * (1 - p) * (1 + inc * t) for t in range(S))
    assert abs(r[0, 0] - want) <= 1e-13 * want


def test_schedule_rejects_bad_parameters():
    for kw in ({"every": 0}, {"first": -1}, {"since": 12}, {"since": -1}, {"escalation": -1.0},
               {"increase": -0.1}, {"steps_per_year": 0}):
        with pytest.raises(ValueError):
            oracle.schedule(10, **kw)


# ------------------------------------------------- brute-force enumeration ----

def death_dist(tab, age, S):
    out, surv = [], 1.0
    for d in range(S):
        p = tab[age + d] if age + d < len(tab) else 0.0
        out.append(surv * (1 - p))
        surv *= p
    out.append(surv)
    return out


def enumerate_cf(product, tx, ty, ax, ay, v, A, rho, S, term, cf):
    """Sum over the death steps (dx, dy; S = alive at the end) of Pr x PV, the
    payment of step u at its end weighted by cf[u]; the maturity sum unweighted."""
    disc = np.concatenate([[1.0], np.cumprod(v[:S])])
    Px = death_dist(tx, ax, S)
    Py = death_dist(ty, ay, S) if ty is not None else [0.0] * S + [1.0]
    total = 0.0
    for dx, dy in itertools.product(range(S + 1), range(S + 1)):
        prob = Px[dx] * Py[dy]
        if prob == 0.0:
            continue
        pv = 0.0
        for u in range(S):
            xa, ya = u < dx, u < dy      # alive at the end of step u
            amt = 0.0
            if product == SL and xa:
                amt = 1.0
            elif product == JL:
                amt = 1.0 if xa else (rho if ya else 0.0)
            elif product == JOINT and xa and ya:
                amt = 1.0
            elif product == LASTS and (xa or ya):
                amt = 1.0
            elif product in (TERM, ENDOW) and dx == u:
                amt = 1.0
            elif product in (JTERM, JENDOW) and min(dx, dy) == u:
                amt = 1.0
            pv += A * cf[u] * amt * disc[u + 1]
        if S == term:
            if product == ENDOW and dx == S:
                pv += A * disc[S]
            if product == JENDOW and dx == S and dy == S:
                pv += A * disc[S]
        total += prob * pv
    return total


@pytest.mark.parametrize("seed", range(3))
def test_brute_force_with_cash_flows(seed):
    rng = np.random.default_rng(700 + seed)
    n_ages = 14
    tx, ty = rng.uniform(0.3, 0.999, n_ages), rng.uniform(0.3, 0.999, n_ages)
    v = rng.uniform(0.85, 1.0, n_ages + 2)
    cf = rng.uniform(0.0, 3.0, len(v))
    cf[rng.uniform(size=len(v)) < 0.3] = 0.0
    for prod in (SL, JL, TERM, ENDOW, JOINT, LASTS, JTERM, JENDOW):
        two = prod in (JL, JOINT, LASTS, JTERM, JENDOW)
        for ax, ay, term in [(0, 3, 8), (9, 4, 0), (2, 2, 5), (11, 6, 3)]:
            if prod in (TERM, ENDOW, JTERM, JENDOW) and term == 0:
                term = 6
            A, rho = float(rng.uniform(1, 50)), float(rng.uniform(0, 1))
            kw = dict(age2=ay, term=term, rho=rho, table_y=ty if two else None, cf=cf)
            r = oracle.chain(prod, ax, A, tx, v, **kw)
            S = r.shape[0] - 1
            want = enumerate_cf(prod, tx, ty if two else None, ax, ay, v, A, rho, S, term, cf)
            assert abs(r[0, 0] - want) <= 1e-13 * A, (prod, ax, ay, term)
            s = oracle.chain(prod, ax, A, tx, v, method="summation", **kw)
            assert abs(s[0, 0] - want) <= 1e-13 * A, (prod, ax, ay, term)


def test_batch_with_cash_flows_matches_chain():
    rng = np.random.default_rng(9)
    n_ages, n_steps, n = 30, 40, 12
    tab = rng.uniform(0.8, 0.999, (2, n_ages))
    v = rng.uniform(0.95, 1.0, (3, n_steps))
    pol = {"product": rng.integers(0, 8, n), "age1_m": rng.integers(0, 20, n),
           "age2_m": rng.integers(0, 20, n), "term_m": rng.integers(1, 12, n),
           "state0": np.zeros(n, int), "table1": rng.integers(0, 2, n), "table2": rng.integers(0, 2, n),
           "amount": rng.uniform(1, 10, n), "reversion": rng.uniform(0, 1, n)}
    cf = rng.uniform(0, 2, (n, n_steps))
    V0, _ = oracle.reserves_batch(pol, tab, v, cf=cf)
    for i in range(n):
        for s in range(3):
            r = oracle.chain(int(pol["product"][i]), int(pol["age1_m"][i]), float(pol["amount"][i]),
                             tab[pol["table1"][i]], v[s], age2=int(pol["age2_m"][i]),
                             term=int(pol["term_m"][i]), rho=float(pol["reversion"][i]),
                             table_y=tab[pol["table2"][i]], cf=cf[i])
            assert V0[i, s] == r[0, 0]
    V1, _ = oracle.reserves_batch(pol, tab, v, cf=cf, method="summation")
    assert np.max(np.abs(V1 - V0)) <= 1e-12 * np.max(np.abs(V0))
