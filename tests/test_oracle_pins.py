"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each check is a closed form, a
brute-force enumeration over death times (which never forms a transition
matrix), one of the scalar recurrences the paper prints, or a structural
invariant.  The summation definition and the backward recurrence are two
separate code paths inside the oracle; their agreement (Section 3.6.2 proves
it exact) is checked too, but only beside the independent pins.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth

SL, JL, TERM, ENDOW = 0, 1, 2, 3
V_FLAT = 1.04 ** (-1.0 / 12.0)     # 4% p.a. effective, monthly steps


def rel(a, b, scale=None):
    a, b = np.asarray(a, float), np.asarray(b, float)
    s = np.maximum(np.abs(b), 1e-300) if scale is None else scale
    return np.max(np.abs(a - b) / s)


# ---------------------------------------------------------------- W and c ----

@pytest.mark.parametrize("product", [SL, JL, TERM, ENDOW])
def test_transition_rows_sum_to_one_and_upper_triangular(product):
    rng = np.random.default_rng(1)
    for _ in range(50):
        px, py = rng.uniform(0, 1, 2)
        W = oracle.transition(product, px, py)
        assert np.allclose(W.sum(axis=1), 1.0, rtol=0, atol=1e-15)
        assert np.all(np.tril(W, -1) == 0.0)          # "0 = alive" labelling (Section 2.4.2)
        assert np.all(W >= 0)


def test_two_life_matrix_entries():
    # Section 4.2: the 4-state binary-labelled matrix, entry by entry.
    px, py = 0.9, 0.7
    qx, qy = 0.1, 0.3
    W = oracle.transition(JL, px, py)
    want = np.array([[px * py, px * qy, qx * py, qx * qy],
                     [0, px, 0, qx],
                     [0, 0, py, qy],
                     [0, 0, 0, 1]])
    assert np.allclose(W, want, rtol=0, atol=1e-16)
    # last-survivor identity printed in Section 4.2.1
    assert math.isclose(1 - qx * qy, W[0, 0] + W[0, 1] + W[0, 2], rel_tol=1e-15)


def test_cashflow_vectors():
    assert np.array_equal(oracle.cashflow(SL, 2.0), [2.0, 0.0])
    assert np.array_equal(oracle.cashflow(JL, 2.0, 0.5), [2.0, 2.0, 1.0, 0.0])
    assert np.array_equal(oracle.cashflow(TERM, 3.0), [0.0, 3.0, 0.0])
    assert np.array_equal(oracle.cashflow(ENDOW, 3.0), [0.0, 3.0, 0.0])


# ------------------------------------------------------------ closed forms ----

def annuity_arrears(g, n):
    return g * (1 - g ** n) / (1 - g)


@pytest.mark.parametrize("mu", [0.01, 0.05, 0.3])
@pytest.mark.parametrize("n", [1, 12, 240, 719])
def test_closed_forms_single_life(mu, n):
    """Flat rate, constant force: level annuity, term assurance, endowment assurance."""
    p = math.exp(-mu / 12)
    tab = synth.constant_force_table(mu, 1440)
    v = np.full(n, V_FLAT)
    g = V_FLAT * p
    A = 123.25
    r = oracle.chain(SL, 0, A, tab, v, term=n)
    for t in (0, n // 2, n - 1, n):
        assert rel(r[t, 0], A * annuity_arrears(g, n - t)) < 1e-13 if t < n else r[t, 0] == 0
    assert np.all(r[:, 1] == 0)                              # dead state: zero reserve state
    term = oracle.chain(TERM, 0, A, tab, v, term=n)
    assert rel(term[0, 0], A * V_FLAT * (1 - p) * (1 - g ** n) / (1 - g)) < 1e-13
    endow = oracle.chain(ENDOW, 0, A, tab, v, term=n)
    assert rel(endow[0, 0], A * (V_FLAT * (1 - p) * (1 - g ** n) / (1 - g) + g ** n)) < 1e-13
    assert np.all(term[:, 1:] == 0) and np.all(endow[:, 1:] == 0)


def test_closed_form_whole_life_to_limiting_age():
    # whole life: a table of L entries means p_k = 0 from L on, so S = L - age
    mu, L, age = 0.02, 1440, 1000
    tab = synth.constant_force_table(mu, L)
    r = oracle.chain(SL, age, 1.0, tab, np.full(L, V_FLAT))
    assert r.shape[0] == L - age + 1
    g = V_FLAT * math.exp(-mu / 12)
    assert rel(r[0, 0], annuity_arrears(g, L - age)) < 1e-13


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.8, 1.0])
def test_closed_forms_two_life(rho):
    """JL reversionary: state 00 = a_x + rho (a_y - a_xy) (Section 2.3.2: a_{x|y} = a_y - a_xy);
    rho = 1 is the last-survivor annuity a_x + a_y - a_xy (Section 4.2.1); state 01 = a_x,
    state 10 = rho a_y; state 11 is a zero reserve state."""
    mux, muy, n = 0.04, 0.07, 300
    px, py = math.exp(-mux / 12), math.exp(-muy / 12)
    tx, ty = synth.constant_force_table(mux), synth.constant_force_table(muy)
    A = 10.0
    r = oracle.chain(JL, 100, A, tx, np.full(n, V_FLAT), age2=200, term=n, rho=rho, table_y=ty)
    ax = annuity_arrears(V_FLAT * px, n)
    ay = annuity_arrears(V_FLAT * py, n)
    axy = annuity_arrears(V_FLAT * px * py, n)
    assert rel(r[0, 0], A * (ax + rho * (ay - axy))) < 1e-13
    assert rel(r[0, 1], A * ax) < 1e-13
    if rho > 0:
        assert rel(r[0, 2], rho * A * ay) < 1e-13
    assert np.all(r[:, 3] == 0)


# ------------------------------------------------- paper's printed relations ----

def random_case(rng, n_ages=60, S=40):
    tab = rng.uniform(0.85, 0.999, n_ages)
    v = rng.uniform(0.95, 0.999, S + 5)
    return tab, v


def test_printed_annuity_due_recurrence():
    """f = 0: annuity-due a''_x = 1 + v p_x a''_{x+1} (Section 2.3.1, 4.1.1)."""
    rng = np.random.default_rng(2)
    tab, v = random_case(rng)
    ones = np.ones_like(tab)
    r = oracle.chain(SL, 10, 1.0, tab, v, table_fx=ones, vf=np.ones_like(v), term=30)
    for t in range(30):
        assert math.isclose(r[t, 0], 1 + v[t] * tab[10 + t] * r[t + 1, 0], rel_tol=1e-14)


def test_printed_general_f_annuity_recurrence():
    """a'_x = fp_x v^f + p_x v a'_{x+1} for f in (0, 1) (Eq. slAnnRecRel)."""
    rng = np.random.default_rng(3)
    tab, v = random_case(rng)
    f = 0.37
    tf = tab ** f
    vf = v ** f
    r = oracle.chain(SL, 5, 1.0, tab, v, table_fx=tf, vf=vf, term=35)
    for t in range(35):
        want = tf[5 + t] * vf[t] + tab[5 + t] * v[t] * r[t + 1, 0]
        assert math.isclose(r[t, 0], want, rel_tol=1e-14)


def test_printed_assurance_and_endowment_recurrences():
    """A_x = v q_x + v p_x A_{x+1} (Section 4.1.3); pure endowment A = v p A' with
    boundary 1 (Section 4.1.2) = endowment assurance minus term assurance."""
    rng = np.random.default_rng(4)
    tab, v = random_case(rng)
    a0, n = 7, 30
    term = oracle.chain(TERM, a0, 1.0, tab, v, term=n)
    endow = oracle.chain(ENDOW, a0, 1.0, tab, v, term=n)
    pure = endow[:, 0] - term[:, 0]
    assert pure[n] == 1.0 and term[n, 0] == 0.0
    for t in range(n):
        p = tab[a0 + t]
        assert math.isclose(term[t, 0], v[t] * (1 - p) + v[t] * p * term[t + 1, 0], rel_tol=1e-14)
        assert math.isclose(pure[t], v[t] * p * pure[t + 1], rel_tol=1e-12)


def test_printed_reversionary_recurrence():
    """a_{x|y} = q_x p_y v + q_x p_y v a_{y+1} + p_x p_y v a_{x+1|y+1} at f = 1 (Eq. revAnnRecRel)."""
    rng = np.random.default_rng(5)
    tx = rng.uniform(0.85, 0.999, 80)
    ty = rng.uniform(0.85, 0.999, 80)
    v = rng.uniform(0.95, 0.999, 60)
    kw = dict(age2=20, term=40, table_y=ty)
    r1 = oracle.chain(JL, 10, 1.0, tx, v, rho=1.0, **kw)
    r0 = oracle.chain(JL, 10, 1.0, tx, v, rho=0.0, **kw)
    a_rev = r1[:, 0] - r0[:, 0]      # a_{x|y}: the rho-part of state 00
    a_y = r1[:, 2]                   # state 10 at rho = 1: annuity on (y)
    for t in range(40):
        px, py = tx[10 + t], ty[20 + t]
        want = (1 - px) * py * v[t] + (1 - px) * py * v[t] * a_y[t + 1] + px * py * v[t] * a_rev[t + 1]
        assert math.isclose(a_rev[t], want, rel_tol=1e-12)


# ------------------------------------------------- brute-force enumeration ----

def enumerate_single(product, tab, age, v, S_term, A, S):
    """Sum over the death step D of the life (or survival past S) of Pr[D] x PV(cash flows)."""
    total = 0.0
    surv = 1.0                       # Pr[alive at start of step d]
    disc = np.concatenate([[1.0], np.cumprod(v[:S])])   # disc[k] = prod_{u<k} v_u
    for d in range(S + 1):
        if d < S:
            p = tab[age + d] if age + d < len(tab) else 0.0
            prob = surv * (1 - p)    # dies during step d
        else:
            prob = surv              # alive at S
        if prob != 0.0:
            if product == SL:        # A at the end of every step survived
                pv = A * sum(disc[u + 1] for u in range(min(d, S)))
            elif product in (TERM, ENDOW):
                pv = A * disc[d + 1] if d < S else 0.0
                if product == ENDOW and d == S and S == S_term:
                    pv += A * disc[S]
            total += prob * pv
        if d < S:
            surv *= tab[age + d] if age + d < len(tab) else 0.0
    return total


def enumerate_jl(tx, ty, ax, ay, v, A, rho, S):
    """Two independent lives: enumerate both death steps."""
    disc = np.concatenate([[1.0], np.cumprod(v[:S])])

    def dist(tab, age):
        out, surv = [], 1.0
        for d in range(S):
            p = tab[age + d] if age + d < len(tab) else 0.0
            out.append(surv * (1 - p))
            surv *= p
        out.append(surv)
        return out

    Px, Py = dist(tx, ax), dist(ty, ay)
    total = 0.0
    for dx, dy in itertools.product(range(S + 1), range(S + 1)):
        prob = Px[dx] * Py[dy]
        if prob == 0.0:
            continue
        pv = 0.0
        for u in range(S):           # payment at the end of step u
            x_alive, y_alive = u < dx, u < dy
            if x_alive:
                pv += A * disc[u + 1]
            elif y_alive:
                pv += rho * A * disc[u + 1]
        total += prob * pv
    return total


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_single_life(seed):
    rng = np.random.default_rng(100 + seed)
    n_ages = 20
    tab = rng.uniform(0.3, 0.999, n_ages)
    v = rng.uniform(0.85, 1.0, n_ages + 4)
    for product in (SL, TERM, ENDOW):
        for age in (0, 5, n_ages - 6, n_ages - 3, n_ages - 1):
            for term in (0, 1, 4, 8) if product == SL else (1, 3, 6, 8):
                A = float(rng.uniform(1, 100))
                r = oracle.chain(product, age, A, tab, v, term=term)
                S = r.shape[0] - 1
                want = enumerate_single(product, tab, age, v, term, A, S)
                s = oracle.chain(product, age, A, tab, v, term=term, method="summation")
                assert abs(r[0, 0] - want) <= 1e-14 * A, (product, age, term)
                assert abs(s[0, 0] - want) <= 1e-14 * A, (product, age, term)


@pytest.mark.parametrize("seed", range(4))
def test_brute_force_two_life(seed):
    rng = np.random.default_rng(200 + seed)
    n_ages = 16
    tx, ty = rng.uniform(0.3, 0.999, n_ages), rng.uniform(0.3, 0.999, n_ages)
    v = rng.uniform(0.85, 1.0, n_ages + 2)
    for ax, ay, term in [(0, 3, 8), (9, 4, 0), (12, 14, 0), (2, 2, 5), (15, 8, 7)]:
        A, rho = float(rng.uniform(1, 50)), float(rng.uniform(0, 1))
        r = oracle.chain(JL, ax, A, tx, v, age2=ay, term=term, rho=rho, table_y=ty)
        S = r.shape[0] - 1
        want = enumerate_jl(tx, ty, ax, ay, v, A, rho, S)
        assert abs(r[0, 0] - want) <= 1e-14 * A
        s = oracle.chain(JL, ax, A, tx, v, age2=ay, term=term, rho=rho, table_y=ty, method="summation")
        assert abs(s[0, 0] - want) <= 1e-14 * A


def test_brute_force_fractional_payment_time():
    """General f: an annuity payment at t+f is made if alive at t+f.  Enumerate death in
    [t, t+f) or [t+f, t+1) with fp and p/fp (Section 2.3.1)."""
    rng = np.random.default_rng(7)
    tab = rng.uniform(0.5, 0.99, 12)
    f = 0.25
    tf = tab ** f                     # any survival over [t, t+f) with tf >= tab works
    v = rng.uniform(0.9, 1.0, 10)
    vf = v ** f
    S = 6
    r = oracle.chain(SL, 2, 1.0, tab, v, table_fx=tf, vf=vf, term=S)
    total, surv = 0.0, 1.0
    disc = np.concatenate([[1.0], np.cumprod(v)])
    for d in range(S + 1):          # d: step in which the life dies (S: survives)
        for half in (0, 1):         # 0: dies before t+f, 1: dies after t+f
            if d == S:
                if half:
                    continue
                prob = surv
            else:
                k = 2 + d
                prob = surv * ((1 - tf[k]) if half == 0 else (tf[k] - tab[k]))
            pv = sum(disc[u] * vf[u] for u in range(min(d, S)))
            if d < S and half == 1:
                pv += disc[d] * vf[d]
            total += prob * pv
        if d < S:
            surv *= tab[2 + d]
    assert math.isclose(r[0, 0], total, rel_tol=1e-14)


# ------------------------------------- summation == recurrence, invariants ----

@pytest.mark.parametrize("scen", ["flat", "vasicek"])
def test_summation_equals_recurrence_config1(scen):
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_single_life(12, seed=3)
    v = synth.flat_scenarios(n_steps=720) if scen == "flat" else synth.vasicek_paths(1, 720, seed=3)
    for p in range(12):
        r = oracle.chain(SL, int(pol["age1_m"][p]), float(pol["amount"][p]), tab, v[0])
        s = oracle.chain(SL, int(pol["age1_m"][p]), float(pol["amount"][p]), tab, v[0], method="summation")
        scale = float(pol["amount"][p])
        assert np.max(np.abs(r - s)) <= 1e-13 * scale * max(1.0, np.max(np.abs(r)) / scale)


def test_summation_equals_recurrence_mix():
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_mix(40, seed=4)
    v = synth.vasicek_paths(1, 1200, seed=4)[0]
    for p in range(40):
        kw = dict(age2=int(pol["age2_m"][p]), term=int(pol["term_m"][p]), rho=float(pol["reversion"][p]))
        a = (int(pol["product"][p]), int(pol["age1_m"][p]), float(pol["amount"][p]), tab, v)
        r = oracle.chain(*a, **kw)
        s = oracle.chain(*a, **kw, method="summation")
        assert np.max(np.abs(r - s)) <= 1e-12 * max(1.0, np.max(np.abs(r)))


def test_reserve_invariants():
    tab = synth.gm_monthly_survival()
    v = synth.flat_scenarios(n_steps=1440)[0]
    # level SL annuity, flat rate, increasing GM force: reserves non-increasing in t
    r = oracle.chain(SL, 60 * 12, 1.0, tab, v)
    assert np.all(np.diff(r[:, 0]) <= 1e-15)
    assert r[-1, 0] == 0.0 and np.all(r >= 0)
    # linear in the amount
    r2 = oracle.chain(SL, 60 * 12, 3.5, tab, v)
    assert np.allclose(r2, 3.5 * r, rtol=1e-14, atol=0)
    # endowment boundary, assurance zero reserve states
    e = oracle.chain(ENDOW, 40 * 12, 7.0, tab, v, term=120)
    assert e[-1, 0] == 7.0 and np.all(e[:, 1:] == 0.0)
    # ages at or past the limiting age: nothing left to pay
    assert oracle.chain(SL, 1440, 1.0, tab, v).shape[0] == 1
    assert oracle.chain(SL, 1439, 1.0, tab, v).shape[0] == 2


def test_horizon_truncation_drops_later_cash_flows():
    tab = synth.gm_monthly_survival()
    v = synth.vasicek_paths(1, 1200, seed=9)[0]
    full = oracle.chain(SL, 300, 1.0, tab, v)
    h = 600
    trunc = oracle.chain(SL, 300, 1.0, tab, v, horizon=h)
    assert trunc.shape[0] == h + 1 and trunc[h, 0] == 0.0
    # the dropped part is the time-h reserve discounted and survival-weighted to 0
    dropped = full[h, 0] * np.prod(v[:h]) * np.prod(tab[300:300 + h])
    assert math.isclose(full[0, 0] - trunc[0, 0], dropped, rel_tol=1e-11)
    e = oracle.chain(ENDOW, 300, 1.0, tab, v, term=700, horizon=h)
    assert e[h, 0] == 0.0         # maturity beyond the horizon is dropped


def test_batch_matches_chain():
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_mix(30, seed=11)
    pol["state0"][pol["product"] == JL] = np.arange((pol["product"] == JL).sum()) % 3
    v = synth.vasicek_paths(3, 1200, seed=11)
    V0, tot = oracle.reserves_batch(pol, tab, v, nthreads=2)
    for p in range(30):
        for s in range(3):
            r = oracle.chain(int(pol["product"][p]), int(pol["age1_m"][p]), float(pol["amount"][p]),
                             tab, v[s], age2=int(pol["age2_m"][p]), term=int(pol["term_m"][p]),
                             rho=float(pol["reversion"][p]))
            assert V0[p, s] == r[0, int(pol["state0"][p])]
    assert np.allclose(tot, V0.sum(axis=0), rtol=1e-15)


# ------------------------------------------------------- input generators ----

def test_gm_table_matches_quadrature():
    from scipy.integrate import quad
    tab = synth.gm_monthly_survival()
    assert len(tab) == 1440
    for k in (0, 240, 720, 1200, 1439):
        I, _ = quad(lambda x: 0.0005 + 0.00003 * 1.1 ** x, k / 12, (k + 1) / 12, epsabs=1e-16, epsrel=1e-13)
        assert math.isclose(tab[k], math.exp(-I), rel_tol=1e-13)


def test_vasicek_moments_and_zero_coupon_price():
    n, T = 40_000, 120
    v, r = synth.vasicek_paths(n, T, seed=5, return_rates=True)
    a, b, sig, r0 = 0.1, 0.04, 0.01, 0.03
    t = T / 12
    mean = b + (r0 - b) * math.exp(-a * t)
    var = sig * sig * (1 - math.exp(-2 * a * t)) / (2 * a)
    se_mean = math.sqrt(var / n)
    assert abs(r[:, T].mean() - mean) < 4 * se_mean
    assert abs(r[:, T].var() - var) < 4 * var * math.sqrt(2 / n)
    D = np.prod(v, axis=1)
    assert abs(D.mean() - synth.vasicek_zcb(t, r0)) < 4 * D.std() / math.sqrt(n)


def test_batch_summation_method_equals_recurrence():
    """The batch entry point by the summation definition at every step agrees
    with the recurrence (Eq. basicReserveSummation against Eq. generalForm)
    on a four-product mix under Vasicek scenarios."""
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_mix(40, seed=31)
    v = synth.vasicek_paths(3, 1200, seed=31)
    a, ta = oracle.reserves_batch(pol, tab, v)
    b, tb = oracle.reserves_batch(pol, tab, v, method="summation")
    assert np.max(np.abs(a - b) / np.maximum(np.abs(a), 1e-9 * pol["amount"][:, None])) <= 1e-12
    assert np.max(np.abs(ta - tb) / ta) <= 1e-12


# ------------------------------------------------------ two-life products ----
JOINT, LASTS, JTERM, JENDOW = (oracle.JOINT_ANNUITY, oracle.LAST_SURVIVOR, oracle.JOINT_TERM,
                               oracle.JOINT_ENDOWMENT)


def test_two_life_products_models():
    """Joint-life and last-survivor annuities use the 4-state two-life matrix
    (Section 4.2) with c = (A, 0, 0, 0) and (A, A, A, 0); the joint-status
    assurances use the assurance model (Section 4.1.3) with survival px py."""
    px, py = 0.9, 0.7
    for prod in (JOINT, LASTS):
        assert np.array_equal(oracle.transition(prod, px, py), oracle.transition(JL, px, py))
    W = oracle.transition(JTERM, px, py)
    assert np.allclose(W, [[px * py, 1 - px * py, 0], [0, 0, 1], [0, 0, 1]], rtol=0, atol=1e-16)
    assert np.array_equal(oracle.cashflow(JOINT, 2.0), [2.0, 0, 0, 0])
    assert np.array_equal(oracle.cashflow(LASTS, 2.0), [2.0, 2.0, 2.0, 0])
    assert np.array_equal(oracle.cashflow(JENDOW, 3.0), [0, 3.0, 0])
    for prod in (JOINT, LASTS, JTERM, JENDOW):
        W = oracle.transition(prod, px, py)
        assert np.allclose(W.sum(axis=1), 1.0, rtol=0, atol=1e-15) and np.all(np.tril(W, -1) == 0.0)


@pytest.mark.parametrize("n", [1, 60, 300])
def test_closed_forms_two_life_products(n):
    """Flat rate, constant forces mux, muy, g = v px py: joint-life annuity
    a_xy = g (1 - g^n) / (1 - g); last survivor a_x + a_y - a_xy; joint term
    assurance v (1 - px py)(1 - g^n) / (1 - g); joint endowment adds g^n."""
    mux, muy = 0.04, 0.09
    px, py = math.exp(-mux / 12), math.exp(-muy / 12)
    tx, ty = synth.constant_force_table(mux), synth.constant_force_table(muy)
    v = np.full(n, V_FLAT)
    A = 7.5
    g = V_FLAT * px * py
    axy = annuity_arrears(g, n)
    ax, ay = annuity_arrears(V_FLAT * px, n), annuity_arrears(V_FLAT * py, n)
    kw = dict(age2=200, term=n, table_y=ty)
    assert rel(oracle.chain(JOINT, 100, A, tx, v, **kw)[0, 0], A * axy) < 1e-13
    assert rel(oracle.chain(LASTS, 100, A, tx, v, **kw)[0, 0], A * (ax + ay - axy)) < 1e-13
    jt = V_FLAT * (1 - px * py) * (1 - g ** n) / (1 - g)
    assert rel(oracle.chain(JTERM, 100, A, tx, v, **kw)[0, 0], A * jt) < 1e-13
    assert rel(oracle.chain(JENDOW, 100, A, tx, v, **kw)[0, 0], A * (jt + g ** n)) < 1e-13


def enumerate_two_life(product, tx, ty, ax, ay, v, A, S, term):
    """Two independent lives, enumerating both death steps (dx, dy in 0..S, S
    meaning alive at the end): PV of the product's cash flows."""
    disc = np.concatenate([[1.0], np.cumprod(v[:S])])

    def dist(tab, age):
        out, surv = [], 1.0
        for d in range(S):
            p = tab[age + d] if age + d < len(tab) else 0.0
            out.append(surv * (1 - p))
            surv *= p
        out.append(surv)
        return out

    Px, Py = dist(tx, ax), dist(ty, ay)
    total = 0.0
    for dx, dy in itertools.product(range(S + 1), range(S + 1)):
        prob = Px[dx] * Py[dy]
        if prob == 0.0:
            continue
        pv = 0.0
        first = min(dx, dy)
        if product == JOINT:
            pv = A * sum(disc[u + 1] for u in range(min(first, S)))
        elif product == LASTS:
            pv = A * sum(disc[u + 1] for u in range(min(max(dx, dy), S)))
        else:
            if first < S:
                pv = A * disc[first + 1]          # end of the step of the first death
            elif product == JENDOW and S == term:
                pv = A * disc[S]                  # both alive at maturity
        total += prob * pv
    return total


@pytest.mark.parametrize("seed", range(3))
def test_brute_force_two_life_products(seed):
    rng = np.random.default_rng(300 + seed)
    n_ages = 14
    tx, ty = rng.uniform(0.3, 0.999, n_ages), rng.uniform(0.3, 0.999, n_ages)
    v = rng.uniform(0.85, 1.0, n_ages + 2)
    for prod in (JOINT, LASTS, JTERM, JENDOW):
        for ax, ay, term in [(0, 3, 8), (9, 4, 0), (2, 2, 5), (11, 6, 3)]:
            if prod in (JTERM, JENDOW) and term == 0:
                term = 6
            A = float(rng.uniform(1, 50))
            r = oracle.chain(prod, ax, A, tx, v, age2=ay, term=term, table_y=ty)
            S = r.shape[0] - 1
            want = enumerate_two_life(prod, tx, ty, ax, ay, v, A, S, term)
            assert abs(r[0, 0] - want) <= 1e-14 * A, (prod, ax, ay, term)
            s = oracle.chain(prod, ax, A, tx, v, age2=ay, term=term, table_y=ty, method="summation")
            assert abs(s[0, 0] - want) <= 1e-14 * A, (prod, ax, ay, term)
