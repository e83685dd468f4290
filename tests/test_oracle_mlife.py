"""Pins of the oracle's two-life assurance model (Section 4.2.3: nine states,
first- and second-death cash flows) and of the m-life tensor-product models
(Section 4.3).

The printed matrices and cash-flow vectors come from a golden fixture typed in
from the paper; the rest are closed forms under constant forces and a flat
rate, brute-force enumerations over the lives' death steps (no transition
matrix), and the counts of non-zero entries the paper states for W^m.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "two_life_transition_matrices.txt")
JL, JTERM, LS_TERM, LS_ENDOW = 1, oracle.JOINT_TERM, oracle.LS_TERM, oracle.LS_ENDOWMENT
V_FLAT = 1.04 ** (-1.0 / 12.0)


def golden():
    """{name: rows of entries} from the fixture."""
    out, cur = {}, None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("["):
            cur = line.strip("[]")
            out[cur] = []
        else:
            out[cur].append(line.split())
    return out


def evaluate(rows, px, py):
    env = {"px": px, "py": py, "qx": 1.0 - px, "qy": 1.0 - py}
    return np.array([[eval(e, {}, env) for e in r] for r in rows], float)


# ------------------------------------------------ printed matrices ----

@pytest.mark.parametrize("px,py", [(0.9, 0.7), (0.999, 0.35), (1.0, 0.0)])
def test_printed_two_life_matrices(px, py):
    g = golden()
    W4, W9 = evaluate(g["W4"], px, py), evaluate(g["W9"], px, py)
    assert np.array_equal(oracle.transition(JL, px, py), W4)
    assert np.array_equal(oracle.transition(LS_TERM, px, py), W9)
    # the Kronecker induction of Section 4.3 gives the same matrices
    assert np.allclose(oracle.mlife_transition(2, 2, [px, py]), W4, rtol=0, atol=1e-16)
    assert np.allclose(oracle.mlife_transition(2, 3, [px, py]), W9, rtol=0, atol=1e-16)
    c2 = np.array(g["c9_second"][0], float)
    assert np.array_equal(oracle.cashflow(LS_TERM, 2.5), 2.5 * c2)
    assert np.array_equal(oracle.cashflow(LS_ENDOW, 1.0), c2)


def test_single_life_factors():
    """m = 1 gives the single-life matrices of Sections 4.1 and 4.1.3."""
    p = 0.83
    assert np.allclose(oracle.mlife_transition(1, 2, [p]), [[p, 1 - p], [0, 1]], rtol=0, atol=1e-16)
    assert np.allclose(oracle.mlife_transition(1, 3, [p]), [[p, 1 - p, 0], [0, 0, 1], [0, 0, 1]], rtol=0, atol=1e-16)
    assert np.array_equal(oracle.mlife_transition(0, 2, []), [[1.0]])


@pytest.mark.parametrize("m", [1, 2, 3, 4])
def test_mlife_nonzero_counts_and_rows(m):
    """Section 4.3: 2^m states with 3^m non-zero entries (two-state model),
    3^m states with 4^m non-zero entries (three-state model); rows sum to 1."""
    p = np.linspace(0.55, 0.95, m)
    W2, W3 = oracle.mlife_transition(m, 2, p), oracle.mlife_transition(m, 3, p)
    assert W2.shape == (2 ** m, 2 ** m) and np.count_nonzero(W2) == 3 ** m
    assert W3.shape == (3 ** m, 3 ** m) and np.count_nonzero(W3) == 4 ** m
    assert np.allclose(W2.sum(axis=1), 1, rtol=0, atol=1e-15)
    assert np.allclose(W3.sum(axis=1), 1, rtol=0, atol=1e-15)
    assert np.all(np.tril(W2, -1) == 0)


def test_full_state_of_the_reduced_valuation_states():
    assert [oracle.full_state(LS_TERM, s) for s in (0, 1, 2)] == [0, 2, 6]
    assert [oracle.full_state(JL, s) for s in (0, 1, 2)] == [0, 1, 2]
    assert oracle.full_state(LS_TERM, 3) == -1


# ------------------------------------------------------- closed forms ----

def assurance(g, vq, n):
    """sum_{t<n} g^t vq: a term assurance with per-step death term vq, survival factor g."""
    return vq * (1 - g ** n) / (1 - g)


@pytest.mark.parametrize("n", [1, 48, 360])
def test_closed_forms_second_and_first_death(n):
    """Constant forces, flat rate.  Second death: A_x + A_y - A_xy (a death
    benefit on the second death is one on each life less one on the first);
    the endowment adds v^n (1 - nqx nqy).  The first-death vector of the
    nine-state model gives the joint-status assurance A_xy."""
    mux, muy = 0.05, 0.11
    px, py = math.exp(-mux / 12), math.exp(-muy / 12)
    tx, ty = synth.constant_force_table(mux), synth.constant_force_table(muy)
    v = np.full(n, V_FLAT)
    Ax = assurance(V_FLAT * px, V_FLAT * (1 - px), n)
    Ay = assurance(V_FLAT * py, V_FLAT * (1 - py), n)
    Axy = assurance(V_FLAT * px * py, V_FLAT * (1 - px * py), n)
    kw = dict(age2=300, term=n, table_y=ty)
    r = oracle.chain(LS_TERM, 100, 3.0, tx, v, **kw)
    # (the closed form cancels: bound the error by the size of its terms)
    assert abs(r[0, 0] - 3.0 * (Ax + Ay - Axy)) <= 1e-13 * 3.0 * (Ax + Ay)
    # the reduced states: only x alive is a single-life assurance on x, likewise y
    assert abs(r[0, 2] - 3.0 * Ax) <= 1e-13 * 3.0 * Ax
    assert abs(r[0, 6] - 3.0 * Ay) <= 1e-13 * 3.0 * Ay
    e = oracle.chain(LS_ENDOW, 100, 3.0, tx, v, **kw)
    want = 3.0 * (Ax + Ay - Axy + V_FLAT ** n * (1 - (1 - px ** n) * (1 - py ** n)))
    assert abs(e[0, 0] - want) <= 1e-13 * (want + 3.0 * (Ax + Ay))
    # first death on the nine-state model
    c1 = np.array(golden()["c9_first"][0], float)
    rf = oracle.mlife_chain(2, 3, np.stack([tx, ty]), [100, 300], c1, np.zeros(9), n, v)
    assert abs(rf[0, 0] - Axy) <= 1e-13 * Axy


@pytest.mark.parametrize("m", [1, 2, 3, 4])
def test_closed_form_joint_life_of_m_lives(m):
    """Paid while all m lives are alive: sum_{t<n} (v prod p_i)^(t+1)."""
    mus = [0.02, 0.05, 0.08, 0.12][:m]
    tabs = np.stack([synth.constant_force_table(u) for u in mus])
    n = 120
    c = np.zeros(2 ** m)
    c[0] = 1.0
    r = oracle.mlife_chain(m, 2, tabs, [10] * m, c, np.zeros(2 ** m), n, np.full(n, V_FLAT))
    g = V_FLAT * math.prod(math.exp(-u / 12) for u in mus)
    want = g * (1 - g ** n) / (1 - g)
    assert abs(r[0, 0] - want) <= 1e-13 * want


# ------------------------------------------------- brute-force enumeration ----

def death_dist(tab, age, S):
    out, surv = [], 1.0
    for d in range(S):
        p = tab[age + d] if age + d < len(tab) else 0.0
        out.append(surv * (1 - p))
        surv *= p
    out.append(surv)
    return out


def enumerate_lives(tabs, ages, v, S, pv_of):
    """sum over the death steps d_i in 0..S (S = alive at the end) of Pr x pv_of(d)."""
    disc = np.concatenate([[1.0], np.cumprod(v[:S])])
    dists = [death_dist(t, a, S) for t, a in zip(tabs, ages)]
    total = 0.0
    for d in itertools.product(range(S + 1), repeat=len(tabs)):
        prob = math.prod(dists[i][d[i]] for i in range(len(tabs)))
        if prob != 0.0:
            total += prob * pv_of(d, disc)
    return total


@pytest.mark.parametrize("seed", range(3))
def test_brute_force_second_death(seed):
    rng = np.random.default_rng(800 + seed)
    n_ages = 14
    tx, ty = rng.uniform(0.3, 0.999, n_ages), rng.uniform(0.3, 0.999, n_ages)
    v = rng.uniform(0.85, 1.0, n_ages + 2)
    for ax, ay, term in [(0, 3, 8), (9, 4, 6), (2, 2, 5), (11, 6, 3)]:
        A = float(rng.uniform(1, 50))
        for prod in (LS_TERM, LS_ENDOW):
            r = oracle.chain(prod, ax, A, tx, v, age2=ay, term=term, table_y=ty)
            S = r.shape[0] - 1

            def pv(d, disc, prod=prod, S=S):
                second = max(d)
                out = A * disc[second + 1] if second < S else 0.0
                if prod == LS_ENDOW and second == S and S == term:
                    out += A * disc[S]
                return out

            want = enumerate_lives([tx, ty], [ax, ay], v, S, pv)
            assert abs(r[0, 0] - want) <= 1e-14 * A, (prod, ax, ay, term)
            s = oracle.chain(prod, ax, A, tx, v, age2=ay, term=term, table_y=ty, method="summation")
            assert abs(s[0, 0] - want) <= 1e-14 * A
            # only x alive (y already dead): the single life's benefit
            want_x = enumerate_lives([tx], [ax], v, S,
                                     lambda d, disc: (A * disc[d[0] + 1] if d[0] < S else
                                                      (A * disc[S] if prod == LS_ENDOW and S == term else 0.0)))
            assert abs(r[0, 2] - want_x) <= 1e-14 * A
    V0, _ = oracle.reserves_batch(
        {"product": [LS_TERM, LS_TERM, LS_ENDOW], "age1_m": [0, 0, 0], "age2_m": [3, 3, 3], "term_m": [8, 8, 8],
         "state0": [0, 2, 1], "table1": [0, 0, 0], "table2": [1, 1, 1], "amount": [1.0, 1.0, 1.0],
         "reversion": [0.0, 0.0, 0.0]}, np.stack([tx, ty]), v[None, :])
    r = oracle.chain(LS_TERM, 0, 1.0, tx, v, age2=3, term=8, table_y=ty)
    e = oracle.chain(LS_ENDOW, 0, 1.0, tx, v, age2=3, term=8, table_y=ty)
    assert V0[0, 0] == r[0, 0] and V0[1, 0] == r[0, 6] and V0[2, 0] == e[0, 2]


def alive_digits(state, m, base):
    """digits of a state index, life 1 first (0 = alive)."""
    out = []
    for _ in range(m):
        out.append(state % base)
        state //= base
    return out[::-1]


@pytest.mark.parametrize("k", [1, 2, 3])
def test_brute_force_three_lives(k):
    """Three lives: an annuity paid while at least k are alive (two-state model,
    c = 1 on the states with >= k digits alive) and a benefit at the end of the
    step of the k-th death (three-state model, c = 1 on the states where the
    k-th death falls in the step: #dead before < k <= #dead before + #died in it)."""
    rng = np.random.default_rng(900 + k)
    n_ages, S = 12, 7
    tabs = [rng.uniform(0.3, 0.99, n_ages) for _ in range(3)]
    ages = [0, 2, 4]
    v = rng.uniform(0.9, 1.0, S)
    c_ann = np.array([1.0 if alive_digits(s, 3, 2).count(0) >= k else 0.0 for s in range(8)])
    r = oracle.mlife_chain(3, 2, np.stack(tabs), ages, c_ann, np.zeros(8), S, v)

    def pv_ann(d, disc):
        return sum(disc[u + 1] for u in range(S) if sum(1 for x in d if u < x) >= k)

    want = enumerate_lives(tabs, ages, v, S, pv_ann)
    assert abs(r[0, 0] - want) <= 1e-14
    c_ass = np.zeros(27)
    for s in range(27):
        dg = alive_digits(s, 3, 3)
        before, now = dg.count(2), dg.count(1)
        c_ass[s] = 1.0 if before < k <= before + now else 0.0
    r = oracle.mlife_chain(3, 3, np.stack(tabs), ages, c_ass, np.zeros(27), S, v)

    def pv_ass(d, disc):
        t = sorted(d)[k - 1]
        return disc[t + 1] if t < S else 0.0

    want = enumerate_lives(tabs, ages, v, S, pv_ass)
    assert abs(r[0, 0] - want) <= 1e-14
