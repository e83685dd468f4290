"""Pins of the nested-valuation oracle (CPU).

* Philox4x32-10 against the known-answer vectors published with the
  generator (Salmon et al., SC'11).
* Box-Muller Gaussians: mean 0 and variance 1 within 4 standard errors.
* Counter-based Vasicek paths: the Monte Carlo mean of the discount product
  matches the Vasicek (1977) zero-coupon price within 4 standard errors.
* The liability at node 0 is the portfolio reserve on the inner path itself.
* With sigma = 0 the short rate is deterministic and every inner path gives
  the same liability, which is the survival-weighted tail of the valuation-time
  reserve written out as a sum.
* The inner Monte Carlo mean matches the recurrence on the model's forward
  curve P(t+1|r)/P(t|r) within 4 standard errors (the inner expectation).
"""
import math

import numpy as np
import pytest

import oracle
import synth


def test_philox_known_answers():
    assert oracle.philox4x32_10([0, 0, 0, 0], [0, 0]) == [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]
    assert oracle.philox4x32_10([0xffffffff] * 4, [0xffffffff] * 2) == [0x408f276d, 0x41c83b0e, 0xa20bc7c6,
                                                                        0x6d5451fd]
    assert oracle.philox4x32_10([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344], [0xa4093822, 0x299f31d0]) == \
        [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]


def test_gaussians_moments():
    z = np.concatenate([oracle.gauss_pairs(7, k, 3, 1, 5 << 24) for k in range(20000)])
    n = len(z)
    assert abs(z.mean()) < 4 / math.sqrt(n)
    assert abs(z.var() - 1) < 4 * math.sqrt(2 / n)


def test_counter_paths_match_zero_coupon_price():
    T, n = 60, 4000
    D = np.array([np.prod(oracle.inner_path(11, 0, 0, i, T, 0.03)[0]) for i in range(n)])
    want = synth.vasicek_zcb(T / 12, 0.03)
    assert abs(D.mean() - want) < 4 * D.std() / math.sqrt(n)


def small_portfolio(n=12, seed=3):
    pol = synth.portfolio_mix(n, seed=seed, age_lo_y=55, age_hi_y=85)
    return pol


def test_node_zero_is_the_portfolio_reserve():
    tab = synth.gm_monthly_survival()
    pol = small_portfolio()
    L, rn, d0 = oracle.nested_node(pol, tab, 5, 2, 0, [0, 7])
    assert rn == 0.03 and d0 == 1.0
    S = max(oracle.steps(int(p), int(a1), int(a2), int(t), 1440)[0] for p, a1, a2, t in
            zip(pol["product"], pol["age1_m"], pol["age2_m"], pol["term_m"]))
    for k, i in enumerate([0, 7]):
        v, _ = oracle.inner_path(5, 2, 0, i, S, 0.03)
        V0, tot = oracle.reserves_batch(pol, tab, v[None, :])
        assert math.isclose(L[k], tot[0], rel_tol=1e-13)


def test_deterministic_rate_liability_is_the_weighted_tail():
    """sigma = 0: L at node n = sum_p A_p sum_{s >= m} [prod_{u<=s} p] prod_{u=m}^{s} v_u for
    single-life annuities (and the assurance analogue), whatever the inner path."""
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_single_life(6, seed=2)
    a, b, r0, n, step = 0.1, 0.04, 0.03, 3, 12
    m = n * step
    L, rn, _ = oracle.nested_node(pol, tab, 1, 0, n, [0, 5], node_step=step, sigma=0.0)
    assert L[0] == L[1]
    # deterministic path: exp(-integral of r) with r_t = b + (r0 - b) e^{-a t}
    def I(t0, t1):
        return b * (t1 - t0) + (r0 - b) * (math.exp(-a * t0) - math.exp(-a * t1)) / a
    want = 0.0
    for age, A in zip(pol["age1_m"], pol["amount"]):
        surv, disc = 1.0, 1.0
        for u in range(m):
            surv *= tab[age + u] if age + u < 1440 else 0.0
        for s in range(m, 1440 - age):
            surv *= tab[age + s]
            disc *= math.exp(-I(s / 12, (s + 1) / 12))
            want += A * surv * disc
    assert math.isclose(rn, b + (r0 - b) * math.exp(-a * m / 12), rel_tol=1e-12)
    assert math.isclose(L[0], want, rel_tol=1e-11)


@pytest.mark.parametrize("node", [0, 2])
def test_inner_mean_matches_forward_curve(node):
    tab = synth.gm_monthly_survival()
    pol = small_portfolio(8, seed=9)
    n_in = 600
    L, rn, _ = oracle.nested_node(pol, tab, 21, 1, node, np.arange(n_in), node_step=24)
    m = node * 24
    want = 0.0
    for p in range(8):
        S = oracle.steps(int(pol["product"][p]), int(pol["age1_m"][p]) + m, int(pol["age2_m"][p]) + m,
                         max(0, int(pol["term_m"][p]) - m), 1440)[0]
        if int(pol["term_m"][p]) and int(pol["term_m"][p]) < m:
            continue
        curve = np.array([synth.vasicek_zcb((t + 1) / 12, rn) / synth.vasicek_zcb(t / 12, rn) for t in range(S)])
        r = oracle.chain(int(pol["product"][p]), int(pol["age1_m"][p]) + m, float(pol["amount"][p]), tab, curve,
                         age2=int(pol["age2_m"][p]) + m, term=max(0, int(pol["term_m"][p]) - m),
                         rho=float(pol["reversion"][p]))
        # in-force state distribution at the node (independent lives)
        px = np.prod([tab[pol["age1_m"][p] + u] for u in range(m)])
        if pol["product"][p] == 1:
            py = np.prod([tab[pol["age2_m"][p] + u] for u in range(m)])
            want += px * py * r[0, 0] + px * (1 - py) * r[0, 1] + (1 - px) * py * r[0, 2]
        else:
            want += px * r[0, 0]
    assert abs(L.mean() - want) < 4 * L.std() / math.sqrt(n_in)
