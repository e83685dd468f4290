"""Seeded synthetic inputs for the reserve recurrence.

This module is the only code shared by the FP64 oracle and the CUDA path.  It
draws inputs and nothing else: it holds none of the reserve arithmetic.  Every
generator is deterministic in its seed.

What it makes (shapes and distributions follow the workloads the library is
measured on; the paper's own data is synthetic too, Section 5):

* ``gm_monthly_survival`` -- a monthly decrement table p_k, k = age in whole
  months, from Gompertz-Makeham mortality mu(x) = A + B c^x integrated exactly
  over each month; p_k = 0 from the limiting age (120) on, the boundary the
  paper uses for whole-life contracts (Section 4.1.1, 4.2.1).
* ``portfolio_single_life`` / ``portfolio_mix`` -- policy records as a dict of
  NumPy arrays (structure of arrays).
* ``flat_scenarios`` / ``vasicek_scenarios`` -- per-step discount factors
  v[s, t] = exp(-integral of the short rate over step t) for scenario s
  (Section 3.4: any interest model may supply the sequence {v_t}).
"""
from __future__ import annotations

import math

import numpy as np

# Product codes.  The numbering is a data format shared with the C ABI.
SL_ANNUITY = 0          # single-life level annuity, monthly in arrears (Section 4.1.1)
JL_REVERSIONARY = 1     # joint-life annuity with reversion rho to the second life (Section 4.2.1)
TERM_ASSURANCE = 2      # level term assurance, benefit at end of month of death (Section 4.1.3)
ENDOWMENT = 3           # endowment assurance: term assurance + maturity payment (Sections 4.1.2-4.1.3)
JOINT_ANNUITY = 4       # paid while both lives are alive
LAST_SURVIVOR = 5       # paid while at least one life is alive
JOINT_TERM = 6          # sum at the end of the month of the first death within the term
JOINT_ENDOWMENT = 7     # joint term assurance + maturity payment if both are alive
LS_TERM = 8             # sum at the end of the month of the second death within the term
LS_ENDOWMENT = 9        # second-death term assurance + maturity payment if either is alive

PRODUCT_NAMES = {SL_ANNUITY: "sl_annuity", JL_REVERSIONARY: "jl_reversionary",
                 TERM_ASSURANCE: "term_assurance", ENDOWMENT: "endowment"}

LIMIT_AGE_M = 1440      # age 120 in months: p_k = 0 for k >= 1440

GM_A, GM_B, GM_C = 0.0005, 0.00003, 1.1


def gm_monthly_survival(A: float = GM_A, B: float = GM_B, c: float = GM_C,
                        limit_age_m: int = LIMIT_AGE_M) -> np.ndarray:
    """Monthly survival probabilities p_k for k = 0 .. limit_age_m - 1 (FP64).

    p_k = exp(-int_{k/12}^{(k+1)/12} (A + B c^x) dx)
        = exp(-A/12 - B c^{k/12} (c^{1/12} - 1) / ln c).
    Entries at and beyond ``limit_age_m`` are not stored: a table of length n
    means p_k = 0 for every k >= n.
    """
    k = np.arange(limit_age_m, dtype=np.float64)
    lnc = math.log(c)
    integral = A / 12.0 + B * np.exp(lnc * k / 12.0) * math.expm1(lnc / 12.0) / lnc
    return np.exp(-integral)


def constant_force_table(mu: float, n_ages: int = LIMIT_AGE_M) -> np.ndarray:
    """Monthly survival under a constant force of mortality mu (per year)."""
    return np.full(n_ages, math.exp(-mu / 12.0))


def _policy_arrays(n: int) -> dict:
    return {
        "product": np.zeros(n, np.int32),
        "age1_m": np.zeros(n, np.int32),
        "age2_m": np.zeros(n, np.int32),
        "term_m": np.zeros(n, np.int32),      # 0 = whole life (to the limiting age)
        "state0": np.zeros(n, np.int32),      # state at valuation, 0 = all lives alive
        "table1": np.zeros(n, np.int32),
        "table2": np.zeros(n, np.int32),
        "amount": np.zeros(n, np.float64),    # per-step annuity amount, or sum assured
        "reversion": np.zeros(n, np.float64), # rho, JL reversionary only
    }


def portfolio_single_life(n: int = 1000, seed: int = 0, age_lo_y: int = 60, age_hi_y: int = 90,
                          annual_median: float = 1.0e4, sigma: float = 0.5) -> dict:
    """Single-life monthly level annuities, whole life (to age 120).

    Ages are uniform over the whole months in [age_lo_y, age_hi_y] years; the
    annual amount is lognormal(ln annual_median, sigma) paid as annual/12 per
    month.
    """
    rng = np.random.default_rng([seed, 0])
    pol = _policy_arrays(n)
    pol["product"][:] = SL_ANNUITY
    pol["age1_m"][:] = rng.integers(age_lo_y * 12, age_hi_y * 12 + 1, size=n)
    pol["amount"][:] = rng.lognormal(math.log(annual_median), sigma, size=n) / 12.0
    return pol


def portfolio_mix(n: int = 100_000, seed: int = 0, age_lo_y: int = 20, age_hi_y: int = 85,
                  shares=(0.4, 0.2, 0.2, 0.2)) -> dict:
    """The four-product mix: SL annuities, JL reversionary annuities (rho ~ U[0.5, 1]),
    level term assurances (terms 5-40 y) and endowment assurances (terms 10-30 y).

    Ages uniform over whole months in [age_lo_y, age_hi_y] years (both lives of a
    JL policy drawn independently from the same range).  Annuity amounts:
    annual lognormal(ln 1e4, 0.5) paid monthly as annual/12; sums assured
    lognormal(ln 1e5, 0.5).  Product counts are exact (n * share, the remainder
    going to the first product) and the records are shuffled.
    """
    rng = np.random.default_rng([seed, 1])
    counts = [int(n * s) for s in shares]
    counts[0] += n - sum(counts)
    prod = np.concatenate([np.full(c, p, np.int32) for p, c in zip(range(4), counts)])
    rng.shuffle(prod)
    pol = _policy_arrays(n)
    pol["product"][:] = prod
    pol["age1_m"][:] = rng.integers(age_lo_y * 12, age_hi_y * 12 + 1, size=n)
    pol["age2_m"][:] = rng.integers(age_lo_y * 12, age_hi_y * 12 + 1, size=n)
    term_y = np.where(prod == TERM_ASSURANCE, rng.integers(5, 41, size=n),
                      np.where(prod == ENDOWMENT, rng.integers(10, 31, size=n), 0))
    pol["term_m"][:] = term_y * 12
    ann = rng.lognormal(math.log(1.0e4), 0.5, size=n) / 12.0
    sums = rng.lognormal(math.log(1.0e5), 0.5, size=n)
    annuity = (prod == SL_ANNUITY) | (prod == JL_REVERSIONARY)
    pol["amount"][:] = np.where(annuity, ann, sums)
    pol["reversion"][:] = np.where(prod == JL_REVERSIONARY, rng.uniform(0.5, 1.0, size=n), 0.0)
    pol["age2_m"][prod != JL_REVERSIONARY] = 0
    return pol


def portfolio_two_life(n: int = 10_000, seed: int = 0, age_lo_y: int = 20, age_hi_y: int = 85,
                       products=(JOINT_ANNUITY, LAST_SURVIVOR, JOINT_TERM, JOINT_ENDOWMENT)) -> dict:
    """Equal shares of the two-life products: by default joint-life annuities,
    last-survivor annuities, joint-life term assurances (terms 5-40 y) and
    joint-life endowments (terms 10-30 y); the second-death term assurances and
    endowments (LS_TERM, LS_ENDOWMENT) take the same terms.  Both ages uniform
    over whole months in [age_lo_y, age_hi_y] years; amounts as in
    ``portfolio_mix``."""
    rng = np.random.default_rng([seed, 2])
    prod = np.resize(np.asarray(products, dtype=np.int32), n)
    rng.shuffle(prod)
    pol = _policy_arrays(n)
    pol["product"][:] = prod
    pol["age1_m"][:] = rng.integers(age_lo_y * 12, age_hi_y * 12 + 1, size=n)
    pol["age2_m"][:] = rng.integers(age_lo_y * 12, age_hi_y * 12 + 1, size=n)
    term_y = np.where(np.isin(prod, (JOINT_TERM, LS_TERM)), rng.integers(5, 41, size=n),
                      np.where(np.isin(prod, (JOINT_ENDOWMENT, LS_ENDOWMENT)), rng.integers(10, 31, size=n), 0))
    pol["term_m"][:] = term_y * 12
    ann = rng.lognormal(math.log(1.0e4), 0.5, size=n) / 12.0
    sums = rng.lognormal(math.log(1.0e5), 0.5, size=n)
    pol["amount"][:] = np.where(prod <= LAST_SURVIVOR, ann, sums)
    return pol


def payment_schedules(n: int, seed: int = 0, annual_share: float = 0.2, escalating_share: float = 0.05,
                      increasing_share: float = 0.0, steps_per_year: int = 12) -> dict:
    """Payment-schedule parameters per policy (the fields of ``rsv_schedule``),
    drawn like the paper's cohort of new annuities (Section 5): about 80% paid
    monthly and the rest annually on the policy anniversary; about 95% level and
    the rest escalating at 3%, 4.25% or 5% on each anniversary; optionally a
    share increasing by 5-20% of the initial level per year.  The months since
    the last anniversary are uniform (inception uniform over the last year).
    Parameters only: the cash flows themselves are the consumer's to expand."""
    rng = np.random.default_rng(seed + 7_000_003)
    since = rng.integers(0, steps_per_year, n).astype(np.int32)
    annual = rng.uniform(size=n) < annual_share
    every = np.where(annual, steps_per_year, 1).astype(np.int32)
    first = np.where(annual, steps_per_year - 1 - since, 0).astype(np.int32)
    esc = np.where(rng.uniform(size=n) < escalating_share, rng.choice([0.03, 0.0425, 0.05], n), 0.0)
    inc = np.where(rng.uniform(size=n) < increasing_share, rng.uniform(0.05, 0.2, n), 0.0)
    return {"every": every, "first": first, "since": since,
            "steps_per_year": np.full(n, steps_per_year, np.int32), "escalation": esc, "increase": inc}


def take(pol: dict, idx) -> dict:
    """Sub-portfolio with the records at ``idx`` (any NumPy index)."""
    return {k: np.ascontiguousarray(v[idx]) for k, v in pol.items()}


def flat_scenarios(annual_rate: float = 0.04, n_steps: int = 720, n_scen: int = 1) -> np.ndarray:
    """Constant monthly discount factor v = (1 + i)^(-1/12), shape [n_scen, n_steps]."""
    return np.full((n_scen, n_steps), (1.0 + annual_rate) ** (-1.0 / 12.0))


def vasicek_step_moments(a: float, b: float, sigma: float, dt: float):
    """Moments of one exact step of the Vasicek model dr = a(b - r)dt + sigma dW.

    Given r_t, (r_{t+dt}, I) with I = int_t^{t+dt} r_u du is bivariate normal:
      E[r'] = b + (r_t - b) e^{-a dt}
      E[I]  = b dt + (r_t - b)(1 - e^{-a dt}) / a
      Var r' = sigma^2 (1 - e^{-2a dt}) / (2a)
      Var I  = sigma^2 / a^2 [dt - 2(1 - e^{-a dt})/a + (1 - e^{-2a dt})/(2a)]
      Cov    = sigma^2 / (2a^2) (1 - e^{-a dt})^2
    (Glasserman, Monte Carlo Methods in Financial Engineering, 2004, Sec. 3.3.)
    Returns (e^{-a dt}, (1 - e^{-a dt})/a, var_r, var_i, cov).
    """
    e = math.exp(-a * dt)
    one_m_e = -math.expm1(-a * dt)
    var_r = sigma * sigma * (-math.expm1(-2 * a * dt)) / (2 * a)
    var_i = sigma * sigma / (a * a) * (dt - 2 * one_m_e / a + (-math.expm1(-2 * a * dt)) / (2 * a))
    cov = sigma * sigma / (2 * a * a) * one_m_e * one_m_e
    return e, one_m_e / a, var_r, var_i, cov


def vasicek_paths(n_scen: int, n_steps: int, seed: int = 0, a: float = 0.1, b: float = 0.04,
                  sigma: float = 0.01, r0: float = 0.03, dt: float = 1.0 / 12.0,
                  stream: int = 1, return_rates: bool = False):
    """Exact-step Vasicek short-rate paths and their monthly discount factors (FP64).

    v[s, t] = exp(-int over step t of r) for scenario s, shape [n_scen, n_steps].
    With ``return_rates`` also returns r[s, t] for t = 0 .. n_steps (r[:, 0] = r0).
    Negative rates are allowed (no floor).
    """
    e, k1, var_r, var_i, cov = vasicek_step_moments(a, b, sigma, dt)
    # Cholesky factor of [[var_r, cov], [cov, var_i]]
    l11 = math.sqrt(var_r)
    l21 = cov / l11
    l22 = math.sqrt(max(var_i - l21 * l21, 0.0))
    rng = np.random.default_rng([seed, stream])
    z = rng.standard_normal((n_steps, 2, n_scen))
    r = np.full(n_scen, r0, np.float64)
    rates = np.empty((n_steps + 1, n_scen)) if return_rates else None
    if return_rates:
        rates[0] = r
    v = np.empty((n_steps, n_scen), np.float64)       # step-major while generating
    for t in range(n_steps):
        z1, z2 = z[t, 0], z[t, 1]
        integral = b * dt + (r - b) * k1 + l21 * z1 + l22 * z2
        r = b + (r - b) * e + l11 * z1
        v[t] = np.exp(-integral)
        if return_rates:
            rates[t + 1] = r
    v = np.ascontiguousarray(v.T)
    if return_rates:
        rates = np.ascontiguousarray(rates.T)
    return (v, rates) if return_rates else v


def vasicek_zcb(tau: float, r: float, a: float = 0.1, b: float = 0.04, sigma: float = 0.01) -> float:
    """Vasicek (1977) zero-coupon bond price P(tau | r) = A(tau) exp(-B(tau) r)."""
    B = -math.expm1(-a * tau) / a
    lnA = (B - tau) * (a * a * b - sigma * sigma / 2) / (a * a) - sigma * sigma * B * B / (4 * a)
    return math.exp(lnA - B * r)
