/*
 * rsv_oracle.c -- plain FP64 CPU oracle for the vector reserve recurrence of
 * M. Tucker and J. M. Bull, "An efficient algorithm for the calculation of
 * reserves for non-unit linked life policies" (arXiv 1401.1757).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  The CUDA library never
 * calls it and the two share no code, headers or tables.
 *
 * What it computes, in the paper's notation (Section 3):
 *   - full-state Markov transition matrices W_{x,t,g} of the use cases in
 *     Section 4 (row j = state at the start of the step, column i = state at
 *     t+g; rows sum to one; "0 = alive" labelling makes them upper triangular);
 *   - the cash-flow vectors c_{x,t} of the four products;
 *   - the reserve vector r_{x,t} for every t, two independent ways:
 *       (a) backward substitution of Eq. (generalForm),
 *             r_t = v_t^f W_{t,f} c_t + v_t W_{t,1} r_{t+1},
 *           from the boundary vector r_S (Section 3.8.2);
 *       (b) the prospective-reserve definition, Eq. (basicReserveSummation),
 *             r_{t,j} = sum_{s>=t} d(t, s+f) sum_i w(t, s+f)_{j,i} c_{s,i},
 *           with multi-step discount factors and transition probabilities
 *           built from one-step ones by Eqs. (recRel_Discounts) and
 *           (recRel_Probabilities) (Section 3.6.1).  O(S^2).
 * No state is removed (no zero-reserve-state reduction, Section 3.6.4): the
 * full vector is returned, and zero-reserve states come out as zeros.
 *
 * Every function is pinned by the CPU tests (closed forms under a flat rate
 * and constant force, brute-force enumeration over death times on tiny
 * inputs, recurrence == summation, the paper's printed scalar recurrences,
 * and the structural invariants of W and r).
 *
 * Build: plain C99, -O2 -ffp-contract=off (no fused multiply-add, so the
 * same IEEE double operations run on x86-64 and AArch64), OpenMP optional.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXN 9

enum {
    ORC_SL_ANNUITY = 0, ORC_JL_REVERSIONARY = 1, ORC_TERM_ASSURANCE = 2, ORC_ENDOWMENT = 3,
    /* two-life products built from the same state models (Section 4.2 and the
     * assurance model of Section 4.1.3 applied to the joint status) */
    ORC_JOINT_ANNUITY = 4,       /* paid while both lives are alive            */
    ORC_LAST_SURVIVOR = 5,       /* paid while at least one life is alive      */
    ORC_JOINT_TERM = 6,          /* sum paid at the end of the step of the first death */
    ORC_JOINT_ENDOWMENT = 7,     /* the same, or at maturity if both are alive */
    /* the two-life assurance model of Section 4.2.3 (nine states) */
    ORC_LS_TERM = 8,             /* sum paid at the end of the step of the second death */
    ORC_LS_ENDOWMENT = 9         /* the same, or at maturity if at least one is alive */
};

static int nine_state(int product) { return product == ORC_LS_TERM || product == ORC_LS_ENDOWMENT; }

static int two_state_life(int product) { return product == ORC_JL_REVERSIONARY || product == ORC_JOINT_ANNUITY || product == ORC_LAST_SURVIVOR; }

/* Number of survival states of the product's full model (Section 4):
 * single life alive/dead (4.1), single life alive/died-in-step/dead for
 * assurances (4.1.3), two lives 00/01/10/11 (4.2); the joint-status
 * assurances use the assurance model with "alive" = both alive. */
int orc_n_states(int product)
{
    switch (product) {
    case ORC_SL_ANNUITY: return 2;
    case ORC_JL_REVERSIONARY:
    case ORC_JOINT_ANNUITY:
    case ORC_LAST_SURVIVOR: return 4;
    case ORC_TERM_ASSURANCE:
    case ORC_ENDOWMENT:
    case ORC_JOINT_TERM:
    case ORC_JOINT_ENDOWMENT: return 3;
    case ORC_LS_TERM:
    case ORC_LS_ENDOWMENT: return 9;
    default: return -1;
    }
}

/* Index in the full state vector of a reduced valuation state (the record's
 * state0: 0 = every life alive; for the two-life models 1 = only the first
 * life alive, 2 = only the second).  The nine-state model labels state
 * 3 i_x + i_y with i = 0 alive, 1 died in the step, 2 dead (Section 4.2.3),
 * so "only x alive" is (0, 2) = 2 and "only y alive" (2, 0) = 6. */
int orc_full_state(int product, int state0)
{
    if (nine_state(product)) return state0 == 0 ? 0 : (state0 == 1 ? 2 : (state0 == 2 ? 6 : -1));
    return state0;
}

/* W_{x,t,g} for survival probabilities px = gp_x (and py = gp_y for two
 * lives) over the interval of length g.  Row-major n x n, W[j*n + i] =
 * w_{j,i} = Pr[state i at t+g | state j at t]. */
int orc_transition(int product, double px, double py, double *W)
{
    int n = orc_n_states(product);
    if (n < 0) return -1;
    double qx = 1.0 - px, qy = 1.0 - py;
    for (int k = 0; k < n * n; ++k) W[k] = 0.0;
    if (product == ORC_SL_ANNUITY) {            /* Eq. (two state, single life) */
        W[0 * 2 + 0] = px; W[0 * 2 + 1] = qx;
        W[1 * 2 + 1] = 1.0;
    } else if (two_state_life(product)) {         /* Section 4.2, binary labels */
        W[0 * 4 + 0] = px * py; W[0 * 4 + 1] = px * qy; W[0 * 4 + 2] = qx * py; W[0 * 4 + 3] = qx * qy;
        W[1 * 4 + 1] = px; W[1 * 4 + 3] = qx;
        W[2 * 4 + 2] = py; W[2 * 4 + 3] = qy;
        W[3 * 4 + 3] = 1.0;
    } else if (nine_state(product)) {
        /* Section 4.2.3: the assurance model of Section 4.1.3 for both lives,
         * state 3 i_x + i_y; a "died in the step" state moves to "dead" */
        W[0 * 9 + 0] = px * py; W[0 * 9 + 1] = px * qy; W[0 * 9 + 3] = qx * py; W[0 * 9 + 4] = qx * qy;
        W[1 * 9 + 2] = px; W[1 * 9 + 5] = qx;
        W[2 * 9 + 2] = px; W[2 * 9 + 5] = qx;
        W[3 * 9 + 6] = py; W[3 * 9 + 7] = qy;
        W[4 * 9 + 8] = 1.0;
        W[5 * 9 + 8] = 1.0;
        W[6 * 9 + 6] = py; W[6 * 9 + 7] = qy;
        W[7 * 9 + 8] = 1.0;
        W[8 * 9 + 8] = 1.0;
    } else if (product == ORC_JOINT_TERM || product == ORC_JOINT_ENDOWMENT) {
        /* three states of the joint status: both alive / first death in the step / after */
        W[0 * 3 + 0] = px * py; W[0 * 3 + 1] = 1.0 - px * py;
        W[1 * 3 + 2] = 1.0;
        W[2 * 3 + 2] = 1.0;
    } else {                                     /* Eq. (three state, single life) */
        W[0 * 3 + 0] = px; W[0 * 3 + 1] = qx;
        W[1 * 3 + 2] = 1.0;
        W[2 * 3 + 2] = 1.0;
    }
    return n;
}

/* Nominal cash-flow vector c_{x,t} (paid at t+f according to the state then).
 *   SL annuity (4.1.1):        (A, 0)
 *   JL reversionary (4.2.1):   (A, A, rho*A, 0): A while (x) lives, rho*A to (y) after (x) dies
 *   joint-life annuity:        (A, 0, 0, 0): while both live
 *   last-survivor annuity:     (A, A, A, 0): while either lives
 *   term / endowment (4.1.3) and their joint-status forms:
 *                              (0, A, 0): benefit in the "died in step" state
 *   second-death term / endowment (4.2.3), nine states 3 i_x + i_y:
 *                              A in (1,1), (1,2), (2,1): the second death in the step */
int orc_cashflow(int product, double amount, double rho, double *c)
{
    int n = orc_n_states(product);
    if (n < 0) return -1;
    for (int k = 0; k < n; ++k) c[k] = 0.0;
    if (product == ORC_SL_ANNUITY) c[0] = amount;
    else if (product == ORC_JL_REVERSIONARY) { c[0] = amount; c[1] = amount; c[2] = rho * amount; }
    else if (product == ORC_JOINT_ANNUITY) c[0] = amount;
    else if (product == ORC_LAST_SURVIVOR) { c[0] = amount; c[1] = amount; c[2] = amount; }
    else if (nine_state(product)) { c[4] = amount; c[5] = amount; c[7] = amount; }   /* second death */
    else c[1] = amount;
    return n;
}

/* Number of projection steps S of a policy and its boundary vector r_S.
 * Whole-life annuities run to the limiting age: a table of n_ages entries
 * means p_k = 0 for k >= n_ages, so S = n_ages - (youngest age) (Sections
 * 4.1.1, 4.2.1: sp_120 = 0).  term_m > 0 limits the term.  Assurances run for
 * their term.  An endowment pays its sum at maturity if alive: boundary
 * r_S = (A, 0, 0) (Section 4.1.2, A_{x+n:0} = 1); the second-death
 * endowment if either life is alive.  A horizon > 0 truncates
 * the projection with r_horizon = 0, dropping later cash flows. */
int orc_steps(int product, int age1, int age2, int term, int n_ages, int horizon,
              double amount, double *rS)
{
    int n = orc_n_states(product), S;
    if (n < 0) return -1;
    if (product == ORC_SL_ANNUITY || product == ORC_JL_REVERSIONARY || product == ORC_LAST_SURVIVOR) {
        /* paid while some life can be alive: to the younger life's limiting age */
        int young = (product != ORC_SL_ANNUITY && age2 < age1) ? age2 : age1;
        S = n_ages - young;
        if (S < 0) S = 0;
        if (term > 0 && term < S) S = term;
    } else if (product == ORC_JOINT_ANNUITY) {
        /* paid while both can be alive: to the older life's limiting age */
        int old = age2 > age1 ? age2 : age1;
        S = n_ages - old;
        if (S < 0) S = 0;
        if (term > 0 && term < S) S = term;
    } else {
        S = term;
    }
    for (int k = 0; k < n; ++k) rS[k] = 0.0;
    if (horizon > 0 && horizon < S) {
        S = horizon;                          /* truncated: r_S = 0 */
    } else if (product == ORC_ENDOWMENT || product == ORC_JOINT_ENDOWMENT) {
        rS[0] = amount;
    } else if (product == ORC_LS_ENDOWMENT) {
        /* at maturity, every state with a life alive: (0,0), (0,1), (0,2), (1,0), (2,0) */
        rS[0] = rS[1] = rS[2] = rS[3] = rS[6] = amount;
    }
    return S;
}

static double table_at(const double *tab, int n_ages, int k)
{
    return (k >= 0 && k < n_ages) ? tab[k] : 0.0;
}

/* y = W x  (n x n times n) */
static void matvec(int n, const double *W, const double *x, double *y)
{
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += W[j * n + i] * x[i];
        y[j] = s;
    }
}

/* C = A B  (n x n) */
static void matmul(int n, const double *A, const double *B, double *C)
{
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += A[j * n + k] * B[k * n + i];
            C[j * n + i] = s;
        }
}

/* One chain (one policy under one discount sequence), every t.
 *
 * p1x/p1y: one-step survival tables of the two lives (p1y unused for one
 * life), indexed by age in months; pfx/pfy: survival over the fraction f of
 * the step (equal to p1x/p1y when f = 1).  v[t]: discount factor over step t;
 * vf[t]: discount from t to t+f (v^f; equal to v when f = 1).
 * cf[t] (NULL: all 1) scales the product's nominal cash-flow vector of
 * step t: c_t = cf[t] c (Section 4.1.1: increasing, escalating and limited
 * term annuities differ only in the sequence c_t; Section 4.6: the sequence
 * carries the timing, e.g. one non-zero step in twelve for annual payments).
 * The boundary r_S (an endowment's maturity sum) is not scaled.
 * method 0: backward recurrence, Eq. (generalForm); method 1: summation,
 * Eq. (basicReserveSummation).
 * r_out[(S+1) * n] receives r_t for t = 0..S (r_S is the boundary).
 * Returns S, or a negative code: -1 bad product, -2 scenario too short. */
int orc_chain_cf(int product, int age1, int age2, int term, double amount, double rho,
                 int n_ages, const double *p1x, const double *p1y,
                 const double *pfx, const double *pfy,
                 int n_steps, const double *v, const double *vf, const double *cf,
                 int horizon, int method, double *r_out)
{
    double rS[ORC_MAXN], c0[ORC_MAXN], c[ORC_MAXN];
    int n = orc_n_states(product);
    if (n < 0) return -1;
    int S = orc_steps(product, age1, age2, term, n_ages, horizon, amount, rS);
    if (S > n_steps) return -2;
    orc_cashflow(product, amount, rho, c0);
    for (int j = 0; j < n; ++j) r_out[S * n + j] = rS[j];

    if (method == 0) {
        double W1[ORC_MAXN * ORC_MAXN], Wf[ORC_MAXN * ORC_MAXN], a[ORC_MAXN], b[ORC_MAXN];
        for (int t = S - 1; t >= 0; --t) {
            orc_transition(product, table_at(p1x, n_ages, age1 + t),
                           p1y ? table_at(p1y, n_ages, age2 + t) : 0.0, W1);
            orc_transition(product, table_at(pfx, n_ages, age1 + t),
                           pfy ? table_at(pfy, n_ages, age2 + t) : 0.0, Wf);
            for (int j = 0; j < n; ++j) c[j] = cf ? cf[t] * c0[j] : c0[j];   /* c_t */
            matvec(n, Wf, c, a);                          /* W_{t,f} c_t     */
            matvec(n, W1, &r_out[(t + 1) * n], b);        /* W_{t,1} r_{t+1} */
            for (int j = 0; j < n; ++j) r_out[t * n + j] = vf[t] * a[j] + v[t] * b[j];
        }
        return S;
    }

    /* Summation: for each t, walk s = t..S-1 keeping the running products
     * prod_{u=t}^{s-1} v_u and prod_{u=t}^{s-1} W_{u,1}. */
    double M[ORC_MAXN * ORC_MAXN], M2[ORC_MAXN * ORC_MAXN], W1[ORC_MAXN * ORC_MAXN],
           Wf[ORC_MAXN * ORC_MAXN], P[ORC_MAXN * ORC_MAXN], a[ORC_MAXN];
    for (int t = 0; t < S; ++t) {
        double acc[ORC_MAXN] = {0};
        double d = 1.0;                                   /* d(t, s) */
        for (int k = 0; k < n * n; ++k) M[k] = (k / n == k % n) ? 1.0 : 0.0;
        for (int s = t; s < S; ++s) {
            orc_transition(product, table_at(p1x, n_ages, age1 + s),
                           p1y ? table_at(p1y, n_ages, age2 + s) : 0.0, W1);
            orc_transition(product, table_at(pfx, n_ages, age1 + s),
                           pfy ? table_at(pfy, n_ages, age2 + s) : 0.0, Wf);
            matmul(n, M, Wf, P);                          /* w(t, s+f) */
            for (int j = 0; j < n; ++j) c[j] = cf ? cf[s] * c0[j] : c0[j];   /* c_s */
            matvec(n, P, c, a);
            for (int j = 0; j < n; ++j) acc[j] += d * vf[s] * a[j];
            matmul(n, M, W1, M2);                         /* w(t, s+1) */
            memcpy(M, M2, sizeof(double) * n * n);
            d *= v[s];                                    /* d(t, s+1) */
        }
        /* the boundary vector r_S acts as a cash flow at time S */
        matvec(n, M, rS, a);
        for (int j = 0; j < n; ++j) r_out[t * n + j] = acc[j] + d * a[j];
    }
    return S;
}

int orc_chain(int product, int age1, int age2, int term, double amount, double rho,
              int n_ages, const double *p1x, const double *p1y,
              const double *pfx, const double *pfy,
              int n_steps, const double *v, const double *vf,
              int horizon, int method, double *r_out)
{
    return orc_chain_cf(product, age1, age2, term, amount, rho, n_ages, p1x, p1y, pfx, pfy,
                        n_steps, v, vf, NULL, horizon, method, r_out);
}

/* Cash-flow multipliers of a payment schedule (Section 4.1.1 and 4.6), for
 * steps t = 0 .. n_steps-1 from valuation:
 *   cf[t] = [t >= first and (t - first) mod every == 0] (1 + increase n_t) (1 + escalation)^n_t,
 *   n_t = floor((t + since) / steps_per_year),
 * i.e. a payment every `every` steps starting at step `first`, with the level
 * in force during step t raised at each policy anniversary: by `increase`
 * times the initial level (arithmetic progression, an increasing annuity) and
 * by the factor 1 + escalation (geometric progression, an escalating
 * annuity).  `since` is the number of steps since the last anniversary at
 * valuation (0 .. steps_per_year-1).  Returns 0, or -1 for bad parameters. */
int orc_schedule(int n_steps, int every, int first, int since, int steps_per_year,
                 double escalation, double increase, double *cf)
{
    if (n_steps < 0 || every < 1 || first < 0 || steps_per_year < 1 || since < 0 ||
        since >= steps_per_year || !(escalation > -1.0) || !(increase >= 0.0))
        return -1;
    for (int t = 0; t < n_steps; ++t) {
        if (t < first || (t - first) % every != 0) {
            cf[t] = 0.0;
            continue;
        }
        int n_t = (t + since) / steps_per_year;
        double g = 1.0;
        for (int k = 0; k < n_t; ++k) g *= 1.0 + escalation;
        cf[t] = (1.0 + increase * n_t) * g;
    }
    return 0;
}

/* ---- m lives (Section 4.3) ----------------------------------------------
 * The transition matrix of m independent lives by induction over the lives,
 *   W^m = W^{m-1} (x) w_m,  W^0 = (1),
 * with w the single-life matrix of the two-state model [[p, q], [0, 1]]
 * (model 2: annuities and endowments, states alive/dead) or of the
 * three-state model [[p, q, 0], [0, 0, 1], [0, 0, 1]] (model 3: assurances,
 * states alive/died in the step/dead).  The Kronecker product makes life 1
 * the most significant digit of the state index (base 2 or 3).  p[i] is the
 * survival probability of life i over the step.  W receives n x n row-major,
 * n = 2^m or 3^m; returns n, or -1 for m outside 0..4 or a bad model. */
int orc_mlife_transition(int m, int model, const double *p, double *W)
{
    if (m < 0 || m > 4 || (model != 2 && model != 3)) return -1;
    double A[81 * 81], w[9];
    int n = 1;
    W[0] = 1.0;
    for (int i = 0; i < m; ++i) {
        const int k = model;
        for (int e = 0; e < k * k; ++e) w[e] = 0.0;
        if (k == 2) {
            w[0] = p[i]; w[1] = 1.0 - p[i]; w[3] = 1.0;
        } else {
            w[0] = p[i]; w[1] = 1.0 - p[i]; w[5] = 1.0; w[8] = 1.0;
        }
        memcpy(A, W, sizeof(double) * n * n);
        const int nn = n * k;
        for (int r1 = 0; r1 < n; ++r1)
            for (int r2 = 0; r2 < k; ++r2)
                for (int c1 = 0; c1 < n; ++c1)
                    for (int c2 = 0; c2 < k; ++c2)
                        W[(r1 * k + r2) * nn + (c1 * k + c2)] = A[r1 * n + c1] * w[r2 * k + c2];
        n = nn;
    }
    return n;
}

/* Reserve vectors of an m-life contract under one discount sequence, for
 * t = 0..S: the backward recurrence of Eq. (generalForm) with f = 1 and a
 * cash-flow vector c fixed over the steps, r_t = v_t W^m_t (c + r_{t+1}),
 * from the boundary r_S.  tables holds m rows of n_ages one-step survival
 * probabilities; life i is aged ages[i] at t = 0 (probability 0 at or beyond
 * the table's end).  r_out receives (S + 1) x n.  Returns n, or -1. */
int orc_mlife_chain(int m, int model, int n_ages, const double *tables, const int *ages,
                    const double *c, const double *rS, int S, const double *v, double *r_out)
{
    if (m < 0 || m > 4 || (model != 2 && model != 3) || S < 0) return -1;
    double p[4], x[81], *W = (double *)malloc(sizeof(double) * 81 * 81);
    if (!W) return -1;
    int n = 1;
    for (int i = 0; i < m; ++i) n *= model;
    memcpy(&r_out[(size_t)S * n], rS, sizeof(double) * n);
    for (int t = S - 1; t >= 0; --t) {
        for (int i = 0; i < m; ++i) p[i] = table_at(tables + (size_t)i * n_ages, n_ages, ages[i] + t);
        orc_mlife_transition(m, model, p, W);
        for (int j = 0; j < n; ++j) x[j] = c[j] + r_out[(size_t)(t + 1) * n + j];
        matvec(n, W, x, &r_out[(size_t)t * n]);
        for (int j = 0; j < n; ++j) r_out[(size_t)t * n + j] *= v[t];
    }
    free(W);
    return n;
}

/* Reserves at valuation for a whole portfolio under n_scen scenarios, f = 1,
 * by the backward recurrence (method 0 of orc_chain) or, in
 * orc_reserves_batch_method with method 1, by the summation definition
 * evaluated at every step (the O(S^2) method the recurrence replaces).
 *
 * Policies are given as arrays (structure of arrays).  tables[n_tables *
 * n_ages] holds one-step survival p_k per table.  v[n_scen * n_steps] holds
 * the per-step discount factors of each scenario.  V0[p * n_scen + s]
 * receives the reserve of policy p in its valuation state state0[p];
 * scen_total[s] (optional) the sum of V0 over policies, summed in policy
 * order.  nthreads <= 0 uses the OpenMP default; policies are shared among
 * threads with a dynamic schedule.  cf (orc_reserves_batch_cf; NULL: level)
 * holds the cash-flow multipliers cf[p * n_steps + t] of every policy (see
 * orc_chain_cf).  Returns 0, or -1 bad record, -2 a scenario shorter than a
 * policy's projection. */
int orc_reserves_batch_cf(int64_t n_pol, const int32_t *product, const int32_t *age1,
                          const int32_t *age2, const int32_t *term, const int32_t *state0,
                          const int32_t *tab1, const int32_t *tab2,
                          const double *amount, const double *rho,
                          int32_t n_tables, int32_t n_ages, const double *tables,
                          int32_t n_scen, int32_t n_steps, const double *v,
                          const double *cf, int32_t horizon, int32_t nthreads, int32_t method,
                          double *V0, double *scen_total)
{
    int status = 0;
    (void)nthreads;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double *r = (double *)malloc(sizeof(double) * ORC_MAXN * ((size_t)n_steps + 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t p = 0; p < n_pol; ++p) {
            int n = orc_n_states(product[p]);
            int full = orc_full_state(product[p], state0[p]);
            if (!r || n < 0 || tab1[p] < 0 || tab1[p] >= n_tables || tab2[p] < 0 ||
                tab2[p] >= n_tables || state0[p] < 0 || full < 0 || full >= n) {
#ifdef _OPENMP
#pragma omp critical
#endif
                status = -1;
                continue;
            }
            const double *tx = tables + (size_t)tab1[p] * n_ages;
            const double *ty = tables + (size_t)tab2[p] * n_ages;
            for (int32_t s = 0; s < n_scen; ++s) {
                const double *vs = v + (size_t)s * n_steps;
                int S = orc_chain_cf(product[p], age1[p], age2[p], term[p], amount[p], rho[p],
                                     n_ages, tx, ty, tx, ty, n_steps, vs, vs,
                                     cf ? cf + (size_t)p * n_steps : NULL, horizon, method, r);
                if (S < 0) {
#ifdef _OPENMP
#pragma omp critical
#endif
                    status = S;
                    V0[p * n_scen + s] = 0.0;
                    continue;
                }
                V0[p * n_scen + s] = r[full];
            }
        }
        free(r);
    }
    if (status == 0 && scen_total) {
        for (int32_t s = 0; s < n_scen; ++s) scen_total[s] = 0.0;
        for (int64_t p = 0; p < n_pol; ++p)
            for (int32_t s = 0; s < n_scen; ++s) scen_total[s] += V0[p * n_scen + s];
    }
    return status;
}

int orc_reserves_batch_method(int64_t n_pol, const int32_t *product, const int32_t *age1,
                              const int32_t *age2, const int32_t *term, const int32_t *state0,
                              const int32_t *tab1, const int32_t *tab2,
                              const double *amount, const double *rho,
                              int32_t n_tables, int32_t n_ages, const double *tables,
                              int32_t n_scen, int32_t n_steps, const double *v,
                              int32_t horizon, int32_t nthreads, int32_t method,
                              double *V0, double *scen_total)
{
    return orc_reserves_batch_cf(n_pol, product, age1, age2, term, state0, tab1, tab2, amount, rho,
                                 n_tables, n_ages, tables, n_scen, n_steps, v, NULL, horizon, nthreads,
                                 method, V0, scen_total);
}

int orc_reserves_batch(int64_t n_pol, const int32_t *product, const int32_t *age1,
                       const int32_t *age2, const int32_t *term, const int32_t *state0,
                       const int32_t *tab1, const int32_t *tab2,
                       const double *amount, const double *rho,
                       int32_t n_tables, int32_t n_ages, const double *tables,
                       int32_t n_scen, int32_t n_steps, const double *v,
                       int32_t horizon, int32_t nthreads,
                       double *V0, double *scen_total)
{
    return orc_reserves_batch_method(n_pol, product, age1, age2, term, state0, tab1, tab2, amount, rho,
                                     n_tables, n_ages, tables, n_scen, n_steps, v, horizon, nthreads, 0,
                                     V0, scen_total);
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
