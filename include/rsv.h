/*
 * rsv.h -- C ABI of the GB300 reserve library.
 *
 * The library evaluates the vector reserve recurrence of Tucker & Bull,
 * "An efficient algorithm for the calculation of reserves for non-unit
 * linked life policies" (arXiv 1401.1757), Eq. (generalForm):
 *
 *     r_{x,t} = v_t^f W_{x,t,f} c_{x,t} + v_t W_{x,t,1} r_{x+1,t},
 *
 * by backward substitution from a boundary vector (Section 3.8.2), for every
 * policy x scenario of a portfolio, with f = 1 (cash flows at the end of each
 * monthly step), after the zero-reserve states of each product are removed
 * (Section 3.6.4).  Products (Section 4):
 *
 *   RSV_SL_ANNUITY       level single-life annuity, 1 reduced state
 *                        (Section 4.1.1: r = v p (A + r')).
 *   RSV_JL_REVERSIONARY  joint-life annuity paying A while the first life
 *                        lives and rho*A to the second life after the first
 *                        dies; two-life binary-labelled model of Section 4.2
 *                        with state 11 removed: 3 reduced states 00, 01, 10.
 *   RSV_TERM_ASSURANCE   level term assurance, benefit at the end of the month
 *                        of death; three-state model of Section 4.1.3 reduced
 *                        to 1 state: r = v (q S + p r').
 *   RSV_ENDOWMENT        endowment assurance: the term assurance plus the sum
 *                        at maturity if alive (Section 4.1.2 boundary
 *                        A_{x+n:0} = 1).
 *   Two-life products on the same models (Section 4.2; the assurances use
 *   the model of Section 4.1.3 on the joint status "both alive"):
 *   RSV_JOINT_ANNUITY    A while both lives are alive: 1 reduced state,
 *                        r = v px py (A + r'), to the older life's limiting age.
 *   RSV_LAST_SURVIVOR    A while at least one life is alive: the RSV_JL_REVERSIONARY
 *                        model with rho = 1 (the reversion field is ignored).
 *   RSV_JOINT_TERM       the sum at the end of the month of the first death
 *                        within the term: r = v ((1 - px py) S + px py r').
 *   RSV_JOINT_ENDOWMENT  RSV_JOINT_TERM plus the sum at maturity if both are alive.
 *   The nine-state two-life assurance model of Section 4.2.3 (each life
 *   alive / died in the step / dead) with the benefit on the second death,
 *   reduced to 3 states: both alive, only the first, only the second:
 *   RSV_LS_TERM          the sum at the end of the month of the second death
 *                        within the term: rx = v (qx S + px rx'), likewise ry,
 *                        r00 = v (qx qy S + px qy rx' + qx py ry' + px py r00').
 *   RSV_LS_ENDOWMENT     RSV_LS_TERM plus the sum at maturity if either is alive.
 *
 * Conventions shared by every entry point:
 *  - Status codes only; no C++ exception crosses the ABI.  On failure the
 *    context keeps a message, read with rsv_last_error().
 *  - Every rsv_load_* copies its input: the caller may free it on return.
 *  - Output buffers are owned and sized by the caller.
 *  - A context is used by one host thread at a time.
 *  - Ages are whole months; one projection step is one month; table entry k
 *    is the probability of surviving one month from age k months.  Ages at or
 *    beyond a table's length have survival probability 0 (the limiting age,
 *    Sections 4.1.1 and 4.2.1).
 *  - The paper's assumptions (Section 3.7) are checked and reported as
 *    RSV_E_ASSUMPTION: survival probabilities in [0, 1], discount factors
 *    finite and > 0, reversion in [0, 1], scenarios at least as long as every
 *    projection, finite amounts.
 */
#ifndef RSV_H
#define RSV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rsv_ctx rsv_ctx;

typedef enum {
    RSV_OK = 0,
    RSV_E_ARG = -1,        /* bad argument, size or pointer                          */
    RSV_E_NOMEM = -2,      /* device or host allocation failed                       */
    RSV_E_CUDA = -3,       /* a CUDA call failed (message in rsv_last_error)         */
    RSV_E_STATE = -4,      /* call order: e.g. compute before the data is loaded     */
    RSV_E_TIMEOUT = -5,    /* a bounded device-side wait ran out                      */
    RSV_E_ASSUMPTION = -6, /* input breaks an assumption of Section 3.7              */
    RSV_E_LIMIT = -7       /* sizes beyond the fixed scratch of rsv_reserves_noalloc  */
} rsv_status;

enum {
    RSV_SL_ANNUITY = 0, RSV_JL_REVERSIONARY = 1, RSV_TERM_ASSURANCE = 2, RSV_ENDOWMENT = 3,
    RSV_JOINT_ANNUITY = 4, RSV_LAST_SURVIVOR = 5, RSV_JOINT_TERM = 6, RSV_JOINT_ENDOWMENT = 7,
    RSV_LS_TERM = 8, RSV_LS_ENDOWMENT = 9
};

/* Arithmetic of the recurrence. */
enum {
    RSV_FORM_F64 = 0,      /* plain FP64 on the GPU                                  */
    RSV_FORM_F32 = 1,      /* plain FP32                                              */
    RSV_FORM_F32_COMP = 2, /* FP32 with compensated (double-float) accumulation and
                              hi/lo-split inputs                                      */
    RSV_FORM_F32_DEFLATED = 3 /* the recurrence in deflated units, compensated FP32:
                              see below                                               */
};

/* RSV_FORM_F32_DEFLATED.  Eq. (generalForm) multiplied at step t by the
 * deflator G_t = D_t l_{x+t} / l_x (D_t = v_0 ... v_{t-1}, the discount-factor
 * product to the start of step t; l the life table {l_{x+t}} of Section 5)
 * becomes U_t = U_{t+1} + G_{t+1} c_t with U = G r: the same backward
 * substitution (Section 3.8.2) whose multiplicative factor is 1 at every
 * step, and r_0 = U_0.  The discount products D are FP64 running products, one
 * per scenario, computed on the device in every call; the life tables are
 * built once in FP64 on the host; each chain-step is one FP32 fused
 * multiply-add, summed in FP32 over 8 steps and folded into a double-float
 * every 16 steps (or every 32, the two spans' sums first added in FP32).
 * Every reserve is within about 15 x 2^-24 (8.9e-7) relative of its value on
 * the FP64 inputs, whatever the projection length.  Products
 * RSV_SL_ANNUITY .. RSV_LAST_SURVIVOR (the reversionary and last-survivor
 * annuities through the reversionary identity of Section 4.2.1, every
 * valuation state); outputs RSV_OUT_V0 and RSV_OUT_SCEN_TOTAL; payment at the
 * end of the step; level cash flows.  Other requests return RSV_E_ARG (a
 * product, output or payment it does not take; tables whose survival falls
 * below 2^-220 or that need more shared memory than the device has) or
 * RSV_E_STATE (a cash-flow sequence loaded). */

/* rsv_opts.outputs bits */
enum {
    RSV_OUT_V0 = 1,         /* reserve at valuation of every policy x scenario        */
    RSV_OUT_SCEN_TOTAL = 2, /* per-scenario portfolio total, FP64, fixed summation order */
    RSV_OUT_PT_MEAN = 4,    /* per-(policy, step) mean over scenarios, FP64            */
    RSV_OUT_TRAJ = 8        /* full trajectory r_t of every chain (small runs only)    */
};

/* One policy record (48 bytes). */
typedef struct {
    int32_t product;   /* RSV_SL_ANNUITY .. RSV_LS_ENDOWMENT                           */
    int32_t age1_m;    /* age of the (first) life at valuation, whole months >= 0      */
    int32_t age2_m;    /* age of the second life; two-life products only               */
    int32_t term_m;    /* term in months; 0 = whole life (annuities only); assurances
                          and endowments need term_m >= 0                              */
    int32_t state0;    /* reduced state at valuation: 0 for every product; the JL,
                          last-survivor and second-death products also accept 1
                          (only the first life alive) and 2 (only the second)          */
    int32_t table1;    /* decrement table of the first life                            */
    int32_t table2;    /* decrement table of the second life (two-life products)       */
    int32_t reserved;  /* must be 0                                                    */
    double amount;     /* annuity amount per monthly step, or sum assured              */
    double reversion;  /* rho in [0, 1]; RSV_JL_REVERSIONARY only                      */
} rsv_policy;

/* rsv_opts.payment: the fraction f of Eq. generalForm at which annuity cash
 * flows are paid within each monthly step,
 *     r_t = v_t^f W_{t,f} c_t + v_t W_{t,1} r_{t+1}.
 * RSV_PAY_END: f = 1 (in arrears).  RSV_PAY_START: f = 0 (in advance,
 * W_{t,0} = I).  RSV_PAY_FRACTION: 0 < f < 1, with the survival over the first
 * fraction of each month from rsv_load_decrements_fraction (every loaded table
 * needs one, of the same length) and the discount over it from
 * rsv_load_scenarios_fraction (the loaded scenario set's shape).  Assurance
 * benefits stay at the end of the month of death (Section 4.1.3 restricts
 * them to f = 1).  The scenario-parallel kernels only; V0 and the totals,
 * not the per-step outputs. */
enum { RSV_PAY_END = 0, RSV_PAY_START = 1, RSV_PAY_FRACTION = 2 };

/* rsv_opts.variant: the backward recurrence as a parallel-in-time scan.  Each
 * step of Eq. generalForm is an affine map of the next step's reserve vector;
 * one warp takes one chain (policy x scenario), its lanes compose the maps of
 * 32 blocks of steps, and a warp suffix scan composes the blocks.  For few
 * scenarios (a flat rate) or very long projections, where the scenario-
 * parallel kernels leave lanes idle.  FP64 form only; outputs V0, the
 * per-scenario totals and the trajectory (not per-step means). */
#define RSV_VARIANT_TIME_SCAN (-2)

/* rsv_opts.variant: the reserves by their summation definition
 * (Eq. basicReserveSummation, Section 3.8.1), O(S^2) per chain: one thread per
 * step t sums the discounted, matrix-weighted cash flows of steps t .. S-1.
 * For measuring the summation against the recurrence; its results equal the
 * recurrence's to rounding.  FP64 form only; outputs V0, the per-scenario
 * totals and the trajectory (not per-step means). */
#define RSV_VARIANT_SUMMATION (-3)

typedef struct {
    int32_t form;      /* RSV_FORM_*                                                   */
    int32_t outputs;   /* RSV_OUT_* bits                                               */
    int32_t horizon;   /* > 0: truncate every projection at this many steps with
                          r_horizon = 0 (later cash flows dropped); 0 = none           */
    int32_t on_device; /* 1: output pointers are device pointers and the call is
                          asynchronous on the context stream; 0: host pointers, the
                          call blocks until the results are in host memory (in the
                          deflated form a page-locked, device-mapped V0 is written
                          by the kernel itself, any other is staged and copied)      */
    int32_t variant;   /* kernel variant index, -1 = the tuned/default one (see
                          rsv_variant_count / rsv_tune), RSV_VARIANT_TIME_SCAN or
                          RSV_VARIANT_SUMMATION                                        */
    int32_t payment;   /* RSV_PAY_*: when in each step the annuity cash flows are
                          paid (0 = at the end, the default)                           */
    int32_t reserved[2];
} rsv_opts;

/* Outputs of rsv_compute_reserves.  Any pointer may be NULL when its bit is
 * clear.  Layouts (n = portfolio size, S = n_scen, T = n_steps):
 *   V0 / V0d     [n][S]        float / double; the reserve in the policy's
 *                              valuation state; either or both may be given
 *   scen_total   [S]           double; sum of V0 over the portfolio
 *   pt_mean      [n][T + 1]    double; mean over scenarios of r_t in state0,
 *                              t = 0..T (entries past a policy's term are its
 *                              boundary value or 0)
 *   traj         [n][T + 1][S] double; r_t in state0 of every chain
 */
typedef struct {
    float *V0;
    double *V0d;
    double *scen_total;
    double *pt_mean;
    double *traj;
} rsv_out;

/* Create a context on CUDA device `device`, issuing work on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream).  The stream is not owned.
 * Errors: RSV_E_ARG (out NULL), RSV_E_CUDA (device unusable). */
rsv_status rsv_create(rsv_ctx **out, int device, void *cuda_stream);

/* Release every device buffer of the context and the context itself.
 * Synchronizes the context stream first.  NULL is accepted. */
rsv_status rsv_destroy(rsv_ctx *ctx);

/* Change the stream later calls are issued on (not owned). */
rsv_status rsv_set_stream(rsv_ctx *ctx, void *cuda_stream);

/* Load decrement table `table_id` (0 <= id < 8): p_monthly[k] = probability
 * of surviving one month from age k months, k = 0..n_ages_m-1 (host FP64,
 * copied).  Survival is 0 from age n_ages_m on.  These are the one-step
 * survival probabilities that populate W_{x,t,1} (Sections 3.5, 4).
 * Errors: RSV_E_ARG (bad id, NULL, n_ages_m < 1 or > 4096),
 * RSV_E_ASSUMPTION (an entry outside [0, 1] or not finite, Section 3.7.3). */
rsv_status rsv_load_decrements(rsv_ctx *ctx, int32_t table_id, const double *p_monthly,
                               int32_t n_ages_m);

/* Survival over the first fraction f of each month of table `table_id`:
 * p_f[k] = probability of surviving from age k months to k + f months (host
 * FP64, copied), for RSV_PAY_FRACTION (it populates W_{x,t,f}).  Survival is 0
 * from age n_ages_m on.
 * Errors: RSV_E_ARG (bad id, NULL, n_ages_m < 1 or > 4096),
 * RSV_E_ASSUMPTION (an entry outside [0, 1] or not finite). */
rsv_status rsv_load_decrements_fraction(rsv_ctx *ctx, int32_t table_id, const double *p_f, int32_t n_ages_m);

/* Discount factors over the first fraction f of each step, v_f[s,t] = v_{s,t}^f
 * in Eq. generalForm, for RSV_PAY_FRACTION; layout as rsv_load_scenarios
 * (host FP64, copied).
 * Errors: RSV_E_ARG (NULL, n_scen < 1, n_steps < 1, bad layout),
 * RSV_E_ASSUMPTION (a factor not finite or <= 0). */
rsv_status rsv_load_scenarios_fraction(rsv_ctx *ctx, const double *v_f, int32_t n_scen, int32_t n_steps,
                                       int32_t layout);

/* ---- Varying cash flows ---------------------------------------------------
 * Section 4.1.1: level, increasing, escalating and limited-term annuities
 * differ only in the cash-flow sequence c_t; Section 4.6: with monthly steps
 * the sequence carries the timing and the escalation (for annual payments,
 * one non-zero step in twelve).  A loaded sequence gives, per policy and step
 * t from valuation, the multiplier cf_t of the product's nominal cash-flow
 * vector c (amount, or amount x (1, 1, rho) for the reversionary annuity):
 * c_t = cf_t c.  It scales annuity payments and assurance death benefits; an
 * endowment's maturity sum stays the amount.  Once loaded it applies to every
 * rsv_compute_reserves call (which then runs the general-cash-flow kernels:
 * unshifted states, V0 and totals; per-step outputs through the time-scan and
 * summation variants) until rsv_clear_cashflows.  Nested runs value level
 * cash flows only (RSV_E_STATE while a sequence is loaded), as do the
 * context-free rsv_reserves_noalloc and the surrogate.  The rows are
 * indexed like the loaded portfolio: a
 * compute with another number of policies, or a projection longer than the
 * rows, fails with RSV_E_STATE. */

/* cf[p * n_steps + t] (host FP64, copied), p < n_pol, t < n_steps.
 * Errors: RSV_E_ARG (NULL, n_pol < 1, n_steps < 1, more than 2^31 entries),
 * RSV_E_ASSUMPTION (an entry negative or not finite), RSV_E_NOMEM, RSV_E_CUDA. */
rsv_status rsv_load_cashflows(rsv_ctx *ctx, const double *cf, int64_t n_pol, int32_t n_steps);

/* A payment schedule (32 bytes): payments every `every` steps from step
 * `first`; the level in force during step t raised at each policy
 * anniversary, n_t = floor((t + since) / steps_per_year) anniversaries after
 * valuation, by the factor 1 + escalation (geometric progression, an
 * escalating annuity) and by increase x the initial level (arithmetic
 * progression, an increasing annuity):
 *   cf_t = [t >= first, (t - first) mod every = 0] (1 + increase n_t) (1 + escalation)^n_t.
 * A level monthly annuity is {1, 0, 0, 12, 0, 0}; annual payments at the end
 * of each policy year with 3% escalation {12, 11, 0, 12, 0.03, 0}. */
typedef struct {
    int32_t every;          /* >= 1: steps between payments                     */
    int32_t first;          /* >= 0: step of the first payment                  */
    int32_t since;          /* 0 .. steps_per_year-1: steps since the last anniversary */
    int32_t steps_per_year; /* >= 1 (12 for monthly steps)                      */
    double escalation;      /* > -1, finite                                     */
    double increase;        /* >= 0, finite                                     */
} rsv_schedule;

/* Expand one schedule per policy into cash-flow multipliers on the device
 * (FP64), rows of n_steps as rsv_load_cashflows.
 * Errors: RSV_E_ARG (NULL, n_pol < 1, n_steps < 1, more than 2^31 entries, a
 * parameter outside the ranges above), RSV_E_NOMEM, RSV_E_CUDA. */
rsv_status rsv_load_schedules(rsv_ctx *ctx, const rsv_schedule *sch, int64_t n_pol, int32_t n_steps);

/* Back to level cash flows (cf_t = 1). */
rsv_status rsv_clear_cashflows(rsv_ctx *ctx);

/* Load the portfolio: n records (host, copied).  Validation of the records
 * against the tables happens at compute time.
 * Errors: RSV_E_ARG (NULL with n > 0, n < 0, n > 2^31 - 1). */
rsv_status rsv_load_portfolio(rsv_ctx *ctx, const rsv_policy *pols, int64_t n);

/* Load a scenario set: v = per-step discount factors (host FP64, copied),
 * v_{s,t} = exp(-integral of the force of interest over step t) in scenario s
 * (Section 3.4).  layout 0: v[s * n_steps + t]; layout 1: v[t * n_scen + s].
 * The same sequence discounts every policy valued under scenario s.
 * Errors: RSV_E_ARG (NULL, n_scen < 1, n_steps < 1, bad layout),
 * RSV_E_ASSUMPTION (a factor not finite or <= 0, Section 3.7.2). */
rsv_status rsv_load_scenarios(rsv_ctx *ctx, const double *v, int32_t n_scen, int32_t n_steps,
                              int32_t layout);

/* Reserves of every policy x scenario by backward substitution of Eq.
 * (generalForm), f = 1, from r_S = 0 (annuities, term assurances) or
 * r_S = (amount) (endowments at maturity), where S is the policy's number of
 * steps: to the limiting age for whole-life annuities (to the younger life's
 * for the JL product), the term otherwise, capped by opts->horizon.
 * Errors: RSV_E_STATE (tables, portfolio or scenarios missing), RSV_E_ARG
 * (bad opts, a NULL output whose bit is set, a trajectory request above 1 GiB,
 * a record with a bad product, table id or state, or whose ages plus steps
 * exceed 4096), RSV_E_ASSUMPTION (reversion outside [0, 1], amount not
 * finite, a projection longer than n_steps), RSV_E_CUDA, RSV_E_NOMEM. */
rsv_status rsv_compute_reserves(rsv_ctx *ctx, const rsv_opts *opts, rsv_out *out);

/* ---- m lives (Section 4.3) -------------------------------------------------
 * Contracts on m = 1..4 independent lives.  The paper builds their transition
 * matrices by induction, W^m = W^{m-1} (x) w_m, from the single-life two-state
 * matrix (annuities) or three-state matrix (assurances).  The library keeps
 * the reduced state "which lives are dead" (2^m states; the three-state
 * model's "died in the step" states only carry the benefit of that step) and
 * applies W^m as m one-life passes of the Kronecker factors, m 2^(m-1)
 * multiply-add pairs per step instead of a dense (2^m)^2 matrix product.
 *   RSV_MLIFE_ANNUITY    the amount at the end of every month in which at
 *                        least k of the m lives are alive (k = m: joint life,
 *                        k = 1: last survivor), to the limiting age of the
 *                        k-th longest-lived table or the term.
 *   RSV_MLIFE_ASSURANCE  the amount at the end of the month of the k-th death
 *                        within the term (term_m >= 1). */
enum { RSV_MLIFE_ANNUITY = 0, RSV_MLIFE_ASSURANCE = 1 };

typedef struct {     /* 64 bytes */
    int32_t m;        /* 1..4 lives                                                    */
    int32_t kind;     /* RSV_MLIFE_ANNUITY or RSV_MLIFE_ASSURANCE                      */
    int32_t k;        /* 1..m                                                          */
    int32_t term_m;   /* months; 0 = whole life (annuities only)                       */
    int32_t age_m[4]; /* ages at valuation in whole months (lives 1..m)                 */
    int32_t table[4]; /* decrement table of each life                                  */
    int32_t dead0;    /* lives already dead at valuation: bit i = life i+1; fewer than
                         k dead for an assurance, at least k alive for an annuity      */
    int32_t reserved; /* must be 0                                                     */
    double amount;
} rsv_mlife_policy;

/* Reserves of n m-life policies under the loaded scenarios (f = 1, level
 * amounts; the loaded cash-flow sequences do not apply), with the decrement
 * tables loaded by rsv_load_decrements.  opts: form (any), outputs RSV_OUT_V0
 * and/or RSV_OUT_SCEN_TOTAL, on_device; horizon, payment and variant 0 / -1.
 * out->V0 / V0d: [n][n_scen]; out->scen_total: [n_scen], summed over the
 * policies in order.  The records are copied.
 * Errors: RSV_E_STATE (tables or scenarios missing), RSV_E_ARG (bad opts or
 * record, a table not loaded, ages plus steps above 4096), RSV_E_ASSUMPTION
 * (amount not finite, a projection longer than the scenarios), RSV_E_CUDA,
 * RSV_E_NOMEM. */
rsv_status rsv_compute_mlife(rsv_ctx *ctx, const rsv_mlife_policy *pols, int64_t n, const rsv_opts *opts,
                             rsv_out *out);

/* ---- Nested ("brute force") valuation -------------------------------------
 * Section 2 of the paper: at each future valuation node every policy is
 * valued under 1000 Monte Carlo scenarios, and the 99.5% liability is the
 * 5th largest of the 1000.  Outer Vasicek paths o start at r0; node n is at
 * month n * node_step_m of the outer path; inner paths (o, n, i) start from
 * the outer path's short rate at the node.  The liability of inner path i is
 *   L_{o,n,i} = sum_p amount_p sum_j pi_{p,n,j} r_{p,j}(node),
 * pi = probability of reduced state j at the node from the valuation state
 * (deterministic mortality), r = reserve at the node by the recurrence of
 * rsv_compute_reserves on the inner path's monthly discount factors.
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed, counter
 * (k, o, 0, 2 << 24) for outer path o and (k, i, n, (3 << 24) | o) for inner
 * path i of node n, words 0,1 -> step 2k and 2,3 -> step 2k+1 as uniforms
 * (w + 1/2) 2^-32, Box-Muller; exact monthly Vasicek steps of (r, integral
 * of r), v = exp(-integral of r), all in FP64. */
enum {
    RSV_NESTED_MC = 0,        /* inner Monte Carlo ("brute force")                       */
    RSV_NESTED_SURROGATE = 1, /* inner expectation by the trained surrogate network, with
                                 the recurrence on the forward curve for flagged buckets
                                 (needs rsv_surrogate_train with the same a, b, sigma)  */
    RSV_NESTED_CURVE = 2      /* inner expectation in closed form: the recurrence on the
                                 Vasicek forward curve P(t+1|r)/P(t|r) (one chain each)   */
};

typedef struct {
    int32_t n_outer;      /* outer paths, >= 1                                         */
    int32_t n_nodes;      /* valuation nodes (months 0, node_step_m, ...), >= 1        */
    int32_t node_step_m;  /* months between nodes, >= 1                                */
    int32_t n_inner;      /* inner paths per (outer path, node), 1 .. 1048576           */
    uint64_t seed;        /* Philox key                                                */
    double a, b, sigma;   /* Vasicek dr = a (b - r) dt + sigma dW; a > 0, sigma >= 0    */
    double r0;            /* short rate at month 0                                     */
    int32_t mode;         /* RSV_NESTED_MC or RSV_NESTED_CURVE                         */
    int32_t batch_outer;  /* outer paths per inner-path batch; 0 = fit 4 GiB           */
    int32_t outer_first;  /* global index of the first outer path: the call values the
                             paths outer_first .. outer_first + n_outer - 1, whose random
                             streams are keyed by that index (below 2^24), so that the
                             outer paths can be split across calls or GPUs with no
                             exchange; the outputs are indexed from 0                    */
} rsv_nested_spec;

/* Outputs (caller-sized; host or device pointers per rsv_opts.on_device):
 *   L_mean [n_outer][n_nodes]  mean over inner paths of L_{o,n,i}
 *   L_q995 [n_outer][n_nodes]  k-th largest of the n_inner values, k =
 *                              ceil(0.005 n_inner) (5th of 1000); with
 *                              RSV_NESTED_CURVE both equal the curve value
 *   r_node [n_outer][n_nodes]  outer short rate at the node (optional)
 *   D0     [n_outer][n_nodes]  outer discount product month 0 -> node (optional)
 *   L_all  [n_outer][n_nodes][n_inner] every L_{o,n,i} (optional; n_inner = 1
 *                              with RSV_NESTED_CURVE and RSV_NESTED_SURROGATE)
 * Values are at the node (not discounted to 0). */
typedef struct {
    double *L_mean, *L_q995, *r_node, *D0, *L_all;
    int64_t *n_fallback;  /* optional, host: queries the surrogate mode valued by the
                             recurrence (its network valued the rest)                  */
} rsv_nested_out;

/* Nested valuation of the loaded portfolio (tables and portfolio needed, no
 * scenario set).  opts->form selects the arithmetic, opts->outputs and
 * opts->horizon must be 0.  With RSV_FORM_F32_DEFLATED the brute-force mode
 * runs in deflated units (products 0-5): each inner path's deflators are the
 * FP64 running products of its discount factors from the node, and
 * L_{o,n,i} = sum_p scale_p sum_{t >= m} D_i(m, t+1) E_p(t) with the policies'
 * expected cash flows E_p of rsv_compute_reserves' deflated form (the in-force
 * weighting at the node is part of them); the curve and surrogate modes then
 * run compensated.  Blocking unless opts->on_device.
 * Errors: RSV_E_STATE, RSV_E_ARG (bad spec, NULL L_mean/L_q995, a record as
 * in rsv_compute_reserves), RSV_E_ASSUMPTION, RSV_E_CUDA, RSV_E_NOMEM. */
rsv_status rsv_compute_nested(rsv_ctx *ctx, const rsv_opts *opts, const rsv_nested_spec *spec,
                              rsv_nested_out *out);

/* ---- Valuation without allocation ------------------------------------------
 * (The paper has no counterpart: this serves a kind of caller, not a step of
 * the method.)
 *
 * For callers that cannot allocate device memory: a serving process whose
 * device memory belongs to another allocator (a fixed arena or pool that must
 * remain its only owner), or latency-bound code that cannot take the
 * device-wide synchronisation a cudaMalloc may imply.  Every input and output
 * is the caller's device memory; the call allocates nothing (no cudaMalloc,
 * no cudaFree, no allocating library routine) and uses no context.
 *
 * Computes what rsv_compute_reserves computes with RSV_FORM_F32_COMP,
 * outputs V0d and scen_total, one decrement table: the reserve at valuation of
 * every policy under every scenario, V0[p * n_scen + s] (FP64), and the
 * per-scenario totals over the portfolio (FP64, fixed summation order).
 *   pols       [n_pol] records (device), table1 (and table2) must be 0
 *   p_monthly  [n_ages] one-month survival by age in months (device), 1..4096
 *   v          [n_steps][n_scen] discount factors, step-major (device)
 *   V0         [n_pol][n_scen] output (device); scen_total [n_scen] (device,
 *              optional, NULL to skip)
 * Working memory is one static 32 MiB device array in the library, held by
 * every GPU that loads it until the process exits.  A call needs
 * 256 B + 64 KiB + n_steps x s_pad x 8 + n_pol x 44 + ceil(n_pol / 256) x
 * n_scen x 8 bytes of it (s_pad = n_scen rounded up to 128, each term rounded
 * up to 256 B); larger calls return RSV_E_LIMIT before any GPU work (100,000
 * policies x 1,000 scenarios x 1,200 steps needs 17.4 MB).
 * The first call on a device looks up the array's device address (with that
 * device current) and keeps it.  Every call shares the array and leaves its
 * contents behind; each call re-initialises what it reads, but calls whose
 * GPU work overlaps (other streams or host threads) race on it: serialise
 * them.  The call is issued on `cuda_stream` (NULL = legacy default) and
 * blocks until its work is done (it reads its status back to the host), so it
 * cannot be issued inside a stream capture.
 * It takes the products RSV_SL_ANNUITY .. RSV_ENDOWMENT on decrement table 0.
 * Errors: RSV_E_ARG (NULL pointer, bad size, a record that breaks an argument
 * rule of the main entry point: product, table, age, term, state, reserved
 * field, age plus steps above 4096), RSV_E_LIMIT (sizes beyond the scratch,
 * refused before any GPU work), RSV_E_ASSUMPTION (a table entry outside
 * [0, 1], a discount factor not finite and positive, or a record with an
 * amount not finite, a reversion outside [0, 1] or more steps than the
 * scenarios; with several bad records, the status of the first in portfolio
 * order, as the main entry point reports), RSV_E_CUDA, RSV_E_TIMEOUT; on an
 * error the outputs are unspecified. */
rsv_status rsv_reserves_noalloc(int device, void *cuda_stream, const rsv_policy *pols, int32_t n_pol,
                                const double *p_monthly, int32_t n_ages, const double *v, int32_t n_scen,
                                int32_t n_steps, double *V0, double *scen_total);

/* ---- Surrogate network ------------------------------------------------------
 * The inner loop of the nested valuation (Section 2) estimates the expected
 * reserve of a policy in a reduced state at a node given the short rate there.
 * Under the Vasicek model with deterministic mortality that expectation is
 * exactly the recurrence (Eq. generalForm) on the forward curve
 * P(t+1|r)/P(t|r), because the reserve is linear in the discount products
 * (Eq. basicReserveSummation).  The surrogate is a perceptron
 * 32 -> 256 -> 256 -> 256 -> 256 -> 1 with GELU (tanh form), BF16 weights and
 * activations and FP32 accumulation on the tensor cores, FP32 master weights
 * and Adam; it predicts ln(reserve per unit amount) minus the ln of a
 * commutation-function base value, from 19 feature slots zero-padded to 32:
 * product one-hot (4), state one-hot (3), the two ages, the reversion, the
 * remaining term, the node rate, ln amount, age^2, term^2, rate x term,
 * ln(1 + remaining months), the ln base value and the flat yield it is taken
 * at.  The parameters are one flat
 * FP32 vector: W1 [32][256], b1 [256], W2 [256][256], b2, W3, b3, W4, b4
 * (each W row-major [in][out]), w5 [256], b5 [1]. */
int64_t rsv_mlp_param_count(void);

/* He-normal initialisation (seeded), or set / read all parameters (host
 * FP32, rsv_mlp_param_count() values).  Setting resets the Adam state. */
rsv_status rsv_mlp_init(rsv_ctx *ctx, uint64_t seed);
rsv_status rsv_mlp_set_params(rsv_ctx *ctx, const float *params, int64_t n);
rsv_status rsv_mlp_get_params(rsv_ctx *ctx, float *params, int64_t n);

/* Kernels that evaluate the network for inference (rsv_mlp_forward,
 * rsv_surrogate_query, the nested surrogate mode): RSV_MLP_TCGEN05 (default)
 * runs all layers and the head in one kernel on the tcgen05 tensor cores with
 * TMEM accumulators; RSV_MLP_MMA_SYNC runs the per-layer mma.sync kernels the
 * training uses.  Both compute the same network in BF16 with FP32
 * accumulation. */
enum { RSV_MLP_MMA_SYNC = 0, RSV_MLP_TCGEN05 = 1 };
rsv_status rsv_mlp_set_backend(rsv_ctx *ctx, int32_t backend);

/* Network output for n rows of 32 host FP32 features (rounded to BF16 on the
 * way in), 1 <= n <= 2^20; y (host) receives n outputs.  The device time of
 * the network's kernels (not the copies) is available from rsv_last_kernel_ms. */
rsv_status rsv_mlp_forward(rsv_ctx *ctx, const float *X, int64_t n, float *y);

/* Gradient of the mean squared error (1/n) sum (y - target)^2 over n rows
 * (n a multiple of 64, <= 2^20), in the flat parameter layout (host); loss
 * receives the mean squared error.  Uses the network's current parameters. */
rsv_status rsv_mlp_gradient(rsv_ctx *ctx, const float *X, const float *target, int64_t n, float *grads,
                            float *loss);

/* Test entry point (the paper has no counterpart): one pass of the network on
 * n rows of 32 host FP32 features (n a multiple of 128, at most 4096) with
 * every layer's values, so that each layer can be checked on its own against
 * a reference fed the same inputs.  All outputs are host buffers owned by the
 * caller.  Xb [n][64]: the BF16 bits of the features as the first layer reads
 * them (hi halves, then lo halves; may be NULL).  y [n]: the outputs.
 * backend RSV_MLP_MMA_SYNC (the training kernels): Z [4][n][256] the FP32
 * pre-activations z_l = A_{l-1} W_l + b_l, A [4][n][256] the BF16 bits of
 * gelu(z_l) as stored for the next product (the head reads layer 4 in FP32);
 * with a target [n] also the backward pass of the mean squared error:
 * dZ [4][n][256] the FP32 gradients with respect to z_l, dZb the BF16 bits the
 * products read, grads [rsv_mlp_param_count()] the parameter gradients.
 * backend RSV_MLP_TCGEN05 (the inference kernel): Z as above and in A the
 * first three layers' BF16 operands as the kernel stores them in tensor
 * memory, 2 gelu(z_l) (its next layer's weights are staged halved); target,
 * dZ, dZb and grads must be NULL.  Blocks until done.
 * Errors: RSV_E_ARG, RSV_E_STATE (no network), RSV_E_CUDA, RSV_E_TIMEOUT. */
rsv_status rsv_mlp_trace(rsv_ctx *ctx, int32_t backend, const float *X, const float *target, int64_t n,
                         uint16_t *Xb, float *Z, uint16_t *A, float *y, float *dZ, uint16_t *dZb, float *grads);

typedef struct {
    int64_t n_train;     /* labelled training queries (>= 1024)                       */
    int64_t n_val;       /* held-out queries scored against the recurrence (>= 1024)  */
    int32_t epochs;      /* passes of n_train / batch random batches                  */
    int32_t batch;       /* multiple of 64, <= 65536                                  */
    double lr;           /* Adam peak learning rate (cosine decay to 2%)              */
    uint64_t seed;       /* query sampling (Philox streams 6, 7), batches, init       */
    double a, b, sigma, r0;  /* Vasicek model of the node rates and of the labels     */
    int32_t max_node_m;  /* nodes sampled at months 0, 12, ... up to this              */
    double widen;        /* node rates drawn from the model's distribution, sd x widen */
    double tol;          /* relative error the network may serve                    */
    double margin;       /* (0, 1]: a bucket is served only if its calibration
                            maximum error is below margin x tol                    */
} rsv_surrogate_cfg;

typedef struct {
    double train_loss;                  /* last batch mean squared error (normalised) */
    double val_max_rel, val_p99_rel, val_median_rel, val_rms_rel;  /* held out     */
    double frac_fallback;               /* held-out share valued by the recurrence  */
    double combined_max_rel;            /* max error of what the network serves     */
    double label_ms, train_ms, infer_ms;/* device times: labels, training, scoring  */
    int64_t n_label, n_infer, n_buckets, n_flagged;
    double y_mean, y_std;               /* target normalisation                     */
} rsv_surrogate_report;

/* Train the surrogate on the loaded portfolio (decrement tables and policies
 * needed): sample n_train + n_val queries (a policy, an annual node before its
 * end, a reduced state its lives can be in, a rate from the model at that
 * month), label them with the FP64 recurrence on the forward curve, train,
 * and score the held-out queries.  Buckets (product and state x age x
 * remaining term x the node rate's z-score under the model) whose error on
 * the first half of the held-out queries exceeds margin x tol, or that hold
 * fewer than 32 of them, are flagged, as are rates beyond 4 standard
 * deviations; the second half measures the error of what the network then
 * serves.  The
 * network is (re)used as initialised if rsv_mlp_init / set_params was called.
 * Errors: RSV_E_ARG, RSV_E_STATE, RSV_E_CUDA, RSV_E_NOMEM. */
rsv_status rsv_surrogate_train(rsv_ctx *ctx, const rsv_surrogate_cfg *cfg, rsv_surrogate_report *report);

/* Write the trained surrogate to a file: the network parameters (FP32), the
 * target normalisation, the fallback map, the tolerance and the Vasicek
 * parameters of its training, with a 64-bit FNV-1a checksum.  Host byte
 * order.  The features refer to the loaded decrement tables and portfolio, so
 * a loaded surrogate is meant for the same tables and policy records.
 * Errors: RSV_E_ARG (NULL path, the file cannot be written), RSV_E_STATE (not
 * trained), RSV_E_CUDA. */
rsv_status rsv_surrogate_save(rsv_ctx *ctx, const char *path);

/* Read a file written by rsv_surrogate_save; the surrogate is then trained.
 * Errors: RSV_E_ARG (NULL path, unreadable file, wrong magic, size, shape or
 * checksum), RSV_E_NOMEM, RSV_E_CUDA. */
rsv_status rsv_surrogate_load(rsv_ctx *ctx, const char *path);

/* A valuation query: policy index (into the loaded portfolio), node month m
 * (0 <= m < the policy's steps), reduced state (0; JL also 1, 2) and the
 * short rate at the node. */
typedef struct {
    int32_t pol, m, state, reserved;
    double r;
} rsv_query;

enum {
    RSV_QUERY_NETWORK = 0,     /* the trained network alone                              */
    RSV_QUERY_RECURRENCE = 1,  /* the FP64 recurrence on the forward curve (the label)    */
    RSV_QUERY_FALLBACK = 2     /* the network, with flagged buckets by the recurrence     */
};

/* Expected reserve (amount x per-unit value) of n host queries into reserve
 * (host FP64, n values).  RSV_QUERY_RECURRENCE needs no trained network; the
 * Vasicek parameters are those of the last rsv_surrogate_train (defaults
 * a = 0.1, b = 0.04, sigma = 0.01 before any).  The device time of the
 * evaluation is available from rsv_last_kernel_ms.
 * Errors: RSV_E_ARG (a bad query), RSV_E_STATE (no portfolio; no trained
 * network for the network modes), RSV_E_CUDA, RSV_E_NOMEM. */
rsv_status rsv_surrogate_query(rsv_ctx *ctx, const rsv_query *queries, int64_t n, int32_t how, double *reserve);

/* Self-test of the bounded device-side wait that every kernel's bulk-copy
 * staging of the decrement tables relies on (failure detection without a GPU
 * fault): one CTA stages 16 KiB into shared memory with the same bulk-copy and
 * mbarrier primitives.  never_completes = 0: a normal staging; RSV_OK if the
 * bytes round-trip.  never_completes = 1: the barrier is told to expect 16
 * bytes more than are copied, so its phase cannot complete; the bounded wait
 * runs out (65,536 polls), the kernel records the timeout, lets its copies
 * land and returns, and the call returns RSV_E_TIMEOUT with the device and any
 * context on it still usable.  Blocks until done.
 * Errors: RSV_E_TIMEOUT (as described), RSV_E_NOMEM, RSV_E_CUDA. */
rsv_status rsv_selftest_bounded_wait(int32_t device, void *cuda_stream, int32_t never_completes);

/* The nested valuation's inner-path generator evaluates its FP64 functions by
 * its own table-driven methods (Tang's logarithm; sine and cosine from a
 * 1,024-entry table and the addition theorems; a series for e^x with
 * |x| < 1/16, exp() beyond).  This entry point runs those device functions on
 * given draws so that tests can compare them with a reference library: for
 * i < n, with u_i = (w[i] + 1/2) 2^-32, out[4 i] = ln u_i,
 * out[4 i + 1] = sin(2 pi u_i), out[4 i + 2] = cos(2 pi u_i) and
 * out[4 i + 3] = e^{x[i]}.  w: n 32-bit draws, x: n doubles, out: 4 n doubles;
 * all host memory owned by the caller.  Blocks until done.
 * Errors: RSV_E_ARG (n < 0, or a null pointer with n > 0), RSV_E_NOMEM,
 * RSV_E_CUDA. */
rsv_status rsv_selftest_generator_math(int32_t device, void *cuda_stream, const uint32_t *w, const double *x,
                                       int64_t n, double *out);

/* Measured fused multiply-add throughput of `device` in TFLOP/s (2 flop per
 * FMA): FP32 (fp64 = 0) or FP64 (fp64 = 1), from a kernel of independent FMA
 * chains filling every SM, best of five timed launches on `cuda_stream`.  It
 * is the measured denominator of the ALU rooflines; the paper has no
 * counterpart.  Blocks until done.  Errors: RSV_E_ARG, RSV_E_CUDA, RSV_E_NOMEM. */
rsv_status rsv_probe_fma_peak(int32_t device, void *cuda_stream, int32_t fp64, double *tflops);

/* Kernel variants of a form (policies x scenarios per thread, CTA size; for
 * the deflated form also the arithmetic: scalar, packed FP32 pairs "x2", the
 * double-float sums in tensor memory "tm", and one fold per 32-step block
 * "tm2"): how many there are, and a printable description of one.  Variants
 * of one form give the same reserves within the form's bound; those that
 * differ only in shape (not in the summation order) give the same bits. */
int32_t rsv_variant_count(int32_t form);
const char *rsv_variant_name(int32_t form, int32_t variant);

/* Autotuner: time every variant of `form` on the loaded data (the same
 * outputs as `opts`), keep the fastest as the context's default for that
 * form and return its index in *best (may be NULL).  reps >= 1 timed runs
 * per variant after one warm-up run; best of reps is compared.
 * ms_out (optional) receives rsv_variant_count(form) times in ms; -1 for a
 * RSV_FORM_F32_DEFLATED variant whose staging does not fit in shared memory
 * beside the loaded tables (it is skipped; without a tuned variant the
 * deflated form falls back to the first that fits).
 * Errors: as rsv_compute_reserves. */
rsv_status rsv_tune(rsv_ctx *ctx, const rsv_opts *opts, int32_t reps, int32_t *best,
                    float *ms_out);

/* Wait for all work issued on the context stream; returns RSV_E_CUDA or
 * RSV_E_TIMEOUT if a kernel reported one. */
rsv_status rsv_synchronize(rsv_ctx *ctx);

/* Message of the last failed call on ctx (owned by ctx, valid until the next
 * call).  Never NULL. */
const char *rsv_last_error(const rsv_ctx *ctx);

/* Device time in ms of the last timed kernel work on ctx: the recurrence
 * kernel of rsv_compute_reserves, or the kernels named by the other calls that
 * say so (CUDA events on the context stream; valid after the call has
 * completed).  Returns -1 if unknown. */
float rsv_last_kernel_ms(rsv_ctx *ctx);

/* Number of streaming multiprocessors of the context's device. */
int32_t rsv_device_sm_count(const rsv_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* RSV_H */
