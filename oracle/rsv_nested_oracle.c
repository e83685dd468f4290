/*
 * rsv_nested_oracle.c -- FP64 CPU oracle of the nested ("brute force")
 * Solvency II valuation built on the reserve recurrence of Tucker & Bull
 * (arXiv 1401.1757, Section 2: 1000 Monte Carlo scenarios at each future
 * step, 99.5% liability = the 5th largest of 1000).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code with
 * the CUDA library; both sides implement the same published random-number
 * generator (Philox4x32-10, Salmon, Moraes, Dror and Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11) from its definition, so that the
 * scenarios can be regenerated here instead of being copied from the GPU.
 *
 * Definitions (all FP64):
 *  - Gaussian pairs: Philox4x32-10 of counter (k, c1, c2, c3) and key (seed
 *    low word, seed high word) gives four words; step 2k uses words 0 and 1,
 *    step 2k+1 words 2 and 3, as uniforms u = (w + 1/2) 2^-32 and the
 *    Box-Muller transform z1 = R cos(2 pi u2), z2 = R sin(2 pi u2),
 *    R = sqrt(-2 ln u1).
 *  - Vasicek short rate, exact joint step of (r, integral of r) over one month
 *    (Glasserman 2004, Sec. 3.3): with e = exp(-a dt),
 *      I  = b dt + (r - b)(1 - e)/a + l21 z1 + l22 z2
 *      r' = b + (r - b) e + l11 z1
 *    where (l11, 0; l21, l22) is the Cholesky factor of the covariance of
 *    (r', I); the step's discount factor is v = exp(-I).
 *  - Outer path o: counters (k, o, 0, 2 << 24), from r0 at month 0.
 *    Inner path i at node n of outer path o: counters (k, i, n, (3 << 24) | o),
 *    from the outer path's rate at the node's month.
 *  - Liability at node n, inner path i: L = sum over policies of
 *    sum_j pi_j r_j, where pi is the distribution of the full survival state
 *    at the node (Chapman-Kolmogorov over the one-step matrices, Eq.
 *    recRel_Probabilities, from the valuation state) times nothing else, and
 *    r_j is the reserve vector at the node by the recurrence on the inner
 *    path (orc_chain from the node: ages advanced, term shortened).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

int orc_n_states(int product);
int orc_transition(int product, double px, double py, double *W);
int orc_steps(int product, int age1, int age2, int term, int n_ages, int horizon, double amount, double *rS);
int orc_full_state(int product, int state0);
int orc_chain(int product, int age1, int age2, int term, double amount, double rho, int n_ages,
              const double *p1x, const double *p1y, const double *pfx, const double *pfy, int n_steps,
              const double *v, const double *vf, int horizon, int method, double *r_out);

/* ---- Philox4x32-10 ---------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t *ctr_in, const uint32_t *key_in, uint32_t *out)
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * c[0];
        uint64_t p1 = (uint64_t)PHILOX_M1 * c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    memcpy(out, c, sizeof c);
}

/* z[0..3]: the two Gaussian pairs of counter (k, c1, c2, c3). */
void orc_gauss_pair(uint64_t seed, uint32_t k, uint32_t c1, uint32_t c2, uint32_t c3, double *z)
{
    const uint32_t ctr[4] = {k, c1, c2, c3};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    const double two32 = 4294967296.0, pi = 3.14159265358979323846;
    for (int h = 0; h < 2; ++h) {
        double u1 = ((double)w[2 * h] + 0.5) / two32;
        double u2 = ((double)w[2 * h + 1] + 0.5) / two32;
        double R = sqrt(-2.0 * log(u1));
        z[2 * h] = R * cos(2.0 * pi * u2);
        z[2 * h + 1] = R * sin(2.0 * pi * u2);
    }
}

typedef struct { double e, k1, l11, l21, l22, b, dt; } vas_step;

static vas_step vasicek_constants(double a, double b, double sigma, double dt)
{
    vas_step s;
    double e = exp(-a * dt), one_m_e = -expm1(-a * dt), one_m_e2 = -expm1(-2.0 * a * dt);
    double var_r = sigma * sigma * one_m_e2 / (2.0 * a);
    double var_i = sigma * sigma / (a * a) * (dt - 2.0 * one_m_e / a + one_m_e2 / (2.0 * a));
    double cov = sigma * sigma / (2.0 * a * a) * one_m_e * one_m_e;
    s.e = e;
    s.k1 = one_m_e / a;
    s.l11 = sqrt(var_r);
    s.l21 = s.l11 > 0.0 ? cov / s.l11 : 0.0;   /* sigma = 0: deterministic rate */
    s.l22 = sqrt(fmax(var_i - s.l21 * s.l21, 0.0));
    s.b = b;
    s.dt = dt;
    return s;
}

/* n_steps monthly steps of one path from rate r_start; counters (k, c1, c2, c3).
 * v[t] = discount factor of step t; r_out (optional) = rate after n_steps. */
static void path(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3, const vas_step *s,
                 double r_start, int n_steps, double *v, double *r_out)
{
    double r = r_start, z[4];
    for (int t = 0; t < n_steps; ++t) {
        if ((t & 1) == 0) orc_gauss_pair(seed, (uint32_t)(t >> 1), c1, c2, c3, z);
        double z1 = z[(t & 1) * 2], z2 = z[(t & 1) * 2 + 1];
        double I = s->b * s->dt + (r - s->b) * s->k1 + s->l21 * z1 + s->l22 * z2;
        r = s->b + (r - s->b) * s->e + s->l11 * z1;
        if (v) v[t] = exp(-I);
    }
    if (r_out) *r_out = r;
}

/* One Vasicek path with counters (k, c1, c2, c3) from rate r_start, monthly
 * steps.  Public for the generator tests. */
void orc_vasicek_path(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3, double a, double b,
                      double sigma, double r_start, int n_steps, double *v, double *r_end)
{
    vas_step s = vasicek_constants(a, b, sigma, 1.0 / 12.0);
    path(seed, c1, c2, c3, &s, r_start, n_steps, v, r_end);
}

/* Liability L_{o,n,i} for the inner paths idx[0..n_idx) of node n (month
 * n * node_step) of outer path o, FP64.
 * ipol[n_pol][6] = (age1, age2, term, state0, table1, table2); dpol[n_pol][2]
 * = (amount, rho); tables [n_tables][n_ages].  L_out[k] receives the
 * liability of inner path idx[k]; r_node_out / d0_out (optional) the outer
 * path's rate at the node and its discount product from 0 to the node.
 * Returns 0 or a negative code. */
int orc_nested_node(int64_t n_pol, const int32_t *prod, const int32_t *ipol, const double *dpol,
                    int32_t n_tables, int32_t n_ages, const double *tables, uint64_t seed, double a,
                    double b, double sigma, double r0, int32_t node_step, int32_t o, int32_t n,
                    int32_t n_idx, const int32_t *idx, double *L_out, double *r_node_out, double *d0_out)
{
    vas_step s = vasicek_constants(a, b, sigma, 1.0 / 12.0);
    const int m = n * node_step;
    /* outer path to the node */
    double *vo = (double *)malloc(sizeof(double) * (m > 0 ? m : 1));
    double r_node;
    if (!vo) return -3;
    path(seed, (uint32_t)o, 0u, 2u << 24, &s, r0, m, vo, &r_node);
    double d0 = 1.0;
    for (int u = 0; u < m; ++u) d0 *= vo[u];
    free(vo);
    if (r_node_out) *r_node_out = r_node;
    if (d0_out) *d0_out = d0;

    /* longest remaining projection at the node */
    int Lmax = 0;
    for (int64_t p = 0; p < n_pol; ++p) {
        double rS[9];
        const int32_t *ip = ipol + 6 * p;
        int S = orc_steps(prod[p], ip[0], ip[1], ip[2], n_ages, 0, 1.0, rS);
        if (S - m > Lmax) Lmax = S - m;
    }
    double *vi = (double *)malloc(sizeof(double) * (Lmax > 0 ? Lmax : 1));
    double *r = (double *)malloc(sizeof(double) * 9 * ((size_t)Lmax + 2));
    if (!vi || !r) { free(vi); free(r); return -3; }
    for (int k = 0; k < n_idx; ++k) {
        path(seed, (uint32_t)idx[k], (uint32_t)n, (3u << 24) | (uint32_t)o, &s, r_node, Lmax, vi, NULL);
        double L = 0.0;
        for (int64_t p = 0; p < n_pol; ++p) {
            const int32_t *ip = ipol + 6 * p;
            const int product = prod[p], a1 = ip[0], a2 = ip[1], term = ip[2], st0 = ip[3];
            const int nst = orc_n_states(product);
            if (nst < 0 || ip[4] < 0 || ip[4] >= n_tables || ip[5] < 0 || ip[5] >= n_tables) {
                free(vi); free(r);
                return -1;
            }
            double rS[9];
            int S = orc_steps(product, a1, a2, term, n_ages, 0, 1.0, rS);
            if (S < m) continue;                                  /* ended before the node */
            const int annuity = product == 0 || product == 1 || product == 4 || product == 5;
            if (annuity && term > 0 && term <= m) continue;       /* limited-term annuity over */
            const double *tx = tables + (size_t)ip[4] * n_ages, *ty = tables + (size_t)ip[5] * n_ages;
            /* full-state distribution at the node: e_{state0} times the one-step matrices */
            double pi[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, nx[9], W[81];
            const int full = orc_full_state(product, st0);
            if (full < 0 || full >= nst) { free(vi); free(r); return -1; }
            pi[full] = 1.0;
            for (int u = 0; u < m; ++u) {
                double px = (a1 + u < n_ages) ? tx[a1 + u] : 0.0;
                double py = (a2 + u < n_ages) ? ty[a2 + u] : 0.0;
                orc_transition(product, px, py, W);
                for (int i = 0; i < nst; ++i) {
                    double acc = 0.0;
                    for (int j = 0; j < nst; ++j) acc += pi[j] * W[j * nst + i];
                    nx[i] = acc;
                }
                memcpy(pi, nx, sizeof(double) * nst);
            }
            int term_left = term > 0 ? term - m : 0;
            int Sn = orc_chain(product, a1 + m, a2 + m, term_left, dpol[2 * p], dpol[2 * p + 1], n_ages, tx, ty,
                               tx, ty, Lmax, vi, vi, 0, 0, r);
            if (Sn < 0) { free(vi); free(r); return Sn; }
            for (int j = 0; j < nst; ++j) L += pi[j] * r[j];
        }
        L_out[k] = L;
    }
    free(vi);
    free(r);
    return 0;
}
