/*
 * fs_oracle.c -- the CPU oracle (TEST INFRASTRUCTURE ONLY; see fs_oracle.h).
 *
 * Plain C11, single-threaded, double precision for every hazard and
 * probability, exact emulation of the storage rounding of ages. Each function
 * names the passage of FlashSpread (arXiv 2604.22092) it restates.
 *
 * Readings of the paper taken here (each is listed with its reason in the
 * design notes of the repository):
 *   - a fixed step dt in fso_step / fso_run; fso_run_adaptive takes the
 *     adaptive rule of Section 5.2 with lambda* the largest per-node rate of
 *     the previous step and dt_max at the first step;
 *   - the hazard is evaluated at the begin-of-step age (Algorithm 3);
 *   - ages of S and R nodes are held at 0; E/I ages advance by one float add
 *     of dt followed by round-to-nearest-even to the storage type (Section
 *     5.7, "promote on load, cast on store");
 *   - the infectivity is the indicator of state I with unit edge weights
 *     (Eq. 8 with s = 1), so the pressure of an S node is beta times the
 *     integer number of infectious in-neighbours (Eq. 3); with a shedding
 *     profile s(tau) (the hazard or the density of a law) the infectivity
 *     beta s(tau) of each I node is evaluated at its begin-of-step age,
 *     stored like an age (fp32, then the storage type), and the pressure is
 *     the double sum of the stored values;
 *   - the paper's Triton PRNG is replaced by Philox4x32-10 keyed by
 *     (seed, replicate, step, node);
 *   - the Markovian engine (Algorithm 1) takes its step size from the rates
 *     of the state the step starts from, Lambda collected by compartment
 *     (beta x S-I edges + sigma |E| + gamma |I|) in double, and SIS returns
 *     recovered nodes to S; its exact reference is a Doob-Gillespie direct
 *     method (fso_gillespie_run).
 */
#include "fs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from the description in Salmon et al., "Parallel  */
/* random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of the Philox    */
/* S-box-free bijection; each round multiplies counter words 0 and 2 by the */
/* two round multipliers (64-bit products split into hi/lo halves), xors    */
/* the high halves with the other two counter words and the round key, and  */
/* the key is bumped by the two Weyl constants between rounds.              */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void fso_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Replaces the paper's tl.rand(seed + step_id, node_id) (Appendix A,
 * Algorithm 3) with a counter-based draw keyed by (seed, rep, step, node). */
double fso_uniform(uint64_t seed, uint32_t rep, int64_t step, int64_t node)
{
    uint32_t ctr[4] = { (uint32_t)node, (uint32_t)step, rep >> 2, 0u };
    uint32_t key[2] = { (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) };
    uint32_t w[4];
    fso_philox4x32_10(ctr, key, w);
    return (double)(w[rep & 3u] >> 8) * (1.0 / 16777216.0);
}

/* ------------------------------------------------------------------------ */
/* Hazards (Section 5.1; Proposition 1 for the log-normal).                 */
/* ------------------------------------------------------------------------ */

/* erfcx(z) = exp(z^2) erfc(z). For z < 26 the definition is evaluated as   */
/* written (erfc(z) > 1 for z < 0, so there is no cancellation; exp(z^2)    */
/* overflows to +inf for z < -26.6, which sends the hazard to 0, the limit  */
/* stated in Appendix A). For z >= 26, where erfc underflows, the           */
/* asymptotic series 1/(z sqrt(pi)) sum_n (-1)^n (2n-1)!! / (2 z^2)^n of    */
/* Appendix A is summed to double precision (the paper stops at 4 terms).   */
double fso_erfcx(double z)
{
    if (z < 26.0)
        return exp(z * z) * erfc(z);
    double inv2z2 = 1.0 / (2.0 * z * z);
    double term = 1.0, sum = 1.0;
    for (int n = 1; n < 40; ++n) {
        term *= -(double)(2 * n - 1) * inv2z2;
        sum += term;
        if (fabs(term) < 1e-18 * fabs(sum))
            break;
    }
    return sum / (z * sqrt(M_PI));
}

double fso_hazard(const fso_law* law, double tau)
{
    switch (law->kind) {
    case FSO_LAW_NONE:
        return 0.0;
    case FSO_LAW_EXP:
        return law->a;
    case FSO_LAW_LOGNORMAL: {
        /* h = sqrt(2/pi) / (tau sigma erfcx(z)), z = (ln tau - mu)/(sigma sqrt 2) */
        double mu = law->a, sigma = law->b;
        if (!(tau > 0.0))
            return 0.0;
        double z = (log(tau) - mu) / (sigma * M_SQRT2);
        return sqrt(2.0 / M_PI) / (tau * sigma * fso_erfcx(z));
    }
    case FSO_LAW_WEIBULL: {
        /* h = (k/s) (tau/s)^(k-1) */
        double k = law->a, s = law->b;
        if (!(tau > 0.0))
            return (k == 1.0) ? 1.0 / s : 0.0;
        return (k / s) * pow(tau / s, k - 1.0);
    }
    case FSO_LAW_ERLANG: {
        /* h = r (r tau)^(k-1)/(k-1)! / sum_{n<k} (r tau)^n / n! */
        int k = law->k;
        double r = law->a, x = r * tau;
        double t = 1.0, sum = 1.0;
        for (int n = 1; n < k; ++n) {
            t *= x / (double)n;
            sum += t;
        }
        return r * t / sum;
    }
    default:
        return NAN;
    }
}

/* Densities f(tau) of the holding-time laws, written from their textbook
 * definitions (used as shedding profiles, Section 5.3). */
double fso_density(const fso_law* law, double tau)
{
    if (tau < 0.0)
        return 0.0;
    switch (law->kind) {
    case FSO_LAW_NONE:
        return 0.0;
    case FSO_LAW_EXP:
        return law->a * exp(-law->a * tau);
    case FSO_LAW_LOGNORMAL: {
        /* f = exp(-(ln tau - mu)^2 / (2 sigma^2)) / (tau sigma sqrt(2 pi)) */
        double mu = law->a, sigma = law->b;
        if (!(tau > 0.0))
            return 0.0;
        double y = (log(tau) - mu) / sigma;
        return exp(-0.5 * y * y) / (tau * sigma * sqrt(2.0 * M_PI));
    }
    case FSO_LAW_WEIBULL: {
        /* f = (k/s) (tau/s)^(k-1) exp(-(tau/s)^k) */
        double k = law->a, s = law->b, x = tau / s;
        return (k / s) * pow(x, k - 1.0) * exp(-pow(x, k));
    }
    case FSO_LAW_ERLANG: {
        /* f = r^k tau^(k-1) exp(-r tau) / (k-1)! */
        int k = law->k;
        double r = law->a;
        double f = r * exp(-r * tau);
        for (int n = 1; n < k; ++n)
            f *= r * tau / (double)n;
        return f;
    }
    default:
        return NAN;
    }
}

/* Eq. 8: rho_j = beta s(tau_j) 1{X_j = I}; s = 1 is the Markovian edge. */
double fso_shedding(const fso_params* prm, double tau)
{
    switch (prm->shed_mode) {
    case FSO_SHED_NONE:
        return 1.0;
    case FSO_SHED_HAZARD:
        return fso_hazard(&prm->shedding, tau);
    case FSO_SHED_DENSITY:
        return fso_density(&prm->shedding, tau);
    default:
        return NAN;
    }
}

/* ------------------------------------------------------------------------ */
/* Storage rounding (Section 5.7, Table "mixed precision dtypes"): all math */
/* in fp32, round-to-nearest-even on the store.                             */
/* ------------------------------------------------------------------------ */
static uint32_t f32_bits(float x) { uint32_t u; memcpy(&u, &x, 4); return u; }
static float bits_f32(uint32_t u) { float x; memcpy(&x, &u, 4); return x; }

uint16_t fso_f32_to_f16_bits(float x)
{
    uint32_t u = f32_bits(x);
    uint32_t sign = (u >> 16) & 0x8000u;
    int32_t  exp8 = (int32_t)((u >> 23) & 0xffu);
    uint32_t mant = u & 0x7fffffu;
    if (exp8 == 0xff)                             /* inf or nan */
        return (uint16_t)(sign | 0x7c00u | (mant ? 0x200u : 0u));
    int32_t e16 = exp8 - 127 + 15;
    if (e16 >= 31)                                /* beyond the largest finite */
        return (uint16_t)(sign | 0x7c00u);
    if (e16 > 0) {                                /* normal binary16 */
        uint32_t h = sign | ((uint32_t)e16 << 10) | (mant >> 13);
        uint32_t rest = mant & 0x1fffu;
        if (rest > 0x1000u || (rest == 0x1000u && (h & 1u)))
            h += 1u;                              /* may carry into inf: correct */
        return (uint16_t)h;
    }
    /* subnormal binary16: value / 2^-24, rounded to nearest even */
    if (exp8 == 0)
        return (uint16_t)sign;                    /* fp32 subnormals are < 2^-126 */
    uint64_t m = (uint64_t)(mant | 0x800000u);
    int shift = 126 - exp8;                       /* >= 14 here */
    if (shift > 25)
        return (uint16_t)sign;
    uint64_t q = m >> shift;
    uint64_t rest = m & ((1ull << shift) - 1ull);
    uint64_t half = 1ull << (shift - 1);
    if (rest > half || (rest == half && (q & 1ull)))
        q += 1ull;
    return (uint16_t)(sign | (uint32_t)q);
}

float fso_f16_bits_to_f32(uint16_t h)
{
    uint32_t sign = ((uint32_t)h & 0x8000u) << 16;
    uint32_t e = ((uint32_t)h >> 10) & 0x1fu;
    uint32_t m = (uint32_t)h & 0x3ffu;
    if (e == 0x1fu)
        return bits_f32(sign | 0x7f800000u | (m << 13));
    if (e == 0) {                                 /* zero or subnormal: m * 2^-24 */
        float v = (float)m * (1.0f / 16777216.0f);
        return sign ? -v : v;
    }
    return bits_f32(sign | ((e - 15u + 127u) << 23) | (m << 13));
}

uint16_t fso_f32_to_bf16_bits(float x)
{
    uint32_t u = f32_bits(x);
    if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x7fffffu))
        return (uint16_t)((u >> 16) | 0x40u);     /* quiet nan */
    /* round to nearest, ties to even, on the 16 dropped bits */
    uint32_t rest = u & 0xffffu;
    uint32_t hi = u >> 16;
    if (rest > 0x8000u || (rest == 0x8000u && (hi & 1u)))
        hi += 1u;
    return (uint16_t)hi;
}

float fso_bf16_bits_to_f32(uint16_t h) { return bits_f32((uint32_t)h << 16); }

float fso_store_age(float x, int32_t age_dtype)
{
    switch (age_dtype) {
    case FSO_AGE_F16:  return fso_f16_bits_to_f32(fso_f32_to_f16_bits(x));
    case FSO_AGE_BF16: return fso_bf16_bits_to_f32(fso_f32_to_bf16_bits(x));
    default:           return x;
    }
}

float fso_age_next(float age, double dt, int32_t age_dtype)
{
    volatile float s = age + (float)dt;           /* one IEEE single add */
    return fso_store_age(s, age_dtype);
}

/* Eq. 8 stored as Section 5.7 stores ages: the product beta * s(tau) in
 * double, rounded to fp32, then to the storage type. */
float fso_infectivity(const fso_params* prm, float tau)
{
    float rho32 = (float)(prm->beta * fso_shedding(prm, (double)tau));
    return fso_store_age(rho32, prm->age_dtype);
}

/* ------------------------------------------------------------------------ */
/* The step (Algorithm 3, fixed step; Section 3 Eqs. 1-3; Section 5.2).     */
/* ------------------------------------------------------------------------ */
int fso_init(int64_t n, const int32_t* index_nodes, int64_t n_index,
             int32_t index_state, uint8_t* X, float* A)
{
    if (index_state < FSO_E || index_state > FSO_I)
        return -1;
    for (int64_t i = 0; i < n; ++i) {
        X[i] = FSO_S;
        A[i] = 0.0f;
    }
    for (int64_t q = 0; q < n_index; ++q) {
        int64_t i = index_nodes[q];
        if (i < 0 || i >= n || X[i] != FSO_S)
            return -1;                            /* out of range or repeated */
        X[i] = (uint8_t)index_state;
    }
    return 0;
}

void fso_counts(int64_t n, const uint8_t* X, uint32_t counts[4])
{
    counts[0] = counts[1] = counts[2] = counts[3] = 0;
    for (int64_t i = 0; i < n; ++i)
        counts[X[i] & 3u] += 1u;
}

static int successor(int32_t model, int x)
{
    switch (x) {
    case FSO_S: return model == FSO_SEIR ? FSO_E : FSO_I;
    case FSO_E: return FSO_I;
    case FSO_I: return FSO_R;
    default:    return FSO_R;
    }
}

int fso_step(int64_t n, const int64_t* row_ptr, const int32_t* col_ind,
             const fso_params* prm, int64_t k,
             const uint8_t* X, const float* A, uint8_t* Xn, float* An,
             double* margin, double* lambda_out)
{
    return fso_step_rho(n, row_ptr, col_ind, prm, k, X, A, NULL, Xn, An, NULL, margin, lambda_out);
}

int fso_step_rho(int64_t n, const int64_t* row_ptr, const int32_t* col_ind,
                 const fso_params* prm, int64_t k,
                 const uint8_t* X, const float* A, const float* rho_in,
                 uint8_t* Xn, float* An, float* rho_out,
                 double* margin, double* lambda_out)
{
    if (prm->shed_mode < FSO_SHED_NONE || prm->shed_mode > FSO_SHED_DENSITY)
        return -1;
    for (int64_t i = 0; i < n; ++i) {
        int x = X[i];
        double tau = (double)A[i];
        double lambda = 0.0;
        if (x == FSO_S && prm->shed_mode == FSO_SHED_NONE) {
            /* Eq. 3 with rho = beta 1{X_j = I}: integer pressure c_i */
            int64_t c = 0;
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
                if (X[col_ind[e]] == FSO_I)
                    c += 1;
            lambda = prm->beta * (double)c;
        } else if (x == FSO_S) {
            /* Eq. 3 with the infectivity of Eq. 8: the sum of the stored
             * rho_j of the infectious in-neighbours, in row order */
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                int32_t j = col_ind[e];
                if (X[j] == FSO_I)
                    lambda += rho_in ? (double)rho_in[j] : (double)fso_infectivity(prm, A[j]);
            }
        } else if (x == FSO_E) {
            if (prm->model != FSO_SEIR)
                return -1;
            lambda = fso_hazard(&prm->latent, tau);
        } else if (x == FSO_I) {
            lambda = fso_hazard(&prm->infectious, tau);
        } else if (x != FSO_R) {
            return -1;
        }
        /* Section 5.2: p = 1 - exp(-lambda dt), Bernoulli(p) */
        double p = (lambda > 0.0) ? -expm1(-lambda * prm->dt) : 0.0;
        int fire = 0;
        double mg = INFINITY;
        if (p > 0.0) {
            double u = fso_uniform(prm->seed, prm->rep, k, i);
            fire = (u < p);
            mg = u - p;
        }
        if (margin)
            margin[i] = mg;
        if (lambda_out)
            lambda_out[i] = lambda;
        /* transition and renewal age (Eq. 1: age resets on any transition) */
        if (fire) {
            Xn[i] = (uint8_t)successor(prm->model, x);
            An[i] = 0.0f;
        } else {
            Xn[i] = (uint8_t)x;
            An[i] = (x == FSO_E || x == FSO_I) ? fso_age_next(A[i], prm->dt, prm->age_dtype)
                                               : 0.0f;
        }
        /* the next step's infectivity, from the new age (Section 5.3) */
        if (rho_out)
            rho_out[i] = (Xn[i] != FSO_I) ? 0.0f
                       : (prm->shed_mode == FSO_SHED_NONE) ? (float)prm->beta : fso_infectivity(prm, An[i]);
    }
    return 0;
}

/* Section 5.2: dt = min(dt_max, eps / (max_i lambda_i + delta)), in double,
 * from the rates of the previous step; the ages advance by its float value. */
float fso_adaptive_dt(double dt_max, double eps, double delta, double lambda_prev)
{
    double dt = eps / (lambda_prev + delta);
    if (dt > dt_max)
        dt = dt_max;
    return (float)dt;
}

int fso_run_adaptive(int64_t n, const int64_t* row_ptr, const int32_t* col_ind,
                     const fso_params* prm, double eps, double delta, double lambda_prev,
                     int64_t k0, int64_t steps, uint8_t* X, float* A, uint32_t* counts,
                     float* dts, double* lambda_last)
{
    const size_t m = (size_t)(n > 0 ? n : 1);
    uint8_t* X2 = (uint8_t*)malloc(m);
    float* A2 = (float*)malloc(sizeof(float) * m);
    double* lam = (double*)malloc(sizeof(double) * m);
    if (!X2 || !A2 || !lam) {
        free(X2); free(A2); free(lam);
        return -1;
    }
    uint8_t* xc = X; float* ac = A;
    uint8_t* xn = X2; float* an = A2;
    fso_params p = *prm;
    int rc = 0;
    if (counts)
        fso_counts(n, xc, counts);
    for (int64_t s = 0; s < steps; ++s) {
        const float dt = fso_adaptive_dt(prm->dt, eps, delta, lambda_prev);
        p.dt = (double)dt;
        rc = fso_step(n, row_ptr, col_ind, &p, k0 + s, xc, ac, xn, an, NULL, lam);
        if (rc)
            break;
        if (dts)
            dts[s] = dt;
        /* the largest rate of this step sets the next step's size */
        double mx = 0.0;
        for (int64_t i = 0; i < n; ++i)
            if (lam[i] > mx)
                mx = lam[i];
        lambda_prev = mx;
        if (counts)
            fso_counts(n, xn, counts + 4 * (s + 1));
        uint8_t* tx = xc; xc = xn; xn = tx;
        float* ta = ac; ac = an; an = ta;
    }
    if (lambda_last)
        *lambda_last = lambda_prev;
    if (xc != X) {
        memcpy(X, xc, (size_t)n);
        memcpy(A, ac, sizeof(float) * (size_t)n);
    }
    free(X2); free(A2); free(lam);
    return rc;
}

int fso_run(int64_t n, const int64_t* row_ptr, const int32_t* col_ind,
            const fso_params* prm, int64_t k0, int64_t steps,
            uint8_t* X, float* A, uint32_t* counts)
{
    uint8_t* X2 = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
    float* A2 = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    if (!X2 || !A2) {
        free(X2); free(A2);
        return -1;
    }
    uint8_t* xc = X; float* ac = A;
    uint8_t* xn = X2; float* an = A2;
    int rc = 0;
    if (counts)
        fso_counts(n, xc, counts);
    for (int64_t s = 0; s < steps; ++s) {
        rc = fso_step(n, row_ptr, col_ind, prm, k0 + s, xc, ac, xn, an, NULL, NULL);
        if (rc)
            break;
        if (counts)
            fso_counts(n, xn, counts + 4 * (s + 1));
        uint8_t* tx = xc; xc = xn; xn = tx;
        float* ta = ac; ac = an; an = ta;
    }
    if (xc != X) {
        memcpy(X, xc, (size_t)n);
        memcpy(A, ac, sizeof(float) * (size_t)n);
    }
    free(X2); free(A2);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Exact event-driven simulator (the exact reference the paper validates    */
/* against, Section 6 "validation" and Appendix C). Only the S -> E rates   */
/* depend on the network state and they are piecewise constant between      */
/* events, so drawing the next contact event from the total rate and the    */
/* E/I exits from holding times sampled at entry is exact.                  */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t s; } sm64;

static uint64_t sm64_next(sm64* g)
{
    uint64_t z = (g->s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double sm64_open01(sm64* g)            /* uniform on (0, 1) */
{
    return ((double)(sm64_next(g) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

static double sm64_normal(sm64* g)            /* Box-Muller */
{
    double u1 = sm64_open01(g), u2 = sm64_open01(g);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

static double sample_holding(const fso_law* law, sm64* g)
{
    switch (law->kind) {
    case FSO_LAW_EXP:
        return -log(sm64_open01(g)) / law->a;
    case FSO_LAW_LOGNORMAL:
        return exp(law->a + law->b * sm64_normal(g));
    case FSO_LAW_WEIBULL:
        return law->b * pow(-log(sm64_open01(g)), 1.0 / law->a);
    case FSO_LAW_ERLANG: {
        double t = 0.0;
        for (int s = 0; s < law->k; ++s)
            t += -log(sm64_open01(g)) / law->a;
        return t;
    }
    default:
        return INFINITY;
    }
}

int fso_exact_run(int64_t n, const int64_t* row_ptr, const int32_t* col_ind,
                  const fso_params* prm, const int32_t* index_nodes,
                  int64_t n_index, int32_t index_state, uint64_t rng_seed,
                  int64_t n_grid, double grid_dt, uint32_t* counts_grid)
{
    if (prm->shed_mode != FSO_SHED_NONE)
        return -1;                   /* rates between events must be constant */
    int64_t nnz = row_ptr[n];
    uint8_t* X = (uint8_t*)malloc((size_t)n);
    double* t_exit = (double*)malloc(sizeof(double) * (size_t)n);
    int64_t* c = (int64_t*)calloc((size_t)n, sizeof(int64_t));
    int64_t* out_ptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t* out_ind = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    if (!X || !t_exit || !c || !out_ptr || !out_ind || !fill) {
        free(X); free(t_exit); free(c); free(out_ptr); free(out_ind); free(fill);
        return -1;
    }
    /* out-neighbour lists: j -> i for every e in row i with col_ind[e] = j */
    for (int64_t e = 0; e < nnz; ++e)
        out_ptr[col_ind[e] + 1] += 1;
    for (int64_t i = 0; i < n; ++i)
        out_ptr[i + 1] += out_ptr[i];
    for (int64_t i = 0; i < n; ++i)
        fill[i] = out_ptr[i];
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            out_ind[fill[col_ind[e]]++] = (int32_t)i;

    sm64 g = { rng_seed };
    for (int64_t i = 0; i < n; ++i) {
        X[i] = FSO_S;
        t_exit[i] = INFINITY;
    }
    for (int64_t q = 0; q < n_index; ++q) {
        int64_t i = index_nodes[q];
        X[i] = (uint8_t)index_state;
        t_exit[i] = sample_holding(index_state == FSO_E ? &prm->latent : &prm->infectious, &g);
        if (index_state == FSO_I)
            for (int64_t e = out_ptr[i]; e < out_ptr[i + 1]; ++e)
                c[out_ind[e]] += 1;
    }
    uint32_t cnt[4];
    fso_counts(n, X, cnt);
    double t = 0.0;
    int64_t gi = 0;
    for (;;) {
        /* total contact rate over S nodes and the earliest scheduled exit */
        int64_t csum = 0;
        for (int64_t i = 0; i < n; ++i)
            if (X[i] == FSO_S)
                csum += c[i];
        double lam = prm->beta * (double)csum;
        int64_t who = -1;
        double t_sched = INFINITY;
        for (int64_t i = 0; i < n; ++i)
            if (t_exit[i] < t_sched) {
                t_sched = t_exit[i];
                who = i;
            }
        double t_inf = (lam > 0.0) ? t - log(sm64_open01(&g)) / lam : INFINITY;
        double t_ev = (t_inf < t_sched) ? t_inf : t_sched;
        while (gi < n_grid && (double)gi * grid_dt < t_ev) {
            memcpy(counts_grid + 4 * gi, cnt, sizeof(cnt));
            ++gi;
        }
        if (gi >= n_grid || !(t_ev < INFINITY))
            break;
        int64_t node;
        int from, to;
        if (t_inf < t_sched) {
            /* choose the infected S node with probability c_i / sum c */
            double target = sm64_open01(&g) * (double)csum;
            double acc = 0.0;
            node = -1;
            for (int64_t i = 0; i < n; ++i)
                if (X[i] == FSO_S && c[i] > 0) {
                    acc += (double)c[i];
                    node = i;
                    if (acc > target)
                        break;
                }
            from = FSO_S;
            to = successor(prm->model, FSO_S);
        } else {
            node = who;
            from = X[node];
            to = successor(prm->model, from);
        }
        X[node] = (uint8_t)to;
        cnt[from] -= 1u;
        cnt[to] += 1u;
        t_exit[node] = INFINITY;
        if (to == FSO_E)
            t_exit[node] = t_ev + sample_holding(&prm->latent, &g);
        else if (to == FSO_I)
            t_exit[node] = t_ev + sample_holding(&prm->infectious, &g);
        if (to == FSO_I)
            for (int64_t e = out_ptr[node]; e < out_ptr[node + 1]; ++e)
                c[out_ind[e]] += 1;
        if (from == FSO_I)
            for (int64_t e = out_ptr[node]; e < out_ptr[node + 1]; ++e)
                c[out_ind[e]] -= 1;
        t = t_ev;
    }
    while (gi < n_grid) {
        memcpy(counts_grid + 4 * gi, cnt, sizeof(cnt));
        ++gi;
    }
    free(X); free(t_exit); free(c); free(out_ptr); free(out_ind); free(fill);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Markovian engine (Section 4, Algorithm 1): constant rates, tau-leaping    */
/* with the step chosen from the total and the largest rate.               */
/* ------------------------------------------------------------------------ */
static int markov_params_ok(const fso_params* prm)
{
    if (prm->model != FSO_SIR && prm->model != FSO_SIS && prm->model != FSO_SEIR)
        return 0;
    if (prm->infectious.kind != FSO_LAW_EXP)
        return 0;
    if (prm->model == FSO_SEIR && prm->latent.kind != FSO_LAW_EXP)
        return 0;
    return 1;
}

/* rate of node i of state X (Eq. 3 for S with rho = beta 1{X_j = I}) */
static double markov_rate(int64_t i, const int64_t* row_ptr, const int32_t* col_ind,
                          const fso_params* prm, const uint8_t* X)
{
    switch (X[i]) {
    case FSO_S: {
        int64_t c = 0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            if (X[col_ind[e]] == FSO_I)
                c += 1;
        return prm->beta * (double)c;
    }
    case FSO_E:
        return prm->latent.a;
    case FSO_I:
        return prm->infectious.a;
    default:
        return 0.0;
    }
}

float fso_markov_tau(int64_t n, const int64_t* row_ptr, const int32_t* col_ind,
                     const fso_params* prm, double theta, double p_max, double tau_max,
                     const uint8_t* X, double* Lambda, double* lambda_max)
{
    /* Lambda collected by compartment, so that its rounding is fixed:
     * beta * (number of S-I edges) + sigma * |E| + gamma * |I| */
    int64_t si = 0, ne = 0, ni = 0, cmax = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (X[i] == FSO_S) {
            int64_t c = 0;
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
                if (X[col_ind[e]] == FSO_I)
                    c += 1;
            si += c;
            if (c > cmax)
                cmax = c;
        } else if (X[i] == FSO_E) {
            ne += 1;
        } else if (X[i] == FSO_I) {
            ni += 1;
        }
    }
    double sigma = prm->model == FSO_SEIR ? prm->latent.a : 0.0;
    double gamma = prm->infectious.a;
    double lam = prm->beta * (double)si + sigma * (double)ne + gamma * (double)ni;
    double lmax = prm->beta * (double)cmax;
    if (ne > 0 && sigma > lmax)
        lmax = sigma;
    if (ni > 0 && gamma > lmax)
        lmax = gamma;
    double tau = tau_max;
    if (lam > 0.0 && theta * (double)n / lam < tau)
        tau = theta * (double)n / lam;
    if (lmax > 0.0 && p_max / lmax < tau)
        tau = p_max / lmax;
    if (Lambda)
        *Lambda = lam;
    if (lambda_max)
        *lambda_max = lmax;
    return (float)tau;
}

int fso_markov_step(int64_t n, const int64_t* row_ptr, const int32_t* col_ind,
                    const fso_params* prm, double theta, double p_max, double tau_max, float tau_in,
                    int64_t k, const uint8_t* X, const float* A, uint8_t* Xn, float* An,
                    double* margin, float* tau_out)
{
    if (!markov_params_ok(prm))
        return -1;
    float tau = tau_in > 0.0f ? tau_in
                              : fso_markov_tau(n, row_ptr, col_ind, prm, theta, p_max, tau_max, X, NULL, NULL);
    if (tau_out)
        *tau_out = tau;
    for (int64_t i = 0; i < n; ++i) {
        int x = X[i];
        if (x > FSO_R || (x == FSO_E && prm->model != FSO_SEIR) || (x == FSO_R && prm->model == FSO_SIS))
            return -1;
        double lambda = markov_rate(i, row_ptr, col_ind, prm, X);
        double p = (lambda > 0.0) ? -expm1(-lambda * (double)tau) : 0.0;
        int fire = 0;
        double mg = INFINITY;
        if (p > 0.0) {
            double u = fso_uniform(prm->seed, prm->rep, k, i);
            fire = (u < p);
            mg = u - p;
        }
        if (margin)
            margin[i] = mg;
        if (fire) {
            int y;
            if (x == FSO_S)
                y = prm->model == FSO_SEIR ? FSO_E : FSO_I;
            else if (x == FSO_E)
                y = FSO_I;
            else
                y = prm->model == FSO_SIS ? FSO_S : FSO_R;
            Xn[i] = (uint8_t)y;
            An[i] = 0.0f;
        } else {
            Xn[i] = (uint8_t)x;
            An[i] = (x == FSO_E || x == FSO_I) ? fso_age_next(A[i], (double)tau, prm->age_dtype) : 0.0f;
        }
    }
    return 0;
}

/* Fenwick tree over the node rates (sums of ranges of rates; the total at
 * the root); selection by descending the implicit tree */
typedef struct {
    int64_t n, top;
    double* t;
} fenwick;

static void fw_add(fenwick* f, int64_t i, double v)
{
    for (int64_t j = i + 1; j <= f->n; j += j & -j)
        f->t[j] += v;
}

static int64_t fw_find(const fenwick* f, double u)   /* smallest i with prefix(i+1) > u */
{
    int64_t pos = 0;
    for (int64_t step = f->top; step > 0; step >>= 1) {
        if (pos + step <= f->n && f->t[pos + step] <= u) {
            pos += step;
            u -= f->t[pos];
        }
    }
    return pos < f->n ? pos : f->n - 1;
}

int fso_gillespie_run(int64_t n, const int64_t* row_ptr, const int32_t* col_ind,
                      const fso_params* prm, const int32_t* index_nodes, int64_t n_index,
                      int32_t index_state, uint64_t rng_seed, int64_t n_grid, double grid_dt,
                      uint32_t* counts_grid)
{
    if (!markov_params_ok(prm) || n <= 0)
        return -1;
    int64_t nnz = row_ptr[n];
    uint8_t* X = (uint8_t*)malloc((size_t)n);
    int64_t* c = (int64_t*)calloc((size_t)n, sizeof(int64_t));
    double* rate = (double*)calloc((size_t)n, sizeof(double));
    int64_t* out_ptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t* out_ind = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    fenwick f = { n, 1, (double*)calloc((size_t)n + 1, sizeof(double)) };
    if (!X || !c || !rate || !out_ptr || !out_ind || !fill || !f.t) {
        free(X); free(c); free(rate); free(out_ptr); free(out_ind); free(fill); free(f.t);
        return -1;
    }
    while (f.top * 2 <= n)
        f.top *= 2;
    for (int64_t e = 0; e < nnz; ++e)
        out_ptr[col_ind[e] + 1] += 1;
    for (int64_t i = 0; i < n; ++i)
        out_ptr[i + 1] += out_ptr[i];
    for (int64_t i = 0; i < n; ++i)
        fill[i] = out_ptr[i];
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            out_ind[fill[col_ind[e]]++] = (int32_t)i;

    const double sigma = prm->model == FSO_SEIR ? prm->latent.a : 0.0;
    const double gamma = prm->infectious.a;
    for (int64_t i = 0; i < n; ++i)
        X[i] = FSO_S;
    for (int64_t q = 0; q < n_index; ++q)
        X[index_nodes[q]] = (uint8_t)index_state;
    for (int64_t i = 0; i < n; ++i)
        if (X[i] == FSO_I)
            for (int64_t e = out_ptr[i]; e < out_ptr[i + 1]; ++e)
                c[out_ind[e]] += 1;
    /* (re)sets the rate of node i in the tree */
#define SET_RATE(i)                                                                  \
    do {                                                                             \
        double r_ = X[i] == FSO_S ? prm->beta * (double)c[i]                         \
                  : X[i] == FSO_E ? sigma : X[i] == FSO_I ? gamma : 0.0;             \
        fw_add(&f, (i), r_ - rate[i]);                                               \
        rate[i] = r_;                                                                \
    } while (0)
    for (int64_t i = 0; i < n; ++i)
        SET_RATE(i);

    sm64 g = { rng_seed };
    uint32_t cnt[4];
    fso_counts(n, X, cnt);
    double t = 0.0;
    int64_t gi = 0, events = 0;
    for (;;) {
        /* the tree's running sums drift by rounding; rebuild them now and then */
        if ((events & 4095) == 0) {
            memset(f.t, 0, sizeof(double) * ((size_t)n + 1));
            for (int64_t i = 0; i < n; ++i)
                fw_add(&f, i, rate[i]);
        }
        double total = 0.0;
        for (int64_t step = f.top, pos = 0; step > 0; step >>= 1)
            if (pos + step <= n) {
                pos += step;
                total += f.t[pos];
            }
        double t_ev = (total > 0.0) ? t - log(sm64_open01(&g)) / total : INFINITY;
        while (gi < n_grid && (double)gi * grid_dt < t_ev) {
            memcpy(counts_grid + 4 * gi, cnt, sizeof(cnt));
            ++gi;
        }
        if (gi >= n_grid || !(total > 0.0))
            break;
        t = t_ev;
        int64_t i = fw_find(&f, sm64_open01(&g) * total);
        while (rate[i] <= 0.0 && i + 1 < n)          /* rounding at a boundary */
            ++i;
        int x = X[i];
        int y = x == FSO_S ? (prm->model == FSO_SEIR ? FSO_E : FSO_I)
              : x == FSO_E ? FSO_I : (prm->model == FSO_SIS ? FSO_S : FSO_R);
        X[i] = (uint8_t)y;
        cnt[x] -= 1;
        cnt[y] += 1;
        if ((x == FSO_I) != (y == FSO_I)) {
            int64_t d = (y == FSO_I) ? 1 : -1;
            for (int64_t e = out_ptr[i]; e < out_ptr[i + 1]; ++e) {
                int64_t j = out_ind[e];
                c[j] += d;
                if (X[j] == FSO_S)
                    SET_RATE(j);
            }
        }
        SET_RATE(i);
        ++events;
    }
#undef SET_RATE
    while (gi < n_grid) {
        memcpy(counts_grid + 4 * gi, cnt, sizeof(cnt));
        ++gi;
    }
    free(X); free(c); free(rate); free(out_ptr); free(out_ind); free(fill); free(f.t);
    return 0;
}

int fso_markov_run(int64_t n, const int64_t* row_ptr, const int32_t* col_ind,
                   const fso_params* prm, double theta, double p_max, double tau_max,
                   int64_t k0, int64_t n_grid, double grid_dt, uint8_t* X, float* A,
                   uint32_t* counts_grid, int64_t* steps_out)
{
    const size_t m = (size_t)(n > 0 ? n : 1);
    uint8_t* X2 = (uint8_t*)malloc(m);
    float* A2 = (float*)malloc(sizeof(float) * m);
    if (!X2 || !A2) {
        free(X2); free(A2);
        return -1;
    }
    uint8_t* xc = X; float* ac = A;
    uint8_t* xn = X2; float* an = A2;
    double t = 0.0;
    int64_t gi = 0, k = k0;
    int rc = 0;
    uint32_t cnt[4];
    fso_counts(n, xc, cnt);
    while (gi < n_grid) {
        while (gi < n_grid && (double)gi * grid_dt <= t) {
            memcpy(counts_grid + 4 * gi, cnt, sizeof(cnt));
            ++gi;
        }
        if (gi >= n_grid)
            break;
        float tau = 0.0f;
        rc = fso_markov_step(n, row_ptr, col_ind, prm, theta, p_max, tau_max, 0.0f, k, xc, ac, xn, an, NULL, &tau);
        if (rc)
            break;
        t += (double)tau;
        ++k;
        fso_counts(n, xn, cnt);
        uint8_t* tx = xc; xc = xn; xn = tx;
        float* ta = ac; ac = an; an = ta;
    }
    if (steps_out)
        *steps_out = k - k0;
    if (xc != X) {
        memcpy(X, xc, (size_t)n);
        memcpy(A, ac, sizeof(float) * (size_t)n);
    }
    free(X2); free(A2);
    return rc;
}
