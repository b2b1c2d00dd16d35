/*
 * fs_oracle.h -- plain, slow, single-threaded CPU oracle for the renewal
 * (age-dependent hazard) Bernoulli tau-leaping step of SIR/SEIR on a CSR
 * contact graph (FlashSpread, arXiv 2604.22092, Sections 3 and 5, Algorithm 3).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, loads or
 * calls this code: it exists so that tests, the smoke check and the CPU
 * baseline leg of the benchmark can compare the CUDA path with an independent
 * restatement of the method. It shares no source with the CUDA path.
 *
 * Conventions (shared with the C ABI only through their definitions):
 *   compartments  S = 0, E = 1, I = 2, R = 3 (SIR leaves E empty)
 *   CSR           row i lists the in-neighbours j of node i (Section 3, Eq. 3;
 *                 Appendix D.1): row_ptr int64[n+1], col_ind int32[E]
 *   ages          stored as the float value of the storage type (f32, f16 or
 *                 bf16 values are all exactly representable in a float)
 *   uniforms      u = (w >> 8) * 2^-24, w = word (rep mod 4) of
 *                 Philox4x32-10(counter = (node, step, rep / 4, 0),
 *                               key = (seed_lo32, seed_hi32))
 */
#ifndef FS_ORACLE_H
#define FS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { FSO_S = 0, FSO_E = 1, FSO_I = 2, FSO_R = 3 };
enum { FSO_SIR = 0, FSO_SEIR = 1, FSO_SIS = 2 };
enum { FSO_LAW_NONE = 0, FSO_LAW_EXP = 1, FSO_LAW_LOGNORMAL = 2,
       FSO_LAW_WEIBULL = 3, FSO_LAW_ERLANG = 4 };
enum { FSO_AGE_F32 = 0, FSO_AGE_F16 = 1, FSO_AGE_BF16 = 2 };
/* shedding profile s(tau) of the infectivity (Section 5.3, Eq. 8) */
enum { FSO_SHED_NONE = 0, FSO_SHED_HAZARD = 1, FSO_SHED_DENSITY = 2 };

/* Holding-time law.  EXP: a = rate.  LOGNORMAL: a = mu, b = sigma (log-days).
 * WEIBULL: a = shape k, b = scale s.  ERLANG: k = stages, a = rate per stage. */
typedef struct {
    int32_t kind;
    int32_t k;
    double a, b;
} fso_law;

typedef struct {
    int32_t model;          /* FSO_SIR or FSO_SEIR                          */
    int32_t age_dtype;      /* FSO_AGE_F32 / F16 / BF16                      */
    fso_law latent;         /* E -> I (SEIR only)                            */
    fso_law infectious;     /* I -> R                                        */
    double beta;            /* per infectious in-neighbour hazard (1/day)    */
    double dt;              /* fixed step (days)                             */
    uint64_t seed;          /* Philox key                                    */
    uint32_t rep;           /* realisation index inside the key's stream     */
    int32_t shed_mode;      /* FSO_SHED_NONE: s = 1 (Markovian edges);
                               FSO_SHED_HAZARD / _DENSITY: s(tau) = the hazard
                               or the density of `shedding`                  */
    fso_law shedding;
} fso_params;

/* ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ------------------ */
void fso_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* The 24-bit uniform of (seed, rep, step, node), as a double in [0, 1). */
double fso_uniform(uint64_t seed, uint32_t rep, int64_t step, int64_t node);

/* ---- hazards in double precision (Section 5.1, Proposition 1) ----------- */
double fso_erfcx(double z);
double fso_hazard(const fso_law* law, double tau);

/* probability density of a law (0 for FSO_LAW_NONE) */
double fso_density(const fso_law* law, double tau);

/* ---- source-node infectivity (Section 5.3, Eq. 8) ------------------------ */
/* s(tau): 1, or the hazard / density of prm->shedding at infection age tau */
double fso_shedding(const fso_params* prm, double tau);
/* The stored infectivity of an I node of age tau: beta * s(tau) rounded to
 * fp32, then to the storage type of the ages (prm->age_dtype). */
float fso_infectivity(const fso_params* prm, float tau);

/* ---- storage rounding (Section 5.7: fp32 math, cast on store) ----------- */
uint16_t fso_f32_to_f16_bits(float x);
float    fso_f16_bits_to_f32(uint16_t h);
uint16_t fso_f32_to_bf16_bits(float x);
float    fso_bf16_bits_to_f32(uint16_t h);
float    fso_store_age(float x, int32_t age_dtype);
/* renewal age update of a node that did not fire and is in E or I */
float    fso_age_next(float age, double dt, int32_t age_dtype);

/* ---- the tau-leaping step (Algorithm 3 with a fixed step) --------------- */
/* Initial condition: every node S with age 0, listed nodes in index_state
 * with age 0. Returns 0, or -1 on a bad index list. */
int fso_init(int64_t n, const int32_t* index_nodes, int64_t n_index,
             int32_t index_state, uint8_t* X, float* A);

void fso_counts(int64_t n, const uint8_t* X, uint32_t counts[4]);

/* One synchronous step k: reads (X, A), writes (Xn, An). When margin is not
 * NULL, margin[i] = u_i - p_i for every node with p_i > 0 and +inf elsewhere.
 * When lambda_out is not NULL it receives lambda_i. Returns 0 or -1. */
int fso_step(int64_t n, const int64_t* row_ptr, const int32_t* col_ind,
             const fso_params* prm, int64_t k,
             const uint8_t* X, const float* A, uint8_t* Xn, float* An,
             double* margin, double* lambda_out);

/* The same step with the infectivity made explicit (shed_mode != NONE: the
 * pressure of an S node is the sum, in double, of the stored infectivities
 * of its infectious in-neighbours). rho_in[n]: the infectivity of every node
 * as stored (read only where X = I), or NULL to compute it from A with
 * fso_infectivity. rho_out[n] (may be NULL): the next step's infectivity,
 * fso_infectivity(An) where Xn = I and 0 elsewhere. With shed_mode = NONE
 * both are ignored (rho_out is filled with beta where Xn = I). */
int fso_step_rho(int64_t n, const int64_t* row_ptr, const int32_t* col_ind,
                 const fso_params* prm, int64_t k,
                 const uint8_t* X, const float* A, const float* rho_in,
                 uint8_t* Xn, float* An, float* rho_out,
                 double* margin, double* lambda_out);

/* steps consecutive steps k0 .. k0+steps-1, in place on (X, A);
 * counts[(steps+1)*4], row 0 = the input state. */
int fso_run(int64_t n, const int64_t* row_ptr, const int32_t* col_ind,
            const fso_params* prm, int64_t k0, int64_t steps,
            uint8_t* X, float* A, uint32_t* counts);

/* ---- adaptive step (Section 5.2) ----------------------------------------- */
/* The step size of step k from the largest rate of step k-1:
 *   dt_k = min(dt_max, eps / (lambda*_{k-1} + delta)),
 * returned as the float value the ages advance by (lambda* = 0 before the
 * first step gives dt_max). */
float fso_adaptive_dt(double dt_max, double eps, double delta, double lambda_prev);

/* steps adaptive steps from k0 (prm->dt = dt_max), in place on (X, A), the
 * rates of the step before k0 summarised by lambda_prev (0 at a start):
 * counts[(steps+1)*4] as fso_run, dts[steps] the step sizes used and
 * *lambda_last the largest rate of the last step (any output may be NULL). */
int fso_run_adaptive(int64_t n, const int64_t* row_ptr, const int32_t* col_ind,
                     const fso_params* prm, double eps, double delta, double lambda_prev,
                     int64_t k0, int64_t steps, uint8_t* X, float* A, uint32_t* counts,
                     float* dts, double* lambda_last);

/* ---- Markovian engine (Section 4, Algorithm 1) --------------------------- */
/* Constant rates: an S node leaves at beta * c_i (c_i = its infectious
 * in-neighbours), E at the latent rate sigma, I at the recovery rate gamma
 * (EXP laws in prm). SIS: I -> S; SIR: I -> R; SEIR: S -> E -> I -> R.
 * The step size of Algorithm 1 from the rates of the current state:
 *   Lambda = sum_i lambda_i, tau = min(theta N / Lambda, p_max / max_i
 *   lambda_i, tau_max) (a term is skipped when its denominator is 0),
 * in double in that order, returned as the float the ages advance by. */
float fso_markov_tau(int64_t n, const int64_t* row_ptr, const int32_t* col_ind,
                     const fso_params* prm, double theta, double p_max, double tau_max,
                     const uint8_t* X, double* Lambda, double* lambda_max);

/* One step k of Algorithm 1: tau from fso_markov_tau (or tau_in if > 0),
 * p_i = 1 - exp(-lambda_i tau), Bernoulli with the step's uniforms, the
 * transitions, renewal ages (age 0 on a transition, E/I ages + tau stored
 * as in fso_age_next). margin as in fso_step. *tau_out = the tau used.
 * Returns 0 or -1 (bad state or parameters). */
int fso_markov_step(int64_t n, const int64_t* row_ptr, const int32_t* col_ind,
                    const fso_params* prm, double theta, double p_max, double tau_max, float tau_in,
                    int64_t k, const uint8_t* X, const float* A, uint8_t* Xn, float* An,
                    double* margin, float* tau_out);

/* Algorithm 1 steps from k0 until the time reaches t_end: counts_grid[n_grid
 * * 4] receives the counts of the state holding at t = g * grid_dt (the
 * state after the last step ending at or before it); in place on (X, A);
 * *steps_out = the steps taken. */
int fso_markov_run(int64_t n, const int64_t* row_ptr, const int32_t* col_ind,
                   const fso_params* prm, double theta, double p_max, double tau_max,
                   int64_t k0, int64_t n_grid, double grid_dt, uint8_t* X, float* A,
                   uint32_t* counts_grid, int64_t* steps_out);

/* Exact Doob-Gillespie direct method for the same Markovian models: the
 * next event after Exp(Lambda), the node chosen with probability
 * lambda_i / Lambda (a Fenwick tree over the rates), its own splitmix64
 * stream. counts_grid[n_grid * 4]: the counts at t = g * grid_dt. */
int fso_gillespie_run(int64_t n, const int64_t* row_ptr, const int32_t* col_ind,
                      const fso_params* prm, const int32_t* index_nodes, int64_t n_index,
                      int32_t index_state, uint64_t rng_seed, int64_t n_grid, double grid_dt,
                      uint32_t* counts_grid);

/* ---- exact continuous-time simulator for tiny graphs -------------------- */
/* Event-driven simulation of the same compartmental process without time
 * discretisation: S -> E (SIR: S -> I) at rate beta * (#infectious
 * in-neighbours), piecewise constant between events; E and I holding times
 * drawn at entry from their laws. Uses its own splitmix64 stream (not
 * Philox). counts_grid[(n_grid)*4] receives the counts at t = g * grid_dt. */
int fso_exact_run(int64_t n, const int64_t* row_ptr, const int32_t* col_ind,
                  const fso_params* prm, const int32_t* index_nodes,
                  int64_t n_index, int32_t index_state, uint64_t rng_seed,
                  int64_t n_grid, double grid_dt, uint32_t* counts_grid);

#ifdef __cplusplus
}
#endif
#endif
