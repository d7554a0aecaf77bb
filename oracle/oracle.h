/*
 * oracle.h -- plain, single-threaded CPU oracle for population annealing
 * Monte Carlo (PAMC) on the D-dimensional Edwards-Anderson spin glass.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * call or execute anything under oracle/.  Only tests/, the smoke check in
 * __graft_entry__.py and the cpu_baseline / reference leg of bench.py use it.
 * It shares no code with the CUDA library (paper_1710_09025_gb300/csrc).
 *
 * What it computes (paper sections cited per function in the .c files):
 *   - Hamiltonian H = -sum_<ij> J_ij S_i S_j - sum_i h_i S_i   (Sec. II.A, Eq. 1;
 *     the field term is an addition; the paper is zero-field)
 *   - the PAMC loop of Sec. II.B: R replicas random at beta = 0, resampling
 *     with mean copy number proportional to exp[-(beta'-beta) E_i] when beta
 *     is raised, then N_S Metropolis sweeps per replica (checkerboard order,
 *     Sec. III.A), free energy by free-energy perturbation (Sec. II.B),
 *     family entropy S_f (Eq. 2), overlap histogram (Sec. V.A)
 *   - exact enumeration of Z, <E>, C, beta F, <s_i s_j>, <s_i> on tiny
 *     lattices (the pin for everything stochastic).
 *
 * Every random number and every rounding that feeds the trajectory is
 * specified (stream layout, exp evaluation, summation order) so that an
 * independent implementation can reproduce the trajectory bit for bit.
 */
#ifndef PAMC_ORACLE_H
#define PAMC_ORACLE_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_PM1 = 0, OR_REAL = 1 };

/* Philox stream ids (bits 28..31 of counter word 3). */
enum { OR_STREAM_INIT = 1, OR_STREAM_PLANE = 2, OR_STREAM_WORD = 3, OR_STREAM_RESAMPLE = 4,
       OR_STREAM_ICM = 5 };

/* ---- primitives (philox.c, specmath.c) ---- */
void     or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint32_t or_counter3(uint32_t stream, uint32_t tag, uint32_t instance);
double   or_spec_exp64(double x);
float    or_spec_expf(float x);
/* out[0..3] = INV_LN2, LN2_HI, LN2_LO, (unused); outf[0..2] = float versions;
 * coef[0..14] = double Taylor coefficients; coeff[0..7] = float ones. */
void     or_spec_constants(double out[4], float outf[3], double coef[15], float coeff[8]);
uint64_t or_threshold_pm(double beta, int dE);      /* floor(spec_exp64(-beta*dE) * 2^32) */
uint64_t or_threshold_real(float x);                /* x = beta*dE in FP32, x > 0 */
double   or_uniform53(uint32_t out0, uint32_t out1);
void     or_philox_batch(int64_t n, const uint32_t* ctr, const uint32_t key[2], uint32_t* out);
void     or_spec_exp64_batch(int64_t n, const double* x, double* y);
void     or_spec_expf_batch(int64_t n, const float* x, float* y);
void     or_threshold_real_batch(int64_t n, const float* x, uint64_t* thr);

/* ---- lattice (pamc.c) ---- */
/* neighbour table nbr[i*2D + 2d + 0] = i - e_d, nbr[i*2D + 2d + 1] = i + e_d;
 * bond[i*2D + 2d + 0] = d*N + (i - e_d), bond[i*2D + 2d + 1] = d*N + i.  */
int or_lattice(int D, int L, int32_t* nbr, int32_t* bond);

/* ---- one PAMC run ---- */
typedef struct or_sim or_sim;

or_sim* or_create(int D, int L, int kind, const float* J, const float* h, int R,
                  const double* betas, int n_temps, int n_sweeps, uint64_t seed,
                  uint32_t rng_instance, uint32_t rng_tag, int accumulate_grad);
/* dynamic population (Sec. III.D, Eq. 6): populations[k] replicas at temperature
 * k, 1 <= populations[k] <= R (R is the capacity); NULL keeps R throughout */
or_sim* or_create_dps(int D, int L, int kind, const float* J, const float* h, int R,
                      const double* betas, int n_temps, int n_sweeps, uint64_t seed,
                      uint32_t rng_instance, uint32_t rng_tag, int accumulate_grad,
                      const int32_t* populations);
/* resampling schemes: multinomial (population exactly R_k) or nearest-integer
 * (population R_k in expectation, Sec. II.B).  For the nearest-integer scheme
 * R (or populations[k]) is the target and `capacity` (0: or_default_capacity
 * of the largest target) bounds the population; copies beyond it are dropped.
 * or_step returns -2 once the population has died out (no copies at all). */
#define OR_RESAMPLE_MULTINOMIAL 0
#define OR_RESAMPLE_NEAREST 1
int     or_default_capacity(int R_max);
or_sim* or_create_ex(int D, int L, int kind, const float* J, const float* h, int R,
                     const double* betas, int n_temps, int n_sweeps, uint64_t seed,
                     uint32_t rng_instance, uint32_t rng_tag, int accumulate_grad,
                     const int32_t* populations, int scheme, int capacity);
/* isoenergetic cluster moves (Sec. II.C): at steps k >= 1 with
 * icm_beta_lo <= beta_k <= icm_beta_hi (hi <= 0: every such step), N_S/2
 * sweeps, two rounds of ICM updates on disjoint random pairs (R updates),
 * then the remaining sweeps.  Needs a zero field. */
int     or_set_icm(or_sim* s, int enable, double icm_beta_lo, double icm_beta_hi);
/* the random pairing: the permutation pi_t of [0, n) of ICM round t at step k */
uint32_t or_icm_perm(uint32_t i, uint32_t n, int k, int t, uint64_t seed, uint32_t inst, uint32_t tag);
/* one ICM update of replicas a and b (int8 rows of N spins, modified in
 * place) with the 32-bit site-choice word r32; returns the island size
 * (0: no update) */
int     or_icm_pair(int D, int L, int8_t* a, int8_t* b, uint32_t r32);
int     or_current_R(const or_sim* s);
void    or_destroy(or_sim* s);
/* runs temperature index k = next step; returns k, -1 after the last one, -2
 * if the population died out */
int     or_step(or_sim* s);
int     or_next_step(const or_sim* s);
int     or_N(const or_sim* s);

void or_get_spins(const or_sim* s, int8_t* out);           /* R*N, +1/-1          */
void or_set_spins(or_sim* s, const int8_t* in);            /* R*N, +1/-1          */
void or_get_energies(const or_sim* s, int64_t* out);       /* 2R: (lo, hi) int128 */
void or_get_parents(const or_sim* s, int32_t* out);        /* R                   */
void or_get_family(const or_sim* s, int32_t* out);         /* R                   */
void or_get_weights(const or_sim* s, double* w, double* P);/* R, R (last resample)*/
/* out[0..7] = E_mean, E2_mean, C, lnQ, betaF, S_f, rho_s, R */
void or_get_obs(const or_sim* s, int k, double* out);
void or_get_grad_counts(const or_sim* s, int64_t* cJ, int64_t* ch); /* n_temps*D*N, n_temps*N */

/* nearest-integer resampling of R replicas with energies E (int128 lo/hi
 * pairs) towards `target` copies in expectation; parent has room for cap
 * slots; returns the new population min(sum counts, cap) */
int or_resample_nearest(int kind, int R, const int64_t* E, double beta_prev, double beta_next, int k,
                        uint64_t seed, uint32_t inst, uint32_t tag, double target, int cap,
                        double* w, double* P, int32_t* parent, int32_t* counts, double* lnQ);

/* ---- components on explicit state (used for sampled parity at full size) ---- */
/* spins of replicas [64*g0, 64*g0+64*ng) intersect [0,R): N_S sweeps at step k.
 * state is R_sub x N int8 for those replicas in order, starting at replica 64*g0. */
int or_sweeps_groups(int D, int L, int kind, const float* J, const float* h,
                     double beta, int k, int n_sweeps, uint64_t seed, uint32_t inst,
                     uint32_t tag, int g0, int ng, int R, int8_t* state);
/* resampling of R replicas with energies E (int128 as lo/hi pairs) from
 * beta_prev to beta_next at step k; outputs w, P, parent, counts and lnQ. */
int or_resample(int kind, int R, const int64_t* E, double beta_prev, double beta_next, int k,
                uint64_t seed, uint32_t inst, uint32_t tag,
                double* w, double* P, int32_t* parent, int32_t* counts, double* lnQ,
                double* u_out /* R or NULL */);
void or_energies(int D, int L, int kind, const float* J, const float* h, int R,
                 const int8_t* spins, int64_t* E /* 2R */);
int  or_overlap(int N, int R, const int8_t* a, const int8_t* b, int64_t* hist /* N+1 */);
/* cumulative resampling weights P (n) of weights w in the fixed summation
 * order, and (if prefix_out is not NULL) the prefix sums before the running
 * maximum */
void or_weight_prefix(const double* w, int n, double* P_out, double* prefix_out);
/* sum_r S_i S_{i+e_d} (cJ, D*N) and sum_r S_i (ch, N) of R int8 rows */
int  or_grad_counts(int D, int L, int R, const int8_t* spins, int64_t* cJ, int64_t* ch);

/* ---- exact enumeration (exact.c), N <= 24 ---- */
/* out[b*8 + 0..7] = lnZ, E_mean, E2_mean, C, betaF, E_ground, (0), (0) */
int or_exact(int D, int L, const double* J, const double* h, int n_betas, const double* betas,
             double* out, double* corr /* n_betas*D*N or NULL */, double* mag /* n_betas*N or NULL */);

#ifdef __cplusplus
}
#endif
#endif
