/*
 * pamc.c -- the oracle's population annealing Monte Carlo run.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Plain loops over replicas and
 * sites; no bit tricks, no blocking, no fusion.  int8 spins (+1/-1) stored
 * replica-major, spins[r*N + i].
 *
 * Paper passages followed (arXiv:1710.09025):
 *   Sec. II.A, Eq. (1): H = -sum_<ij> J_ij S_i S_j on an L^D lattice (periodic
 *     boundaries are our reading; the paper does not state them).  A field
 *     term -sum_i h_i S_i is added for the gradient with respect to h.
 *   Sec. II.B: R replicas initialised at random at beta = 0; at each lowering
 *     of the temperature beta -> beta' the population is resampled so that
 *     replica i has on average R exp[-(beta'-beta)E_i] / sum_j exp[...]
 *     copies (the expected population is R); then N_S Metropolis sweeps of
 *     N spin-update attempts per replica.  Work W = R N_S N_T sweeps, so the
 *     sweeps also run at the first temperature.  The resampling scheme is not
 *     stated; we use multinomial resampling (R independent draws).
 *   Sec. II.B: free energy by free-energy perturbation:
 *     Q_k = (1/R) sum_i exp[-(beta_k - beta_{k-1}) E_i],
 *     beta_k F_k = -N ln 2 - sum_{l<=k} ln Q_l   (Z(beta=0) = 2^N).
 *   Sec. II.B, Eq. (2): family entropy S_f = -sum_i nu_i ln nu_i, rho_s = R/e^S_f.
 *   Sec. III.A: checkerboard spin selection; sweep = parity-0 sites then
 *     parity-1 sites (the order is our reading).
 *   Sec. V.A, Eq. (9): observables are plain population averages.
 *   Sec. V.A: spin overlap between uncorrelated replicas (here: slot r of two
 *     independently seeded populations).
 *
 * Random streams (Philox4x32-10, key = (seed lo, seed hi), counter word 3 =
 * stream<<28 | tag<<24 | instance):
 *   INIT   : word(g, i) = out0 | out1<<32 of counter (i, g, 0, c3); replica
 *            64g+j has S_i = -1 iff bit j of the word is set.
 *   PLANE  : (+-J) half-sweep hs = 2(k N_S + s) + parity, site i, q = i>>1,
 *            group g: 16 calls with counter (q, hs, 16g+m, c3), m = 0..15,
 *            give 32 planes, plane 2m = out0|out1<<32, plane 2m+1 = out2|out3<<32;
 *            replica 64g+j draws r = sum_b bit_j(plane_b) 2^(31-b).
 *   WORD   : (real couplings) r(rho, hs, q) = out[q&3] of counter (q>>2, hs, rho, c3).
 *   RESAMPLE: draw q at step k: counter (q, k, 0, c3), u = 53-bit uniform.
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

struct or_sim {
    int D, L, N, kind, R, G, n_temps, n_sweeps, k_next, acc_grad;
    int Rcap, R_src_last;      /* capacity; source population of the last resampling */
    int scheme, dead;          /* resampling scheme; population died out */
    int icm;                   /* isoenergetic cluster moves (Sec. II.C) */
    double icm_lo, icm_hi;     /* beta window of the cluster moves */
    int32_t* Rk;               /* population at each temperature (Sec. III.D, Eq. 6) */
    uint64_t seed;
    uint32_t inst, tag;
    float *J, *h;
    double* betas;
    int32_t *nbr, *bond;
    int8_t *s, *tmp;
    i128* E;
    int32_t *parent, *family, *family_tmp, *counts;
    double *w, *P;
    double* obs;
    double sum_lnQ;
    int64_t *cJ, *ch;
};

static int ipow(int L, int D)
{
    int n = 1;
    for (int d = 0; d < D; ++d) n *= L;
    return n;
}

/* Sec. II.A: nearest neighbours on the periodic L^D lattice, site index
 * i = x + L y + L^2 z.  Neighbour order (-x, +x, -y, +y, -z, +z).  Bond
 * (d, i) joins i and i + e_d and carries J[d*N + i]. */
int or_lattice(int D, int L, int32_t* nbr, int32_t* bond)
{
    if (D < 1 || D > 3 || L < 2) return -1;
    int N = ipow(L, D);
    for (int i = 0; i < N; ++i) {
        int stride = 1;
        for (int d = 0; d < D; ++d) {
            int c = (i / stride) % L;
            int cm = (c + L - 1) % L, cp = (c + 1) % L;
            int im = i + (cm - c) * stride, ip = i + (cp - c) * stride;
            nbr[i * 2 * D + 2 * d + 0] = im;
            nbr[i * 2 * D + 2 * d + 1] = ip;
            bond[i * 2 * D + 2 * d + 0] = d * N + im;
            bond[i * 2 * D + 2 * d + 1] = d * N + i;
            stride *= L;
        }
    }
    return N;
}

static int parity_of(int i, int D, int L)
{
    int p = 0;
    for (int d = 0; d < D; ++d) {
        p += i % L;
        i /= L;
    }
    return p & 1;
}

static i128 fix96(float v) { return (i128)ldexp((double)v, 96); }

/* couplings as used by both acceptance rules: real values are flushed to 0
 * below 2^-73 in magnitude (so that v * 2^96 is an integer) */
static float flush_real(float v) { return (fabsf(v) < 0x1p-73f) ? 0.0f : v; }

/* ---------------- init (Sec. II.B: random replicas at beta = 0) ---------------- */

static void init_spins(int N, int R, uint64_t seed, uint32_t inst, uint32_t tag, int8_t* s)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t c3 = or_counter3(OR_STREAM_INIT, tag, inst);
    int G = (R + 63) / 64;
    for (int g = 0; g < G; ++g)
        for (int i = 0; i < N; ++i) {
            uint32_t ctr[4] = {(uint32_t)i, (uint32_t)g, 0u, c3}, out[4];
            or_philox4x32_10(ctr, key, out);
            uint64_t word = (uint64_t)out[0] | ((uint64_t)out[1] << 32);
            for (int j = 0; j < 64; ++j) {
                int r = 64 * g + j;
                if (r >= R) break;
                s[(size_t)r * N + i] = ((word >> j) & 1u) ? (int8_t)-1 : (int8_t)1;
            }
        }
}

/* ---------------- Metropolis half-sweeps (Sec. II.B, Sec. III.A) ---------------- */

typedef struct {
    int D, L, N;
    const int32_t *nbr, *bond;
    const float *J, *h;
    uint32_t key[2];
    uint32_t inst, tag;
} lat_ctx;

/* +-J couplings: the energy change of flipping S_i is dE = 2 S_i sum_nb J S_nb
 * = 4D - 4 n_unsat, n_unsat = number of the 2D bonds of i with J S_i S_nb = -1.
 * Accept iff dE <= 0 or r < floor(exp(-beta dE) 2^32). */
static void halfsweep_pm(const lat_ctx* c, int8_t* s, int r0, int nrep, double beta, int hs,
                         int parity)
{
    uint64_t thr[4];
    for (int n = 1; n <= 3; ++n) thr[n] = or_threshold_pm(beta, 4 * n);
    uint32_t c3 = or_counter3(OR_STREAM_PLANE, c->tag, c->inst);
    int twoD = 2 * c->D;
    for (int rb = 0; rb < nrep; rb += 64) {
        int g = (r0 + rb) / 64;
        for (int i = 0; i < c->N; ++i) {
            if (parity_of(i, c->D, c->L) != parity) continue;
            uint32_t q = (uint32_t)(i >> 1);
            int have_planes = 0;
            uint64_t planes[32];
            for (int j = 0; j < 64 && rb + j < nrep; ++j) {
                int8_t* sr = s + (size_t)(rb + j) * c->N;
                int n_unsat = 0;
                for (int nb = 0; nb < twoD; ++nb) {
                    int jsign = c->J[c->bond[i * twoD + nb]] > 0.0f ? 1 : -1;
                    if (jsign * sr[i] * sr[c->nbr[i * twoD + nb]] < 0) ++n_unsat;
                }
                int dE = 4 * c->D - 4 * n_unsat;
                int flip;
                if (dE <= 0) {
                    flip = 1;
                } else {
                    if (!have_planes) {
                        for (uint32_t m = 0; m < 16; ++m) {
                            uint32_t ctr[4] = {q, (uint32_t)hs, 16u * (uint32_t)g + m, c3}, out[4];
                            or_philox4x32_10(ctr, c->key, out);
                            planes[2 * m] = (uint64_t)out[0] | ((uint64_t)out[1] << 32);
                            planes[2 * m + 1] = (uint64_t)out[2] | ((uint64_t)out[3] << 32);
                        }
                        have_planes = 1;
                    }
                    uint64_t r = 0;
                    for (int b = 0; b < 32; ++b) r |= ((planes[b] >> j) & 1u) << (31 - b);
                    flip = r < thr[dE / 4];
                }
                if (flip) sr[i] = (int8_t)-sr[i];
            }
        }
    }
}

/* real couplings: local field f = ((((t_-x + t_+x) + t_-y) + t_+y) + ...) + h_i
 * in FP32 with t = J S_nb (exact sign flip); dE = 2 S_i f (exact);
 * x = f32(beta) * dE (FP32); accept iff x <= 0 or r < floor(expf(-x) 2^32). */
static void halfsweep_real(const lat_ctx* c, int8_t* s, int r0, int nrep, double beta, int hs,
                           int parity)
{
    uint32_t c3 = or_counter3(OR_STREAM_WORD, c->tag, c->inst);
    float bf = (float)beta;
    int twoD = 2 * c->D;
    for (int rr = 0; rr < nrep; ++rr) {
        int8_t* sr = s + (size_t)rr * c->N;
        uint32_t rho = (uint32_t)(r0 + rr);
        for (int i = 0; i < c->N; ++i) {
            if (parity_of(i, c->D, c->L) != parity) continue;
            uint32_t q = (uint32_t)(i >> 1);
            uint32_t ctr[4] = {q >> 2, (uint32_t)hs, rho, c3}, out[4];
            or_philox4x32_10(ctr, c->key, out);
            uint32_t r = out[q & 3u];
            float f = 0.0f;
            for (int nb = 0; nb < twoD; ++nb) {
                float Jb = c->J[c->bond[i * twoD + nb]];
                float t = sr[c->nbr[i * twoD + nb]] > 0 ? Jb : -Jb;
                f = (nb == 0) ? t : f + t;
            }
            f = f + (c->h ? c->h[i] : 0.0f);
            float dE = sr[i] > 0 ? 2.0f * f : -2.0f * f;
            float x = bf * dE;
            int flip = (x <= 0.0f) || ((uint64_t)r < or_threshold_real(x));
            if (flip) sr[i] = (int8_t)-sr[i];
        }
    }
}

/* sweeps sw0 .. sw1-1 of the n_sweeps at step k (half-sweep index
 * hs = 2 (k n_sweeps + sw) + parity whatever the split) */
static void sweeps_range(const lat_ctx* c, int kind, int8_t* s, int r0, int nrep, double beta, int k,
                         int n_sweeps, int sw0, int sw1)
{
    for (int sw = sw0; sw < sw1; ++sw)
        for (int p = 0; p < 2; ++p) {
            int hs = 2 * (k * n_sweeps + sw) + p;
            if (kind == OR_PM1)
                halfsweep_pm(c, s, r0, nrep, beta, hs, p);
            else
                halfsweep_real(c, s, r0, nrep, beta, hs, p);
        }
}

static void sweeps(const lat_ctx* c, int kind, int8_t* s, int r0, int nrep, double beta, int k,
                   int n_sweeps)
{
    for (int sw = 0; sw < n_sweeps; ++sw)
        for (int p = 0; p < 2; ++p) {
            int hs = 2 * (k * n_sweeps + sw) + p;
            if (kind == OR_PM1)
                halfsweep_pm(c, s, r0, nrep, beta, hs, p);
            else
                halfsweep_real(c, s, r0, nrep, beta, hs, p);
        }
}

/* ---------------- isoenergetic cluster moves (Sec. II.C) ----------------
 *
 * Two replicas a, b: the overlap q_i = S^a_i S^b_i splits the lattice into
 * islands (connected sets of sites of equal q).  One island is drawn from
 * the sector (q = -1 or q = +1) with fewer sites (ties: q = -1), its spins
 * are flipped in both replicas; E_a + E_b is unchanged for a zero field, so
 * the move is always accepted.  The island is the lattice-connected
 * component, in that sector, of the idx-th sector site in site order,
 * idx = floor(r32 n_sector / 2^32).
 *
 * Random pairing: round t of step k pairs pi_t(2i) with pi_t(2i+1),
 * i < floor(R/2), where pi_t is a 4-round Feistel permutation of
 * [0, 2^m) (m even, the smallest with 2^m >= R, at least 2) walked in
 * cycles back into [0, R): halves of m/2 bits, (Lh, Rh) -> (Rh, Lh ^ F_j(Rh)),
 * F_j(v) = out0 of Philox at counter (v, k, 4t + j, ICM stream) masked to
 * m/2 bits.  The site-choice word of pair i in round t is out0 at counter
 * (i, k, 16 + t, ICM stream). */

static uint32_t icm_feistel(uint32_t x, int h, int k, int t, const uint32_t key[2], uint32_t c3)
{
    const uint32_t mask = (h >= 32) ? 0xFFFFFFFFu : ((1u << h) - 1u);
    uint32_t Lh = (x >> h) & mask, Rh = x & mask;
    for (int j = 0; j < 4; ++j) {
        uint32_t ctr[4] = {Rh, (uint32_t)k, (uint32_t)(4 * t + j), c3}, out[4];
        or_philox4x32_10(ctr, key, out);
        uint32_t nl = Rh, nr = Lh ^ (out[0] & mask);
        Lh = nl;
        Rh = nr;
    }
    return (Lh << h) | Rh;
}

uint32_t or_icm_perm(uint32_t i, uint32_t n, int k, int t, uint64_t seed, uint32_t inst, uint32_t tag)
{
    int m = 2;
    while (m < 32 && (1ull << m) < (unsigned long long)n) m += 2;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t c3 = or_counter3(OR_STREAM_ICM, tag, inst);
    uint32_t y = icm_feistel(i, m / 2, k, t, key, c3);
    while (y >= n) y = icm_feistel(y, m / 2, k, t, key, c3);
    return y;
}

int or_icm_pair(int D, int L, int8_t* a, int8_t* b, uint32_t r32)
{
    int N = ipow(L, D);
    int32_t* nbr = (int32_t*)malloc(sizeof(int32_t) * (size_t)N * 2 * D);
    int32_t* bond = (int32_t*)malloc(sizeof(int32_t) * (size_t)N * 2 * D);
    or_lattice(D, L, nbr, bond);
    int nneg = 0;
    for (int i = 0; i < N; ++i) nneg += (a[i] * b[i] < 0);
    int sigma = (nneg <= N - nneg) ? -1 : 1;
    int nsec = sigma < 0 ? nneg : N - nneg;
    int size = 0;
    if (nsec > 0) {
        uint32_t idx = (uint32_t)(((uint64_t)r32 * (uint64_t)nsec) >> 32);
        int c = -1;
        for (int i = 0, seen = 0; i < N; ++i)
            if (a[i] * b[i] == sigma) {
                if ((uint32_t)seen == idx) { c = i; break; }
                ++seen;
            }
        /* breadth-first search of the island of c */
        int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
        uint8_t* in = (uint8_t*)calloc((size_t)N, 1);
        int head = 0, tail = 0;
        queue[tail++] = c;
        in[c] = 1;
        while (head < tail) {
            int i = queue[head++];
            for (int nb = 0; nb < 2 * D; ++nb) {
                int j = nbr[i * 2 * D + nb];
                if (!in[j] && a[j] * b[j] == sigma) {
                    in[j] = 1;
                    queue[tail++] = j;
                }
            }
        }
        for (int q = 0; q < tail; ++q) {
            a[queue[q]] = (int8_t)-a[queue[q]];
            b[queue[q]] = (int8_t)-b[queue[q]];
        }
        size = tail;
        free(queue);
        free(in);
    }
    free(nbr);
    free(bond);
    return size;
}

static void icm_rounds(or_sim* s, int k)
{
    uint32_t key[2] = {(uint32_t)s->seed, (uint32_t)(s->seed >> 32)};
    uint32_t c3 = or_counter3(OR_STREAM_ICM, s->tag, s->inst);
    for (int t = 0; t < 2; ++t)
        for (int i = 0; i < s->R / 2; ++i) {
            uint32_t pa_ = or_icm_perm((uint32_t)(2 * i), (uint32_t)s->R, k, t, s->seed, s->inst, s->tag);
            uint32_t pb_ = or_icm_perm((uint32_t)(2 * i + 1), (uint32_t)s->R, k, t, s->seed, s->inst, s->tag);
            uint32_t ctr[4] = {(uint32_t)i, (uint32_t)k, (uint32_t)(16 + t), c3}, out[4];
            or_philox4x32_10(ctr, key, out);
            or_icm_pair(s->D, s->L, s->s + (size_t)pa_ * s->N, s->s + (size_t)pb_ * s->N, out[0]);
        }
}

int or_set_icm(or_sim* s, int enable, double icm_beta_lo, double icm_beta_hi)
{
    if (enable && s->h)
        for (int i = 0; i < s->N; ++i)
            if (s->h[i] != 0.0f) return -1; /* the moves conserve energy only without a field */
    s->icm = enable ? 1 : 0;
    s->icm_lo = icm_beta_lo;
    s->icm_hi = icm_beta_hi;
    return 0;
}

/* ---------------- energies (Eq. 1 plus field) ---------------- */

static i128 energy_one(const lat_ctx* c, int kind, const int8_t* sr)
{
    i128 e = 0;
    for (int i = 0; i < c->N; ++i) {
        for (int d = 0; d < c->D; ++d) {
            int b = d * c->N + i;
            int j = c->nbr[i * 2 * c->D + 2 * d + 1];
            int ss = sr[i] * sr[j];
            if (kind == OR_PM1)
                e -= (i128)((c->J[b] > 0.0f ? 1 : -1) * ss);
            else
                e -= (ss > 0) ? fix96(c->J[b]) : -fix96(c->J[b]);
        }
        if (kind == OR_REAL && c->h) e -= (sr[i] > 0) ? fix96(c->h[i]) : -fix96(c->h[i]);
    }
    return e;
}

/* ---------------- resampling (Sec. II.B) ---------------- */

/* Fan-out of the fixed summation order of the resampling weights. */
#define OR_FANOUT 32

/* Inclusive prefix sums of x[0..n) in a fixed hierarchical order (a reading
 * of Sec. II.B, which fixes only the normalisation S = sum w): runs of
 * OR_FANOUT consecutive entries are summed sequentially (left to right, the
 * first term taken as is); the run totals form a sequence that is summed the
 * same way, recursively, until one run is left; entry j of run c is then
 * Q_{c-1} + l_j, with l_j its sum inside the run and Q_{c-1} the inclusive
 * prefix of the run totals before run c (entries of run 0 are l_j alone). */
static void prefix_fixed_order(const double* x, int n, double* out)
{
    if (n <= OR_FANOUT) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j) {
            acc = (j == 0) ? x[j] : acc + x[j];
            out[j] = acc;
        }
        return;
    }
    int m = (n + OR_FANOUT - 1) / OR_FANOUT;
    double* tot = (double*)malloc(sizeof(double) * (size_t)m);
    double* Q = (double*)malloc(sizeof(double) * (size_t)m);
    for (int c = 0; c < m; ++c) {
        int j0 = c * OR_FANOUT, j1 = j0 + OR_FANOUT < n ? j0 + OR_FANOUT : n;
        double acc = 0.0;
        for (int j = j0; j < j1; ++j) {
            acc = (j == j0) ? x[j] : acc + x[j];
            out[j] = acc;
        }
        tot[c] = acc;
    }
    prefix_fixed_order(tot, m, Q);
    for (int j = OR_FANOUT; j < n; ++j) out[j] = Q[j / OR_FANOUT - 1] + out[j];
    free(tot);
    free(Q);
}

/* The cumulative weights the draws search: the fixed-order prefix sums made
 * non-decreasing by a running maximum (exact in floating point; rounding in
 * two different orders can leave the last sum of a run one unit above the
 * first of the next), P_i = max_{j <= i} prefix_j.  S = P_{R-1}. */
static void cumulative_weights(const double* w, int R, double* P)
{
    prefix_fixed_order(w, R, P);
    for (int i = 1; i < R; ++i)
        if (P[i] < P[i - 1]) P[i] = P[i - 1];
}

void or_weight_prefix(const double* w, int n, double* P_out, double* prefix_out)
{
    if (prefix_out) prefix_fixed_order(w, n, prefix_out);
    cumulative_weights(w, n, P_out);
}

static double e_to_double(int kind, i128 v)
{
    return (kind == OR_PM1) ? (double)v : (double)v * 0x1p-96;
}

/* Resampling R (source replicas) -> Rn (new population): Rn multinomial draws
 * with probabilities w_i / S, so replica i gets Rn w_i / S copies on average
 * and the expected new population is Rn (Sec. II.B; Rn = R(beta') of Sec.
 * III.D, Eq. 6, for a dynamic population).  Q averages over the R sources. */
static int resample_core2(int kind, int R, int Rn, const i128* E, double beta_prev, double beta_next,
                          int k, uint64_t seed, uint32_t inst, uint32_t tag, double* w, double* P,
                          int32_t* parent, int32_t* counts, double* lnQ, double* u_out)
{
    double db = beta_next - beta_prev;
    i128 emin = E[0];
    for (int r = 1; r < R; ++r)
        if (E[r] < emin) emin = E[r];
    /* weights relative to the lowest energy: w_r = exp(-db (E_r - E_min)) */
    for (int r = 0; r < R; ++r) w[r] = or_spec_exp64(-(db * e_to_double(kind, E[r] - emin)));
    /* cumulative weights in the fixed order, S their last entry */
    cumulative_weights(w, R, P);
    double S = P[R - 1];
    *lnQ = (-(db * e_to_double(kind, emin)) + log(S)) - log((double)R);
    /* multinomial draws: parent of draw q = smallest i with u_q S < P_i */
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t c3 = or_counter3(OR_STREAM_RESAMPLE, tag, inst);
    memset(counts, 0, sizeof(int32_t) * (size_t)R);
    for (int q = 0; q < Rn; ++q) {
        uint32_t ctr[4] = {(uint32_t)q, (uint32_t)k, 0u, c3}, out[4];
        or_philox4x32_10(ctr, key, out);
        double u = or_uniform53(out[0], out[1]);
        if (u_out) u_out[q] = u;
        double x = u * S;
        int lo = 0, hi = R; /* first index with P > x */
        while (lo < hi) {
            int mid = lo + (hi - lo) / 2;
            if (x < P[mid]) hi = mid; else lo = mid + 1;
        }
        if (lo == R) { /* x == S after rounding: first index with P >= x */
            lo = 0; hi = R;
            while (lo < hi) {
                int mid = lo + (hi - lo) / 2;
                if (P[mid] >= x) hi = mid; else lo = mid + 1;
            }
        }
        counts[lo] += 1;
    }
    /* slots [C_i, C_i + n_i) receive replica i: families stay contiguous */
    int j = 0;
    for (int i = 0; i < R; ++i)
        for (int t = 0; t < counts[i]; ++t) parent[j++] = i;
    return j == Rn ? 0 : -1;
}

/* Nearest-integer resampling R sources -> population conserved in expectation
 * (Sec. II.B: the mean number of copies of replica i is proportional to
 * exp[-(beta'-beta) E_i], normalised so that the expected new population is
 * the target T = R(beta')).  tau_i = T w_i / S; replica i gets floor(tau_i)
 * copies plus one more with probability tau_i - floor(tau_i) (uniform u_i of
 * the RESAMPLE stream, counter (i, k, 1)).  Copies are placed as in the
 * multinomial scheme; slots beyond the capacity are dropped.  Returns the new
 * population min(sum n_i, cap). */
static int resample_nearest(int kind, int R, double target, int cap, const i128* E, double beta_prev,
                            double beta_next, int k, uint64_t seed, uint32_t inst, uint32_t tag,
                            double* w, double* P, int32_t* parent, int32_t* counts, double* lnQ)
{
    double db = beta_next - beta_prev;
    i128 emin = E[0];
    for (int r = 1; r < R; ++r)
        if (E[r] < emin) emin = E[r];
    for (int r = 0; r < R; ++r) w[r] = or_spec_exp64(-(db * e_to_double(kind, E[r] - emin)));
    /* cumulative weights in the fixed order, S their last entry */
    cumulative_weights(w, R, P);
    double S = P[R - 1];
    *lnQ = (-(db * e_to_double(kind, emin)) + log(S)) - log((double)R);
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t c3 = or_counter3(OR_STREAM_RESAMPLE, tag, inst);
    for (int i = 0; i < R; ++i) {
        uint32_t ctr[4] = {(uint32_t)i, (uint32_t)k, 1u, c3}, out[4];
        or_philox4x32_10(ctr, key, out);
        double u = or_uniform53(out[0], out[1]);
        double tau = (target * w[i]) / S;
        double fl = floor(tau);
        counts[i] = (int32_t)fl + (u < tau - fl ? 1 : 0);
    }
    int j = 0;
    for (int i = 0; i < R; ++i)
        for (int t = 0; t < counts[i]; ++t) {
            if (j < cap) parent[j] = i;
            ++j;
        }
    return j < cap ? j : cap;
}

static int resample_core(int kind, int R, const i128* E, double beta_prev, double beta_next, int k,
                         uint64_t seed, uint32_t inst, uint32_t tag, double* w, double* P,
                         int32_t* parent, int32_t* counts, double* lnQ, double* u_out)
{
    return resample_core2(kind, R, R, E, beta_prev, beta_next, k, seed, inst, tag, w, P, parent,
                          counts, lnQ, u_out);
}

int or_resample(int kind, int R, const int64_t* E, double beta_prev, double beta_next, int k,
                uint64_t seed, uint32_t inst, uint32_t tag, double* w, double* P, int32_t* parent,
                int32_t* counts, double* lnQ, double* u_out)
{
    i128* e = (i128*)malloc(sizeof(i128) * (size_t)R);
    if (!e) return -1;
    for (int r = 0; r < R; ++r)
        e[r] = (i128)(((unsigned __int128)(uint64_t)E[2 * r + 1] << 64) | (uint64_t)E[2 * r]);
    int rc = resample_core(kind, R, e, beta_prev, beta_next, k, seed, inst, tag, w, P, parent,
                           counts, lnQ, u_out);
    free(e);
    return rc;
}

int or_resample_nearest(int kind, int R, const int64_t* E, double beta_prev, double beta_next, int k,
                        uint64_t seed, uint32_t inst, uint32_t tag, double target, int cap,
                        double* w, double* P, int32_t* parent, int32_t* counts, double* lnQ)
{
    i128* e = (i128*)malloc(sizeof(i128) * (size_t)R);
    if (!e) return -1;
    for (int r = 0; r < R; ++r)
        e[r] = (i128)(((unsigned __int128)(uint64_t)E[2 * r + 1] << 64) | (uint64_t)E[2 * r]);
    int Rn = resample_nearest(kind, R, target, cap, e, beta_prev, beta_next, k, seed, inst, tag, w, P,
                              parent, counts, lnQ);
    free(e);
    return Rn;
}

/* ---------------- the run ---------------- */

static lat_ctx lat_of(const or_sim* s)
{
    lat_ctx c;
    c.D = s->D; c.L = s->L; c.N = s->N;
    c.nbr = s->nbr; c.bond = s->bond; c.J = s->J; c.h = s->h;
    c.key[0] = (uint32_t)s->seed; c.key[1] = (uint32_t)(s->seed >> 32);
    c.inst = s->inst; c.tag = s->tag;
    return c;
}

or_sim* or_create(int D, int L, int kind, const float* J, const float* h, int R,
                  const double* betas, int n_temps, int n_sweeps, uint64_t seed,
                  uint32_t rng_instance, uint32_t rng_tag, int accumulate_grad)
{
    return or_create_dps(D, L, kind, J, h, R, betas, n_temps, n_sweeps, seed, rng_instance, rng_tag,
                         accumulate_grad, NULL);
}

or_sim* or_create_dps(int D, int L, int kind, const float* J, const float* h, int R,
                      const double* betas, int n_temps, int n_sweeps, uint64_t seed,
                      uint32_t rng_instance, uint32_t rng_tag, int accumulate_grad,
                      const int32_t* populations)
{
    return or_create_ex(D, L, kind, J, h, R, betas, n_temps, n_sweeps, seed, rng_instance, rng_tag,
                        accumulate_grad, populations, OR_RESAMPLE_MULTINOMIAL, 0);
}

int or_default_capacity(int R_max) { return R_max + 64 + 8 * (int)ceil(sqrt((double)R_max)); }

or_sim* or_create_ex(int D, int L, int kind, const float* J, const float* h, int R,
                     const double* betas, int n_temps, int n_sweeps, uint64_t seed,
                     uint32_t rng_instance, uint32_t rng_tag, int accumulate_grad,
                     const int32_t* populations, int scheme, int capacity)
{
    if (R < 1 || n_temps < 1 || capacity < 0) return NULL;
    if (scheme != OR_RESAMPLE_MULTINOMIAL && scheme != OR_RESAMPLE_NEAREST) return NULL;
    int tmax = R;
    if (populations) {
        tmax = 0;
        for (int k = 0; k < n_temps; ++k) {
            if (populations[k] < 1) return NULL;
            if (populations[k] > tmax) tmax = populations[k];
        }
    }
    int cap;
    if (scheme == OR_RESAMPLE_MULTINOMIAL) {
        /* exact populations: R (or the given capacity) bounds them */
        cap = capacity > R ? capacity : R;
        if (tmax > cap) return NULL;
    } else {
        cap = capacity > 0 ? capacity : or_default_capacity(tmax);
        if (tmax > cap) return NULL;
    }
    if (D < 2 || D > 3 || L < 2 || (L & 1) || n_temps < 1 || n_sweeps < 0) return NULL;
    if (kind != OR_PM1 && kind != OR_REAL) return NULL;
    if (betas[0] != 0.0) return NULL;
    for (int k = 1; k < n_temps; ++k)
        if (!(betas[k] >= betas[k - 1]) || !isfinite(betas[k])) return NULL;
    or_sim* s = (or_sim*)calloc(1, sizeof(or_sim));
    int N = ipow(L, D);
    s->D = D; s->L = L; s->N = N; s->kind = kind; s->R = R; s->G = (R + 63) / 64;
    s->Rcap = cap; s->R_src_last = R; s->scheme = scheme; s->dead = 0;
    s->Rk = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_temps);
    for (int k = 0; k < n_temps; ++k) s->Rk[k] = populations ? populations[k] : R;
    s->n_temps = n_temps; s->n_sweeps = n_sweeps; s->k_next = 0; s->acc_grad = accumulate_grad;
    s->seed = seed; s->inst = rng_instance; s->tag = rng_tag;
    s->J = (float*)malloc(sizeof(float) * (size_t)D * N);
    s->h = (kind == OR_REAL && h) ? (float*)malloc(sizeof(float) * (size_t)N) : NULL;
    for (int b = 0; b < D * N; ++b) {
        float v = J[b];
        if (!isfinite(v)) goto fail;
        if (kind == OR_PM1 && v != 1.0f && v != -1.0f) goto fail;
        if (kind == OR_REAL && fabsf(v) >= 4096.0f) goto fail;
        s->J[b] = kind == OR_REAL ? flush_real(v) : v;
    }
    if (kind == OR_PM1 && h)
        for (int i = 0; i < N; ++i)
            if (h[i] != 0.0f) goto fail;
    if (s->h)
        for (int i = 0; i < N; ++i) {
            if (!isfinite(h[i]) || fabsf(h[i]) >= 4096.0f) goto fail;
            s->h[i] = flush_real(h[i]);
        }
    s->betas = (double*)malloc(sizeof(double) * (size_t)n_temps);
    memcpy(s->betas, betas, sizeof(double) * (size_t)n_temps);
    s->nbr = (int32_t*)malloc(sizeof(int32_t) * (size_t)N * 2 * D);
    s->bond = (int32_t*)malloc(sizeof(int32_t) * (size_t)N * 2 * D);
    or_lattice(D, L, s->nbr, s->bond);
    s->s = (int8_t*)malloc((size_t)cap * N);
    s->tmp = (int8_t*)malloc((size_t)cap * N);
    s->E = (i128*)calloc((size_t)cap, sizeof(i128));
    s->parent = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
    s->family = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
    s->family_tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
    s->counts = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
    s->w = (double*)calloc((size_t)cap, sizeof(double));
    s->P = (double*)calloc((size_t)cap, sizeof(double));
    s->obs = (double*)calloc((size_t)n_temps * 8, sizeof(double));
    if (accumulate_grad) {
        s->cJ = (int64_t*)calloc((size_t)n_temps * D * N, sizeof(int64_t));
        s->ch = (int64_t*)calloc((size_t)n_temps * N, sizeof(int64_t));
    }
    return s;
fail:
    free(s->J);
    free(s->h);
    free(s);
    return NULL;
}

void or_destroy(or_sim* s)
{
    if (!s) return;
    free(s->J); free(s->h); free(s->betas); free(s->nbr); free(s->bond);
    free(s->s); free(s->tmp); free(s->E); free(s->parent); free(s->family);
    free(s->family_tmp); free(s->counts); free(s->w); free(s->P); free(s->obs);
    free(s->cJ); free(s->ch); free(s->Rk);
    free(s);
}

/* Population sums for the gradient of beta F (from Eq. 1 with the field term
 * and Z = sum exp(-beta H)): c_b += sum_r S_i S_{i+e_d} for bond b = d N + i,
 * m_i += sum_r S_i, over R replicas given as int8 rows. */
static void grad_counts_add(int D, int N, const int32_t* nbr, int R, const int8_t* spins,
                            int64_t* cJ, int64_t* ch)
{
    for (int r = 0; r < R; ++r) {
        const int8_t* sr = spins + (size_t)r * N;
        for (int i = 0; i < N; ++i) {
            ch[i] += sr[i];
            for (int d = 0; d < D; ++d)
                cJ[d * N + i] += sr[i] * sr[nbr[i * 2 * D + 2 * d + 1]];
        }
    }
}

static void measure(or_sim* s, int k, double lnQ)
{
    lat_ctx c = lat_of(s);
    for (int r = 0; r < s->R; ++r) s->E[r] = energy_one(&c, s->kind, s->s + (size_t)r * s->N);
    double Em, E2m;
    if (s->kind == OR_PM1) {
        int64_t se = 0, se2 = 0;
        for (int r = 0; r < s->R; ++r) {
            int64_t e = (int64_t)s->E[r];
            se += e;
            se2 += e * e;
        }
        Em = (double)se / s->R;
        E2m = (double)se2 / s->R;
    } else {
        double se = 0.0, se2 = 0.0;
        for (int r = 0; r < s->R; ++r) {
            double e = e_to_double(s->kind, s->E[r]);
            se += e;
            se2 += e * e;
        }
        Em = se / s->R;
        E2m = se2 / s->R;
    }
    double beta = s->betas[k];
    s->sum_lnQ += lnQ;
    double Sf = 0.0;
    for (int r = 0; r < s->R;) {
        int t = r;
        while (t < s->R && s->family[t] == s->family[r]) ++t;
        double nu = (double)(t - r) / s->R;
        Sf -= nu * log(nu);
        r = t;
    }
    double* o = s->obs + (size_t)k * 8;
    o[0] = Em;
    o[1] = E2m;
    o[2] = beta * beta * (E2m - Em * Em) / s->N;
    o[3] = lnQ;
    o[4] = -(double)s->N * log(2.0) - s->sum_lnQ;
    o[5] = Sf;
    o[6] = (double)s->R / exp(Sf);
    o[7] = (double)s->R;
    if (s->acc_grad)
        grad_counts_add(s->D, s->N, s->nbr, s->R, s->s, s->cJ + (size_t)k * s->D * s->N,
                        s->ch + (size_t)k * s->N);
}

int or_step(or_sim* s)
{
    int k = s->k_next;
    if (s->dead) return -2;
    if (k >= s->n_temps) return -1;
    double lnQ = 0.0;
    if (k == 0) {
        s->R = s->Rk[0];
        init_spins(s->N, s->R, s->seed, s->inst, s->tag, s->s);
        for (int r = 0; r < s->R; ++r) s->family[r] = s->parent[r] = r;
    } else {
        int Rn = s->Rk[k];
        if (s->scheme == OR_RESAMPLE_NEAREST) {
            Rn = resample_nearest(s->kind, s->R, (double)s->Rk[k], s->Rcap, s->E, s->betas[k - 1],
                                  s->betas[k], k, s->seed, s->inst, s->tag, s->w, s->P, s->parent,
                                  s->counts, &lnQ);
            if (Rn == 0) { /* every replica left without copies: the run ends */
                s->dead = 1;
                s->R_src_last = s->R;
                s->R = 0;
                s->k_next = k + 1;
                return -2;
            }
        } else {
            resample_core2(s->kind, s->R, Rn, s->E, s->betas[k - 1], s->betas[k], k, s->seed, s->inst,
                           s->tag, s->w, s->P, s->parent, s->counts, &lnQ, NULL);
        }
        s->R_src_last = s->R;
        s->R = Rn;
        for (int j = 0; j < s->R; ++j) {
            memcpy(s->tmp + (size_t)j * s->N, s->s + (size_t)s->parent[j] * s->N, (size_t)s->N);
            s->family_tmp[j] = s->family[s->parent[j]];
        }
        int8_t* t = s->s; s->s = s->tmp; s->tmp = t;
        int32_t* f = s->family; s->family = s->family_tmp; s->family_tmp = f;
    }
    lat_ctx c = lat_of(s);
    const double beta = s->betas[k];
    if (s->icm && k > 0 && beta >= s->icm_lo && (s->icm_hi <= 0.0 || beta <= s->icm_hi)) {
        const int h1 = s->n_sweeps / 2;
        sweeps_range(&c, s->kind, s->s, 0, s->R, beta, k, s->n_sweeps, 0, h1);
        icm_rounds(s, k);
        sweeps_range(&c, s->kind, s->s, 0, s->R, beta, k, s->n_sweeps, h1, s->n_sweeps);
    } else {
        sweeps(&c, s->kind, s->s, 0, s->R, beta, k, s->n_sweeps);
    }
    measure(s, k, lnQ);
    s->k_next = k + 1;
    return k;
}

int or_next_step(const or_sim* s) { return s->k_next; }
int or_N(const or_sim* s) { return s->N; }

void or_get_spins(const or_sim* s, int8_t* out) { memcpy(out, s->s, (size_t)s->R * s->N); }
void or_set_spins(or_sim* s, const int8_t* in) { memcpy(s->s, in, (size_t)s->R * s->N); }

void or_get_energies(const or_sim* s, int64_t* out)
{
    for (int r = 0; r < s->R; ++r) {
        unsigned __int128 u = (unsigned __int128)s->E[r];
        out[2 * r] = (int64_t)(uint64_t)u;
        out[2 * r + 1] = (int64_t)(uint64_t)(u >> 64);
    }
}

void or_get_parents(const or_sim* s, int32_t* out) { memcpy(out, s->parent, sizeof(int32_t) * (size_t)s->R); }
void or_get_family(const or_sim* s, int32_t* out) { memcpy(out, s->family, sizeof(int32_t) * (size_t)s->R); }
void or_get_weights(const or_sim* s, double* w, double* P)
{
    memcpy(w, s->w, sizeof(double) * (size_t)s->R_src_last);
    memcpy(P, s->P, sizeof(double) * (size_t)s->R_src_last);
}

int or_current_R(const or_sim* s) { return s->R; }
void or_get_obs(const or_sim* s, int k, double* out) { memcpy(out, s->obs + (size_t)k * 8, 8 * sizeof(double)); }
void or_get_grad_counts(const or_sim* s, int64_t* cJ, int64_t* ch)
{
    if (!s->acc_grad) return;
    memcpy(cJ, s->cJ, sizeof(int64_t) * (size_t)s->n_temps * s->D * s->N);
    memcpy(ch, s->ch, sizeof(int64_t) * (size_t)s->n_temps * s->N);
}

/* ---------------- components on explicit state ---------------- */

int or_sweeps_groups(int D, int L, int kind, const float* J, const float* h, double beta, int k,
                     int n_sweeps, uint64_t seed, uint32_t inst, uint32_t tag, int g0, int ng,
                     int R, int8_t* state)
{
    int N = ipow(L, D);
    lat_ctx c;
    int32_t* nbr = (int32_t*)malloc(sizeof(int32_t) * (size_t)N * 2 * D);
    int32_t* bond = (int32_t*)malloc(sizeof(int32_t) * (size_t)N * 2 * D);
    float* Jf = (float*)malloc(sizeof(float) * (size_t)D * N);
    float* hf = (kind == OR_REAL && h) ? (float*)malloc(sizeof(float) * (size_t)N) : NULL;
    or_lattice(D, L, nbr, bond);
    for (int b = 0; b < D * N; ++b) Jf[b] = kind == OR_REAL ? flush_real(J[b]) : J[b];
    if (hf)
        for (int i = 0; i < N; ++i) hf[i] = flush_real(h[i]);
    c.D = D; c.L = L; c.N = N; c.nbr = nbr; c.bond = bond; c.J = Jf; c.h = hf;
    c.key[0] = (uint32_t)seed; c.key[1] = (uint32_t)(seed >> 32); c.inst = inst; c.tag = tag;
    int r0 = 64 * g0;
    int r1 = 64 * (g0 + ng) < R ? 64 * (g0 + ng) : R;
    sweeps(&c, kind, state, r0, r1 - r0, beta, k, n_sweeps);
    free(nbr); free(bond); free(Jf); free(hf);
    return r1 - r0;
}

void or_energies(int D, int L, int kind, const float* J, const float* h, int R,
                 const int8_t* spins, int64_t* E)
{
    int N = ipow(L, D);
    lat_ctx c;
    int32_t* nbr = (int32_t*)malloc(sizeof(int32_t) * (size_t)N * 2 * D);
    int32_t* bond = (int32_t*)malloc(sizeof(int32_t) * (size_t)N * 2 * D);
    float* Jf = (float*)malloc(sizeof(float) * (size_t)D * N);
    float* hf = (kind == OR_REAL && h) ? (float*)malloc(sizeof(float) * (size_t)N) : NULL;
    or_lattice(D, L, nbr, bond);
    for (int b = 0; b < D * N; ++b) Jf[b] = kind == OR_REAL ? flush_real(J[b]) : J[b];
    if (hf)
        for (int i = 0; i < N; ++i) hf[i] = flush_real(h[i]);
    c.D = D; c.L = L; c.N = N; c.nbr = nbr; c.bond = bond; c.J = Jf; c.h = hf;
    for (int r = 0; r < R; ++r) {
        unsigned __int128 u = (unsigned __int128)energy_one(&c, kind, spins + (size_t)r * N);
        E[2 * r] = (int64_t)(uint64_t)u;
        E[2 * r + 1] = (int64_t)(uint64_t)(u >> 64);
    }
    free(nbr); free(bond); free(Jf); free(hf);
}

/* Sec. V.A: overlap q_r = (1/N) sum_i S^A_i S^B_i; histogram index
 * (N + sum_i S^A_i S^B_i)/2 = N - n_diff. */
int or_overlap(int N, int R, const int8_t* a, const int8_t* b, int64_t* hist)
{
    memset(hist, 0, sizeof(int64_t) * (size_t)(N + 1));
    for (int r = 0; r < R; ++r) {
        int ndiff = 0;
        for (int i = 0; i < N; ++i) ndiff += a[(size_t)r * N + i] != b[(size_t)r * N + i];
        hist[N - ndiff] += 1;
    }
    return 0;
}

/* Gradient counts of one population given as int8 rows (R x N): cJ (D*N) and
 * ch (N) are overwritten with sum_r S_i S_{i+e_d} and sum_r S_i. */
int or_grad_counts(int D, int L, int R, const int8_t* spins, int64_t* cJ, int64_t* ch)
{
    int N = ipow(L, D);
    int32_t* nbr = (int32_t*)malloc(sizeof(int32_t) * (size_t)N * 2 * D);
    int32_t* bond = (int32_t*)malloc(sizeof(int32_t) * (size_t)N * 2 * D);
    if (!nbr || !bond) { free(nbr); free(bond); return -1; }
    or_lattice(D, L, nbr, bond);
    memset(cJ, 0, sizeof(int64_t) * (size_t)D * N);
    memset(ch, 0, sizeof(int64_t) * (size_t)N);
    grad_counts_add(D, N, nbr, R, spins, cJ, ch);
    free(nbr); free(bond);
    return 0;
}
