/*
 * exact.c -- brute-force enumeration of all 2^N spin states (N <= 24).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  This is the definition of the
 * canonical ensemble of Eq. (1) (plus the field term) written out:
 *   Z(beta) = sum_s exp(-beta H(s)),  beta F = -ln Z,
 *   <E> = sum_s H(s) e^{-beta H} / Z,  C = beta^2 (<E^2> - <E>^2) / N,
 *   <s_i s_j> and <s_i> as Boltzmann averages.
 * Couplings are taken in binary64 so that tests can differentiate in J.
 * Sums use long double accumulators; exponentials are shifted by the ground
 * state energy (log-sum-exp).
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>

int or_exact(int D, int L, const double* J, const double* h, int n_betas, const double* betas,
             double* out, double* corr, double* mag)
{
    int N = 1;
    for (int d = 0; d < D; ++d) N *= L;
    if (N > 24 || N < 1) return -1;
    int32_t* nbr = (int32_t*)malloc(sizeof(int32_t) * (size_t)N * 2 * D);
    int32_t* bond = (int32_t*)malloc(sizeof(int32_t) * (size_t)N * 2 * D);
    or_lattice(D, L, nbr, bond);
    size_t ns = (size_t)1 << N;
    double* E = (double*)malloc(sizeof(double) * ns);
    double emin = INFINITY;
    for (size_t st = 0; st < ns; ++st) {
        double e = 0.0;
        for (int i = 0; i < N; ++i) {
            int si = ((st >> i) & 1u) ? -1 : 1;
            for (int d = 0; d < D; ++d) {
                int j = nbr[i * 2 * D + 2 * d + 1];
                int sj = ((st >> j) & 1u) ? -1 : 1;
                e -= J[d * N + i] * (double)(si * sj);
            }
            if (h) e -= h[i] * (double)si;
        }
        E[st] = e;
        if (e < emin) emin = e;
    }
    int nb = D * N;
    long double* ac = corr ? (long double*)malloc(sizeof(long double) * (size_t)nb) : NULL;
    long double* am = mag ? (long double*)malloc(sizeof(long double) * (size_t)N) : NULL;
    for (int t = 0; t < n_betas; ++t) {
        double beta = betas[t];
        long double z = 0.0L, s1 = 0.0L;
        if (ac) for (int b = 0; b < nb; ++b) ac[b] = 0.0L;
        if (am) for (int i = 0; i < N; ++i) am[i] = 0.0L;
        for (size_t st = 0; st < ns; ++st) {
            long double wt = expl(-(long double)beta * ((long double)E[st] - emin));
            z += wt;
            s1 += wt * E[st];
            if (ac || am) {
                for (int i = 0; i < N; ++i) {
                    int si = ((st >> i) & 1u) ? -1 : 1;
                    if (am) am[i] += wt * si;
                    if (ac)
                        for (int d = 0; d < D; ++d) {
                            int j = nbr[i * 2 * D + 2 * d + 1];
                            int sj = ((st >> j) & 1u) ? -1 : 1;
                            ac[d * N + i] += wt * (si * sj);
                        }
                }
            }
        }
        long double em = s1 / z;
        long double s2 = 0.0L, sq = 0.0L;
        for (size_t st = 0; st < ns; ++st) {
            long double wt = expl(-(long double)beta * ((long double)E[st] - emin));
            long double de = (long double)E[st] - em;
            s2 += wt * de * de;
            sq += wt * (long double)E[st] * E[st];
        }
        double lnZ = (double)(-(long double)beta * emin + logl(z));
        double* o = out + (size_t)t * 8;
        o[0] = lnZ;
        o[1] = (double)em;
        o[2] = (double)(sq / z);
        o[3] = (double)((long double)beta * beta * (s2 / z) / N);
        o[4] = -lnZ;
        o[5] = emin;
        o[6] = 0.0;
        o[7] = 0.0;
        if (ac) for (int b = 0; b < nb; ++b) corr[(size_t)t * nb + b] = (double)(ac[b] / z);
        if (am) for (int i = 0; i < N; ++i) mag[(size_t)t * N + i] = (double)(am[i] / z);
    }
    free(ac); free(am); free(E); free(nbr); free(bond);
    return 0;
}
