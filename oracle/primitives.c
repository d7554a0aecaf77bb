/*
 * primitives.c -- random numbers and the specified exponential of the oracle.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Random numbers.  The paper does not name its generator; the method only
 * needs uniform random numbers for Metropolis acceptance (Sec. II.B, N_S
 * sweeps) and for drawing copy numbers in resampling (Sec. II.B).  Both
 * sides of the parity check use the counter-based Philox4x32-10 generator
 * defined in Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3" (SC'11): a 4x32-bit counter, a 2x32-bit key, ten rounds of
 * two 32x32->64 multiplications, with the key bumped by the Weyl constants
 * between rounds.  This file implements it from that definition.
 *
 * Exponential.  Metropolis acceptance needs exp(-beta dE) and resampling
 * needs exp[-(beta'-beta) E_i] (Sec. II.B).  To make every accept/reject and
 * every copy-number decision reproducible across machines, exp is pinned to
 * one IEEE operation sequence: Cody-Waite argument reduction
 * x = k ln2 + r with a two-word ln 2 and fused multiply-adds, a Taylor
 * polynomial in r evaluated by Horner's rule with fused multiply-adds, and
 * an exact scaling by 2^k.  The constants are defined, not tuned:
 *   INV_LN2   = RN(1/ln 2)
 *   LN2_HI    = ln 2 truncated to 32 significant bits (so k*LN2_HI is exact)
 *   LN2_LO    = RN(ln 2 - LN2_HI)
 *   c_n       = RN(1/n!),  n = 0..14
 * and the FP32 version uses 16 significant bits for LN2_HI_F and degree 7.
 * The oracle derives c_n at run time as 1/n! (n! is exact in binary64 for
 * n <= 18, so one correctly rounded division gives RN(1/n!)).
 */
#include "oracle.h"
#include <math.h>
#include <string.h>

/* ---------------- Philox4x32-10 ---------------- */

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    /* round multipliers and key increments from Salmon et al. (SC'11) */
    const uint32_t MUL_A = 0xD2511F53u, MUL_B = 0xCD9E8D57u;
    const uint32_t WEYL_A = 0x9E3779B9u, WEYL_B = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod_a = (uint64_t)MUL_A * (uint64_t)x0;
        uint64_t prod_b = (uint64_t)MUL_B * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(prod_b >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)prod_b;
        uint32_t y2 = (uint32_t)(prod_a >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)prod_a;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += WEYL_A;
        k1 += WEYL_B;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

uint32_t or_counter3(uint32_t stream, uint32_t tag, uint32_t instance)
{
    return (stream << 28) | ((tag & 0xFu) << 24) | (instance & 0xFFFFFFu);
}

/* u = ((out0 >> 5) * 2^26 + (out1 >> 6)) * 2^-53 : 53 uniform bits in [0, 1) */
double or_uniform53(uint32_t out0, uint32_t out1)
{
    uint64_t a = out0 >> 5, b = out1 >> 6;
    return (double)(a * 67108864ull + b) * 0x1p-53;
}

/* ---------------- specified exponentials ---------------- */

static const double OR_INV_LN2 = 0x1.71547652b82fep+0;
static const double OR_LN2_HI = 0x1.62e42feep-1;
static const double OR_LN2_LO = 0x1.a39ef35793c76p-33;
static const float OR_INV_LN2_F = 0x1.715476p+0f;
static const float OR_LN2_HI_F = 0x1.62e4p-1f;
static const float OR_LN2_LO_F = 0x1.7f7d1cp-20f;

static double coef64(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i; /* exact for n <= 18 */
    return 1.0 / f;
}

static float coef32(int n)
{
    float f = 1.0f;
    for (int i = 2; i <= n; ++i) f *= (float)i; /* exact for n <= 10 */
    return 1.0f / f;
}

void or_spec_constants(double out[4], float outf[3], double coef[15], float coeff[8])
{
    out[0] = OR_INV_LN2; out[1] = OR_LN2_HI; out[2] = OR_LN2_LO; out[3] = 0.0;
    outf[0] = OR_INV_LN2_F; outf[1] = OR_LN2_HI_F; outf[2] = OR_LN2_LO_F;
    for (int n = 0; n <= 14; ++n) coef[n] = coef64(n);
    for (int n = 0; n <= 7; ++n) coeff[n] = coef32(n);
}

/* exp(x) for x <= 0: 1 at x == 0, 0 below -708. */
double or_spec_exp64(double x)
{
    if (x == 0.0) return 1.0;
    if (x < -708.0) return 0.0;
    double kd = rint(x * OR_INV_LN2);
    double r = fma(-kd, OR_LN2_HI, x);
    r = fma(-kd, OR_LN2_LO, r);
    double p = coef64(14);
    for (int n = 13; n >= 0; --n) p = fma(p, r, coef64(n));
    int k = (int)kd; /* -1021 <= k <= 0 */
    uint64_t bits = (uint64_t)(k + 1023) << 52;
    double scale;
    memcpy(&scale, &bits, sizeof scale);
    return p * scale;
}

/* expf(x) for x <= 0: 1 at x == 0, 0 below -87. */
float or_spec_expf(float x)
{
    if (x == 0.0f) return 1.0f;
    if (x < -87.0f) return 0.0f;
    float kf = rintf(x * OR_INV_LN2_F);
    float r = fmaf(-kf, OR_LN2_HI_F, x);
    r = fmaf(-kf, OR_LN2_LO_F, r);
    float p = coef32(7);
    for (int n = 6; n >= 0; --n) p = fmaf(p, r, coef32(n));
    int k = (int)kf; /* -126 <= k <= 0 */
    uint32_t bits = (uint32_t)(k + 127) << 23;
    float scale;
    memcpy(&scale, &bits, sizeof scale);
    return p * scale;
}

/* Metropolis threshold for a +-J energy increase dE > 0 at inverse
 * temperature beta: accept iff the 32-bit uniform r satisfies r < thr,
 * thr = floor(exp(-beta*dE) * 2^32) in [0, 2^32]. */
uint64_t or_threshold_pm(double beta, int dE)
{
    double e = or_spec_exp64(-(beta * (double)dE));
    return (uint64_t)(e * 4294967296.0);
}

/* Same for the real-coupling path; x = f32(beta) * dE computed in FP32. */
uint64_t or_threshold_real(float x)
{
    if (x <= 0.0f) return 4294967296ull;
    float e = or_spec_expf(-x);
    return (uint64_t)(e * 4294967296.0f);
}

/* ---------------- batch helpers for the tests ---------------- */

void or_philox_batch(int64_t n, const uint32_t* ctr, const uint32_t key[2], uint32_t* out)
{
    for (int64_t t = 0; t < n; ++t) or_philox4x32_10(ctr + 4 * t, key, out + 4 * t);
}

void or_spec_exp64_batch(int64_t n, const double* x, double* y)
{
    for (int64_t t = 0; t < n; ++t) y[t] = or_spec_exp64(x[t]);
}

void or_spec_expf_batch(int64_t n, const float* x, float* y)
{
    for (int64_t t = 0; t < n; ++t) y[t] = or_spec_expf(x[t]);
}

void or_threshold_real_batch(int64_t n, const float* x, uint64_t* thr)
{
    for (int64_t t = 0; t < n; ++t) thr[t] = or_threshold_real(x[t]);
}
