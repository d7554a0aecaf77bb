// pa_device.cuh -- device primitives of the GB300 PAMC library.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Ten
// rounds; each round multiplies counter words 0 and 2 by the round constants
// (32x32 -> 64 bit), XORs the high halves with the other counter words and
// the key, and bumps the key by the two Weyl increments.  Stream layout
// (counter word 3 = stream << 28 | tag << 24 | instance):
//   INIT  (1): counter (site, group, 0, c3) -> 64 spin bits of one replica group
//   PLANE (2): counter (q, hs, 16 g + m, c3), m = 0..15 -> 32 bit planes of
//              64 lanes; replica 64g+j's 32-bit uniform is sum_b bit_j(plane_b) 2^(31-b)
//   WORD  (3): counter (q >> 2, hs, replica, c3) -> word q & 3 is the uniform
//   RES   (4): counter (draw, k, 0, c3) -> 53-bit uniform from words 0 and 1
// (hs = 2 (k N_S + sweep) + parity, q = site >> 1).
//
// Exponentials: exp(-beta dE) of Metropolis acceptance and exp[-(beta'-beta)E]
// of resampling (Sec. II.B) follow one fixed IEEE operation sequence so that
// accept/reject and copy-number decisions are reproducible: Cody-Waite
// reduction x = k ln 2 + r (two-word ln 2, fused multiply-adds), a Taylor
// polynomial by Horner's rule with fused multiply-adds, exact scaling by 2^k.
// Constants: RN(1/ln2); ln 2 truncated to 32 (FP32: 16) significant bits and
// RN of the remainder; c_n = RN(1/n!) for n <= 14 (FP32: n <= 7).
#pragma once
#include <cstdint>

#ifndef PA_HD
#define PA_HD __host__ __device__ __forceinline__
#endif

namespace pa {

enum : uint32_t { STREAM_INIT = 1, STREAM_PLANE = 2, STREAM_WORD = 3, STREAM_RES = 4, STREAM_ICM = 5 };

PA_HD uint32_t counter3(uint32_t stream, uint32_t tag, uint32_t instance)
{
    return (stream << 28) | ((tag & 0xFu) << 24) | (instance & 0xFFFFFFu);
}

struct u32x4 {
    uint32_t x, y, z, w;
};

PA_HD void mulhilo(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo)
{
    // one wide multiply gives both halves
    const uint64_t p = (uint64_t)a * (uint64_t)b;
    lo = (uint32_t)p;
    hi = (uint32_t)(p >> 32);
}

PA_HD u32x4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int rnd = 0; rnd < 10; ++rnd) {
        uint32_t hi0, lo0, hi2, lo2;
        mulhilo(0xD2511F53u, c0, hi0, lo0);
        mulhilo(0xCD9E8D57u, c2, hi2, lo2);
        uint32_t n0 = hi2 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo2;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return {c0, c1, c2, c3};
}

// Philox4x32-10 with the ten round keys precomputed (rk[2r] = k0 + r W0,
// rk[2r+1] = k1 + r W1); identical output to philox().
__device__ __forceinline__ u32x4 philox_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                           const uint32_t (&rk)[20])
{
#pragma unroll
    for (int rnd = 0; rnd < 10; ++rnd) {
        // one wide multiply gives both halves of each product
        const uint64_t p0 = (uint64_t)c0 * 0xD2511F53u, p2 = (uint64_t)c2 * 0xCD9E8D57u;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo2 = (uint32_t)p2, hi2 = (uint32_t)(p2 >> 32);
        const uint32_t n0 = hi2 ^ c1 ^ rk[2 * rnd];
        const uint32_t n2 = hi0 ^ c3 ^ rk[2 * rnd + 1];
        c0 = n0;
        c1 = lo2;
        c2 = n2;
        c3 = lo0;
    }
    return {c0, c1, c2, c3};
}

// The same with counter word 2 taken as c2 + d, given add2 = d * 0xCD9E8D57
// as a 64-bit product: word 2 enters Philox only through its first-round
// product, and (c2 + d) M = c2 M + d M exactly while c2 + d < 2^32, so the
// offset rides in the multiply's addend (identical output to
// philox_rk(c0, c1, c2 + d, c3, rk)).
__device__ __forceinline__ u32x4 philox_rk_add2(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                const uint32_t (&rk)[20], uint64_t add2)
{
    {
        const uint64_t p0 = (uint64_t)c0 * 0xD2511F53u, p2 = (uint64_t)c2 * 0xCD9E8D57u + add2;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo2 = (uint32_t)p2, hi2 = (uint32_t)(p2 >> 32);
        const uint32_t n0 = hi2 ^ c1 ^ rk[0];
        const uint32_t n2 = hi0 ^ c3 ^ rk[1];
        c0 = n0;
        c1 = lo2;
        c2 = n2;
        c3 = lo0;
    }
#pragma unroll
    for (int rnd = 1; rnd < 10; ++rnd) {
        const uint64_t p0 = (uint64_t)c0 * 0xD2511F53u, p2 = (uint64_t)c2 * 0xCD9E8D57u;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo2 = (uint32_t)p2, hi2 = (uint32_t)(p2 >> 32);
        const uint32_t n0 = hi2 ^ c1 ^ rk[2 * rnd];
        const uint32_t n2 = hi0 ^ c3 ^ rk[2 * rnd + 1];
        c0 = n0;
        c1 = lo2;
        c2 = n2;
        c3 = lo0;
    }
    return {c0, c1, c2, c3};
}

// 53-bit uniform in [0, 1) from two 32-bit words
PA_HD double uniform53(uint32_t a, uint32_t b)
{
    return (double)((uint64_t)(a >> 5) * 67108864ull + (uint64_t)(b >> 6)) * 0x1p-53;
}

// ---------------- specified exponentials ----------------

PA_HD double fma64(double a, double b, double c)
{
#ifdef __CUDA_ARCH__
    return __fma_rn(a, b, c);
#else
    return __builtin_fma(a, b, c);
#endif
}
PA_HD float fma32(float a, float b, float c)
{
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return __builtin_fmaf(a, b, c);
#endif
}
PA_HD double mul64(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    return a * b;
#endif
}
PA_HD float mul32(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
PA_HD float add32(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
PA_HD double add64(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dadd_rn(a, b);
#else
    return a + b;
#endif
}
PA_HD double rint64(double x)
{
#ifdef __CUDA_ARCH__
    return rint(x);
#else
    return __builtin_rint(x);
#endif
}
PA_HD float rint32(float x)
{
#ifdef __CUDA_ARCH__
    return rintf(x);
#else
    return __builtin_rintf(x);
#endif
}
PA_HD double pow2_64(int k)  // 2^k for -1022 <= k <= 1023
{
    uint64_t bits = (uint64_t)(k + 1023) << 52;
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)bits);
#else
    double d;
    __builtin_memcpy(&d, &bits, sizeof d);
    return d;
#endif
}
PA_HD float pow2_32(int k)  // 2^k for -126 <= k <= 127
{
    uint32_t bits = (uint32_t)(k + 127) << 23;
#ifdef __CUDA_ARCH__
    return __uint_as_float(bits);
#else
    float f;
    __builtin_memcpy(&f, &bits, sizeof f);
    return f;
#endif
}

// 1/n! rounded to nearest, n = 0..14 (exact rational 1/n! rounded once)
#define PA_C64_TABLE                                                                      \
    {0x1p+0, 0x1p+0, 0x1p-1, 0x1.5555555555555p-3, 0x1.5555555555555p-5,                 \
     0x1.1111111111111p-7, 0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13, 0x1.a01a01a01a01ap-16, \
     0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22, 0x1.ae64567f544e4p-26,                 \
     0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33, 0x1.93974a8c07c9dp-37}
#define PA_C32_TABLE \
    {0x1p+0f, 0x1p+0f, 0x1p-1f, 0x1.555556p-3f, 0x1.555556p-5f, 0x1.111112p-7f, 0x1.6c16c2p-10f, 0x1.a01a02p-13f}

// exp(x) for x <= 0; 1 at 0, 0 below -708
PA_HD double spec_exp64(double x)
{
    if (x == 0.0) return 1.0;
    if (x < -708.0) return 0.0;
    const double c[15] = PA_C64_TABLE;
    double kd = rint64(mul64(x, 0x1.71547652b82fep+0));
    double r = fma64(-kd, 0x1.62e42feep-1, x);
    r = fma64(-kd, 0x1.a39ef35793c76p-33, r);
    double p = c[14];
#pragma unroll
    for (int n = 13; n >= 0; --n) p = fma64(p, r, c[n]);
    return mul64(p, pow2_64((int)kd));
}

// expf(x) for x <= 0; 1 at 0, 0 below -87
PA_HD float spec_expf(float x)
{
    if (x == 0.0f) return 1.0f;
    if (x < -87.0f) return 0.0f;
    const float c[8] = PA_C32_TABLE;
    float kf = rint32(mul32(x, 0x1.715476p+0f));
    float r = fma32(-kf, 0x1.62e4p-1f, x);
    r = fma32(-kf, 0x1.7f7d1cp-20f, r);
    float p = c[7];
#pragma unroll
    for (int n = 6; n >= 0; --n) p = fma32(p, r, c[n]);
    return mul32(p, pow2_32((int)kf));
}

// +-J acceptance threshold for an energy increase dE > 0: floor(exp(-beta dE) 2^32)
PA_HD uint64_t threshold_pm(double beta, int dE)
{
    double e = spec_exp64(-mul64(beta, (double)dE));
    return (uint64_t)mul64(e, 4294967296.0);
}

// ---------------- int128 -> double, round to nearest even ----------------

__device__ __forceinline__ double i128_to_double(__int128 v)
{
    bool neg = v < 0;
    unsigned __int128 u = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    uint64_t hi = (uint64_t)(u >> 64), lo = (uint64_t)u;
    if (hi == 0 && lo < (1ull << 53)) {
        double d = (double)lo;  // exact
        return neg ? -d : d;
    }
    int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
    int top = 127 - lz;       // index of the leading one, >= 53
    int shift = top - 52;     // drop `shift` low bits
    unsigned __int128 m = u >> shift;
    unsigned __int128 rem = u - (m << shift);
    unsigned __int128 half = (unsigned __int128)1 << (shift - 1);
    uint64_t mm = (uint64_t)m;
    if (rem > half || (rem == half && (mm & 1u))) ++mm;
    double d = __dmul_rn((double)mm, pow2_64(shift));  // mm <= 2^53: exact
    return neg ? -d : d;
}

// ---------------- lattice helpers ----------------
//
// Site i = x + L y + L^2 z; parity p(i) = (x + y + z) & 1; for even L the
// sublattice index q = i >> 1 numbers the N/2 sites of each parity.
// Given parity p and q: xh = q mod L/2, y, z from q div L/2, and
// x = 2 xh + b with b = (p + y + z) & 1.

template <int D, int L>
struct Lat {
    static constexpr int N = (D == 3) ? L * L * L : L * L;
    static constexpr int NH = N / 2;
    static constexpr int LH = L / 2;
    // neighbour sublattice indices (in the other parity's array) of (p, q),
    // order (-x, +x, -y, +y, -z, +z); also the site index i of (p, q) and the
    // site indices of the -e_d neighbours (for coupling lookup J[d][i - e_d]).
    struct Nb {
        int q[2 * D];
        int site;
        int site_m[D];
    };
    static __device__ __forceinline__ Nb neighbours(int p, int q)
    {
        Nb nb;
        int xh = q % LH;
        int row = q / LH;
        int y = row % L;
        int z = (D == 3) ? row / L : 0;
        int b = (p + y + z) & 1;
        int x = 2 * xh + b;
        nb.site = 2 * q + b;
        int xm = (x == 0) ? L - 1 : x - 1;
        int xp = (x == L - 1) ? 0 : x + 1;
        int ym = (y == 0) ? L - 1 : y - 1;
        int yp = (y == L - 1) ? 0 : y + 1;
        int rowq = row * LH;
        nb.q[0] = rowq + (xm >> 1);
        nb.q[1] = rowq + (xp >> 1);
        int zq = (D == 3) ? z * L : 0;
        nb.q[2] = (ym + zq) * LH + xh;
        nb.q[3] = (yp + zq) * LH + xh;
        nb.site_m[0] = x == 0 ? nb.site + (L - 1) : nb.site - 1;
        nb.site_m[1] = (y == 0) ? nb.site + (L - 1) * L : nb.site - L;
        if (D == 3) {
            int zm = (z == 0) ? L - 1 : z - 1;
            int zp = (z == L - 1) ? 0 : z + 1;
            nb.q[4] = (y + zm * L) * LH + xh;
            nb.q[5] = (y + zp * L) * LH + xh;
            nb.site_m[2] = (z == 0) ? nb.site + (L - 1) * L * L : nb.site - L * L;
        }
        return nb;
    }
    // the same for a site whose column (xh, y) is known (3D): only z is decoded
    static __device__ __forceinline__ Nb neighbours_column(int p, int q, int xh, int y)
    {
        static_assert(D == 3, "column walk is three-dimensional");
        Nb nb;
        const int z = q / (LH * L);
        const int b = (p + y + z) & 1;
        nb.site = 2 * q + b;
        // x: b = 0 -> (q - 1 or row wrap, q); b = 1 -> (q, q + 1 or row wrap)
        const int dxm = b ? 0 : (xh == 0 ? LH - 1 : -1);
        const int dxp = b ? (xh == LH - 1 ? -(LH - 1) : 1) : 0;
        nb.q[0] = q + dxm;
        nb.q[1] = q + dxp;
        nb.q[2] = q + (y == 0 ? (L - 1) * LH : -LH);
        nb.q[3] = q + (y == L - 1 ? -(L - 1) * LH : LH);
        nb.q[4] = q + (z == 0 ? (L - 1) * LH * L : -LH * L);
        nb.q[5] = q + (z == L - 1 ? -(L - 1) * LH * L : LH * L);
        const int x = 2 * xh + b;
        nb.site_m[0] = x == 0 ? nb.site + (L - 1) : nb.site - 1;
        nb.site_m[1] = (y == 0) ? nb.site + (L - 1) * L : nb.site - L;
        nb.site_m[2] = (z == 0) ? nb.site + (L - 1) * L * L : nb.site - L * L;
        return nb;
    }
};

}  // namespace pa
