// pa_packed.cu -- +-J couplings: multi-spin-coded checkerboard Metropolis.
//
// Sec. II.B (N_S Metropolis sweeps per temperature) with the checkerboard
// spin selection of Sec. III.A.  64 replicas of one instance share a uint64
// word per site (bit j = replica 64g+j, bit set = spin -1), so one bitwise
// operation updates 64 replicas.  A block stages GPB replica groups in shared
// memory, split by parity (word of site i at [group][parity(i)][i>>1]), runs
// all N_S sweeps there, and writes the tile back: the state crosses HBM once
// per temperature.  Couplings are shared by every replica: one 6-bit sign
// mask per site in shared memory.
//
// Acceptance (+-J): flipping S_i changes the energy by dE = 4D - 4 n with n
// the number of unsatisfied bonds of i (J S_i S_j = -1).  Lanes with dE <= 0
// flip.  For dE = 4c > 0 the lane flips iff its 32-bit uniform r is below
// thr_c = floor(exp(-beta dE) 2^32).  The uniforms are stored as 32 bit
// planes (plane b holds bit 31-b of all 64 lanes' r), so "r < thr" is decided
// MSB first: a lane is decided at the first plane where its bit differs from
// thr's bit.  Planes are generated two at a time only while undecided lanes
// remain, which gives the same decisions as generating all 32.
//
// Energies: per-lane unsatisfied-bond counts are accumulated in bit-sliced
// (vertical) counters, reduced across the threads of a group with warp
// shuffles, and E = 2 n_unsat - D N.
#include "pa_device.cuh"
#include "pa_internal.h"

namespace pa {

__device__ __forceinline__ uint64_t maj3(uint64_t a, uint64_t b, uint64_t c)
{
    return (a & b) | (c & (a ^ b));
}

template <int D, int L>
__device__ __forceinline__ int site_parity(int i)
{
    int x = i % L, y = (i / L) % L, z = (D == 3) ? i / (L * L) : 0;
    return (x + y + z) & 1;
}

// One plane of the comparison r < thr for the undecided lanes U.  T (the
// threshold's bit for each lane's class) is selected by the count bits:
// n = 0 -> v00, n = 1 -> v01, n = 2 -> v10 (0 / ~0 masks of this plane).
// A lane whose plane bit differs from T is decided: accepted if T = 1.
__device__ __forceinline__ void plane_step(uint64_t pl, uint32_t v00, uint32_t v01, uint32_t v10,
                                           uint64_t b0, uint64_t b1, uint64_t& U, uint64_t& acc)
{
    const uint64_t V00 = (uint64_t)(int64_t)(int32_t)v00;
    const uint64_t V01 = (uint64_t)(int64_t)(int32_t)v01;
    const uint64_t V10 = (uint64_t)(int64_t)(int32_t)v10;
    const uint64_t inner = (b0 & V01) | (~b0 & V00);
    const uint64_t T = (b1 & V10) | (~b1 & inner);
    acc |= U & T & ~pl;
    U &= ~(T ^ pl);
}

// bits needed to count up to v
__host__ __device__ constexpr int bits_for(int v) { return v <= 0 ? 1 : 1 + bits_for(v >> 1); }

template <int D, int L, int GPB, int THREADS, bool I8>
__global__ void __launch_bounds__(THREADS, 4) sweep_packed_kernel(PackedSweepArgs a)
{
    using LT = Lat<D, L>;
    constexpr int N = LT::N, NH = LT::NH;
    constexpr int TPG = THREADS / GPB;           // threads per group in the energy phase
    constexpr int SEGW = TPG < 32 ? TPG : 32;    // shuffle segment width
    constexpr int NSEG = TPG / SEGW;             // segments (warps) per group
    constexpr int B = bits_for(D * N);           // counter width
    static_assert(THREADS % GPB == 0 && (TPG & (TPG - 1)) == 0, "threads per group");

    extern __shared__ uint64_t sm[];             // [GPB][2][NH]
    __shared__ uint8_t sj[N];
    __shared__ uint64_t cnt[GPB * NSEG * B];

    const int g0 = blockIdx.x * GPB;
    const int ng = min(GPB, a.G - g0);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int NWARP = THREADS / 32;

    for (int t = tid; t < N; t += THREADS) sj[t] = a.jneg[t];

    if (!I8 && !a.parent) {
        for (int t = tid; t < ng * N; t += THREADS) {
            int gl = t / N, i = t - gl * N;
            uint64_t w = a.Sin[(size_t)(g0 + gl) * N + i];
            sm[(gl * 2 + site_parity<D, L>(i)) * NH + (i >> 1)] = w;
        }
    } else if (!I8) {
        // fused resampling gather: lane j of group g takes the bit of replica
        // parent[64g+j]; parents are non-decreasing, so the 64 sources of a word
        // sit in one to a few neighbouring groups.  Each thread owns destination
        // lanes `lane` and `lane+32`; two ballots assemble a word; the word of
        // site base+t is kept by lane t and stored once per 32 sites.
        constexpr int NCH = (N + 31) / 32;
        for (int tup = warp; tup < ng * NCH; tup += NWARP) {
            const int gl = tup / NCH, base = (tup - gl * NCH) * 32;
            const int r0 = 64 * (g0 + gl) + lane, r1 = r0 + 32;
            const int s0 = r0 < a.R ? a.parent[r0] : r0;
            const int s1 = r1 < a.R ? a.parent[r1] : r1;
            const uint64_t* p0 = a.Sin + (size_t)(s0 >> 6) * N + base;
            const uint64_t* p1 = a.Sin + (size_t)(s1 >> 6) * N + base;
            const int sb0 = s0 & 63, sb1 = s1 & 63;
            const int cnt = min(32, N - base);
            uint64_t mine = 0;
#pragma unroll 4
            for (int t = 0; t < cnt; ++t) {
                const uint64_t w0 = __ldg(p0 + t), w1 = __ldg(p1 + t);
                const uint32_t lo = __ballot_sync(0xffffffffu, (uint32_t)(w0 >> sb0) & 1u);
                const uint32_t hi = __ballot_sync(0xffffffffu, (uint32_t)(w1 >> sb1) & 1u);
                if (lane == t) mine = (uint64_t)lo | ((uint64_t)hi << 32);
            }
            const int i = base + lane;
            if (lane < cnt) sm[(gl * 2 + site_parity<D, L>(i)) * NH + (i >> 1)] = mine;
        }
    } else {
        // int8 rows -> bit words: one ballot per site and 32-lane half
        const int nchunk = a.NP / 16;
        for (int tup = warp; tup < ng * 2 * nchunk; tup += NWARP) {
            int gl = tup / (2 * nchunk), rem = tup - gl * 2 * nchunk;
            int h = rem / nchunk, c = rem - h * nchunk;
            int r = 64 * (g0 + gl) + 32 * h + lane;
            uint4 v = make_uint4(0x01010101u, 0x01010101u, 0x01010101u, 0x01010101u);
            if (r < a.R) {
                int src = a.parent ? a.parent[r] : r;
                v = *reinterpret_cast<const uint4*>(a.S8_in + (size_t)src * a.NP + 16 * c);
            }
            uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                int byte = (int)(int8_t)(wv[t >> 2] >> (8 * (t & 3)));
                uint32_t bal = __ballot_sync(0xffffffffu, byte < 0);
                int i = 16 * c + t;
                if (lane == t && i < N)
                    reinterpret_cast<uint32_t*>(&sm[(gl * 2 + site_parity<D, L>(i)) * NH + (i >> 1)])[h] = bal;
            }
        }
    }
    __syncthreads();

    const uint64_t und1 = (a.und & 2u) ? ~0ull : 0ull, und2 = (a.und & 4u) ? ~0ull : 0ull,
                   und3 = (a.und & 8u) ? ~0ull : 0ull;
    const uint64_t alw1 = (a.always & 2u) ? ~0ull : 0ull, alw2 = (a.always & 4u) ? ~0ull : 0ull,
                   alw3 = (a.always & 8u) ? ~0ull : 0ull;

    for (int sw = 0; sw < a.n_sweeps; ++sw) {
        for (int p = 0; p < 2; ++p) {
            const uint32_t hs = 2u * (uint32_t)(a.k * a.n_sweeps + sw) + (uint32_t)p;
            for (int t = tid; t < ng * NH; t += THREADS) {
                const int gl = t / NH, q = t - gl * NH;
                uint64_t* cur = sm + (gl * 2 + p) * NH;
                const uint64_t* oth = sm + (gl * 2 + (p ^ 1)) * NH;
                const auto nb = LT::neighbours(p, q);
                const uint64_t s = cur[q];
                const uint32_t jm = sj[nb.site];
                uint64_t u[2 * D];
#pragma unroll
                for (int kk = 0; kk < 2 * D; ++kk)
                    u[kk] = s ^ oth[nb.q[kk]] ^ (((jm >> kk) & 1u) ? ~0ull : 0ull);
                uint64_t m1, m2, m3, b0, b1;
                if (D == 3) {
                    uint64_t s1 = u[0] ^ u[1] ^ u[2], c1 = maj3(u[0], u[1], u[2]);
                    uint64_t s2 = u[3] ^ u[4] ^ u[5], c2 = maj3(u[3], u[4], u[5]);
                    b0 = s1 ^ s2;
                    uint64_t k0 = s1 & s2;
                    b1 = c1 ^ c2 ^ k0;
                    uint64_t b2 = maj3(c1, c2, k0);
                    m3 = ~b2 & ~b1 & ~b0;  // n = 0: dE = 12
                    m2 = ~b2 & ~b1 & b0;   // n = 1: dE = 8
                    m1 = ~b2 & b1 & ~b0;   // n = 2: dE = 4
                } else {
                    uint64_t s1 = u[0] ^ u[1] ^ u[2], c1 = maj3(u[0], u[1], u[2]);
                    b0 = s1 ^ u[3];
                    uint64_t k0 = s1 & u[3];
                    b1 = c1 ^ k0;
                    uint64_t b2 = c1 & k0;
                    m3 = 0;
                    m2 = ~b2 & ~b1 & ~b0;  // n = 0: dE = 8
                    m1 = ~b2 & ~b1 & b0;   // n = 1: dE = 4
                }
                uint64_t acc = ~(m1 | m2 | m3) | (m1 & alw1) | (m2 & alw2) | (m3 & alw3);
                uint64_t U = (m1 & und1) | (m2 & und2) | (m3 & und3);
                const uint32_t g = (uint32_t)(g0 + gl);
                // MSB-first comparison r < thr over the planes still needed
#pragma unroll
                for (int m = 0; m < 16; ++m) {
                    if (!U) break;
                    const u32x4 o = philox_rk((uint32_t)q, hs, 16u * g + (uint32_t)m, a.c3, a.rk);
                    plane_step((uint64_t)o.x | ((uint64_t)o.y << 32), a.v00[2 * m], a.v01[2 * m],
                               a.v10[2 * m], b0, b1, U, acc);
                    plane_step((uint64_t)o.z | ((uint64_t)o.w << 32), a.v00[2 * m + 1], a.v01[2 * m + 1],
                               a.v10[2 * m + 1], b0, b1, U, acc);
                }
                cur[q] = s ^ acc;
            }
            __syncthreads();
        }
    }

    // ---- write back ----
    if (!I8) {
        for (int t = tid; t < ng * N; t += THREADS) {
            int gl = t / N, i = t - gl * N;
            a.S[(size_t)(g0 + gl) * N + i] = sm[(gl * 2 + site_parity<D, L>(i)) * NH + (i >> 1)];
        }
    } else {
        const int nchunk = a.NP / 16;
        for (int tup = warp; tup < ng * 2 * nchunk; tup += NWARP) {
            int gl = tup / (2 * nchunk), rem = tup - gl * 2 * nchunk;
            int h = rem / nchunk, c = rem - h * nchunk;
            int r = 64 * (g0 + gl) + 32 * h + lane;
            uint32_t wv[4] = {0x01010101u, 0x01010101u, 0x01010101u, 0x01010101u};
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                int i = 16 * c + t;
                if (i < N) {
                    uint32_t half = reinterpret_cast<const uint32_t*>(
                        &sm[(gl * 2 + site_parity<D, L>(i)) * NH + (i >> 1)])[h];
                    uint32_t byte = ((half >> lane) & 1u) ? 0xFFu : 0x01u;
                    wv[t >> 2] = (wv[t >> 2] & ~(0xFFu << (8 * (t & 3)))) | (byte << (8 * (t & 3)));
                }
            }
            if (r < a.R)
                *reinterpret_cast<uint4*>(a.S8_out + (size_t)r * a.NP + 16 * c) =
                    make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
    }

    // ---- energies: vertical counters of unsatisfied bonds ----
    {
        const int gl = tid / TPG, lt = tid - gl * TPG;
        uint64_t C[B];
#pragma unroll
        for (int b = 0; b < B; ++b) C[b] = 0;
        if (gl < ng) {
            const uint64_t* base = sm + gl * 2 * NH;
            for (int i = lt; i < N; i += TPG) {
                const int x = i % L, y = (i / L) % L, z = (D == 3) ? i / (L * L) : 0;
                const int p = (x + y + z) & 1;
                const uint64_t si = base[p * NH + (i >> 1)];
                const uint32_t jm = sj[i];
                int nbs[3];
                nbs[0] = i - x + (x == L - 1 ? 0 : x + 1);
                nbs[1] = i + ((y == L - 1) ? -(L - 1) * L : L);
                if (D == 3) nbs[2] = i + ((z == L - 1) ? -(L - 1) * L * L : L * L);
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    const int j = nbs[d];
                    const uint64_t sjw = base[(p ^ 1) * NH + (j >> 1)];
                    uint64_t carry = si ^ sjw ^ (((jm >> (2 * d + 1)) & 1u) ? ~0ull : 0ull);
#pragma unroll
                    for (int b = 0; b < B; ++b) {
                        uint64_t tt = C[b] & carry;
                        C[b] ^= carry;
                        carry = tt;
                    }
                }
            }
        }
        // segmented shuffle reduction (bit-sliced addition)
#pragma unroll
        for (int off = SEGW / 2; off > 0; off >>= 1) {
            uint64_t carry = 0;
#pragma unroll
            for (int b = 0; b < B; ++b) {
                uint64_t o = __shfl_xor_sync(0xffffffffu, C[b], off);
                uint64_t sum = C[b] ^ o ^ carry;
                carry = maj3(C[b], o, carry);
                C[b] = sum;
            }
        }
        if (gl < ng && (lt % SEGW) == 0) {
            const int seg = lt / SEGW;
#pragma unroll
            for (int b = 0; b < B; ++b) cnt[(gl * NSEG + seg) * B + b] = C[b];
        }
    }
    __syncthreads();
    for (int t = tid; t < ng * 64; t += THREADS) {
        const int gl = t >> 6, j = t & 63;
        int n = 0;
        for (int seg = 0; seg < NSEG; ++seg)
#pragma unroll
            for (int b = 0; b < B; ++b) n += (int)((cnt[(gl * NSEG + seg) * B + b] >> j) & 1ull) << b;
        const int r = 64 * (g0 + gl) + j;
        if (r < a.R) a.E[r] = 2 * n - D * N;
    }
}

// ---------------- shapes and dispatch ----------------

struct Shape { int gpb, threads; };

template <int D, int L> constexpr Shape default_shape()
{
    constexpr int N = (D == 3) ? L * L * L : L * L;
    return N <= 16 ? Shape{32, 256}
         : N <= 64 ? Shape{8, 256}
         : N <= 256 ? Shape{8, 256}
         : N <= 512 ? Shape{4, 256}
         : N <= 1024 ? Shape{2, 256}
         : Shape{1, 256};
}

template <int D, int L, int GPB, int THREADS, bool I8>
static cudaError_t launch_one(const PackedSweepArgs& a, cudaStream_t st)
{
    constexpr int NH = Lat<D, L>::NH;
    size_t smem = (size_t)GPB * 2 * NH * sizeof(uint64_t);
    auto kern = sweep_packed_kernel<D, L, GPB, THREADS, I8>;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    int grid = (a.G + GPB - 1) / GPB;
    kern<<<grid, THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

template <int D, int L>
static cudaError_t launch_dl(const PackedSweepArgs& a, int gpb, int threads, cudaStream_t st)
{
    constexpr Shape s = default_shape<D, L>();
    const bool i8 = a.S8_out != nullptr;
    // the one tuned alternative: twice the groups per block, same thread count
    if (gpb == 2 * s.gpb && threads == s.threads)
        return i8 ? launch_one<D, L, 2 * s.gpb, s.threads, true>(a, st)
                  : launch_one<D, L, 2 * s.gpb, s.threads, false>(a, st);
    if (gpb != s.gpb || threads != s.threads) return cudaErrorInvalidConfiguration;
    return i8 ? launch_one<D, L, s.gpb, s.threads, true>(a, st)
              : launch_one<D, L, s.gpb, s.threads, false>(a, st);
}

#define PA_PACKED_CASES(X) \
    X(3, 2) X(3, 4) X(3, 6) X(3, 8) X(3, 10) X(3, 12) X(3, 16) \
    X(2, 2) X(2, 4) X(2, 6) X(2, 8) X(2, 10) X(2, 12) X(2, 16) X(2, 32) X(2, 64)

bool packed_supported(int D, int L)
{
#define X(d, l) if (D == d && L == l) return true;
    PA_PACKED_CASES(X)
#undef X
    return false;
}

void packed_default_shape(int D, int L, int* gpb, int* threads)
{
#define X(d, l) if (D == d && L == l) { constexpr Shape s = default_shape<d, l>(); *gpb = s.gpb; *threads = s.threads; return; }
    PA_PACKED_CASES(X)
#undef X
    *gpb = 1; *threads = 256;
}

cudaError_t launch_sweep_packed(int D, int L, const PackedSweepArgs& a, int gpb, int threads,
                                cudaStream_t st)
{
#define X(d, l) if (D == d && L == l) return launch_dl<d, l>(a, gpb, threads, st);
    PA_PACKED_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

// ---------------- init, gather, unpack, overlap ----------------

// Sec. II.B: replicas start at random (beta = 0).  INIT stream word per (group, site).
__global__ void init_packed_kernel(uint64_t* S, int N, int G, uint32_t k0, uint32_t k1, uint32_t c3)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)N * G) return;
    int g = (int)(t / N), i = (int)(t - (size_t)g * N);
    u32x4 o = philox((uint32_t)i, (uint32_t)g, 0u, c3, k0, k1);
    S[t] = (uint64_t)o.x | ((uint64_t)o.y << 32);
}

cudaError_t launch_init_packed(uint64_t* S, int N, int G, uint32_t k0, uint32_t k1, uint32_t c3,
                               cudaStream_t st)
{
    size_t n = (size_t)N * G;
    init_packed_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(S, N, G, k0, k1, c3);
    return cudaGetLastError();
}

__global__ void unpack_packed_kernel(const uint64_t* S, int8_t* out, int N, int r0, int n)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)n * N) return;
    int rr = (int)(t / N), i = (int)(t - (size_t)rr * N);
    int r = r0 + rr;
    uint64_t w = S[(size_t)(r >> 6) * N + i];
    out[t] = ((w >> (r & 63)) & 1ull) ? (int8_t)-1 : (int8_t)1;
}

cudaError_t launch_unpack_packed(const uint64_t* S, int8_t* out, int N, int r0, int n, cudaStream_t st)
{
    size_t tot = (size_t)N * n;
    unpack_packed_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(S, out, N, r0, n);
    return cudaGetLastError();
}

// Sec. V.A overlap: lane j of group g counts sites where the two populations differ.
__global__ void overlap_packed_kernel(const uint64_t* A, const uint64_t* B, int N, int R,
                                      unsigned long long* hist)
{
    const int g = blockIdx.x, j = threadIdx.x;  // 64 threads
    const int r = 64 * g + j;
    const uint64_t* a = A + (size_t)g * N;
    const uint64_t* b = B + (size_t)g * N;
    int nd = 0;
    for (int i = 0; i < N; ++i) nd += (int)(((a[i] ^ b[i]) >> j) & 1ull);
    if (r < R) atomicAdd(&hist[N - nd], 1ull);
}

cudaError_t launch_overlap_packed(const uint64_t* A, const uint64_t* B, int N, int R,
                                  unsigned long long* hist, cudaStream_t st)
{
    int G = (R + 63) / 64;
    overlap_packed_kernel<<<G, 64, 0, st>>>(A, B, N, R, hist);
    return cudaGetLastError();
}

}  // namespace pa
