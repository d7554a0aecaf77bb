// pa_sweep_tiles.cuh -- the Metropolis sweep of one tile of replicas, shared by
// the single-instance kernels and the batched persistent kernel.
//
// Sec. II.B: N_S Metropolis sweeps per temperature; Sec. III.A: checkerboard
// spin selection (all parity-0 sites, then all parity-1 sites).
//
// +-J tile (multi-spin coding): 64 replicas of one instance share a uint64 word
// per site (bit j = replica 64g+j, bit set = spin -1).  A tile is GPB replica
// groups staged in shared memory split by parity ([group][parity(i)][i>>1]);
// all N_S sweeps run there and the tile is written back once per temperature.
// Flipping S_i changes the energy by dE = 4D - 4n, n = unsatisfied bonds of i
// (J S_i S_j = -1).  Lanes with dE <= 0 flip; for dE = 4c > 0 a lane flips iff
// its 32-bit uniform r < thr_c = floor(exp(-beta dE) 2^32).  The uniforms are
// stored as 32 bit planes (plane b holds bit 31-b of the 64 lanes' r), so
// r < thr is decided MSB first at the first plane where a lane's bit differs
// from thr's; planes are generated two at a time only while undecided lanes
// remain (same decisions as generating all 32).  Words still undecided after
// the first calls (mode 1: any; modes 0 and 2 at L=16: after four calls) are
// compacted into a block queue and finished on full warps.  Energies: per-lane counts of
// unsatisfied bonds in bit-sliced counters, reduced across the threads of a
// group with warp shuffles; E = 2 n_unsat - D N.
//
// Real-coupling tile: 32 replicas staged transposed to [parity][q][replica]
// bytes so that a warp (one lane per replica) updates one site of 32
// replicas; couplings are warp-uniform broadcast loads.  Local field
// f = ((((t_-x + t_+x) + t_-y) + t_+y) + ...) + h_i in FP32 with t = J S_nb,
// dE = 2 S_i f (exact), x = f32(beta) dE; accept iff x <= 0 or
// r < floor(spec_expf(-x) 2^32), decided through a device-verified guard band
// around that threshold (same decisions; see accept_band).  Energies are
// exact int128 sums of J * 2^96.
#pragma once
#include <type_traits>
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

// a 0 / ~0 32-bit mask widened to 64 bits (both halves the same register)
__device__ __forceinline__ uint64_t rep32(uint32_t v) { return ((uint64_t)v << 32) | v; }

// One plane of the comparison r < thr for the undecided lanes U.  T (the
// threshold's bit for each lane's class) is selected by the count bits:
// n = 0 -> v00, n = 1 -> v01, n = 2 -> v10 (0 / ~0 masks of this plane).
// A lane whose plane bit differs from T is decided: accepted if T = 1.
__device__ __forceinline__ void plane_step(uint64_t pl, uint32_t v00, uint32_t v01, uint32_t v10,
                                           uint64_t b0, uint64_t b1, uint64_t& U, uint64_t& acc)
{
    const uint64_t V00 = rep32(v00), V01 = rep32(v01), V10 = rep32(v10);
    const uint64_t inner = (b0 & V01) | (~b0 & V00);
    const uint64_t T = (b1 & V10) | (~b1 & inner);
    acc |= U & T & ~pl;
    U &= ~(T ^ pl);
}

// The same step when every undecided lane has the same threshold: its plane
// bit t is uniform, so the decision needs no per-lane selection.
__device__ __forceinline__ void plane_step_uniform(uint64_t pl, uint32_t t, uint64_t& U, uint64_t& acc)
{
    if (t) {
        acc |= U & ~pl;
        U &= pl;
    } else {
        U &= ~pl;
    }
}

// Two classes: sel picks the class with threshold bit ta (sel = 1) or tb.
__device__ __forceinline__ void plane_step_two(uint64_t pl, uint32_t ta, uint32_t tb, uint64_t sel,
                                               uint64_t& U, uint64_t& acc)
{
    const uint64_t A = rep32(ta), B = rep32(tb);
    const uint64_t T = (sel & A) | (~sel & B);
    acc |= U & T & ~pl;
    U &= ~(T ^ pl);
}

// bits needed to count up to v
__host__ __device__ constexpr int bits_for(int v) { return v <= 0 ? 1 : 1 + bits_for(v >> 1); }

// LATE: the late compaction of modes 0, 2 and 3 (single 3D instances with
// L >= 8): its queue entries also carry the class bits of the undecided lanes
template <int D, int L, int GPB, int THREADS, bool LATE = true>
struct PackedShape {
    static constexpr int N = Lat<D, L>::N, NH = Lat<D, L>::NH;
    static constexpr bool kLate = LATE && D == 3 && L >= 8;
    static constexpr int TPG = THREADS / GPB;         // threads per group in the energy phase
    static constexpr int SEGW = TPG < 32 ? TPG : 32;  // shuffle segment width
    static constexpr int NSEG = TPG / SEGW;           // segments (warps) per group
    static constexpr int B = bits_for(D * N);         // counter width
    static constexpr size_t TILE = (size_t)GPB * 2 * NH * 8;
    static constexpr size_t SJ = ((size_t)N + 15) / 16 * 16;
    static constexpr size_t CNT = (size_t)GPB * NSEG * B * 8;
    static constexpr int QIPT = 4;  // items per thread per queue round
    static constexpr int QCAP = QIPT * THREADS;  // queue entries (every item of a round)
    // queue of undecided words: counters, masks (two with the class bits), item indices
    static constexpr size_t QUEUE = 32 + (size_t)QCAP * ((kLate ? 16 : 8) + 2);
    static_assert(GPB * NH <= 65535, "item indices fit 16 bits");
    static constexpr size_t SMEM = TILE + SJ + CNT + QUEUE;
    static_assert(THREADS % GPB == 0 && (TPG & (TPG - 1)) == 0, "threads per group");
};

struct Shape {
    int gpb, threads;
};

// default groups per block and threads of the packed sweep for a lattice
template <int D, int L> __host__ __device__ constexpr Shape default_shape()
{
    constexpr int N = (D == 3) ? L * L * L : L * L;
    return N <= 16 ? Shape{32, 256}
         : N <= 64 ? Shape{8, 256}
         : N <= 256 ? Shape{8, 256}
         : N <= 512 ? Shape{4, 256}
         : N <= 1024 ? Shape{2, 256}
         : Shape{1, 256};
}

// groups [g0, g0 + GPB) of one instance; smem holds PackedShape::SMEM bytes
// LATE: allow the late compaction of modes 0 and 2 (the single-instance
// kernels; the disorder batch measured slower with it)
// SHARD: the instance is a shard of a larger population; its PLANE counters
// carry the global group index g0 + in.goff (a separate instantiation, so
// that the counters of every other launch cost nothing extra)
template <int D, int L, int GPB, int THREADS, bool I8, bool LATE = true, bool SHARD = false>
__device__ __forceinline__ void sweep_packed_tile(const PackedStep& s, const PackedInst& in, int g0,
                                                  unsigned char* smem)
{
    using LT = Lat<D, L>;
    using SH = PackedShape<D, L, GPB, THREADS, LATE>;
    constexpr int N = SH::N, NH = SH::NH, TPG = SH::TPG, SEGW = SH::SEGW, NSEG = SH::NSEG, B = SH::B;
    constexpr int NWARP = THREADS / 32;
    uint64_t* sm = reinterpret_cast<uint64_t*>(smem);
    uint8_t* sj = smem + SH::TILE;
    uint64_t* cnt = reinterpret_cast<uint64_t*>(smem + SH::TILE + SH::SJ);
    unsigned char* qbuf = smem + SH::TILE + SH::SJ + SH::CNT;

    const int R = in.Rdev ? __ldg(in.Rdev) : in.R;
    const int G = in.Rdev ? (R + 63) >> 6 : in.G;
    if (g0 >= G) return;  // block-uniform: past the population held in device memory
    const uint32_t c3 = in.c3;
    // a shard's groups carry their global index in the PLANE counters:
    // 16 goff added to counter word 2 through its first-round product
    const uint64_t gadd = SHARD ? (uint64_t)(16u * (uint32_t)in.goff) * 0xCD9E8D57ull : 0ull;
    auto plane_call = [&](uint32_t q, uint32_t hs, uint32_t c2) {
        if constexpr (SHARD) return philox_rk_add2(q, hs, c2, c3, s.rk, gadd);
        else return philox_rk(q, hs, c2, c3, s.rk);
    };
    // (the group index passed to the comparisons is written g0 when a block
    // holds one group, so that the compiler sees it block-uniform and keeps the
    // first-round products that depend on it alone off the vector pipes:
    // L=16, k=5..24: 2837 -> 2875 attempts/ns)
    const int32_t* __restrict__ parent = in.parent;
    const int ng = GPB == 1 ? 1 : min(GPB, G - g0);  // g0 < G: one group is always full
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;

    for (int t = tid; t < N; t += THREADS) sj[t] = in.jneg[t];

    if (!I8 && !parent) {
        for (int t = tid; t < ng * N; t += THREADS) {
            int gl = t / N, i = t - gl * N;
            uint64_t w = in.Sin[(size_t)(g0 + gl) * N + i];
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
            const int s0 = r0 < R ? parent[r0] : r0;
            const int s1 = r1 < R ? parent[r1] : r1;
            const uint64_t* p0 = in.Sin + (size_t)(s0 >> 6) * N + base;
            const uint64_t* p1 = in.Sin + (size_t)(s1 >> 6) * N + base;
            const int sb0 = s0 & 63, sb1 = s1 & 63;
            const int cnt32 = min(32, N - base);
            uint64_t mine = 0;
#pragma unroll 4
            for (int t = 0; t < cnt32; ++t) {
                const uint64_t w0 = __ldg(p0 + t), w1 = __ldg(p1 + t);
                const uint32_t lo = __ballot_sync(0xffffffffu, (uint32_t)(w0 >> sb0) & 1u);
                const uint32_t hi = __ballot_sync(0xffffffffu, (uint32_t)(w1 >> sb1) & 1u);
                if (lane == t) mine = (uint64_t)lo | ((uint64_t)hi << 32);
            }
            const int i = base + lane;
            if (lane < cnt32) sm[(gl * 2 + site_parity<D, L>(i)) * NH + (i >> 1)] = mine;
        }
    } else {
        // int8 rows -> bit words: one ballot per site and 32-lane half
        const int nchunk = in.NP / 16;
        for (int tup = warp; tup < ng * 2 * nchunk; tup += NWARP) {
            int gl = tup / (2 * nchunk), rem = tup - gl * 2 * nchunk;
            int h = rem / nchunk, c = rem - h * nchunk;
            int r = 64 * (g0 + gl) + 32 * h + lane;
            uint4 v = make_uint4(0x01010101u, 0x01010101u, 0x01010101u, 0x01010101u);
            if (r < R) {
                int src = parent ? parent[r] : r;
                v = *reinterpret_cast<const uint4*>(in.S8_in + (size_t)src * in.NP + 16 * c);
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

    const uint64_t und1 = (s.und & 2u) ? ~0ull : 0ull, und2 = (s.und & 4u) ? ~0ull : 0ull,
                   und3 = (s.und & 8u) ? ~0ull : 0ull;
    const uint64_t alw1 = (s.always & 2u) ? ~0ull : 0ull, alw2 = (s.always & 4u) ? ~0ull : 0ull,
                   alw3 = (s.always & 8u) ? ~0ull : 0ull;

    // this thread's x-y column (used when every item of the thread shares it)
    const int xh_c = (tid % NH) % LT::LH, y_c = ((tid % NH) / LT::LH) % L;
    // item t = (group gl, sublattice index q) of parity p: neighbour decoding,
    // unsatisfied-bond counts n = b0 + 2 b1 + 4 b2 per lane, lanes with dE <= 0
    auto classify = [&](int t, int p, const typename LT::Nb& nb_fixed, uint64_t*& cur, int& q,
                        uint64_t& sw0, uint64_t& b0, uint64_t& b1, uint64_t& b2, uint64_t& down) {
        const int gl = t / NH;
        q = t - gl * NH;
        cur = sm + (gl * 2 + p) * NH;
        const uint64_t* oth = sm + (gl * 2 + (p ^ 1)) * NH;
        typename LT::Nb nb;
        // when every item of this thread sits on the same sublattice site
        // (THREADS a multiple of N/2) decode once; when it sits on the same x-y
        // column (3D, THREADS a multiple of L^2/2) only z moves
        if constexpr (THREADS % NH == 0) {
            nb = nb_fixed;
        } else if constexpr (D == 3 && THREADS % (LT::LH * L) == 0) {
            nb = LT::neighbours_column(p, q, xh_c, y_c);
        } else {
            nb = LT::neighbours(p, q);
        }
        sw0 = cur[q];
        const uint32_t jm = sj[nb.site];
        uint64_t u[2 * D];
        // bond signs moved to bit 7 of bytes 0..5 of (ja, jb) by two multiplies
        // (the shifted copies do not overlap), then replicated over a word by
        // the sign-replicating byte permute
        const uint32_t ja = jm * 0x10204080u, jb = jm * 0x408u;
#pragma unroll
        for (int kk = 0; kk < 2 * D; ++kk) {
            uint32_t m32;
            asm("prmt.b32 %0, %1, %2, %3;" : "=r"(m32) : "r"(ja), "r"(jb), "r"((uint32_t)(8 | kk) * 0x1111u));
            u[kk] = sw0 ^ oth[nb.q[kk]] ^ (((uint64_t)m32 << 32) | m32);
        }
        if (D == 3) {
            uint64_t s1 = u[0] ^ u[1] ^ u[2], c1 = maj3(u[0], u[1], u[2]);
            uint64_t s2 = u[3] ^ u[4] ^ u[5], c2 = maj3(u[3], u[4], u[5]);
            b0 = s1 ^ s2;
            uint64_t k0 = s1 & s2;
            b1 = c1 ^ c2 ^ k0;
            b2 = maj3(c1, c2, k0);
            down = b2 | (b1 & b0);  // n >= 3: dE <= 0
        } else {
            uint64_t s1 = u[0] ^ u[1] ^ u[2], c1 = maj3(u[0], u[1], u[2]);
            b0 = s1 ^ u[3];
            uint64_t k0 = s1 & u[3];
            b1 = c1 ^ k0;
            b2 = c1 & k0;
            down = b1 | b2;         // n >= 2: dE <= 0
        }
    };
    // MSB-first comparison r < thr over the planes still needed, per mode
    // (s.mode is uniform over the launch; mode 1 runs on the compacted queue):
    //   1: only dE = 4 lanes (n = D - 1) undecided, one threshold, uniform bit
    //   2: dE = 4 and dE = 8 lanes (n = D - 1, D - 2), bit picked by one count bit
    //   0: any set of classes, bit picked by the two low count bits
    auto compare_mode1 = [&](uint32_t q, uint32_t g, uint32_t hs, uint64_t U, uint64_t& acc) {
        // one call at a time: queue words need few calls here (side-by-side
        // pairs measured 4141 vs 4255 attempts/ns at L=16, k=200..219)
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            if (!U) break;
            const u32x4 o = plane_call(q, hs, 16u * g + (uint32_t)m);
            // the dE = 4 class has n = 2 unsatisfied bonds in 3D (v10), n = 1 in 2D (v01)
            plane_step_uniform((uint64_t)o.x | ((uint64_t)o.y << 32),
                               (D == 3) ? s.v10[2 * m] : s.v01[2 * m], U, acc);
            plane_step_uniform((uint64_t)o.z | ((uint64_t)o.w << 32),
                               (D == 3) ? s.v10[2 * m + 1] : s.v01[2 * m + 1], U, acc);
        }
    };
    auto compare_mode02 = [&](uint32_t q, uint32_t g, uint32_t hs, uint64_t& U, uint64_t b0, uint64_t b1,
                              uint64_t& acc, auto M0, auto M1) {
        constexpr int m0 = decltype(M0)::value, m1 = decltype(M1)::value;
        // planes where every threshold bit is 0 only reject (a 1 in r decides
        // r > thr): one masking step instead of the class selection
        const uint32_t zp = s.zero_planes;
        // the calls of a word are made kCP at a time (independent Philox
        // chains side by side, so that their multiplies overlap); a call made
        // after its word is decided changes nothing, since every step only
        // acts on the undecided lanes U.  L=16, k=5..24 (attempts/ns): one at a
        // time 2713; the first four calls together and then groups of
        // 2 / 3 / 4: 2817 / 2829 / 2797; first calls 3 + 1 or 2 + 2: 2767 / 2776
        constexpr int kCPI = 4, kCPQ = 3, kCPN = 1;
        // kCPN: the loop without late compaction (small lattices, the batch:
        // 512 instances at k=3..12, 1 / 2 / 4 calls side by side: 580.9 /
        // 578.2 / 565.9 attempts/ns)
        constexpr int kCP = m1 - m0 == 16 ? kCPN : m0 == 0 ? kCPI : kCPQ;
        auto run_calls = [&](auto step2) {
#pragma unroll
            for (int m = m0; m < m1; m += kCP) {
                if (!U) break;
                u32x4 o[kCP];
#pragma unroll
                for (int j = 0; j < kCP; ++j)
                    if (m + j < m1) o[j] = plane_call(q, hs, 16u * g + (uint32_t)(m + j));
#pragma unroll
                for (int j = 0; j < kCP; ++j)
                    if (m + j < m1) step2(m + j, o[j]);
            }
        };
        if (s.mode == 2) {
            const uint64_t sel = (D == 3) ? b1 : b0;  // 1 selects the dE = 4 class
            run_calls([&](int m, const u32x4& o) {
                const uint64_t p0 = (uint64_t)o.x | ((uint64_t)o.y << 32);
                const uint64_t p1 = (uint64_t)o.z | ((uint64_t)o.w << 32);
                if ((zp >> (2 * m)) & 1u) U &= ~p0;
                else plane_step_two(p0, (D == 3) ? s.v10[2 * m] : s.v01[2 * m],
                                    (D == 3) ? s.v01[2 * m] : s.v00[2 * m], sel, U, acc);
                if ((zp >> (2 * m + 1)) & 1u) U &= ~p1;
                else plane_step_two(p1, (D == 3) ? s.v10[2 * m + 1] : s.v01[2 * m + 1],
                                    (D == 3) ? s.v01[2 * m + 1] : s.v00[2 * m + 1], sel, U, acc);
            });
        } else if ((zp & 3u) == 3u) {
            // thresholds below 2^30: leading planes only reject
            run_calls([&](int m, const u32x4& o) {
                const uint64_t p0 = (uint64_t)o.x | ((uint64_t)o.y << 32);
                const uint64_t p1 = (uint64_t)o.z | ((uint64_t)o.w << 32);
                if ((zp >> (2 * m)) & 1u) U &= ~p0;
                else plane_step(p0, s.v00[2 * m], s.v01[2 * m], s.v10[2 * m], b0, b1, U, acc);
                if ((zp >> (2 * m + 1)) & 1u) U &= ~p1;
                else plane_step(p1, s.v00[2 * m + 1], s.v01[2 * m + 1], s.v10[2 * m + 1], b0, b1, U, acc);
            });
        } else {
            // high temperature: threshold bits of 1 from the first planes on
            run_calls([&](int m, const u32x4& o) {
                plane_step((uint64_t)o.x | ((uint64_t)o.y << 32), s.v00[2 * m], s.v01[2 * m],
                           s.v10[2 * m], b0, b1, U, acc);
                plane_step((uint64_t)o.z | ((uint64_t)o.w << 32), s.v00[2 * m + 1], s.v01[2 * m + 1],
                           s.v10[2 * m + 1], b0, b1, U, acc);
            });
        }
    };
    // lanes that flip without a comparison (acc) and lanes that need one (U)
    auto start = [&](uint64_t b0, uint64_t b1, uint64_t b2, uint64_t down, uint64_t& acc, uint64_t& U) {
        acc = down;  // in modes 2 and 3 no uphill class is always accepted
        if (s.mode == 3) {
            U = ~down;  // every uphill class undecided
        } else if (s.mode == 2) {
            U = ~down & ((D == 3) ? (b0 | b1) : ~0ull);
        } else {
            uint64_t m1, m2, m3;
            if (D == 3) {
                m3 = ~b2 & ~b1 & ~b0;  // n = 0: dE = 12
                m2 = ~b2 & ~b1 & b0;   // n = 1: dE = 8
                m1 = ~b2 & b1 & ~b0;   // n = 2: dE = 4
            } else {
                m3 = 0;
                m2 = ~b2 & ~b1 & ~b0;  // n = 0: dE = 8
                m1 = ~b2 & ~b1 & b0;   // n = 1: dE = 4
            }
            acc |= (m1 & alw1) | (m2 & alw2) | (m3 & alw3);
            U = (m1 & und1) | (m2 & und2) | (m3 & und3);
        }
    };
    // block queue: per round two counters (entries, next entry to take), then
    // the undecided masks and item indices
    int* qn = reinterpret_cast<int*>(qbuf);
    uint64_t* QU = reinterpret_cast<uint64_t*>(qbuf + 32);  // undecided lanes (late: class A)
    uint64_t* QB = QU + SH::QCAP;                              // late: class B
    uint16_t* Qt = reinterpret_cast<uint16_t*>(QU + (SH::kLate ? 2 : 1) * SH::QCAP);
    if (tid < 4) qn[tid] = 0;
    __syncthreads();
    int round = 0;
    // queue entries are claimed a warp at a time (one shared atomic per 32
    // entries); lane l takes entry e0 + l, and the loop ends for the whole warp
    // once a chunk starts past the queue
    auto claim = [&](int* next) {
        int e0 = 0;
        if (lane == 0) e0 = atomicAdd(next, 32);
        return __shfl_sync(0xffffffffu, e0, 0) + lane;
    };
    // mode 1 compacts every word with undecided lanes (at low temperature
    // most words have none: L=16 mode-1 steps 14.5 -> 12.0 ms); modes 0 and 2,
    // where most words have undecided lanes, compact only the words still
    // undecided after the first calls (below)
    const bool compact = s.mode == 1;
    // late compaction is measured faster for single 3D instances with L >= 8
    // (L=8: 2182 -> 2273 attempts/ns; L=16: 3108 -> 3197); the disorder batch
    // (L = 4..10, doubled groups per block) measured slower and keeps the loop
    constexpr bool kLate = SH::kLate;

    for (int sw = 0; sw < s.n_sweeps; ++sw) {
        for (int p = 0; p < 2; ++p) {
            const uint32_t hs = s.hs0 + 2u * (uint32_t)sw + (uint32_t)p;
            typename LT::Nb nb_fixed;
            if constexpr (THREADS % NH == 0) nb_fixed = LT::neighbours(p, tid % NH);
            if (compact) {
                // Words with undecided lanes are compacted into a block queue so
                // that the comparison loop runs on full warps: at low temperature
                // most words have no dE = 4 lane, the others need several planes.
                // Lanes with dE <= 0 are flipped at once; the queue entries, taken
                // one at a time by whichever thread is free, add the accepted ones.
                for (int base = 0; base < ng * NH; base += SH::QIPT * THREADS, ++round) {
                    int* cnt_r = qn + 2 * (round & 1);
#pragma unroll
                    for (int it = 0; it < SH::QIPT; ++it) {
                        const int t = base + it * THREADS + tid;
                        uint64_t U = 0;
                        if (t < ng * NH) {
                            uint64_t* cur;
                            int q;
                            uint64_t sw0, b0, b1, b2, down;
                            classify(t, p, nb_fixed, cur, q, sw0, b0, b1, b2, down);
                            cur[q] = sw0 ^ down;  // no uphill class is always accepted in mode 1
                            U = ~down & ((D == 3) ? b1 : b0);
                        }
                        const unsigned bal = __ballot_sync(0xffffffffu, U != 0);
                        int wb = 0;
                        if (lane == 0 && bal) wb = atomicAdd(cnt_r, __popc(bal));
                        wb = __shfl_sync(0xffffffffu, wb, 0);
                        if (U) {
                            const int slot = wb + __popc(bal & ((1u << lane) - 1u));
                            QU[slot] = U;
                            Qt[slot] = (uint16_t)t;
                        }
                    }
                    __syncthreads();
                    const int n = cnt_r[0];
                    if (tid == 0) { qn[2 * ((round + 1) & 1)] = 0; qn[2 * ((round + 1) & 1) + 1] = 0; }
                    for (int e = claim(cnt_r + 1); e - lane < n; e = claim(cnt_r + 1)) {
                        if (e < n) {
                            const int t2 = Qt[e], gl2 = t2 / NH, q2 = t2 - gl2 * NH;
                            uint64_t acc2 = 0;
                            compare_mode1((uint32_t)q2, (GPB == 1 ? (uint32_t)g0 : (uint32_t)(g0 + gl2)), hs, QU[e], acc2);
                            sm[(gl2 * 2 + p) * NH + q2] ^= acc2;
                        }
                    }
                    __syncthreads();
                }
            } else if constexpr (!kLate) {
                for (int t = tid; t < ng * NH; t += THREADS) {
                    uint64_t* cur;
                    int q;
                    uint64_t sw0, b0, b1, b2, down, acc, U;
                    classify(t, p, nb_fixed, cur, q, sw0, b0, b1, b2, down);
                    start(b0, b1, b2, down, acc, U);
                    compare_mode02((uint32_t)q, (GPB == 1 ? (uint32_t)g0 : (uint32_t)(g0 + t / NH)), hs, U, b0, b1, acc,
                                   std::integral_constant<int, 0>{}, std::integral_constant<int, 16>{});
                    cur[q] = sw0 ^ acc;
                }
                __syncthreads();
            } else {
                // Late compaction: every word gets its first KLATE Philox calls
                // in place; a warp then waits for its slowest word only that
                // far (L=16, k=5..24, queue claimed a warp at a time: 2 calls
                // 2293, 3 calls 2666, 4 calls 2714 attempts/ns; 5 calls measured
                // 2328 with per-thread claims).  The words still undecided go to the block queue with
                // the class bits of their undecided lanes (those lanes did not
                // flip, so their classes are unchanged) and finish there on full
                // warps, one word per thread, without classifying it again.
                // Class code of an undecided lane: A = n <= 1, B = n >= 1
                // (n = 0: A; n = 1: A and B; n = 2: B), so U = A | B,
                // b0 = A & B, b1 = B & ~A.
                constexpr int KLATE = 4;
                for (int base = 0; base < ng * NH; base += SH::QIPT * THREADS, ++round) {
                    int* cnt_r = qn + 2 * (round & 1);
#pragma unroll
                    for (int it = 0; it < SH::QIPT; ++it) {
                        const int t = base + it * THREADS + tid;
                        uint64_t U = 0, b0 = 0, b1 = 0;
                        if (t < ng * NH) {
                            uint64_t* cur;
                            int q;
                            uint64_t sw0, b2, down, acc;
                            classify(t, p, nb_fixed, cur, q, sw0, b0, b1, b2, down);
                            start(b0, b1, b2, down, acc, U);
                            compare_mode02((uint32_t)q, (GPB == 1 ? (uint32_t)g0 : (uint32_t)(g0 + t / NH)), hs, U, b0, b1, acc,
                                           std::integral_constant<int, 0>{}, std::integral_constant<int, KLATE>{});
                            cur[q] = sw0 ^ acc;
                        }
                        const unsigned bal = __ballot_sync(0xffffffffu, U != 0);
                        int wb = 0;
                        if (lane == 0 && bal) wb = atomicAdd(cnt_r, __popc(bal));
                        wb = __shfl_sync(0xffffffffu, wb, 0);
                        if (U) {
                            const int slot = wb + __popc(bal & ((1u << lane) - 1u));
                            QU[slot] = U & ~b1;         // A: n <= 1
                            QB[slot] = U & (b0 | b1);   // B: n >= 1
                            Qt[slot] = (uint16_t)t;
                        }
                    }
                    __syncthreads();
                    const int n = cnt_r[0];
                    if (tid == 0) { qn[2 * ((round + 1) & 1)] = 0; qn[2 * ((round + 1) & 1) + 1] = 0; }
                    for (int e = claim(cnt_r + 1); e - lane < n; e = claim(cnt_r + 1)) {
                        if (e < n) {
                            const int t2 = Qt[e], gl2 = t2 / NH, q2 = t2 - gl2 * NH;
                            const uint64_t A = QU[e], Bm = QB[e];
                            uint64_t U2 = A | Bm, acc2 = 0;
                            compare_mode02((uint32_t)q2, (GPB == 1 ? (uint32_t)g0 : (uint32_t)(g0 + gl2)), hs, U2, A & Bm, Bm & ~A, acc2,
                                           std::integral_constant<int, KLATE>{}, std::integral_constant<int, 16>{});
                            sm[(gl2 * 2 + p) * NH + q2] ^= acc2;  // lanes accepted in the queue
                        }
                    }
                    __syncthreads();
                }
            }
        }
    }

    // ---- write back ----
    if (!I8) {
        for (int t = tid; t < ng * N; t += THREADS) {
            int gl = t / N, i = t - gl * N;
            in.S[(size_t)(g0 + gl) * N + i] = sm[(gl * 2 + site_parity<D, L>(i)) * NH + (i >> 1)];
        }
    } else {
        const int nchunk = in.NP / 16;
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
            if (r < R)
                *reinterpret_cast<uint4*>(in.S8_out + (size_t)r * in.NP + 16 * c) =
                    make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
    }

    // ---- energies: vertical counters of unsatisfied bonds ----
    {
        const int gl = tid / TPG, lt = tid - gl * TPG;
        // a thread counts at most ceil(N / TPG) sites of D bonds each
        constexpr int W = bits_for(((N + TPG - 1) / TPG) * D) > 2 ? bits_for(((N + TPG - 1) / TPG) * D) : 2;
        static_assert(W <= B, "per-thread counter fits the block counter");
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
                uint64_t ub[3] = {0, 0, 0};  // unsatisfied +e_d bonds of site i
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    const int j = nbs[d];
                    const uint64_t sjw = base[(p ^ 1) * NH + (j >> 1)];
                    ub[d] = si ^ sjw ^ (((jm >> (2 * d + 1)) & 1u) ? ~0ull : 0ull);
                }
                // the site's count (0..D) as two bit-sliced bits, added into the
                // thread's counter, whose width W covers this thread's sites only
                const uint64_t lo = ub[0] ^ ub[1] ^ ub[2], hi = maj3(ub[0], ub[1], ub[2]);
                uint64_t carry = C[0] & lo;
                C[0] ^= lo;
                uint64_t c2 = maj3(C[1], hi, carry);
                C[1] ^= hi ^ carry;
                carry = c2;
#pragma unroll
                for (int b = 2; b < W; ++b) {
                    const uint64_t tt = C[b] & carry;
                    C[b] ^= carry;
                    carry = tt;
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
        if (r < R) in.E[r] = 2 * n - D * N;
    }
    __syncthreads();  // the tile's shared memory is reused by the next tile
}

// ---------------- real couplings, int8 spins ----------------
//
// Shared memory: the spin tile T[parity][q][32] (bytes), then per site record
// (parity, q) the couplings to the 2D neighbours in field order, h_i, and the
// neighbours' byte offsets in the other parity's tile:
//   Jrec[(p NH + q)] = {J_-x, J_+x, J_-y, J_+y}, {J_-z, J_+z, h_i, offsets 0|1}
//   Orec[(p NH + q)] = {offsets 2|3, offsets 4|5}      (16-bit each)
// then (only with gradient counts) the block's integer bond/site sums.  The
// energy epilogue's int128 partials reuse the spin tile after a barrier.

template <int D, int L, int WARPS>
struct RealShape {
    static constexpr int N = Lat<D, L>::N, NH = Lat<D, L>::NH;
    // spin tile, also holding the epilogue's int128 partials (one per lane and warp)
    static constexpr size_t T8 = ((size_t)N * 32 > (size_t)WARPS * 32 * 16) ? (size_t)N * 32
                                                                              : (size_t)WARPS * 32 * 16;
    static constexpr size_t JREC = (size_t)N * 32;    // 2 x float4 per site
    static constexpr size_t OREC = (size_t)N * 8;     // uint2 per site
    static constexpr size_t GR = (size_t)(D + 1) * N * 4;
    static constexpr size_t SMEM = T8 + JREC + OREC;
    static constexpr size_t SMEM_GRAD = SMEM + GR;
    static_assert(NH * 32 < 65536, "16-bit neighbour offsets");
};

// site records (once per instance); zero the block's gradient sums if asked
template <int D, int L, int WARPS>
__device__ __forceinline__ void real_stage(const RealInst& in, unsigned char* smem, bool zero_grad)
{
    using LT = Lat<D, L>;
    using SH = RealShape<D, L, WARPS>;
    constexpr int N = SH::N, NH = SH::NH;
    float4* Jrec = reinterpret_cast<float4*>(smem + SH::T8);
    uint2* Orec = reinterpret_cast<uint2*>(smem + SH::T8 + SH::JREC);
    for (int t = threadIdx.x; t < N; t += WARPS * 32) {
        const int p = t / NH, q = t - p * NH;
        const auto nb = LT::neighbours(p, q);
        float Jn[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        uint32_t off[6] = {0u, 0u, 0u, 0u, 0u, 0u};
#pragma unroll
        for (int kk = 0; kk < 2 * D; ++kk) {
            const int d = kk >> 1;
            Jn[kk] = in.J[d * N + ((kk & 1) ? nb.site : nb.site_m[d])];
            off[kk] = (uint32_t)nb.q[kk] * 32u;
        }
        Jrec[2 * t] = make_float4(Jn[0], Jn[1], Jn[2], Jn[3]);
        Jrec[2 * t + 1] = make_float4(Jn[4], Jn[5], in.h[nb.site], __uint_as_float(off[0] | (off[1] << 16)));
        Orec[t] = make_uint2(off[2] | (off[3] << 16), off[4] | (off[5] << 16));
    }
    if (zero_grad) {
        int* gJ = reinterpret_cast<int*>(smem + SH::SMEM);
        for (int t = threadIdx.x; t < (D + 1) * N; t += WARPS * 32) gJ[t] = 0;
    }
    __syncthreads();
}

// add this block's gradient counts to the step's global counters
template <int D, int L, int WARPS>
__device__ __forceinline__ void real_flush_grad(const RealInst& in, unsigned char* smem)
{
    using SH = RealShape<D, L, WARPS>;
    constexpr int N = SH::N;
    const int* gJ = reinterpret_cast<const int*>(smem + SH::SMEM);
    const int* gh = gJ + D * N;
    __syncthreads();
    for (int t = threadIdx.x; t < D * N; t += WARPS * 32)
        if (gJ[t]) atomicAdd(&in.cJ[t], (unsigned long long)(long long)gJ[t]);
    for (int t = threadIdx.x; t < N; t += WARPS * 32)
        if (gh[t]) atomicAdd(&in.ch[t], (unsigned long long)(long long)gh[t]);
}

// ---- Metropolis acceptance for real couplings (Sec. II.B) ----
// The specified rule for x = beta dE: accept iff x <= 0, or e == 1, or
// r < floor(e 2^32) with e = spec_expf(-x).
__device__ __forceinline__ bool accept_real_exact(float x, uint32_t r)
{
    const float e = spec_expf(fminf(-x, 0.0f));
    return (x <= 0.0f) || (e == 1.0f) || (r < __float2uint_rz(mul32(e, 4294967296.0f)));
}

// Guard band around the specified threshold, from the hardware base-2
// exponential g = 2^(-x log2 e) (ex2.approx.ftz, about 2^-20 from exp(-x)):
// lo = trunc(g 2^32 (1 - 2^-14)), hi = trunc(g 2^32 (1 + 2^-14)).  A lane with
// r < lo accepts and a lane with r > hi rejects under the specified rule too,
// provided lo <= thr(x) and hi + 1 >= thr(x) for the specified threshold
// thr(x) (2^32 when e == 1, else floor(e 2^32)).  accept_band_check verifies
// both inequalities on the device for every positive finite float x; lanes
// with lo <= r <= hi (probability about 2^-13 e) take the specified rule.
struct AcceptBand {
    uint32_t lo, hi;
};
__device__ __forceinline__ float ex2_approx(float y)
{
    float g;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(g) : "f"(y));
    return g;
}
__device__ __forceinline__ AcceptBand accept_band(float x)
{
    const float g = ex2_approx(mul32(x, -0x1.715476p+0f));
    return {__float2uint_rz(mul32(g, 0x1.fff8p+31f)), __float2uint_rz(mul32(g, 0x1.0004p+32f))};
}

// replicas [32 tile, 32 tile + 32) of one instance
template <int D, int L, int WARPS>
__device__ __forceinline__ void sweep_real_tile(const RealStep& s, const RealInst& in, int tile,
                                                unsigned char* smem, bool grad)
{
    using LT = Lat<D, L>;
    using SH = RealShape<D, L, WARPS>;
    constexpr int N = SH::N, NH = SH::NH;
    constexpr int NB = (NH + 3) / 4;
    int8_t* T = reinterpret_cast<int8_t*>(smem);
    const float4* Jrec = reinterpret_cast<const float4*>(smem + SH::T8);
    const uint2* Orec = reinterpret_cast<const uint2*>(smem + SH::T8 + SH::JREC);
    __int128* Ep = reinterpret_cast<__int128*>(smem);  // reuses the spin tile after the epilogue
    int* gJ = reinterpret_cast<int*>(smem + SH::SMEM);
    int* gh = gJ + D * N;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int R = in.Rdev ? __ldg(in.Rdev) : in.R, NP = in.NP;
    const uint32_t c3 = in.c3;
    const int nchunk = NP / 16;
    const int r0 = tile * 32;
    const int r = r0 + lane;
    const bool valid = r < R;
    // ---- prologue: rows (gathered through parent) -> T[parity][q][lane]
    const int src = valid ? (in.parent ? in.parent[r] : r) : 0;
    for (int c = warp; c < nchunk; c += WARPS) {
        uint4 v = make_uint4(0x01010101u, 0x01010101u, 0x01010101u, 0x01010101u);
        if (valid) v = *reinterpret_cast<const uint4*>(in.Sin + (size_t)src * NP + 16 * c);
        const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int i = 16 * c + t;
            if (i < N) {
                const int x = i % L, y = (i / L) % L, z = (D == 3) ? i / (L * L) : 0;
                const int p = (x + y + z) & 1;
                T[(p * NH + (i >> 1)) * 32 + lane] = (int8_t)(wv[t >> 2] >> (8 * (t & 3)));
            }
        }
    }
    __syncthreads();
    // ---- N_S sweeps
    for (int sw = 0; sw < s.n_sweeps; ++sw) {
        for (int p = 0; p < 2; ++p) {
            const uint32_t hsw = s.hs0 + 2u * (uint32_t)sw + (uint32_t)p;
            const int8_t* oth = T + (p ^ 1) * NH * 32;
            int8_t* cur = T + p * NH * 32;
            for (int blk = warp; blk < NB; blk += WARPS) {
                const u32x4 o = philox_rk((uint32_t)blk, hsw, (uint32_t)r, c3, s.rk);
                const uint32_t rs[4] = {o.x, o.y, o.z, o.w};
                // the four sites of one random-number block are independent (same
                // parity): fields and energy changes first, then decisions, then stores
                float xs[4];
                int sis[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int q = (NH % 4 != 0 && 4 * blk + t >= NH) ? 4 * blk : 4 * blk + t;
                    const int rec = p * NH + q;
                    const float4 ja = Jrec[2 * rec], jb = Jrec[2 * rec + 1];
                    const uint2 ob = Orec[rec];
                    const uint32_t o01 = __float_as_uint(jb.w);
                    const float Jn[6] = {ja.x, ja.y, ja.z, ja.w, jb.x, jb.y};
                    const uint32_t off[6] = {o01 & 0xFFFFu, o01 >> 16, ob.x & 0xFFFFu, ob.x >> 16,
                                             ob.y & 0xFFFFu, ob.y >> 16};
                    const int si = cur[q * 32 + lane];
                    float f = 0.0f;
#pragma unroll
                    for (int kk = 0; kk < 2 * D; ++kk) {
                        const int sn = oth[off[kk] + lane];
                        const float tt = __int_as_float(__float_as_int(Jn[kk]) ^ (sn & (int)0x80000000));
                        f = (kk == 0) ? tt : add32(f, tt);
                    }
                    f = add32(f, jb.z);
                    const float dE = mul32(f, si > 0 ? 2.0f : -2.0f);
                    xs[t] = mul32(s.beta, dE);
                    sis[t] = si;
                }
                // decisions: the guard band settles almost every lane; a lane
                // inside it (or every lane without a verified band) takes the
                // specified rule, the same decision either way
                bool accs[4], und[4];
                bool any = false;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const AcceptBand bd = accept_band(xs[t]);
                    const bool up = xs[t] > 0.0f;
                    accs[t] = !up || rs[t] < bd.lo;
                    und[t] = up && (!s.band || (rs[t] >= bd.lo && rs[t] <= bd.hi));
                    any |= und[t];
                }
                if (__any_sync(0xffffffffu, any)) {
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (und[t]) accs[t] = accept_real_exact(xs[t], rs[t]);
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int q = 4 * blk + t;
                    if (NH % 4 != 0 && q >= NH) break;
                    if (accs[t]) cur[q * 32 + lane] = (int8_t)(-sis[t]);
                }
            }
            __syncthreads();
        }
    }
    // ---- epilogue: rows out
    for (int c = warp; c < nchunk; c += WARPS) {
        uint32_t wv[4] = {0x01010101u, 0x01010101u, 0x01010101u, 0x01010101u};
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int i = 16 * c + t;
            if (i < N) {
                const int x = i % L, y = (i / L) % L, z = (D == 3) ? i / (L * L) : 0;
                const int p = (x + y + z) & 1;
                const uint32_t b = (uint8_t)T[(p * NH + (i >> 1)) * 32 + lane];
                wv[t >> 2] = (wv[t >> 2] & ~(0xFFu << (8 * (t & 3)))) | (b << (8 * (t & 3)));
            }
        }
        if (valid)
            *reinterpret_cast<uint4*>(in.Sout + (size_t)r * NP + 16 * c) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
    }
    // ---- energies (exact, int128) and gradient counts
    __int128 e = 0;
    for (int i = warp; i < N; i += WARPS) {
        const int x = i % L, y = (i / L) % L, z = (D == 3) ? i / (L * L) : 0;
        const int p = (x + y + z) & 1;
        const int si = T[(p * NH + (i >> 1)) * 32 + lane];
        int nbs[3];
        nbs[0] = i - x + (x == L - 1 ? 0 : x + 1);
        nbs[1] = i + ((y == L - 1) ? -(L - 1) * L : L);
        if (D == 3) nbs[2] = i + ((z == L - 1) ? -(L - 1) * L * L : L * L);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int j = nbs[d];
            const int sj = T[((p ^ 1) * NH + (j >> 1)) * 32 + lane];
            const longlong2 jf = __ldg(&in.Jfix[d * N + i]);
            __int128 v = ((__int128)jf.y << 64) | (unsigned long long)jf.x;
            const int sig = si * sj;
            e -= (sig > 0) ? v : -v;
            if (grad) {
                const int tot = __reduce_add_sync(0xffffffffu, valid ? sig : 0);
                if (lane == 0) gJ[d * N + i] += tot;
            }
        }
        {
            const longlong2 hf = __ldg(&in.hfix[i]);
            __int128 v = ((__int128)hf.y << 64) | (unsigned long long)hf.x;
            e -= (si > 0) ? v : -v;
        }
        if (grad) {
            const int tot = __reduce_add_sync(0xffffffffu, valid ? si : 0);
            if (lane == 0) gh[i] += tot;
        }
    }
    __syncthreads();  // every warp is done reading the spin tile
    Ep[warp * 32 + lane] = e;
    __syncthreads();
    if (warp == 0) {
        __int128 tot = 0;
        for (int w = 0; w < WARPS; ++w) tot += Ep[w * 32 + lane];
        if (valid) {
            longlong2 out;
            out.x = (long long)(unsigned long long)tot;
            out.y = (long long)(tot >> 64);
            in.E[r] = out;
        }
    }
    __syncthreads();  // T and Ep are reused by the next tile
}

}  // namespace pa
