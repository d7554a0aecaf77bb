// pa_real.cu -- real (Gaussian) couplings: int8 spins, FP32 local fields.
//
// Sec. II.B Metropolis sweeps (checkerboard order of Sec. III.A) for
// H = -sum J_ij S_i S_j - sum h_i S_i with FP32 couplings (Sec. II.A draws
// J from a Gaussian).  A block takes tiles of 32 replicas; the tile is staged
// in shared memory transposed to [parity][q][replica] bytes so that a warp
// (one lane per replica) updates the same site of 32 replicas: couplings are
// warp-uniform broadcast loads and spin loads are 32 consecutive bytes.
// Resampling's replica gather is fused into the tile load (row parent[r]).
//
// Acceptance: f = ((((t_-x + t_+x) + t_-y) + t_+y) + ...) + h_i in FP32 with
// t = J S_nb (exact sign flip), dE = 2 S_i f (exact), x = f32(beta) * dE;
// accept iff x <= 0 or r < floor(spec_expf(-x) 2^32).  r comes from the WORD
// stream: one Philox call per replica and four consecutive sublattice sites.
//
// Energies are exact: E * 2^96 is an integer for FP32 couplings of magnitude
// >= 2^-73, accumulated in int128, so the sum does not depend on order.
#include "pa_device.cuh"
#include "pa_internal.h"

namespace pa {

template <int D, int L, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) sweep_real_kernel(RealSweepArgs a)
{
    using LT = Lat<D, L>;
    constexpr int N = LT::N, NH = LT::NH;
    constexpr int NB = (NH + 3) / 4;
    extern __shared__ __align__(16) unsigned char smraw[];
    int8_t* T = reinterpret_cast<int8_t*>(smraw);                                   // N*32
    float* Js = reinterpret_cast<float*>(smraw + N * 32);                            // D*N
    float* hs = Js + D * N;                                                          // N
    __int128* Ep = reinterpret_cast<__int128*>(hs + N + ((4 - (((D + 1) * N) & 3)) & 3)); // WARPS*32
    int* gJ = reinterpret_cast<int*>(Ep + WARPS * 32);                               // D*N
    int* gh = gJ + D * N;                                                            // N

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool grad = a.cJ != nullptr;
    for (int t = tid; t < D * N; t += WARPS * 32) Js[t] = a.J[t];
    for (int t = tid; t < N; t += WARPS * 32) hs[t] = a.h[t];
    if (grad) {
        for (int t = tid; t < D * N; t += WARPS * 32) gJ[t] = 0;
        for (int t = tid; t < N; t += WARPS * 32) gh[t] = 0;
    }
    const int ntiles = (a.R + 31) / 32;
    const int nchunk = a.NP / 16;

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int r0 = tile * 32;
        const int r = r0 + lane;
        const bool valid = r < a.R;
        __syncthreads();  // previous tile's epilogue finished with T
        // ---- prologue: rows (gathered through parent) -> T[parity][q][lane]
        const int src = valid ? (a.parent ? a.parent[r] : r) : 0;
        for (int c = warp; c < nchunk; c += WARPS) {
            uint4 v = make_uint4(0x01010101u, 0x01010101u, 0x01010101u, 0x01010101u);
            if (valid) v = *reinterpret_cast<const uint4*>(a.Sin + (size_t)src * a.NP + 16 * c);
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
        for (int sw = 0; sw < a.n_sweeps; ++sw) {
            for (int p = 0; p < 2; ++p) {
                const uint32_t hsw = 2u * (uint32_t)(a.k * a.n_sweeps + sw) + (uint32_t)p;
                const int8_t* oth = T + (p ^ 1) * NH * 32;
                int8_t* cur = T + p * NH * 32;
                for (int blk = warp; blk < NB; blk += WARPS) {
                    const u32x4 o = philox((uint32_t)blk, hsw, (uint32_t)r, a.c3, a.key0, a.key1);
                    const uint32_t rs[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int q = 4 * blk + t;
                        if (NH % 4 != 0 && q >= NH) break;
                        const auto nb = LT::neighbours(p, q);
                        const int si = cur[q * 32 + lane];
                        float f = 0.0f;
#pragma unroll
                        for (int kk = 0; kk < 2 * D; ++kk) {
                            const int d = kk >> 1;
                            const float Jb = Js[d * N + ((kk & 1) ? nb.site : nb.site_m[d])];
                            const int sn = oth[nb.q[kk] * 32 + lane];
                            const float tt = __int_as_float(__float_as_int(Jb) ^ (sn & (int)0x80000000));
                            f = (kk == 0) ? tt : add32(f, tt);
                        }
                        f = add32(f, hs[nb.site]);
                        const float dE = mul32(f, si > 0 ? 2.0f : -2.0f);
                        const float x = mul32(a.beta, dE);
                        bool acc = x <= 0.0f;
                        if (!acc) {
                            const float e = spec_expf(-x);
                            const unsigned long long thr = __float2ull_rz(mul32(e, 4294967296.0f));
                            acc = (unsigned long long)rs[t] < thr;
                        }
                        if (acc) cur[q * 32 + lane] = (int8_t)(-si);
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
                *reinterpret_cast<uint4*>(a.Sout + (size_t)r * a.NP + 16 * c) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
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
                const longlong2 jf = __ldg(&a.Jfix[d * N + i]);
                __int128 v = ((__int128)jf.y << 64) | (unsigned long long)jf.x;
                const int sig = si * sj;
                e -= (sig > 0) ? v : -v;
                if (grad) {
                    const int tot = __reduce_add_sync(0xffffffffu, valid ? sig : 0);
                    if (lane == 0) gJ[d * N + i] += tot;
                }
            }
            if (a.hfix) {
                const longlong2 hf = __ldg(&a.hfix[i]);
                __int128 v = ((__int128)hf.y << 64) | (unsigned long long)hf.x;
                e -= (si > 0) ? v : -v;
            }
            if (grad) {
                const int tot = __reduce_add_sync(0xffffffffu, valid ? si : 0);
                if (lane == 0) gh[i] += tot;
            }
        }
        Ep[warp * 32 + lane] = e;
        __syncthreads();
        if (warp == 0) {
            __int128 tot = 0;
            for (int w = 0; w < WARPS; ++w) tot += Ep[w * 32 + lane];
            if (valid) {
                longlong2 out;
                out.x = (long long)(unsigned long long)tot;
                out.y = (long long)(tot >> 64);
                a.E[r] = out;
            }
        }
    }
    if (grad) {
        __syncthreads();
        for (int t = tid; t < D * N; t += WARPS * 32)
            if (gJ[t]) atomicAdd(&a.cJ[t], (unsigned long long)(long long)gJ[t]);
        for (int t = tid; t < N; t += WARPS * 32)
            if (gh[t]) atomicAdd(&a.ch[t], (unsigned long long)(long long)gh[t]);
    }
}

template <int D, int L>
static size_t real_smem(int warps)
{
    constexpr int N = Lat<D, L>::N;
    size_t off = (size_t)N * 32 + (size_t)(D + 1) * N * 4;
    off = (off + 15) & ~(size_t)15;
    off += (size_t)warps * 32 * 16;
    off += (size_t)(D + 1) * N * 4;
    return off;
}

template <int D, int L, int WARPS>
static cudaError_t launch_real_one(const RealSweepArgs& a, int grid, cudaStream_t st)
{
    size_t smem = real_smem<D, L>(WARPS);
    auto kern = sweep_real_kernel<D, L, WARPS>;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    if (grid <= 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, WARPS * 32, smem);
        int ntiles = (a.R + 31) / 32;
        grid = sms * (per > 0 ? per : 1);
        if (grid > ntiles) grid = ntiles;
    }
    kern<<<grid, WARPS * 32, smem, st>>>(a);
    return cudaGetLastError();
}

#define PA_REAL_CASES(X) \
    X(3, 2) X(3, 4) X(3, 6) X(3, 8) X(3, 10) X(3, 12) \
    X(2, 2) X(2, 4) X(2, 6) X(2, 8) X(2, 10) X(2, 12) X(2, 16) X(2, 32)

bool real_supported(int D, int L)
{
#define X(d, l) if (D == d && L == l) return true;
    PA_REAL_CASES(X)
#undef X
    return false;
}

cudaError_t launch_sweep_real(int D, int L, const RealSweepArgs& a, int warps, int grid,
                              cudaStream_t st)
{
#define X(d, l)                                                                \
    if (D == d && L == l) {                                                    \
        if (warps == 4) return launch_real_one<d, l, 4>(a, grid, st);          \
        return launch_real_one<d, l, 8>(a, grid, st);                          \
    }
    PA_REAL_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

// Sec. II.B: random initial replicas; same INIT stream as the packed layout.
__global__ void init_i8_kernel(int8_t* S, int N, int NP, int R, uint32_t k0, uint32_t k1, uint32_t c3)
{
    const int G = (R + 63) / 64;
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)N * G) return;
    int g = (int)(t / N), i = (int)(t - (size_t)g * N);
    u32x4 o = philox((uint32_t)i, (uint32_t)g, 0u, c3, k0, k1);
    uint64_t w = (uint64_t)o.x | ((uint64_t)o.y << 32);
    for (int j = 0; j < 64; ++j) {
        int r = 64 * g + j;
        if (r >= R) break;
        S[(size_t)r * NP + i] = ((w >> j) & 1ull) ? (int8_t)-1 : (int8_t)1;
    }
}

cudaError_t launch_init_i8(int8_t* S, int N, int NP, int R, uint32_t k0, uint32_t k1, uint32_t c3,
                           cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(S, 0x01, (size_t)R * NP, st);
    if (e != cudaSuccess) return e;
    size_t n = (size_t)N * ((R + 63) / 64);
    init_i8_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(S, N, NP, R, k0, k1, c3);
    return cudaGetLastError();
}

__global__ void overlap_i8_kernel(const int8_t* A, const int8_t* B, int N, int NP, int R,
                                  unsigned long long* hist)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int8_t* a = A + (size_t)r * NP;
    const int8_t* b = B + (size_t)r * NP;
    int nd = 0;
    for (int i = 0; i < N; ++i) nd += a[i] != b[i];
    atomicAdd(&hist[N - nd], 1ull);
}

cudaError_t launch_overlap_i8(const int8_t* A, const int8_t* B, int N, int NP, int R,
                              unsigned long long* hist, cudaStream_t st)
{
    overlap_i8_kernel<<<(R + 127) / 128, 128, 0, st>>>(A, B, N, NP, R, hist);
    return cudaGetLastError();
}

}  // namespace pa
