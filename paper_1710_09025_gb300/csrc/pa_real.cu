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
#include "pa_sweep_tiles.cuh"

#include <cstring>
#include <mutex>

namespace pa {

// ---- verification of the acceptance guard band ----
__device__ unsigned long long g_band_violations;
__device__ unsigned int g_band_maxdev;  // float bits of the largest relative deviation

// every positive finite float x (bit patterns 1 .. 0x7f7fffff)
__global__ void __launch_bounds__(256) accept_band_check_kernel()
{
    unsigned long long viol = 0;
    float dev = 0.0f;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t u = 1 + blockIdx.x * blockDim.x + threadIdx.x; u <= 0x7f7fffffu; u += stride) {
        const float x = __uint_as_float(u);
        const float e = spec_expf(-x);
        const unsigned long long thr = (e == 1.0f) ? (1ull << 32) : __float2uint_rz(mul32(e, 4294967296.0f));
        const AcceptBand bd = accept_band(x);
        viol += (bd.lo > thr) || ((unsigned long long)bd.hi + 1ull < thr);
        if (x <= 87.0f && e > 0.0f) {
            const float g = ex2_approx(mul32(x, -0x1.715476p+0f));
            const double d = fabs((double)g - (double)e) / (double)e;
            dev = fmaxf(dev, __double2float_ru(d));
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        viol += __shfl_down_sync(0xffffffffu, viol, off);
        dev = fmaxf(dev, __shfl_down_sync(0xffffffffu, dev, off));
    }
    if ((threadIdx.x & 31) == 0) {
        if (viol) atomicAdd(&g_band_violations, viol);
        atomicMax(&g_band_maxdev, __float_as_uint(dev));  // non-negative floats order as their bits
    }
}

cudaError_t accept_band_check(cudaStream_t st, unsigned long long* violations, double* max_rel_dev)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned long long z = 0;
    const unsigned int zu = 0;
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(g_band_violations, &z, sizeof z, 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(g_band_maxdev, &zu, sizeof zu, 0, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    accept_band_check_kernel<<<sms * 8, 256, 0, st>>>();
    e = cudaGetLastError();
    unsigned long long v = 0;
    unsigned int d = 0;
    if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(&v, g_band_violations, sizeof v, 0, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(&d, g_band_maxdev, sizeof d, 0, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    float df;
    std::memcpy(&df, &d, sizeof df);
    if (violations) *violations = v;
    if (max_rel_dev) *max_rel_dev = df;
    return cudaSuccess;
}

int accept_band_ok(cudaStream_t st)
{
    static std::mutex mu;
    static int verdict[64];  // 0 unknown, 1 verified, 2 failed
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    std::lock_guard<std::mutex> g(mu);
    if (verdict[dev] == 0) {
        unsigned long long v = 1;
        if (accept_band_check(st, &v, nullptr) != cudaSuccess) return 0;
        verdict[dev] = v == 0 ? 1 : 2;
    }
    return verdict[dev] == 1;
}

// persistent over the instance's tiles of 32 replicas
template <int D, int L, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) sweep_real_kernel(RealSweepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_real[];
    const bool grad = a.i.cJ != nullptr;
    real_stage<D, L, WARPS>(a.i, smem_real, grad);
    const int ntiles = ((a.i.Rdev ? __ldg(a.i.Rdev) : a.i.R) + 31) / 32;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
        sweep_real_tile<D, L, WARPS>(a.s, a.i, tile, smem_real, grad);
    if (grad) real_flush_grad<D, L, WARPS>(a.i, smem_real);
}

template <int D, int L, int WARPS>
static cudaError_t launch_real_one(const RealSweepArgs& a, int grid, cudaStream_t st)
{
    const size_t smem = a.i.cJ ? RealShape<D, L, WARPS>::SMEM_GRAD : RealShape<D, L, WARPS>::SMEM;
    auto kern = sweep_real_kernel<D, L, WARPS>;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)RealShape<D, L, WARPS>::SMEM_GRAD);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    if (grid <= 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, WARPS * 32, smem);
        int ntiles = (a.i.R + 31) / 32;
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
__global__ void init_i8_kernel(int8_t* S, int N, int NP, int R, uint32_t k0, uint32_t k1, uint32_t c3, int goff)
{
    const int G = (R + 63) / 64;
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)N * G) return;
    int g = (int)(t / N), i = (int)(t - (size_t)g * N);
    u32x4 o = philox((uint32_t)i, (uint32_t)(g + goff), 0u, c3, k0, k1);
    uint64_t w = (uint64_t)o.x | ((uint64_t)o.y << 32);
    for (int j = 0; j < 64; ++j) {
        int r = 64 * g + j;
        if (r >= R) break;
        S[(size_t)r * NP + i] = ((w >> j) & 1ull) ? (int8_t)-1 : (int8_t)1;
    }
}

cudaError_t launch_init_i8(int8_t* S, int N, int NP, int R, uint32_t k0, uint32_t k1, uint32_t c3,
                           cudaStream_t st, int goff)
{
    cudaError_t e = cudaMemsetAsync(S, 0x01, (size_t)R * NP, st);
    if (e != cudaSuccess) return e;
    size_t n = (size_t)N * ((R + 63) / 64);
    init_i8_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(S, N, NP, R, k0, k1, c3, goff);
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
