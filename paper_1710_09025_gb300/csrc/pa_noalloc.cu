// pa_noalloc.cu -- resampling without any device allocation.
//
// Some callers cannot call cudaMalloc at all: allocator-less embedded
// runtimes, or hosts whose memory manager owns every device byte and hands
// out only the input and output buffers.  pa_resample_static gives them the resampling step of
// pa_anneal_step (weights, fixed-order prefix, multinomial draws, parents,
// ln Q) with its scratch in one file-scope device array instead of a
// context workspace.  The caller passes only inputs and outputs.
//
// The array is a module global: every GPU that loads the library holds its
// PA_STATIC_SCRATCH_BYTES until the process exits.  Host code may not pass
// the array's name to a kernel (on the host it is only a stand-in symbol),
// so the device address is looked up once per device with
// cudaGetSymbolAddress while that device is current, and cached for the life
// of the process (a device reset after the first call is not supported).
#include "pa.h"
#include "pa_device.cuh"
#include "pa_internal.h"

#include <cmath>
#include <mutex>
#include <string>

namespace {

constexpr int kMaxR = PA_STATIC_MAX_R;
constexpr int kMaxLeaves = (kMaxR + pa::kFan - 1) / pa::kFan;
constexpr int kMaxUpper = 2 * ((kMaxR + pa::kWBlock - 1) / pa::kWBlock) + 64;  // levels >= 2
constexpr int kMaxScanBlocks = (kMaxR + pa::kScanBlock - 1) / pa::kScanBlock;

// carve-up of the scratch array (byte offsets, each 256-byte aligned)
constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffW = 0;
constexpr size_t kOffP = kOffW + al(sizeof(double) * kMaxR);
constexpr size_t kOffCounts = kOffP + al(sizeof(double) * kMaxR);
constexpr size_t kOffFamIn = kOffCounts + al(sizeof(int32_t) * kMaxR);
constexpr size_t kOffFamOut = kOffFamIn + al(sizeof(int32_t) * kMaxR);
constexpr size_t kOffLev1 = kOffFamOut + al(sizeof(int32_t) * kMaxR);
constexpr size_t kOffBmax = kOffLev1 + al(sizeof(double) * kMaxLeaves);
constexpr size_t kOffUpper = kOffBmax + al(sizeof(double) * 2 * ((kMaxR + pa::kWBlock - 1) / pa::kWBlock));
constexpr size_t kOffBlock = kOffUpper + al(sizeof(double) * kMaxUpper);
constexpr size_t kOffAcc = kOffBlock + al(sizeof(int32_t) * (kMaxScanBlocks + 1));
constexpr size_t kBytes = kOffAcc + al(2 * sizeof(pa::StepAcc));
static_assert(kBytes <= PA_STATIC_SCRATCH_BYTES, "scratch layout exceeds the stated size");
static_assert(pa::rs_upper_size(kMaxR) <= kMaxUpper, "upper prefix levels fit");

}  // namespace

// The scratch itself: zero-initialised at module load, shared by every call.
static __device__ __align__(256) unsigned char pa_static_scratch[PA_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

// E_min into prev (as pa_anneal_step takes it from the previous step's
// observables), zero copy counts, identity families, zero running sums.
__global__ void __launch_bounds__(1024) static_prep_kernel(const int32_t* E, int R, unsigned char* base)
{
    __shared__ int wmin[32];
    int32_t* counts = reinterpret_cast<int32_t*>(base + kOffCounts);
    int32_t* fam = reinterpret_cast<int32_t*>(base + kOffFamIn);
    pa::StepAcc* acc = reinterpret_cast<pa::StepAcc*>(base + kOffAcc);
    int mn = 0x7fffffff;
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        mn = min(mn, E[r]);
        counts[r] = 0;
        fam[r] = r;
    }
    mn = __reduce_min_sync(0xffffffffu, mn);
    if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = mn;
    __syncthreads();
    if (threadIdx.x < 32) {
        int v = __reduce_min_sync(0xffffffffu, wmin[threadIdx.x]);
        if (threadIdx.x == 0) {
            acc[0] = pa::StepAcc{};
            acc[1] = pa::StepAcc{};
            acc[0].emin_lo = v;
            acc[0].emin_hi = v < 0 ? -1 : 0;
        }
    }
}

__global__ void static_lnq_kernel(const unsigned char* base, double* lnQ)
{
    *lnQ = reinterpret_cast<const pa::StepAcc*>(base + kOffAcc)[1].lnQ;
}

}  // namespace

extern "C" int pa_resample_static(const int32_t* d_E, int R, double beta_prev, double beta_next,
                                  int k, uint64_t seed, uint32_t rng_instance, uint32_t rng_tag,
                                  int32_t* d_parent, double* d_lnQ, void* stream)
{
    if (R < 1 || R > kMaxR) {
        pa::set_global_error("pa_resample_static: R must be in [1, PA_STATIC_MAX_R = 65536]");
        return PA_EINVAL;
    }
    if (!d_E || !d_parent || !d_lnQ) {
        pa::set_global_error("pa_resample_static: NULL pointer argument");
        return PA_EINVAL;
    }
    if (!std::isfinite(beta_prev) || !std::isfinite(beta_next) || beta_next < beta_prev || k < 0) {
        pa::set_global_error("pa_resample_static: need finite beta_prev <= beta_next and k >= 0");
        return PA_EINVAL;
    }
    if (rng_instance >= (1u << 24) || rng_tag >= 16u) {
        pa::set_global_error("pa_resample_static: rng_instance < 2^24 and rng_tag < 16 required");
        return PA_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        pa::set_global_error("pa_resample_static: no usable current CUDA device");
        return PA_ECUDA;
    }
    unsigned char* base;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, pa_static_scratch);
            if (e != cudaSuccess || !p) {
                pa::set_global_error((std::string("pa_resample_static: cudaGetSymbolAddress: ") +
                                      cudaGetErrorString(e)).c_str());
                return PA_ECUDA;
            }
            g_addr[dev] = static_cast<unsigned char*>(p);
        }
        base = g_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    static_prep_kernel<<<1, 1024, 0, st>>>(d_E, R, base);
    pa::ResampleArgs ra{};
    ra.R = R;
    ra.Rn = R;
    ra.kind = 0;
    ra.E32 = d_E;
    ra.E128 = nullptr;
    ra.prev = reinterpret_cast<const pa::StepAcc*>(base + kOffAcc);
    ra.cur = reinterpret_cast<pa::StepAcc*>(base + kOffAcc) + 1;
    ra.w = reinterpret_cast<double*>(base + kOffW);
    ra.P = reinterpret_cast<double*>(base + kOffP);
    ra.lev1 = reinterpret_cast<double*>(base + kOffLev1);
    ra.bmax = reinterpret_cast<double*>(base + kOffBmax);
    ra.upper = reinterpret_cast<double*>(base + kOffUpper);
    ra.counts = reinterpret_cast<int32_t*>(base + kOffCounts);
    ra.blocksum = reinterpret_cast<int32_t*>(base + kOffBlock);
    ra.parent = d_parent;
    ra.fam_in = reinterpret_cast<const int32_t*>(base + kOffFamIn);
    ra.fam_out = reinterpret_cast<int32_t*>(base + kOffFamOut);
    ra.dbeta = beta_next - beta_prev;
    ra.log_R = std::log((double)R);
    ra.betaF0 = 0.0;
    ra.k = k;
    ra.key0 = (uint32_t)seed;
    ra.key1 = (uint32_t)(seed >> 32);
    ra.c3 = pa::counter3(pa::STREAM_RES, rng_tag, rng_instance);
    e = pa::launch_resample(ra, st);
    if (e == cudaSuccess) {
        static_lnq_kernel<<<1, 1, 0, st>>>(base, d_lnQ);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        pa::set_global_error((std::string("pa_resample_static: ") + cudaGetErrorString(e)).c_str());
        return PA_ECUDA;
    }
    return PA_OK;
}
