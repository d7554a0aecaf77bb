// pa_gather_grad.cu -- the replica gather as its own launch, and the
// gradient counts of +-J populations.
//
// Gather (Sec. II.B resampling): slot j of the new population takes the
// spins of replica parent[j].  By default the gather is fused into the
// sweep's tile load; with pa_options.separate_gather it runs here first and
// the sweeps then work in place on the gathered buffer (same results).
//   packed words: lane j of group g takes bit (parent & 63) of the word of
//   group parent >> 6; parents are non-decreasing, so the 64 sources of a
//   word sit in one to a few neighbouring groups; one warp builds 32 words
//   (32 sites of one group) with two ballots per site.
//   int8 rows: 16-byte copies of row parent[j].
//
// Gradient counts (from Eq. 1 with Z = sum exp(-beta H)): after the sweeps
// at beta_k, c_b = sum_r S_i S_{i+e_d} and m_i = sum_r S_i over the
// population.  Packed words (bit set = spin -1): c_b = n - 2 popc(w_i ^ w_j),
// m_i = n - 2 popc(w_i) over the n valid lanes; int8 rows: direct sums.
// Each block adds the partial sums of its share of replicas atomically.
#include "pa_internal.h"

namespace pa {

__global__ void gather_packed_kernel(const uint64_t* __restrict__ Sin, uint64_t* __restrict__ Sout,
                                     const int32_t* __restrict__ parent, int N, int G, int R,
                                     const int* Rdev)
{
    const int lane = threadIdx.x & 31;
    const int nch = (N + 31) / 32;
    const int tup = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);  // (group, 32-site chunk)
    const int Rn = Rdev ? *Rdev : R;
    const int Gn = Rdev ? (Rn + 63) >> 6 : G;
    if (tup >= Gn * nch) return;  // warp-uniform
    const int g = tup / nch, base = (tup - g * nch) * 32;
    const int r0 = 64 * g + lane, r1 = r0 + 32;
    const int s0 = r0 < Rn ? parent[r0] : r0;  // padding lanes keep their own bits
    const int s1 = r1 < Rn ? parent[r1] : r1;
    const uint64_t* p0 = Sin + (size_t)(s0 >> 6) * N + base;
    const uint64_t* p1 = Sin + (size_t)(s1 >> 6) * N + base;
    const int sb0 = s0 & 63, sb1 = s1 & 63;
    const int cnt = min(32, N - base);
    uint64_t mine = 0;
    for (int t = 0; t < cnt; ++t) {
        const uint32_t lo = __ballot_sync(0xffffffffu, (uint32_t)(__ldg(p0 + t) >> sb0) & 1u);
        const uint32_t hi = __ballot_sync(0xffffffffu, (uint32_t)(__ldg(p1 + t) >> sb1) & 1u);
        if (lane == t) mine = (uint64_t)lo | ((uint64_t)hi << 32);
    }
    if (lane < cnt) Sout[(size_t)g * N + base + lane] = mine;
}

__global__ void gather_rows_kernel(const int8_t* __restrict__ Sin, int8_t* __restrict__ Sout,
                                   const int32_t* __restrict__ parent, int NP, int R, const int* Rdev)
{
    const int nv = NP / 16;  // 16-byte vectors per row
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int Rn = Rdev ? *Rdev : R;
    if (t >= (long long)Rn * nv) return;
    const int j = (int)(t / nv), v = (int)(t - (long long)j * nv);
    const uint4 x = reinterpret_cast<const uint4*>(Sin + (size_t)parent[j] * NP)[v];
    reinterpret_cast<uint4*>(Sout + (size_t)j * NP)[v] = x;
}

cudaError_t launch_gather(const uint64_t* Sin, uint64_t* Sout, const int8_t* S8in, int8_t* S8out,
                          const int32_t* parent, int N, int NP, int R, const int* Rdev, cudaStream_t st)
{
    if (Sin) {
        const int G = (R + 63) / 64, nch = (N + 31) / 32;
        const long long warps = (long long)G * nch;
        gather_packed_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(Sin, Sout, parent, N, G, R, Rdev);
    } else {
        const long long n = (long long)R * (NP / 16);
        gather_rows_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(S8in, S8out, parent, NP, R, Rdev);
    }
    return cudaGetLastError();
}

// neighbour i + e_d of site i (periodic), d = 0, 1, 2 -> x, y, z
__device__ __forceinline__ int nb_plus(int i, int d, int L)
{
    const int x = i % L, y = (i / L) % L;
    if (d == 0) return i - x + (x == L - 1 ? 0 : x + 1);
    if (d == 1) return i + (y == L - 1 ? -(L - 1) * L : L);
    const int z = i / (L * L);
    return i + (z == L - 1 ? -(L - 1) * L * L : L * L);
}

// blockIdx.y: a share of the replica groups; one thread per site
__global__ void grad_counts_packed_kernel(const uint64_t* __restrict__ S, int D, int L, int N, int R,
                                          const int* Rdev, unsigned long long* cJ, unsigned long long* ch)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int Rn = Rdev ? *Rdev : R;
    const int G = (Rn + 63) >> 6;
    const int ns = gridDim.y, sp = blockIdx.y;
    const int g0 = (int)((long long)G * sp / ns), g1 = (int)((long long)G * (sp + 1) / ns);
    if (g0 >= g1) return;
    int nb[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) nb[d] = nb_plus(i, d, L);
    long long n = 0, neg = 0, diff[3] = {0, 0, 0};
    for (int g = g0; g < g1; ++g) {
        const int left = Rn - 64 * g;
        const uint64_t mask = left >= 64 ? ~0ull : ((1ull << left) - 1ull);
        const uint64_t* row = S + (size_t)g * N;
        const uint64_t w = row[i] & mask;
        n += __popcll(mask);
        neg += __popcll(w);
        for (int d = 0; d < D; ++d) diff[d] += __popcll((w ^ row[nb[d]]) & mask);
    }
    atomicAdd(&ch[i], (unsigned long long)(n - 2 * neg));
    for (int d = 0; d < D; ++d) atomicAdd(&cJ[(size_t)d * N + i], (unsigned long long)(n - 2 * diff[d]));
}

__global__ void grad_counts_i8_kernel(const int8_t* __restrict__ S8, int NP, int D, int L, int N, int R,
                                      const int* Rdev, unsigned long long* cJ, unsigned long long* ch)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int Rn = Rdev ? *Rdev : R;
    const int ns = gridDim.y, sp = blockIdx.y;
    const int r0 = (int)((long long)Rn * sp / ns), r1 = (int)((long long)Rn * (sp + 1) / ns);
    if (r0 >= r1) return;
    int nb[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) nb[d] = nb_plus(i, d, L);
    long long m = 0, c[3] = {0, 0, 0};
    for (int r = r0; r < r1; ++r) {
        const int8_t* row = S8 + (size_t)r * NP;
        const int s = row[i];
        m += s;
        for (int d = 0; d < D; ++d) c[d] += s * row[nb[d]];
    }
    atomicAdd(&ch[i], (unsigned long long)m);
    for (int d = 0; d < D; ++d) atomicAdd(&cJ[(size_t)d * N + i], (unsigned long long)c[d]);
}

cudaError_t launch_grad_counts_pm(const uint64_t* S, const int8_t* S8, int NP, int D, int L, int R,
                                  const int* Rdev, unsigned long long* cJ, unsigned long long* ch,
                                  cudaStream_t st)
{
    const int N = D == 3 ? L * L * L : L * L;
    const int bx = (N + 127) / 128;
    // enough blocks for the GPU, each share at least a few hundred replicas
    int ns = (R + 1023) / 1024;
    if (ns > 64) ns = 64;
    if (ns < 1) ns = 1;
    if (S)
        grad_counts_packed_kernel<<<dim3(bx, ns), 128, 0, st>>>(S, D, L, N, R, Rdev, cJ, ch);
    else
        grad_counts_i8_kernel<<<dim3(bx, ns), 128, 0, st>>>(S8, NP, D, L, N, R, Rdev, cJ, ch);
    return cudaGetLastError();
}

}  // namespace pa
