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
#include "pa_packed_sweep.cuh"

namespace pa {

// ---------------- shapes and dispatch ----------------

#define PA_PACKED_CASES(X) \
    X(3, 2) X(3, 4) X(3, 6) X(3, 8) X(3, 10) X(3, 12) X(3, 14) X(3, 16) \
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
    bool handled = false;
    cudaError_t e = launch_sweep_packed_part0(D, L, a, gpb, threads, st, &handled);
    if (!handled) e = launch_sweep_packed_part1(D, L, a, gpb, threads, st, &handled);
    if (!handled) e = launch_sweep_packed_part2(D, L, a, gpb, threads, st, &handled);
    if (!handled) e = launch_sweep_packed_part3(D, L, a, gpb, threads, st, &handled);
    return handled ? e : cudaErrorInvalidValue;
}

// ---------------- init, gather, unpack, overlap ----------------

// Sec. II.B: replicas start at random (beta = 0).  INIT stream word per (group, site).
__global__ void init_packed_kernel(uint64_t* S, int N, int G, uint32_t k0, uint32_t k1, uint32_t c3, int goff)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)N * G) return;
    int g = (int)(t / N), i = (int)(t - (size_t)g * N);
    u32x4 o = philox((uint32_t)i, (uint32_t)(g + goff), 0u, c3, k0, k1);
    S[t] = (uint64_t)o.x | ((uint64_t)o.y << 32);
}

cudaError_t launch_init_packed(uint64_t* S, int N, int G, uint32_t k0, uint32_t k1, uint32_t c3,
                               cudaStream_t st, int goff)
{
    size_t n = (size_t)N * G;
    init_packed_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(S, N, G, k0, k1, c3, goff);
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
