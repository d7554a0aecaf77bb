// pa_icm.cu -- isoenergetic cluster moves (Sec. II.C) between random pairs.
//
// Round t of step k pairs replicas pi_t(2i) and pi_t(2i+1), i < floor(R/2);
// pi_t is a 4-round Feistel permutation of [0, 2^m) (m even, the smallest
// with 2^m >= R, at least 2) walked in cycles back into [0, R): halves of m/2
// bits, (Lh, Rh) -> (Rh, Lh ^ F_j(Rh)), F_j(v) = out0 of Philox at counter
// (v, k, 4t + j) of the ICM stream.  For a pair, the overlap q_i = S^a_i S^b_i
// splits the lattice into islands; the sector (q = -1 or +1) with fewer
// sites is used (ties: -1), its idx-th site in site order is drawn with
// idx = floor(r32 n_sector / 2^32), r32 = out0 at counter (i, k, 16 + t), and
// the spins of that site's island are flipped in both replicas.  With a zero
// field E_a + E_b is unchanged, so the move is always accepted.
//
// One block per pair (pairs of a round are disjoint replicas).  The island
// is found by a lock-free union-find in shared memory: roots always link to
// the smaller index, so every parent chain decreases and every loop ends;
// each loop also has an iteration bound that sets an error flag.
#include "pa_device.cuh"
#include "pa_internal.h"

namespace pa {

constexpr int kIcmThreads = 256;
constexpr int kIcmMaxN = 4096;

__device__ __forceinline__ uint32_t icm_feistel(uint32_t x, int h, int k, int t, uint32_t k0, uint32_t k1,
                                                uint32_t c3)
{
    const uint32_t mask = (1u << h) - 1u;  // h <= 16
    uint32_t Lh = (x >> h) & mask, Rh = x & mask;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const u32x4 o = philox(Rh, (uint32_t)k, (uint32_t)(4 * t + j), c3, k0, k1);
        const uint32_t nr = Lh ^ (o.x & mask);
        Lh = Rh;
        Rh = nr;
    }
    return (Lh << h) | Rh;
}

__device__ uint32_t icm_perm(uint32_t i, uint32_t n, int k, int t, uint32_t k0, uint32_t k1, uint32_t c3)
{
    int m = 2;
    while (m < 32 && (1ull << m) < (unsigned long long)n) m += 2;
    uint32_t y = icm_feistel(i, m / 2, k, t, k0, k1, c3);
    // cycle walking: the permutation of [0, 2^m) restricted to [0, n); each
    // step leaves [0, n) with probability below 3/4, and n <= 2^26 bounds the walk
    for (int guard = 0; y >= n && guard < (1 << 26); ++guard) y = icm_feistel(y, m / 2, k, t, k0, k1, c3);
    return y;
}

__device__ __forceinline__ int uf_find(volatile int* par, int x, int N, int* bad)
{
    for (int guard = 0; guard <= N; ++guard) {
        const int p = par[x];
        if (p == x) return x;
        const int gp = par[p];
        if (gp != p) par[x] = gp;  // path halving: an ancestor, never a root entry
        x = gp;
    }
    *bad = 1;
    return x;
}

__device__ __forceinline__ void uf_union(int* par, int x, int y, int N, int* bad)
{
    volatile int* vp = par;
    for (int guard = 0; guard <= 4 * N + 8; ++guard) {
        x = uf_find(vp, x, N, bad);
        y = uf_find(vp, y, N, bad);
        if (x == y) return;
        if (x > y) { const int tmp = x; x = y; y = tmp; }
        if (atomicCAS(&par[y], y, x) == y) return;  // y was a root: linked under x
    }
    *bad = 1;
}

__device__ __forceinline__ int spin_neg(const IcmArgs& a, int r, int j)
{
    if (a.S8) return a.S8[(size_t)r * a.NP + j] < 0;
    return (int)((a.S[(size_t)(r >> 6) * a.N + j] >> (r & 63)) & 1ull);
}

// +e_d neighbour of site j (x fastest, periodic)
__device__ __forceinline__ int nb_plus(int j, int d, int L)
{
    int stride = 1;
    for (int e = 0; e < d; ++e) stride *= L;
    const int c = (j / stride) % L;
    return c == L - 1 ? j - (L - 1) * stride : j + stride;
}

__global__ void __launch_bounds__(kIcmThreads) icm_kernel(IcmArgs a)
{
    __shared__ uint8_t qneg[kIcmMaxN];
    __shared__ int par[kIcmMaxN];
    __shared__ int s_cnt[kIcmThreads];
    __shared__ int s_pair[4];  // a, b, chosen site, root
    __shared__ uint32_t s_r32;
    __shared__ int s_nneg, s_bad;
    const int N = a.N, tid = threadIdx.x;
    const int R = a.Rdev ? *a.Rdev : a.R;
    const int npairs = R / 2;
    // contiguous chunk of sites per thread (site order for the idx-th sector site)
    const int per = (N + kIcmThreads - 1) / kIcmThreads;
    const int j0 = min(N, tid * per), j1 = min(N, j0 + per);
    if (tid == 0) s_bad = 0;
    for (int i = blockIdx.x; i < npairs; i += gridDim.x) {
        if (tid == 0) {
            s_pair[0] = (int)icm_perm((uint32_t)(2 * i), (uint32_t)R, a.k, a.t, a.key0, a.key1, a.c3);
            s_pair[1] = (int)icm_perm((uint32_t)(2 * i + 1), (uint32_t)R, a.k, a.t, a.key0, a.key1, a.c3);
            s_r32 = philox((uint32_t)i, (uint32_t)a.k, (uint32_t)(16 + a.t), a.c3, a.key0, a.key1).x;
            s_nneg = 0;
        }
        __syncthreads();
        const int ra = s_pair[0], rb = s_pair[1];
        int cnt = 0;
        for (int j = j0; j < j1; ++j) {
            const uint8_t v = (uint8_t)(spin_neg(a, ra, j) ^ spin_neg(a, rb, j));
            qneg[j] = v;
            cnt += v;
        }
        atomicAdd(&s_nneg, cnt);
        __syncthreads();
        const int nneg = s_nneg;
        const uint8_t want = nneg <= N - nneg ? 1 : 0;  // the sector with fewer sites (ties: q = -1)
        const int nsec = want ? nneg : N - nneg;
        if (nsec > 0) {  // block-uniform
            // sector sites of this thread's chunk, then an exclusive scan over threads
            int c = 0;
            for (int j = j0; j < j1; ++j) c += (qneg[j] == want);
            s_cnt[tid] = c;
            for (int j = j0; j < j1; ++j) par[j] = (qneg[j] == want) ? j : -1;
            __syncthreads();
            if (tid == 0) {
                const uint32_t idx = (uint32_t)(((uint64_t)s_r32 * (uint64_t)nsec) >> 32);
                int acc = 0, th = 0;
                while (th < kIcmThreads - 1 && acc + s_cnt[th] <= (int)idx) acc += s_cnt[th++];
                const int t0 = min(N, th * per), t1 = min(N, t0 + per);
                int site = -1;
                for (int j = t0; j < t1 && site < 0; ++j)
                    if (qneg[j] == want) {
                        if (acc == (int)idx) site = j;
                        ++acc;
                    }
                s_pair[2] = site;
            }
            // islands: union along +e_d bonds inside the sector
            for (int j = j0; j < j1; ++j) {
                if (qneg[j] != want) continue;
                for (int d = 0; d < a.D; ++d) {
                    const int nb = nb_plus(j, d, a.L);
                    if (qneg[nb] == want) uf_union(par, j, nb, N, &s_bad);
                }
            }
            __syncthreads();
            if (tid == 0) s_pair[3] = s_pair[2] >= 0 ? uf_find(par, s_pair[2], N, &s_bad) : -1;
            __syncthreads();
            const int root = s_pair[3];
            if (root >= 0) {
                for (int j = j0; j < j1; ++j) {
                    if (qneg[j] != want || uf_find(par, j, N, &s_bad) != root) continue;
                    if (a.S8) {
                        int8_t* pa_ = a.S8 + (size_t)ra * a.NP + j;
                        int8_t* pb_ = a.S8 + (size_t)rb * a.NP + j;
                        *pa_ = (int8_t)-*pa_;
                        *pb_ = (int8_t)-*pb_;
                    } else if ((ra >> 6) == (rb >> 6)) {
                        atomicXor((unsigned long long*)&a.S[(size_t)(ra >> 6) * N + j],
                                  (1ull << (ra & 63)) | (1ull << (rb & 63)));
                    } else {
                        atomicXor((unsigned long long*)&a.S[(size_t)(ra >> 6) * N + j], 1ull << (ra & 63));
                        atomicXor((unsigned long long*)&a.S[(size_t)(rb >> 6) * N + j], 1ull << (rb & 63));
                    }
                }
            }
        }
        __syncthreads();  // shared arrays are reused by the next pair
    }
    if (tid == 0 && s_bad) atomicExch(a.err, 1);
}

cudaError_t launch_icm(const IcmArgs& a, cudaStream_t st)
{
    if (a.N > kIcmMaxN) return cudaErrorInvalidValue;
    const int npairs_max = a.R / 2;
    if (npairs_max == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::min(npairs_max, sms * 8);
    icm_kernel<<<grid, kIcmThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace pa
