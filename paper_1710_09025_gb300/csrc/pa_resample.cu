// pa_resample.cu -- resampling, observables and the gradient backward pass.
//
// Resampling (Sec. II.B): when beta rises to beta', replica i gets on average
// R w_i / S copies, w_i = exp[-(beta'-beta)(E_i - E_min)], S = sum_i w_i
// (multinomial: R independent draws).  Free-energy perturbation: ln Q =
// -(beta'-beta) E_min + ln S - ln R and beta F_k = -N ln 2 - sum_{l<=k} ln Q_l.
//
// Fixed order, so that the draws do not depend on the launch geometry:
// runs of 32 weights are summed left to right; the run totals are summed the
// same way, recursively, until one run is left; entry j of run c is
// Q_{c-1} + l_j (l_j its sum inside the run, Q the inclusive prefix of the
// run totals; run 0: l_j alone).  P_i is the running maximum of those sums
// (exact; it only repairs the one-unit steps that two summation orders can
// leave at a run boundary) and S = P_{R-1}.  Draw q (RES stream) picks the
// smallest i with u_q S < P_i (if u_q S == S after rounding: the smallest i
// with P_i >= u_q S).  Copy numbers are exact integer counts; their exclusive
// scan places the copies of replica i in slots [C_i, C_i + n_i), so families
// stay contiguous (Sec. V.A).
#include "pa_device.cuh"
#include "pa_internal.h"

namespace pa {

__device__ __forceinline__ __int128 ll2_to_i128(longlong2 v)
{
    return ((__int128)v.y << 64) | (unsigned long long)v.x;
}

__device__ __forceinline__ double e_minus_min_to_double(const ResampleArgs& a, int i)
{
    if (a.kind == 0) return (double)(a.E32[i] - (int)a.prev->emin_lo);  // exact integer
    __int128 emin = ((__int128)a.prev->emin_hi << 64) | (unsigned long long)a.prev->emin_lo;
    return __dmul_rn(i128_to_double(ll2_to_i128(a.E128[i]) - emin), 0x1p-96);
}

// true in the block that finishes last (every block calls it once); the
// counter is reset for the next launch.  Writes before the call are visible
// to the last block (fence before the count).
__device__ __forceinline__ bool last_block(int* counter)
{
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const int done = atomicAdd(counter, 1);
        s_last = done == (int)(gridDim.x * gridDim.y) - 1;
        if (s_last) *counter = 0;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

// source population: in device memory for the nearest-integer scheme
__device__ __forceinline__ int rs_src(const ResampleArgs& a) { return a.Rsrc ? *a.Rsrc : a.R; }

// Weights and the two lowest levels of the prefix, one block of kWThreads
// threads per kWBlock weights (small blocks, so that several blocks' FP64
// chains overlap on an SM).  GB300 has little FP64 throughput, so every
// addition of the specified order is executed once: lane c of warp 0 sums
// run c (32 weights, staged in shared memory, loaded eight at a time) left
// to right, then lane 0 sums the block's run totals left to right.
constexpr int kWThreads = 256;
__device__ __forceinline__ void rs_weights_body(const ResampleArgs& a, int b)
{
    __shared__ double s_w[kFan * (kFan + 1)];  // run c at [c (kFan + 1)], padded against bank conflicts
    __shared__ double s_t[kFan];
    const int R = rs_src(a);
    const int i0 = b * kWBlock;
    if (i0 >= R) return;  // block-uniform: past the source population
    const int tid = threadIdx.x;
    const int n = min(kWBlock, R - i0);
    for (int t = tid; t < n; t += kWThreads) {
        const int i = i0 + t;
        double w;
        const int lv = a.kind == 0 ? a.E32[i] - (int)a.prev->emin_lo : 0;
        if (a.wtab && (lv & 3) == 0 && (lv >> 2) < a.wtab_n) {
            w = a.wtab[lv >> 2];  // +-J: E - E_min is a multiple of 4, the weight a table entry
        } else {
            const double d = e_minus_min_to_double(a, i);
            w = spec_exp64(-__dmul_rn(a.dbeta, d));
        }
        a.w[i] = w;
        s_w[(t / kFan) * (kFan + 1) + t % kFan] = w;
    }
    __syncthreads();
    const int nruns = (n + kFan - 1) / kFan;
    if (tid < nruns) {  // run tid, left to right
        double* x = s_w + tid * (kFan + 1);
        const int cnt = min(kFan, n - tid * kFan);
        double acc = 0.0;
        for (int j0 = 0; j0 < cnt; j0 += 8) {
            double v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = j0 + j < cnt ? x[j0 + j] : 0.0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (j0 + j < cnt) {
                    acc = (j0 + j == 0) ? v[0] : __dadd_rn(acc, v[j]);
                    x[j0 + j] = acc;
                }
            }
        }
        s_t[tid] = acc;
    }
    __syncthreads();
    for (int t = tid; t < n; t += kWThreads) a.P[i0 + t] = s_w[(t / kFan) * (kFan + 1) + t % kFan];
    if (tid == 0) {  // the block's run totals, left to right
        double acc = s_t[0];
        a.lev1[b * kFan] = acc;
        for (int c = 1; c < nruns; ++c) {
            acc = __dadd_rn(acc, s_t[c]);
            a.lev1[b * kFan + c] = acc;
        }
        a.upper[b] = acc;
    }
}
__device__ __forceinline__ void rs_top_body(const ResampleArgs& a);
__global__ void __launch_bounds__(kWThreads) rs_weights_kernel(ResampleArgs a)
{
    rs_weights_body(a, blockIdx.x);
    if (a.sync && last_block(a.sync)) rs_top_body(a);  // levels >= 2 of the prefix
}
__global__ void __launch_bounds__(kWThreads) rs_weights_batched(const ResampleArgs* tab)
{
    const ResampleArgs& a = tab[blockIdx.y];
    rs_weights_body(a, blockIdx.x);
}

// +-J: all energies are congruent modulo 4 (Delta E of a flip is 4D - 4n),
// so E - E_min takes the values 4l, l < wtab_n; the weight of level l,
// spec_exp64(-(dbeta * 4l)), is the same arithmetic as for a replica
__global__ void rs_table_kernel(ResampleArgs a)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < a.wtab_n) const_cast<double*>(a.wtab)[l] = spec_exp64(-__dmul_rn(a.dbeta, (double)(4 * l)));
}

// Levels >= 2 of the prefix, by one block of kWBlock threads after every
// weights block is done: bottom-up sums inside runs of the block totals (each
// thread loads its run, then adds in order), then top-down Q_{c-1} + l_j.
__device__ __forceinline__ void rs_top_body(const ResampleArgs& a)
{
    constexpr int kMaxLev = 8;  // kFan^(kMaxLev+1) > 2^31 weights
    const int tid = threadIdx.x, nt = blockDim.x;
    const int R = a.gR ? a.gR : rs_src(a);  // a shard sums the global block totals
    int base[kMaxLev], len[kMaxLev], nl = 0;
    int n = rs_wblocks(R), off = 0;
    for (;;) {
        base[nl] = off; len[nl] = n; ++nl;
        const int nc = n <= kFan ? 1 : (n + kFan - 1) / kFan;
        for (int c = tid; c < nc; c += nt) {
            double* x = a.upper + off + c * kFan;
            const int cnt = min(kFan, n - c * kFan);
            double acc = 0.0;
            for (int j0 = 0; j0 < cnt; j0 += 8) {  // eight independent loads, then the additions
                double v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = j0 + j < cnt ? x[j0 + j] : 0.0;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    acc = (j0 + j == 0) ? v[0] : __dadd_rn(acc, v[j]);  // +0 past the run: no change
                    v[j] = acc;
                }
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (j0 + j < cnt) x[j0 + j] = v[j];
            }
            if (n > kFan) a.upper[off + n + c] = acc;
        }
        __syncthreads();
        if (n <= kFan) break;  // one run left: its sums are the prefix of this level
        off += n;
        n = nc;
    }
    for (int v = nl - 2; v >= 0; --v) {
        double* x = a.upper + base[v];
        const double* q = a.upper + base[v + 1];
        for (int j = kFan + tid; j < len[v]; j += nt) x[j] = __dadd_rn(q[j / kFan - 1], x[j]);
        __syncthreads();
    }
}
__global__ void __launch_bounds__(kWBlock) rs_top_kernel(ResampleArgs a) { rs_top_body(a); }
// one block per instance
__global__ void __launch_bounds__(kWBlock) rs_top_batched(const ResampleArgs* tab, int n_inst)
{
    if ((int)blockIdx.x < n_inst) rs_top_body(tab[blockIdx.x]);
}

// Non-negative doubles compare as their bit patterns do (as signed 64-bit
// integers): maxima and the draw search use the integer compare, which is
// exact and leaves GB300's scarce FP64 units to the specified additions.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

// Level 0 and the running maximum inside one weights block: weight i of run
// c gets Q1_{c-1} + l_i (Q1_{c-1} = Q2_{b'-1} + l1_{c-1} with b' the block of
// run c - 1, the level-1 sums alone in block 0), then P_i = the largest of
// these up to i within the block; bmax[b] = the block's largest.
__device__ __forceinline__ void rs_finalize_body(const ResampleArgs& a, int b)
{
    constexpr int PER = kWBlock / kWThreads;  // consecutive weights per thread
    __shared__ double s_q[kFan];
    __shared__ long long s_m[kWThreads / 32];
    const int R = rs_src(a);
    const int i0 = b * kWBlock;
    if (i0 >= R) return;  // block-uniform
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cg0 = a.gb0 * kFan;  // global index of local run 0 (0 unless a shard)
    if (tid < kFan) {  // Q1 of the run before run c = b kFan + tid (one addition per run)
        const int c = b * kFan + tid;
        double q = 0.0;
        if (cg0 + c > 0 && c * kFan < R) {
            const int cb = (cg0 + c - 1) / kFan;  // global block of run c - 1
            // l1 of run c - 1; before a shard's first run it is the last run of
            // the previous (remote) block, whose l1 is that block's total
            const double l1 = c > 0 ? a.lev1[c - 1] : a.t2g[cb];
            q = cb == 0 ? l1 : __dadd_rn(a.upper[cb - 1], l1);
        }
        s_q[tid] = q;
    }
    __syncthreads();
    long long v[PER];
    long long m = 0;  // bits of +0.0: weights are >= 0
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int i = i0 + tid * PER + j;
        long long x = 0;
        if (i < R) {
            const double l = a.P[i];
            x = dbits(cg0 == 0 && i < kFan ? l : __dadd_rn(s_q[(tid * PER + j) / kFan], l));
        }
        m = max(m, x);
        v[j] = m;  // inclusive maximum within this thread's weights
    }
    long long incl = m;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl = max(incl, u);
    }
    if (lane == 31) s_m[warp] = incl;
    const long long up = __shfl_up_sync(0xffffffffu, incl, 1);
    __syncthreads();
    long long before = lane > 0 ? up : 0;
    for (int w = 0; w < warp; ++w) before = max(before, s_m[w]);
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int i = i0 + tid * PER + j;
        if (i < R) a.P[i] = __longlong_as_double(max(before, v[j]));
    }
    if (tid == 0) {
        long long bm = 0;
        for (int w = 0; w < kWThreads / 32; ++w) bm = max(bm, s_m[w]);
        a.bmax[b] = __longlong_as_double(bm);
    }
}
// running maximum over the weights blocks (bmax[nb + b] = the largest
// cumulative weight before block b), S = the largest cumulative weight, ln Q
// and the running free energy; one block, as many block maxima per pass as it
// has threads (integer maxima of the bit patterns)
__device__ __forceinline__ void rs_blockmax_body(const ResampleArgs& a)
{
    __shared__ long long s_w[32];
    __shared__ long long s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int R = a.gR ? a.gR : rs_src(a);  // a shard: the global block maxima
    const int nb = rs_wblocks(R);
    if (tid == 0) s_carry = 0;
    __syncthreads();
    const int nt = blockDim.x;
    for (int b0 = 0; b0 < nb; b0 += nt) {
        const int b = b0 + tid;
        long long m = b < nb ? dbits(a.bmax[b]) : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, m, o);
            if (lane >= o) m = max(m, u);
        }
        if (lane == 31) s_w[warp] = m;
        const long long carry = s_carry;
        __syncthreads();
        long long before = carry;
        for (int w = 0; w < warp; ++w) before = max(before, s_w[w]);
        const long long up = __shfl_up_sync(0xffffffffu, m, 1);
        const long long excl = lane > 0 ? max(before, up) : before;
        if (b < nb) a.bmax[nb + b] = __longlong_as_double(excl);
        if (tid == nt - 1) s_carry = max(before, m);
        __syncthreads();
    }
    if (tid != 0) return;
    const double S = __longlong_as_double(s_carry);
    double emin_d;
    if (a.kind == 0) {
        emin_d = (double)(int)a.prev->emin_lo;
    } else {
        __int128 emin = ((__int128)a.prev->emin_hi << 64) | (unsigned long long)a.prev->emin_lo;
        emin_d = __dmul_rn(i128_to_double(emin), 0x1p-96);
    }
    const double log_R = a.Rsrc ? log((double)R) : a.log_R;
    const double lnQ = __dsub_rn(__dadd_rn(-__dmul_rn(a.dbeta, emin_d), log(S)), log_R);
    const double sum = __dadd_rn(a.prev->sum_lnQ, lnQ);
    a.cur->lnQ = lnQ;
    a.cur->sum_lnQ = sum;
    a.cur->betaF = __dsub_rn(a.betaF0, sum);
    a.cur->S = S;
}
__global__ void __launch_bounds__(kWThreads) rs_finalize_kernel(ResampleArgs a)
{
    rs_finalize_body(a, blockIdx.x);
    if (a.sync && last_block(a.sync + 3)) rs_blockmax_body(a);
}
__global__ void __launch_bounds__(kWThreads) rs_finalize_batched(const ResampleArgs* tab)
{
    rs_finalize_body(tab[blockIdx.y], blockIdx.x);
}
__global__ void __launch_bounds__(kWBlock) rs_blockmax_kernel(ResampleArgs a) { rs_blockmax_body(a); }
// one block per instance
__global__ void __launch_bounds__(kWBlock) rs_blockmax_batched(const ResampleArgs* tab, int n_inst)
{
    if ((int)blockIdx.x < n_inst) rs_blockmax_body(tab[blockIdx.x]);
}

// Multinomial draws.  P is non-decreasing, so the smallest i with x < P_i
// lies in the first segment (of s consecutive weights, whole weights blocks)
// whose last P exceeds x: each block stages the segment ends in shared memory,
// finds the segment there and bisects only inside it in global memory.  P_i
// is the stored block-local value raised to the largest value before its
// weights block.
constexpr int kDrawThreads = 512;
constexpr int kMaxSeg = 2048;
__device__ __forceinline__ int rs_seg_blocks(int nb)
{
    int s = 1;
    while ((nb + s - 1) / s > kMaxSeg) s *= 2;
    return s;
}
__device__ __forceinline__ long long rs_P(const ResampleArgs& a, int nb, int i)
{
    return max(dbits(a.bmax[nb + i / kWBlock]), dbits(a.P[i]));
}
__device__ __forceinline__ void rs_draws_body(const ResampleArgs& a, int q)
{
    __shared__ long long s_end[kMaxSeg];
    const int R = a.R;
    const int nb = rs_wblocks(R);
    const int sb = rs_seg_blocks(nb), seg = sb * kWBlock, nseg = (nb + sb - 1) / sb;
    const double S = a.cur->S;
    for (int k = threadIdx.x; k < nseg; k += blockDim.x) {
        const int lb = min(nb - 1, k * sb + sb - 1);  // last weights block of segment k
        // its largest P: the largest before the next block, or S for the last block
        s_end[k] = lb + 1 < nb ? dbits(a.bmax[nb + lb + 1]) : dbits(S);
    }
    __syncthreads();
    if (q >= a.Rn) return;
    const u32x4 o = philox((uint32_t)q, (uint32_t)a.k, 0u, a.c3, a.key0, a.key1);
    const long long x = dbits(__dmul_rn(uniform53(o.x, o.y), S));  // x >= 0
    int lo = 0, hi = nseg;  // first segment whose end exceeds x
    while (lo < hi) {
        const int mid = lo + ((hi - lo) >> 1);
        if (x < s_end[mid]) hi = mid; else lo = mid + 1;
    }
    if (lo < nseg) {
        const int k = lo;
        lo = k * seg;
        hi = min(R - 1, k * seg + seg - 1);  // x < P[hi]
        if (sb == 1) {
            // one weights block: x is at least the largest P before it, so
            // x < max(that, stored P_i) reduces to x < stored P_i
            while (lo < hi) {
                const int mid = lo + ((hi - lo) >> 1);
                if (x < dbits(a.P[mid])) hi = mid; else lo = mid + 1;
            }
        } else {
            while (lo < hi) {
                const int mid = lo + ((hi - lo) >> 1);
                if (x < rs_P(a, nb, mid)) hi = mid; else lo = mid + 1;
            }
        }
    } else {
        // x == S after rounding: the smallest i with P_i >= x
        lo = 0; hi = R;
        while (lo < hi) {
            const int mid = lo + ((hi - lo) >> 1);
            if (rs_P(a, nb, mid) >= x) hi = mid; else lo = mid + 1;
        }
        if (lo >= R) lo = R - 1;  // unreachable: x = u S <= S = P[R-1]
    }
    atomicAdd(&a.counts[lo], 1);
}
// A shard's draws: all gR global draws are evaluated, a draw's weights block
// is found from the global block ends, and only draws that land on a local
// block are resolved (bisection in the local P) and counted.
__device__ __forceinline__ void rs_draws_shard_body(const ResampleArgs& a, int q)
{
    __shared__ long long s_end[kMaxSeg];
    const int nb = rs_wblocks(a.gR), nloc = rs_wblocks(a.R);
    const int sb = rs_seg_blocks(nb), nseg = (nb + sb - 1) / sb;
    const double S = a.cur->S;
    // largest P up to the end of block b: the largest before block b + 1, or S
    auto block_end = [&](int b) { return b + 1 < nb ? dbits(a.bmax[nb + b + 1]) : dbits(S); };
    for (int k = threadIdx.x; k < nseg; k += blockDim.x) s_end[k] = block_end(min(nb - 1, k * sb + sb - 1));
    __syncthreads();
    if (q >= a.Rn) return;
    const u32x4 o = philox((uint32_t)q, (uint32_t)a.k, 0u, a.c3, a.key0, a.key1);
    const long long x = dbits(__dmul_rn(uniform53(o.x, o.y), S));  // x >= 0
    int lo = 0, hi = nseg;
    while (lo < hi) {
        const int mid = lo + ((hi - lo) >> 1);
        if (x < s_end[mid]) hi = mid; else lo = mid + 1;
    }
    const bool strict = lo < nseg;  // some P exceeds x; else x == S: the first P >= x
    int b0 = strict ? lo * sb : 0, b1 = strict ? min(nb - 1, lo * sb + sb - 1) : nb - 1;
    while (b0 < b1) {  // the first block whose end exceeds x (or reaches x)
        const int mid = b0 + ((b1 - b0) >> 1);
        const long long e = block_end(mid);
        if (strict ? x < e : e >= x) b1 = mid; else b0 = mid + 1;
    }
    const int bl = b0 - a.gb0;
    if (bl < 0 || bl >= nloc) return;  // another shard's draw
    const long long before = dbits(a.bmax[nb + b0]);
    int i = bl * kWBlock, j = min(a.R, i + kWBlock) - 1;
    while (i < j) {
        const int mid = i + ((j - i) >> 1);
        const long long p = max(before, dbits(a.P[mid]));
        if (strict ? x < p : p >= x) j = mid; else i = mid + 1;
    }
    atomicAdd(&a.counts[i], 1);
}
__global__ void __launch_bounds__(kDrawThreads) rs_draws_shard_kernel(ResampleArgs a)
{
    rs_draws_shard_body(a, blockIdx.x * blockDim.x + threadIdx.x);
}
__global__ void __launch_bounds__(kDrawThreads) rs_draws_kernel(ResampleArgs a)
{
    rs_draws_body(a, blockIdx.x * blockDim.x + threadIdx.x);
}
__global__ void __launch_bounds__(kDrawThreads) rs_draws_batched(const ResampleArgs* tab)
{
    const ResampleArgs& a = tab[blockIdx.y];
    if ((int)(blockIdx.x * blockDim.x) >= a.Rn) return;  // block-uniform: no draw of this instance
    rs_draws_body(a, blockIdx.x * blockDim.x + threadIdx.x);
}

// nearest-integer copy numbers (Sec. II.B, population in expectation):
// tau_i = target w_i / S, n_i = floor(tau_i) + [u_i < tau_i - floor(tau_i)],
// u_i from the RESAMPLE stream at counter (i, k, 1)
__device__ __forceinline__ void rs_nearest_body(const ResampleArgs& a, int i)
{
    const int R = rs_src(a);
    if (i >= R) return;
    const double S = a.cur->S;
    const u32x4 o = philox((uint32_t)i, (uint32_t)a.k, 1u, a.c3, a.key0, a.key1);
    const double u = uniform53(o.x, o.y);
    const double tau = __ddiv_rn(__dmul_rn(a.target, a.w[i]), S);
    const double fl = floor(tau);
    a.counts[i] = (int32_t)fl + (u < __dsub_rn(tau, fl) ? 1 : 0);
}
__global__ void rs_nearest_kernel(ResampleArgs a) { rs_nearest_body(a, blockIdx.x * blockDim.x + threadIdx.x); }

__device__ __forceinline__ void rs_blocksum_body(const int32_t* counts, int R, int32_t* blocksum, int b)
{
    __shared__ int ws[32];
    const int tid = threadIdx.x;
    int s = 0;
    for (int t = 0; t < kScanBlock / 1024; ++t) {
        const int i = b * kScanBlock + t * 1024 + tid;
        if (i < R) s += counts[i];
    }
    s = __reduce_add_sync(0xffffffffu, s);
    if ((tid & 31) == 0) ws[tid >> 5] = s;
    __syncthreads();
    if (tid < 32) {
        int v = __reduce_add_sync(0xffffffffu, ws[tid]);
        if (tid == 0) blocksum[b] = v;
    }
}
__device__ __forceinline__ void rs_scan_finish(const ResampleArgs& a);
__global__ void __launch_bounds__(1024) rs_blocksum_kernel(ResampleArgs a)
{
    const int R = rs_src(a);
    if ((int)blockIdx.x * kScanBlock < R) rs_blocksum_body(a.counts, R, a.blocksum, blockIdx.x);
    if (a.sync && last_block(a.sync + 1) && threadIdx.x == 0) rs_scan_finish(a);  // block offsets
}
__global__ void __launch_bounds__(1024) rs_blocksum_batched(const ResampleArgs* tab)
{
    const ResampleArgs& a = tab[blockIdx.y];
    if ((int)blockIdx.x * kScanBlock < a.R) rs_blocksum_body(a.counts, a.R, a.blocksum, blockIdx.x);
}

__device__ __forceinline__ int rs_scan_blocks_body(int32_t* blocksum, int nb)
{
    int acc = 0;
    for (int b = 0; b < nb; ++b) {
        const int v = blocksum[b];
        blocksum[b] = acc;
        acc += v;
    }
    return acc;
}
__device__ __forceinline__ void rs_scan_finish(const ResampleArgs& a)
{
    const int R = rs_src(a);
    const int nbs = (R + kScanBlock - 1) / kScanBlock;
    const int total = rs_scan_blocks_body(a.blocksum, nbs);
    a.blocksum[nbs] = total;  // the copies placed (a shard reads it)
    if (a.Rdst) {  // the drawn population, copies beyond the capacity dropped
        const int Rn = min(total, a.cap);
        *a.Rdst = Rn;
        *a.Rdst_d = (double)Rn;
    }
}
__global__ void rs_scan_blocks_kernel(ResampleArgs a)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) rs_scan_finish(a);
}
__global__ void rs_scan_blocks_batched(const ResampleArgs* tab, int n_inst)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_inst) rs_scan_blocks_body(tab[i].blocksum, (tab[i].R + kScanBlock - 1) / kScanBlock);
}

// exclusive scan inside the block + block offset; write parents and families
__device__ __forceinline__ void rs_fill_body(const ResampleArgs& a, int b)
{
    __shared__ int ws[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int PER = kScanBlock / 1024;
    const int i0 = b * kScanBlock + tid * PER;
    int c[PER];
    int s = 0;
    const int R = rs_src(a);
    const int cap = a.Rdst ? a.cap : 0x7fffffff;
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        c[t] = (i0 + t < R) ? a.counts[i0 + t] : 0;
        s += c[t];
    }
    int incl = s;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int v = ws[lane];
        int inc = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += u;
        }
        ws[lane] = inc - v;  // exclusive warp offsets
    }
    __syncthreads();
    int off = a.blocksum[b] + ws[warp] + (incl - s);
    const int pbase = a.gb0 * kWBlock;  // a shard writes global replica indices
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        const int i = i0 + t;
        if (i < R) {
            const int f = a.fam_in[i];
            const int n = min(c[t], max(cap - off, 0));  // slots past the capacity are dropped
            for (int u = 0; u < n; ++u) {
                a.parent[off + u] = pbase + i;
                a.fam_out[off + u] = f;
            }
            off += c[t];
            a.counts[i] = 0;
        }
    }
}
__global__ void __launch_bounds__(1024) rs_fill_kernel(ResampleArgs a)
{
    if ((int)blockIdx.x * kScanBlock < rs_src(a)) rs_fill_body(a, blockIdx.x);
}
__global__ void __launch_bounds__(1024) rs_fill_batched(const ResampleArgs* tab)
{
    const ResampleArgs& a = tab[blockIdx.y];
    if ((int)blockIdx.x * kScanBlock < a.R) rs_fill_body(a, blockIdx.x);
}

cudaError_t launch_resample(const ResampleArgs& a, cudaStream_t st)
{
    const int nb = (a.R + kScanBlock - 1) / kScanBlock;
    // one level per thread, small blocks spread over the SMs (FP64-bound)
    if (a.wtab) rs_table_kernel<<<(a.wtab_n + 31) / 32, 32, 0, st>>>(a);
    rs_weights_kernel<<<rs_wblocks(a.R), kWThreads, 0, st>>>(a);
    if (!a.sync) rs_top_kernel<<<1, kWBlock, 0, st>>>(a);
    rs_finalize_kernel<<<rs_wblocks(a.R), kWThreads, 0, st>>>(a);
    if (!a.sync) rs_blockmax_kernel<<<1, kWBlock, 0, st>>>(a);
    if (a.scheme == 1)
        rs_nearest_kernel<<<(a.R + 255) / 256, 256, 0, st>>>(a);
    else
        rs_draws_kernel<<<(a.Rn + kDrawThreads - 1) / kDrawThreads, kDrawThreads, 0, st>>>(a);
    rs_blocksum_kernel<<<nb, 1024, 0, st>>>(a);
    if (!a.sync) rs_scan_blocks_kernel<<<1, 32, 0, st>>>(a);
    rs_fill_kernel<<<nb, 1024, 0, st>>>(a);
    return cudaGetLastError();
}

// the phases of a shard's resampling (the host exchanges the block totals,
// the block maxima and the copy totals between them)
cudaError_t launch_resample_shard(const ResampleArgs& a, int phase, cudaStream_t st)
{
    const int nb = (a.R + kScanBlock - 1) / kScanBlock;
    switch (phase) {
    case 0:  // weights, levels 0 and 1 of the local blocks -> local block totals in upper
        if (a.wtab) rs_table_kernel<<<(a.wtab_n + 31) / 32, 32, 0, st>>>(a);
        rs_weights_kernel<<<rs_wblocks(a.R), kWThreads, 0, st>>>(a);
        break;
    case 1:  // global levels >= 2 (upper holds every shard's block totals), local P, block maxima
        rs_top_kernel<<<1, kWBlock, 0, st>>>(a);
        rs_finalize_kernel<<<rs_wblocks(a.R), kWThreads, 0, st>>>(a);
        break;
    case 2:  // running maximum over every shard's blocks, S, ln Q; draws; copy totals
        rs_blockmax_kernel<<<1, kWBlock, 0, st>>>(a);
        rs_draws_shard_kernel<<<(a.Rn + kDrawThreads - 1) / kDrawThreads, kDrawThreads, 0, st>>>(a);
        rs_blocksum_kernel<<<nb, 1024, 0, st>>>(a);
        rs_scan_blocks_kernel<<<1, 32, 0, st>>>(a);
        break;
    default:  // placement: global parent indices and families of the local copies
        rs_fill_kernel<<<nb, 1024, 0, st>>>(a);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_resample_batched(const ResampleArgs* tab, int n_inst, int maxR, cudaStream_t st)
{
    const unsigned nb = (maxR + kScanBlock - 1) / kScanBlock;
    const unsigned ni = (unsigned)n_inst;
    rs_weights_batched<<<dim3(rs_wblocks(maxR), ni), kWThreads, 0, st>>>(tab);
    rs_top_batched<<<ni, kWBlock, 0, st>>>(tab, n_inst);
    rs_finalize_batched<<<dim3(rs_wblocks(maxR), ni), kWThreads, 0, st>>>(tab);
    rs_blockmax_batched<<<ni, kWBlock, 0, st>>>(tab, n_inst);
    rs_draws_batched<<<dim3((maxR + kDrawThreads - 1) / kDrawThreads, ni), kDrawThreads, 0, st>>>(tab);
    rs_blocksum_batched<<<dim3(nb, ni), 1024, 0, st>>>(tab);
    rs_scan_blocks_batched<<<(ni + 63) / 64, 64, 0, st>>>(tab, n_inst);
    rs_fill_batched<<<dim3(nb, ni), 1024, 0, st>>>(tab);
    return cudaGetLastError();
}

// log(c) for c < kLogC (entries 0 and 1 are never read: a run of one adds 0)
__global__ void logc_table_kernel(double* t)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < kLogC) t[c] = c > 0 ? log((double)c) : 0.0;
}
cudaError_t launch_logc_table(double* t, cudaStream_t st)
{
    logc_table_kernel<<<(kLogC + 255) / 256, 256, 0, st>>>(t);
    return cudaGetLastError();
}

// ---------------- observables (Sec. V.A, Eq. 9; Sec. II.B, Eq. 2) ----------------
// kObsBlocks blocks each reduce a contiguous slice of the population in a
// fixed order; one block combines the partials in block order.  The result
// does not depend on the GPU (the partition depends only on R).
__device__ __forceinline__ void observe_partial_body(const ObsArgs& a)
{
    __shared__ long long s_ll[2][32];
    __shared__ double s_d[3][32];
    __shared__ __int128 s_min[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int R = a.Rdev ? *a.Rdev : a.R;
    const int nb = obs_blocks(R);
    if ((int)blockIdx.x >= nb) return;  // block-uniform
    const int per = (R + nb - 1) / nb;
    const int j0 = blockIdx.x * per, j1 = min(R, j0 + per);
    long long se = 0, se2 = 0;
    double sed = 0.0, se2d = 0.0, clnc = 0.0;
    __int128 mn = (__int128)(((unsigned __int128)1 << 127) - 1);
    for (int j = j0 + tid; j < j1; j += 1024) {
        if (a.kind == 0) {
            const long long e = a.E32[j];
            se += e;
            se2 += e * e;
            if ((__int128)e < mn) mn = e;
        } else {
            const longlong2 v = a.E128[j];
            const __int128 e = ((__int128)v.y << 64) | (unsigned long long)v.x;
            const double ed = __dmul_rn(i128_to_double(e), 0x1p-96);
            sed = __dadd_rn(sed, ed);
            se2d = __fma_rn(ed, ed, se2d);
            if (e < mn) mn = e;
        }
        const int f = a.family[j];
        if (j == 0 || a.family[j - 1] != f) {
            // end of the run of family f (families are sorted): a short
            // forward look first, bisection for long runs
            int e = j + 1;
            while (e < R && e < j + 8 && a.family[e] == f) ++e;
            if (e < R && a.family[e] == f) {
                int lo = e + 1, hi = R;  // first index with family > f
                while (lo < hi) {
                    const int mid = lo + ((hi - lo) >> 1);
                    if (a.family[mid] > f) hi = mid; else lo = mid + 1;
                }
                e = lo;
            }
            // c ln c of the run; a run of one adds exactly 0 (GB300's FP64 log
            // is costly: short runs read it from the context's table, which
            // holds the same device log of the same argument)
            const int cn = e - j;
            if (cn > 1) {
                const double c = (double)cn;
                const double lc = (a.logc && cn < kLogC) ? a.logc[cn] : log(c);
                clnc = __fma_rn(c, lc, clnc);
            }
        }
    }
    // fixed shuffle trees; the FP64 ones only where they can add something
    // (GB300 has little FP64 throughput): +-J energies are integer sums, and a
    // warp without a family start has clnc = 0 in every lane
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        se += __shfl_down_sync(0xffffffffu, se, off);
        se2 += __shfl_down_sync(0xffffffffu, se2, off);
        const long long lo = __shfl_down_sync(0xffffffffu, (long long)(unsigned long long)mn, off);
        const long long hi = __shfl_down_sync(0xffffffffu, (long long)(mn >> 64), off);
        const __int128 o = ((__int128)hi << 64) | (unsigned long long)lo;
        if (o < mn) mn = o;
    }
    if (a.kind != 0) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            sed = __dadd_rn(sed, __shfl_down_sync(0xffffffffu, sed, off));
            se2d = __dadd_rn(se2d, __shfl_down_sync(0xffffffffu, se2d, off));
        }
    }
    if (__any_sync(0xffffffffu, clnc != 0.0)) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) clnc = __dadd_rn(clnc, __shfl_down_sync(0xffffffffu, clnc, off));
    }
    if (lane == 0) {
        s_ll[0][warp] = se; s_ll[1][warp] = se2;
        s_d[0][warp] = sed; s_d[1][warp] = se2d; s_d[2][warp] = clnc;
        s_min[warp] = mn;
    }
    __syncthreads();
    if (tid == 0) {
        ObsPartial p;
        p.sumE = 0; p.sumE2 = 0; p.sumEd = 0.0; p.sumE2d = 0.0; p.clnc = 0.0; p.pad = 0.0;
        __int128 M = s_min[0];
        for (int w = 0; w < 32; ++w) {
            p.sumE += s_ll[0][w]; p.sumE2 += s_ll[1][w];
            p.sumEd = __dadd_rn(p.sumEd, s_d[0][w]); p.sumE2d = __dadd_rn(p.sumE2d, s_d[1][w]);
            p.clnc = __dadd_rn(p.clnc, s_d[2][w]);
            if (s_min[w] < M) M = s_min[w];
        }
        p.min_lo = (long long)(unsigned long long)M;
        p.min_hi = (long long)(M >> 64);
        a.part[blockIdx.x] = p;
    }
}
__device__ __forceinline__ void observe_final_body(const ObsArgs& a);
__global__ void __launch_bounds__(1024) observe_partial_kernel(ObsArgs a)
{
    observe_partial_body(a);
    if (a.sync && last_block(a.sync) && threadIdx.x < 32) observe_final_body(a);  // combine in a fixed order
}
__global__ void __launch_bounds__(1024) observe_partial_batched(const ObsArgs* tab)
{
    observe_partial_body(tab[blockIdx.y]);
}

// partials combined by one warp: lane l adds blocks l, l + 32, ... in order,
// then the 32 lane sums are added by a fixed shuffle tree (the same order on
// every GPU)
__device__ __forceinline__ void observe_final_body(const ObsArgs& a)
{
    const int lane = threadIdx.x & 31;
    long long A = 0, B = 0;
    double C = 0.0, Dd = 0.0, F = 0.0;
    __int128 M = (__int128)(((unsigned __int128)1 << 127) - 1);
    const int nb = obs_blocks(a.Rdev ? *a.Rdev : a.R);
    for (int b = lane; b < nb; b += 32) {
        const ObsPartial p = a.part[b];
        A += p.sumE; B += p.sumE2;
        C = __dadd_rn(C, p.sumEd); Dd = __dadd_rn(Dd, p.sumE2d); F = __dadd_rn(F, p.clnc);
        const __int128 m = ((__int128)p.min_hi << 64) | (unsigned long long)p.min_lo;
        if (m < M) M = m;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        A += __shfl_down_sync(0xffffffffu, A, off);
        B += __shfl_down_sync(0xffffffffu, B, off);
        C = __dadd_rn(C, __shfl_down_sync(0xffffffffu, C, off));
        Dd = __dadd_rn(Dd, __shfl_down_sync(0xffffffffu, Dd, off));
        F = __dadd_rn(F, __shfl_down_sync(0xffffffffu, F, off));
        const long long lo = __shfl_down_sync(0xffffffffu, (long long)(unsigned long long)M, off);
        const long long hi = __shfl_down_sync(0xffffffffu, (long long)(M >> 64), off);
        const __int128 o = ((__int128)hi << 64) | (unsigned long long)lo;
        if (o < M) M = o;
    }
    if (lane != 0) return;
    a.cur->sumE = A; a.cur->sumE2 = B;
    a.cur->sumEd = C; a.cur->sumE2d = Dd;
    a.cur->sum_clnc = F;
    a.cur->emin_lo = (long long)(unsigned long long)M;
    a.cur->emin_hi = (long long)(M >> 64);
}
__global__ void observe_final_kernel(ObsArgs a)
{
    if (threadIdx.x < 32) observe_final_body(a);
}
// one warp per instance
__global__ void observe_final_batched(const ObsArgs* tab, int n_inst)
{
    const int i = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (i < n_inst) observe_final_body(tab[i]);
}

cudaError_t launch_observe(const ObsArgs& a, cudaStream_t st)
{
    observe_partial_kernel<<<obs_blocks(a.R), 1024, 0, st>>>(a);
    if (!a.sync) observe_final_kernel<<<1, 32, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_observe_batched(const ObsArgs* tab, int n_inst, int maxR, cudaStream_t st)
{
    observe_partial_batched<<<dim3(obs_blocks(maxR), (unsigned)n_inst), 1024, 0, st>>>(tab);
    observe_final_batched<<<(n_inst + 7) / 8, 256, 0, st>>>(tab, n_inst);
    return cudaGetLastError();
}

// ---------------- backward pass of sum_k gbar_k beta_k F_k ----------------
// d(beta F)/dJ_b = -beta <S_i S_j>, d(beta F)/dh_i = -beta <S_i> (from Eq. 1),
// estimated with the exact population sums after the sweeps at beta_k.
__global__ void grad_backward_kernel(const unsigned long long* cJ, const unsigned long long* ch,
                                     const double* gbar, const double* betas, const double* Rk,
                                     int n_temps, int nJ, int N, double* dJ, double* dh)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nJ + N) return;
    const bool isJ = b < nJ;
    const int idx = isJ ? b : b - nJ;
    const int stride = isJ ? nJ : N;
    const unsigned long long* c = isJ ? cJ : ch;
    double acc = 0.0;
    for (int k = 0; k < n_temps; ++k) {
        const double m = __ddiv_rn((double)(long long)c[(size_t)k * stride + idx], Rk[k]);
        acc = __dadd_rn(acc, __dmul_rn(gbar[k], -__dmul_rn(betas[k], m)));
    }
    if (isJ) dJ[idx] = acc; else dh[idx] = acc;
}

cudaError_t launch_grad_backward(const unsigned long long* cJ, const unsigned long long* ch,
                                 const double* gbar, const double* betas, const double* Rk,
                                 int n_temps, int nJ, int N, double* dJ, double* dh, cudaStream_t st)
{
    const int n = nJ + N;
    grad_backward_kernel<<<(n + 255) / 256, 256, 0, st>>>(cJ, ch, gbar, betas, Rk, n_temps, nJ, N, dJ, dh);
    return cudaGetLastError();
}

}  // namespace pa
