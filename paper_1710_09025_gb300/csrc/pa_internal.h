// pa_internal.h -- declarations shared by the CUDA translation units of libpamc.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace pa {

// Per-temperature accumulators kept on the device (one per step k).
struct StepAcc {
    long long sumE, sumE2;     // +-J: exact integer sums over the population
    double sumEd, sumE2d;      // real couplings: FP64 sums (fixed order)
    long long emin_lo, emin_hi;// lowest energy as int128 (+-J: sign-extended int32)
    double lnQ;                // ln Q_k (0 at k = 0)
    double sum_lnQ;            // sum_{l <= k} ln Q_l (sequential in l)
    double betaF;              // beta_k F_k = -N ln 2 - sum_lnQ
    double S;                  // sum of resampling weights (relative to E_min)
    double sum_clnc;           // sum over families of c ln c (family entropy)
    long long pad;
};
static_assert(sizeof(StepAcc) == 96, "StepAcc layout");

// ---------------- packed +-J path ----------------
// Parameters of one temperature, uniform over every instance of a launch.
struct PackedStep {
    int k, n_sweeps;         // n_sweeps: sweeps of this launch
    uint32_t hs0;            // half-sweep index of its first half-sweep, 2 (k N_S + first sweep)
    int mode;                // undecided uphill classes: 1 = {dE=4}, 2 = {dE=4, dE=8},
                             // 3 = every uphill class (3D, none always accepted), 0 = any set
    uint32_t und;            // bit c: class c (dE = 4c) needs a random comparison (0 < thr < 2^32)
    uint32_t always;         // bit c: class c always accepted (thr == 2^32)
    uint32_t rk[20];         // Philox round keys: rk[2r] = k0 + r W0, rk[2r+1] = k1 + r W1
    // per plane b (bit 31-b of the thresholds) as 0 / ~0 masks, selected by the
    // two low bits (b1 b0) of the unsatisfied-bond count n of an uphill lane:
    // v00: n = 0, v01: n = 1, v10: n = 2
    uint32_t v00[32], v01[32], v10[32];
    uint32_t zero_planes;    // bit b: every threshold bit of plane b is 0 (a 1 in r rejects)
};
// Parameters of one instance.
struct PackedInst {
    uint64_t* S;             // [G][N] words out
    const uint64_t* Sin;     // [G][N] words in (== S without resampling); with parent != null,
                             // lane j of group g reads replica parent[64g+j]
    const uint8_t* jneg;     // [N] bit k: coupling to neighbour k (-x,+x,-y,+y,-z,+z) negative
    int32_t* E;              // [R] energies out
    int8_t* S8_in;           // int8 storage of the same algorithm (layout I8): rows of NP bytes
    int8_t* S8_out;          // non-null selects the int8 storage
    const int32_t* parent;   // or null (identity)
    const int* Rdev;         // population in device memory (or null: R); G, R then size the grid
    int G, R, NP;
    uint32_t c3;             // Philox counter word 3 of the PLANE stream
    int goff;                // global index of group 0 (a shard of a larger population; else 0)
};
struct PackedSweepArgs {
    PackedStep s;
    PackedInst i;
};
cudaError_t launch_sweep_packed(int D, int L, const PackedSweepArgs& a, int gpb, int threads,
                                cudaStream_t st);
bool packed_supported(int D, int L);
void packed_default_shape(int D, int L, int* gpb, int* threads);
cudaError_t launch_init_packed(uint64_t* S, int N, int G, uint32_t k0, uint32_t k1, uint32_t c3,
                               cudaStream_t st, int goff = 0);
cudaError_t launch_unpack_packed(const uint64_t* S, int8_t* out, int N, int r0, int n, cudaStream_t st);
cudaError_t launch_overlap_packed(const uint64_t* A, const uint64_t* B, int N, int R,
                                  unsigned long long* hist, cudaStream_t st);

// the replica gather as its own launch (packed words if Sin, else int8 rows):
// slot j of the new population takes replica parent[j]
cudaError_t launch_gather(const uint64_t* Sin, uint64_t* Sout, const int8_t* S8in, int8_t* S8out,
                          const int32_t* parent, int N, int NP, int R, const int* Rdev, cudaStream_t st);
// gradient counts of a +-J population after the sweeps (packed words if S,
// else int8 rows), added to cJ (D*N) and ch (N) of this step
cudaError_t launch_grad_counts_pm(const uint64_t* S, const int8_t* S8, int NP, int D, int L, int R,
                                  const int* Rdev, unsigned long long* cJ, unsigned long long* ch,
                                  cudaStream_t st);

// ---------------- int8 path ----------------
struct RealStep {
    int k, n_sweeps;         // n_sweeps: sweeps of this launch
    uint32_t hs0;            // 2 (k N_S + first sweep)
    float beta;
    uint32_t key0, key1;
    int band;                // 1: the acceptance guard band is verified on this device
    uint32_t rk[20];         // Philox round keys of (key0, key1), as in PackedStep
};
struct RealInst {
    const int8_t* Sin;       // rows of NP bytes (+1/-1)
    int8_t* Sout;
    const int32_t* parent;   // gather rows parent[r] (or null)
    const float* J;          // [D*N] (flushed)
    const float* h;          // [N] (zeros without a field)
    const longlong2* Jfix;   // [D*N] J * 2^96 as int128 (lo, hi)
    const longlong2* hfix;   // [N]
    longlong2* E;            // [R] energies * 2^96 out
    unsigned long long* cJ;  // [D*N] grad counts of this step (or null)
    unsigned long long* ch;  // [N]
    const int* Rdev;         // population in device memory (or null: R); R then sizes the grid
    int R, NP;
    uint32_t c3;             // Philox counter word 3 of the WORD stream
};
struct RealSweepArgs {
    RealStep s;
    RealInst i;
};
cudaError_t launch_sweep_real(int D, int L, const RealSweepArgs& a, int warps, int grid,
                              cudaStream_t st);
bool real_supported(int D, int L);
// verifies the acceptance guard band for every positive finite float
// (violations: count of x where it fails; max_rel_dev: largest |g/e - 1| for
// 0 < x <= 87); synchronises st
cudaError_t accept_band_check(cudaStream_t st, unsigned long long* violations, double* max_rel_dev);
// the verdict for the current device, checked once per process
int accept_band_ok(cudaStream_t st);
cudaError_t launch_init_i8(int8_t* S, int N, int NP, int R, uint32_t k0, uint32_t k1, uint32_t c3,
                           cudaStream_t st, int goff = 0);
cudaError_t launch_overlap_i8(const int8_t* A, const int8_t* B, int N, int NP, int R,
                              unsigned long long* hist, cudaStream_t st);

// ---------------- batched sweep ----------------
constexpr int kBatchRealBase = 100;   // class ids >= this are real-coupling tiles
struct BatchSweepInst {
    int cls;                 // packed: 2 * lattice index (+1 for the doubled groups per block)
    int pad;
    PackedInst pk;
    RealInst re;
};
bool batch_class(int D, int L, int kind, int mult, int G, int R, int* cls, int* tiles, size_t* smem);
cudaError_t batch_sweep_occupancy(size_t smem, int* blocks_per_sm);
cudaError_t launch_sweep_batched(const PackedStep& ps, const RealStep& rs, const BatchSweepInst* insts,
                                 const int2* items, int n_items, int mult, int* counter, int blocks,
                                 size_t smem, cudaStream_t st);

// ---------------- isoenergetic cluster moves (Sec. II.C) ----------------
struct IcmArgs {
    int D, L, N, NP;
    uint64_t* S;             // packed words [G][N] (or null)
    int8_t* S8;              // int8 rows [R][NP] (or null)
    const int* Rdev;         // population in device memory (or null: R)
    int R;                   // population, or the capacity with Rdev
    int k, t;                // step, round (0 or 1)
    uint32_t key0, key1, c3; // Philox key, counter word 3 of the ICM stream
    int* err;                // set if a bounded union-find loop gave up
};
cudaError_t launch_icm(const IcmArgs& a, cudaStream_t st);

// ---------------- resampling and observables ----------------
struct ResampleArgs {
    int R, kind;                 // R: source replicas; kind 0: E32, 1: E128
    int Rn;                      // copies drawn (the new population)
    // nearest-integer scheme (scheme 1): populations live in device memory;
    // R above is then the capacity and sizes the grids
    int scheme, cap;
    double target;               // expected new population R(beta')
    const int* Rsrc;             // source population (or null: R)
    int* Rdst;                   // new population min(sum n_i, cap) out
    double* Rdst_d;              // the same as a double (gradient normalisation)
    const int32_t* E32;
    const longlong2* E128;
    const StepAcc* prev;         // acc[k-1]: E_min, sum_lnQ
    StepAcc* cur;                // acc[k]: lnQ, sum_lnQ, betaF, S
    double* w;                   // [R] weights
    const double* wtab;          // +-J: weight per level (E - E_min) / 4, or null
    int wtab_n;                  // levels in wtab
    // two zeroed block counters: with them the last block of the weights
    // launch completes the prefix (upper levels, run offsets, running maximum,
    // S, ln Q) and the last block of the block-sum launch scans the block sums
    // (no separate launches); null: separate launches
    int* sync;
    double* P;                   // [R] sums inside runs of 32, then the cumulative weights
                                 // up to the running maximum over earlier weights blocks
    double* lev1;                // [rs_leaves(R)] level-1 sums inside runs of 32 runs, then
                                 // the inclusive prefix of the run totals
    double* bmax;                // [2 rs_wblocks(R)] largest prefix sum of each weights block,
                                 // then the largest before each block (running maximum)
    double* upper;               // [rs_upper_size(R)] levels 2, 3, ... of the prefix
    // a shard of a population of gR replicas spread over several contexts
    // (gR = 0: not sharded): the local replicas are the global replicas
    // [kWBlock gb0, kWBlock gb0 + R); upper and bmax then hold the global
    // levels (rs_upper_size(gR), 2 rs_wblocks(gR)), t2g the global block
    // totals, the draws are the gR global ones (only those landing on local
    // replicas are counted), and parents are written as global indices
    int gR, gb0;
    const double* t2g;
    int32_t* counts;             // [R] copy numbers (zero on entry, zeroed again on exit)
    int32_t* blocksum;           // [nblocks] scratch for the count scan
    int32_t* parent;             // [R] out
    const int32_t* fam_in;       // [R]
    int32_t* fam_out;            // [R]
    double dbeta, log_R, betaF0;
    int k;
    uint32_t key0, key1, c3;
};
// Weight prefix in a fixed order of fan-out kFan: runs of kFan weights summed
// left to right, the run totals likewise, recursively; each weights block
// covers kFan runs (kFan^2 weights, levels 0 and 1).
constexpr int kFan = 32;
constexpr int kWBlock = kFan * kFan;
__host__ __device__ constexpr inline int rs_leaves(int R) { return (R + kFan - 1) / kFan; }
__host__ __device__ constexpr inline int rs_wblocks(int R) { return (R + kWBlock - 1) / kWBlock; }
// doubles of the levels >= 2 (block totals, then their run totals, ...)
__host__ __device__ constexpr inline int rs_upper_size(int R)
{
    int n = rs_wblocks(R), t = 0;
    for (;;) {
        t += n;
        if (n <= kFan) return t;
        n = (n + kFan - 1) / kFan;
    }
}
constexpr int kScanBlock = 4096; // elements per block of the copy-number scan
cudaError_t launch_resample(const ResampleArgs& a, cudaStream_t st);
// one phase (0..3) of a shard's resampling (a.gR > 0, a.sync null)
cudaError_t launch_resample_shard(const ResampleArgs& a, int phase, cudaStream_t st);
// all instances of a batch at once: tab[i] describes instance i (device memory)
cudaError_t launch_resample_batched(const ResampleArgs* tab, int n_inst, int maxR, cudaStream_t st);

struct ObsPartial {
    long long sumE, sumE2, min_lo, min_hi;
    double sumEd, sumE2d, clnc, pad;
};
constexpr int kObsBlocks = 608;  // most blocks of the observables reduction (4 per SM of GB300)
// blocks of the observables reduction for a population of R (a function of R
// only, non-decreasing, so that a grid sized for a capacity covers any smaller
// population): about 4096 replicas each, but at least min(ceil(R / 1024), 304)
// blocks, so that small populations spread their FP64 work over many SMs
// (R = 10^5: 0.048 -> 0.026 ms per step), at most kObsBlocks
__host__ __device__ constexpr inline int obs_blocks(int R)
{
    const int a = (R + 4095) / 4096, b = (R + 1023) / 1024 < 304 ? (R + 1023) / 1024 : 304;
    const int n = a > b ? a : b;
    return n < 1 ? 1 : (n > kObsBlocks ? kObsBlocks : n);
}
struct ObsArgs {
    int R, kind;
    const int* Rdev;             // population in device memory (or null: R)
    const int32_t* E32;
    const longlong2* E128;
    const int32_t* family;
    ObsPartial* part;            // [kObsBlocks] scratch
    const double* logc;          // [kLogC] log(c) for the family entropy (or null)
    StepAcc* cur;
    int* sync;                   // zeroed block counter: the last block combines (or null)
};
// family sizes below kLogC take log(c) from a table that the context fills
// once with the same device log; larger ones evaluate it
constexpr int kLogC = 4096;
cudaError_t launch_logc_table(double* t, cudaStream_t st);
cudaError_t launch_observe(const ObsArgs& a, cudaStream_t st);
cudaError_t launch_observe_batched(const ObsArgs* tab, int n_inst, int maxR, cudaStream_t st);
cudaError_t launch_grad_backward(const unsigned long long* cJ, const unsigned long long* ch,
                                 const double* gbar, const double* betas, const double* Rk,
                                 int n_temps, int nJ, int N, double* dJ, double* dh, cudaStream_t st);

// message returned by pa_last_error(NULL) for calls without a context
void set_global_error(const char* msg);

}  // namespace pa
