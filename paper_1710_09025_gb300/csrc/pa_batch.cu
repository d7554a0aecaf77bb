// pa_batch.cu -- the batched sweep: one persistent launch over the replica
// tiles of many instances (mixed L, +-J and real couplings).
//
// Blocks take work items (instance, tile) from a queue in global memory (one
// atomic counter per temperature) and run the same tile functions as the
// single-instance kernels, so every instance gets exactly the results of its
// own context.  Items are ordered by decreasing cost so that the expensive
// tiles start first and the tail is made of cheap ones.
#include "pa_sweep_tiles.cuh"

namespace pa {

constexpr int kBatchThreads = 256;

// 3D lattices the batched sweep dispatches to: packed +-J (two groups-per-
// block choices) and int8 real couplings.
#define PA_BATCH_PACKED(X) X(0, 4) X(1, 6) X(2, 8) X(3, 10) X(4, 12) X(5, 16)
#define PA_BATCH_REAL(X) X(0, 4) X(1, 6) X(2, 8) X(3, 10) X(4, 12)

__global__ void __launch_bounds__(kBatchThreads, 3) sweep_batch_kernel(PackedStep ps, RealStep rs,
                                                                    const BatchSweepInst* insts,
                                                                    const int2* items, int n_items,
                                                                    int mult, int* counter)
{
    extern __shared__ __align__(16) unsigned char smem_b[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) return;
        const int2 w = items[it];
        const BatchSweepInst& bi = insts[w.x];
        const int cls = bi.cls < kBatchRealBase ? bi.cls + (mult - 1) : bi.cls;
        switch (cls) {
#define XP(idx, l)                                                                                  \
    case 2 * idx: {                                                                                 \
        constexpr int g = default_shape<3, l>().gpb;                                                \
        sweep_packed_tile<3, l, g, kBatchThreads, false, false>(ps, bi.pk, w.y * g, smem_b);               \
    } break;                                                                                        \
    case 2 * idx + 1: {                                                                             \
        constexpr int g = 2 * default_shape<3, l>().gpb;                                            \
        sweep_packed_tile<3, l, g, kBatchThreads, false, false>(ps, bi.pk, w.y * g, smem_b);               \
    } break;
            PA_BATCH_PACKED(XP)
#undef XP
#define XR(idx, l)                                                                                  \
    case kBatchRealBase + idx:                                                                      \
        real_stage<3, l, kBatchThreads / 32>(bi.re, smem_b, false);                                 \
        sweep_real_tile<3, l, kBatchThreads / 32>(rs, bi.re, w.y, smem_b, false);                   \
        break;
            PA_BATCH_REAL(XR)
#undef XR
            default:
                break;
        }
    }
}

// class id, tiles and shared memory of an instance in the batched sweep
bool batch_class(int D, int L, int kind, int mult, int G, int R, int* cls, int* tiles, size_t* smem)
{
    if (D != 3) return false;
    if (kind == 0) {
#define XP(idx, l)                                                                            \
    if (L == l) {                                                                             \
        constexpr int g = default_shape<3, l>().gpb;                                          \
        *cls = 2 * idx;                                                                       \
        *tiles = (G + g * mult - 1) / (g * mult);                                             \
        *smem = mult == 1 ? PackedShape<3, l, g, kBatchThreads, false>::SMEM                  \
                          : PackedShape<3, l, 2 * g, kBatchThreads, false>::SMEM;             \
        return true;                                                                          \
    }
        PA_BATCH_PACKED(XP)
#undef XP
        return false;
    }
#define XR(idx, l)                                                                            \
    if (L == l) {                                                                             \
        *cls = kBatchRealBase + idx;                                                          \
        *tiles = (R + 31) / 32;                                                               \
        *smem = RealShape<3, l, kBatchThreads / 32>::SMEM;                                    \
        return true;                                                                          \
    }
    PA_BATCH_REAL(XR)
#undef XR
    return false;
}

cudaError_t batch_sweep_occupancy(size_t smem, int* blocks_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(sweep_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, sweep_batch_kernel,
                                                         kBatchThreads, smem);
}

cudaError_t launch_sweep_batched(const PackedStep& ps, const RealStep& rs, const BatchSweepInst* insts,
                                 const int2* items, int n_items, int mult, int* counter, int blocks,
                                 size_t smem, cudaStream_t st)
{
    sweep_batch_kernel<<<blocks, kBatchThreads, smem, st>>>(ps, rs, insts, items, n_items, mult, counter);
    return cudaGetLastError();
}

}  // namespace pa
