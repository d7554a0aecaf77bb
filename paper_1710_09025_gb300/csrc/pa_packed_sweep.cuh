// pa_packed_sweep.cuh -- the packed (+-J) sweep kernel and its launch
// templates.  Each lattice size instantiates four kernels (two groups-per-
// block choices, packed or int8 storage); the sizes are spread over the
// translation units pa_packed_part0..3.cu so that they compile in parallel.
#pragma once
#include "pa_sweep_tiles.cuh"

namespace pa {

template <int D, int L, int GPB, int THREADS, bool I8, bool SHARD = false>
__global__ void __launch_bounds__(THREADS, 4) sweep_packed_kernel(PackedSweepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_packed[];
    sweep_packed_tile<D, L, GPB, THREADS, I8, true, SHARD>(a.s, a.i, blockIdx.x * GPB, smem_packed);
}

// ---------------- shapes and dispatch ----------------

template <int D, int L, int GPB, int THREADS, bool I8, bool SHARD = false>
static cudaError_t launch_one(const PackedSweepArgs& a, cudaStream_t st)
{
    const size_t smem = PackedShape<D, L, GPB, THREADS>::SMEM;
    auto kern = sweep_packed_kernel<D, L, GPB, THREADS, I8, SHARD>;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    int grid = (a.i.G + GPB - 1) / GPB;
    kern<<<grid, THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

template <int D, int L>
static cudaError_t launch_dl(const PackedSweepArgs& a, int gpb, int threads, cudaStream_t st)
{
    constexpr Shape s = default_shape<D, L>();
    const bool i8 = a.i.S8_out != nullptr;
    if (a.i.goff != 0) {  // a shard (packed words, default shape)
        if (i8 || gpb != s.gpb || threads != s.threads) return cudaErrorInvalidConfiguration;
        return launch_one<D, L, s.gpb, s.threads, false, true>(a, st);
    }
    // the one tuned alternative: twice the groups per block, same thread count
    if (gpb == 2 * s.gpb && threads == s.threads)
        return i8 ? launch_one<D, L, 2 * s.gpb, s.threads, true>(a, st)
                  : launch_one<D, L, 2 * s.gpb, s.threads, false>(a, st);
    if (gpb != s.gpb || threads != s.threads) return cudaErrorInvalidConfiguration;
    return i8 ? launch_one<D, L, s.gpb, s.threads, true>(a, st)
              : launch_one<D, L, s.gpb, s.threads, false>(a, st);
}

// launch for the lattice sizes of one part: *handled is false when (D, L)
// belongs to another part
cudaError_t launch_sweep_packed_part0(int D, int L, const PackedSweepArgs& a, int gpb, int threads,
                                      cudaStream_t st, bool* handled);
cudaError_t launch_sweep_packed_part1(int D, int L, const PackedSweepArgs& a, int gpb, int threads,
                                      cudaStream_t st, bool* handled);
cudaError_t launch_sweep_packed_part2(int D, int L, const PackedSweepArgs& a, int gpb, int threads,
                                      cudaStream_t st, bool* handled);
cudaError_t launch_sweep_packed_part3(int D, int L, const PackedSweepArgs& a, int gpb, int threads,
                                      cudaStream_t st, bool* handled);

}  // namespace pa
