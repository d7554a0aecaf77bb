// pa_packed_part2.cu -- packed sweep kernels for 3D L=10, 3D L=6, 3D L=14, 2D L=10, 2D L=12
// (one of four translation units that share the lattice sizes).
#include "pa_packed_sweep.cuh"

namespace pa {

cudaError_t launch_sweep_packed_part2(int D, int L, const PackedSweepArgs& a, int gpb, int threads,
                                      cudaStream_t st, bool* handled)
{
    *handled = true;
#define X(d, l) if (D == d && L == l) return launch_dl<d, l>(a, gpb, threads, st);
    X(3, 10) X(3, 6) X(3, 14) X(2, 10) X(2, 12)
#undef X
    *handled = false;
    return cudaSuccess;
}

}  // namespace pa
