// pa_packed_part1.cu -- packed sweep kernels for 3D L=12, 3D L=4, 2D L=6, 2D L=8
// (one of four translation units that share the lattice sizes).
#include "pa_packed_sweep.cuh"

namespace pa {

cudaError_t launch_sweep_packed_part1(int D, int L, const PackedSweepArgs& a, int gpb, int threads,
                                      cudaStream_t st, bool* handled)
{
    *handled = true;
#define X(d, l) if (D == d && L == l) return launch_dl<d, l>(a, gpb, threads, st);
    X(3, 12) X(3, 4) X(2, 6) X(2, 8)
#undef X
    *handled = false;
    return cudaSuccess;
}

}  // namespace pa
