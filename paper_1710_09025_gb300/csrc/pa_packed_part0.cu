// pa_packed_part0.cu -- packed sweep kernels for 3D L=16, 3D L=2, 2D L=2, 2D L=4
// (one of four translation units that share the lattice sizes).
#include "pa_packed_sweep.cuh"

namespace pa {

cudaError_t launch_sweep_packed_part0(int D, int L, const PackedSweepArgs& a, int gpb, int threads,
                                      cudaStream_t st, bool* handled)
{
    *handled = true;
#define X(d, l) if (D == d && L == l) return launch_dl<d, l>(a, gpb, threads, st);
    X(3, 16) X(3, 2) X(2, 2) X(2, 4)
#undef X
    *handled = false;
    return cudaSuccess;
}

}  // namespace pa
