// pa_packed_part3.cu -- packed sweep kernels for 3D L=8, 2D L=16, 2D L=32, 2D L=64
// (one of four translation units that share the lattice sizes).
#include "pa_packed_sweep.cuh"

namespace pa {

cudaError_t launch_sweep_packed_part3(int D, int L, const PackedSweepArgs& a, int gpb, int threads,
                                      cudaStream_t st, bool* handled)
{
    *handled = true;
#define X(d, l) if (D == d && L == l) return launch_dl<d, l>(a, gpb, threads, st);
    X(3, 8) X(2, 16) X(2, 32) X(2, 64)
#undef X
    *handled = false;
    return cudaSuccess;
}

}  // namespace pa
