// Host instantiation of the library's device primitives (pa_device.cuh), for
// CPU tests that compare them with the oracle.  Test infrastructure only.
#include "pa_device.cuh"

extern "C" void shim_philox(long n, const unsigned* ctr, const unsigned* key, unsigned* out)
{
    for (long t = 0; t < n; ++t) {
        pa::u32x4 o = pa::philox(ctr[4 * t], ctr[4 * t + 1], ctr[4 * t + 2], ctr[4 * t + 3], key[0], key[1]);
        out[4 * t] = o.x; out[4 * t + 1] = o.y; out[4 * t + 2] = o.z; out[4 * t + 3] = o.w;
    }
}
extern "C" void shim_exp64(long n, const double* x, double* y)
{
    for (long t = 0; t < n; ++t) y[t] = pa::spec_exp64(x[t]);
}
extern "C" void shim_expf(long n, const float* x, float* y)
{
    for (long t = 0; t < n; ++t) y[t] = pa::spec_expf(x[t]);
}
extern "C" unsigned long long shim_threshold_pm(double beta, int dE) { return pa::threshold_pm(beta, dE); }
extern "C" double shim_uniform53(unsigned a, unsigned b) { return pa::uniform53(a, b); }
