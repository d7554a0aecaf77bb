// pa_api.cu -- the C ABI of libpamc (declared in include/pa.h).
//
// Host orchestration of one population annealing run (Sec. II.B):
//   k = 0 : random replicas (INIT stream), family id = slot
//   k > 0 : resampling beta_{k-1} -> beta_k (weights, prefix, draws, parents,
//           families), replica gather
//   every k: N_S checkerboard sweeps at beta_k with energies in the epilogue,
//           then the observables reduction.
// All device work is enqueued on the context's stream; pa_anneal captures a
// run of steps into one CUDA graph.
#include "pa.h"
#include "pa_device.cuh"
#include "pa_internal.h"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using pa::StepAcc;

struct pa_ctx {
    int D, L, N, kind, R, G, n_temps, n_sweeps, k_next, layout, NP;
    uint64_t seed;
    uint32_t inst, tag;
    int acc_grad;
    cudaStream_t st;
    int gpb, threads, real_warps;
    double betaF0, log_R;
    std::vector<double> betas;
    std::vector<float> Jh, hh;  // flushed host copies
    // device
    void* ws;
    bool own_ws;
    float* J;
    float* h;
    uint8_t* jneg;
    longlong2* Jfix;
    longlong2* hfix;
    double* betas_d;
    uint64_t* S[2];
    int8_t* S8[2];
    int cur;
    int32_t* E32;
    longlong2* E128;
    int32_t* parent;
    int32_t* fam[2];
    int famcur;
    int32_t* counts;
    int32_t* blocksum;
    double *w, *P, *tot, *T;
    StepAcc* acc;
    unsigned long long *cJ, *ch;
    int8_t* tmp8;
    unsigned long long* hist;
    double *gbar_d, *dJ_d, *dh_d;
    pa::ObsPartial* obspart;
    cudaGraphExec_t gexec;
    std::string err;
    // profiling: event pairs per phase, launch counter
    int profiling;
    bool capturing;
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
    long long launches;
};

// records the start of a phase; returns the start event (or null)
static cudaEvent_t phase_begin(pa_ctx* c)
{
    if (!c->profiling || c->capturing) return nullptr;
    cudaEvent_t e;
    if (!c->ev_free.empty()) { e = c->ev_free.back(); c->ev_free.pop_back(); }
    else if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    cudaEventRecord(e, c->st);
    return e;
}

static void phase_end(pa_ctx* c, int phase, cudaEvent_t start)
{
    if (!start) return;
    cudaEvent_t e;
    if (!c->ev_free.empty()) { e = c->ev_free.back(); c->ev_free.pop_back(); }
    else if (cudaEventCreate(&e) != cudaSuccess) { c->ev_free.push_back(start); return; }
    cudaEventRecord(e, c->st);
    c->ev_pending.push_back({phase, {start, e}});
}

static thread_local std::string g_create_err;

void pa::set_global_error(const char* msg) { g_create_err = msg ? msg : ""; }

#define PA_CK(ctx, call)                                                                 \
    do {                                                                                 \
        cudaError_t e__ = (call);                                                        \
        if (e__ != cudaSuccess) {                                                        \
            (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e__);            \
            return PA_ECUDA;                                                             \
        }                                                                                \
    } while (0)

// ---------------- small kernels of the orchestration ----------------

__global__ void iota_kernel(int32_t* a, int32_t* b, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        a[i] = i;
        if (b) b[i] = i;
    }
}

__global__ void acc0_kernel(StepAcc* acc, double betaF0, int R)
{
    acc->lnQ = 0.0;
    acc->sum_lnQ = 0.0;
    acc->betaF = betaF0;
    acc->S = (double)R;
}

// ---------------- workspace layout ----------------

struct Layout {
    size_t off[32];
    size_t total;
};

enum {
    W_J, W_H, W_JNEG, W_JFIX, W_HFIX, W_BETAS, W_S0, W_S1, W_E32, W_E128, W_PARENT, W_FAM0, W_FAM1,
    W_COUNTS, W_BLOCKSUM, W_W, W_P, W_TOT, W_T, W_ACC, W_CJ, W_CH, W_TMP8, W_HIST, W_GBAR, W_DJ,
    W_DH, W_OBSPART, W_COUNT
};

static Layout make_layout(int D, int L, int kind, int layout, int R, int n_temps, int acc_grad)
{
    int N = (D == 3) ? L * L * L : L * L;
    int G = (R + 63) / 64;
    int NP = (N + 15) / 16 * 16;
    size_t sz[W_COUNT] = {};
    sz[W_J] = sizeof(float) * D * N;
    sz[W_H] = sizeof(float) * N;
    sz[W_JNEG] = N;
    sz[W_JFIX] = kind == PA_REAL ? sizeof(longlong2) * D * N : 0;
    sz[W_HFIX] = kind == PA_REAL ? sizeof(longlong2) * N : 0;
    sz[W_BETAS] = sizeof(double) * n_temps;
    size_t state = layout == PA_LAYOUT_PACKED ? sizeof(uint64_t) * (size_t)G * N : (size_t)R * NP;
    sz[W_S0] = state;
    sz[W_S1] = state;
    sz[W_E32] = kind == PA_PM1 ? sizeof(int32_t) * (size_t)R : 0;
    sz[W_E128] = kind == PA_REAL ? sizeof(longlong2) * (size_t)R : 0;
    sz[W_PARENT] = sizeof(int32_t) * (size_t)R;
    sz[W_FAM0] = sizeof(int32_t) * (size_t)R;
    sz[W_FAM1] = sizeof(int32_t) * (size_t)R;
    sz[W_COUNTS] = sizeof(int32_t) * (size_t)R;
    sz[W_BLOCKSUM] = sizeof(int32_t) * ((R + pa::kScanBlock - 1) / pa::kScanBlock + 1);
    sz[W_W] = sizeof(double) * (size_t)R;
    sz[W_P] = sizeof(double) * (size_t)R;
    int nch = (R + pa::kChunk - 1) / pa::kChunk;
    sz[W_TOT] = sizeof(double) * nch;
    sz[W_T] = sizeof(double) * (nch + 1);
    sz[W_ACC] = sizeof(StepAcc) * n_temps;
    sz[W_CJ] = acc_grad ? sizeof(unsigned long long) * (size_t)n_temps * D * N : 0;
    sz[W_CH] = acc_grad ? sizeof(unsigned long long) * (size_t)n_temps * N : 0;
    sz[W_TMP8] = layout == PA_LAYOUT_PACKED ? (size_t)R * N : 0;
    sz[W_HIST] = sizeof(unsigned long long) * (N + 1);
    sz[W_GBAR] = acc_grad ? sizeof(double) * n_temps : 0;
    sz[W_DJ] = acc_grad ? sizeof(double) * D * N : 0;
    sz[W_DH] = acc_grad ? sizeof(double) * N : 0;
    sz[W_OBSPART] = sizeof(pa::ObsPartial) * pa::kObsBlocks;
    Layout lay;
    size_t off = 0;
    for (int i = 0; i < W_COUNT; ++i) {
        lay.off[i] = off;
        off += (sz[i] + 255) & ~(size_t)255;
    }
    lay.total = off;
    return lay;
}

// ---------------- validation ----------------

static int resolve_layout(int kind, const pa_options* o)
{
    int lay = o ? o->layout : PA_LAYOUT_AUTO;
    if (lay == PA_LAYOUT_AUTO) lay = kind == PA_PM1 ? PA_LAYOUT_PACKED : PA_LAYOUT_I8;
    return lay;
}

static int validate(std::string& err, int D, int L, int kind, const float* J, const float* h, int R,
                    const double* betas, int n_temps, int n_sweeps, const pa_options* o)
{
    if (D != 2 && D != 3) { err = "D must be 2 or 3"; return PA_EINVAL; }
    if (L < 2 || (L & 1)) { err = "L must be even and >= 2 (checkerboard on a periodic lattice)"; return PA_EINVAL; }
    if (kind != PA_PM1 && kind != PA_REAL) { err = "kind must be PA_PM1 or PA_REAL"; return PA_EINVAL; }
    int lay = resolve_layout(kind, o);
    if (lay != PA_LAYOUT_PACKED && lay != PA_LAYOUT_I8) { err = "unknown layout"; return PA_EINVAL; }
    if (lay == PA_LAYOUT_PACKED && kind != PA_PM1) { err = "packed layout needs +-J couplings"; return PA_EINVAL; }
    bool sup = (kind == PA_PM1) ? pa::packed_supported(D, L) : pa::real_supported(D, L);
    if (!sup) { err = "lattice size not compiled in (3D: L in 2..12 even or 16; 2D: up to 32/64)"; return PA_EINVAL; }
    if (R < 1 || R > (1 << 26)) { err = "R must be in [1, 2^26]"; return PA_EINVAL; }
    if (n_temps < 1 || !betas) { err = "need at least one temperature"; return PA_EINVAL; }
    if (betas[0] != 0.0) { err = "betas[0] must be 0 (beta F starts from -N ln 2)"; return PA_EINVAL; }
    for (int k = 1; k < n_temps; ++k)
        if (!std::isfinite(betas[k]) || betas[k] < betas[k - 1]) { err = "betas must be finite and non-decreasing"; return PA_EINVAL; }
    if (n_sweeps < 0) { err = "n_sweeps must be >= 0"; return PA_EINVAL; }
    if (!J) { err = "J is NULL"; return PA_EINVAL; }
    int N = (D == 3) ? L * L * L : L * L;
    for (int b = 0; b < D * N; ++b) {
        float v = J[b];
        if (!std::isfinite(v)) { err = "J has NaN or Inf"; return PA_EINVAL; }
        if (kind == PA_PM1 && v != 1.0f && v != -1.0f) { err = "PA_PM1 needs J exactly +1 or -1"; return PA_EINVAL; }
        if (kind == PA_REAL && std::fabs(v) >= 4096.0f) { err = "|J| must be < 4096"; return PA_EINVAL; }
    }
    if (h) {
        for (int i = 0; i < N; ++i) {
            float v = h[i];
            if (!std::isfinite(v)) { err = "h has NaN or Inf"; return PA_EINVAL; }
            if (kind == PA_PM1 && v != 0.0f) { err = "PA_PM1 takes no field (use PA_REAL)"; return PA_EINVAL; }
            if (std::fabs(v) >= 4096.0f) { err = "|h| must be < 4096"; return PA_EINVAL; }
        }
    }
    if (o) {
        if (o->accumulate_grad && kind != PA_REAL) { err = "accumulate_grad needs PA_REAL"; return PA_EINVAL; }
        if (o->rng_instance >= (1u << 24)) { err = "rng_instance must be < 2^24"; return PA_EINVAL; }
        if (o->rng_tag >= 16u) { err = "rng_tag must be < 16"; return PA_EINVAL; }
    }
    return PA_OK;
}

// ---------------- public API ----------------

extern "C" int pa_options_default(pa_options* opt)
{
    if (!opt) return PA_EINVAL;
    std::memset(opt, 0, sizeof *opt);
    return PA_OK;
}

extern "C" int pa_workspace_size(int D, int L, int kind, int R, int n_temps, const pa_options* opt,
                                 size_t* bytes)
{
    if (!bytes || (D != 2 && D != 3) || L < 2 || R < 1 || n_temps < 1) return PA_EINVAL;
    int lay = resolve_layout(kind, opt);
    Layout l = make_layout(D, L, kind, lay, R, n_temps, opt ? opt->accumulate_grad : 0);
    *bytes = l.total;
    return PA_OK;
}

static float flush73(float v) { return std::fabs(v) < 0x1p-73f ? 0.0f : v; }

static longlong2 fix96(float v)
{
    __int128 x = (__int128)std::ldexp((double)v, 96);
    longlong2 r;
    r.x = (long long)(unsigned long long)x;
    r.y = (long long)(x >> 64);
    return r;
}

static int create_impl(pa_ctx** out, int D, int L, int kind, const float* J, const float* h, int R,
                       const double* betas, int n_temps, int n_sweeps, uint64_t seed,
                       const pa_options* opt, void* stream, void* workspace, size_t ws_bytes)
{
    if (!out) return PA_EINVAL;
    *out = nullptr;
    int rc = validate(g_create_err, D, L, kind, J, h, R, betas, n_temps, n_sweeps, opt);
    if (rc) return rc;
    pa_options o;
    pa_options_default(&o);
    if (opt) o = *opt;
    pa_ctx* c = new pa_ctx();
    c->D = D; c->L = L; c->N = (D == 3) ? L * L * L : L * L; c->kind = kind; c->R = R;
    c->G = (R + 63) / 64; c->n_temps = n_temps; c->n_sweeps = n_sweeps; c->k_next = 0;
    c->layout = resolve_layout(kind, &o); c->NP = (c->N + 15) / 16 * 16;
    c->seed = seed; c->inst = o.rng_instance; c->tag = o.rng_tag; c->acc_grad = o.accumulate_grad ? 1 : 0;
    c->st = (cudaStream_t)stream;
    c->betas.assign(betas, betas + n_temps);
    c->betaF0 = -(double)c->N * std::log(2.0);
    c->log_R = std::log((double)R);
    c->gexec = nullptr;
    c->profiling = 0;
    c->capturing = false;
    c->launches = 0;
    pa::packed_default_shape(D, L, &c->gpb, &c->threads);
    if (o.groups_per_block > 0) c->gpb = o.groups_per_block;
    if (o.threads > 0) c->threads = o.threads;
    c->real_warps = (kind == PA_REAL && o.threads == 128) ? 4 : 8;
    const int N = c->N;
    int nflush = 0;
    c->Jh.resize((size_t)D * N);
    c->hh.assign(N, 0.0f);
    for (int b = 0; b < D * N; ++b) {
        c->Jh[b] = kind == PA_REAL ? flush73(J[b]) : J[b];
        nflush += (c->Jh[b] != J[b]);
    }
    if (h && kind == PA_REAL)
        for (int i = 0; i < N; ++i) {
            c->hh[i] = flush73(h[i]);
            nflush += (c->hh[i] != h[i]);
        }
    if (nflush) c->err = "warning: " + std::to_string(nflush) + " coupling/field magnitudes below 2^-73 flushed to 0";

    Layout lay = make_layout(D, L, kind, c->layout, R, n_temps, c->acc_grad);
    if (workspace) {
        if (ws_bytes < lay.total || ((uintptr_t)workspace & 255)) {
            g_create_err = "workspace too small or not 256-byte aligned";
            delete c;
            return PA_ENOMEM;
        }
        c->ws = workspace;
        c->own_ws = false;
    } else {
        cudaError_t e = cudaMalloc(&c->ws, lay.total);
        if (e != cudaSuccess) {
            g_create_err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
            delete c;
            return PA_ENOMEM;
        }
        c->own_ws = true;
    }
    char* base = (char*)c->ws;
    auto at = [&](int w) -> void* { return base + lay.off[w]; };
    c->J = (float*)at(W_J); c->h = (float*)at(W_H); c->jneg = (uint8_t*)at(W_JNEG);
    c->Jfix = kind == PA_REAL ? (longlong2*)at(W_JFIX) : nullptr;
    c->hfix = kind == PA_REAL ? (longlong2*)at(W_HFIX) : nullptr;
    c->betas_d = (double*)at(W_BETAS);
    if (c->layout == PA_LAYOUT_PACKED) {
        c->S[0] = (uint64_t*)at(W_S0); c->S[1] = (uint64_t*)at(W_S1); c->S8[0] = c->S8[1] = nullptr;
    } else {
        c->S8[0] = (int8_t*)at(W_S0); c->S8[1] = (int8_t*)at(W_S1); c->S[0] = c->S[1] = nullptr;
    }
    c->cur = 0;
    c->E32 = kind == PA_PM1 ? (int32_t*)at(W_E32) : nullptr;
    c->E128 = kind == PA_REAL ? (longlong2*)at(W_E128) : nullptr;
    c->parent = (int32_t*)at(W_PARENT);
    c->fam[0] = (int32_t*)at(W_FAM0); c->fam[1] = (int32_t*)at(W_FAM1); c->famcur = 0;
    c->counts = (int32_t*)at(W_COUNTS); c->blocksum = (int32_t*)at(W_BLOCKSUM);
    c->w = (double*)at(W_W); c->P = (double*)at(W_P); c->tot = (double*)at(W_TOT); c->T = (double*)at(W_T);
    c->acc = (StepAcc*)at(W_ACC);
    c->cJ = c->acc_grad ? (unsigned long long*)at(W_CJ) : nullptr;
    c->ch = c->acc_grad ? (unsigned long long*)at(W_CH) : nullptr;
    c->tmp8 = c->layout == PA_LAYOUT_PACKED ? (int8_t*)at(W_TMP8) : nullptr;
    c->hist = (unsigned long long*)at(W_HIST);
    c->gbar_d = c->acc_grad ? (double*)at(W_GBAR) : nullptr;
    c->dJ_d = c->acc_grad ? (double*)at(W_DJ) : nullptr;
    c->dh_d = c->acc_grad ? (double*)at(W_DH) : nullptr;
    c->obspart = (pa::ObsPartial*)at(W_OBSPART);

    // couplings: sign masks (+-J), fixed-point copies (real)
    std::vector<uint8_t> jn(N, 0);
    std::vector<longlong2> jf, hf;
    for (int i = 0; i < N; ++i) {
        int stride = 1;
        for (int d = 0; d < D; ++d) {
            int cc = (i / stride) % L;
            int im = i + (((cc + L - 1) % L) - cc) * stride;
            if (c->Jh[(size_t)d * N + im] < 0.0f) jn[i] |= (uint8_t)(1u << (2 * d));
            if (c->Jh[(size_t)d * N + i] < 0.0f) jn[i] |= (uint8_t)(1u << (2 * d + 1));
            stride *= L;
        }
    }
    if (kind == PA_REAL) {
        jf.resize((size_t)D * N);
        hf.resize(N);
        for (int b = 0; b < D * N; ++b) jf[b] = fix96(c->Jh[b]);
        for (int i = 0; i < N; ++i) hf[i] = fix96(c->hh[i]);
    }
    int rc2 = PA_OK;
    auto up = [&](void* dst, const void* src, size_t n) {
        if (rc2 == PA_OK && n) {
            cudaError_t e = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, c->st);
            if (e != cudaSuccess) { g_create_err = cudaGetErrorString(e); rc2 = PA_ECUDA; }
        }
    };
    up(c->J, c->Jh.data(), sizeof(float) * D * N);
    up(c->h, c->hh.data(), sizeof(float) * N);
    up(c->jneg, jn.data(), N);
    if (kind == PA_REAL) {
        up(c->Jfix, jf.data(), sizeof(longlong2) * D * N);
        up(c->hfix, hf.data(), sizeof(longlong2) * N);
    }
    up(c->betas_d, c->betas.data(), sizeof(double) * n_temps);
    if (rc2 == PA_OK) {
        cudaError_t e = cudaMemsetAsync(c->counts, 0, sizeof(int32_t) * (size_t)R, c->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->acc, 0, sizeof(StepAcc) * n_temps, c->st);
        if (e == cudaSuccess && c->acc_grad) {
            e = cudaMemsetAsync(c->cJ, 0, sizeof(unsigned long long) * (size_t)n_temps * D * N, c->st);
            if (e == cudaSuccess) e = cudaMemsetAsync(c->ch, 0, sizeof(unsigned long long) * (size_t)n_temps * N, c->st);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);  // host vectors above go out of scope
        if (e != cudaSuccess) { g_create_err = cudaGetErrorString(e); rc2 = PA_ECUDA; }
    }
    if (rc2 != PA_OK) {
        if (c->own_ws) cudaFree(c->ws);
        delete c;
        return rc2;
    }
    *out = c;
    return PA_OK;
}

extern "C" int pa_create(pa_ctx** out, int D, int L, int kind, const float* J, const float* h, int R,
                         const double* betas, int n_temps, int n_sweeps, uint64_t seed,
                         const pa_options* opt, void* stream)
{
    return create_impl(out, D, L, kind, J, h, R, betas, n_temps, n_sweeps, seed, opt, stream, nullptr, 0);
}

extern "C" int pa_create_ws(pa_ctx** out, int D, int L, int kind, const float* J, const float* h,
                            int R, const double* betas, int n_temps, int n_sweeps, uint64_t seed,
                            const pa_options* opt, void* stream, void* workspace, size_t workspace_bytes)
{
    if (!workspace) { g_create_err = "workspace is NULL"; return PA_EINVAL; }
    return create_impl(out, D, L, kind, J, h, R, betas, n_temps, n_sweeps, seed, opt, stream,
                       workspace, workspace_bytes);
}

// enqueue step k (no synchronisation)
static int enqueue_step(pa_ctx* c)
{
    const int k = c->k_next;
    if (k >= c->n_temps) { c->err = "schedule finished"; return PA_EDONE; }
    const uint32_t k0 = (uint32_t)c->seed, k1 = (uint32_t)(c->seed >> 32);
    const int N = c->N, R = c->R;
    const double beta = c->betas[k];
    cudaEvent_t ev;
    if (k == 0) {
        ev = phase_begin(c);
        const uint32_t c3 = pa::counter3(pa::STREAM_INIT, c->tag, c->inst);
        if (c->layout == PA_LAYOUT_PACKED)
            PA_CK(c, pa::launch_init_packed(c->S[c->cur], N, c->G, k0, k1, c3, c->st));
        else
            PA_CK(c, pa::launch_init_i8(c->S8[c->cur], N, c->NP, R, k0, k1, c3, c->st));
        iota_kernel<<<(R + 255) / 256, 256, 0, c->st>>>(c->fam[c->famcur], c->parent, R);
        acc0_kernel<<<1, 1, 0, c->st>>>(c->acc, c->betaF0, R);
        PA_CK(c, cudaGetLastError());
        c->launches += 3;
        phase_end(c, PA_PHASE_INIT, ev);
    } else {
        ev = phase_begin(c);
        pa::ResampleArgs ra;
        ra.R = R; ra.kind = c->kind == PA_PM1 ? 0 : 1;
        ra.E32 = c->E32; ra.E128 = c->E128;
        ra.prev = c->acc + (k - 1); ra.cur = c->acc + k;
        ra.w = c->w; ra.P = c->P; ra.tot = c->tot; ra.T = c->T;
        ra.counts = c->counts; ra.blocksum = c->blocksum; ra.parent = c->parent;
        ra.fam_in = c->fam[c->famcur]; ra.fam_out = c->fam[c->famcur ^ 1];
        ra.dbeta = c->betas[k] - c->betas[k - 1];
        ra.log_R = c->log_R; ra.betaF0 = c->betaF0; ra.k = k;
        ra.key0 = k0; ra.key1 = k1; ra.c3 = pa::counter3(pa::STREAM_RES, c->tag, c->inst);
        PA_CK(c, pa::launch_resample(ra, c->st));
        c->launches += 7;
        phase_end(c, PA_PHASE_RESAMPLE, ev);
        c->famcur ^= 1;
    }
    ev = phase_begin(c);
    if (c->kind == PA_PM1) {
        pa::PackedSweepArgs a;
        std::memset(&a, 0, sizeof a);
        a.jneg = c->jneg; a.E = c->E32; a.G = c->G; a.R = R; a.k = k; a.n_sweeps = c->n_sweeps;
        a.key0 = k0; a.key1 = k1; a.c3 = pa::counter3(pa::STREAM_PLANE, c->tag, c->inst);
        for (int cl = 1; cl <= 3; ++cl) {
            const uint64_t thr = pa::threshold_pm(beta, 4 * cl);
            a.thr[cl] = (uint32_t)thr;
            if (thr >= 4294967296ull) a.always |= 1u << cl;
            else if (thr > 0) a.und |= 1u << cl;
        }
        for (int r = 0; r < 10; ++r) {
            a.rk[2 * r] = k0 + (uint32_t)r * 0x9E3779B9u;
            a.rk[2 * r + 1] = k1 + (uint32_t)r * 0xBB67AE85u;
        }
        // class of an uphill lane by its unsatisfied-bond count n: dE = 4D - 4n
        const int cls_n0 = c->D, cls_n1 = c->D - 1, cls_n2 = c->D - 2;  // dE / 4
        for (int b = 0; b < 32; ++b) {
            auto bit = [&](int cl) -> uint32_t {
                if (cl < 1 || cl > 3) return 0u;
                return ((a.thr[cl] >> (31 - b)) & 1u) ? 0xFFFFFFFFu : 0u;
            };
            a.v00[b] = bit(cls_n0);
            a.v01[b] = bit(cls_n1);
            a.v10[b] = bit(cls_n2);
        }
        if (c->layout == PA_LAYOUT_PACKED) {
            // k > 0: the replica gather is fused into the sweep's tile load
            a.Sin = c->S[c->cur];
            if (k > 0) {
                a.parent = c->parent;
                c->cur ^= 1;
            }
            a.S = c->S[c->cur];
        } else {
            a.S8_in = c->S8[c->cur]; a.S8_out = c->S8[c->cur ^ 1];
            a.parent = k > 0 ? c->parent : nullptr; a.NP = c->NP;
            c->cur ^= 1;
        }
        PA_CK(c, pa::launch_sweep_packed(c->D, c->L, a, c->gpb, c->threads, c->st));
    } else {
        pa::RealSweepArgs a;
        a.Sin = c->S8[c->cur]; a.Sout = c->S8[c->cur ^ 1];
        a.parent = k > 0 ? c->parent : nullptr;
        a.J = c->J; a.h = c->h; a.Jfix = c->Jfix; a.hfix = c->hfix; a.E = c->E128;
        a.cJ = c->acc_grad ? c->cJ + (size_t)k * c->D * N : nullptr;
        a.ch = c->acc_grad ? c->ch + (size_t)k * N : nullptr;
        a.R = R; a.NP = c->NP; a.k = k; a.n_sweeps = c->n_sweeps; a.beta = (float)beta;
        a.key0 = k0; a.key1 = k1; a.c3 = pa::counter3(pa::STREAM_WORD, c->tag, c->inst);
        PA_CK(c, pa::launch_sweep_real(c->D, c->L, a, c->real_warps, 0, c->st));
        c->cur ^= 1;
    }
    c->launches += 1;
    phase_end(c, PA_PHASE_SWEEP, ev);
    ev = phase_begin(c);
    pa::ObsArgs oa;
    oa.R = R; oa.kind = c->kind == PA_PM1 ? 0 : 1; oa.E32 = c->E32; oa.E128 = c->E128;
    oa.family = c->fam[c->famcur]; oa.part = c->obspart; oa.cur = c->acc + k;
    PA_CK(c, pa::launch_observe(oa, c->st));
    c->launches += 2;
    phase_end(c, PA_PHASE_OBSERVE, ev);
    c->k_next = k + 1;
    return PA_OK;
}

extern "C" int pa_anneal_step(pa_ctx* c)
{
    if (!c) return PA_EINVAL;
    return enqueue_step(c);
}

extern "C" int pa_anneal(pa_ctx* c, int n_steps)
{
    if (!c) return PA_EINVAL;
    if (c->k_next >= c->n_temps) { c->err = "schedule finished"; return PA_EDONE; }
    int n = (n_steps < 0) ? c->n_temps - c->k_next : n_steps;
    if (n == 0) return PA_OK;
    if (c->k_next + n > c->n_temps) { c->err = "n_steps past the end of the schedule"; return PA_EINVAL; }
    if (c->gexec) {
        PA_CK(c, cudaStreamSynchronize(c->st));
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    if (!c->st) {
        // capture needs a non-legacy stream: run eagerly instead
        for (int t = 0; t < n; ++t) {
            int rc = enqueue_step(c);
            if (rc) return rc;
        }
        return PA_OK;
    }
    const int k_save = c->k_next, cur_save = c->cur, fam_save = c->famcur;
    const long long launches_save = c->launches;
    PA_CK(c, cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    int rc = PA_OK;
    for (int t = 0; t < n && rc == PA_OK; ++t) rc = enqueue_step(c);
    c->capturing = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->st, &g);
    if (rc != PA_OK || e != cudaSuccess) c->launches = launches_save;
    if (rc != PA_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        c->k_next = k_save; c->cur = cur_save; c->famcur = fam_save;
        if (rc == PA_OK) { c->err = std::string("stream capture: ") + cudaGetErrorString(e); rc = PA_ECUDA; }
        return rc;
    }
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->k_next = k_save; c->cur = cur_save; c->famcur = fam_save;
        c->gexec = nullptr;
        c->err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
        return PA_ECUDA;
    }
    PA_CK(c, cudaGraphLaunch(c->gexec, c->st));
    return PA_OK;
}

extern "C" int pa_current_step(const pa_ctx* c) { return c ? c->k_next : PA_EINVAL; }

extern "C" int pa_synchronize(pa_ctx* c)
{
    if (!c) return PA_EINVAL;
    PA_CK(c, cudaStreamSynchronize(c->st));
    return PA_OK;
}

extern "C" int pa_observables(pa_ctx* c, int k, pa_obs* out)
{
    if (!c || !out) return PA_EINVAL;
    if (k < 0 || k >= c->k_next) { c->err = "step not run yet"; return PA_ESTATE; }
    StepAcc a;
    PA_CK(c, cudaMemcpyAsync(&a, c->acc + k, sizeof a, cudaMemcpyDeviceToHost, c->st));
    PA_CK(c, cudaStreamSynchronize(c->st));
    const double R = (double)c->R;
    double Em, E2m;
    if (c->kind == PA_PM1) {
        Em = (double)a.sumE / R;
        E2m = (double)a.sumE2 / R;
    } else {
        Em = a.sumEd / R;
        E2m = a.sumE2d / R;
    }
    const double beta = c->betas[k];
    out->E_mean = Em;
    out->E2_mean = E2m;
    out->C = beta * beta * (E2m - Em * Em) / c->N;
    out->lnQ = a.lnQ;
    out->betaF = a.betaF;
    out->S_f = c->log_R - a.sum_clnc / R;
    out->rho_s = R / std::exp(out->S_f);
    out->R = c->R;
    return PA_OK;
}

extern "C" int pa_free_energy(pa_ctx* c, double* betaF)
{
    if (!c || !betaF) return PA_EINVAL;
    std::vector<StepAcc> a(c->n_temps);
    PA_CK(c, cudaMemcpyAsync(a.data(), c->acc, sizeof(StepAcc) * c->n_temps, cudaMemcpyDeviceToHost, c->st));
    PA_CK(c, cudaStreamSynchronize(c->st));
    for (int k = 0; k < c->n_temps; ++k) betaF[k] = k < c->k_next ? a[k].betaF : NAN;
    return PA_OK;
}

extern "C" int pa_grad(pa_ctx* c, const double* gbar, double* dJ, double* dh)
{
    if (!c || !gbar || !dJ) return PA_EINVAL;
    if (!c->acc_grad) { c->err = "context created without accumulate_grad"; return PA_ESTATE; }
    for (int k = c->k_next; k < c->n_temps; ++k)
        if (gbar[k] != 0.0) { c->err = "gbar weights a step that has not run"; return PA_ESTATE; }
    const int nJ = c->D * c->N;
    PA_CK(c, cudaMemcpyAsync(c->gbar_d, gbar, sizeof(double) * c->n_temps, cudaMemcpyHostToDevice, c->st));
    PA_CK(c, pa::launch_grad_backward(c->cJ, c->ch, c->gbar_d, c->betas_d, c->n_temps, nJ, c->N, c->R,
                                      c->dJ_d, c->dh_d, c->st));
    PA_CK(c, cudaMemcpyAsync(dJ, c->dJ_d, sizeof(double) * nJ, cudaMemcpyDeviceToHost, c->st));
    if (dh) PA_CK(c, cudaMemcpyAsync(dh, c->dh_d, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->st));
    PA_CK(c, cudaStreamSynchronize(c->st));
    return PA_OK;
}

extern "C" int pa_overlap(pa_ctx* a, pa_ctx* b, int64_t* hist)
{
    if (!a || !b || !hist) return PA_EINVAL;
    if (a->D != b->D || a->L != b->L || a->R != b->R || a->layout != b->layout) {
        a->err = "overlap needs two contexts of the same lattice, R and layout";
        return PA_EINVAL;
    }
    PA_CK(a, cudaStreamSynchronize(b->st));
    PA_CK(a, cudaMemsetAsync(a->hist, 0, sizeof(unsigned long long) * (a->N + 1), a->st));
    if (a->layout == PA_LAYOUT_PACKED)
        PA_CK(a, pa::launch_overlap_packed(a->S[a->cur], b->S[b->cur], a->N, a->R, a->hist, a->st));
    else
        PA_CK(a, pa::launch_overlap_i8(a->S8[a->cur], b->S8[b->cur], a->N, a->NP, a->R, a->hist, a->st));
    PA_CK(a, cudaMemcpyAsync(hist, a->hist, sizeof(int64_t) * (a->N + 1), cudaMemcpyDeviceToHost, a->st));
    PA_CK(a, cudaStreamSynchronize(a->st));
    return PA_OK;
}

extern "C" int pa_get_spins_range(pa_ctx* c, int r0, int n, int8_t* dst)
{
    if (!c || !dst || r0 < 0 || n < 0 || r0 + n > c->R) return PA_EINVAL;
    if (n == 0) return PA_OK;
    if (c->layout == PA_LAYOUT_PACKED) {
        PA_CK(c, pa::launch_unpack_packed(c->S[c->cur], c->tmp8, c->N, r0, n, c->st));
        PA_CK(c, cudaMemcpyAsync(dst, c->tmp8, (size_t)n * c->N, cudaMemcpyDeviceToHost, c->st));
    } else {
        PA_CK(c, cudaMemcpy2DAsync(dst, c->N, c->S8[c->cur] + (size_t)r0 * c->NP, c->NP, c->N, n,
                                   cudaMemcpyDeviceToHost, c->st));
    }
    PA_CK(c, cudaStreamSynchronize(c->st));
    return PA_OK;
}

extern "C" int pa_get_spins(pa_ctx* c, int8_t* dst)
{
    if (!c) return PA_EINVAL;
    return pa_get_spins_range(c, 0, c->R, dst);
}

extern "C" int pa_get_energies(pa_ctx* c, int64_t* dst)
{
    if (!c || !dst) return PA_EINVAL;
    if (c->kind == PA_PM1) {
        std::vector<int32_t> e(c->R);
        PA_CK(c, cudaMemcpyAsync(e.data(), c->E32, sizeof(int32_t) * c->R, cudaMemcpyDeviceToHost, c->st));
        PA_CK(c, cudaStreamSynchronize(c->st));
        for (int r = 0; r < c->R; ++r) dst[r] = e[r];
    } else {
        PA_CK(c, cudaMemcpyAsync(dst, c->E128, sizeof(longlong2) * c->R, cudaMemcpyDeviceToHost, c->st));
        PA_CK(c, cudaStreamSynchronize(c->st));
    }
    return PA_OK;
}

extern "C" int pa_get_parents(pa_ctx* c, int32_t* dst)
{
    if (!c || !dst) return PA_EINVAL;
    PA_CK(c, cudaMemcpyAsync(dst, c->parent, sizeof(int32_t) * c->R, cudaMemcpyDeviceToHost, c->st));
    PA_CK(c, cudaStreamSynchronize(c->st));
    return PA_OK;
}

extern "C" int pa_get_family(pa_ctx* c, int32_t* dst)
{
    if (!c || !dst) return PA_EINVAL;
    PA_CK(c, cudaMemcpyAsync(dst, c->fam[c->famcur], sizeof(int32_t) * c->R, cudaMemcpyDeviceToHost, c->st));
    PA_CK(c, cudaStreamSynchronize(c->st));
    return PA_OK;
}

extern "C" int pa_get_grad_counts(pa_ctx* c, int64_t* cJ, int64_t* ch)
{
    if (!c || !cJ || !ch) return PA_EINVAL;
    if (!c->acc_grad) { c->err = "context created without accumulate_grad"; return PA_ESTATE; }
    PA_CK(c, cudaMemcpyAsync(cJ, c->cJ, sizeof(int64_t) * (size_t)c->n_temps * c->D * c->N, cudaMemcpyDeviceToHost, c->st));
    PA_CK(c, cudaMemcpyAsync(ch, c->ch, sizeof(int64_t) * (size_t)c->n_temps * c->N, cudaMemcpyDeviceToHost, c->st));
    PA_CK(c, cudaStreamSynchronize(c->st));
    return PA_OK;
}

extern "C" int pa_sizes(const pa_ctx* c, int* D, int* L, int* N, int* R, int* n_temps, int* layout)
{
    if (!c) return PA_EINVAL;
    if (D) *D = c->D;
    if (L) *L = c->L;
    if (N) *N = c->N;
    if (R) *R = c->R;
    if (n_temps) *n_temps = c->n_temps;
    if (layout) *layout = c->layout;
    return PA_OK;
}

extern "C" int pa_profile(pa_ctx* c, int enable)
{
    if (!c) return PA_EINVAL;
    c->profiling = enable ? 1 : 0;
    return PA_OK;
}

extern "C" int pa_phase_times(pa_ctx* c, double* ms, int64_t* n, int64_t* launches)
{
    if (!c) return PA_EINVAL;
    PA_CK(c, cudaStreamSynchronize(c->st));
    double acc[PA_NPHASE] = {0};
    int64_t cnt[PA_NPHASE] = {0};
    for (auto& pe : c->ev_pending) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, pe.second.first, pe.second.second) == cudaSuccess) {
            acc[pe.first] += t;
            cnt[pe.first] += 1;
        }
        c->ev_free.push_back(pe.second.first);
        c->ev_free.push_back(pe.second.second);
    }
    c->ev_pending.clear();
    for (int p = 0; p < PA_NPHASE; ++p) {
        if (ms) ms[p] = acc[p];
        if (n) n[p] = cnt[p];
    }
    if (launches) *launches = c->launches;
    return PA_OK;
}

extern "C" const char* pa_last_error(const pa_ctx* c)
{
    return c ? c->err.c_str() : g_create_err.c_str();
}

extern "C" void pa_destroy(pa_ctx* c)
{
    if (!c) return;
    cudaStreamSynchronize(c->st);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    for (auto& pe : c->ev_pending) {
        cudaEventDestroy(pe.second.first);
        cudaEventDestroy(pe.second.second);
    }
    for (auto e : c->ev_free) cudaEventDestroy(e);
    if (c->own_ws) cudaFree(c->ws);
    delete c;
}
