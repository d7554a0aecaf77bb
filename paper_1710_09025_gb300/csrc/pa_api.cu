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

#include <nvtx3/nvToolsExt.h>

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
    int sep_gather;             // the replica gather as its own launch before the sweeps
    int shard_off, shard_total; // a shard: global replicas [shard_off, shard_off + R) of shard_total
    int shard_copies;           // copies placed by the last pa_shard_draw
    cudaStream_t st;
    int gpb, threads, real_warps;
    int band;                   // real couplings: acceptance guard band verified on this device
    double betaF0, log_R;
    std::vector<double> betas;
    std::vector<int> Rk;        // population (target) at each temperature; R = capacity
    int scheme;                 // PA_RESAMPLE_*; nearest-integer: populations in Rdev
    int icm;                    // isoenergetic cluster moves and their beta window
    double icm_lo, icm_hi;
    int* icm_err;               // device flag: a bounded union-find loop gave up
    double* wtab;               // +-J: resampling weight per energy level
    int* sync;                  // block counters of the merged launches (zeroed)
    int* Rdev;                  // [n_temps] populations in device memory
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
    double *w, *P, *lev1, *bmax, *upper;
    double *sh_upper, *sh_t2g, *sh_bmax;  // a shard: global prefix levels, block totals, maxima
    int32_t *sh_pout, *sh_fout;           // a shard: parents and families of its outgoing copies
    uint64_t* sh_stage;                   // a shard: incoming replica groups
    StepAcc* acc;
    unsigned long long *cJ, *ch;
    int8_t* tmp8;
    unsigned long long* hist;
    double *gbar_d, *dJ_d, *dh_d;
    pa::ObsPartial* obspart;
    double* logc;               // log(c) table of the family entropy
    double* Rk_d;               // populations as doubles (gradient normalisation)
    cudaGraphExec_t gexec;
    std::string err;
    // profiling: event pairs per phase, launch counter
    int profiling;
    bool capturing;
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
    long long launches;
};

// NVTX range names of the phases (host-side ranges around each phase's
// launches, for timeline and kernel-filter tools; no-ops without a tool)
static const char* const kPhaseName[PA_NPHASE] = {"pa/init", "pa/resample", "pa/gather", "pa/sweep",
                                                   "pa/observe"};

// records the start of a phase; returns the start event (or null)
static cudaEvent_t phase_begin(pa_ctx* c, int phase)
{
    nvtxRangePushA(kPhaseName[phase]);
    if (!c->profiling || c->capturing) return nullptr;
    cudaEvent_t e;
    if (!c->ev_free.empty()) { e = c->ev_free.back(); c->ev_free.pop_back(); }
    else if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    cudaEventRecord(e, c->st);
    return e;
}

static void phase_end(pa_ctx* c, int phase, cudaEvent_t start)
{
    nvtxRangePop();
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

// a[i] = off + i (families: the global index of the initial replica), b[i] = i
__global__ void iota_kernel(int32_t* a, int32_t* b, int n, int off)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        a[i] = off + i;
        if (b) b[i] = i;
    }
}

__global__ void acc0_kernel(StepAcc* acc, double betaF0, int R, int* Rdev)
{
    *Rdev = R;
    acc->lnQ = 0.0;
    acc->sum_lnQ = 0.0;
    acc->betaF = betaF0;
    acc->S = (double)R;
}

// ---------------- workspace layout ----------------

enum {
    W_J, W_H, W_JNEG, W_JFIX, W_HFIX, W_BETAS, W_S0, W_S1, W_E32, W_E128, W_PARENT, W_FAM0, W_FAM1,
    W_COUNTS, W_BLOCKSUM, W_W, W_P, W_LEV1, W_BMAX, W_UPPER, W_ACC, W_CJ, W_CH, W_TMP8, W_HIST, W_GBAR, W_DJ,
    W_DH, W_OBSPART, W_RK, W_RDEV, W_ICMERR, W_WTAB, W_SYNC, W_LOGC,
    W_SH_UPPER, W_SH_T2G, W_SH_BMAX, W_SH_POUT, W_SH_FOUT, W_SH_STAGE, W_COUNT
};

struct Layout {
    size_t off[W_COUNT];  // byte offset of every buffer in the workspace
    size_t total;
};

// incoming replica groups of a shard beyond its own groups: one partial group
// per sending shard (at most this many shards)
constexpr int kShardStageExtra = 64;

// shard_total > 0: the context is a shard of a population of shard_total
// replicas (global prefix levels, outgoing copies, incoming replica groups)
static Layout make_layout(int D, int L, int kind, int layout, int R, int n_temps, int acc_grad,
                          int shard_total = 0)
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
    sz[W_LEV1] = sizeof(double) * (size_t)pa::rs_leaves(R);
    sz[W_BMAX] = sizeof(double) * 2 * (size_t)pa::rs_wblocks(R);
    sz[W_UPPER] = sizeof(double) * (size_t)pa::rs_upper_size(R);
    sz[W_ACC] = sizeof(StepAcc) * n_temps;
    sz[W_CJ] = acc_grad ? sizeof(unsigned long long) * (size_t)n_temps * D * N : 0;
    sz[W_CH] = acc_grad ? sizeof(unsigned long long) * (size_t)n_temps * N : 0;
    sz[W_TMP8] = layout == PA_LAYOUT_PACKED ? (size_t)R * N : 0;
    sz[W_HIST] = sizeof(unsigned long long) * (N + 1);
    sz[W_GBAR] = acc_grad ? sizeof(double) * n_temps : 0;
    sz[W_DJ] = acc_grad ? sizeof(double) * D * N : 0;
    sz[W_DH] = acc_grad ? sizeof(double) * N : 0;
    sz[W_OBSPART] = sizeof(pa::ObsPartial) * pa::kObsBlocks;
    sz[W_LOGC] = sizeof(double) * pa::kLogC;
    sz[W_RK] = sizeof(double) * n_temps;
    sz[W_RDEV] = sizeof(int) * n_temps;
    sz[W_ICMERR] = sizeof(int);
    sz[W_SYNC] = sizeof(int) * 4;
    sz[W_WTAB] = kind == PA_PM1 ? sizeof(double) * (size_t)(D * N / 2 + 1) : 0;
    if (shard_total > 0) {
        sz[W_SH_UPPER] = sizeof(double) * (size_t)pa::rs_upper_size(shard_total);
        sz[W_SH_T2G] = sizeof(double) * (size_t)pa::rs_wblocks(shard_total);
        sz[W_SH_BMAX] = sizeof(double) * 2 * (size_t)pa::rs_wblocks(shard_total);
        sz[W_SH_POUT] = sizeof(int32_t) * (size_t)shard_total;
        sz[W_SH_FOUT] = sizeof(int32_t) * (size_t)shard_total;
        sz[W_SH_STAGE] = sizeof(uint64_t) * (size_t)(G + kShardStageExtra) * N;  // incoming replica groups
    }
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

// replica slots: the multinomial scheme draws exact populations (at most
// max(R, capacity)); the nearest-integer scheme fluctuates around its targets
// (the largest target T, default capacity T + 64 + 8 ceil(sqrt T))
static long long capacity_of(int R, int n_temps, const pa_options* o)
{
    const int scheme = o ? o->resampling : PA_RESAMPLE_MULTINOMIAL;
    const int given = o ? o->capacity : 0;
    if (scheme == PA_RESAMPLE_MULTINOMIAL) return given > R ? given : R;
    long long tmax = R;
    if (o && o->populations) {
        tmax = 0;
        for (int k = 0; k < n_temps; ++k) tmax = std::max<long long>(tmax, o->populations[k]);
    }
    if (given > 0) return given;
    return tmax + 64 + 8 * (long long)std::ceil(std::sqrt((double)tmax));
}

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
    if (!sup) { err = "lattice size not compiled in (3D: even L in 2..16, real couplings 2..12; 2D: up to 32/64)"; return PA_EINVAL; }
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
        if (o->rng_instance >= (1u << 24)) { err = "rng_instance must be < 2^24"; return PA_EINVAL; }
        if (o->rng_tag >= 16u) { err = "rng_tag must be < 16"; return PA_EINVAL; }
        if (o->resampling != PA_RESAMPLE_MULTINOMIAL && o->resampling != PA_RESAMPLE_NEAREST) {
            err = "resampling must be PA_RESAMPLE_MULTINOMIAL or PA_RESAMPLE_NEAREST";
            return PA_EINVAL;
        }
        if (o->capacity < 0) { err = "capacity must be >= 0"; return PA_EINVAL; }
        if (o->icm) {
            if (h)
                for (int i = 0; i < N; ++i)
                    if (h[i] != 0.0f) { err = "cluster moves (icm) need a zero field"; return PA_EINVAL; }
            if (!std::isfinite(o->icm_beta_lo) || !std::isfinite(o->icm_beta_hi)) {
                err = "icm beta window must be finite";
                return PA_EINVAL;
            }
            if (N > 4096) { err = "cluster moves support N <= 4096"; return PA_EINVAL; }
        }
        if (o->shard_total > 0) {
            if (kind != PA_PM1 || lay != PA_LAYOUT_PACKED) { err = "shards need +-J couplings in the packed layout"; return PA_EINVAL; }
            if (o->shard_offset < 0 || o->shard_offset % pa::kWBlock != 0 ||
                (long long)o->shard_offset + R > o->shard_total || o->shard_total > (1 << 26)) {
                err = "shard: offset a multiple of 1024, offset + R <= shard_total <= 2^26";
                return PA_EINVAL;
            }
            if (o->populations || o->resampling || o->icm || o->accumulate_grad || o->separate_gather || o->capacity ||
                o->threads || o->groups_per_block) {
                err = "shard: fixed population, multinomial resampling, default tile; no cluster moves, gradient "
                      "counts or separate gather";
                return PA_EINVAL;
            }
        } else if (o->shard_total < 0 || o->shard_offset != 0) {
            err = "shard_offset needs shard_total > 0";
            return PA_EINVAL;
        }
        const long long cap = capacity_of(R, n_temps, o);
        if (cap > (1 << 26)) { err = "capacity must be <= 2^26"; return PA_EINVAL; }
        if (o->resampling == PA_RESAMPLE_NEAREST && !o->populations && cap < R) {
            err = "capacity below the population R";
            return PA_EINVAL;
        }
        if (o->populations)
            for (int k = 0; k < n_temps; ++k)
                if (o->populations[k] < 1 || o->populations[k] > cap) {
                    err = "populations[k] must be in [1, capacity]";
                    return PA_EINVAL;
                }
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
    const long long cap = capacity_of(R, n_temps, opt);
    if (cap > (1 << 26)) return PA_EINVAL;
    Layout l = make_layout(D, L, kind, lay, (int)cap, n_temps, opt ? opt->accumulate_grad : 0,
                           opt ? opt->shard_total : 0);
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
    const int cap = (int)capacity_of(R, n_temps, &o);
    c->D = D; c->L = L; c->N = (D == 3) ? L * L * L : L * L; c->kind = kind; c->R = cap;
    c->G = (cap + 63) / 64; c->scheme = o.resampling;
    c->icm = o.icm ? 1 : 0; c->icm_lo = o.icm_beta_lo; c->icm_hi = o.icm_beta_hi; c->n_temps = n_temps; c->n_sweeps = n_sweeps; c->k_next = 0;
    c->layout = resolve_layout(kind, &o); c->NP = (c->N + 15) / 16 * 16;
    c->seed = seed; c->inst = o.rng_instance; c->tag = o.rng_tag; c->acc_grad = o.accumulate_grad ? 1 : 0;
    c->sep_gather = o.separate_gather ? 1 : 0;
    c->shard_off = o.shard_total > 0 ? o.shard_offset : 0;
    c->shard_total = o.shard_total > 0 ? o.shard_total : 0;
    c->shard_copies = 0;
    c->st = (cudaStream_t)stream;
    c->betas.assign(betas, betas + n_temps);
    c->Rk.assign(n_temps, R);
    if (o.populations) c->Rk.assign(o.populations, o.populations + n_temps);
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

    Layout lay = make_layout(D, L, kind, c->layout, cap, n_temps, c->acc_grad, c->shard_total);
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
    c->w = (double*)at(W_W); c->P = (double*)at(W_P);
    c->lev1 = (double*)at(W_LEV1); c->bmax = (double*)at(W_BMAX); c->upper = (double*)at(W_UPPER);
    c->acc = (StepAcc*)at(W_ACC);
    c->cJ = c->acc_grad ? (unsigned long long*)at(W_CJ) : nullptr;
    c->ch = c->acc_grad ? (unsigned long long*)at(W_CH) : nullptr;
    c->tmp8 = c->layout == PA_LAYOUT_PACKED ? (int8_t*)at(W_TMP8) : nullptr;
    c->hist = (unsigned long long*)at(W_HIST);
    c->gbar_d = c->acc_grad ? (double*)at(W_GBAR) : nullptr;
    c->dJ_d = c->acc_grad ? (double*)at(W_DJ) : nullptr;
    c->dh_d = c->acc_grad ? (double*)at(W_DH) : nullptr;
    c->obspart = (pa::ObsPartial*)at(W_OBSPART);
    c->logc = (double*)at(W_LOGC);
    c->Rk_d = (double*)at(W_RK);
    c->Rdev = (int*)at(W_RDEV);
    c->icm_err = (int*)at(W_ICMERR);
    c->sync = (int*)at(W_SYNC);
    c->sh_upper = (double*)at(W_SH_UPPER); c->sh_t2g = (double*)at(W_SH_T2G); c->sh_bmax = (double*)at(W_SH_BMAX);
    c->sh_pout = (int32_t*)at(W_SH_POUT); c->sh_fout = (int32_t*)at(W_SH_FOUT);
    c->sh_stage = (uint64_t*)at(W_SH_STAGE);
    c->wtab = kind == PA_PM1 ? (double*)at(W_WTAB) : nullptr;

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
    std::vector<double> rkd(c->Rk.begin(), c->Rk.end());
    up(c->Rk_d, rkd.data(), sizeof(double) * n_temps);
    if (rc2 == PA_OK) {
        cudaError_t e = cudaMemsetAsync(c->counts, 0, sizeof(int32_t) * (size_t)R, c->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->acc, 0, sizeof(StepAcc) * n_temps, c->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->icm_err, 0, sizeof(int), c->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->sync, 0, sizeof(int) * 4, c->st);
        if (e == cudaSuccess) e = pa::launch_logc_table(c->logc, c->st);
        if (e == cudaSuccess && c->acc_grad) {
            e = cudaMemsetAsync(c->cJ, 0, sizeof(unsigned long long) * (size_t)n_temps * D * N, c->st);
            if (e == cudaSuccess) e = cudaMemsetAsync(c->ch, 0, sizeof(unsigned long long) * (size_t)n_temps * N, c->st);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);  // host vectors above go out of scope
        if (e != cudaSuccess) { g_create_err = cudaGetErrorString(e); rc2 = PA_ECUDA; }
    }
    c->band = (rc2 == PA_OK && kind == PA_REAL && !o.exact_accept) ? pa::accept_band_ok(c->st) : 0;
    if (rc2 != PA_OK) {
        if (c->own_ws) cudaFree(c->ws);
        delete c;
        return rc2;
    }
    *out = c;
    return PA_OK;
}

extern "C" int pa_check_accept_band(int64_t* violations, double* max_rel_dev)
{
    unsigned long long v = 0;
    double d = 0.0;
    cudaError_t e = pa::accept_band_check(nullptr, &v, &d);
    if (e != cudaSuccess) {
        pa::set_global_error(cudaGetErrorString(e));
        return PA_ECUDA;
    }
    if (violations) *violations = (int64_t)v;
    if (max_rel_dev) *max_rel_dev = d;
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

// Per-temperature parameters of the +-J sweep: Metropolis thresholds of the
// uphill classes dE = 4c as plane masks, and the Philox round keys.
static void fill_round_keys(uint32_t* rk, uint32_t k0, uint32_t k1)
{
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = k0 + (uint32_t)r * 0x9E3779B9u;
        rk[2 * r + 1] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
}

static void fill_packed_step(pa::PackedStep* s, int D, double beta, int k, int n_sweeps,
                             uint32_t k0, uint32_t k1)
{
    std::memset(s, 0, sizeof *s);
    s->k = k;
    s->n_sweeps = n_sweeps;
    s->hs0 = 2u * (uint32_t)(k * n_sweeps);
    uint32_t thr[4] = {0, 0, 0, 0};
    for (int cl = 1; cl <= 3; ++cl) {
        const uint64_t t = pa::threshold_pm(beta, 4 * cl);
        thr[cl] = (uint32_t)t;
        if (t >= 4294967296ull) s->always |= 1u << cl;
        else if (t > 0) s->und |= 1u << cl;
    }
    // undecided class sets with a cheaper comparison loop (thresholds fall with
    // dE, so classes never accepted are the large-dE ones)
    if (s->always == 0 && s->und == 2u) s->mode = 1;
    else if (s->always == 0 && s->und == 6u) s->mode = 2;
    else if (D == 3 && s->always == 0 && s->und == 14u) s->mode = 3;  // every uphill class undecided
    else s->mode = 0;
    fill_round_keys(s->rk, k0, k1);
    // class of an uphill lane by its unsatisfied-bond count n: dE / 4 = D - n
    const int cls_n0 = D, cls_n1 = D - 1, cls_n2 = D - 2;
    for (int b = 0; b < 32; ++b) {
        auto bit = [&](int cl) -> uint32_t {
            if (cl < 1 || cl > 3) return 0u;
            return ((thr[cl] >> (31 - b)) & 1u) ? 0xFFFFFFFFu : 0u;
        };
        s->v00[b] = bit(cls_n0);
        s->v01[b] = bit(cls_n1);
        s->v10[b] = bit(cls_n2);
        if ((s->v00[b] | s->v01[b] | s->v10[b]) == 0) s->zero_planes |= 1u << b;
    }
}

// Everything one anneal step launches, with the context's ping-pong state
// advanced to after the step.
struct StepPlan {
    int k;
    pa::ResampleArgs rs;       // k > 0
    pa::PackedSweepArgs pk;    // PA_PM1
    pa::RealSweepArgs re;      // PA_REAL
    // cluster moves: pk / re run the first N_S/2 sweeps, then two rounds of
    // moves, then pk2 / re2 the remaining sweeps (no gather, in place)
    bool icm;
    pa::IcmArgs ic;
    pa::PackedSweepArgs pk2;
    pa::RealSweepArgs re2;
    pa::ObsArgs ob;
    // separate_gather (k > 0): the gather launch, then the sweeps in place
    bool gather;
    const uint64_t* g_Sin;
    uint64_t* g_Sout;
    const int8_t* g_S8in;
    int8_t* g_S8out;
    // +-J gradient counts of the population after the sweeps
    bool grad_pm;
    // context state after the step
    int cur, famcur;
};

static void plan_step(pa_ctx* c, StepPlan* pl)
{
    const int k = c->k_next;
    const uint32_t k0 = (uint32_t)c->seed, k1 = (uint32_t)(c->seed >> 32);
    const int R = c->Rk[k];                      // population after this step
    const int G = (R + 63) / 64;
    const double beta = c->betas[k];
    std::memset(pl, 0, sizeof *pl);
    pl->k = k;
    // nearest-integer scheme: every kernel reads the population from Rdev and
    // the grids cover the capacity
    const bool dyn = c->scheme == PA_RESAMPLE_NEAREST;
    if (k > 0) {
        pa::ResampleArgs& ra = pl->rs;
        const int Rprev = c->Rk[k - 1];
        ra.R = Rprev; ra.Rn = R; ra.kind = c->kind == PA_PM1 ? 0 : 1;
        if (dyn) {
            ra.R = c->R; ra.Rn = 0;
            ra.scheme = 1; ra.cap = c->R; ra.target = (double)c->Rk[k];
            ra.Rsrc = c->Rdev + (k - 1); ra.Rdst = c->Rdev + k; ra.Rdst_d = c->Rk_d + k;
        }
        ra.E32 = c->E32; ra.E128 = c->E128;
        ra.prev = c->acc + (k - 1); ra.cur = c->acc + k;
        ra.w = c->w; ra.P = c->P; ra.lev1 = c->lev1; ra.bmax = c->bmax; ra.upper = c->upper;
        ra.counts = c->counts; ra.blocksum = c->blocksum; ra.parent = c->parent;
        ra.fam_in = c->fam[c->famcur]; ra.fam_out = c->fam[c->famcur ^ 1];
        ra.dbeta = c->betas[k] - c->betas[k - 1];
        ra.log_R = std::log((double)Rprev); ra.betaF0 = c->betaF0; ra.k = k;
        ra.wtab = c->wtab; ra.wtab_n = c->wtab ? c->D * c->N / 2 + 1 : 0;  // E - E_min <= 2 D N
        ra.sync = c->sync;
        ra.key0 = k0; ra.key1 = k1; ra.c3 = pa::counter3(pa::STREAM_RES, c->tag, c->inst);
        c->famcur ^= 1;
    }
    const bool icm = c->icm && k > 0 && beta >= c->icm_lo && (c->icm_hi <= 0.0 || beta <= c->icm_hi);
    const int h1 = c->n_sweeps / 2;
    pl->icm = icm;
    if (c->kind == PA_PM1) {
        fill_packed_step(&pl->pk.s, c->D, beta, k, c->n_sweeps, k0, k1);
        if (icm) pl->pk.s.n_sweeps = h1;
        pa::PackedInst& in = pl->pk.i;
        in.jneg = c->jneg; in.E = c->E32; in.G = G; in.R = R; in.NP = c->NP;
        if (dyn) { in.Rdev = c->Rdev + k; in.G = c->G; in.R = c->R; }
        in.c3 = pa::counter3(pa::STREAM_PLANE, c->tag, c->inst);
        in.goff = c->shard_off / 64;  // a shard's groups carry their global index
        if (c->layout == PA_LAYOUT_PACKED) {
            // k > 0: the replica gather is fused into the sweep's tile load
            in.Sin = c->S[c->cur];
            if (k > 0) {
                in.parent = c->parent;
                c->cur ^= 1;
            }
            in.S = c->S[c->cur];
        } else {
            in.S8_in = c->S8[c->cur]; in.S8_out = c->S8[c->cur ^ 1];
            in.parent = k > 0 ? c->parent : nullptr;
            c->cur ^= 1;
        }
        if (icm) {
            pl->pk2 = pl->pk;
            pl->pk2.s.n_sweeps = c->n_sweeps - h1;
            pl->pk2.s.hs0 = 2u * (uint32_t)(k * c->n_sweeps + h1);
            pa::PackedInst& i2 = pl->pk2.i;
            i2.parent = nullptr;
            if (c->layout == PA_LAYOUT_PACKED) {
                i2.Sin = c->S[c->cur]; i2.S = c->S[c->cur];  // in place
            } else {
                i2.S8_in = c->S8[c->cur]; i2.S8_out = c->S8[c->cur ^ 1];
            }
        }
    } else {
        pa::RealStep& st = pl->re.s;
        st.k = k; st.n_sweeps = icm ? h1 : c->n_sweeps; st.beta = (float)beta; st.key0 = k0; st.key1 = k1;
        st.band = c->band;
        fill_round_keys(st.rk, k0, k1);
        st.hs0 = 2u * (uint32_t)(k * c->n_sweeps);
        pa::RealInst& in = pl->re.i;
        in.Sin = c->S8[c->cur]; in.Sout = c->S8[c->cur ^ 1];
        in.parent = k > 0 ? c->parent : nullptr;
        in.J = c->J; in.h = c->h; in.Jfix = c->Jfix; in.hfix = c->hfix; in.E = c->E128;
        in.cJ = c->acc_grad ? c->cJ + (size_t)k * c->D * c->N : nullptr;
        in.ch = c->acc_grad ? c->ch + (size_t)k * c->N : nullptr;
        in.R = R; in.NP = c->NP; in.c3 = pa::counter3(pa::STREAM_WORD, c->tag, c->inst);
        if (dyn) { in.Rdev = c->Rdev + k; in.R = c->R; }
        c->cur ^= 1;
        if (icm) {
            pl->re2 = pl->re;
            pl->re2.s.n_sweeps = c->n_sweeps - h1;
            pl->re2.s.hs0 = 2u * (uint32_t)(k * c->n_sweeps + h1);
            in.cJ = nullptr; in.ch = nullptr;  // counts after the last sweep only
            pa::RealInst& i2 = pl->re2.i;
            i2.parent = nullptr;
            i2.Sin = c->S8[c->cur]; i2.Sout = c->S8[c->cur ^ 1];
        }
    }
    if (icm) {
        pa::IcmArgs& ic = pl->ic;
        ic.D = c->D; ic.L = c->L; ic.N = c->N; ic.NP = c->NP;
        if (c->layout == PA_LAYOUT_PACKED) { ic.S = c->S[c->cur]; ic.S8 = nullptr; }
        else { ic.S = nullptr; ic.S8 = c->S8[c->cur]; }
        ic.Rdev = dyn ? c->Rdev + k : nullptr;
        ic.R = dyn ? c->R : R;
        ic.k = k; ic.t = 0;
        ic.key0 = k0; ic.key1 = k1; ic.c3 = pa::counter3(pa::STREAM_ICM, c->tag, c->inst);
        ic.err = c->icm_err;
        if (c->layout != PA_LAYOUT_PACKED || c->kind == PA_REAL) c->cur ^= 1;  // the second sweep launch ping-pongs
    }
    if (c->sep_gather && k > 0) {
        // the gather the first sweep launch would fuse runs as its own launch
        // into the buffer that launch writes; that launch then sweeps in place
        pl->gather = true;
        if (c->kind == PA_PM1) {
            pa::PackedInst& in = pl->pk.i;
            if (c->layout == PA_LAYOUT_PACKED) {
                pl->g_Sin = in.Sin; pl->g_Sout = in.S;
                in.Sin = in.S;
            } else {
                pl->g_S8in = in.S8_in; pl->g_S8out = in.S8_out;
                in.S8_in = in.S8_out;
            }
            in.parent = nullptr;
        } else {
            pa::RealInst& in = pl->re.i;
            pl->g_S8in = in.Sin; pl->g_S8out = in.Sout;
            in.Sin = in.Sout;
            in.parent = nullptr;
        }
    }
    pl->grad_pm = c->acc_grad && c->kind == PA_PM1;
    pa::ObsArgs& oa = pl->ob;
    oa.R = R; oa.kind = c->kind == PA_PM1 ? 0 : 1; oa.E32 = c->E32; oa.E128 = c->E128;
    if (dyn) { oa.Rdev = c->Rdev + k; oa.R = c->R; }
    oa.family = c->fam[c->famcur]; oa.part = c->obspart; oa.cur = c->acc + k; oa.logc = c->logc;
    oa.sync = c->sync + 2;
    c->k_next = k + 1;
    pl->cur = c->cur;
    pl->famcur = c->famcur;
}

// enqueue the k = 0 initialisation of one context
static int enqueue_init(pa_ctx* c)
{
    const uint32_t k0 = (uint32_t)c->seed, k1 = (uint32_t)(c->seed >> 32);
    const uint32_t c3 = pa::counter3(pa::STREAM_INIT, c->tag, c->inst);
    const int R0 = c->Rk[0];
    if (c->layout == PA_LAYOUT_PACKED)
        PA_CK(c, pa::launch_init_packed(c->S[c->cur], c->N, (R0 + 63) / 64, k0, k1, c3, c->st, c->shard_off / 64));
    else
        PA_CK(c, pa::launch_init_i8(c->S8[c->cur], c->N, c->NP, R0, k0, k1, c3, c->st));
    iota_kernel<<<(c->R + 255) / 256, 256, 0, c->st>>>(c->fam[c->famcur], c->parent, c->R, c->shard_off);
    acc0_kernel<<<1, 1, 0, c->st>>>(c->acc, c->betaF0, R0, c->Rdev);
    PA_CK(c, cudaGetLastError());
    c->launches += 3;
    return PA_OK;
}

// enqueue step k (no synchronisation)
static int enqueue_step(pa_ctx* c)
{
    const int k = c->k_next;
    if (k >= c->n_temps) { c->err = "schedule finished"; return PA_EDONE; }
    if (c->shard_total > 0 && k > 0) {
        c->err = "a shard resamples across shards: steps k >= 1 run with the pa_shard_* phases";
        return PA_ESTATE;
    }
    cudaEvent_t ev;
    if (k == 0) {
        ev = phase_begin(c, PA_PHASE_INIT);
        int rc = enqueue_init(c);
        if (rc) return rc;
        phase_end(c, PA_PHASE_INIT, ev);
    }
    StepPlan pl;
    plan_step(c, &pl);
    if (k > 0) {
        ev = phase_begin(c, PA_PHASE_RESAMPLE);
        PA_CK(c, pa::launch_resample(pl.rs, c->st));
        c->launches += pl.rs.wtab ? 6 : 5;
        phase_end(c, PA_PHASE_RESAMPLE, ev);
    }
    if (pl.gather) {
        ev = phase_begin(c, PA_PHASE_GATHER);
        const bool dyn = c->scheme == PA_RESAMPLE_NEAREST;
        PA_CK(c, pa::launch_gather(pl.g_Sin, pl.g_Sout, pl.g_S8in, pl.g_S8out, c->parent, c->N, c->NP,
                                   dyn ? c->R : c->Rk[k], dyn ? c->Rdev + k : nullptr, c->st));
        c->launches += 1;
        phase_end(c, PA_PHASE_GATHER, ev);
    }
    ev = phase_begin(c, PA_PHASE_SWEEP);
    if (c->kind == PA_PM1)
        PA_CK(c, pa::launch_sweep_packed(c->D, c->L, pl.pk, c->gpb, c->threads, c->st));
    else
        PA_CK(c, pa::launch_sweep_real(c->D, c->L, pl.re, c->real_warps, 0, c->st));
    c->launches += 1;
    if (pl.icm) {
        for (int t = 0; t < 2; ++t) {
            pa::IcmArgs ic = pl.ic;
            ic.t = t;
            PA_CK(c, pa::launch_icm(ic, c->st));
        }
        if (c->kind == PA_PM1)
            PA_CK(c, pa::launch_sweep_packed(c->D, c->L, pl.pk2, c->gpb, c->threads, c->st));
        else
            PA_CK(c, pa::launch_sweep_real(c->D, c->L, pl.re2, c->real_warps, 0, c->st));
        c->launches += 3;
    }
    if (pl.grad_pm) {
        const bool dyn = c->scheme == PA_RESAMPLE_NEAREST;
        const bool packed = c->layout == PA_LAYOUT_PACKED;
        PA_CK(c, pa::launch_grad_counts_pm(packed ? c->S[pl.cur] : nullptr, packed ? nullptr : c->S8[pl.cur],
                                           c->NP, c->D, c->L, dyn ? c->R : c->Rk[k],
                                           dyn ? c->Rdev + k : nullptr, c->cJ + (size_t)k * c->D * c->N,
                                           c->ch + (size_t)k * c->N, c->st));
        c->launches += 1;
    }
    phase_end(c, PA_PHASE_SWEEP, ev);
    ev = phase_begin(c, PA_PHASE_OBSERVE);
    PA_CK(c, pa::launch_observe(pl.ob, c->st));
    c->launches += 1;
    phase_end(c, PA_PHASE_OBSERVE, ev);
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

// population after the last completed step (before any step: the initial
// one); the nearest-integer scheme keeps it in device memory (synchronises)
static int pop_now(pa_ctx* c, int* R)
{
    const int k = c->k_next > 0 ? c->k_next - 1 : 0;
    *R = c->Rk[k];
    if (c->scheme == PA_RESAMPLE_NEAREST && c->k_next > 0) {
        PA_CK(c, cudaMemcpyAsync(R, c->Rdev + k, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        PA_CK(c, cudaStreamSynchronize(c->st));
        if (*R == 0) { c->err = "population died out"; return PA_EEMPTY; }
    }
    return PA_OK;
}
#define PA_POP(ctx, var)                      \
    int var;                                  \
    do {                                      \
        int rc__ = pop_now((ctx), &var);      \
        if (rc__ != PA_OK) return rc__;       \
    } while (0)

extern "C" int pa_synchronize(pa_ctx* c)
{
    if (!c) return PA_EINVAL;
    PA_CK(c, cudaStreamSynchronize(c->st));
    if (c->icm) {
        int bad = 0;
        PA_CK(c, cudaMemcpy(&bad, c->icm_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (bad) { c->err = "a cluster-move union-find loop reached its bound"; return PA_ETIMEOUT; }
    }
    int R;
    return pop_now(c, &R);  // PA_EEMPTY once the population died out
}

extern "C" int pa_observables(pa_ctx* c, int k, pa_obs* out)
{
    if (!c || !out) return PA_EINVAL;
    if (k < 0 || k >= c->k_next) { c->err = "step not run yet"; return PA_ESTATE; }
    StepAcc a;
    int Rk = c->Rk[k];
    PA_CK(c, cudaMemcpyAsync(&a, c->acc + k, sizeof a, cudaMemcpyDeviceToHost, c->st));
    if (c->scheme == PA_RESAMPLE_NEAREST)
        PA_CK(c, cudaMemcpyAsync(&Rk, c->Rdev + k, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    PA_CK(c, cudaStreamSynchronize(c->st));
    if (Rk == 0) { c->err = "population died out"; return PA_EEMPTY; }
    const double R = (double)Rk;
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
    out->S_f = std::log(R) - a.sum_clnc / R;
    out->rho_s = R / std::exp(out->S_f);
    out->R = Rk;
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
    PA_CK(c, pa::launch_grad_backward(c->cJ, c->ch, c->gbar_d, c->betas_d, c->Rk_d, c->n_temps, nJ, c->N,
                                      c->dJ_d, c->dh_d, c->st));
    PA_CK(c, cudaMemcpyAsync(dJ, c->dJ_d, sizeof(double) * nJ, cudaMemcpyDeviceToHost, c->st));
    if (dh) PA_CK(c, cudaMemcpyAsync(dh, c->dh_d, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->st));
    PA_CK(c, cudaStreamSynchronize(c->st));
    return PA_OK;
}

extern "C" int pa_overlap(pa_ctx* a, pa_ctx* b, int64_t* hist)
{
    if (!a || !b || !hist) return PA_EINVAL;
    PA_POP(a, Ra);
    PA_POP(b, Rb);
    if (a->D != b->D || a->L != b->L || Ra != Rb || a->layout != b->layout) {
        a->err = "overlap needs two contexts of the same lattice, R and layout";
        return PA_EINVAL;
    }
    PA_CK(a, cudaStreamSynchronize(b->st));
    PA_CK(a, cudaMemsetAsync(a->hist, 0, sizeof(unsigned long long) * (a->N + 1), a->st));
    if (a->layout == PA_LAYOUT_PACKED)
        PA_CK(a, pa::launch_overlap_packed(a->S[a->cur], b->S[b->cur], a->N, Ra, a->hist, a->st));
    else
        PA_CK(a, pa::launch_overlap_i8(a->S8[a->cur], b->S8[b->cur], a->N, a->NP, Ra, a->hist, a->st));
    PA_CK(a, cudaMemcpyAsync(hist, a->hist, sizeof(int64_t) * (a->N + 1), cudaMemcpyDeviceToHost, a->st));
    PA_CK(a, cudaStreamSynchronize(a->st));
    return PA_OK;
}

extern "C" int pa_get_spins_range(pa_ctx* c, int r0, int n, int8_t* dst)
{
    if (!c || !dst) return PA_EINVAL;
    PA_POP(c, Rn);
    if (r0 < 0 || n < 0 || r0 + n > Rn) return PA_EINVAL;
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
    PA_POP(c, Rn);
    return pa_get_spins_range(c, 0, Rn, dst);
}

extern "C" int pa_get_energies(pa_ctx* c, int64_t* dst)
{
    if (!c || !dst) return PA_EINVAL;
    PA_POP(c, Rn);
    if (c->kind == PA_PM1) {
        std::vector<int32_t> e(Rn);
        PA_CK(c, cudaMemcpyAsync(e.data(), c->E32, sizeof(int32_t) * Rn, cudaMemcpyDeviceToHost, c->st));
        PA_CK(c, cudaStreamSynchronize(c->st));
        for (int r = 0; r < Rn; ++r) dst[r] = e[r];
    } else {
        PA_CK(c, cudaMemcpyAsync(dst, c->E128, sizeof(longlong2) * Rn, cudaMemcpyDeviceToHost, c->st));
        PA_CK(c, cudaStreamSynchronize(c->st));
    }
    return PA_OK;
}

extern "C" int pa_get_parents(pa_ctx* c, int32_t* dst)
{
    if (!c || !dst) return PA_EINVAL;
    PA_POP(c, Rn);
    PA_CK(c, cudaMemcpyAsync(dst, c->parent, sizeof(int32_t) * Rn, cudaMemcpyDeviceToHost, c->st));
    PA_CK(c, cudaStreamSynchronize(c->st));
    return PA_OK;
}

extern "C" int pa_get_family(pa_ctx* c, int32_t* dst)
{
    if (!c || !dst) return PA_EINVAL;
    PA_POP(c, Rn);
    PA_CK(c, cudaMemcpyAsync(dst, c->fam[c->famcur], sizeof(int32_t) * Rn, cudaMemcpyDeviceToHost, c->st));
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
    if (R) {
        int rc = pop_now(const_cast<pa_ctx*>(c), R);
        if (rc != PA_OK && rc != PA_EEMPTY) return rc;  // an empty population reports R = 0
    }
    if (n_temps) *n_temps = c->n_temps;
    if (layout) *layout = c->layout;
    return PA_OK;
}

// ---------------- checkpoint / resume ----------------
//
// A checkpoint holds the state that the next step reads: the spin buffer in
// use, energies, parents, families, the per-temperature accumulators, the
// populations and (with accumulate_grad) the gradient counts, behind a
// header that pins the configuration (sizes, options, seed, and an FNV-1a
// fingerprint of the couplings, field, schedule and population targets).

namespace {
struct CkptHeader {
    char magic[8];
    uint32_t version;
    int32_t D, L, kind, cap, n_temps, n_sweeps, layout, scheme, acc_grad;
    uint32_t inst, tag;
    uint64_t seed, fingerprint;
    int32_t k_next, cur, famcur, pad;
};
constexpr char kCkptMagic[8] = {'P', 'A', 'M', 'C', 'C', 'K', 'P', 'T'};

uint64_t fnv1a(uint64_t h, const void* p, size_t n)
{
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    return h;
}

struct CkptSection {
    void* dev;
    size_t bytes;
};
}  // namespace

static std::vector<CkptSection> ckpt_sections(pa_ctx* c)
{
    std::vector<CkptSection> v;
    const size_t cap = (size_t)c->R;
    if (c->layout == PA_LAYOUT_PACKED) v.push_back({c->S[c->cur], sizeof(uint64_t) * (size_t)c->G * c->N});
    else v.push_back({c->S8[c->cur], cap * c->NP});
    if (c->kind == PA_PM1) v.push_back({c->E32, sizeof(int32_t) * cap});
    else v.push_back({c->E128, sizeof(longlong2) * cap});
    v.push_back({c->parent, sizeof(int32_t) * cap});
    v.push_back({c->fam[c->famcur], sizeof(int32_t) * cap});
    v.push_back({c->acc, sizeof(StepAcc) * c->n_temps});
    v.push_back({c->Rdev, sizeof(int) * c->n_temps});
    v.push_back({c->Rk_d, sizeof(double) * c->n_temps});
    if (c->acc_grad) {
        v.push_back({c->cJ, sizeof(unsigned long long) * (size_t)c->n_temps * c->D * c->N});
        v.push_back({c->ch, sizeof(unsigned long long) * (size_t)c->n_temps * c->N});
    }
    return v;
}

static CkptHeader ckpt_header(const pa_ctx* c)
{
    CkptHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = 1;
    h.D = c->D; h.L = c->L; h.kind = c->kind; h.cap = c->R; h.n_temps = c->n_temps;
    h.n_sweeps = c->n_sweeps; h.layout = c->layout; h.scheme = c->scheme; h.acc_grad = c->acc_grad;
    h.inst = c->inst; h.tag = c->tag; h.seed = c->seed;
    uint64_t f = 1469598103934665603ull;
    f = fnv1a(f, c->Jh.data(), sizeof(float) * c->Jh.size());
    f = fnv1a(f, c->hh.data(), sizeof(float) * c->hh.size());
    f = fnv1a(f, c->betas.data(), sizeof(double) * c->betas.size());
    f = fnv1a(f, c->Rk.data(), sizeof(int) * c->Rk.size());
    const double icmw[3] = {(double)c->icm, c->icm_lo, c->icm_hi};
    f = fnv1a(f, icmw, sizeof icmw);
    h.fingerprint = f;
    h.k_next = c->k_next; h.cur = c->cur; h.famcur = c->famcur;
    return h;
}

extern "C" int pa_checkpoint_size(const pa_ctx* c, size_t* bytes)
{
    if (!c || !bytes) return PA_EINVAL;
    size_t n = sizeof(CkptHeader);
    for (const auto& sct : ckpt_sections(const_cast<pa_ctx*>(c))) n += sct.bytes;
    *bytes = n;
    return PA_OK;
}

extern "C" int pa_checkpoint_save(pa_ctx* c, void* buf, size_t bytes)
{
    if (!c || !buf) return PA_EINVAL;
    size_t need = 0;
    pa_checkpoint_size(c, &need);
    if (bytes < need) { c->err = "checkpoint buffer too small"; return PA_EINVAL; }
    const CkptHeader h = ckpt_header(c);
    std::memcpy(buf, &h, sizeof h);
    char* p = (char*)buf + sizeof h;
    for (const auto& sct : ckpt_sections(c)) {
        PA_CK(c, cudaMemcpyAsync(p, sct.dev, sct.bytes, cudaMemcpyDeviceToHost, c->st));
        p += sct.bytes;
    }
    PA_CK(c, cudaStreamSynchronize(c->st));
    return PA_OK;
}

extern "C" int pa_checkpoint_load(pa_ctx* c, const void* buf, size_t bytes)
{
    if (!c || !buf) return PA_EINVAL;
    CkptHeader h;
    if (bytes < sizeof h) { c->err = "checkpoint truncated"; return PA_EINVAL; }
    std::memcpy(&h, buf, sizeof h);
    CkptHeader mine = ckpt_header(c);
    if (std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != 1) { c->err = "not a checkpoint"; return PA_EINVAL; }
    mine.k_next = h.k_next; mine.cur = h.cur; mine.famcur = h.famcur;
    if (std::memcmp(&h, &mine, sizeof h) != 0) {
        c->err = "checkpoint of a different configuration (sizes, options, seed, couplings or schedule)";
        return PA_EINVAL;
    }
    if (h.k_next < 0 || h.k_next > c->n_temps || (h.cur & ~1) || (h.famcur & ~1)) {
        c->err = "checkpoint state out of range";
        return PA_EINVAL;
    }
    PA_CK(c, cudaStreamSynchronize(c->st));
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    c->k_next = h.k_next; c->cur = h.cur; c->famcur = h.famcur;
    size_t need = 0;
    pa_checkpoint_size(c, &need);
    if (bytes < need) { c->err = "checkpoint truncated"; return PA_EINVAL; }
    const char* p = (const char*)buf + sizeof h;
    for (const auto& sct : ckpt_sections(c)) {
        PA_CK(c, cudaMemcpyAsync(sct.dev, p, sct.bytes, cudaMemcpyHostToDevice, c->st));
        p += sct.bytes;
    }
    PA_CK(c, cudaStreamSynchronize(c->st));
    return PA_OK;
}

// ---------------- shards of one population (Sec. V.A) ----------------
//
// A step k >= 1 of a shard runs in phases; between them the caller exchanges
// small arrays among the shards (in shard order) and finally the replicas
// each shard's new slots descend from.  Every phase synchronises the stream.

static int shard_check(pa_ctx* c, int min_k)
{
    if (!c) return PA_EINVAL;
    if (c->shard_total <= 0) { c->err = "not a shard"; return PA_ESTATE; }
    if (c->k_next < min_k || c->k_next >= c->n_temps) { c->err = "no step to run"; return PA_ESTATE; }
    return PA_OK;
}

// the resampling arguments of step k of a shard
static void shard_args(pa_ctx* c, pa::ResampleArgs* ra)
{
    const int k = c->k_next;
    std::memset(ra, 0, sizeof *ra);
    ra->R = c->R; ra->Rn = c->shard_total; ra->kind = 0;
    ra->gR = c->shard_total; ra->gb0 = c->shard_off / pa::kWBlock;
    ra->E32 = c->E32;
    ra->prev = c->acc + (k - 1); ra->cur = c->acc + k;
    ra->w = c->w; ra->P = c->P; ra->lev1 = c->lev1; ra->t2g = c->sh_t2g;
    ra->counts = c->counts; ra->blocksum = c->blocksum;
    ra->parent = c->sh_pout; ra->fam_in = c->fam[c->famcur]; ra->fam_out = c->sh_fout;
    ra->dbeta = c->betas[k] - c->betas[k - 1];
    ra->log_R = std::log((double)c->shard_total); ra->betaF0 = c->betaF0; ra->k = k;
    ra->wtab = c->wtab; ra->wtab_n = c->D * c->N / 2 + 1;
    ra->key0 = (uint32_t)c->seed; ra->key1 = (uint32_t)(c->seed >> 32);
    ra->c3 = pa::counter3(pa::STREAM_RES, c->tag, c->inst);
}

extern "C" int pa_shard_emin(pa_ctx* c, int64_t* emin)
{
    int rc = shard_check(c, 1);
    if (rc) return rc;
    if (!emin) return PA_EINVAL;
    StepAcc a;
    PA_CK(c, cudaMemcpyAsync(&a, c->acc + (c->k_next - 1), sizeof a, cudaMemcpyDeviceToHost, c->st));
    PA_CK(c, cudaStreamSynchronize(c->st));
    *emin = a.emin_lo;
    return PA_OK;
}

extern "C" int pa_shard_weights(pa_ctx* c, int64_t emin_global, double* host_block_totals)
{
    int rc = shard_check(c, 1);
    if (rc) return rc;
    if (!host_block_totals) return PA_EINVAL;
    // the weights are taken relative to the lowest energy of the whole population
    const long long em[2] = {(long long)emin_global, emin_global < 0 ? -1ll : 0ll};
    PA_CK(c, cudaMemcpyAsync(&c->acc[c->k_next - 1].emin_lo, em, sizeof em, cudaMemcpyHostToDevice, c->st));
    pa::ResampleArgs ra;
    shard_args(c, &ra);
    ra.upper = c->upper;  // the local block totals
    PA_CK(c, pa::launch_resample_shard(ra, 0, c->st));
    PA_CK(c, cudaMemcpyAsync(host_block_totals, c->upper, sizeof(double) * pa::rs_wblocks(c->R),
                             cudaMemcpyDeviceToHost, c->st));
    PA_CK(c, cudaStreamSynchronize(c->st));
    c->launches += 2;
    return PA_OK;
}

extern "C" int pa_shard_prefix(pa_ctx* c, const double* host_all_totals, double* host_block_max)
{
    int rc = shard_check(c, 1);
    if (rc) return rc;
    if (!host_all_totals || !host_block_max) return PA_EINVAL;
    const size_t nbg = (size_t)pa::rs_wblocks(c->shard_total);
    PA_CK(c, cudaMemcpyAsync(c->sh_upper, host_all_totals, sizeof(double) * nbg, cudaMemcpyHostToDevice, c->st));
    PA_CK(c, cudaMemcpyAsync(c->sh_t2g, host_all_totals, sizeof(double) * nbg, cudaMemcpyHostToDevice, c->st));
    pa::ResampleArgs ra;
    shard_args(c, &ra);
    ra.upper = c->sh_upper;  // every shard's block totals -> the global levels >= 2
    ra.bmax = c->bmax;       // the local block maxima
    PA_CK(c, pa::launch_resample_shard(ra, 1, c->st));
    PA_CK(c, cudaMemcpyAsync(host_block_max, c->bmax, sizeof(double) * pa::rs_wblocks(c->R),
                             cudaMemcpyDeviceToHost, c->st));
    PA_CK(c, cudaStreamSynchronize(c->st));
    c->launches += 2;
    return PA_OK;
}

extern "C" int pa_shard_draw(pa_ctx* c, const double* host_all_block_max, int32_t* copies)
{
    int rc = shard_check(c, 1);
    if (rc) return rc;
    if (!host_all_block_max || !copies) return PA_EINVAL;
    const size_t nbg = (size_t)pa::rs_wblocks(c->shard_total);
    PA_CK(c, cudaMemcpyAsync(c->sh_bmax, host_all_block_max, sizeof(double) * nbg, cudaMemcpyHostToDevice, c->st));
    pa::ResampleArgs ra;
    shard_args(c, &ra);
    ra.bmax = c->sh_bmax;
    PA_CK(c, pa::launch_resample_shard(ra, 2, c->st));
    const int nbs = (c->R + pa::kScanBlock - 1) / pa::kScanBlock;
    int32_t n = 0;
    PA_CK(c, cudaMemcpyAsync(&n, c->blocksum + nbs, sizeof n, cudaMemcpyDeviceToHost, c->st));
    PA_CK(c, cudaStreamSynchronize(c->st));
    c->launches += 4;
    c->shard_copies = n;
    *copies = n;
    return PA_OK;
}

extern "C" int pa_shard_copies(pa_ctx* c, int32_t* host_parent, int32_t* host_family)
{
    int rc = shard_check(c, 1);
    if (rc) return rc;
    if (!host_parent || !host_family) return PA_EINVAL;
    pa::ResampleArgs ra;
    shard_args(c, &ra);
    PA_CK(c, pa::launch_resample_shard(ra, 3, c->st));
    const size_t n = (size_t)c->shard_copies;
    PA_CK(c, cudaMemcpyAsync(host_parent, c->sh_pout, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c->st));
    PA_CK(c, cudaMemcpyAsync(host_family, c->sh_fout, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c->st));
    PA_CK(c, cudaStreamSynchronize(c->st));
    c->launches += 1;
    return PA_OK;
}

extern "C" int pa_shard_pack(pa_ctx* c, const int32_t* host_replicas, int n, void* dst, int dst_on_device)
{
    int rc = shard_check(c, 1);
    if (rc) return rc;
    if (n < 0 || n > c->R || (n > 0 && (!host_replicas || !dst))) return PA_EINVAL;
    if (n == 0) return PA_OK;
    for (int i = 0; i < n; ++i)
        if (host_replicas[i] < c->shard_off || host_replicas[i] >= c->shard_off + c->R ||
            (i > 0 && host_replicas[i] <= host_replicas[i - 1])) {
            c->err = "pa_shard_pack: replicas must be increasing global indices of this shard";
            return PA_EINVAL;
        }
    // the local indices of the replicas, then the packed gather of those replicas
    std::vector<int32_t> loc(n);
    for (int i = 0; i < n; ++i) loc[i] = host_replicas[i] - c->shard_off;
    PA_CK(c, cudaMemcpyAsync(c->sh_pout, loc.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, c->st));
    const int ng = (n + 63) / 64;
    uint64_t* out = c->sh_stage;  // scratch until pa_shard_finish receives
    PA_CK(c, pa::launch_gather(c->S[c->cur], out, nullptr, nullptr, c->sh_pout, c->N, c->NP, n, nullptr, c->st));
    PA_CK(c, cudaMemcpyAsync(dst, out, sizeof(uint64_t) * (size_t)ng * c->N,
                             dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st));
    PA_CK(c, cudaStreamSynchronize(c->st));
    c->launches += 1;
    return PA_OK;
}

extern "C" int pa_shard_finish(pa_ctx* c, const void* groups, int n_groups, int src_on_device,
                               const int32_t* host_parent, const int32_t* host_family)
{
    int rc = shard_check(c, 1);
    if (rc) return rc;
    const int G = (c->R + 63) / 64;
    if (!groups || !host_parent || !host_family || n_groups < 1 || n_groups > G + kShardStageExtra) {
        c->err = "pa_shard_finish: need 1..(own groups + 64) incoming groups, parents and families";
        return PA_EINVAL;
    }
    for (int j = 0; j < c->R; ++j)
        if (host_parent[j] < 0 || host_parent[j] >= 64 * n_groups) {
            c->err = "pa_shard_finish: a parent index is outside the incoming groups";
            return PA_EINVAL;
        }
    PA_CK(c, cudaMemcpyAsync(c->sh_stage, groups, sizeof(uint64_t) * (size_t)n_groups * c->N,
                             src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st));
    StepPlan pl;
    plan_step(c, &pl);  // advances k, the ping-pong buffers and the family buffer
    PA_CK(c, cudaMemcpyAsync(c->parent, host_parent, sizeof(int32_t) * c->R, cudaMemcpyHostToDevice, c->st));
    PA_CK(c, cudaMemcpyAsync(c->fam[c->famcur], host_family, sizeof(int32_t) * c->R, cudaMemcpyHostToDevice,
                             c->st));
    pl.pk.i.Sin = c->sh_stage;  // the gather reads the incoming replicas
    pl.pk.i.parent = c->parent;
    cudaEvent_t ev = phase_begin(c, PA_PHASE_SWEEP);
    PA_CK(c, pa::launch_sweep_packed(c->D, c->L, pl.pk, c->gpb, c->threads, c->st));
    phase_end(c, PA_PHASE_SWEEP, ev);
    ev = phase_begin(c, PA_PHASE_OBSERVE);
    PA_CK(c, pa::launch_observe(pl.ob, c->st));
    phase_end(c, PA_PHASE_OBSERVE, ev);
    PA_CK(c, cudaStreamSynchronize(c->st));
    c->launches += 2;
    return PA_OK;
}

extern "C" int pa_shard_sums(pa_ctx* c, int k, int64_t* sums)
{
    if (!c || !sums) return PA_EINVAL;
    if (c->shard_total <= 0) { c->err = "not a shard"; return PA_ESTATE; }
    if (k < 0 || k >= c->k_next) { c->err = "step not run yet"; return PA_ESTATE; }
    StepAcc a;
    PA_CK(c, cudaMemcpyAsync(&a, c->acc + k, sizeof a, cudaMemcpyDeviceToHost, c->st));
    PA_CK(c, cudaStreamSynchronize(c->st));
    sums[0] = a.sumE;
    sums[1] = a.sumE2;
    sums[2] = a.emin_lo;
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

// ====================== batched instances ======================
//
// A batch owns one context per instance (carved from one workspace) plus
// device tables with every instance's kernel arguments for every temperature
// (built by plan_step, so the batched launches and the per-instance launches
// follow the same ping-pong sequence).  A batched step is: k = 0 initialisation
// per instance; resampling for all instances (one launch per kernel); one
// persistent sweep launch over a work queue of (instance, tile) items; the
// observables for all instances.

#include <algorithm>
#include <map>
#include <mutex>

struct pa_batch {
    int D, n_inst, n_temps, n_sweeps, k_next;
    uint64_t seed;
    cudaStream_t st;
    void* ws;
    std::vector<pa_ctx*> ctx;
    std::vector<double> betas;
    pa::ResampleArgs* d_rs;        // [n_temps][n_inst]
    pa::BatchSweepInst* d_sw;      // [n_temps][n_inst]
    pa::ObsArgs* d_ob;             // [n_temps][n_inst]
    int2* d_items[2];              // work items per groups-per-block multiplier
    int n_items[2];
    size_t smem[2];
    int* d_counters;               // [n_temps + kTuneSlots]
    std::vector<int> after_cur, after_fam;  // [k * n_inst + i]: context state after step k
    int maxR;
    bool has_packed;
    int band;                      // acceptance guard band verified (real instances)
    int tune_mode;                 // 0 tune, -1 defaults
    bool tuned;
    int blocks, mult, tune_slot;
    double tuned_ms;
    std::string sig;
    cudaGraphExec_t gexec;
    long long launches;
    std::string err;
};

static constexpr int kTuneSlots = 64;
static std::mutex g_tune_mu;
static std::map<std::string, std::pair<int, int>> g_tune_cache;  // signature -> (blocks, mult)

#define PB_CK(b, call)                                                                   \
    do {                                                                                 \
        cudaError_t e__ = (call);                                                        \
        if (e__ != cudaSuccess) {                                                        \
            (b)->err = std::string(#call) + ": " + cudaGetErrorString(e__);              \
            return PA_ECUDA;                                                             \
        }                                                                                \
    } while (0)

static void batch_free(pa_batch* b)
{
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (auto* c : b->ctx) pa_destroy(c);
    cudaFree(b->d_rs);
    cudaFree(b->d_sw);
    cudaFree(b->d_ob);
    cudaFree(b->d_items[0]);
    cudaFree(b->d_items[1]);
    cudaFree(b->d_counters);
    cudaFree(b->ws);
    delete b;
}

extern "C" int pa_batch_create(pa_batch** out, int D, int n_inst, const pa_inst_desc* descs,
                               const double* betas, int n_temps, int n_sweeps, uint64_t seed,
                               const pa_options* opt, void* stream)
{
    if (!out) return PA_EINVAL;
    *out = nullptr;
    if (D != 3) { g_create_err = "batched sweeps support D = 3"; return PA_EINVAL; }
    if (n_inst < 1 || !descs) { g_create_err = "need at least one instance"; return PA_EINVAL; }
    if (opt && (opt->layout != PA_LAYOUT_AUTO || opt->accumulate_grad || opt->populations || opt->separate_gather ||
                opt->resampling != PA_RESAMPLE_MULTINOMIAL || opt->capacity || opt->icm)) {
        g_create_err = "batch: layout must be AUTO, accumulate_grad 0, populations NULL, multinomial "
                       "resampling and no capacity";
        return PA_EINVAL;
    }
    pa_batch* b = new pa_batch();
    b->D = D; b->n_inst = n_inst; b->n_temps = n_temps; b->n_sweeps = n_sweeps; b->k_next = 0;
    b->seed = seed; b->st = (cudaStream_t)stream; b->ws = nullptr;
    b->d_rs = nullptr; b->d_sw = nullptr; b->d_ob = nullptr;
    b->d_items[0] = b->d_items[1] = nullptr; b->d_counters = nullptr; b->gexec = nullptr;
    b->tune_mode = (opt && opt->threads < 0) ? -1 : 0;
    b->tuned = b->tune_mode < 0;
    b->blocks = 0; b->mult = 1; b->tune_slot = 0; b->tuned_ms = 0.0; b->launches = 0;
    b->maxR = 0; b->has_packed = false; b->band = 0;
    // validate every instance and size the workspace
    std::vector<size_t> offs(n_inst);
    size_t total = 0;
    for (int i = 0; i < n_inst; ++i) {
        const pa_inst_desc& d = descs[i];
        pa_options o;
        pa_options_default(&o);
        o.rng_instance = d.rng_instance;
        std::string err;
        int rc = validate(err, D, d.L, d.kind, d.J, d.h, d.R, betas, n_temps, n_sweeps, &o);
        int cls, tiles;
        size_t sm;
        int G = (d.R + 63) / 64;
        if (rc == PA_OK && !pa::batch_class(D, d.L, d.kind, 1, G, d.R, &cls, &tiles, &sm)) {
            err = "lattice size not supported by the batched sweep (3D L in 4..12 even or 16)";
            rc = PA_EINVAL;
        }
        if (rc) {
            g_create_err = "instance " + std::to_string(i) + ": " + err;
            delete b;
            return rc;
        }
        int lay = resolve_layout(d.kind, &o);
        offs[i] = total;
        total += make_layout(D, d.L, d.kind, lay, d.R, n_temps, 0).total;
        b->maxR = std::max(b->maxR, d.R);
        b->has_packed |= d.kind == PA_PM1;
    }
    cudaError_t e = cudaMalloc(&b->ws, total);
    if (e != cudaSuccess) {
        g_create_err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        delete b;
        return PA_ENOMEM;
    }
    b->betas.assign(betas, betas + n_temps);
    for (int i = 0; i < n_inst; ++i) {
        const pa_inst_desc& d = descs[i];
        pa_options o;
        pa_options_default(&o);
        o.rng_instance = d.rng_instance;
        o.exact_accept = opt ? opt->exact_accept : 0;
        pa_ctx* c = nullptr;
        size_t sz = make_layout(D, d.L, d.kind, resolve_layout(d.kind, &o), d.R, n_temps, 0).total;
        int rc = create_impl(&c, D, d.L, d.kind, d.J, d.h, d.R, betas, n_temps, n_sweeps, seed, &o, stream,
                             (char*)b->ws + offs[i], sz);
        if (rc) {
            g_create_err = "instance " + std::to_string(i) + ": " + g_create_err;
            batch_free(b);
            return rc;
        }
        b->ctx.push_back(c);
        if (d.kind == PA_REAL) b->band = c->band;  // one verdict per device
    }
    // argument tables for every (temperature, instance)
    const size_t nt = (size_t)n_temps * n_inst;
    std::vector<pa::ResampleArgs> rs(nt);
    std::vector<pa::BatchSweepInst> sw(nt);
    std::vector<pa::ObsArgs> ob(nt);
    b->after_cur.resize(nt);
    b->after_fam.resize(nt);
    for (int i = 0; i < n_inst; ++i) {
        pa_ctx* c = b->ctx[i];
        int cls, tiles;
        size_t sm;
        pa::batch_class(D, c->L, c->kind, 1, c->G, c->R, &cls, &tiles, &sm);
        for (int k = 0; k < n_temps; ++k) {
            StepPlan pl;
            plan_step(c, &pl);
            const size_t at = (size_t)k * n_inst + i;
            rs[at] = pl.rs;
            rs[at].wtab = nullptr;  // the batched resampling computes every weight
            rs[at].wtab_n = 0;
            rs[at].sync = nullptr;  // and launches every stage
            std::memset(&sw[at], 0, sizeof sw[at]);
            sw[at].cls = cls;
            sw[at].pk = pl.pk.i;
            sw[at].re = pl.re.i;
            ob[at] = pl.ob;
            ob[at].sync = nullptr;
            b->after_cur[at] = pl.cur;
            b->after_fam[at] = pl.famcur;
        }
        c->k_next = 0; c->cur = 0; c->famcur = 0;
    }
    // work items, most expensive first (estimated thread-instructions per tile)
    for (int m = 1; m <= 2; ++m) {
        struct It { double cost; int inst, tile; };
        std::vector<It> items;
        size_t smax = 0;
        for (int i = 0; i < n_inst; ++i) {
            pa_ctx* c = b->ctx[i];
            int cls, tiles;
            size_t sm;
            pa::batch_class(D, c->L, c->kind, m, c->G, c->R, &cls, &tiles, &sm);
            smax = std::max(smax, sm);
            int gpb = 0, thr = 0;
            pa::packed_default_shape(D, c->L, &gpb, &thr);
            double cost = c->kind == PA_PM1 ? (double)gpb * m * c->N * 700.0 : 32.0 * c->N * 70.0;
            for (int t = 0; t < tiles; ++t) items.push_back({cost, i, t});
        }
        std::stable_sort(items.begin(), items.end(), [](const It& x, const It& y) { return x.cost > y.cost; });
        std::vector<int2> h(items.size());
        for (size_t t = 0; t < items.size(); ++t) h[t] = make_int2(items[t].inst, items[t].tile);
        b->n_items[m - 1] = (int)items.size();
        b->smem[m - 1] = smax;
        e = cudaMalloc(&b->d_items[m - 1], sizeof(int2) * h.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_items[m - 1], h.data(), sizeof(int2) * h.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->d_rs, sizeof(pa::ResampleArgs) * nt);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_sw, sizeof(pa::BatchSweepInst) * nt);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ob, sizeof(pa::ObsArgs) * nt);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counters, sizeof(int) * (n_temps + kTuneSlots));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_rs, rs.data(), sizeof(pa::ResampleArgs) * nt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_sw, sw.data(), sizeof(pa::BatchSweepInst) * nt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_ob, ob.data(), sizeof(pa::ObsArgs) * nt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->d_counters, 0, sizeof(int) * (n_temps + kTuneSlots));
    if (e != cudaSuccess) {
        g_create_err = std::string("batch tables: ") + cudaGetErrorString(e);
        batch_free(b);
        return PA_ECUDA;
    }
    // default sweep configuration: groups-per-block x1, as many blocks as fit
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (pa::batch_sweep_occupancy(std::max(b->smem[0], b->smem[1]), &per) != cudaSuccess || per < 1) per = 1;
    b->blocks = sms * per;
    // signature of the batch for the tuning cache: SM count and class histogram
    std::map<std::pair<int, int>, int> hist;
    for (auto* c : b->ctx) hist[{c->kind, c->L}] += 1;
    b->sig = std::to_string(sms) + "|" + std::to_string(n_sweeps);
    for (auto& kv : hist)
        b->sig += "|" + std::to_string(kv.first.first) + ":" + std::to_string(kv.first.second) + "x" +
                  std::to_string(kv.second);
    if (b->tune_mode == 0) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(b->sig);
        if (it != g_tune_cache.end()) {
            b->blocks = it->second.first;
            b->mult = it->second.second;
            b->tuned = true;
        }
    }
    *out = b;
    return PA_OK;
}

static void batch_step_params(pa_batch* b, int k, pa::PackedStep* ps, pa::RealStep* rs)
{
    const uint32_t k0 = (uint32_t)b->seed, k1 = (uint32_t)(b->seed >> 32);
    fill_packed_step(ps, b->D, b->betas[k], k, b->n_sweeps, k0, k1);
    rs->k = k; rs->n_sweeps = b->n_sweeps; rs->beta = (float)b->betas[k]; rs->key0 = k0; rs->key1 = k1;
    rs->hs0 = 2u * (uint32_t)(k * b->n_sweeps);
    rs->band = b->band;
    fill_round_keys(rs->rk, k0, k1);
}

// time every candidate sweep configuration on step k; a sweep with k >= 1
// reads its input replicas from one buffer and writes another, so re-running
// it gives the same outputs, and every candidate gives identical results
static int batch_tune(pa_batch* b, int k)
{
    pa::PackedStep ps;
    pa::RealStep rs;
    batch_step_params(b, k, &ps, &rs);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaEvent_t e0, e1;
    PB_CK(b, cudaEventCreate(&e0));
    PB_CK(b, cudaEventCreate(&e1));
    double best = 1e30;
    int bb = b->blocks, bm = 1;
    const pa::BatchSweepInst* tab = b->d_sw + (size_t)k * b->n_inst;
    for (int m = 1; m <= (b->has_packed ? 2 : 1); ++m) {
        int per = 0;
        if (pa::batch_sweep_occupancy(b->smem[m - 1], &per) != cudaSuccess || per < 1) continue;
        for (int bps = 1; bps <= per; ++bps) {
            if (b->tune_slot >= kTuneSlots) break;
            int* ctr = b->d_counters + b->n_temps + b->tune_slot++;
            PB_CK(b, cudaEventRecord(e0, b->st));
            PB_CK(b, pa::launch_sweep_batched(ps, rs, tab, b->d_items[m - 1], b->n_items[m - 1], m, ctr,
                                              sms * bps, b->smem[m - 1], b->st));
            PB_CK(b, cudaEventRecord(e1, b->st));
            PB_CK(b, cudaEventSynchronize(e1));
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) { best = ms; bb = sms * bps; bm = m; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->blocks = bb;
    b->mult = bm;
    b->tuned_ms = best;
    b->tuned = true;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[b->sig] = {bb, bm};
    return PA_OK;
}

static int batch_enqueue(pa_batch* b, bool allow_tune)
{
    const int k = b->k_next;
    if (k >= b->n_temps) { b->err = "schedule finished"; return PA_EDONE; }
    if (k == 0) {
        for (auto* c : b->ctx) {
            int rc = enqueue_init(c);
            if (rc) { b->err = c->err; return rc; }
            b->launches += 3;
        }
    } else {
        PB_CK(b, pa::launch_resample_batched(b->d_rs + (size_t)k * b->n_inst, b->n_inst, b->maxR, b->st));
        b->launches += 8;
    }
    if (!b->tuned && allow_tune && k >= 1) {
        int rc = batch_tune(b, k);
        if (rc) return rc;
    }
    pa::PackedStep ps;
    pa::RealStep rs;
    batch_step_params(b, k, &ps, &rs);
    PB_CK(b, pa::launch_sweep_batched(ps, rs, b->d_sw + (size_t)k * b->n_inst, b->d_items[b->mult - 1],
                                      b->n_items[b->mult - 1], b->mult, b->d_counters + k, b->blocks,
                                      b->smem[b->mult - 1], b->st));
    PB_CK(b, pa::launch_observe_batched(b->d_ob + (size_t)k * b->n_inst, b->n_inst, b->maxR, b->st));
    b->launches += 3;
    for (int i = 0; i < b->n_inst; ++i) {
        pa_ctx* c = b->ctx[i];
        c->k_next = k + 1;
        c->cur = b->after_cur[(size_t)k * b->n_inst + i];
        c->famcur = b->after_fam[(size_t)k * b->n_inst + i];
    }
    b->k_next = k + 1;
    return PA_OK;
}

extern "C" int pa_batch_step(pa_batch* b)
{
    if (!b) return PA_EINVAL;
    for (auto* c : b->ctx)
        if (c->k_next != b->k_next) { b->err = "an instance was stepped on its own"; return PA_ESTATE; }
    return batch_enqueue(b, true);
}

extern "C" int pa_batch_run(pa_batch* b, int n_steps)
{
    if (!b) return PA_EINVAL;
    if (b->k_next >= b->n_temps) { b->err = "schedule finished"; return PA_EDONE; }
    int n = n_steps < 0 ? b->n_temps - b->k_next : n_steps;
    if (b->k_next + n > b->n_temps) { b->err = "n_steps past the end of the schedule"; return PA_EINVAL; }
    // the first steps run eagerly: k = 0 initialises, the first k >= 1 tunes
    while (n > 0 && (b->k_next == 0 || !b->tuned || !b->st)) {
        int rc = pa_batch_step(b);
        if (rc) return rc;
        --n;
    }
    if (n == 0) return PA_OK;
    if (b->gexec) {
        PB_CK(b, cudaStreamSynchronize(b->st));
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    const int k_save = b->k_next;
    const long long l_save = b->launches;
    std::vector<int> st_save;
    for (auto* c : b->ctx) { st_save.push_back(c->k_next); st_save.push_back(c->cur); st_save.push_back(c->famcur); }
    PB_CK(b, cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    int rc = PA_OK;
    for (int t = 0; t < n && rc == PA_OK; ++t) rc = batch_enqueue(b, false);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->st, &g);
    if (rc == PA_OK && e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (rc != PA_OK || e != cudaSuccess) {
        b->k_next = k_save;
        b->launches = l_save;
        for (size_t i = 0; i < b->ctx.size(); ++i) {
            b->ctx[i]->k_next = st_save[3 * i];
            b->ctx[i]->cur = st_save[3 * i + 1];
            b->ctx[i]->famcur = st_save[3 * i + 2];
        }
        b->gexec = nullptr;
        if (rc == PA_OK) { b->err = std::string("batch graph: ") + cudaGetErrorString(e); rc = PA_ECUDA; }
        return rc;
    }
    PB_CK(b, cudaGraphLaunch(b->gexec, b->st));
    return PA_OK;
}

extern "C" int pa_batch_current_step(const pa_batch* b) { return b ? b->k_next : PA_EINVAL; }

extern "C" int pa_batch_instance(pa_batch* b, int i, pa_ctx** out)
{
    if (!b || !out || i < 0 || i >= b->n_inst) return PA_EINVAL;
    *out = b->ctx[i];
    return PA_OK;
}

extern "C" int pa_batch_sweep_config(const pa_batch* b, int* blocks, int* gpb_mult, double* ms)
{
    if (!b) return PA_EINVAL;
    if (blocks) *blocks = b->blocks;
    if (gpb_mult) *gpb_mult = b->mult;
    if (ms) *ms = b->tuned_ms;
    return PA_OK;
}

extern "C" const char* pa_batch_last_error(const pa_batch* b)
{
    return b ? b->err.c_str() : g_create_err.c_str();
}

extern "C" void pa_batch_destroy(pa_batch* b) { batch_free(b); }
