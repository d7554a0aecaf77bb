/*
 * pa.h -- C ABI of the GB300 population annealing library (libpamc.so).
 *
 * Population annealing Monte Carlo (PAMC) for the Edwards-Anderson spin
 * glass, arXiv:1710.09025:
 *   Hamiltonian            Sec. II.A, Eq. (1): H = -sum_<ij> J_ij S_i S_j
 *                          (plus -sum_i h_i S_i, an addition for the field gradient)
 *   anneal step            Sec. II.B: resample beta -> beta' with copy numbers of mean
 *                          proportional to exp[-(beta'-beta) E_i], then N_S Metropolis sweeps
 *   spin selection         Sec. III.A: checkerboard (parity-0 sites, then parity-1 sites)
 *   free energy            Sec. II.B: free-energy perturbation, beta F_k = -N ln 2 - sum ln Q_l
 *   family entropy         Sec. II.B, Eq. (2)-(3): S_f, rho_s = R / e^{S_f}
 *   overlap                Sec. V.A: overlap histogram of uncorrelated replicas
 *   observable averages    Sec. V.A, Eq. (9)
 *
 * Conventions common to all calls
 *   - Lattice: D in {2,3}, even L >= 2, periodic, N = L^D sites; site index
 *     i = x + L y + L^2 z.  Bond (d, i) joins i and i + e_d; couplings are
 *     passed as J[d*N + i] (D*N floats), the field as h[i] (N floats).
 *   - Pointers named host_* or documented "host" are host memory owned by the
 *     caller; the library copies from/to them before returning.  All device
 *     memory is owned by the context (or by the caller for the *_ws variant).
 *   - Every call returns PA_OK (0) or a negative PA_E* status; nothing aborts
 *     or throws across the ABI.  pa_last_error() gives a message.
 *   - One context per CUDA stream / host thread; calls on one context are not
 *     thread-safe.
 *   - Results are bit-for-bit reproducible: every random number comes from a
 *     counter-based Philox4x32-10 stream keyed by (seed, instance, tag) and
 *     addressed by (temperature index, sweep, site, replica); every rounding
 *     that feeds the trajectory is specified (see the library's design notes).
 */
#ifndef PAMC_GB300_PA_H
#define PAMC_GB300_PA_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    PA_OK = 0,
    PA_EINVAL = -1,   /* invalid argument (message says which)                 */
    PA_ENOMEM = -2,   /* device or host allocation failed / workspace too small */
    PA_ECUDA = -3,    /* a CUDA call failed (message has the CUDA error)        */
    PA_ETIMEOUT = -4, /* a bounded device wait gave up                           */
    PA_EDONE = -5,    /* the schedule is finished                                */
    PA_ESTATE = -6,   /* call not valid in the current state                     */
    PA_EEMPTY = -7    /* the population died out (nearest-integer resampling)    */
};

enum { PA_PM1 = 0, /* J in {-1,+1}, no field */
       PA_REAL = 1 /* FP32 couplings, optional FP32 field */ };

/* Resampling (Sec. II.B: replica i gets on average R(beta') w_i / sum_j w_j
 * copies, w_i = exp[-(beta'-beta) E_i]). */
enum { PA_RESAMPLE_MULTINOMIAL = 0, /* R(beta') independent draws: population exactly R(beta') */
       PA_RESAMPLE_NEAREST = 1 };   /* floor(tau_i) copies, one more with probability
                                     * tau_i - floor(tau_i), tau_i = R(beta') w_i / sum w:
                                     * population R(beta') in expectation */

enum { PA_LAYOUT_AUTO = 0,   /* PM1 -> packed, REAL -> int8                          */
       PA_LAYOUT_PACKED = 1, /* PM1 only: 64 replicas per uint64 word, bit 1 = spin -1 */
       PA_LAYOUT_I8 = 2 };   /* one int8 (+1/-1) per spin, rows of N padded to 16     */

typedef struct {
    int32_t layout;          /* PA_LAYOUT_*                                            */
    int32_t accumulate_grad; /* 1: keep per-temperature <s_i s_j>, <s_i> population counts */
    uint32_t rng_instance;   /* 24-bit instance id in the Philox counter               */
    uint32_t rng_tag;        /* 4-bit tag: independent populations (overlap)           */
    int32_t threads;         /* tile override: 0 = tuned default; else threads per block */
    int32_t groups_per_block;/* tile override: 0 = tuned default (packed layout)       */
    /* dynamic population (Sec. III.D, Eq. 6): host array of n_temps replica
     * counts, populations[k] >= 1, the population R(beta_k) at temperature k
     * (exact for the multinomial scheme, the expectation for the
     * nearest-integer one).  NULL keeps R throughout. */
    const int32_t* populations;
    int32_t resampling;      /* PA_RESAMPLE_*                                          */
    /* replica slots (buffers, grids).  Multinomial: max(R, capacity), and every
     * populations[k] must fit.  Nearest-integer: 0 selects T + 64 + 8 ceil(sqrt T)
     * for the largest target T; copies placed beyond the capacity are dropped.
     * Kernels then read the population from device memory, so one CUDA graph
     * serves any population sequence. */
    int32_t capacity;
    /* isoenergetic cluster moves (Sec. II.C), zero field only: at steps k >= 1
     * with icm_beta_lo <= beta_k <= icm_beta_hi (icm_beta_hi <= 0: every step),
     * N_S/2 sweeps, then two rounds of moves on disjoint random pairs (R moves),
     * then the remaining sweeps */
    int32_t icm;
    double icm_beta_lo, icm_beta_hi;
    /* real couplings: 1 takes the specified Metropolis rule (spec_expf
     * threshold, Sec. II.B) in every lane instead of the verified guard band
     * of pa_check_accept_band; the decisions, and so every result, are the
     * same (0: the band where it is verified on the device) */
    int32_t exact_accept;
    /* 1: the replica gather of a resampling step (slot j takes replica
     * parent[j], Sec. II.B) runs as its own launch before the sweeps, which
     * then work in place; 0: it is fused into the first sweep launch's tile
     * load.  Same results either way.  Single contexts only. */
    int32_t separate_gather;
    /* a shard of one population spread over several contexts (one per GPU;
     * Sec. V.A: replicas numbered globally, every rank holding an equal share):
     * the context holds the global replicas [shard_offset, shard_offset + R)
     * of shard_total (shard_offset a multiple of 1024; +-J couplings, packed
     * layout, fixed population, multinomial resampling).  Step 0 runs with
     * pa_anneal_step; later steps with the pa_shard_* phases below.
     * shard_total = 0: not a shard. */
    int32_t shard_offset, shard_total;
} pa_options;

/* Per-temperature observables (Sec. II.B, Eq. 2-3; Sec. V.A, Eq. 9). */
typedef struct {
    double E_mean;   /* (1/R) sum_r E_r after the N_S sweeps at beta_k             */
    double E2_mean;  /* (1/R) sum_r E_r^2                                           */
    double C;        /* specific heat beta_k^2 (E2_mean - E_mean^2) / N             */
    double lnQ;      /* ln Q_k, Q_k = (1/R) sum_r exp[-(beta_k-beta_{k-1}) E_r]; 0 at k=0 */
    double betaF;    /* beta_k F_k = -N ln 2 - sum_{l=1..k} ln Q_l                  */
    double S_f;      /* family entropy -sum_f nu_f ln nu_f                           */
    double rho_s;    /* R / exp(S_f)                                                 */
    int64_t R;       /* population size                                              */
} pa_obs;

typedef struct pa_ctx pa_ctx;

/* Fills *opt with the defaults (auto layout, no grad, instance 0, tag 0, tuned). */
int pa_options_default(pa_options* opt);

/*
 * pa_create -- allocate a population of R replicas on the current CUDA device.
 *   D, L      lattice (D in {2,3}, L even; 3D: 2 <= L <= 16 for PA_PM1, <= 12 for
 *             PA_REAL; 2D: L <= 64 for PA_PM1, <= 32 for PA_REAL)
 *   kind      PA_PM1 (J exactly +-1, h must be NULL or all zero) or PA_REAL
 *             (|J|,|h| < 4096; magnitudes below 2^-73 are flushed to zero so
 *             that energies are exact fixed-point integers at scale 2^-96)
 *   J         host, D*N floats, J[d*N+i] couples i and i+e_d
 *   h         host, N floats or NULL (PA_REAL only)
 *   R         replicas, 1 <= R <= 2^26 (with pa_options.populations or the
 *             nearest-integer scheme: see pa_options for R, targets and capacity)
 *   betas     host, n_temps doubles, betas[0] == 0, non-decreasing, finite
 *   n_sweeps  Metropolis sweeps per temperature (N_S >= 0)
 *   seed      Philox key
 *   opt       NULL for defaults
 *   stream    cudaStream_t to run on (NULL = legacy default stream)
 * J, h and betas are deep-copied; the caller may free them on return.
 * Errors: PA_EINVAL (bad argument), PA_ENOMEM, PA_ECUDA.  *out is NULL on error.
 */
int pa_create(pa_ctx** out, int D, int L, int kind, const float* J, const float* h, int R,
              const double* betas, int n_temps, int n_sweeps, uint64_t seed,
              const pa_options* opt, void* stream);

/* Device workspace in bytes that pa_create_ws needs for these sizes. */
int pa_workspace_size(int D, int L, int kind, int R, int n_temps, const pa_options* opt,
                      size_t* bytes);
/* As pa_create, but all large device buffers are carved from a caller-owned
 * device allocation `workspace` of at least pa_workspace_size() bytes (256-byte
 * aligned).  The caller keeps it alive until pa_destroy. */
int pa_create_ws(pa_ctx** out, int D, int L, int kind, const float* J, const float* h, int R,
                 const double* betas, int n_temps, int n_sweeps, uint64_t seed,
                 const pa_options* opt, void* stream, void* workspace, size_t workspace_bytes);

/* One anneal step at temperature index k = pa_current_step(): resampling from
 * beta_{k-1} (k > 0), N_S sweeps at beta_k, energies and observables.
 * Asynchronous on the context's stream.  PA_EDONE after the last temperature. */
int pa_anneal_step(pa_ctx* ctx);
/* n_steps steps (-1: the rest of the schedule) captured once into a CUDA graph
 * and replayed; identical results to repeated pa_anneal_step. */
int pa_anneal(pa_ctx* ctx, int n_steps);
int pa_current_step(const pa_ctx* ctx);
int pa_synchronize(pa_ctx* ctx);

/* Observables of a completed step k (synchronises); out->R is the population
 * at beta_k.  PA_EEMPTY if the population had died out by step k. */
int pa_observables(pa_ctx* ctx, int k, pa_obs* out);
/* beta F_k for every completed k (host, n_temps doubles; unfinished k -> NaN). */
int pa_free_energy(pa_ctx* ctx, double* host_betaF);

/*
 * pa_grad -- backward pass of the free-energy estimate.  For the function
 *   f = sum_k gbar[k] * beta_k F_k
 * returns df/dJ_b = sum_k gbar[k] (-beta_k c_b(k) / R_k) and
 *         df/dh_i = sum_k gbar[k] (-beta_k m_i(k) / R_k),
 * with c_b(k) = sum_r S_i S_{i+e_d} and m_i(k) = sum_r S_i the exact integer
 * population sums after the sweeps at beta_k (d(beta F)/dJ = -beta <S_i S_j>,
 * d(beta F)/dh = -beta <S_i>; from Eq. 1 and Z = sum exp(-beta H)), R_k the
 * population at beta_k.
 * Needs accumulate_grad; gbar host n_temps doubles (entries for steps not yet
 * run must be 0); dJ host D*N doubles, dh host N doubles (or NULL). FP64,
 * summed over k in increasing order. */
int pa_grad(pa_ctx* ctx, const double* gbar, double* dJ, double* dh);

/* Histogram of the overlap sum_i S^a_i S^b_i between slot r of two contexts of
 * the same lattice and R (Sec. V.A); hist host int64[N+1], index
 * (N + sum_i S^a_i S^b_i) / 2. */
int pa_overlap(pa_ctx* a, pa_ctx* b, int64_t* hist);

/* Verifies, on the current device (default stream, synchronises), the guard
 * band that real-coupling sweeps use to take the Metropolis decision of
 * Sec. II.B without evaluating the specified spec_expf in most lanes: a hardware
 * estimate g of exp(-x) brackets the specified threshold thr(x) as
 * trunc(g 2^32 (1 - 2^-14)) <= thr(x) <= trunc(g 2^32 (1 + 2^-14)) + 1.  Every
 * positive finite float x is checked (about 2^31 values, a few milliseconds).
 * violations (may be NULL): floats where the bracket fails (0 expected; real
 * contexts created on a device with violations take the specified rule in every
 * lane).  max_rel_dev (may be NULL): largest |g / spec_expf(-x) - 1| over
 * 0 < x <= 87.  Each context runs the check once per device and process at
 * creation.  PA_ECUDA on a CUDA error (message from pa_last_error(NULL)). */
int pa_check_accept_band(int64_t* violations, double* max_rel_dev);

/* Copies of the current state to host memory (synchronise).  R below is the
 * current population: populations[last completed step] for the multinomial
 * scheme, the drawn population for the nearest-integer one (pa_sizes reports
 * it).  PA_EEMPTY once a nearest-integer resampling left no replica (every
 * later step does no work). */
int pa_get_spins(pa_ctx* ctx, int8_t* host_spins /* R*N, +1/-1, replica-major */);
/* Replicas [r0, r0 + n) only (0 <= r0, r0 + n <= R): n*N bytes, +1/-1. */
int pa_get_spins_range(pa_ctx* ctx, int r0, int n, int8_t* host_spins);
int pa_get_energies(pa_ctx* ctx, int64_t* host_E /* PM1: R values; REAL: 2R (lo, hi) of E*2^96 */);
int pa_get_parents(pa_ctx* ctx, int32_t* host_parent /* R: parent of slot j at the last resampling */);
int pa_get_family(pa_ctx* ctx, int32_t* host_family /* R: initial ancestor of slot j */);
/* Grad counts (accumulate_grad): cJ n_temps*D*N, ch n_temps*N int64, host. */
int pa_get_grad_counts(pa_ctx* ctx, int64_t* host_cJ, int64_t* host_ch);
int pa_sizes(const pa_ctx* ctx, int* D, int* L, int* N, int* R, int* n_temps, int* layout);

/* Checkpoint / resume.  A checkpoint is the state the next step reads (the
 * spins in use, energies, parents, families, per-temperature accumulators,
 * populations, gradient counts) behind a header that pins the configuration.
 * pa_checkpoint_save (synchronises) writes pa_checkpoint_size() bytes to a
 * host buffer; pa_checkpoint_load restores them into a context created with
 * the same arguments and options (PA_EINVAL otherwise), after which the run
 * continues exactly as the saved one would have. */
int pa_checkpoint_size(const pa_ctx* ctx, size_t* bytes);
int pa_checkpoint_save(pa_ctx* ctx, void* host_buf, size_t bytes);
int pa_checkpoint_load(pa_ctx* ctx, const void* host_buf, size_t bytes);

/* Per-phase timing with CUDA events recorded on the context's stream around
 * each phase of pa_anneal_step (off by default; not recorded inside pa_anneal
 * graphs).  Phases: 0 init, 1 resampling (weights..parents), 2 replica gather,
 * 3 sweeps (+ energies), 4 observables. */
enum { PA_PHASE_INIT = 0, PA_PHASE_RESAMPLE, PA_PHASE_GATHER, PA_PHASE_SWEEP, PA_PHASE_OBSERVE,
       PA_NPHASE };
int pa_profile(pa_ctx* ctx, int enable);
/* Synchronises; writes the summed milliseconds and the number of timed phase
 * instances per phase since the previous call (host ms[PA_NPHASE], n[PA_NPHASE],
 * either may be NULL), and *launches = kernels enqueued by this context so far. */
int pa_phase_times(pa_ctx* ctx, double* ms, int64_t* n, int64_t* launches);

/* ---------------- batched instances ----------------
 * Many disorder realisations annealed together: one persistent sweep launch
 * covers every instance's replica tiles (mixed L, +-J and real couplings),
 * resampling and observables run as one launch each for all instances, and
 * pa_batch_run captures the schedule into a CUDA graph.  All instances share
 * D, the schedule (betas, n_sweeps) and the Philox key (seed); each has its
 * own rng_instance, so its results are identical to a single-instance
 * context created with the same arguments.  Sweep shapes (groups per block of
 * the packed tiles, persistent grid size) are chosen by timing candidates on
 * the first step with k >= 1; every candidate gives bit-identical results. */
typedef struct {
    int L, kind;              /* lattice size, PA_PM1 or PA_REAL                    */
    const float* J;           /* host, D*N                                          */
    const float* h;           /* host, N or NULL                                    */
    int R;                    /* replicas                                           */
    uint32_t rng_instance;    /* < 2^24, distinct per instance                      */
} pa_inst_desc;
typedef struct pa_batch pa_batch;
/* opt: layout must be AUTO; accumulate_grad must be 0; threads = 0 tunes the
 * sweep shapes, threads = -1 keeps the defaults.  Errors as pa_create. */
int pa_batch_create(pa_batch** out, int D, int n_inst, const pa_inst_desc* descs,
                    const double* betas, int n_temps, int n_sweeps, uint64_t seed,
                    const pa_options* opt, void* stream);
int pa_batch_step(pa_batch* b);               /* one temperature for every instance       */
int pa_batch_run(pa_batch* b, int n_steps);   /* n_steps (-1: the rest), graph-captured   */
int pa_batch_current_step(const pa_batch* b);
/* the context of instance i (owned by the batch: do not destroy); all getters
 * (pa_observables, pa_get_spins, ...) work on it, and pa_anneal_step on it runs
 * the same step with per-instance launches instead of the batched ones. */
int pa_batch_instance(pa_batch* b, int i, pa_ctx** out);
/* chosen sweep configuration: persistent blocks, packed groups-per-block
 * multiplier (1 or 2), and the tuned sweep time of one step in ms */
int pa_batch_sweep_config(const pa_batch* b, int* blocks, int* gpb_mult, double* ms);
const char* pa_batch_last_error(const pa_batch* b);  /* NULL: last pa_batch_create failure */
void pa_batch_destroy(pa_batch* b);

/* ---------------- shards of one population (Sec. V.A) ----------------
 * One population of shard_total replicas split over several contexts, one per
 * GPU, each holding the replicas [shard_offset, shard_offset + R) (the
 * paper's global replica numbering); after every resampling each shard again
 * holds its own range of slots (equal shares, the paper's load balancing).
 * Random streams follow the global replica numbers, and the summation order
 * of the weights is that of one context, so a sharded run gives bit for bit
 * the results of one context of shard_total replicas (spins, energies,
 * parents, families, ln Q, beta F).  Step 0 runs with pa_anneal_step; a step
 * k >= 1 runs these phases in order, the caller exchanging between them (in
 * shard order): every phase synchronises the context's stream.
 *   1. pa_shard_emin: this shard's lowest energy after step k-1 (the caller
 *      takes the minimum over the shards).
 *   2. pa_shard_weights(E_min of all shards): resampling weights and the two
 *      lowest summation levels of the local weights blocks; writes the
 *      rs = ceil(R / 1024) local block totals (host doubles).
 *   3. pa_shard_prefix(all shards' block totals, ceil(shard_total / 1024),
 *      concatenated in shard order): the higher levels (identical on every
 *      shard) and the local cumulative weights; writes the rs local block
 *      maxima.
 *   4. pa_shard_draw(all shards' block maxima): S, ln Q and beta F of step k
 *      (the same on every shard), then the shard_total draws, of which the
 *      local ones are counted; *copies = the copies of local replicas.
 *   5. pa_shard_copies: the global parent index and family of every local
 *      copy (host int32 [copies] each), in slot order.  The copies of shard s
 *      take the global slots [sum_{t<s} copies_t, ...).  The caller sends each
 *      slot's parent, family and replica to the shard owning the slot.
 *   6. pa_shard_pack(replicas, n, dst): the spins of n increasing global
 *      replica indices of this shard packed into ceil(n/64) groups of N
 *      uint64 words (replica i at bit i % 64 of group i / 64) at dst (host,
 *      or device memory of this GPU when dst_on_device).
 *   7. pa_shard_finish(groups, n_groups, parent, family): the incoming
 *      replica groups (at most ceil(R/64) + 64), and for each of the R local
 *      slots the index of its parent among them and its family; then the N_S
 *      sweeps of step k (the gather reading the incoming replicas) and the
 *      local observables.
 * pa_shard_sums(k): the exact local sum of E and E^2 after step k and the
 * local lowest energy (the caller adds the shards' sums for <E>, <E^2>).
 * pa_observables on a shard gives the global ln Q and beta F and the local
 * averages.  Errors: PA_EINVAL, PA_ESTATE (not a shard, or no step to run),
 * PA_ECUDA. */
int pa_shard_emin(pa_ctx* ctx, int64_t* emin);
int pa_shard_weights(pa_ctx* ctx, int64_t emin_global, double* host_block_totals);
int pa_shard_prefix(pa_ctx* ctx, const double* host_all_totals, double* host_block_max);
int pa_shard_draw(pa_ctx* ctx, const double* host_all_block_max, int32_t* copies);
int pa_shard_copies(pa_ctx* ctx, int32_t* host_parent, int32_t* host_family);
int pa_shard_pack(pa_ctx* ctx, const int32_t* host_replicas, int n, void* dst, int dst_on_device);
int pa_shard_finish(pa_ctx* ctx, const void* groups, int n_groups, int src_on_device,
                    const int32_t* host_parent, const int32_t* host_family);
int pa_shard_sums(pa_ctx* ctx, int k, int64_t* sums /* 3: sum E, sum E^2, lowest E */);

/*
 * pa_resample_static -- the resampling step of pa_anneal_step for a +-J
 * population, for callers that cannot allocate device memory: allocator-less
 * embedded runtimes, and hosts whose memory manager owns every device byte and
 * hands the library only its input and output buffers.  The paper has no
 * counterpart; it exists for those callers.  No cudaMalloc, cudaFree or
 * allocating library call is made: the scratch (weights, prefix sums, copy
 * numbers, families) lives in one file-scope device array of
 * PA_STATIC_SCRATCH_BYTES, which every GPU that loads the library keeps until
 * the process exits.
 *   d_E        device, R int32 energies (+-J only: integer energies of the
 *              population at beta_prev, i.e. after the sweeps of step k-1);
 *              E_min is taken as the minimum of d_E (pa_anneal_step takes the
 *              same minimum from the previous step's observables)
 *   R          1 <= R <= PA_STATIC_MAX_R; larger R returns PA_EINVAL
 *   beta_prev, beta_next   finite, beta_prev <= beta_next
 *   k          temperature index of the step (selects the draw stream)
 *   seed, rng_instance (< 2^24), rng_tag (< 16)   as in pa_create / pa_options
 *   d_parent   device, R int32 out: slot j takes replica d_parent[j]
 *   d_lnQ      device, 1 double out: ln Q of this step
 *   stream     cudaStream_t (NULL = legacy default stream)
 * Results are bit-identical to what pa_anneal_step computes for the same
 * energies and step (parents and ln Q).  The first call on a device looks up
 * the array's device address with cudaGetSymbolAddress (that device must be
 * current) and caches it for the life of the process; make that first call
 * before any stream capture.  A device reset (cudaDeviceReset) after the first
 * call is not supported: the cached address would be stale.  Every call shares
 * the one array and keeps the last call's contents (each call clears what it
 * needs zeroed): calls whose kernels overlap on the GPU (two streams, two host
 * threads) race and must be serialised by the caller.
 * Errors: PA_EINVAL, PA_ECUDA; message in pa_last_error(NULL).
 */
#define PA_STATIC_MAX_R 65536
#define PA_STATIC_SCRATCH_BYTES (2u * 1024u * 1024u)
int pa_resample_static(const int32_t* d_E, int R, double beta_prev, double beta_next, int k,
                       uint64_t seed, uint32_t rng_instance, uint32_t rng_tag,
                       int32_t* d_parent, double* d_lnQ, void* stream);

const char* pa_last_error(const pa_ctx* ctx); /* NULL ctx: last pa_create failure */
void pa_destroy(pa_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
