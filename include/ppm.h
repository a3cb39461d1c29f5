/*
 * ppm.h -- C ABI of libppm: hypothesis-tested progressive kernel estimation
 * (FPPM, and the VM part of VCM+) on one GB300 (sm_103a).
 *
 * Method: "Hypothesis Testing for Progressive Kernel Estimation and VCM
 * Framework" (Lin, Hu, Jia, Li).  Every iteration i the caller hands in the
 * iteration's photons (light vertices); the library
 *   1. builds a hashed uniform grid over them (cell key + stable LSD radix
 *      sort + cell ranges) -- the range-search structure of Sec. 5.1;
 *   2. gathers, for every hit point, the photons inside its disk of radius
 *      r_i, maps them into the unified 2D space of Eq. (map-function), and
 *      accumulates per group (2 equi-areal annuli x 6 sectors, Sec. 3.2.1 /
 *      6.1.1) the count, the sum of psi and the sum of psi^2 (Sec. 5.1 step 2);
 *   3. evaluates the ANOVA F statistic of Eq. (f-statistic) with m = t*J
 *      samples per group (Sec. 3.2.1, 5.1), compares it with the critical
 *      value F_c of F(11, 12(m-1)) at significance alpha_F (Sec. 3.2.2), and
 *      applies Eq. (radiusupdate); the window of samples is kept while the
 *      radius is kept and cleared when it shrinks (Sec. 5.1);
 *   4. accumulates the progressive estimate of Eq. (progressive-VCM-estimator):
 *      tau += Phi_i / (pi r_i^2).  For VCM+ every gathered pair carries the
 *      balance-heuristic merge weight of Eq. (mis-weight) (Sec. 4.2).
 *
 * Conventions (all entry points):
 *   - Return PPM_OK (0) or a negative PPM_E* code; ppm_strerror() names it.
 *   - Pointers in ppm_hitpoints / ppm_photons and output pointers are DEVICE
 *     pointers on the current CUDA device, borrowed for the duration of the
 *     work the call enqueues (stream-ordered); the library never frees them.
 *   - All work is enqueued on the stream given to ppm_create (or
 *     ppm_set_stream).  No entry point synchronizes the host except
 *     ppm_create, ppm_stats, ppm_get_state/ppm_set_state (which wait for
 *     their own copies) and ppm_destroy.
 *   - Floating-point layouts are row-major: an "n x 3" array holds x,y,z of
 *     element 0, then of element 1, ...
 *   - Packed directions ("snorm8") are uint32 words holding four signed
 *     bytes (x | y<<8 | z<<16 | 0<<24), each round(127 * component).
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef PPM_H
#define PPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PPM_OK        0
#define PPM_EINVAL   (-1)   /* bad argument (NULL, size, layout, range) */
#define PPM_ENOMEM   (-2)   /* device allocation failed */
#define PPM_ECUDA    (-3)   /* a CUDA runtime call or launch failed */
#define PPM_ETIMEOUT (-4)   /* a bounded device-side wait gave up */
#define PPM_ESTATE   (-5)   /* call out of order (iteration sequence) */
#define PPM_EINCOMPLETE (-6) /* a gather skipped cells: a hit point's sphere
                               spanned more grid cells than a hash block, so
                               some of its photons were not gathered */

#define PPM_NGROUPS 12      /* 2 annuli x 6 sectors, Sec. 6.1.1 */

typedef struct ppm_ctx ppm_ctx;  /* opaque; owned by the library */

/* Hit points (eye vertices / gather points, Sec. 3.1), fixed for the life of
 * a context.  pos, u, v: n x 3 float; (u, v) is an orthonormal tangent frame
 * of Eq. (map-function).  nq: n packed snorm8 surface normals, or NULL for a
 * single-surface scene (no same-surface filter).  rho: n x 2 float
 * (rho_vm_h, rho_vc_h), the eye-side pdf ratios of the VCM+ merge weight;
 * required iff params->vcm. */
typedef struct {
    int64_t n;
    const float* pos;
    const float* u;
    const float* v;
    const uint32_t* nq;
    const float* rho;
} ppm_hitpoints;

/* Photons (light vertices) of one iteration.  pos: n x 3 float.  flux: n
 * float (channels = 1) or n x 3 float RGB (channels = 3).  J: light
 * sub-paths emitted this iteration = samples per group per iteration
 * (Sec. 3.2.1); must be >= 2 and the same in every iteration of a context.
 * nq: n packed snorm8 normals, or NULL (then the hit points' normals are
 * ignored too).  VCM+ only: rho n x 2 float (rho_vm_l, rho_vc_l) and wq n
 * packed incoming directions. */
typedef struct {
    int64_t n;
    int64_t J;
    const float* pos;
    const float* flux;
    int32_t channels;
    int32_t pad;
    const uint32_t* nq;
    const float* rho;
    const uint32_t* wq;
} ppm_photons;

/* Method parameters.  ppm_default_params() fills the paper's defaults. */
typedef struct {
    double alpha_f;     /* significance level alpha_F, 0.01 (Sec. 6.1.1) */
    float k;            /* shrinking ratio of Eq. (radiusupdate), 0.7 (Sec. 6.1.1) */
    float rmin_ratio;   /* r_min = rmin_ratio * r0, 0.001 (Sec. 6.1.2) */
    float cell_factor;  /* grid cell edge = cell_factor * max radius along y and
                           z (half of it along x), in [0.5, 4]; 1 */
    int32_t channels;   /* flux channels of every iteration: 1 or 3 */
    int32_t rgb_test;   /* 0: F-test on luminance (default); 1: one F-test per
                           RGB channel, reject if any rejects (Sec. 5.1) */
    int32_t vcm;        /* 1: weight samples by the VCM+ merge weight */
    float n_vm;         /* VCM+: light sub-paths used for merging; 0 = J */
    int32_t mapping;    /* gather traversal: 0 = each thread walks its own cells,
                           1 / 2 = warp walks the union of its 32 hit points'
                           cells (32 / 64-entry in-disk queues per lane),
                           3 = union walk with one pair queue per warp and
                           fixed-point group sums (one tested channel:
                           PPM_EINVAL with rgb_test), 4 = a warp per hit point
                           with shuffle-reduced group sums (one flux channel:
                           PPM_EINVAL with channels = 3).  The features of
                           the learned proposer and CPPM's count test always
                           run traversal 0. */
    int32_t tile;       /* batches: hit points per tile of the persistent
                           gather, a multiple of 64 in [64, 1024]; 0 = 64.
                           Contexts ignore it.  Results do not depend on it. */
    int32_t test;       /* 0: the ANOVA F-test of the paper (FPPM, default);
                           1: CPPM's chi-square test (Sec. 3.2.3, settings of
                           Sec. 6.1.1): reject iff Pearson's X^2 of the
                           window's in-disk counts c_g over the 12 equal-area
                           groups exceeds chi_c, the (1 - alpha_f) quantile of
                           chi^2(11) (24.725 at alpha_f = 0.01).  The counts
                           alone decide, not the flux.  X^2 is computed from
                           exact integers, (12 sum c_g^2 - C^2) / C with
                           C = sum c_g (0 when C = 0), and is what the F
                           array of ppm_get_state then holds.  Contexts only
                           (batches: PPM_EINVAL); not with rgb_test, features
                           or the proposer (PPM_EINVAL); traversal 0. */
    int32_t wait_limit; /* polls before a wait between the blocks of the grid's
                           sort gives up (decoupled look-back); 0 = the default
                           (2^22, each poll sleeping ~32 ns).  The waits always
                           end on a healthy GPU; a small limit only exists to
                           test the error path (PPM_ETIMEOUT below). */
    int32_t reserved[3];
} ppm_params;

/* Per-iteration counters of the last ppm_gather_test_update. */
typedef struct {
    int32_t iter;          /* last completed iteration (0 = none) */
    int32_t flags;         /* device error flags, sticky for the life of the
                              context; bit 0: a sphere spanned more cells
                              than a hash block (results incomplete; the
                              counters' call returns PPM_EINCOMPLETE); bit 1:
                              a window length outside the F_c table (from
                              ppm_set_state), clamped; bit 2: a wait between
                              the blocks of the grid's sort gave up (the
                              grid is unusable: the cell ranges, the permute
                              and every later gather of the context do
                              nothing, and the counters' call returns
                              PPM_ETIMEOUT) */
    int64_t pairs;         /* in-disk photon/hit-point pairs gathered */
    int64_t candidates;    /* photons visited in the scanned cells */
    int64_t rejects;       /* hit points whose null hypothesis was rejected */
    int64_t pairs_total;   /* pairs summed over all iterations */
    float r_max;           /* largest radius after the update */
    float cell;            /* grid cell edge along y and z used by the last
                              build (the edge along x is half of it) */
    int32_t launches;      /* kernels launched by the last build + gather */
    float gather_ms;       /* batches: device time of the last gather launch
                              (events recorded around it); contexts: -1 */
    int64_t proposals;     /* radii shrunk by the learned proposer */
} ppm_iter_stats;

/* State per hit point, in the caller's hit-point order (device pointers;
 * any may be NULL to skip it).  ntc = 3 if rgb_test else 1.
 *   r: n float radius; t: n int32 iterations in the current window;
 *   counts: n x 12 int32 in-disk photons per group in the window;
 *   S, Q: n x ntc x 12 float window sums of psi and psi^2 per group;
 *   tau: n x channels double accumulated estimate sum; F: n float F of the
 *   last test (luminance / channel 0). */
typedef struct {
    float* r;
    int32_t* t;
    int32_t* counts;
    float* S;
    float* Q;
    double* tau;
    float* F;
} ppm_state_view;

void ppm_default_params(ppm_params* p);

/* Create a context over n hit points with initial radius r0 > 0 for all of
 * them and radius-bound exponent alpha in (0,1) (Eq. radiusupdate; 0.75 in
 * Sec. 6.1.2).  params may be NULL (defaults).  stream is a cudaStream_t (or
 * NULL for the legacy default stream).  Copies the hit points into a
 * spatially sorted internal layout; the caller may free its arrays once the
 * call returns.  Synchronizes the stream once.  *out is NULL on error. */
int ppm_create(const ppm_hitpoints* hp, float r0, float alpha,
               const ppm_params* params, void* stream, ppm_ctx** out);

/* Change the stream later work is enqueued on. */
int ppm_set_stream(ppm_ctx* ctx, void* stream);

/* Hit points traced anew (stochastic eye paths through each pixel, as in
 * SPPM, which the paper's distributed ray tracing stage follows, Sec. 7):
 * replace the positions, frames, normals and VCM+ ratios of all n hit
 * points before an iteration's ppm_build_grid / ppm_gather_test_update.
 * hp has the same count and order as at ppm_create: entry h is the same
 * pixel, whose radius, window statistics and estimate carry over.  The
 * context keeps the spatial order it computed at ppm_create.  hp->nq must
 * be given iff it was at create (the same-surface test stays on or off),
 * hp->rho when the context is VCM+.  The arrays may be reused once the
 * stream passes this work.  PPM_EINVAL on a count or array mismatch. */
int ppm_set_hitpoints(ppm_ctx* ctx, const ppm_hitpoints* hp);

/* Step 1 of an iteration (Sec. 5.1: build the range-search structure):
 * hash every photon to a grid cell of edge cell_factor * max_h r_h, sort
 * (cell, index) pairs with a stable radix sort, and copy the photons into
 * cell order.  The photon arrays may be reused once the stream passes this
 * work.  n = 0 is allowed (an iteration without photons). */
int ppm_build_grid(ppm_ctx* ctx, const ppm_photons* ph);

/* Steps 2-4 of iteration iter (Sec. 5.1 steps 2-4 and Eq. progressive-VCM-
 * estimator) over the grid of the last ppm_build_grid.  iter must be the
 * previous iteration + 1, starting at 1, with a grid built since
 * (PPM_ESTATE otherwise). */
int ppm_gather_test_update(ppm_ctx* ctx, int32_t iter);

/* Radiance estimate L = tau / iter (Eq. progressive-VCM-estimator) into out:
 * n float (channels = 1) or n x 3 float, device, caller's hit-point order. */
int ppm_radiance(ppm_ctx* ctx, float* out);

/* Copy the state out of / into the context (checkpoint / resume, tests).
 * Both wait for the copies to finish.  set_state leaves the iteration
 * counter untouched; use ppm_set_iteration to resume a sequence.
 * get_state copies the state and then returns PPM_ETIMEOUT or
 * PPM_EINCOMPLETE when the context's error flags hold bit 2 or bit 0 (see
 * ppm_iter_stats.flags). */
int ppm_get_state(ppm_ctx* ctx, const ppm_state_view* v);
int ppm_set_state(ppm_ctx* ctx, const ppm_state_view* v);
int ppm_set_iteration(ppm_ctx* ctx, int32_t iter);

/* Counters of the last iteration; waits for the stream.  *out is filled in
 * every case; the return value is PPM_ETIMEOUT if a bounded device wait of
 * the context has given up (flags bit 2), else PPM_EINCOMPLETE if a gather
 * skipped cells (flags bit 0), else PPM_OK. */
int ppm_stats(ppm_ctx* ctx, ppm_iter_stats* out);

/* One whole iteration fed from HOST memory: the grid build of
 * ppm_build_grid and the gather/test/update of ppm_gather_test_update for
 * iteration iter (Sec. 5.1 steps 1-4), with host_ph's arrays (same layout
 * and rules as ppm_photons, host pointers) first copied into one of two
 * context-owned device buffers, used in turn, on a private copy stream.
 * With page-locked host arrays the copy of iteration i overlaps the gather
 * of iteration i - 1; pageable arrays work, without that overlap.  After
 * the gather the iteration's counters are copied to page-locked memory.
 * Returns without waiting.  The caller keeps host_ph's arrays unchanged
 * until ppm_stats_host has returned for this iteration (or the context's
 * stream has been synchronized).  PPM_ESTATE unless iter = last + 1.  The
 * device buffers grow (with one synchronization) when n grows. */
int ppm_iterate_host(ppm_ctx* ctx, const ppm_photons* host_ph, int32_t iter);

/* Counters of host-fed iteration iter, which must be one of the last two
 * ppm_iterate_host iterations (PPM_ESTATE otherwise): waits only for that
 * iteration's counter copy, not for later work.  gather_ms is -1.  Returns
 * PPM_ETIMEOUT / PPM_EINCOMPLETE from the flags as ppm_stats does. */
int ppm_stats_host(ppm_ctx* ctx, int32_t iter, ppm_iter_stats* out);

/* F-test critical values on their own (Sec. 3.2.2): out[t] = the
 * (1 - alpha_f) quantile of F(11, 12 (t J - 1)) for t = 1 .. t_max, FP64,
 * out[0] = 0.  out: device array of t_max + 1 doubles.  Enqueued on stream. */
int ppm_f_critical(int64_t J, double alpha_f, int32_t t_max, double* out, void* stream);

/* Chi-square critical value on its own (the count test of CPPM, Sec. 3.2.3):
 * out[0] = the (1 - alpha) quantile of chi^2(dof), FP64, dof in [1, 1000].
 * out: device array of one double.  Enqueued on stream. */
int ppm_chi2_critical(int32_t dof, double alpha, double* out, void* stream);

/* Stable LSD radix sort of (key, value) pairs on the low `bits` bits of the
 * keys (1..32), the sort that orders photons by grid bucket in
 * ppm_build_grid: pairs with equal keys keep their input order.  keys_in,
 * vals_in: n uint32 each (device, read only); keys_out, vals_out: n uint32
 * each (device, written; may alias the inputs).  n in [0, 2^32 - 1).
 * One kernel per 8-bit pass: the blocks of a pass wait for the counts of
 * earlier blocks (decoupled look-back).  Every such wait ends, because a
 * block waits only for blocks that started before it; each is capped all
 * the same, and were a cap ever reached the output order would be
 * unspecified.  Scratch (2n words + 2 KB per 2048 pairs + 4 KB) comes from
 * cudaMallocAsync on the stream and is released with cudaFreeAsync, so the
 * call does not block.  PPM_EINVAL for bad sizes or NULL pointers with
 * n > 0, PPM_ENOMEM if the scratch cannot be allocated. */
int ppm_sort_pairs(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                   uint32_t* vals_out, int64_t n, int32_t bits, void* stream);

/* ---- learned radius proposer (not in the paper) ----------------------------
 * A 12 -> 64 -> 64 -> 2 MLP with ReLU hidden layers: BF16 weights, FP32
 * biases and accumulation, every layer's input (features, h1, h2) rounded
 * to BF16 (nearest even); inference runs on the tensor cores.  The
 * gradient treats that rounding as the identity.  Input: 12 features of the window a
 * hit point's F-test just used -- log(1+C), log(1+t'), log i, r/r0,
 * log(r/r0), log(1+F), F/F_c, max_g S_g/S, min_g S_g/S, fraction of empty
 * groups, coefficient of variation of the group sums, max_g c_g/C (C, S:
 * window count and psi sum; channel 0).  Outputs: o0 = predicted
 * log(r_final / r), o1 = logit of "will be rejected within a few tests".
 * Weight blob (device, 16-byte aligned, PPM_MLP_BLOB_BYTES): W1 [64][12],
 * W2 [64][64], W3 [2][64] as bf16 row-major, then b1[64], b2[64], b3[2] as
 * float.  Master parameters (FP32, PPM_MLP_PARAMS floats): the same order. */
#define PPM_MLP_IN 12
#define PPM_MLP_HIDDEN 64
#define PPM_MLP_OUT 2
#define PPM_MLP_PARAMS (64 * 12 + 64 * 64 + 2 * 64 + 64 + 64 + 2)
#define PPM_MLP_BLOB_BYTES 10504

/* Allocate (enable != 0) or free the per-hit-point feature buffer; while it
 * exists every ppm_gather_test_update writes the features of its tests. */
int ppm_set_features(ppm_ctx* ctx, int32_t enable);
/* Features of the last iteration's tests into out (device, n x 12,
 * caller's hit-point order); PPM_ESTATE if features are not enabled. */
int ppm_get_features(ppm_ctx* ctx, float* out);
/* Enable (blob != NULL) or disable the proposer.  After the F-test update
 * of each iteration, a hit point the test did not reject gets
 * r <- max(r max(exp(o0), min_ratio), bound of Eq. radiusupdate) when
 * sigmoid(o1) > doom_threshold and o0 < 0, and its window is cleared; the
 * F-test keeps testing every radius.  The blob is borrowed (caller-owned)
 * until the proposer is disabled or the context destroyed. */
int ppm_set_mlp(ppm_ctx* ctx, const void* blob, float doom_threshold, float min_ratio);
/* Inference: X n x 12 float, Y n x 2 float (device). */
int ppm_mlp_forward(const void* blob, const float* X, int64_t n, float* Y, void* stream);
/* Gradient of scale * sum_s [0.5 M0 (o0 - Y0)^2 + M1 BCE(o1, Y1)] over the
 * n samples (X n x 12, Y and M n x 2) with respect to the master
 * parameters, ADDED to grad (PPM_MLP_PARAMS floats); the loss is added to
 * *loss.  Forward passes use the blob's BF16 weights.  Deterministic: the
 * sums of each 128-sample tile go to scratch memory allocated on the stream
 * (at most about 5 MB) and are added in tile order, so equal inputs give
 * bitwise equal grad and loss.  PPM_ENOMEM if the scratch cannot be had. */
int ppm_mlp_grad(const void* blob, const float* X, const float* Y, const float* M, int64_t n,
                 float scale, float* grad, float* loss, void* stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, step >= 1) on master with
 * moments m, v; rewrites the blob from the new master and zeroes grad. */
int ppm_mlp_adam(float* master, float* grad, float* m, float* v, int32_t step, float lr,
                 void* blob, void* stream);
/* Blob from master (BF16 round to nearest even). */
int ppm_mlp_pack(const float* master, void* blob, void* stream);

/* ---- batches: many independent problems per launch --------------------
 * A batch holds n_problems independent problem instances (hit points,
 * radii, per-iteration photons, window statistics, estimates), each
 * exactly as one context would hold it: for the same mapping and cell
 * factor a problem's results are bit-identical to a context's (traversal
 * 4: identical counts, windows, radii and decisions; its lanes' partial
 * sums, and so the rounding of the window sums, can differ).  One
 * iteration of all of them is one grid build over all photons (the
 * problem id is mixed into the bucket hash and checked in the gather) and
 * ONE persistent gather launch whose resident blocks pull tiles of
 * params->tile hit points (64 by default) from an atomic queue, heaviest
 * problems first.  From the second
 * iteration on, the whole iteration is replayed as a CUDA graph on a
 * private stream ordered after the caller's stream. */
typedef struct ppm_batch ppm_batch;

/* hp: n_problems hit-point sets (device arrays as for ppm_create); r0:
 * n_problems initial radii (host); J: n_problems light paths per iteration
 * (host) -- every iteration problem p must bring exactly J[p] photons;
 * cell_factor: n_problems grid cell factors in [0.5, 4] (host; from the
 * autotuner) or NULL for params->cell_factor.  Normals: for every problem
 * or for none.  Synchronizes the stream; copies the hit points. */
int ppm_batch_create(int32_t n_problems, const ppm_hitpoints* hp, const float* r0,
                     const int64_t* J, float alpha, const ppm_params* params,
                     const float* cell_factor, void* stream, ppm_batch** out);

/* Iteration iter (previous + 1, from 1) of every problem; ph: n_problems
 * photon sets.  The photon arrays are read by work ordered after the
 * caller's stream at the time of the call and must stay valid until the
 * caller's stream passes this call. */
int ppm_batch_iterate(ppm_batch* b, const ppm_photons* ph, int32_t iter);

/* Radiance of one problem into out (device, that problem's n or n x 3). */
int ppm_batch_radiance(ppm_batch* b, int32_t problem, float* out);

/* State of one problem (as ppm_get_state, error returns included); waits. */
int ppm_batch_get_state(ppm_batch* b, int32_t problem, const ppm_state_view* v);

/* Counters of the last iteration, one entry per problem; waits.  Returns
 * PPM_ETIMEOUT / PPM_EINCOMPLETE from the batch's flags as ppm_stats does. */
int ppm_batch_stats(ppm_batch* b, ppm_iter_stats* out);

/* 1 once the iteration has been captured into a CUDA graph, else 0. */
int ppm_batch_graph_ready(ppm_batch* b);

void ppm_batch_destroy(ppm_batch* b);

/* Frees everything the context owns (waits for the stream first). */
void ppm_destroy(ppm_ctx* ctx);

const char* ppm_strerror(int code);

/* ---- no-allocation variant (the paper has no counterpart) ----------------
 * ppm_sort_pairs_noalloc: the same stable radix sort as ppm_sort_pairs, with
 * the same arguments, results and error codes (computed by three kernels a
 * pass, with no waits between blocks), for callers that cannot call
 * cudaMalloc while they run -- real-time loops that cannot pay for an
 * allocator call or the synchronization it may bring, hosts whose device
 * memory belongs to another allocator.  It calls no cudaMalloc, cudaFree
 * or other allocating routine: its scratch is a fixed device array of the
 * library, sized for PPM_NOALLOC_MAX_PAIRS = n pairs (2n + n/8 + 34 words,
 * 8.9 MB), which every GPU that loads the library holds until the process
 * exits.
 *   - n > PPM_NOALLOC_MAX_PAIRS returns PPM_EINVAL (use ppm_sort_pairs).
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and keeps it for the
 *     life of the process: make that first call before any stream capture,
 *     and cudaDeviceReset after it is not supported.
 *   - All calls share the array: calls whose work overlaps on the GPU
 *     (several streams or host threads on one device) race on it; order
 *     them on one stream.  It keeps the last call's contents; nothing in it
 *     needs clearing between calls. */
#define PPM_NOALLOC_MAX_PAIRS (1 << 20)
int ppm_sort_pairs_noalloc(const uint32_t* keys_in, const uint32_t* vals_in,
                           uint32_t* keys_out, uint32_t* vals_out, int64_t n,
                           int32_t bits, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PPM_H */
