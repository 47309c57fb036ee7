/*
 * fmm.h -- C ABI of the GB300 (sm_103a) shift-free 2D FMM library (libfmm.so).
 *
 * The library evaluates the 2D log potential of N charges in the square
 * [0, box]^2,
 *
 *     phi(z_i) = sum_{j != i} q_j log|z_i - z_j|,
 *
 * with the shift-free Fast Multipole Method of Kajima, "Summation of certain
 * locally bilinear forms and its applications to the Fast Multipole Method"
 * (arXiv 2009.00767):
 *   - the computation box is split into a uniform quadtree of depth `levels`
 *     (Sec. 2.1 items 1-4);
 *   - for EVERY level k = 2..levels the multipole moments of every square are
 *     formed directly from the particles (the upward pass U-bar of Sec. 2.2.1,
 *     with no multipole-to-multipole shift);
 *   - each square's interaction list (Sec. 2.1 item 5) is converted into a
 *     local expansion (D-bar-1 of Sec. 2.2.1);
 *   - each level's local expansion is evaluated directly at the particles and
 *     the levels are summed (D-bar-2 of Sec. 2.2.1 by linearity, with no
 *     local-to-local shift);
 *   - the near field of the own and eight adjacent finest squares is summed
 *     directly (Sec. 2.1 E-2).
 * The vectors and bilinear forms of Sec. 2.2.1 are realised as complex
 * multipole moments of order p (coefficients 0..p) and the multipole-to-local
 * conversion of Greengard's 2D expansions (the paper's ref. [101]); the
 * conversion operators depend only on the relative offset of two squares
 * (40 offsets) and are built once per plan in FP64 (Sec. 4, Discussions (2)
 * and (3)).
 *
 * Conventions for every entry point:
 *   - Device pointers are CUDA global-memory pointers on the plan's device;
 *     the caller owns them.  Host pointers are ordinary host memory.
 *   - Arrays are dense and C-ordered.  xy is [N][2] (x then y), FP64.
 *   - Work is enqueued on the plan's CUDA stream and returns without waiting
 *     unless the entry point says otherwise.  Errors that only the device can
 *     see (a particle outside the box, a non-finite value) are latched in the
 *     plan and returned by fmm_sync; phi is then left unwritten for that call.
 *   - A plan is not thread-safe: calls on one plan must not overlap.
 *   - fmm_status values are returned; no entry point aborts or prints.
 */
#ifndef FMM_H_
#define FMM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmm_plan_s* fmm_plan_t;

typedef enum {
    FMM_OK = 0,
    FMM_ERR_INVALID_ARG = 1,   /* a host-side argument check failed */
    FMM_ERR_OUT_OF_BOX = 2,    /* a particle lies outside [0, box]^2 (device check) */
    FMM_ERR_NONFINITE = 3,     /* a coordinate or charge is NaN or infinite (device check) */
    FMM_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    FMM_ERR_OOM = 5,           /* device memory allocation failed in fmm_plan */
    FMM_ERR_TIMEOUT = 6,       /* a bounded device-side wait ran out */
    FMM_ERR_UNSUPPORTED = 7    /* valid request this build does not implement */
} fmm_status;

/* Arithmetic of the hot path.  FMM_FP64 runs every stage in FP64.  The mixed
 * modes run particle-side stages (P2M, L2P, P2P) in FP32 on coordinates local
 * to each square, keep the cross-level sum and the final phi in FP64, and run
 * M2L as stated: FP32 on the CUDA cores, or, for levels 6 and finer, on the
 * tensor cores (tcgen05) with FP32 accumulation in TF32 or BF16, where the x3
 * forms split each operand into parts to recover FP32-level accuracy
 * (3xTF32: hi + lo, three products; BF16x2: hi + lo in BF16, three products;
 * BF16x3: hi + mid + lo, six products).
 * Measured relative L2 error against the FP64 oracle at 2^20 uniform
 * particles, levels 8, p = 20: FP32 / 3xTF32 / BF16x3 about 2e-7, TF32 about
 * 3e-6, BF16 about 2e-5. */
typedef enum {
    FMM_FP64 = 0,
    FMM_MIXED_FP32 = 1,
    FMM_MIXED_TF32 = 2,
    FMM_MIXED_3XTF32 = 3,
    FMM_MIXED_BF16 = 4,
    FMM_MIXED_BF16X3 = 5,
    FMM_MIXED_BF16X2 = 6
} fmm_precision;

/* Per-call statistics of the last completed fmm_potential (valid after fmm_sync). */
typedef struct {
    int64_t n;                 /* particles */
    int levels, p, precision;
    double ms_total;           /* enqueue of the first stage to the end of the last, CUDA events */
    double ms_sort;            /* bin + scan + scatter */
    double ms_p2m;             /* moments of levels 2..levels */
    double ms_m2l;             /* interaction-list conversion of levels 2..levels */
    double ms_l2p;             /* local evaluation of levels 2..levels */
    double ms_p2p;             /* near field + final phi in input order */
    int64_t p2p_pairs;         /* ordered source-target pairs of the near field (counted on device) */
    int64_t max_leaf;          /* largest finest-square population */
    int kernel_launches;       /* kernels the library launched for that call */
    uint64_t workspace_bytes;  /* device memory the plan owns */
    double ms_m2l_tc;          /* the tensor-core M2L kernel alone (0 when none ran) */
    double ms_p2p_kernel;      /* the mixed path's near-field kernel alone (0 when none ran) */
    /* Mixed path: the near field (from the sort on), the coarse levels' chain (from the fine P2M
     * on: upward pass to levels levels-3 .. 2, M2L and L2P of levels 2..5) and the fine levels'
     * P2M and M2L run on three streams at once, so ms_p2m, ms_m2l and ms_l2p above are sums of
     * these spans and the stages overlap in time.  FP64 path: ms_m2l_fine = ms_m2l, the others 0. */
    double ms_p2m_fine;        /* P2M of the finest three levels */
    double ms_p2m_coarse;      /* the coarser levels' moments by the upward pass (M2M) */
    double ms_m2l_fine;        /* M2L of levels 6 and finer (tensor-core prep + kernel, or FP32) */
    double ms_m2l_coarse;      /* M2L of levels 2..5 on the CUDA cores */
} fmm_stats;

/* Create a plan for exactly n particles, a quadtree of depth `levels` over
 * [0, box]^2 and expansion order p (coefficients 0..p).
 *   out        receives the plan; unchanged on error.
 *   n          1 <= n <= 2^31 - 1.
 *   levels     0 <= levels <= 12 (levels 0 and 1 have no far field: the
 *              interaction list exists from level 2, Sec. 2.1 item 5).
 *   p          1 <= p <= 40 (FP64, FP32 and the batched form); the tensor-core
 *              modes (TF32, 3xTF32, BF16, BF16x2, BF16x3) take p <= 31 and return
 *              FMM_ERR_UNSUPPORTED above.
 *   box        side of the computation box (the paper's 5), > 0 and finite.
 *   precision  an fmm_precision value.
 *   stream     cudaStream_t to enqueue on (NULL = legacy default stream).
 * The plan allocates all device workspaces and builds the 40 M2L operators in
 * FP64 on the host (uploaded once); this cost is not part of fmm_potential.
 * Returns FMM_ERR_INVALID_ARG, FMM_ERR_UNSUPPORTED, FMM_ERR_OOM or
 * FMM_ERR_CUDA on failure. */
fmm_status fmm_plan(fmm_plan_t* out, int64_t n, int levels, int p, double box,
                    int precision, void* stream);

/* How many streams a mixed-precision call spreads its work over: 3 (the default: after the
 * fine levels' P2M the near field, the coarse levels' chain and the fine levels' M2L run at
 * once on the plan's stream and two streams of its own, joined back before L2P) or 1 (every
 * kernel in turn on the plan's stream, so that fmm_plan_stats times each kernel alone).  The
 * results are the same either way.  FMM_ERR_INVALID_ARG for another count or a NULL plan. */
fmm_status fmm_set_concurrency(fmm_plan_t plan, int streams);

/* Change the stream later calls enqueue on. */
fmm_status fmm_set_stream(fmm_plan_t plan, void* stream);

/* phi[i] = potential at particle i, in input order (the whole method above).
 *   xy   device, const double[n][2]; every point must lie in [0, box]^2.
 *   q    device, const double[n].
 *   phi  device, double[n]; written only if the device checks pass.
 * Asynchronous on the plan's stream; allocates nothing.  Device-detected
 * errors are reported by fmm_sync.  Coincident particles (r = 0) contribute 0. */
fmm_status fmm_potential(fmm_plan_t plan, const double* xy, const double* q, double* phi);

/* phi and the force field E = -grad phi at every particle, in input order (Sec. 3: the paper
 * times the method for "potential and force fields").  With phi = Re f(z), f analytic, grad phi
 * = (Re f', -Im f'): the far field differentiates each level's local expansion (sum over l of
 * l b_l w^(l-1) / s_k for w = (z - c) / s_k), the near field adds q_j (z - z_j) / |z - z_j|^2 of
 * the own and adjacent squares' particles; coincident particles contribute 0.
 *   xy, q, phi  as for fmm_potential.
 *   field       device, double[n][2]: (Ex, Ey) of particle i at field[2i], field[2i + 1];
 *               written only if the device checks pass.
 * Asynchronous on the plan's stream; allocates nothing.  Every precision. */
fmm_status fmm_potential_field(fmm_plan_t plan, const double* xy, const double* q, double* phi, double* field);

/* As fmm_potential, with HOST arrays: copies xy and q to plan-owned device
 * buffers, runs the method and copies phi back, then waits for the stream.
 * Host arrays may be pageable or pinned (pinned is faster).  Returns the
 * device-detected status, like fmm_sync; after a device-detected error the
 * contents of phi_host are unspecified.  Equivalent to fmm_potential_host_async
 * followed by fmm_sync. */
fmm_status fmm_potential_host(fmm_plan_t plan, const double* xy_host, const double* q_host,
                              double* phi_host);

/* fmm_potential_host without the wait: enqueues the uploads, the method and the download of phi
 * and returns.  The host arrays must stay valid, and xy_host / q_host unmodified, until the
 * next fmm_sync returns; phi_host is written when the call's work completes.  The plan holds two
 * staging sets, so in the mixed precisions successive calls overlap: a call's inputs go up (in
 * chunks, each binned as it lands) while the previous call computes, and its phi comes down while
 * the next one computes.  The device link carries about 200 GB/s each way on GB300, so this
 * overlap, not a faster copy, is what hides the transfers.  fmm_sync waits for every call since
 * the previous one and returns the first device-detected error among them. */
fmm_status fmm_potential_host_async(fmm_plan_t plan, const double* xy_host, const double* q_host,
                                    double* phi_host);

/* Wait for the plan's stream; return the first device-detected error of the
 * calls since the previous fmm_sync (FMM_OK if none) and clear it. */
fmm_status fmm_sync(fmm_plan_t plan);

/* Copy the statistics of the last synced call into *out (host struct). */
fmm_status fmm_plan_stats(fmm_plan_t plan, fmm_stats* out);

/* The finest square each particle of the last fmm_potential call was binned into (Sec. 2.1
 * items 1-4: ix = floor(x 2^levels / box) evaluated in FP64 in that order and clamped to
 * [0, 2^levels - 1], likewise iy), as the Morton key ix_0 iy_0 ix_1 iy_1 ... (bit 2b of the key
 * is bit b of ix, bit 2b + 1 is bit b of iy), in input order.
 *   keys  device, uint32_t[n], owned by the caller.
 * Asynchronous on the plan's stream (a device-to-device copy); allocates nothing.  Valid once
 * a call has been enqueued; FMM_ERR_INVALID_ARG for a null pointer. */
fmm_status fmm_leaf_keys(fmm_plan_t plan, uint32_t* keys);

/* Error-path test hook (no counterpart in the paper): with enable != 0, later calls run the
 * tensor-core M2L kernel with its copy producers switched off and its bounded mbarrier waits cut
 * to 4096 polls, so its first wait runs out with no copy or MMA in flight; the kernel then stores
 * nothing, frees its tensor memory and returns, phi is left unwritten and fmm_sync returns
 * FMM_ERR_TIMEOUT.  enable = 0 restores normal calls.  FMM_ERR_UNSUPPORTED for a plan that runs
 * no tensor-core level (an FP64 or FP32 plan, or levels < 6); FMM_ERR_INVALID_ARG for NULL. */
fmm_status fmm_inject_timeout(fmm_plan_t plan, int enable);

/* Free the plan and every device buffer it owns.  NULL is ignored. */
void fmm_plan_destroy(fmm_plan_t plan);

/* Static English text for a status code; never NULL. */
const char* fmm_status_string(int status);

/* FP64 direct sum at selected targets (the reference of every accuracy figure):
 *   phi_t[t] = sum_{j != targets[t], r > 0} q_j log|z_targets[t] - z_j|.
 *   xy, q      device, the n particles as in fmm_potential.
 *   targets    device, const int64_t[n_targets], each in [0, n).
 *   phi_t      device, double[n_targets].
 *   stream     cudaStream_t (NULL = default stream).
 * Asynchronous; allocates nothing; returns FMM_ERR_INVALID_ARG for n < 0,
 * n_targets < 0 or null pointers with nonzero sizes. */
fmm_status fmm_direct_targets(int64_t n, const double* xy, const double* q, int64_t n_targets,
                              const int64_t* targets, double* phi_t, void* stream);

/* Throughput probes for the roofline denominators of the arithmetic-bound stages.  They have no
 * counterpart in the paper; they measure the units its near field (Sec. 2.1, E-2: one logarithm
 * per pair) and its FP32 expansion sums run on.
 *   unit       FMM_PROBE_FP32_FMA: FP32 flop/s (an FMA counts 2);
 *              FMM_PROBE_MUFU_LG2: lg2.approx results/s;
 *              FMM_PROBE_FP64_FMA: FP64 flop/s.
 *   ops_per_s  host, written with the best rate of three timed launches (0 on failure).
 *   stream     cudaStream_t (NULL = default stream), on the current device.
 * Runs four launches of a few milliseconds each and blocks until they finish; allocates 4 bytes of
 * device memory for the call.  FMM_ERR_INVALID_ARG for an unknown unit or a null ops_per_s,
 * FMM_ERR_OOM or FMM_ERR_CUDA when a CUDA call fails. */
enum { FMM_PROBE_FP32_FMA = 0, FMM_PROBE_MUFU_LG2 = 1, FMM_PROBE_FP64_FMA = 2 };
fmm_status fmm_probe_peak(int unit, double* ops_per_s, void* stream);

/* ---------------------------------------------------------------------------------------
 * Batched form: many independent systems of uneven size, each an independent instance of
 * the method above (its own box [0, box]^2 and quadtree depth), evaluated by one launch per
 * stage that spans all systems, replayed as one CUDA graph.  M2L of levels 2..5 runs on the
 * CUDA cores in FP32; in the tensor-core precisions every system's levels 6 and finer run in
 * one tcgen05 launch whose tiles come from any system.  The near field is the symmetric one
 * of the single-system path, on a second branch of the graph beside P2M and M2L.
 * --------------------------------------------------------------------------------------- */
typedef struct fmm_batch_s* fmm_batch_t;

/* Create a batch plan for nsys systems (1 <= nsys <= 1536; total particles < 2^31).
 *   n[i], levels[i]  host arrays: particles (>= 1) and quadtree depth (0..12) of system i.
 *   p, box           expansion order and box side shared by all systems.
 *   precision        FMM_MIXED_FP32, or a tensor-core precision (FMM_MIXED_TF32, _3XTF32,
 *                    _BF16, _BF16X2, _BF16X3; p <= 31); FMM_FP64 returns FMM_ERR_UNSUPPORTED.
 *   stream           cudaStream_t the calls run on (NULL = default stream).
 * Allocates every workspace, builds the operators and captures the launch sequence into a
 * CUDA graph. */
fmm_status fmm_batch_plan(fmm_batch_t* out, int nsys, const int64_t* n, const int* levels, int p,
                          double box, int precision, void* stream);

/* phi of every system: xy [sum n][2], q [sum n], phi [sum n] are device arrays with the
 * systems concatenated in order (system i starts at n[0] + ... + n[i-1]).  Asynchronous;
 * allocates nothing; errors found on the device are reported by fmm_batch_sync. */
fmm_status fmm_batch_potential(fmm_batch_t batch, const double* xy, const double* q, double* phi);

/* Wait for the batch's stream; return the device-detected status of the calls since the
 * last sync and clear it.  ms (may be NULL) receives the device time of the last call. */
fmm_status fmm_batch_sync(fmm_batch_t batch, double* ms);

/* Autotuner: times the batch on the given inputs (device arrays as for fmm_batch_potential)
 * for every launch shape of a small grid -- persistent blocks per SM of the grid-stride
 * kernels (2, 4, 8), tensor-core M2L tiles per CTA (the default, 2, 4; tensor-core
 * precisions only) and near-field targets per block (16, 24) -- keeps the fastest and
 * rebuilds the graph.  grid_mult_out (may be NULL) receives the blocks per SM.  Runs and
 * waits for about 70 calls on the batch's stream. */
fmm_status fmm_batch_autotune(fmm_batch_t batch, const double* xy, const double* q, double* phi,
                              int* grid_mult_out);

/* As fmm_batch_autotune, with a cache: cache_path (may be NULL: no cache) names a text file
 * of lines "key grid_mult tc_rows p2p_block ms", the key naming the device (name, SMs,
 * driver version), p, the precision and the batch's shape (systems, total particles to a
 * power of two, systems per depth).  A line with this batch's key is applied without timing;
 * otherwise the search runs and its result is appended.  The file is created if missing. */
fmm_status fmm_batch_autotune_cached(fmm_batch_t batch, const double* xy, const double* q, double* phi,
                                     const char* cache_path);

/* The batch's current launch shape and the autotuner's best time (0 before a search); any
 * pointer may be NULL. */
fmm_status fmm_batch_tuning(fmm_batch_t batch, int* grid_mult, int* tc_rows, int* p2p_block, double* ms);

/* Kernels (and memsets) the batch graph launches per call, or -1 for NULL. */
int fmm_batch_launches(fmm_batch_t batch);

/* Free the batch plan and everything it owns.  NULL is ignored. */
void fmm_batch_destroy(fmm_batch_t batch);

/* ---------------------------------------------------------------------------------------
 * Learned (levels, p) selector.  Features of a system: for every level k = 3..11 of the
 * uniform quadtree over [0, box]^2, the fraction of squares whose population c falls in bin
 * floor(log2(c + 1)) (12 bins, the last one open), then log2(N) / 22 -- 109 values.  A small
 * MLP (IN = 111: the features, levels / 12 and p / 32 of one candidate; two hidden ReLU
 * layers; 2 outputs) predicts log10(relative L2 error) / 8 and log(milliseconds) of the method
 * at that candidate.  Training, inference and the statistics run in the library's kernels.
 * --------------------------------------------------------------------------------------- */
typedef struct fmm_selector_s* fmm_selector_t;

/* Input, output and feature widths of the network (111, 2, 109); any pointer may be NULL. */
int fmm_selector_dims(int* in, int* out, int* feat);

/* A network with `hidden` units per hidden layer, He-uniform weights from a SplitMix64 seed. */
fmm_status fmm_selector_create(fmm_selector_t* out, int hidden, uint64_t seed, void* stream);
void fmm_selector_destroy(fmm_selector_t sel);
int fmm_selector_num_params(fmm_selector_t sel);

/* The 109 features of xy (device, [n][2]) into feat_host (host); waits for the stream. */
fmm_status fmm_selector_features(fmm_selector_t sel, const double* xy, int64_t n, double box, float* feat_host);

/* Parameters in / out as host arrays of fmm_selector_num_params floats, layout
 * [W1 (IN x H) | b1 | W2 (H x H) | b2 | W3 (H x 2) | b3], row-major [input][output]. */
fmm_status fmm_selector_get_params(fmm_selector_t sel, float* host);
fmm_status fmm_selector_set_params(fmm_selector_t sel, const float* host);

/* y[rows][2] = network(x[rows][IN]); host arrays; waits for the stream. */
fmm_status fmm_selector_predict(fmm_selector_t sel, const float* x_host, int rows, float* y_host);

/* Loss (1/rows) sum_r sum_j (y - t)^2 and its gradient (grad_host may be NULL); host arrays. */
fmm_status fmm_selector_loss_grad(fmm_selector_t sel, const float* x_host, const float* t_host, int rows,
                                  float* loss, float* grad_host);

/* `epochs` full-batch Adam steps (learning rate lr); loss_out (may be NULL) gets the final
 * loss.  The Adam state persists in the selector, so repeated calls continue training. */
fmm_status fmm_selector_train(fmm_selector_t sel, const float* x_host, const float* t_host, int rows,
                              int epochs, float lr, float* loss_out);

/* Save / load parameters and Adam state (a versioned binary file) to resume training. */
fmm_status fmm_selector_save(fmm_selector_t sel, const char* path);
fmm_status fmm_selector_load(fmm_selector_t sel, const char* path);

/* Choose (levels, p) for xy (device, [n][2]): candidates levels = round(log4(n/16)) - 2 .. + 2
 * (clamped to 2..11) x p = 8, 12, .., 28 (every precision takes them); returns the cheapest
 * predicted time among those
 * whose predicted log10 error is at most log10(target_err) - margin_decades, else the fixed
 * fallback (8, 20) with *used_fallback = 1. */
fmm_status fmm_select(fmm_selector_t sel, const double* xy, int64_t n, double box, double target_err,
                      double margin_decades, int* levels_out, int* p_out, int* used_fallback);

/* The FP64 method of fmm_potential for callers that cannot allocate device memory.
 * The paper has no counterpart: this is a library convenience.  Some callers cannot call
 * cudaMalloc -- a loop that forbids allocation once it has started, a device whose free
 * memory belongs to another allocator, a plugin that may not own allocations -- and
 * fmm_plan allocates.  This entry point creates no plan and allocates nothing: its
 * workspaces live in one fixed device array of 8.5 MB inside libfmm.so, which every GPU
 * that loads the library reserves until the process exits.  The CUDA runtime reserves it
 * when the library's module is loaded on a device; with lazy loading (the default) that is
 * the first call of this entry point or of any library kernel there, so a caller whose
 * allocator later claims the free memory should make one call before it does.  If that
 * reservation fails the call returns FMM_ERR_OOM.
 *   n, levels, p, box   as for fmm_plan, FP64 only, limited to 1 <= n <= 65536,
 *                       0 <= levels <= 6 and 1 <= p <= 20; larger requests return
 *                       FMM_ERR_INVALID_ARG and touch nothing.
 *   xy, q, phi          device arrays as for fmm_potential, owned by the caller.
 *   stream              cudaStream_t to run on (NULL = default stream).
 * The call waits for `stream` and returns the device checks' status (phi is left unwritten
 * when a particle is outside the box or a value is not finite).  The first call on a device
 * looks up the array's device address and creates the stage events for that device; make
 * that first call before any stream capture.  A CUDA error already pending on the calling
 * thread is left for its owner: the call returns FMM_ERR_CUDA without clearing it.  Every call on a device shares the one array,
 * so calls that overlap on the GPU (other threads, other streams) race and must be
 * serialised by the caller. */
fmm_status fmm_potential_noalloc(int64_t n, int levels, int p, double box, const double* xy,
                                 const double* q, double* phi, void* stream);

#ifdef __cplusplus
}
#endif

#endif  /* FMM_H_ */
