/*
 * fmm_lagrange.h -- C ABI of the Lagrange-node form of the shift-free FMM in libfmm.so.
 *
 * The paper's own realisation of its method (arXiv 2009.00767, Appendix, STEP1-STEP5, Eq. 1-2,
 * with the summation scheme of Sec. 2.2.1): the charges of a square (2D) or cube (3D) are
 * represented by charges fixed at n^D Lagrange nodes, n = 4 (16 nodes per square, 64 per
 * cube).  It evaluates, for N charges in [0, box]^D,
 *
 *     phi(c_i) = sum_{j != i} q_j K(c_i, c_j),   K = log|r| (D = 2) or 1/|r| (D = 3, Coulomb),
 *
 * with coincident pairs contributing 0.
 *
 * Geometry (readings of the paper, whose Fig. 3 and Fig. 4 are missing):
 *   - uniform tree of depth `levels` over [0, box]^D; a charge's finest cell is
 *     floor(x 2^levels / box) per axis in FP64, clamped to [0, 2^levels - 1];
 *   - in a cell of side s centred at c the nodes are c + (s/5) a per axis, a in {-2,-1,1,2}
 *     (Eq. 2's node values for the paper's box of side 5, scaled with the cell);
 *   - h_m(c) = q_c f_i(x) f_j(y) [f_k(z)], f the Lagrange basis on those nodes (Eq. 1) at the
 *     charge's local coordinate (position - c) / (s/5);
 *   - interaction list of a level-k cell (k >= 2): children of its parent and the parent's
 *     neighbours that are not adjacent to it (27 in 2D, 189 in 3D); near field: the own and
 *     adjacent finest cells (Sec. 2.1 E-2).
 *
 * Forms (fmm_lag_form):
 *   FMM_LAG_LITERAL_F64  the paper's steps as written, FP64: v_c = h_{m^0}(c) (the charges at
 *                        the root box's nodes), U-bar-1 / U-bar-2 sums up the tree with no
 *                        shift, D-bar-1 with B_{m_i,m} = M_{m_i}^T M_b M_m formed once per
 *                        interaction-list pair at plan time and kept in device memory (STEP5;
 *                        Sec. 4 Discussions (2) and (5)), D-bar-2 sums of dual vectors down
 *                        the tree, F(v) = L_{m^l}(v).  M_m's entries grow like (2^k)^(3D)
 *                        (STEP4 extrapolates the root nodes into a small cell), so FP64 loses
 *                        about 3D*log10(2^k) digits at level k (Sec. 4 Discussion (3)): this
 *                        form is offered for levels <= 7 (2D) and <= 3 (3D) and is accurate
 *                        to the method's own error only to about level 4 (2D) and 3 (3D).
 *   FMM_LAG_NODE_F64     the same bilinear forms with the change of basis applied on the
 *                        particle side (STEP4: M_m h_{m^0}(c) = h_m(c) exactly): node charges
 *                        of every cell at every level straight from its charges, the node-to-
 *                        node matrix M_b over each interaction list, the node potentials
 *                        interpolated back at the charges; equal to the literal form in exact
 *                        arithmetic and free of its cancellation.  FP64 throughout.
 *   FMM_LAG_NODE_F32     the node form in FP32 arithmetic with FP64 accumulation across
 *                        levels and source tiles; near-field differences from two-word (hi, lo)
 *                        FP32 coordinates.  About 1e-7 relative to the FP64 node form.
 * The method's own error (4 nodes per axis) is about 1e-4 .. 1e-3 of the potential.
 *
 * Conventions (as in fmm.h): device pointers on the plan's device, owned by the caller;
 * pos is [N][D] FP64 C-ordered, q and phi [N] FP64; work is enqueued on the plan's stream;
 * device-side input errors (out of box, non-finite) are latched and returned by fmm_lag_sync,
 * with phi left unwritten; a plan is not thread-safe; fmm_status values are returned.
 */
#ifndef FMM_LAGRANGE_H_
#define FMM_LAGRANGE_H_

#include <stdint.h>

#include "fmm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmm_lag_plan_s* fmm_lag_plan_t;

typedef enum {
    FMM_LAG_NODE_F32 = 0,
    FMM_LAG_NODE_F64 = 1,
    FMM_LAG_LITERAL_F64 = 2
} fmm_lag_form;

/* Per-call statistics of the last completed fmm_lag_potential (valid after fmm_lag_sync).
 * Stage names follow the node forms; for the literal form ms_up covers U-bar-1 and U-bar-2,
 * ms_down D-bar-1 and D-bar-2, ms_eval F(v). */
typedef struct {
    int64_t n;
    int dim, levels, form;
    double ms_total;           /* first kernel to last, CUDA events */
    double ms_sort;            /* bin, scan, scatter */
    double ms_up;              /* node charges of levels 2..levels (literal: U-bar sums) */
    double ms_down;            /* node potentials over the interaction lists (literal: D-bar) */
    double ms_eval;            /* interpolation at the charges + far/near sum in input order */
    double ms_p2p;             /* near field (on a second stream, overlapping the far field) */
    int64_t p2p_pairs;         /* ordered pairs of the near field, self pairs included */
    int64_t m2l_pairs;         /* interaction-list pairs of levels 2..levels */
    uint64_t workspace_bytes;  /* device memory the plan owns (the literal form's B included) */
    int kernel_launches;
} fmm_lag_stats;

/* Create a plan for up to n_max charges in dimension `dim` (2 or 3).
 *   levels  0..8 (dim 2) or 0..5 (dim 3) for the node forms; 0..7 / 0..3 for the literal form;
 *           levels 0 and 1 have no far field (everything is near field).
 *   box     side of the computation box, > 0 and finite.
 *   form    an fmm_lag_form value.
 *   stream  cudaStream_t to enqueue on (NULL = legacy default stream).
 * Builds the node-to-node operators of every level in FP64 on the host (and, for the literal
 * form, every pair's B on the device in FP64).  FMM_ERR_INVALID_ARG, FMM_ERR_OOM or
 * FMM_ERR_CUDA on failure; *out unchanged then. */
fmm_status fmm_lag_plan(fmm_lag_plan_t* out, int dim, int64_t n_max, int levels, double box, int form,
                        void* stream);

/* phi[i] = potential at charge i, input order.  0 <= n <= n_max; n = 0 enqueues nothing. */
fmm_status fmm_lag_potential(fmm_lag_plan_t plan, const double* pos, const double* q, int64_t n, double* phi);

/* Wait for the plan's work; returns the first latched device-side error (and clears it). */
fmm_status fmm_lag_sync(fmm_lag_plan_t plan);

/* Statistics of the last call (call after fmm_lag_sync). */
fmm_status fmm_lag_stats_get(fmm_lag_plan_t plan, fmm_lag_stats* out);

/* Change the stream later calls enqueue on. */
fmm_status fmm_lag_set_stream(fmm_lag_plan_t plan, void* stream);

/* 2 (the default): the near field runs on a stream of the plan's own beside the far field, joined
 * back before the final sum.  1: every kernel in turn on the plan's stream, so that the stage
 * times of fmm_lag_stats_get are those of each stage alone.  Same results either way.
 * FMM_ERR_INVALID_ARG for another count or a NULL plan. */
fmm_status fmm_lag_set_concurrency(fmm_lag_plan_t plan, int streams);

/* The finest cell of every charge of the last call, [n][dim] int32 device array, input order
 * (the binning the tree used, for bit-exact checks).  Enqueued on the plan's stream. */
fmm_status fmm_lag_cells(fmm_lag_plan_t plan, int32_t* cells);

/* FP64 direct sum at chosen targets on the device: phi[t] = sum_{j != tgt[t]} q_j K(c_tgt[t], c_j),
 * all device arrays; enqueued on `stream`.  The reference for error figures at full size. */
fmm_status fmm_lag_direct_targets(int dim, int64_t n, const double* pos, const double* q, int64_t nt,
                                  const int64_t* tgt, double* phi, void* stream);

/* Release the plan (synchronises its stream first).  NULL is ignored. */
void fmm_lag_plan_destroy(fmm_lag_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* FMM_LAGRANGE_H_ */
