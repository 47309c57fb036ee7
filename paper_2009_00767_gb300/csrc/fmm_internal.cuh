// fmm_internal.cuh -- plan layout and kernel launchers shared by the library's .cu files.
//
// Data layout in device memory (all owned by the plan):
//   keys[n], rank[n]         finest-square Morton key and rank inside it, input order
//   counts[M], leaf_start[M+1]   M = 4^levels finest squares in Morton order (CSR)
//   sorted_key[n]            Morton key of each particle, box-sorted order
//   sorted64[n]              fmm_p64 {x, y, q, input index} in box-sorted order (FP64 path)
//   sorted32[n]              float4 {x - cx, y - cy (relative to the finest-square centre), q,
//                            input index as int bits} (mixed paths)
//   A[k]  (k = 2..levels)    multipole moments of level k on a (2^k + 6)^2 grid with a 3-square
//                            zero halo, row-major, p+1 complex coefficients per square
//   B[k]                     local coefficients of level k, (2^k)^2 row-major, p+1 complex each
//   A32[k]                   (mixed) FP32 moments of level k, same layout (the mixed path has no
//                            FP64 A[k]); slot 0 holds M_0 as a float-float pair
//   (mixed) B[k] slot 0 holds Re b'_0 as a float-float pair
//   phi_far[n]               FP64 path: far field summed over levels, box-sorted order; mixed
//                            path: the near field as float-float pairs (log2 r^2 units)
//   T64                      49 x (p+1) x (p+1) complex FP64 M2L operators, layout [d][k][l],
//                            d = (dx + 3) + 7 (dy + 3), zero for the 9 adjacent offsets
// Because keys are Morton-ordered, the particles of every square of every level are one
// contiguous range of the sorted arrays (square key = finest key >> 2 (levels - k)).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fmm.h"

#define FMM_MAX_LEVELS 12

// box-sorted particle record of the FP64 path: one 32-byte sector per particle
struct __align__(32) fmm_p64 {
    double x, y, q, w;   // w = input index (exact in FP64)
};
#define FMM_MAX_P 40
#define FMM_HALO 3

// device status bits (latched until fmm_sync)
#define FMM_FLAG_OUT_OF_BOX 1u
#define FMM_FLAG_NONFINITE 2u
#define FMM_FLAG_TIMEOUT 4u

// Near-field statistics are spread over this many counter slots (one update per CTA each) so
// that no single L2 address serialises the updates.
#define FMM_COUNTER_SLOTS 64
#define FMM_LANE_MAX 128   // finest squares above this many particles are "crowded" in the fine P2M

// Conversions between FP32 and FP64 by integer bit operations, so that they do not occupy
// GB300's narrow FP64 pipe.  Zero, subnormal and out-of-range inputs flush to zero (their
// magnitudes are below 2^-126, far under the rounding of the results they feed).
__device__ __forceinline__ double fmm_f2d_bits(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return 0.0;
    const uint32_t m = u & 0x7fffffu;
    const uint32_t hi = (u & 0x80000000u) | ((e + 896u) << 20) | (m >> 3);
    return __hiloint2double((int)hi, (int)((m & 7u) << 29));
}
// double -> (hi, lo) float pair with hi = the double truncated to 24 bits and lo the rest
// (rounded to FP32); hi + lo carries about 48 bits of the double.
__device__ __forceinline__ float2 fmm_d2ff_bits(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7ffu);
    if (e <= 896 || e >= 1151) return make_float2(0.f, 0.f);
    const uint32_t sign = (uint32_t)(b >> 63) << 31;
    const unsigned long long m = b & 0xfffffffffffffull;
    const float hi = __uint_as_float(sign | ((uint32_t)(e - 896) << 23) | (uint32_t)(m >> 29));
    float lo = 0.f;
    if (e > 948) {   // 2^(e - 1075) is a normal float
        lo = (float)(uint32_t)(m & 0x1fffffffu) * __uint_as_float((uint32_t)(e - 948) << 23);
        if (sign) lo = -lo;
    }
    return make_float2(hi, lo);
}

struct FmmLevelPtrs {
    void* A[FMM_MAX_LEVELS + 1];    // FP64 moments (FP64 path), double2 [cell][p+1]
    void* B[FMM_MAX_LEVELS + 1];    // local coefficients: double2 (FP64 path) or float2 (mixed)
    void* A32[FMM_MAX_LEVELS + 1];  // mixed path: float2 copy of A, coefficient 0 as (hi, lo) of M_0
};

struct FmmTc;   // tensor-core M2L state (m2l_tc.cu)

struct fmm_plan_s {
    int device;
    int64_t n;
    int levels, p, precision;
    double box;
    cudaStream_t stream;

    uint32_t* keys;
    uint32_t* rank;
    uint32_t* counts;
    uint32_t* leaf_start;
    uint32_t* block_sums;        // scan partials, scan_blocks + 1 entries (64-bit in the mixed path)
    int scan_blocks;
    uint32_t* leaf_bstart;       // near-field target blocks: exclusive scan over the squares, 4^levels + 1
    uint2* blk_map;              // near-field block -> (square, block inside it), mixed path
    int clean;                   // mixed path: the square populations are zero (each call's scan
                                 // leaves them so; a call that failed to enqueue does not)
    uint32_t* sorted_key;
    fmm_p64* sorted64;
    float4* sorted32;
    float2* sorted_lo;           // mixed path, field calls: the local coordinates' FP32 rounding residues
    FmmLevelPtrs grids;
    size_t a_bytes[FMM_MAX_LEVELS + 1];
    double* phi_far;                  // FP64 path: far field; mixed path: near-field accumulator per particle
    double2* near_grad;               // mixed path: near-field gradient accumulator (fmm_potential_field)
    float2* far_part;                 // mixed path: float-float far field of the coarse levels per particle

    double2* T64;       // FP64 operators [49][p+1][p+1]
    float2* T32;        // FP32 operators [49][p1b][p1b], zero-padded, [d][0][0] = 0 (mixed SIMT M2L)
    float2* U32;        // mixed path: upward-pass translations [child position][j][m] (p1b each), zero-padded
    int p1b;            // padded coefficient count of the FP32 M2L kernel instance
    FmmTc* tc;          // tensor-core M2L state (TF32 modes), or null

    unsigned int* d_status;
    unsigned long long* d_counters;   // [0..63] near-field pair partials, [64..127] max leaf population
    unsigned int* h_status;           // pinned
    unsigned long long* h_counters;   // pinned [128]
    // mixed path: set to 1 by the scan of a call that finds a finest square above FMM_LANE_MAX
    // particles (mapped host memory, read without a sync by the next call's enqueue, which then
    // sums crowded squares' fine-level moments with k_p2m_crowded instead of one warp each)
    int* crowd_hint_h;
    int* crowd_hint_d;

    // host-array calls: two staging sets, so a call's uploads overlap the previous call's compute
    double* d_xy_stage[2];
    double* d_q_stage[2];
    double* d_phi_stage[2];
    int stage_next;                          // the set the next host call uses
    int host_chunks;                         // chunks the current host call binned itself
    cudaStream_t s_up, s_down;               // mixed path: uploads + binning, result downloads
    cudaEvent_t ev_sorted;                   // the sort no longer needs keys, ranks or populations
    cudaEvent_t ev_stage_free[2];            // the set's inputs were consumed (scatter done)
    cudaEvent_t ev_up_done, ev_l2p_done;     // a host call's uploads / compute are complete
    cudaEvent_t ev_down_done[2];             // the set's result was downloaded

    // Mixed path: after the sort (or, when the coarse M2L reaches a fine level, after the fine P2M)
    // the work forks three ways -- the near field on stream2, the coarse levels' chain (P2M,
    // conversion, M2L and L2P of levels 2..5) on stream3, the fine levels' P2M and M2L on the plan's
    // stream -- and joins back before the fine levels' L2P.
    cudaStream_t stream2, stream3;
    cudaEvent_t ev_fork, ev_join, ev_join3;   // untimed fork / join events
    cudaEvent_t ev_a32;   // stream3's FP32 moment grids are written (levels 2 .. l-3; from l = 9 on the
                          // fine levels' M2L on the plan's stream reads some of them)
    // Timing events.  FP64 path: stage boundaries [0..5] (sort, P2M, M2L, L2P, P2P).  Mixed path:
    // [0] start, [1] sort done, [2] fine P2M done, [14] fine M2L start, [3] fine M2L done, [4] L2P
    // start (after the joins), [5] end, all on the plan's stream; [6, 7] the tensor-core M2L
    // kernel; [8, 9] the near-field kernel (stream2); [10, 11] the coarse P2M and its conversion,
    // [12, 13] the coarse M2L, [15, 16] the coarse levels' L2P (stream3).
    static constexpr int kEvents = 17;
    cudaEvent_t ev[kEvents];
    int ev_kernels;       // bits: 1 [6, 7], 2 [8, 9], 4 [10, 11], 8 [12, 13], 16 [15, 16] recorded this call
    int serial;           // fmm_set_concurrency(plan, 1): every stage on the plan's stream
    int events_recorded;
    int launches;
    fmm_stats last;
    uint64_t workspace_bytes;
    int test_stall;       // fmm_inject_timeout: the tensor-core M2L's producers issue nothing
};

// --- Morton helpers ----------------------------------------------------------------------------
__host__ __device__ inline uint32_t fmm_spread2(uint32_t v) {
    v &= 0x0000ffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}
__host__ __device__ inline uint32_t fmm_compact2(uint32_t v) {
    v &= 0x55555555u;
    v = (v | (v >> 1)) & 0x33333333u;
    v = (v | (v >> 2)) & 0x0f0f0f0fu;
    v = (v | (v >> 4)) & 0x00ff00ffu;
    v = (v | (v >> 8)) & 0x0000ffffu;
    return v;
}
__host__ __device__ inline uint32_t fmm_morton(uint32_t ix, uint32_t iy) {
    return fmm_spread2(ix) | (fmm_spread2(iy) << 1);
}

__host__ __device__ inline int fmm_grid_width(int k) { return (1 << k) + 2 * FMM_HALO; }

// Finest-square coordinate floor(fl(x 2^l / box)) clamped to [0, side - 1], the rule the oracle
// uses, without occupying the narrow FP64 pipe in the common case: an FP32 estimate of the
// quotient (error below 1e-3 for side <= 4096) decides whenever it is more than 2e-3 away from
// an integer; otherwise the exact FP64 division decides.  t = x 2^l is exact.
static __device__ __forceinline__ int finest_coord(double x, double scale, float scale_over_box32, double box, int side) {
    const float2 xf = fmm_d2ff_bits(x);   // hi word: x truncated to 24 bits
    const float q32 = xf.x * scale_over_box32;
    const float fl = floorf(q32);
    const float fr = q32 - fl;
    float f;
    if (fr > 2e-3f && fr < 1.0f - 2e-3f) {
        f = fl;
    } else {
        f = (float)floor(x * scale / box);
    }
    return f < 0.f ? 0 : (f > (float)(side - 1) ? side - 1 : (int)f);
}

// x in [0, box] for finite x, by integer comparison of the bit patterns (monotone for
// non-negative doubles; -0.0 counts as 0).
static __device__ __forceinline__ bool in_box_bits(double x, long long box_bits) {
    const long long b = __double_as_longlong(x);
    if (b == (long long)0x8000000000000000ull) return true;
    return b >= 0 && b <= box_bits;
}

static __device__ __forceinline__ bool finite_bits(double x) {
    return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

// the rounding error of s = fl(a + b) (Knuth's TwoSum): a + b = s + err exactly
static __device__ __forceinline__ float two_sum_err(float a, float b, float s) {
    const float bb = s - a;
    return (a - (s - bb)) + (b - bb);
}

// a * (s.x + s.y) as an FP32 pair (FMA-exact product of the high word)
static __device__ __forceinline__ float2 scatter_mul(float a, float2 s) {
    const float h = a * s.x;
    const float e = fmaf(a, s.x, -h) + a * s.y;
    const float hh = h + e;
    return make_float2(hh, e - (hh - h));
}


// --- launchers (each returns the number of kernels it launched, or -1 on a launch error) ---------
// with_lo: also the rounding residues of the mixed path's local coordinates (sorted_lo); binned: the
// particles were already binned (fmm_launch_bin_range over all of them)
int fmm_launch_sort(fmm_plan_s* pl, const double* xy, const double* q, bool with_lo = false, bool binned = false);
int fmm_launch_bin_range(fmm_plan_s* pl, const double* xy, const double* q, int64_t i0, int64_t i1, cudaStream_t s);
int fmm_scan_blocks(int64_t m);
int fmm_launch_scan(const uint32_t* counts, int64_t m, uint32_t* block_sums, uint32_t* leaf_start, uint32_t n_total,
                    cudaStream_t st);
// Near-field target blocks: nb[i] = ceil(population of square i / block), bstart = their exclusive
// scan (m + 1 entries), and, if map is not null, map[b] = (square, index of b inside it).
int fmm_launch_leaf_blocks(const uint32_t* leaf_start, int64_t m, uint32_t block, uint32_t* nb, uint32_t* block_sums,
                           uint32_t* bstart, uint2* map, cudaStream_t st);
// targets per near-field block of the mixed path (the batched form uses 32)
#define FMM_P2P_BLOCK 24

// largest i in [0, m) with pre[i] <= w, for a non-decreasing pre with pre[0] <= w: a 32-ary
// search by the whole warp (each step probes 32 evenly spaced entries), about log32(m) loads
static __device__ __forceinline__ uint32_t fmm_warp_search(const uint32_t* pre, uint32_t m, uint32_t w, int lane) {
    uint32_t lo = 0, hi = m;
    for (int it = 0; it < 8 && hi - lo > 1; ++it) {
        const uint32_t step = (hi - lo + 31u) / 32u;
        const uint32_t pos = lo + (uint32_t)lane * step;
        const bool le = pos < hi && pre[pos] <= w;
        const unsigned msk = __ballot_sync(0xffffffffu, le);
        const int last = 31 - __clz(msk);
        lo = lo + (uint32_t)last * step;
        hi = min(hi, lo + step);
    }
    return lo;
}
int fmm_launch_fp64(fmm_plan_s* pl, double* phi, double* field = nullptr);
int fmm_launch_mixed(fmm_plan_s* pl, double* phi, double* field);
int fmm_m2l_bucket(int p1);
int fmm_launch_direct_f64(int64_t n, const double* xy, const double* q, int64_t nt, const int64_t* targets,
                          double* phi_t, cudaStream_t stream);
