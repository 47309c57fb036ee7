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
//   B0[k]                    (mixed) Re b'_0 of each level-k square in FP64
//   phi_far[n]               far field summed over levels, FP64, box-sorted order
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

struct FmmLevelPtrs {
    void* A[FMM_MAX_LEVELS + 1];    // FP64 moments (both paths), double2 [cell][p+1]
    void* B[FMM_MAX_LEVELS + 1];    // local coefficients: double2 (FP64 path) or float2 (mixed)
    void* B0[FMM_MAX_LEVELS + 1];   // mixed path: Re b'_0 in FP64, one per square
};

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
    uint32_t* block_sums;
    int scan_blocks;
    uint32_t* sorted_key;
    fmm_p64* sorted64;
    float4* sorted32;

    FmmLevelPtrs grids;
    size_t a_bytes[FMM_MAX_LEVELS + 1];
    double* phi_far;

    double2* T64;       // FP64 operators [49][p+1][p+1]
    float2* T32;        // FP32 operators [49][p1b][p1b], zero-padded, [d][0][0] = 0 (mixed SIMT M2L)
    int p1b;            // padded coefficient count of the FP32 M2L kernel instance

    unsigned int* d_status;
    unsigned long long* d_counters;   // [0] = near-field pairs, [1] = max leaf population
    unsigned int* h_status;           // pinned
    unsigned long long* h_counters;   // pinned [2]

    double* d_xy_stage;
    double* d_q_stage;
    double* d_phi_stage;

    cudaEvent_t ev[6];
    int events_recorded;
    int launches;
    fmm_stats last;
    uint64_t workspace_bytes;
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

// --- launchers (each returns the number of kernels it launched, or -1 on a launch error) ---------
int fmm_launch_sort(fmm_plan_s* pl, const double* xy, const double* q);
int fmm_scan_blocks(int64_t m);
int fmm_launch_fp64(fmm_plan_s* pl, double* phi);
int fmm_launch_mixed(fmm_plan_s* pl, double* phi);
int fmm_m2l_bucket(int p1);
int fmm_launch_direct_f64(int64_t n, const double* xy, const double* q, int64_t nt, const int64_t* targets,
                          double* phi_t, cudaStream_t stream);
