// mixed_common.cuh -- helpers shared by the mixed-precision kernels (mixed.cu, m2l_tc.cu).
#pragma once

#include <cmath>

#include "fmm_internal.cuh"

// ---------------------------------------------------------------- float-float helpers
// Knuth's TwoSum and an FMA-based product (error-free transformations): a value is hi + lo
// with |lo| <= ulp(hi)/2, about 48 significant bits from FP32 arithmetic alone.
static __device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return make_float2(s, e);
}
static __device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
    const float2 s = two_sum(a.x, b.x);
    const float e = s.y + (a.y + b.y);
    const float h = s.x + e;
    return make_float2(h, e - (h - s.x));
}
static __device__ __forceinline__ float2 ff_add_f(float2 a, float b) {
    const float2 s = two_sum(a.x, b);
    const float e = s.y + a.y;
    const float h = s.x + e;
    return make_float2(h, e - (h - s.x));
}
static __device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
    const float pr = a.x * b.x;
    float e = fmaf(a.x, b.x, -pr);
    e = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
    const float h = pr + e;
    return make_float2(h, e - (h - pr));
}

// Per-level constants, formed on the host in FP64 and rounded once.
struct MixedLevels {
    float inv_s[FMM_MAX_LEVELS + 1];      // 2^k / box
    float s_leaf;                         // box / 2^levels
    float2 logc[FMM_MAX_LEVELS + 1][49];  // log|w0_d| + ln s_k as float-float, 0 for adjacent d
};

// w of a particle in its level-k square, from its offset (dx, dy) to the centre of its finest
// square (ix, iy): w = ((i_local + 1/2) 2^-(l-k) - 1/2) + d 2^k / box.  The first part is an
// exact dyadic number in FP32.
static __device__ __forceinline__ float2 level_w(float dx, float dy, uint32_t ix, uint32_t iy, int sh, float inv_s) {
    const uint32_t mask = (1u << sh) - 1u;
    const float sc = __int_as_float((127 - sh) << 23);   // 2^-sh
    const float ox = fmaf((float)(ix & mask) + 0.5f, sc, -0.5f);
    const float oy = fmaf((float)(iy & mask) + 0.5f, sc, -0.5f);
    return make_float2(fmaf(dx, inv_s, ox), fmaf(dy, inv_s, oy));
}


inline MixedLevels fmm_make_levels(const fmm_plan_s* pl) {

    MixedLevels lv{};
    for (int k = 0; k <= FMM_MAX_LEVELS; ++k) {
        lv.inv_s[k] = (float)((double)(1 << k) / pl->box);
        const double ln_s = log(pl->box / (double)(1 << k));
        for (int d = 0; d < 49; ++d) {
            const int dx = d % 7 - 3, dy = d / 7 - 3;
            const bool adj = dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1;
            const double c = adj ? 0.0 : 0.5 * log((double)(dx * dx + dy * dy)) + ln_s;
            const float h = (float)c;
            lv.logc[k][d] = make_float2(h, (float)(c - (double)h));
        }
    }
    lv.s_leaf = (float)(pl->box / (double)(1 << pl->levels));
    return lv;
}


// tensor-core M2L (m2l_tc.cu)
#include <vector>
// one level of one system for the tensor cores: its FP32 moment grid (3-cell halo) and local grid
struct FmmTcLevel {
    const float2* a32;
    float2* B;
    int k;
};
bool fmm_tc_precision(int precision);
FmmTc* fmm_tc_new(int p, int precision, const std::vector<double>& Tre, const std::vector<double>& Tim, int* err,
                  uint64_t* bytes);
int fmm_tc_set_levels(FmmTc* tc, const std::vector<FmmTcLevel>& levels, uint64_t* bytes);
void fmm_tc_free(FmmTc* tc);
int fmm_tc_enqueue(FmmTc* tc, const MixedLevels& lv, cudaStream_t st, unsigned int* status, int stall, int rows_max,
                   cudaEvent_t e0, cudaEvent_t e1);
int fmm_tc_create(fmm_plan_s* pl, const std::vector<double>& Tre, const std::vector<double>& Tim);
void fmm_tc_destroy(fmm_plan_s* pl);
int fmm_launch_m2l_tc(fmm_plan_s* pl, const MixedLevels& lv);
// the FP64 M2L operators T[49][p+1][p+1] (api.cu), real and imaginary parts
void fmm_build_operators_f64(int p, std::vector<double>& re, std::vector<double>& im);
// the near field on the plan's second stream (mixed.cu); kernels launched, or -1
int fmm_launch_p2p_concurrent(fmm_plan_s* pl, const MixedLevels& lv, bool with_field, bool record_fork);
int fmm_tc_kmin();
