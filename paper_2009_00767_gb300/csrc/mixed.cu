// mixed.cu -- the mixed-precision path: FP32 particle stages and FP32 M2L on the CUDA cores,
// with float-float (two FP32 words) wherever magnitudes are large.  GB300's FP64 pipe is far
// narrower than its FP32 pipe, so no FP64 arithmetic runs inside the hot loops: FP64 appears
// only in the atomic moment sums (executed in L2), in the one-off conversion of each moment
// cell, and in the final phi written for the caller.
//
// Scaled form as in fp64.cu (w = (z - c) / s, power-sum moments M_m = sum q w^m):
//   P2M  every level straight from the particles (U-bar of Sec. 2.2.1): w in FP32 from the
//        particle's offset to its finest-square centre (an exact dyadic square offset plus an
//        FP32 product), q w^m in FP32, warp-segmented FP32 sums of at most 32 terms, then FP64
//        atomics into the level's grid.
//   prep each moment cell once to FP32; the total charge M_0 (real) is kept as a float-float
//        pair (hi, lo) in the slot of coefficient 0.
//   M2L  (D-bar-1) per target: b'_l = sum_d sum_k T_d[k][l] M[t+d][k] in FP32 (k, l = 0..p),
//        except the monopole-log term sum_d M_0 (log|w0| + ln s) of b'_0, summed in
//        float-float; Re b'_0 is stored as a float-float pair in the slot of coefficient 0.
//   L2P  (D-bar-2 by linearity) per particle and level: Re sum_{l>=1} b'_l w^l by Horner in
//        FP32, plus Re b'_0; the levels are summed in float-float.
//   P2P  (E-2 of Sec. 2.1) in FP32 on square-local coordinates, log via the MUFU lg2 unit,
//        sources staged in shared memory by the bulk-copy (TMA) engine; phi = far + near.
#include "mixed_common.cuh"

namespace {

constexpr int kWarpsPerBlock = 4;
constexpr int kM2LThreads = 128;

// -------------------------------------------------------------------------------- P2M
// Every level straight from the particles (U-bar of Sec. 2.2.1).  Squares of a level are
// contiguous Morton ranges of the sorted particles, so the sums need no global sort of their own.
//
// Fine levels (at most kFineMean particles per square on average): one lane per square walks its
// range and keeps the p+1 sums in registers; the lane owns the square, so it stores the FP32
// moments (total charge as a float-float pair) straight into the FP32 grid, with no reduction
// and no atomics.  Squares above kLaneMax particles are left to the whole warp afterwards.
//
// Coarse levels: each warp walks kCoarseChunk consecutive particles; lanes add their particles'
// terms in registers while the square stays the same and flush (a column sum over the warp's
// lanes in shared memory, then FP64 atomics into the level's grid) when it changes.
constexpr int kFineMean = 64;
constexpr int kLaneMax = 128;
constexpr int kCoarseChunk = 256;

struct P2MFineArgs {
    int base[FMM_MAX_LEVELS + 2];   // first thread of each fine level
    int kf, levels, p;
};

// powers q w^m, m = 1..P1B-1 added into acc (entries at m >= p1 stay untouched: the caller masks)
template <int P1B>
__device__ __forceinline__ void add_powers(float2 (&acc)[P1B], float q, float2 w) {
    float pr = q, pi = 0.f;
#pragma unroll
    for (int m = 1; m < P1B; ++m) {
        const float nr = fmaf(pr, w.x, -pi * w.y);
        const float ni = fmaf(pr, w.y, pi * w.x);
        pr = nr;
        pi = ni;
        acc[m].x += pr;
        acc[m].y += pi;
    }
}

template <int P1B>
__global__ void __launch_bounds__(128)
k_p2m_fine(const float4* __restrict__ sp, const uint32_t* __restrict__ skey, const uint32_t* __restrict__ leaf_start,
           P2MFineArgs fa, MixedLevels lv, FmmLevelPtrs g) {
    __shared__ float red[4][32][2 * P1B + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    int k = fa.kf;
    while (k < fa.levels && gt >= fa.base[k + 1]) ++k;
    const bool valid = gt < fa.base[fa.levels + 1];
    const uint32_t b = valid ? (uint32_t)(gt - fa.base[k]) : 0u;
    const int sh = fa.levels - k;
    const int p1 = fa.p + 1;
    const uint32_t lo = valid ? leaf_start[(size_t)b << (2 * sh)] : 0u;
    const uint32_t hi = valid ? leaf_start[(size_t)(b + 1) << (2 * sh)] : 0u;
    const int W = fmm_grid_width(k);
    const size_t cell = (size_t)(fmm_compact2(b >> 1) + FMM_HALO) * W + fmm_compact2(b) + FMM_HALO;
    const bool large = hi - lo > (uint32_t)kLaneMax;
    float2 acc[P1B];
#pragma unroll
    for (int m = 0; m < P1B; ++m) acc[m] = make_float2(0.f, 0.f);
    float2 m0 = make_float2(0.f, 0.f);
    if (valid && !large) {
        for (uint32_t j = lo; j < hi; ++j) {
            const float4 P = sp[j];
            const uint32_t key = skey[j];
            const float2 w = level_w(P.x, P.y, fmm_compact2(key), fmm_compact2(key >> 1), sh, lv.inv_s[k]);
            m0 = ff_add_f(m0, P.z);
            add_powers<P1B>(acc, P.z, w);
        }
        float2* A = reinterpret_cast<float2*>(g.A32[k]) + cell * p1;
        A[0] = m0;
#pragma unroll
        for (int m = 1; m < P1B; ++m)
            if (m < p1) A[m] = acc[m];
    }
    // squares above kLaneMax particles: the whole warp, then a column sum in shared memory
    unsigned todo = __ballot_sync(0xffffffffu, valid && large);
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const uint32_t lo2 = __shfl_sync(0xffffffffu, lo, src), hi2 = __shfl_sync(0xffffffffu, hi, src);
        const int k2 = __shfl_sync(0xffffffffu, k, src);
        const unsigned long long cell2 = __shfl_sync(0xffffffffu, (unsigned long long)cell, src);
        const int sh2 = fa.levels - k2;
#pragma unroll
        for (int m = 0; m < P1B; ++m) acc[m] = make_float2(0.f, 0.f);
        m0 = make_float2(0.f, 0.f);
        for (uint32_t j = lo2 + lane; j < hi2; j += 32) {
            const float4 P = sp[j];
            const uint32_t key = skey[j];
            const float2 w = level_w(P.x, P.y, fmm_compact2(key), fmm_compact2(key >> 1), sh2, lv.inv_s[k2]);
            m0 = ff_add_f(m0, P.z);
            add_powers<P1B>(acc, P.z, w);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            m0 = ff_add(m0, make_float2(__shfl_xor_sync(0xffffffffu, m0.x, o), __shfl_xor_sync(0xffffffffu, m0.y, o)));
        float* row = red[warp][lane];
#pragma unroll
        for (int m = 1; m < P1B; ++m) {
            row[2 * m] = acc[m].x;
            row[2 * m + 1] = acc[m].y;
        }
        __syncwarp();
        float2* A = reinterpret_cast<float2*>(g.A32[k2]) + cell2 * p1;
        for (int col = 2 + lane; col < 2 * p1; col += 32) {
            float s = 0.f;
#pragma unroll
            for (int r = 0; r < 32; ++r) s += red[warp][r][col];
            reinterpret_cast<float*>(A)[col] = s;
        }
        if (lane == 0) A[0] = m0;
        __syncwarp();
    }
}

template <int P1B>
__global__ void __launch_bounds__(128)
k_p2m_coarse(const float4* __restrict__ sp, const uint32_t* __restrict__ skey, int64_t n, int levels, int kc_max,
             int p, MixedLevels lv, FmmLevelPtrs g) {
    __shared__ float red[4][32][2 * P1B + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = ((int64_t)blockIdx.x * 4 + warp) * kCoarseChunk;
    if (base >= n) return;
    const int p1 = p + 1, ncol = 2 * p1;
    float* row = red[warp][lane];
    for (int k = 2; k <= kc_max; ++k) {
        const int sh = levels - k;
        const int W = fmm_grid_width(k);
        double* A = reinterpret_cast<double*>(g.A[k]);
        float2 acc[P1B];
#pragma unroll
        for (int m = 0; m < P1B; ++m) acc[m] = make_float2(0.f, 0.f);
        uint32_t cur = skey[base] >> (2 * sh);
        auto flush = [&](uint32_t box) {
#pragma unroll
            for (int m = 0; m < P1B; ++m) {
                row[2 * m] = acc[m].x;
                row[2 * m + 1] = acc[m].y;
                acc[m] = make_float2(0.f, 0.f);
            }
            __syncwarp();
            const size_t cell = (size_t)(fmm_compact2(box >> 1) + FMM_HALO) * W + fmm_compact2(box) + FMM_HALO;
            for (int col = lane; col < ncol; col += 32) {
                float s = 0.f;
#pragma unroll
                for (int r = 0; r < 32; ++r) s += red[warp][r][col];
                atomicAdd(A + cell * ncol + col, fmm_f2d_bits(s));
            }
            __syncwarp();
        };
        for (int r = 0; r < kCoarseChunk / 32; ++r) {
            const int64_t j = base + 32 * r + lane;
            const bool valid = j < n;
            float2 c[P1B];
            uint32_t bx = 0xffffffffu;
            if (valid) {
                const float4 P = sp[j];
                const uint32_t key = skey[j];
                bx = key >> (2 * sh);
                const float2 w = level_w(P.x, P.y, fmm_compact2(key), fmm_compact2(key >> 1), sh, lv.inv_s[k]);
                c[0] = make_float2(P.z, 0.f);
                float pr = P.z, pi = 0.f;
#pragma unroll
                for (int m = 1; m < P1B; ++m) {
                    const float nr = fmaf(pr, w.x, -pi * w.y);
                    const float ni = fmaf(pr, w.y, pi * w.x);
                    pr = nr;
                    pi = ni;
                    c[m] = make_float2(pr, pi);
                }
            } else {
#pragma unroll
                for (int m = 0; m < P1B; ++m) c[m] = make_float2(0.f, 0.f);
            }
            // keys are sorted, so lanes with a square above cur are the ones not yet added; each
            // pass adds at least one lane, so at most 32 passes close the chunk
            for (int pass = 0; pass < 33; ++pass) {
                if (valid && bx == cur) {
#pragma unroll
                    for (int m = 0; m < P1B; ++m) {
                        acc[m].x += c[m].x;
                        acc[m].y += c[m].y;
                    }
                }
                const unsigned later = __ballot_sync(0xffffffffu, valid && bx > cur);
                if (!later) break;
                flush(cur);
                cur = __shfl_sync(0xffffffffu, bx, __ffs(later) - 1);
            }
            if (!__any_sync(0xffffffffu, valid)) break;
        }
        flush(cur);
    }
}

// -------------------------------------------------------------------------------- moment prep
// FP64 moment grid -> FP32 grid, once per coefficient; coefficient 0 (the real total charge)
// becomes a float-float pair.
__global__ void k_prep_a32(const double2* __restrict__ a64, float2* __restrict__ a32, int64_t count, int p1) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    const double2 v = a64[e];
    a32[e] = (e % p1 == 0) ? fmm_d2ff_bits(v.x) : make_float2(fmm_d2ff_bits(v.x).x, fmm_d2ff_bits(v.y).x);
}

// -------------------------------------------------------------------------------- M2L (FP32 SIMT)
struct M2LMixedArgs {
    FmmLevelPtrs g;
    const float2* T;                    // [49][P1B][P1B] FP32, zero beyond p and at [d][0][0]
    int cta_base[FMM_MAX_LEVELS + 2];   // first CTA of each level
    int levels, p, kmin, kmax;          // levels kmin..kmax run here
};

// Coarse levels (few targets, so one thread per target would leave the GPU idle and wait on
// one long dependent chain): a CTA takes 4 x kM2LWarpTargets targets of one parity class, one
// warp per kM2LWarpTargets targets, lanes over the outputs b'_l (l = lane, lane + 32).  The 27
// offsets of the class run in sequence; each offset's operator is staged in shared memory (two
// buffers), and the next offset's operator and source moments are loaded into registers while
// the current one is applied, so the loads' latency hides behind the FMAs.  Same arithmetic as
// the thread-per-target kernel: FP32 FMAs, the monopole-log term in float-float.
constexpr int kM2LWarpTargets = 2;
constexpr int kM2LWarpMaxLevel = 6;   // 4^6 targets: the finest level this kernel takes

struct M2LWarpArgs {
    FmmLevelPtrs g;
    const float2* T;
    int cbase[FMM_MAX_LEVELS + 2];      // first CTA of each level
    int kw, p;                          // levels 2..kw run here
};

template <int P1B>
__global__ void __launch_bounds__(128) k_m2l_coarse(M2LWarpArgs a, MixedLevels lv) {
    constexpr int NT = kM2LWarpTargets, NL = (P1B + 31) / 32;
    constexpr int TE = P1B * P1B, RT = (TE + 127) / 128;   // operator entries, per thread
    __shared__ float2 Ts[2][TE];
    __shared__ float2 src_s[4][NT][P1B];
    __shared__ int dl[27];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cta = blockIdx.x;
    int k = 2;
    while (cta >= a.cbase[k + 1]) ++k;
    const int w2 = 1 << (k - 1);
    const int per_class = (w2 * w2 + 4 * NT - 1) / (4 * NT);
    const int rel = cta - a.cbase[k];
    const int cls = rel / per_class;
    const int u0 = (rel - cls * per_class) * 4 * NT + warp * NT;
    const int px = cls & 1, py = cls >> 1;
    const int p1 = a.p + 1, W = fmm_grid_width(k);
    const float2* A = reinterpret_cast<const float2*>(a.g.A32[k]);
    if (threadIdx.x == 0) {
        int c = 0;
        for (int dy = -2 - py; dy <= 3 - py; ++dy)
            for (int dx = -2 - px; dx <= 3 - px; ++dx)
                if (!(dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1)) dl[c++] = (dx + 3) + 7 * (dy + 3);
    }
    int tx[NT], ty[NT];
    bool act[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const int u = u0 + j;
        act[j] = u < w2 * w2;
        tx[j] = act[j] ? 2 * (u % w2) + px : px;
        ty[j] = act[j] ? 2 * (u / w2) + py : py;
    }
    __syncthreads();
    // registers holding the next offset's operator share and source moments
    float2 tr[RT], sr[NT][NL];
    auto fetch = [&](int i) {
        const int d = dl[i];
        const float2* Td = a.T + (size_t)d * TE;
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            const int e = threadIdx.x + 128 * r;
            tr[r] = (e < TE) ? __ldg(Td + e) : make_float2(0.f, 0.f);
        }
        const int dx = d % 7 - 3, dy = d / 7 - 3;
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            // sources outside the domain read the zero halo
            const float2* src = A + ((size_t)(ty[j] + dy + FMM_HALO) * W + (tx[j] + dx + FMM_HALO)) * p1;
#pragma unroll
            for (int i2 = 0; i2 < NL; ++i2) {
                const int kk = lane + 32 * i2;
                sr[j][i2] = (kk < p1) ? src[kk] : make_float2(0.f, 0.f);
            }
        }
    };
    float2 acc[NT][NL];
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
        for (int i = 0; i < NL; ++i) acc[j][i] = make_float2(0.f, 0.f);
    float2 mono = make_float2(0.f, 0.f);   // lane j < NT: target j
    fetch(0);
    for (int i = 0; i < 27; ++i) {
        const int buf = i & 1;
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            const int e = threadIdx.x + 128 * r;
            if (e < TE) Ts[buf][e] = tr[r];
        }
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int i2 = 0; i2 < NL; ++i2) {
                const int kk = lane + 32 * i2;
                if (kk < P1B) src_s[warp][j][kk] = sr[j][i2];
            }
        const int d = dl[i];
        __syncthreads();   // Ts[buf] complete; the previous reader of this buffer is two offsets back
        if (i + 1 < 27) fetch(i + 1);
        if (lane < NT) mono = ff_add(mono, ff_mul(src_s[warp][lane][0], lv.logc[k][d]));
#pragma unroll
        for (int kk = 0; kk < P1B; ++kk) {
            float2 t[NL];
#pragma unroll
            for (int i2 = 0; i2 < NL; ++i2) {
                const int l = lane + 32 * i2;
                t[i2] = (l < P1B) ? Ts[buf][kk * P1B + l] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                float2 m = src_s[warp][j][kk];
                if (kk == 0) m.y = 0.f;   // M_0 is real; .y held its low word
#pragma unroll
                for (int i2 = 0; i2 < NL; ++i2) {
                    acc[j][i2].x = fmaf(t[i2].x, m.x, fmaf(-t[i2].y, m.y, acc[j][i2].x));
                    acc[j][i2].y = fmaf(t[i2].x, m.y, fmaf(t[i2].y, m.x, acc[j][i2].y));
                }
            }
        }
        __syncwarp();   // src_s of this warp is rewritten at the next offset
    }
    float2* B = reinterpret_cast<float2*>(a.g.B[k]);
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const float2 mj = make_float2(__shfl_sync(0xffffffffu, mono.x, j), __shfl_sync(0xffffffffu, mono.y, j));
        if (!act[j]) continue;
        const size_t t = (size_t)ty[j] * (1u << k) + tx[j];
#pragma unroll
        for (int i2 = 0; i2 < NL; ++i2) {
            const int l = lane + 32 * i2;
            if (l < p1) B[t * p1 + l] = (l == 0) ? ff_add_f(mj, acc[j][i2].x) : acc[j][i2];   // Re b'_0 as float-float
        }
    }
}

// One thread per target square; the CTA's 128 targets share one parity class (so one list of
// 27 offsets) and stage each offset's operator in shared memory, read as broadcasts.
template <int P1B>
__global__ void __launch_bounds__(kM2LThreads) k_m2l_f32(M2LMixedArgs a, MixedLevels lv) {
    __shared__ float2 Ts[P1B * P1B];
    const int cta = blockIdx.x;
    int k = a.kmin;
    while (cta >= a.cta_base[k + 1]) ++k;
    const int w2 = 1 << (k - 1);                       // parity sub-grid width
    const int per_class = (w2 * w2 + kM2LThreads - 1) / kM2LThreads;
    const int rel = cta - a.cta_base[k];
    const int cls = rel / per_class;
    const int u = (rel - cls * per_class) * kM2LThreads + threadIdx.x;
    const bool active = u < w2 * w2;
    const int px = cls & 1, py = cls >> 1;
    const int tx = 2 * (active ? u % w2 : 0) + px;
    const int ty = 2 * (active ? u / w2 : 0) + py;
    const int p1 = a.p + 1, W = fmm_grid_width(k);
    const float2* A = reinterpret_cast<const float2*>(a.g.A32[k]);
    float2 acc[P1B];
#pragma unroll
    for (int l = 0; l < P1B; ++l) acc[l] = make_float2(0.f, 0.f);
    float2 mono = make_float2(0.f, 0.f);
    for (int dy = -2 - py; dy <= 3 - py; ++dy) {
        for (int dx = -2 - px; dx <= 3 - px; ++dx) {
            if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
            const int d = (dx + 3) + 7 * (dy + 3);
            __syncthreads();
            const float2* Td = a.T + (size_t)d * P1B * P1B;
            for (int e = threadIdx.x; e < P1B * P1B; e += kM2LThreads) Ts[e] = Td[e];
            __syncthreads();
            // sources outside the domain read the zero halo
            const float2* src = A + ((size_t)(ty + dy + FMM_HALO) * W + (tx + dx + FMM_HALO)) * p1;
            float2 m[P1B];
#pragma unroll
            for (int kk = 0; kk < P1B; ++kk) m[kk] = (kk < p1) ? src[kk] : make_float2(0.f, 0.f);
            mono = ff_add(mono, ff_mul(m[0], lv.logc[k][d]));   // M_0 (log|w0| + ln s), float-float
            m[0].y = 0.f;                                        // M_0 is real; .y held its low word
#pragma unroll
            for (int kk = 0; kk < P1B; ++kk) {
#pragma unroll
                for (int l = 0; l < P1B; ++l) {
                    const float2 t = Ts[kk * P1B + l];
                    acc[l].x = fmaf(t.x, m[kk].x, fmaf(-t.y, m[kk].y, acc[l].x));
                    acc[l].y = fmaf(t.x, m[kk].y, fmaf(t.y, m[kk].x, acc[l].y));
                }
            }
        }
    }
    if (!active) return;
    const size_t t = (size_t)ty * (1u << k) + tx;
    float2* B = reinterpret_cast<float2*>(a.g.B[k]);
    B[t * p1] = ff_add_f(mono, acc[0].x);   // Re b'_0 as float-float
#pragma unroll
    for (int l = 1; l < P1B; ++l)
        if (l < p1) B[t * p1 + l] = acc[l];
}

// -------------------------------------------------------------------------------- L2P
// One thread per particle; per level the square's p+1 coefficients are loaded together (the
// order is padded to P1B at compile time, so all loads issue before the Horner chain).
template <int P1B>
__global__ void __launch_bounds__(128)
k_l2p_mixed(const float4* __restrict__ sp, const uint32_t* __restrict__ skey, int64_t n, int levels, int p,
            MixedLevels lv, FmmLevelPtrs g, float2* __restrict__ phi_far) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 P = sp[i];
    const uint32_t key = skey[i];
    const uint32_t ix = fmm_compact2(key), iy = fmm_compact2(key >> 1);
    const int p1 = p + 1;
    float2 far = make_float2(0.f, 0.f);
    for (int k = 2; k <= levels; ++k) {
        const int sh = levels - k;
        const float2 w = level_w(P.x, P.y, ix, iy, sh, lv.inv_s[k]);
        const size_t t = (size_t)(iy >> sh) * (1u << k) + (ix >> sh);
        const float2* Bt = reinterpret_cast<const float2*>(g.B[k]) + t * p1;
        float2 b[P1B];
#pragma unroll
        for (int l = 0; l < P1B; ++l) b[l] = (l < p1) ? __ldg(Bt + l) : make_float2(0.f, 0.f);
        float2 u = b[P1B - 1];
#pragma unroll
        for (int l = P1B - 2; l >= 1; --l) {
            const float ur = fmaf(u.x, w.x, fmaf(-u.y, w.y, b[l].x));
            const float ui = fmaf(u.x, w.y, fmaf(u.y, w.x, b[l].y));
            u.x = ur;
            u.y = ui;
        }
        const float v = fmaf(u.x, w.x, -u.y * w.y);   // Re(u w) = Re sum_{l>=1} b'_l w^l
        far = ff_add(far, ff_add_f(b[0], v));         // b[0] = Re b'_0 as (hi, lo)
    }
    phi_far[i] = far;
}

// -------------------------------------------------------------------------------- P2P + final phi
// One warp per finest square.  When the square and its (up to) eight neighbours hold at most
// kP2PCap sources, the bulk-copy (TMA) engine moves their contiguous Morton ranges into the
// warp's shared-memory buffer (cp.async.bulk completing on an mbarrier, with a bounded wait);
// otherwise the warp reads them from global memory.  With T targets the warp splits into
// 32 / T' groups (T' = T rounded up to a power of two, at most 32) that take interleaved
// sources and combine by shuffles.  Each neighbour's sum runs in FP32 and the neighbours are
// combined in float-float, so crowded squares keep their accuracy.
constexpr int kP2PWarps = 4;
constexpr int kP2PCap = 512;                  // sources per warp buffer (8 KB)
constexpr unsigned kSpinLimit = 1u << 22;     // bounded mbarrier wait

// q-weight of one pair: log2 r^2 by the MUFU unit (flush-to-zero: r^2 of distinct particles is
// normal); self and coincident pairs (r^2 = 0) give 0.
__device__ __forceinline__ float p2p_lg2(float dx, float dy) {
    const float r2 = fmaf(dx, dx, dy * dy);
    float lg;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lg) : "f"(r2));
    return r2 > 0.f ? lg : 0.f;
}

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
    return (uint32_t)__cvta_generic_to_shared(ptr);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (unsigned it = 0; it < kSpinLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred P;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, P;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__global__ void __launch_bounds__(kP2PWarps * 32)
k_p2p_mixed(const float4* __restrict__ sp, const uint32_t* __restrict__ leaf_start,
            const uint32_t* __restrict__ bstart, uint32_t nleaf, int levels, float s_leaf,
            const float2* __restrict__ phi_far, double* __restrict__ phi, unsigned int* __restrict__ status,
            unsigned long long* __restrict__ counters) {
    __shared__ __align__(16) float4 buf[kP2PWarps][kP2PCap];
    __shared__ __align__(8) uint64_t bar[kP2PWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // one warp per block of up to 32 targets of one finest square: crowded squares spread
    // over as many warps as they have target blocks
    const uint32_t w = (uint32_t)blockIdx.x * kP2PWarps + warp;
    if (w >= bstart[nleaf]) return;
    if (*(volatile const unsigned int*)status != 0u) return;   // inputs failed the device checks
    const uint32_t leaf = fmm_warp_search(bstart, nleaf, w, lane);
    const uint32_t tb = w - bstart[leaf];
    const uint32_t t0 = leaf_start[leaf], t1 = leaf_start[leaf + 1];
    const uint32_t b0 = t0 + 32u * tb;
    const int T = (int)min(32u, t1 - b0);
    const int side = 1 << levels;
    const int ix = (int)fmm_compact2(leaf), iy = (int)fmm_compact2(leaf >> 1);
    // the nine neighbour slots, fully unrolled so that they live in registers
    uint32_t nb0[9], ncnt[9], noff[9];
    uint32_t nsrc = 0;
#pragma unroll
    for (int b = 0; b < 9; ++b) {
        const int jx = ix + (b % 3) - 1, jy = iy + (b / 3) - 1;
        const bool in = jx >= 0 && jy >= 0 && jx < side && jy < side;
        const uint32_t nl = in ? fmm_morton((uint32_t)jx, (uint32_t)jy) : 0u;
        nb0[b] = in ? leaf_start[nl] : 0u;
        ncnt[b] = in ? leaf_start[nl + 1] - nb0[b] : 0u;
        noff[b] = nsrc;
        nsrc += ncnt[b];
    }
    if (lane == 0) {
        const unsigned slot = leaf % FMM_COUNTER_SLOTS;
        atomicAdd(&counters[slot], (unsigned long long)T * nsrc - (unsigned long long)T);
        atomicMax(&counters[FMM_COUNTER_SLOTS + slot], (unsigned long long)(t1 - t0));
    }
    const bool staged = nsrc <= (uint32_t)kP2PCap;
    const uint32_t mb = smem_u32(&bar[warp]);
    if (staged) {
        if (lane == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(16u * nsrc)
                         : "memory");
            const uint32_t dst0 = smem_u32(buf[warp]);
#pragma unroll
            for (int b = 0; b < 9; ++b)
                if (ncnt[b] > 0)
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            dst0 + 16u * noff[b]),
                        "l"(sp + nb0[b]), "r"(16u * ncnt[b]), "r"(mb)
                        : "memory");
        }
        __syncwarp();
        if (!mbar_wait(mb, 0)) {
            if (lane == 0) atomicOr(status, FMM_FLAG_TIMEOUT);
            return;   // the copies were issued with valid sizes; nothing else waits on them
        }
        // move every staged source into the target square's frame: x_j + (jx - ix) s, y_j + (jy - iy) s
        float4* sb = buf[warp];
#pragma unroll
        for (int b = 0; b < 9; ++b) {
            const float ox = (float)((b % 3) - 1) * s_leaf, oy = (float)((b / 3) - 1) * s_leaf;
            for (uint32_t j = lane; j < ncnt[b]; j += 32) {
                float4 v = sb[noff[b] + j];
                v.x += ox;
                v.y += oy;
                sb[noff[b] + j] = v;
            }
        }
        __syncwarp();
    }
    int tp = 1;
    while (tp < T) tp <<= 1;
    const uint32_t groups = 32 / tp;
    const int slot = lane & (tp - 1);
    const uint32_t grp = lane / tp;
    const bool active = slot < T;
    const uint32_t gi = b0 + (active ? slot : 0);
    const float4 Pi = sp[gi];
    float2 near = make_float2(0.f, 0.f);
    if (staged) {
        // at most kP2PCap / groups terms per lane: one FP32 sum, four sources per step
        const float4* src = buf[warp];
        float acc0 = 0.f, acc1 = 0.f;
        uint32_t j = grp;
        for (; j + 3u * groups < nsrc; j += 4u * groups) {
            const float4 a0 = src[j], a1 = src[j + groups], a2 = src[j + 2u * groups], a3 = src[j + 3u * groups];
            acc0 = fmaf(a0.z, p2p_lg2(Pi.x - a0.x, Pi.y - a0.y), acc0);
            acc1 = fmaf(a1.z, p2p_lg2(Pi.x - a1.x, Pi.y - a1.y), acc1);
            acc0 = fmaf(a2.z, p2p_lg2(Pi.x - a2.x, Pi.y - a2.y), acc0);
            acc1 = fmaf(a3.z, p2p_lg2(Pi.x - a3.x, Pi.y - a3.y), acc1);
        }
        for (; j < nsrc; j += groups) {
            const float4 a0 = src[j];
            acc0 = fmaf(a0.z, p2p_lg2(Pi.x - a0.x, Pi.y - a0.y), acc0);
        }
        near = make_float2(acc0 + acc1, 0.f);
    } else {
        // crowded squares: FP32 sums over runs of kP2PCap sources from global memory, combined
        // in float-float
#pragma unroll
        for (int b = 0; b < 9; ++b) {
            const float bx = Pi.x - (float)((b % 3) - 1) * s_leaf;   // target-centre minus source-centre
            const float by = Pi.y - (float)((b / 3) - 1) * s_leaf;
            const float4* src = sp + nb0[b];
            for (uint32_t r0 = 0; r0 < ncnt[b]; r0 += kP2PCap) {
                const uint32_t r1 = min(ncnt[b], r0 + kP2PCap);
                float acc0 = 0.f, acc1 = 0.f;
                uint32_t j = r0 + grp;
                for (; j + groups < r1; j += 2u * groups) {
                    const float4 a0 = src[j], a1 = src[j + groups];
                    acc0 = fmaf(a0.z, p2p_lg2(bx - a0.x, by - a0.y), acc0);
                    acc1 = fmaf(a1.z, p2p_lg2(bx - a1.x, by - a1.y), acc1);
                }
                if (j < r1) {
                    const float4 a0 = src[j];
                    acc0 = fmaf(a0.z, p2p_lg2(bx - a0.x, by - a0.y), acc0);
                }
                near = ff_add_f(near, acc0 + acc1);
            }
        }
    }
    for (int o = tp; o < 32; o <<= 1) {
        const float2 other = make_float2(__shfl_xor_sync(0xffffffffu, near.x, o),
                                         __shfl_xor_sync(0xffffffffu, near.y, o));
        near = ff_add(near, other);
    }
    if (active && grp == 0) {
        const float2 v = ff_add(phi_far[gi], ff_mul(near, make_float2(0.3465736f, -9.523271e-10f)));
        phi[__float_as_int(Pi.w)] = fmm_f2d_bits(v.x) + fmm_f2d_bits(v.y);   // ln2 / 2 as float-float above
    }
    if (staged && lane == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(mb) : "memory");
}

template <int P1B>
void launch_m2l(const M2LMixedArgs& a, const MixedLevels& lv, int blocks, cudaStream_t st) {
    k_m2l_f32<P1B><<<blocks, kM2LThreads, 0, st>>>(a, lv);
}

template <int P1B>
void launch_m2l_coarse(const M2LWarpArgs& a, const MixedLevels& lv, int blocks, cudaStream_t st) {
    k_m2l_coarse<P1B><<<blocks, 128, 0, st>>>(a, lv);
}

}  // namespace

int fmm_m2l_bucket(int p1) {
    const int b[] = {9, 13, 17, 21, 25, 33, 41};
    for (int v : b)
        if (p1 <= v) return v;
    return -1;
}

int fmm_launch_mixed(fmm_plan_s* pl, double* phi) {
    if (pl->precision != FMM_MIXED_FP32 && pl->precision != FMM_MIXED_TF32 && pl->precision != FMM_MIXED_3XTF32)
        return -2;
    // in the TF32 modes the tensor-core M2L takes the levels from fmm_tc_kmin() on
    const bool use_tc = pl->tc != nullptr && pl->levels >= fmm_tc_kmin();
    cudaStream_t st = pl->stream;
    const int64_t n = pl->n;
    const int L = pl->levels, p = pl->p, p1 = p + 1;
    const MixedLevels lv = fmm_make_levels(pl);
    int launches = 0;
    cudaEventRecord(pl->ev[1], st);
    if (L >= 2) {
        // fine levels: at most kFineMean particles per square on average
        int kf = L;
        while (kf > 2 && (n >> (2 * (kf - 1))) <= kFineMean) --kf;
        const int kc_max = kf - 1;
        for (int k = 2; k <= kc_max; ++k)
            if (cudaMemsetAsync(pl->grids.A[k], 0, pl->a_bytes[k], st) != cudaSuccess) return -1;
        P2MFineArgs fa{};
        int acc = 0;
        for (int k = kf; k <= L; ++k) {
            fa.base[k] = acc;
            acc += 1 << (2 * k);
        }
        fa.base[L + 1] = acc;
        fa.kf = kf;
        fa.levels = L;
        fa.p = p;
        const unsigned fblocks = (unsigned)((acc + 127) / 128);
        const unsigned cblocks = (unsigned)((n + 4 * kCoarseChunk - 1) / (4 * kCoarseChunk));
        switch (pl->p1b) {
#define FMM_P2M(PB)                                                                                          \
    case PB:                                                                                                 \
        k_p2m_fine<PB><<<fblocks, 128, 0, st>>>(pl->sorted32, pl->sorted_key, pl->leaf_start, fa, lv,        \
                                                pl->grids);                                                  \
        if (kc_max >= 2)                                                                                     \
            k_p2m_coarse<PB><<<cblocks, 128, 0, st>>>(pl->sorted32, pl->sorted_key, n, L, kc_max, p, lv,     \
                                                      pl->grids);                                            \
        break;
            FMM_P2M(9) FMM_P2M(13) FMM_P2M(17) FMM_P2M(21) FMM_P2M(25) FMM_P2M(33) FMM_P2M(41)
#undef FMM_P2M
            default: return -2;
        }
        launches += kc_max >= 2 ? 2 : 1;
        for (int k = 2; k <= kc_max; ++k) {
            const int64_t count = (int64_t)fmm_grid_width(k) * fmm_grid_width(k) * p1;
            k_prep_a32<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(
                reinterpret_cast<const double2*>(pl->grids.A[k]), reinterpret_cast<float2*>(pl->grids.A32[k]), count,
                p1);
            ++launches;
        }
    }
    cudaEventRecord(pl->ev[2], st);
    if (L >= 2) {
        // coarse levels: a CTA per 4 x kM2LWarpTargets targets of one class
        M2LWarpArgs wa;
        wa.g = pl->grids;
        wa.T = pl->T32;
        wa.p = p;
        wa.kw = L < kM2LWarpMaxLevel ? L : kM2LWarpMaxLevel;
        int wacc = 0;
        for (int k = 0; k <= FMM_MAX_LEVELS + 1; ++k) wa.cbase[k] = 0;
        for (int k = 2; k <= wa.kw; ++k) {
            wa.cbase[k] = wacc;
            wacc += 4 * (((1 << (2 * (k - 1))) + 4 * kM2LWarpTargets - 1) / (4 * kM2LWarpTargets));
        }
        wa.cbase[wa.kw + 1] = wacc;
        switch (pl->p1b) {
            case 9: launch_m2l_coarse<9>(wa, lv, wacc, st); break;
            case 13: launch_m2l_coarse<13>(wa, lv, wacc, st); break;
            case 17: launch_m2l_coarse<17>(wa, lv, wacc, st); break;
            case 21: launch_m2l_coarse<21>(wa, lv, wacc, st); break;
            case 25: launch_m2l_coarse<25>(wa, lv, wacc, st); break;
            case 33: launch_m2l_coarse<33>(wa, lv, wacc, st); break;
            case 41: launch_m2l_coarse<41>(wa, lv, wacc, st); break;
            default: return -2;
        }
        ++launches;
        // finer levels: one thread per target, or the tensor cores
        M2LMixedArgs a;
        a.g = pl->grids;
        a.T = pl->T32;
        a.levels = L;
        a.p = p;
        a.kmin = wa.kw + 1;
        a.kmax = use_tc ? fmm_tc_kmin() - 1 : L;
        int acc = 0;
        for (int k = 0; k <= FMM_MAX_LEVELS + 1; ++k) a.cta_base[k] = 0;
        for (int k = a.kmin; k <= a.kmax; ++k) {
            a.cta_base[k] = acc;
            const int w2 = 1 << (k - 1);
            acc += 4 * ((w2 * w2 + kM2LThreads - 1) / kM2LThreads);
        }
        a.cta_base[a.kmax + 1] = acc;
        if (acc > 0) {
            switch (pl->p1b) {
                case 9: launch_m2l<9>(a, lv, acc, st); break;
                case 13: launch_m2l<13>(a, lv, acc, st); break;
                case 17: launch_m2l<17>(a, lv, acc, st); break;
                case 21: launch_m2l<21>(a, lv, acc, st); break;
                case 25: launch_m2l<25>(a, lv, acc, st); break;
                case 33: launch_m2l<33>(a, lv, acc, st); break;
                case 41: launch_m2l<41>(a, lv, acc, st); break;
                default: return -2;
            }
            ++launches;
        }
        if (use_tc) {
            const int t = fmm_launch_m2l_tc(pl, lv);
            if (t < 0) return -1;
            launches += t;
        }
    }
    cudaEventRecord(pl->ev[3], st);
    float2* far = reinterpret_cast<float2*>(pl->phi_far);
    {
        const unsigned blocks = (unsigned)((n + 127) / 128);
        switch (pl->p1b) {
#define FMM_L2P(PB)                                                                                          \
    case PB:                                                                                                 \
        k_l2p_mixed<PB><<<blocks, 128, 0, st>>>(pl->sorted32, pl->sorted_key, n, L, p, lv, pl->grids, far);  \
        break;
            FMM_L2P(9) FMM_L2P(13) FMM_L2P(17) FMM_L2P(21) FMM_L2P(25) FMM_L2P(33) FMM_L2P(41)
#undef FMM_L2P
            default: return -2;
        }
        ++launches;
    }
    cudaEventRecord(pl->ev[4], st);
    {
        const uint32_t nleaf = 1u << (2 * L);
        const int r = fmm_launch_leaf_blocks(pl->leaf_start, nleaf, pl->leaf_nb, pl->block_sums, pl->leaf_bstart, st);
        if (r < 0) return -1;
        launches += r;
        // upper bound of the target blocks: each square adds at most one partial block
        const uint64_t wmax = (uint64_t)nleaf + (uint64_t)(n / 32) + 1;
        const unsigned blocks = (unsigned)((wmax + kP2PWarps - 1) / kP2PWarps);
        k_p2p_mixed<<<blocks, kP2PWarps * 32, 0, st>>>(pl->sorted32, pl->leaf_start, pl->leaf_bstart, nleaf, L,
                                                      lv.s_leaf, far, phi, pl->d_status, pl->d_counters);
        ++launches;
    }
    cudaEventRecord(pl->ev[5], st);
    if (cudaGetLastError() != cudaSuccess) return -1;
    return launches;
}
