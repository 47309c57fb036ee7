// mixed.cu -- the mixed-precision path: FP32 particle stages and FP32 M2L on the CUDA cores,
// with float-float (two FP32 words) wherever magnitudes are large.  GB300's FP64 pipe is far
// narrower than its FP32 pipe, so no FP64 arithmetic runs inside the hot loops: FP64 appears
// only in the near field's atomic sums (executed in L2) and in the final phi written for the
// caller.
//
// Scaled form as in fp64.cu (w = (z - c) / s, power-sum moments M_m = sum q w^m):
//   P2M  the finest three levels straight from the particles (U-bar-1 of Sec. 2.2.1): w in FP32
//        from the particle's offset to its finest-square centre (an exact dyadic square offset
//        plus an FP32 product), q w^m in FP32, register and shuffle sums; the total charge M_0
//        (real) is kept as a float-float pair (hi, lo) in the slot of coefficient 0.
//   M2M  the coarser levels by the upward pass (U-bar-2): each parent the sum of its four
//        children's moments re-expanded about its centre (exact for truncated expansions).
//   M2L  (D-bar-1) per target: b'_l = sum_d sum_k T_d[k][l] M[t+d][k] in FP32 (k, l = 0..p),
//        except the monopole-log term sum_d M_0 (log|w0| + ln s) of b'_0, summed in
//        float-float; Re b'_0 is stored as a float-float pair in the slot of coefficient 0.
//   L2P  (D-bar-2 by linearity) per particle and level: Re sum_{l>=1} b'_l w^l by Horner in
//        FP32, plus Re b'_0; the levels are summed in float-float.
//   P2P  (E-2 of Sec. 2.1) in FP32 on square-local coordinates, log via the MUFU lg2 unit,
//        lanes over sources and one register partial per target; phi = far + near.
#include "mixed_common.cuh"
#include "p2p_block.cuh"

namespace {

constexpr int kM2LThreads = 128;

// -------------------------------------------------------------------------------- P2M
// The fine levels straight from the particles (U-bar-1 of Sec. 2.2.1).  Squares of a level are
// contiguous Morton ranges of the sorted particles, so the sums need no global sort of their own.
//
// Fine levels (the finest three, l - 2 .. l): two lanes per finest square, 16 consecutive squares
// per warp in Morton order, so that each group of 2 * 4^(l - k) consecutive lanes is one level-k
// square.  For each level a lane sums its half of the square's particles in registers (the
// square fixes the particles' offsets inside every coarser square, so no key is read), then the
// group's partial sums are combined by a shuffle reduce-scatter that leaves each lane of the
// group with a share of the coefficients to store: no atomics, coalesced stores.  Squares above
// kLaneMax particles are summed by the whole warp and added by the owning group before the store.
//
// Coarse levels (2 .. l - 3): the upward pass from the fine levels' moments (k_m2m_f32).
constexpr int kFineLevels = 3;
constexpr int kLaneMax = FMM_LANE_MAX;
constexpr int kCoarseChunk = 256;

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

// Sum over each aligned group of G lanes of v[0 .. VP), scattered: afterwards the lane of rank r
// in its group holds entries [r VP / G, (r + 1) VP / G) of the group's sum in v[0 .. VP / G).
// At the step with mask m a lane keeps the half of its live blocks whose bit m matches its own
// rank bit and sends the other half to its partner.
template <int G, int VP>
__device__ __forceinline__ void group_reduce_scatter(float (&v)[VP], int lane) {
    constexpr int B = VP / G;
#pragma unroll
    for (int m = G / 2; m >= 1; m >>= 1) {
        const bool up = (lane & m) != 0;
#pragma unroll
        for (int i = 0; i < m * B; ++i) {
            const float send = up ? v[i] : v[i + m * B];
            const float keep = up ? v[i + m * B] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
        }
    }
}

// Level k = l - log4(G) of the lane's finest square sq (particles [lo, hi), offset (ox, oy) of
// its centre in units of the level-k square): the group's sums of the lane partials acc and m0,
// the crowded squares of the warp added, stored by the group's lanes.
template <int P1B, int G, int SH>
__device__ __forceinline__ void p2m_fine_finish(const float2 (&acc)[P1B], float2 m0, const float4* __restrict__ sp,
                                                uint32_t sq, uint32_t lo, uint32_t hi, bool valid, bool owner,
                                                int levels, int p1, float inv_s, float ox, float oy, float* red,
                                                int lane, FmmLevelPtrs g, bool ext) {
    constexpr int V = 2 * (P1B - 1);              // Re, Im of coefficients 1 .. P1B - 1
    constexpr int VP = (V + G - 1) / G * G;
    constexpr int B = VP / G;
    const int k = levels - SH;
    const bool large = hi - lo > (uint32_t)kLaneMax;
    float v[VP];
#pragma unroll
    for (int i = 0; i < VP; ++i) v[i] = i < V ? ((i & 1) ? acc[1 + i / 2].y : acc[1 + i / 2].x) : 0.f;
    group_reduce_scatter<G, VP>(v, lane);
#pragma unroll
    for (int m = 1; m < G; m <<= 1)
        m0 = ff_add(m0, make_float2(__shfl_xor_sync(0xffffffffu, m0.x, m), __shfl_xor_sync(0xffffffffu, m0.y, m)));
    // crowded squares: the whole warp sums the particles, the owning group adds its share (with
    // `ext`, k_p2m_crowded adds their coefficients 1..p afterwards and the warp sums only the
    // total charge, in float-float)
    unsigned todo = __ballot_sync(0xffffffffu, valid && large && owner);
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const uint32_t lo2 = __shfl_sync(0xffffffffu, lo, src), hi2 = __shfl_sync(0xffffffffu, hi, src);
        const float ox2 = __shfl_sync(0xffffffffu, ox, src), oy2 = __shfl_sync(0xffffffffu, oy, src);
        float2 a2[P1B];
#pragma unroll
        for (int m = 0; m < P1B; ++m) a2[m] = make_float2(0.f, 0.f);
        float2 mm = make_float2(0.f, 0.f);
        if (ext) {
            for (uint32_t j = lo2 + lane; j < hi2; j += 32) mm = ff_add_f(mm, sp[j].z);
        } else {
            for (uint32_t j = lo2 + lane; j < hi2; j += 32) {
                const float4 P = sp[j];
                mm = ff_add_f(mm, P.z);
                add_powers<P1B>(a2, P.z, make_float2(fmaf(P.x, inv_s, ox2), fmaf(P.y, inv_s, oy2)));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mm = ff_add(mm, make_float2(__shfl_xor_sync(0xffffffffu, mm.x, o), __shfl_xor_sync(0xffffffffu, mm.y, o)));
            if (!ext) {
#pragma unroll
                for (int m = 1; m < P1B; ++m) {
                    a2[m].x += __shfl_xor_sync(0xffffffffu, a2[m].x, o);
                    a2[m].y += __shfl_xor_sync(0xffffffffu, a2[m].y, o);
                }
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int m = 1; m < P1B; ++m) {
                red[2 * (m - 1)] = a2[m].x;
                red[2 * (m - 1) + 1] = a2[m].y;
            }
        }
        __syncwarp();
        if ((lane & ~(G - 1)) == (src & ~(G - 1))) {
            const int r = lane & (G - 1);
#pragma unroll
            for (int i = 0; i < B; ++i)
                if (r * B + i < V) v[i] += red[r * B + i];
            m0 = ff_add(m0, mm);
        }
        __syncwarp();
    }
    if (!valid) return;
    const uint32_t b = sq >> (2 * SH);
    const int W = fmm_grid_width(k);
    const size_t cell = (size_t)(fmm_compact2(b >> 1) + FMM_HALO) * W + fmm_compact2(b) + FMM_HALO;
    float* A = reinterpret_cast<float*>(reinterpret_cast<float2*>(g.A32[k]) + cell * p1);
    const int r = lane & (G - 1);
#pragma unroll
    for (int i = 0; i < B; ++i) {
        const int e = r * B + i;
        if (e < 2 * (p1 - 1)) A[2 + e] = v[i];
    }
    if (r == 0) {
        A[0] = m0.x;   // total charge as a float-float pair
        A[1] = m0.y;
    }
}

// offset of the finest square's centre in units of its ancestor SH levels up: exact dyadic
__device__ __forceinline__ float fine_offset(uint32_t i, int sh) {
    const uint32_t mask = (1u << sh) - 1u;
    return fmaf((float)(i & mask) + 0.5f, __int_as_float((127 - sh) << 23), -0.5f);
}

// two particles' power chains in packed FP32x2 (lane a, lane b of each register pair): ar[m]
// accumulates (Re of a, Re of b), ai[m] (Im of a, Im of b)
template <int P1B>
__device__ __forceinline__ void add_powers_pair(float2 (&ar)[P1B], float2 (&ai)[P1B], float2 q2, float2 wx,
                                                float2 wy) {
    const float2 nwy = make_float2(-wy.x, -wy.y);
    float2 pr = q2, pi = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 1; m < P1B; ++m) {
        const float2 nr = __ffma2_rn(pr, wx, __fmul2_rn(pi, nwy));
        const float2 ni = __ffma2_rn(pr, wy, __fmul2_rn(pi, wx));
        pr = nr;
        pi = ni;
        ar[m] = __fadd2_rn(ar[m], pr);
        ai[m] = __fadd2_rn(ai[m], pi);
    }
}

// levels max(2, l - 2) .. l, two lanes per finest square, each taking half of its particles.  Per
// level a lane walks its half two particles at a time, the pair's power chains in packed FP32x2
// arithmetic (the particles stay in L1 between the levels' passes); the total charge is summed
// once, in float-float.  The two halves join in the group reductions (2, 8 and 32 lanes).
template <int P1B>
__global__ void __launch_bounds__(128, P1B <= 25 ? 4 : 1)
k_p2m_fine(const float4* __restrict__ sp, const uint32_t* __restrict__ leaf_start, int levels, int p, MixedLevels lv,
           FmmLevelPtrs g, int ext) {
    __shared__ float red[4][2 * P1B];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t t = blockIdx.x * 128u + threadIdx.x;
    const uint32_t sq = t >> 1;
    const bool owner = (t & 1u) == 0u;
    const bool valid = sq < (1u << (2 * levels));
    const uint32_t lo = valid ? leaf_start[sq] : 0u, hi = valid ? leaf_start[sq + 1] : 0u;
    const bool walk = valid && hi - lo <= (uint32_t)kLaneMax;   // crowded squares: the whole warp
    const uint32_t mid = lo + ((hi - lo + 1u) >> 1);
    const uint32_t a0 = owner ? lo : mid, a1 = owner ? mid : hi;   // this lane's half
    const int p1 = p + 1;
    const uint32_t ix = fmm_compact2(sq), iy = fmm_compact2(sq >> 1);
    float2 m0 = make_float2(0.f, 0.f);
    if (walk)
        for (uint32_t j = a0; j < a1; ++j) m0 = ff_add_f(m0, sp[j].z);
#pragma unroll 1
    for (int sh = 0; sh < kFineLevels; ++sh) {
        if (levels - sh < 2) break;
        const float s = lv.inv_s[levels - sh];
        const float ox = sh == 0 ? 0.f : fine_offset(ix, sh), oy = sh == 0 ? 0.f : fine_offset(iy, sh);
        const float2 s2 = make_float2(s, s), ox2 = make_float2(ox, ox), oy2 = make_float2(oy, oy);
        float2 ar[P1B], ai[P1B];
#pragma unroll
        for (int m = 0; m < P1B; ++m) ar[m] = ai[m] = make_float2(0.f, 0.f);
        if (walk && a0 < a1) {
            // pairs (j, j + 1); an odd count ends with a zero-charge partner
            float4 na = sp[a0], nb = a0 + 1 < a1 ? sp[a0 + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
            for (uint32_t j = a0; j < a1; j += 2) {
                const float4 a = na, b = nb;
                if (j + 2 < a1) na = sp[j + 2];
                nb = j + 3 < a1 ? sp[j + 3] : make_float4(0.f, 0.f, 0.f, 0.f);
                add_powers_pair<P1B>(ar, ai, make_float2(a.z, b.z), __ffma2_rn(make_float2(a.x, b.x), s2, ox2),
                                     __ffma2_rn(make_float2(a.y, b.y), s2, oy2));
            }
        }
        float2 acc[P1B];
#pragma unroll
        for (int m = 0; m < P1B; ++m) acc[m] = make_float2(ar[m].x + ar[m].y, ai[m].x + ai[m].y);
        if (sh == 0)
            p2m_fine_finish<P1B, 2, 0>(acc, m0, sp, sq, lo, hi, valid, owner, levels, p1, s, ox, oy, red[warp], lane,
                                       g, ext != 0);
        else if (sh == 1)
            p2m_fine_finish<P1B, 8, 1>(acc, m0, sp, sq, lo, hi, valid, owner, levels, p1, s, ox, oy, red[warp], lane,
                                       g, ext != 0);
        else
            p2m_fine_finish<P1B, 32, 2>(acc, m0, sp, sq, lo, hi, valid, owner, levels, p1, s, ox, oy, red[warp],
                                        lane, g, ext != 0);
    }
}

// Fine levels of crowded finest squares (above kLaneMax particles), spread over the whole grid
// instead of one warp per square: each warp walks kCoarseChunk consecutive sorted particles, takes
// those of crowded squares and, per fine level, adds their power chains in registers while their
// level-k square stays the same, flushing (a warp butterfly sum, then FP32 atomics into the level's
// FP32 grid) when it changes.  k_p2m_fine, run first in its `ext` mode, has stored every square's
// other shares and the crowded squares' total charge, so these adds complete coefficients 1..p.
template <int P1B>
__global__ void __launch_bounds__(128)
k_p2m_crowded(const float4* __restrict__ sp, const uint32_t* __restrict__ skey, const uint32_t* __restrict__ leaf_start,
              int64_t n, int levels, int p, MixedLevels lv, FmmLevelPtrs g) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = ((int64_t)blockIdx.x * 4 + warp) * kCoarseChunk;
    if (base >= n) return;
    const int p1 = p + 1;
    uint32_t cmask = 0;   // bit r: particle base + 32 r + lane lies in a crowded finest square
#pragma unroll
    for (int r = 0; r < kCoarseChunk / 32; ++r) {
        const int64_t j = base + 32 * r + lane;
        if (j < n) {
            const uint32_t key = skey[j];
            if (leaf_start[key + 1] - leaf_start[key] > (uint32_t)kLaneMax) cmask |= 1u << r;
        }
    }
    if (!__any_sync(0xffffffffu, cmask != 0u)) return;
#pragma unroll 1
    for (int sh = 0; sh < kFineLevels; ++sh) {
        const int k = levels - sh;
        if (k < 2) break;
        const int W = fmm_grid_width(k);
        float2* A = reinterpret_cast<float2*>(g.A32[k]);
        const float inv_s = lv.inv_s[k];
        float2 acc[P1B];
#pragma unroll
        for (int m = 0; m < P1B; ++m) acc[m] = make_float2(0.f, 0.f);
        uint32_t cur = 0xffffffffu;   // the level-k square the sums belong to (warp-uniform)
        auto flush = [&]() {
#pragma unroll
            for (int m = 1; m < P1B; ++m)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    acc[m].x += __shfl_xor_sync(0xffffffffu, acc[m].x, o);
                    acc[m].y += __shfl_xor_sync(0xffffffffu, acc[m].y, o);
                }
            const size_t cell = (size_t)(fmm_compact2(cur >> 1) + FMM_HALO) * W + fmm_compact2(cur) + FMM_HALO;
            float2* Ac = A + cell * p1;
#pragma unroll
            for (int m = 1; m < P1B; ++m) {
                if (m < p1 && lane == (m & 31)) {
                    atomicAdd(&Ac[m].x, acc[m].x);
                    atomicAdd(&Ac[m].y, acc[m].y);
                }
                acc[m] = make_float2(0.f, 0.f);
            }
        };
#pragma unroll 1
        for (int r = 0; r < kCoarseChunk / 32; ++r) {
            const bool act = (cmask >> r) & 1u;
            const int64_t j = base + 32 * r + lane;
            float4 P = make_float4(0.f, 0.f, 0.f, 0.f);
            uint32_t key = 0u, box = 0xffffffffu;
            if (act) {
                P = sp[j];
                key = skey[j];
                box = key >> (2 * sh);
            }
            // the keys are sorted, so the lanes of one square are consecutive: each pass takes the
            // square of the first lane still to add, at most 32 passes
            unsigned todo = __ballot_sync(0xffffffffu, act);
            while (todo) {
                const uint32_t first = __shfl_sync(0xffffffffu, box, __ffs(todo) - 1);
                if (first != cur) {
                    if (cur != 0xffffffffu) flush();
                    cur = first;
                }
                const bool mine = ((todo >> lane) & 1u) && box == cur;
                if (mine)
                    add_powers<P1B>(acc, P.z, level_w(P.x, P.y, fmm_compact2(key), fmm_compact2(key >> 1), sh, inv_s));
                todo &= ~__ballot_sync(0xffffffffu, mine);
            }
        }
        if (cur != 0xffffffffu) flush();
    }
}

// Upward pass (U-bar-2 of Sec. 2.2.1) for the coarse levels: the parent's moments are the sum of
// its four children's, each re-expanded about the parent's centre.  With w = (z - c) / s_k per
// level, a child's w' relates to its parent's as w = w' / 2 + d_c, so
//     M_m(parent) = sum_c sum_{j <= m} U_c[m][j] M_j(child c),   U_c[m][j] = C(m, j) 2^-j d_c^(m-j),
// a finite sum, exact for the truncated expansions (the same moments the particles give directly).
// U comes from the plan ([c][j][m]: FP64 build, one FP32 rounding, zero above the diagonal and
// past p).  Two parents a CTA, one thread per coefficient m; the total charge (slot 0, a
// float-float pair) is the children's float-float sum.
constexpr int kM2MThreads = 64;   // per parent: coefficients 0 .. P1B - 1 (P1B <= 41)

template <int P1B>
__global__ void __launch_bounds__(2 * kM2MThreads)
k_m2m_f32(const float2* __restrict__ child, float2* __restrict__ parent, const float2* __restrict__ U, int k,
          int p1) {
    static_assert(P1B <= kM2MThreads, "one thread per coefficient");
    // U is staged in shared memory, all four children's at once where they fit (one round trip to
    // L2 instead of a chain of dependent loads per thread), else one child's at a time
    constexpr int UC = 4 * P1B * P1B * (int)sizeof(float2) <= 40 * 1024 ? 4 : 1;
    __shared__ float2 mom[2][4][P1B];   // the children's moments, slot 0 = M_0 as (hi, lo)
    __shared__ float2 us[UC * P1B * P1B];
    const int half = threadIdx.x / kM2MThreads, m = threadIdx.x % kM2MThreads;
    const uint32_t side = 1u << k;
    const uint32_t par = blockIdx.x * 2u + (uint32_t)half;   // row-major parent index
    const bool live = par < side * side;
    const uint32_t px = par % side, py = par / side;
    const int Wc = fmm_grid_width(k + 1), Wp = fmm_grid_width(k);
    if (m < P1B) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float2 v = make_float2(0.f, 0.f);
            if (live && m < p1) {
                const size_t cell = (size_t)(2 * py + (c >> 1) + FMM_HALO) * Wc + 2 * px + (c & 1) + FMM_HALO;
                v = child[cell * p1 + m];
            }
            mom[half][c][m] = v;
        }
    }
    const bool work = live && m >= 1 && m < p1;
    float re = 0.f, im = 0.f;
#pragma unroll
    for (int c0 = 0; c0 < 4; c0 += UC) {
        // every thread's loads issued before its stores: one round trip to L2, not one per element
        constexpr int NU = UC * P1B * P1B, R = (NU + 2 * kM2MThreads - 1) / (2 * kM2MThreads);
        float2 stage[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = threadIdx.x + r * 2 * kM2MThreads;
            stage[r] = i < NU ? __ldg(U + (size_t)c0 * P1B * P1B + i) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = threadIdx.x + r * 2 * kM2MThreads;
            if (i < NU) us[i] = stage[r];
        }
        __syncthreads();
        if (work) {
#pragma unroll
            for (int cc = 0; cc < UC; ++cc) {
                const float2* u = us + cc * P1B * P1B + m;   // U_c[m][j] at u[j P1B]
                const float2 m0 = mom[half][c0 + cc][0];
                const float q0 = m0.x + m0.y;   // M_0 from its float-float pair
                float r = u[0].x * q0, t = u[0].y * q0;
#pragma unroll
                for (int j = 1; j < P1B; ++j) {   // U is zero past m
                    const float2 uj = u[j * P1B], mj = mom[half][c0 + cc][j];
                    r = fmaf(uj.x, mj.x, fmaf(-uj.y, mj.y, r));
                    t = fmaf(uj.x, mj.y, fmaf(uj.y, mj.x, t));
                }
                re += r;
                im += t;
            }
        }
        __syncthreads();
    }
    if (!live || m >= p1) return;
    float2 out;
    if (m == 0) {
        out = mom[half][0][0];
#pragma unroll
        for (int c = 1; c < 4; ++c) out = ff_add(out, mom[half][c][0]);
    } else {
        out = make_float2(re, im);
    }
    const size_t pcell = (size_t)(py + FMM_HALO) * Wp + px + FMM_HALO;
    parent[pcell * p1 + m] = out;
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
constexpr int kM2LWarpMaxLevel = 5;   // 4^5 targets: the finest level this kernel takes

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

// -------------------------------------------------------------------------------- L2P + final phi
// One thread per particle; per level the square's p+1 coefficients are loaded together (the
// order is padded to P1B at compile time, so all loads issue before the Horner chain; kExact:
// p + 1 == P1B, so no load needs a guard).  The levels are summed in float-float, the particle's
// near field (from the P2P kernel, which runs concurrently with P2P and M2L on a second stream)
// is added, and phi is written in input order unless the inputs failed the device checks.
// u z + c for complex u, z, c (FP32)
__device__ __forceinline__ float2 cfma(float2 u, float2 z, float2 c) {
    return make_float2(fmaf(u.x, z.x, fmaf(-u.y, z.y, c.x)), fmaf(u.x, z.y, fmaf(u.y, z.x, c.y)));
}

// Re sum_{l=1}^{P1B-1} b_l w^l, the even and odd powers as two Horner chains in z = w^2
template <int P1B>
__device__ __forceinline__ float l2p_split_horner(const float2 (&b)[P1B], float2 w) {
    static_assert(P1B >= 2, "at least b_0 and b_1");
    constexpr int LO = (P1B - 1) % 2 == 1 ? P1B - 1 : P1B - 2;   // highest odd index
    constexpr int LE = (P1B - 1) % 2 == 0 ? P1B - 1 : P1B - 2;   // highest even index
    const float2 z = make_float2(fmaf(w.x, w.x, -w.y * w.y), 2.f * w.x * w.y);
    float2 o = b[LO];
#pragma unroll
    for (int l = LO - 2; l >= 1; l -= 2) o = cfma(o, z, b[l]);
    float v = fmaf(o.x, w.x, -o.y * w.y);   // Re(w O)
    if constexpr (LE >= 2) {
        float2 e = b[LE];
#pragma unroll
        for (int l = LE - 2; l >= 2; l -= 2) e = cfma(e, z, b[l]);
        v += fmaf(e.x, z.x, -e.y * z.y);   // Re(z E)
    }
    return v;
}

// Levels k_lo..k_hi.  far_out: the float-float sum of those levels is stored per particle and
// nothing else (the coarse levels, on the third stream once their M2L is done); otherwise the sum
// continues from far_in (if given), the near field is added and phi written.  Either way the
// levels are added in the same order as in one pass over 2..levels, so the result is the same.
template <int P1B, bool kExact>
__global__ void __launch_bounds__(128)
k_l2p_mixed(const float4* __restrict__ sp, const uint32_t* __restrict__ skey, int64_t n, int levels, int k_lo,
            int k_hi, int p, MixedLevels lv, FmmLevelPtrs g, const float2* __restrict__ far_in,
            float2* __restrict__ far_out, const double* __restrict__ near, const unsigned int* __restrict__ status,
            double* __restrict__ phi) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double nd = far_out ? 0.0 : near[i];
    const float4 P = sp[i];
    const uint32_t key = skey[i];
    const uint32_t ix = fmm_compact2(key), iy = fmm_compact2(key >> 1);
    const int p1 = p + 1;
    float2 far = far_in ? far_in[i] : make_float2(0.f, 0.f);
    for (int k = k_lo; k <= k_hi; ++k) {
        const int sh = levels - k;
        const float2 w = level_w(P.x, P.y, ix, iy, sh, lv.inv_s[k]);
        const size_t t = (size_t)(iy >> sh) * (1u << k) + (ix >> sh);
        const float2* Bt = reinterpret_cast<const float2*>(g.B[k]) + t * p1;
        float2 b[P1B];
#pragma unroll
        for (int l = 0; l < P1B; ++l) b[l] = (kExact || l < p1) ? __ldg(Bt + l) : make_float2(0.f, 0.f);
        // Re sum_{l>=1} b'_l w^l = Re(z E(z) + w O(z)) with z = w^2, E(z) = sum_{m>=1} b'_{2m} z^(m-1),
        // O(z) = sum_{m>=0} b'_{2m+1} z^m: two independent Horner chains of half the length
        const float v = l2p_split_horner<P1B>(b, w);
        far = ff_add(far, ff_add_f(b[0], v));         // b[0] = Re b'_0 as (hi, lo)
    }
    if (far_out) {
        far_out[i] = far;
        return;
    }
    if (*(volatile const unsigned int*)status != 0u) return;   // inputs failed the device checks
    phi[__float_as_int(P.w)] = p2p_phi(far, fmm_d2ff_bits(nd));
}

// L2P with the field: per level the local expansion F(w) = sum_{l>=1} b'_l w^l and its derivative by
// one Horner pass (q <- q w + b_l, d <- d w + q), f'(z) = F'(w) / s_k, grad phi = (Re f', -Im f'),
// levels summed in float-float; E = -(far + near gradient) written as (Ex, Ey) in input order.
template <int P1B>
__global__ void __launch_bounds__(128)
k_l2p_field(const float4* __restrict__ sp, const uint32_t* __restrict__ skey, int64_t n, int levels, int p,
            MixedLevels lv, FmmLevelPtrs g, const double* __restrict__ near, const double2* __restrict__ nearg,
            const unsigned int* __restrict__ status, double* __restrict__ phi, double* __restrict__ field) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double nd = near[i];
    const double2 ng = nearg[i];
    const float4 P = sp[i];
    const uint32_t key = skey[i];
    const uint32_t ix = fmm_compact2(key), iy = fmm_compact2(key >> 1);
    const int p1 = p + 1;
    float2 far = make_float2(0.f, 0.f), gx = make_float2(0.f, 0.f), gy = make_float2(0.f, 0.f);
    for (int k = 2; k <= levels; ++k) {
        const int sh = levels - k;
        const float2 w = level_w(P.x, P.y, ix, iy, sh, lv.inv_s[k]);
        const size_t t = (size_t)(iy >> sh) * (1u << k) + (ix >> sh);
        const float2* Bt = reinterpret_cast<const float2*>(g.B[k]) + t * p1;
        float2 b[P1B];
#pragma unroll
        for (int l = 0; l < P1B; ++l) b[l] = l < p1 ? __ldg(Bt + l) : make_float2(0.f, 0.f);
        float2 q = b[P1B - 1], d = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = P1B - 2; l >= 1; --l) {
            d = cfma(d, w, q);
            q = cfma(q, w, b[l]);
        }
        d = cfma(d, w, q);                                  // F'(w)
        const float v = fmaf(q.x, w.x, -q.y * w.y);        // Re F(w)
        far = ff_add(far, ff_add_f(b[0], v));
        gx = ff_add_f(gx, d.x * lv.inv_s[k]);
        gy = ff_add_f(gy, -d.y * lv.inv_s[k]);
    }
    if (*(volatile const unsigned int*)status != 0u) return;   // inputs failed the device checks
    const int idx = __float_as_int(P.w);
    phi[idx] = p2p_phi(far, fmm_d2ff_bits(nd));
    field[2 * (int64_t)idx] = -(fmm_f2d_bits(gx.x) + fmm_f2d_bits(gx.y) + ng.x);
    field[2 * (int64_t)idx + 1] = -(fmm_f2d_bits(gy.x) + fmm_f2d_bits(gy.y) + ng.y);
}

// -------------------------------------------------------------------------------- P2P
// One warp per block of up to FMM_P2P_BLOCK targets of one finest square (the block -> square map
// spares the warp a search); crowded squares spread over as many warps as they have blocks.  The
// block's near field is p2p_near_sym (p2p_block.cuh): the own square in full and the four forward
// neighbours once for both sides, every result added in FP64 to the per-particle accumulator
// `acc` (log2 r^2 units, sorted order; cleared at the start of each call), which L2P adds to phi.
// The kernel needs only the sort's output, so it runs on a second stream beside P2M and M2L.
constexpr int kP2PWarps = 4;

__global__ void __launch_bounds__(kP2PWarps * 32, 8)
k_p2p_mixed(const float4* __restrict__ sp, const uint32_t* __restrict__ leaf_start,
            const uint32_t* __restrict__ bstart, const uint2* __restrict__ bmap, uint32_t nleaf, int levels,
            float s_leaf, double* __restrict__ acc, unsigned int* __restrict__ status,
            unsigned long long* __restrict__ counters) {
    __shared__ __align__(16) float4 tgt[kP2PWarps][16];   // zero past the block's targets
    __shared__ __align__(16) float2 tq[kP2PWarps][16];
    __shared__ __align__(16) int4 seg[kP2PWarps][4];      // forward neighbours: {index - slot, ox, oy, -}
    static_assert(FMM_P2P_BLOCK <= 24, "p2p_near_sym takes blocks of up to 24 targets");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t w = (uint32_t)blockIdx.x * kP2PWarps + warp;
    // the map has an entry for every warp of the grid (its size is the grid's bound), so it is
    // read together with the bound and the status word
    const uint2 lt = bmap[w];   // (square, block inside it)
    if (w >= bstart[nleaf]) return;
    if (*(volatile const unsigned int*)status != 0u) return;   // inputs failed the device checks
    const uint32_t leaf = lt.x;
    const uint32_t t0 = leaf_start[leaf], t1 = leaf_start[leaf + 1];
    const uint32_t b0 = t0 + (uint32_t)FMM_P2P_BLOCK * lt.y;
    const int T = (int)min((uint32_t)FMM_P2P_BLOCK, t1 - b0);
    uint32_t pairs;
    const float2 near = p2p_near_sym(sp, leaf_start, leaf, t0, t1, b0, T, levels, s_leaf, tgt[warp], tq[warp],
                                     seg[warp], lane, acc, &pairs);
    if (lane == 0) {
        const unsigned slot = leaf % FMM_COUNTER_SLOTS;
        atomicAdd(&counters[slot], (unsigned long long)pairs);
        atomicMax(&counters[FMM_COUNTER_SLOTS + slot], (unsigned long long)(t1 - t0));
    }
    if (lane < T) atomicAdd(acc + b0 + lane, fmm_f2d_bits(near.x) + fmm_f2d_bits(near.y));
}

// The near field with the gradient (fmm_potential_field): p2p_near_sym_field, the gradient sums
// added to accg beside phi's to acc.  Three accumulators per target: fewer warps per SM.
__global__ void __launch_bounds__(kP2PWarps * 32, 4)
k_p2p_field(const float4* __restrict__ sp, const uint32_t* __restrict__ leaf_start,
            const uint32_t* __restrict__ bstart, const uint2* __restrict__ bmap, uint32_t nleaf, int levels,
            float s_leaf, const float2* __restrict__ lo, double* __restrict__ acc, double2* __restrict__ accg,
            unsigned int* __restrict__ status, unsigned long long* __restrict__ counters) {
    __shared__ __align__(16) float4 tgt[kP2PWarps][16];
    __shared__ __align__(16) float4 tlo[kP2PWarps][16];
    __shared__ __align__(16) float2 tq[kP2PWarps][16];
    __shared__ __align__(16) int4 seg[kP2PWarps][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t w = (uint32_t)blockIdx.x * kP2PWarps + warp;
    const uint2 lt = bmap[w];
    if (w >= bstart[nleaf]) return;
    if (*(volatile const unsigned int*)status != 0u) return;
    const uint32_t leaf = lt.x;
    const uint32_t t0 = leaf_start[leaf], t1 = leaf_start[leaf + 1];
    const uint32_t b0 = t0 + (uint32_t)FMM_P2P_BLOCK * lt.y;
    const int T = (int)min((uint32_t)FMM_P2P_BLOCK, t1 - b0);
    uint32_t pairs;
    const NearField nf = p2p_near_sym_field(sp, lo, leaf_start, leaf, t0, t1, b0, T, levels, s_leaf, tgt[warp],
                                            tlo[warp], tq[warp], seg[warp], lane, acc, accg, &pairs);
    if (lane == 0) {
        const unsigned slot = leaf % FMM_COUNTER_SLOTS;
        atomicAdd(&counters[slot], (unsigned long long)pairs);
        atomicMax(&counters[FMM_COUNTER_SLOTS + slot], (unsigned long long)(t1 - t0));
    }
    if (lane < T) {
        atomicAdd(acc + b0 + lane, fmm_f2d_bits(nf.phi.x) + fmm_f2d_bits(nf.phi.y));
        atomicAdd(&accg[b0 + lane].x, fmm_f2d_bits(nf.gx.x) + fmm_f2d_bits(nf.gx.y));
        atomicAdd(&accg[b0 + lane].y, fmm_f2d_bits(nf.gy.x) + fmm_f2d_bits(nf.gy.y));
    }
}

}  // namespace

// The near field on the plan's second stream: forked from the plan's stream at this point of its
// work (record_fork) or at the fork event recorded earlier (any point after the sort will do),
// joined back before L2P.
int fmm_launch_p2p_concurrent(fmm_plan_s* pl, const MixedLevels& lv, bool with_field, bool record_fork) {
    cudaStream_t st = pl->stream, s2 = pl->serial ? pl->stream : pl->stream2;
    // the near-field accumulator starts at zero: cleared on stream2 as soon as the call starts (the
    // start event follows the previous call's L2P, its last reader), beside the sort and fine P2M
    if (s2 != st && cudaStreamWaitEvent(s2, pl->ev[0], 0) != cudaSuccess) return -1;
    if (cudaMemsetAsync(pl->phi_far, 0, sizeof(double) * (size_t)pl->n, s2) != cudaSuccess) return -1;
    if (with_field && cudaMemsetAsync(pl->near_grad, 0, sizeof(double2) * (size_t)pl->n, s2) != cudaSuccess) return -1;
    if ((record_fork && cudaEventRecord(pl->ev_fork, st) != cudaSuccess) ||
        cudaStreamWaitEvent(s2, pl->ev_fork, 0) != cudaSuccess)
        return -1;
    const int L = pl->levels;
    const int64_t n = pl->n;
    const uint32_t nleaf = 1u << (2 * L);
    // the near-field blocks (leaf_bstart, blk_map) came with the sort's scan; upper bound of the
    // blocks: each square adds at most one partial block
    const uint64_t wmax = (uint64_t)nleaf + (uint64_t)(n / FMM_P2P_BLOCK) + 1;
    const unsigned blocks = (unsigned)((wmax + kP2PWarps - 1) / kP2PWarps);
    cudaEventRecord(pl->ev[8], s2);
    if (with_field)
        k_p2p_field<<<blocks, kP2PWarps * 32, 0, s2>>>(pl->sorted32, pl->leaf_start, pl->leaf_bstart, pl->blk_map,
                                                      nleaf, L, lv.s_leaf, pl->sorted_lo, pl->phi_far, pl->near_grad,
                                                      pl->d_status, pl->d_counters);
    else
        k_p2p_mixed<<<blocks, kP2PWarps * 32, 0, s2>>>(pl->sorted32, pl->leaf_start, pl->leaf_bstart, pl->blk_map,
                                                      nleaf, L, lv.s_leaf, pl->phi_far, pl->d_status, pl->d_counters);
    cudaEventRecord(pl->ev[9], s2);
    pl->ev_kernels |= 2;
    if (cudaEventRecord(pl->ev_join, s2) != cudaSuccess) return -1;
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

namespace {

template <int P1B>
void launch_m2l(const M2LMixedArgs& a, const MixedLevels& lv, int blocks, cudaStream_t st) {
    k_m2l_f32<P1B><<<blocks, kM2LThreads, 0, st>>>(a, lv);
}

template <int P1B>
void launch_m2l_coarse(const M2LWarpArgs& a, const MixedLevels& lv, int blocks, cudaStream_t st) {
    k_m2l_coarse<P1B><<<blocks, 128, 0, st>>>(a, lv);
}

}  // namespace

// L2P of levels k_lo..k_hi on stream s (k_l2p_mixed); -1 if the coefficient bucket is unknown
static int launch_l2p(fmm_plan_s* pl, const MixedLevels& lv, int k_lo, int k_hi, const float2* far_in, float2* far_out,
               double* phi, cudaStream_t s) {
    const int64_t n = pl->n;
    const unsigned blocks = (unsigned)((n + 127) / 128);
    const int p = pl->p, p1 = p + 1;
    switch (pl->p1b) {
#define FMM_L2P(PB)                                                                                          \
    case PB:                                                                                                 \
        if (p1 == PB)                                                                                        \
            k_l2p_mixed<PB, true><<<blocks, 128, 0, s>>>(pl->sorted32, pl->sorted_key, n, pl->levels, k_lo, k_hi, \
                                                         p, lv, pl->grids, far_in, far_out, pl->phi_far,     \
                                                         pl->d_status, phi);                                 \
        else                                                                                                 \
            k_l2p_mixed<PB, false><<<blocks, 128, 0, s>>>(pl->sorted32, pl->sorted_key, n, pl->levels, k_lo, k_hi, \
                                                          p, lv, pl->grids, far_in, far_out, pl->phi_far,    \
                                                          pl->d_status, phi);                                \
        return 0;
        FMM_L2P(9) FMM_L2P(13) FMM_L2P(17) FMM_L2P(21) FMM_L2P(25) FMM_L2P(33) FMM_L2P(41)
#undef FMM_L2P
        default: return -1;
    }
}

int fmm_m2l_bucket(int p1) {
    const int b[] = {9, 13, 17, 21, 25, 33, 41};
    for (int v : b)
        if (p1 <= v) return v;
    return -1;
}

int fmm_launch_mixed(fmm_plan_s* pl, double* phi, double* field) {
    if (pl->precision != FMM_MIXED_FP32 && pl->precision != FMM_MIXED_TF32 && pl->precision != FMM_MIXED_3XTF32 &&
        pl->precision != FMM_MIXED_BF16 && pl->precision != FMM_MIXED_BF16X3 && pl->precision != FMM_MIXED_BF16X2)
        return -2;
    // in the tensor-core modes the tensor-core M2L takes the levels from fmm_tc_kmin() on
    const bool use_tc = pl->tc != nullptr && pl->levels >= fmm_tc_kmin();
    cudaStream_t st = pl->stream, s3 = pl->serial ? pl->stream : pl->stream3;
    const int64_t n = pl->n;
    const int L = pl->levels, p = pl->p, p1 = p + 1;
    const MixedLevels lv = fmm_make_levels(pl);
    int launches = 0;
    const double* near = pl->phi_far;   // near-field accumulator per sorted particle
    cudaEventRecord(pl->ev[1], st);
    // fine levels: the finest kFineLevels from the particles; coarser ones by the upward pass
    const int kf = L - (kFineLevels - 1) > 2 ? L - (kFineLevels - 1) : 2;
    const int kc_max = kf - 1;
    const int kw = L < kM2LWarpMaxLevel ? L : kM2LWarpMaxLevel;   // levels 2..kw: the coarse M2L kernel
    // The near field needs only the sort: it forks right after it.  The coarse levels' chain (upward
    // pass, M2L and L2P of levels 2..kw) needs the fine P2M's moments: it forks after it.  The fine
    // P2M is launched before the near field, so that its blocks (the head of the longest chain: fine
    // P2M, tensor-core prep, tensor-core M2L) reach the SMs first.
    // Potential calls with levels above kw evaluate the coarse levels' locals on the third stream as
    // soon as their M2L is done; the final L2P adds the fine levels, the near field and writes phi.
    const bool split_l2p = field == nullptr && L > kw && kw >= 2;
    if (cudaEventRecord(pl->ev_fork, st) != cudaSuccess) return -1;
    if (L >= 2) {
        // crowded squares (a previous call's scan found a finest square above kLaneMax particles):
        // their fine-level coefficients come from k_p2m_crowded, spread over the grid; the hint is
        // only a guess about this call's input, and either way the result is the same
        const bool ext = pl->crowd_hint_h != nullptr && *(volatile int*)pl->crowd_hint_h != 0;
        if (pl->crowd_hint_h) *(volatile int*)pl->crowd_hint_h = 0;
        const unsigned fblocks = (unsigned)(((2ull << (2 * L)) + 127) / 128);   // two lanes per finest square
        const unsigned cwblocks = (unsigned)((n + 4 * kCoarseChunk - 1) / (4 * kCoarseChunk));
        switch (pl->p1b) {
#define FMM_P2M(PB)                                                                                          \
    case PB:                                                                                                 \
        k_p2m_fine<PB><<<fblocks, 128, 0, st>>>(pl->sorted32, pl->leaf_start, L, p, lv, pl->grids, ext ? 1 : 0);   \
        if (ext)                                                                                             \
            k_p2m_crowded<PB><<<cwblocks, 128, 0, st>>>(pl->sorted32, pl->sorted_key, pl->leaf_start, n, L, p, lv, \
                                                        pl->grids);                                          \
        break;
            FMM_P2M(9) FMM_P2M(13) FMM_P2M(17) FMM_P2M(21) FMM_P2M(25) FMM_P2M(33) FMM_P2M(41)
#undef FMM_P2M
            default: return -2;
        }
        launches += ext ? 2 : 1;
    }
    cudaEventRecord(pl->ev[2], st);
    // the near field on stream2, from the sort's fork event; all three streams join before the
    // final L2P (with fmm_set_concurrency(plan, 1) everything runs in turn on the plan's stream)
    {
        const int r = fmm_launch_p2p_concurrent(pl, lv, field != nullptr, false);
        if (r < 0) return -1;
        launches += r;
    }
    if (L >= 2) {
        if (s3 != st && cudaStreamWaitEvent(s3, pl->ev[2], 0) != cudaSuccess) return -1;   // the fine P2M is done
        cudaEventRecord(pl->ev[10], s3);
        // upward pass, levels kc_max .. 2, each from the level below it
        for (int k = kc_max; k >= 2; --k) {
            const unsigned mblocks = (unsigned)(((1u << (2 * k)) + 1u) / 2u);
            const float2* ch = reinterpret_cast<const float2*>(pl->grids.A32[k + 1]);
            float2* par = reinterpret_cast<float2*>(pl->grids.A32[k]);
            switch (pl->p1b) {
#define FMM_M2M(PB)                                                                                          \
    case PB:                                                                                                 \
        k_m2m_f32<PB><<<mblocks, 2 * kM2MThreads, 0, s3>>>(ch, par, pl->U32, k, p1);                         \
        break;
                FMM_M2M(9) FMM_M2M(13) FMM_M2M(17) FMM_M2M(21) FMM_M2M(25) FMM_M2M(33) FMM_M2M(41)
#undef FMM_M2M
                default: return -2;
            }
            ++launches;
        }
        // from level 9 on the upward pass forms moments of levels 6 .. l-3, which the fine levels'
        // M2L on the plan's stream reads
        if (kc_max > kw && cudaEventRecord(pl->ev_a32, s3) != cudaSuccess) return -1;
        cudaEventRecord(pl->ev[11], s3);
        cudaEventRecord(pl->ev[12], s3);
        // coarse levels: a CTA per 4 x kM2LWarpTargets targets of one class
        M2LWarpArgs wa;
        wa.g = pl->grids;
        wa.T = pl->T32;
        wa.p = p;
        wa.kw = kw;
        int wacc = 0;
        for (int k = 0; k <= FMM_MAX_LEVELS + 1; ++k) wa.cbase[k] = 0;
        for (int k = 2; k <= wa.kw; ++k) {
            wa.cbase[k] = wacc;
            wacc += 4 * (((1 << (2 * (k - 1))) + 4 * kM2LWarpTargets - 1) / (4 * kM2LWarpTargets));
        }
        wa.cbase[wa.kw + 1] = wacc;
        switch (pl->p1b) {
            case 9: launch_m2l_coarse<9>(wa, lv, wacc, s3); break;
            case 13: launch_m2l_coarse<13>(wa, lv, wacc, s3); break;
            case 17: launch_m2l_coarse<17>(wa, lv, wacc, s3); break;
            case 21: launch_m2l_coarse<21>(wa, lv, wacc, s3); break;
            case 25: launch_m2l_coarse<25>(wa, lv, wacc, s3); break;
            case 33: launch_m2l_coarse<33>(wa, lv, wacc, s3); break;
            case 41: launch_m2l_coarse<41>(wa, lv, wacc, s3); break;
            default: return -2;
        }
        ++launches;
        cudaEventRecord(pl->ev[13], s3);
        pl->ev_kernels |= 4 | 8;
        if (split_l2p) {
            // the coarse levels' L2P, beside the near field and the fine levels' M2L
            cudaEventRecord(pl->ev[15], s3);
            if (launch_l2p(pl, lv, 2, kw, nullptr, pl->far_part, nullptr, s3) < 0) return -2;
            cudaEventRecord(pl->ev[16], s3);
            pl->ev_kernels |= 16;
            ++launches;
        }
        if (cudaEventRecord(pl->ev_join3, s3) != cudaSuccess) return -1;

        // finer levels on the plan's stream: one thread per target, or the tensor cores.  Their
        // moments of levels kw+1 .. kc_max (l >= 9) come from the third stream's coarse P2M.
        if (kc_max > kw && s3 != st && cudaStreamWaitEvent(st, pl->ev_a32, 0) != cudaSuccess) return -1;
        cudaEventRecord(pl->ev[14], st);
        M2LMixedArgs a;
        a.g = pl->grids;
        a.T = pl->T32;
        a.levels = L;
        a.p = p;
        a.kmin = kw + 1;
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
    if (L < 2) cudaEventRecord(pl->ev[14], st);
    cudaEventRecord(pl->ev[3], st);
    if (cudaStreamWaitEvent(st, pl->ev_join, 0) != cudaSuccess) return -1;   // the near field is done
    if (L >= 2 && cudaStreamWaitEvent(st, pl->ev_join3, 0) != cudaSuccess) return -1;   // and the coarse levels
    cudaEventRecord(pl->ev[4], st);
    if (field != nullptr) {
        const unsigned blocks = (unsigned)((n + 127) / 128);
        switch (pl->p1b) {
#define FMM_L2PF(PB)                                                                                         \
    case PB:                                                                                                 \
        k_l2p_field<PB><<<blocks, 128, 0, st>>>(pl->sorted32, pl->sorted_key, n, L, p, lv, pl->grids, near,      \
                                                pl->near_grad, pl->d_status, phi, field);                    \
        break;
            FMM_L2PF(9) FMM_L2PF(13) FMM_L2PF(17) FMM_L2PF(21) FMM_L2PF(25) FMM_L2PF(33) FMM_L2PF(41)
#undef FMM_L2PF
            default: return -2;
        }
        ++launches;
    } else {
        if (split_l2p ? launch_l2p(pl, lv, kw + 1, L, pl->far_part, nullptr, phi, st) < 0
                      : launch_l2p(pl, lv, 2, L, nullptr, nullptr, phi, st) < 0)
            return -2;
        ++launches;
    }
    cudaEventRecord(pl->ev[5], st);
    if (cudaGetLastError() != cudaSuccess) return -1;
    return launches;
}
