// batch.cu -- many independent systems of uneven size in one launch per stage (the batched form
// of the mixed-precision path), replayed as one CUDA graph.
//
// Every system is an independent instance of the method (its own box [0, box]^2, its own
// quadtree depth); the particles of all systems are concatenated in system order.  The stages
// are the single-system ones (sort, P2M per level, M2L, L2P per level, P2P), each run as one
// grid-stride (persistent) kernel over a flattened work space that spans all systems.  A work
// item finds its system by binary search over per-system prefix counts held in shared memory.
// One exclusive scan over the concatenated finest-square populations gives every system's CSR
// offsets already shifted by the system's first particle.  The coarse levels' moments come from the
// upward pass over every system's squares of one level per launch.  M2L runs levels 2..5 on the CUDA cores
// in FP32 and, in the tensor-core precisions, every system's levels 6 and finer in one tcgen05
// launch whose tiles come from any system (one segment per system and level).  The near field is
// the symmetric one of the single-system path, on a second branch of the graph beside P2M and M2L;
// L2P then adds each particle's near field and writes phi.  The sequence of launches is captured
// once into a CUDA graph; the call's array pointers live in a small device block written before
// each replay, so one graph serves every call.  fmm_batch_autotune times candidate launch shapes
// (persistent blocks per SM, tensor-core tiles per CTA, near-field targets per block).
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mixed_common.cuh"
#include "p2p_block.cuh"

namespace {

constexpr int kT = 128;   // threads per block of every batched kernel
constexpr int kLaneMax = 128;
constexpr int kFineMean = 64;
constexpr int kP2PBlockMin = 16;   // the smallest near-field block the autotuner tries

struct BatchSys {
    long long p_off;                       // first particle of the system (input and sorted order)
    long long leaf_off;                    // first finest square in the concatenated CSR
    long long a_off[FMM_MAX_LEVELS + 1];   // first cell of level k's moment grid (3-cell halo layout)
    long long b_off[FMM_MAX_LEVELS + 1];   // first cell of level k's local-coefficient grid
    int n, levels, kf;                     // particles, depth, first fine P2M level
};

struct BatchCall {
    const double* xy;
    const double* q;
    double* phi;
};

struct BatchArgs {
    const BatchSys* sys;
    const BatchCall* call;
    // per-system prefix counts (nsys + 1 entries each) of the flattened work spaces
    const long long* wp_part;     // particles
    const long long* wp_leaf;     // finest squares
    const long long* wp_fine;     // fine-level P2M squares
    const long long* wp_m2l;      // M2L blocks
    const long long* wp_m2m;      // upward-pass parents of level 2; level k's prefix is (k - 2) (nsys + 1) further
    int nsys, p;
    double box;
    float2 box_ff;
    uint32_t* keys;
    uint32_t* rank;
    uint32_t* counts;
    uint32_t* leaf_start;
    const uint32_t* bstart;   // near-field target blocks: exclusive scan over the concatenated squares
    const uint2* bmap;        // near-field block -> (concatenated square, block inside it)
    long long nl;             // concatenated finest squares
    uint32_t* sorted_key;
    float4* sorted32;
    float2* a32;     // all moment grids (FP32; coarse region first)
    float2* b32;     // local coefficients
    const float2* T; // FP32 operators [49][P1B][P1B]
    const float2* U; // upward-pass translations [child position][j][m], P1B each (the single-system plan's)
    double* acc;     // near field per sorted particle (log2 r^2 units), zeroed at the start of a call
    unsigned int* status;
    int m2l_kmax;    // levels 2..m2l_kmax of each system run in kb_m2l_f32 (the tensor cores take the rest)
    int p2p_block;   // near-field targets per block (16 or 24)
};

// largest s with pre[s] <= w, for pre[0] = 0 <= w < pre[nsys]
__device__ __forceinline__ int find_sys(const long long* pre, int nsys, long long w) {
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= w) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void load_prefix(long long* dst, const long long* src, int nsys) {
    for (int i = threadIdx.x; i <= nsys; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
}

// -------------------------------------------------------------------------------- sort
__global__ void __launch_bounds__(kT) kb_bin(BatchArgs a, MixedLevels lv) {
    extern __shared__ long long pre[];
    load_prefix(pre, a.wp_part, a.nsys);
    const long long total = pre[a.nsys];
    const double2* xy = reinterpret_cast<const double2*>(a.call->xy);
    const double* q = a.call->q;
    const long long bb = __double_as_longlong(a.box);
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < total; i += (long long)gridDim.x * kT) {
        const BatchSys& S = a.sys[find_sys(pre, a.nsys, i)];
        const double2 p = xy[i];
        const double qq = q[i];
        const int side = 1 << S.levels;
        uint32_t key = 0;
        if (!(finite_bits(p.x) && finite_bits(p.y) && finite_bits(qq))) {
            atomicOr(a.status, FMM_FLAG_NONFINITE);
        } else {
            if (!(in_box_bits(p.x, bb) && in_box_bits(p.y, bb))) atomicOr(a.status, FMM_FLAG_OUT_OF_BOX);
            const double scale = (double)side;
            const float sob = lv.inv_s[S.levels];
            key = fmm_morton((uint32_t)finest_coord(p.x, scale, sob, a.box, side),
                             (uint32_t)finest_coord(p.y, scale, sob, a.box, side));
        }
        a.keys[i] = key;
        a.rank[i] = atomicAdd(&a.counts[S.leaf_off + key], 1u);
    }
}

__global__ void __launch_bounds__(kT) kb_scatter(BatchArgs a) {
    extern __shared__ long long pre[];
    load_prefix(pre, a.wp_part, a.nsys);
    const long long total = pre[a.nsys];
    const double2* xy = reinterpret_cast<const double2*>(a.call->xy);
    const double* q = a.call->q;
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < total; i += (long long)gridDim.x * kT) {
        const BatchSys& S = a.sys[find_sys(pre, a.nsys, i)];
        const uint32_t key = a.keys[i];
        const uint32_t pos = a.leaf_start[S.leaf_off + key] + a.rank[i];
        const double2 p = xy[i];
        // the square side box / 2^l as an FP32 pair: exact power-of-two scaling of box
        const float sc = __int_as_float((127 - S.levels) << 23);
        const float2 s_ff = make_float2(a.box_ff.x * sc, a.box_ff.y * sc);
        const float2 cx = scatter_mul((float)fmm_compact2(key) + 0.5f, s_ff);
        const float2 cy = scatter_mul((float)fmm_compact2(key >> 1) + 0.5f, s_ff);
        const float2 xf = fmm_d2ff_bits(p.x), yf = fmm_d2ff_bits(p.y), qf = fmm_d2ff_bits(q[i]);
        a.sorted_key[pos] = key;
        a.sorted32[pos] = make_float4((xf.x - cx.x) + (xf.y - cx.y), (yf.x - cy.x) + (yf.y - cy.y), qf.x + qf.y,
                                      __int_as_float((int)(i - S.p_off)));
    }
}

// -------------------------------------------------------------------------------- P2M
template <int P1B>
__device__ __forceinline__ void add_powers_b(float2 (&acc)[P1B], float q, float2 w) {
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

// fine levels: one lane per square (see mixed.cu); 32 consecutive work items per warp step
template <int P1B>
__global__ void __launch_bounds__(kT) kb_p2m_fine(BatchArgs a, MixedLevels lv) {
    extern __shared__ long long pre[];
    __shared__ float red[kT / 32][32][2 * P1B + 1];
    load_prefix(pre, a.wp_fine, a.nsys);
    const long long total = pre[a.nsys];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p1 = a.p + 1;
    const long long stride = (long long)gridDim.x * kT;
    for (long long wbase = (long long)blockIdx.x * kT + warp * 32; wbase < total; wbase += stride) {
        const long long gt = wbase + lane;
        const bool valid = gt < total;
        int s = valid ? find_sys(pre, a.nsys, gt) : 0;
        const BatchSys& S = a.sys[s];
        long long local = valid ? gt - pre[s] : 0;
        int k = S.kf;
        while (k < S.levels && local >= (1ll << (2 * k))) {
            local -= 1ll << (2 * k);
            ++k;
        }
        const uint32_t b = (uint32_t)local;
        const int sh = S.levels - k;
        const uint32_t lo = valid ? a.leaf_start[S.leaf_off + ((long long)b << (2 * sh))] : 0u;
        const uint32_t hi = valid ? a.leaf_start[S.leaf_off + ((long long)(b + 1) << (2 * sh))] : 0u;
        const long long cell =
            S.a_off[k] + (long long)(fmm_compact2(b >> 1) + FMM_HALO) * fmm_grid_width(k) + fmm_compact2(b) + FMM_HALO;
        const bool large = hi - lo > (uint32_t)kLaneMax;
        float2 acc[P1B];
#pragma unroll
        for (int m = 0; m < P1B; ++m) acc[m] = make_float2(0.f, 0.f);
        float2 m0 = make_float2(0.f, 0.f);
        if (valid && !large) {
            for (uint32_t j = lo; j < hi; ++j) {
                const float4 P = a.sorted32[j];
                const uint32_t key = a.sorted_key[j];
                const float2 w = level_w(P.x, P.y, fmm_compact2(key), fmm_compact2(key >> 1), sh, lv.inv_s[k]);
                m0 = ff_add_f(m0, P.z);
                add_powers_b<P1B>(acc, P.z, w);
            }
            float2* A = a.a32 + cell * p1;
            A[0] = m0;
#pragma unroll
            for (int m = 1; m < P1B; ++m)
                if (m < p1) A[m] = acc[m];
        }
        unsigned todo = __ballot_sync(0xffffffffu, valid && large);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const uint32_t lo2 = __shfl_sync(0xffffffffu, lo, src), hi2 = __shfl_sync(0xffffffffu, hi, src);
            const int k2 = __shfl_sync(0xffffffffu, k, src);
            const int sh2 = __shfl_sync(0xffffffffu, sh, src);
            const long long cell2 = __shfl_sync(0xffffffffu, cell, src);
#pragma unroll
            for (int m = 0; m < P1B; ++m) acc[m] = make_float2(0.f, 0.f);
            m0 = make_float2(0.f, 0.f);
            for (uint32_t j = lo2 + lane; j < hi2; j += 32) {
                const float4 P = a.sorted32[j];
                const uint32_t key = a.sorted_key[j];
                const float2 w = level_w(P.x, P.y, fmm_compact2(key), fmm_compact2(key >> 1), sh2, lv.inv_s[k2]);
                m0 = ff_add_f(m0, P.z);
                add_powers_b<P1B>(acc, P.z, w);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                m0 = ff_add(m0,
                            make_float2(__shfl_xor_sync(0xffffffffu, m0.x, o), __shfl_xor_sync(0xffffffffu, m0.y, o)));
            float* row = red[warp][lane];
#pragma unroll
            for (int m = 1; m < P1B; ++m) {
                row[2 * m] = acc[m].x;
                row[2 * m + 1] = acc[m].y;
            }
            __syncwarp();
            float2* A = a.a32 + cell2 * p1;
            for (int col = 2 + lane; col < 2 * p1; col += 32) {
                float sum = 0.f;
#pragma unroll
                for (int r = 0; r < 32; ++r) sum += red[warp][r][col];
                reinterpret_cast<float*>(A)[col] = sum;
            }
            if (lane == 0) A[0] = m0;
            __syncwarp();
        }
    }
}

// Upward pass for the coarse levels (U-bar-2, as in mixed.cu's k_m2m_f32): level k of every
// system whose coarse levels include k, one parent per half-CTA of 64 threads (a thread per
// coefficient), grid-stride over pairs of parents.  Each parent sums its four children's moments
// re-expanded about its centre with the tables U; its total charge is a float-float sum.
constexpr int kM2MHalf = 64;

template <int P1B>
__global__ void __launch_bounds__(2 * kM2MHalf) kb_m2m(BatchArgs a, int k) {
    static_assert(P1B <= kM2MHalf, "one thread per coefficient");
    // the four tables staged at once where they take at most 24 KB (the prefix array shares the
    // 48 KB of shared memory), else one child's at a time
    constexpr int UC = 4 * P1B * P1B * (int)sizeof(float2) <= 24 * 1024 ? 4 : 1;
    extern __shared__ long long pre[];
    __shared__ float2 mom[2][4][P1B];
    __shared__ float2 us[UC * P1B * P1B];
    load_prefix(pre, a.wp_m2m + (long long)(k - 2) * (a.nsys + 1), a.nsys);
    const long long total = pre[a.nsys];
    const int half = threadIdx.x / kM2MHalf, m = threadIdx.x % kM2MHalf;
    const int p1 = a.p + 1;
    auto stage = [&](int c0) {
        constexpr int NU = UC * P1B * P1B, R = (NU + 2 * kM2MHalf - 1) / (2 * kM2MHalf);
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = threadIdx.x + r * 2 * kM2MHalf;
            v[r] = i < NU ? __ldg(a.U + (size_t)c0 * P1B * P1B + i) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = threadIdx.x + r * 2 * kM2MHalf;
            if (i < NU) us[i] = v[r];
        }
    };
    if (UC == 4) stage(0);   // once for all the CTA's parents (load_prefix's barrier came before)
    for (long long wp = blockIdx.x; 2 * wp < total; wp += gridDim.x) {
        const long long w = 2 * wp + half;
        const bool live = w < total;
        int s = 0;
        uint32_t px = 0, py = 0;
        if (live) {
            s = find_sys(pre, a.nsys, w);
            const uint32_t par = (uint32_t)(w - pre[s]), side = 1u << k;
            px = par % side;
            py = par / side;
        }
        const BatchSys& S = a.sys[s];
        if (m < P1B) {
            const int Wc = fmm_grid_width(k + 1);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float2 v = make_float2(0.f, 0.f);
                if (live && m < p1) {
                    const long long cell =
                        S.a_off[k + 1] + (long long)(2 * py + (c >> 1) + FMM_HALO) * Wc + 2 * px + (c & 1) + FMM_HALO;
                    v = a.a32[cell * p1 + m];
                }
                mom[half][c][m] = v;
            }
        }
        const bool work = live && m >= 1 && m < p1;
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int c0 = 0; c0 < 4; c0 += UC) {
            if (UC == 1) stage(c0);
            __syncthreads();
            if (work) {
#pragma unroll
                for (int cc = 0; cc < UC; ++cc) {
                    const float2* u = us + cc * P1B * P1B + m;   // U_c[m][j] at u[j P1B]
                    const float2 m0 = mom[half][c0 + cc][0];
                    const float q0 = m0.x + m0.y;
                    float r = u[0].x * q0, t = u[0].y * q0;
#pragma unroll
                    for (int j = 1; j < P1B; ++j) {
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
        if (live && m < p1) {
            float2 out;
            if (m == 0) {
                out = mom[half][0][0];
#pragma unroll
                for (int c = 1; c < 4; ++c) out = ff_add(out, mom[half][c][0]);
            } else {
                out = make_float2(re, im);
            }
            const int Wp = fmm_grid_width(k);
            const long long pcell = S.a_off[k] + (long long)(py + FMM_HALO) * Wp + px + FMM_HALO;
            a.a32[pcell * p1 + m] = out;
        }
    }
}

// -------------------------------------------------------------------------------- M2L (FP32)
template <int P1B>
__global__ void __launch_bounds__(kT) kb_m2l_f32(BatchArgs a, MixedLevels lv) {
    extern __shared__ long long pre[];
    __shared__ float2 Ts[P1B * P1B];
    load_prefix(pre, a.wp_m2l, a.nsys);
    const long long total = pre[a.nsys];
    const int p1 = a.p + 1;
    for (long long cta = blockIdx.x; cta < total; cta += gridDim.x) {
        const int s = find_sys(pre, a.nsys, cta);
        const BatchSys& S = a.sys[s];
        long long rel = cta - pre[s];
        int k = 2;
        const int kmax = S.levels < a.m2l_kmax ? S.levels : a.m2l_kmax;
        for (; k < kmax; ++k) {
            const long long w2 = 1ll << (k - 1);
            const long long cnt = 4 * ((w2 * w2 + kT - 1) / kT);
            if (rel < cnt) break;
            rel -= cnt;
        }
        const int w2 = 1 << (k - 1);
        const int per_class = (w2 * w2 + kT - 1) / kT;
        const int cls = (int)(rel / per_class);
        const int u = (int)(rel - (long long)cls * per_class) * kT + threadIdx.x;
        const bool active = u < w2 * w2;
        const int px = cls & 1, py = cls >> 1;
        const int tx = 2 * (active ? u % w2 : 0) + px;
        const int ty = 2 * (active ? u / w2 : 0) + py;
        const int W = fmm_grid_width(k);
        const float2* A = a.a32 + S.a_off[k] * p1;
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
                for (int e = threadIdx.x; e < P1B * P1B; e += kT) Ts[e] = Td[e];
                __syncthreads();
                const float2* src = A + ((size_t)(ty + dy + FMM_HALO) * W + (tx + dx + FMM_HALO)) * p1;
                float2 m[P1B];
#pragma unroll
                for (int kk = 0; kk < P1B; ++kk) m[kk] = (kk < p1) ? src[kk] : make_float2(0.f, 0.f);
                mono = ff_add(mono, ff_mul(m[0], lv.logc[k][d]));
                m[0].y = 0.f;
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
        if (active) {
            float2* B = a.b32 + (S.b_off[k] + (long long)ty * (1ll << k) + tx) * p1;
            B[0] = ff_add_f(mono, acc[0].x);
#pragma unroll
            for (int l = 1; l < P1B; ++l)
                if (l < p1) B[l] = acc[l];
        }
    }
}

// -------------------------------------------------------------------------------- L2P + final phi
// One thread per particle: the levels' local expansions summed in float-float, the particle's near
// field (kb_p2p, already complete) added, phi written in input order unless the checks failed.
template <int P1B>
__global__ void __launch_bounds__(kT) kb_l2p(BatchArgs a, MixedLevels lv) {
    extern __shared__ long long pre[];
    load_prefix(pre, a.wp_part, a.nsys);
    const long long total = pre[a.nsys];
    const int p1 = a.p + 1;
    const bool bad = *(volatile const unsigned int*)a.status != 0u;
    double* phi = a.call->phi;
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < total && !bad; i += (long long)gridDim.x * kT) {
        const BatchSys& S = a.sys[find_sys(pre, a.nsys, i)];
        const double nd = a.acc[i];
        const float4 P = a.sorted32[i];
        const uint32_t key = a.sorted_key[i];
        const uint32_t ix = fmm_compact2(key), iy = fmm_compact2(key >> 1);
        float2 far = make_float2(0.f, 0.f);
        for (int k = 2; k <= S.levels; ++k) {
            const int sh = S.levels - k;
            const float2 w = level_w(P.x, P.y, ix, iy, sh, lv.inv_s[k]);
            const float2* Bt = a.b32 + (S.b_off[k] + (long long)(iy >> sh) * (1ll << k) + (ix >> sh)) * p1;
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
            far = ff_add(far, ff_add_f(b[0], fmaf(u.x, w.x, -u.y * w.y)));
        }
        phi[S.p_off + __float_as_int(P.w)] = p2p_phi(far, fmm_d2ff_bits(nd));
    }
}

// One warp per near-field block of any system (blocks of up to p2p_block targets, the block map
// giving the square), grid-stride; the block's near field is p2p_near_sym (p2p_block.cuh), as in
// the single-system path: the own square in full, the four forward neighbours once for both sides,
// every result added in FP64 to the per-particle accumulator.
__global__ void __launch_bounds__(kT, 8) kb_p2p(BatchArgs a, MixedLevels lv) {
    extern __shared__ long long pre[];
    __shared__ __align__(16) float4 tgt[kT / 32][16];
    __shared__ __align__(16) float2 tq[kT / 32][16];
    __shared__ __align__(16) int4 seg[kT / 32][4];
    load_prefix(pre, a.wp_leaf, a.nsys);
    const long long total = a.bstart[a.nl];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool bad = *(volatile const unsigned int*)a.status != 0u;
    for (long long w = (long long)blockIdx.x * (kT / 32) + warp; w < total && !bad;
         w += (long long)gridDim.x * (kT / 32)) {
        const uint2 lt = a.bmap[w];
        const int s = find_sys(pre, a.nsys, (long long)lt.x);
        const BatchSys& S = a.sys[s];
        const uint32_t leaf = (uint32_t)((long long)lt.x - pre[s]);
        const uint32_t* ls = a.leaf_start + S.leaf_off;
        const uint32_t t0 = ls[leaf], t1 = ls[leaf + 1];
        const uint32_t b0 = t0 + (uint32_t)a.p2p_block * lt.y;
        const int T = (int)min((uint32_t)a.p2p_block, t1 - b0);
        const float s_leaf = a.box_ff.x * __int_as_float((127 - S.levels) << 23);
        uint32_t pairs;
        const float2 near = p2p_near_sym(a.sorted32, ls, leaf, t0, t1, b0, T, S.levels, s_leaf, tgt[warp], tq[warp],
                                         seg[warp], lane, a.acc, &pairs);
        if (lane < T) atomicAdd(a.acc + b0 + lane, fmm_f2d_bits(near.x) + fmm_f2d_bits(near.y));
        __syncwarp();   // tgt, tq and seg are rewritten by the next block
    }
}

}  // namespace

// ---------------------------------------------------------------- the batch plan
struct fmm_batch_s {
    int device, nsys, p, p1b;
    double box;
    long long nt, nl, coarse_cells, a_cells, b_cells;   // coarse_cells: the coarse levels' grid cells
    cudaStream_t stream;
    int precision;
    int grid_mult;                    // persistent blocks per SM (autotuned)
    int tc_rows;                      // tensor-core tiles per CTA, 0 = the kernel's default (autotuned)
    int p2p_block;                    // near-field targets per block, 16 or 24 (autotuned)
    double tuned_ms;                  // the autotuner's best time (0 before a search)
    FmmTc* tc;                        // tensor-core M2L of levels 6 and finer (tensor-core precisions)
    std::vector<BatchSys> host_sys;
    BatchSys* d_sys;
    long long* d_pre;                 // prefix arrays, (nsys + 1) each: particles, squares, fine P2M
                                      // squares, M2L blocks, then upward-pass parents of levels 2..max
    BatchCall* d_call;
    BatchCall* h_call;                // pinned
    uint32_t *keys, *rank, *counts, *leaf_start, *block_sums, *sorted_key, *leaf_nb, *bstart;
    uint2* bmap;
    float4* sorted32;
    float2 *a32, *b32;
    double* acc;                      // near field per sorted particle
    float2* T32;
    float2* U32;                      // upward-pass translations (the single-system plan's layout)
    int m2m_kmax;                     // the highest coarse level of any system (the upward pass runs
                                      // levels m2m_kmax .. 2), 1 when no system has one
    unsigned int* d_status;
    unsigned int* h_status;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    cudaEvent_t ev0, ev1;
    int launches;
    uint64_t workspace_bytes;
};

namespace {

void batch_free(fmm_batch_s* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    void* bufs[] = {b->d_sys, b->d_pre, b->d_call, b->keys, b->rank, b->counts, b->leaf_start, b->block_sums,
                    b->leaf_nb, b->bstart, b->bmap,
                    b->sorted_key, b->sorted32, b->a32, b->b32, b->acc, b->T32, b->U32, b->d_status};
    fmm_tc_free(b->tc);
    for (void* p : bufs)
        if (p) cudaFree(p);
    if (b->h_call) cudaFreeHost(b->h_call);
    if (b->h_status) cudaFreeHost(b->h_status);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    delete b;
}

template <class T>
bool balloc(fmm_batch_s* b, T** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(reinterpret_cast<void**>(p), bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    b->workspace_bytes += bytes;
    return true;
}

// The call's launches: the sort on st, then two branches -- the near field on st2, P2M and M2L on
// st -- joined before L2P.  (st2 == st runs them in turn.)
template <int P1B>
int enqueue_batch_kernels(fmm_batch_s* b, const BatchArgs& a, const MixedLevels& lv, cudaStream_t st,
                          cudaStream_t st2, cudaEvent_t ev_fork, cudaEvent_t ev_join) {
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    const unsigned grid = (unsigned)(sms * b->grid_mult);
    const size_t pre_bytes = sizeof(long long) * (b->nsys + 1);
    int launches = 0;
    if (cudaMemsetAsync(b->counts, 0, sizeof(uint32_t) * b->nl, st) != cudaSuccess ||
        cudaMemsetAsync(b->acc, 0, sizeof(double) * b->nt, st) != cudaSuccess)
        return -1;
    kb_bin<<<grid, kT, pre_bytes, st>>>(a, lv);
    ++launches;
    const int sc = fmm_launch_scan(b->counts, b->nl, b->block_sums, b->leaf_start, (uint32_t)b->nt, st);
    if (sc < 0) return -1;
    launches += sc;
    kb_scatter<<<grid, kT, pre_bytes, st>>>(a);
    ++launches;
    // the near field needs only the sorted particles
    if (st2 != st && (cudaEventRecord(ev_fork, st) != cudaSuccess || cudaStreamWaitEvent(st2, ev_fork, 0) != cudaSuccess))
        return -1;
    const int lb = fmm_launch_leaf_blocks(b->leaf_start, b->nl, (uint32_t)b->p2p_block, b->leaf_nb, b->block_sums,
                                          b->bstart, b->bmap, st2);
    if (lb < 0) return -1;
    kb_p2p<<<grid, kT, pre_bytes, st2>>>(a, lv);
    launches += lb + 1;
    if (st2 != st && cudaEventRecord(ev_join, st2) != cudaSuccess) return -1;
    kb_p2m_fine<P1B><<<grid, kT, pre_bytes, st>>>(a, lv);
    ++launches;
    // upward pass: one launch per coarse level, the finest first
    for (int k = b->m2m_kmax; k >= 2; --k) {
        kb_m2m<P1B><<<grid, 2 * kM2MHalf, pre_bytes, st>>>(a, k);
        ++launches;
    }
    kb_m2l_f32<P1B><<<grid, kT, pre_bytes, st>>>(a, lv);
    ++launches;
    if (b->tc) {
        const int t = fmm_tc_enqueue(b->tc, lv, st, b->d_status, 0, b->tc_rows, nullptr, nullptr);
        if (t < 0) return -1;
        launches += t;
    }
    if (st2 != st && cudaStreamWaitEvent(st, ev_join, 0) != cudaSuccess) return -1;
    kb_l2p<P1B><<<grid, kT, pre_bytes, st>>>(a, lv);
    ++launches;
    return cudaGetLastError() == cudaSuccess ? launches : -1;
}

int enqueue_all(fmm_batch_s* b, cudaStream_t st, cudaStream_t st2, cudaEvent_t ev_fork, cudaEvent_t ev_join) {
    BatchArgs a{};
    const long long stride = b->nsys + 1;
    a.sys = b->d_sys;
    a.call = b->d_call;
    a.wp_part = b->d_pre;
    a.wp_leaf = b->d_pre + stride;
    a.wp_fine = b->d_pre + 2 * stride;
    a.wp_m2l = b->d_pre + 3 * stride;
    a.wp_m2m = b->d_pre + 4 * stride;
    a.nsys = b->nsys;
    a.p = b->p;
    a.box = b->box;
    const float bh = (float)b->box;
    a.box_ff = make_float2(bh, (float)(b->box - (double)bh));
    a.keys = b->keys;
    a.rank = b->rank;
    a.counts = b->counts;
    a.leaf_start = b->leaf_start;
    a.bstart = b->bstart;
    a.bmap = b->bmap;
    a.nl = b->nl;
    a.sorted_key = b->sorted_key;
    a.sorted32 = b->sorted32;
    a.a32 = b->a32;
    a.b32 = b->b32;
    a.T = b->T32;
    a.U = b->U32;
    a.acc = b->acc;
    a.status = b->d_status;
    a.m2l_kmax = b->tc ? fmm_tc_kmin() - 1 : FMM_MAX_LEVELS;
    a.p2p_block = b->p2p_block;
    fmm_plan_s shim{};
    shim.box = b->box;
    shim.levels = 0;
    const MixedLevels lv = fmm_make_levels(&shim);
    switch (b->p1b) {
        case 9: return enqueue_batch_kernels<9>(b, a, lv, st, st2, ev_fork, ev_join);
        case 13: return enqueue_batch_kernels<13>(b, a, lv, st, st2, ev_fork, ev_join);
        case 17: return enqueue_batch_kernels<17>(b, a, lv, st, st2, ev_fork, ev_join);
        case 21: return enqueue_batch_kernels<21>(b, a, lv, st, st2, ev_fork, ev_join);
        case 25: return enqueue_batch_kernels<25>(b, a, lv, st, st2, ev_fork, ev_join);
        case 33: return enqueue_batch_kernels<33>(b, a, lv, st, st2, ev_fork, ev_join);
        case 41: return enqueue_batch_kernels<41>(b, a, lv, st, st2, ev_fork, ev_join);
        default: return -2;
    }
}

// capture the launch sequence into a graph (on a private stream) and instantiate it
fmm_status build_graph(fmm_batch_s* b) {
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    cudaStream_t cap = nullptr, cap2 = nullptr;
    cudaEvent_t evf = nullptr, evj = nullptr;
    auto release = [&]() {
        if (cap) cudaStreamDestroy(cap);
        if (cap2) cudaStreamDestroy(cap2);
        if (evf) cudaEventDestroy(evf);
        if (evj) cudaEventDestroy(evj);
    };
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&cap2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&evf, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&evj, cudaEventDisableTiming) != cudaSuccess) {
        release();
        return FMM_ERR_CUDA;
    }
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        release();
        return FMM_ERR_CUDA;
    }
    const int n = enqueue_all(b, cap, cap2, evf, evj);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cap, &g);
    release();
    if (n < 0 || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return n == -2 ? FMM_ERR_UNSUPPORTED : FMM_ERR_CUDA;
    }
    b->graph = g;
    b->launches = n;
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) return FMM_ERR_CUDA;
    return FMM_OK;
}

fmm_status batch_run(fmm_batch_s* b, const double* xy, const double* q, double* phi) {
    b->h_call->xy = xy;
    b->h_call->q = q;
    b->h_call->phi = phi;
    cudaStream_t st = b->stream;
    if (cudaMemcpyAsync(b->d_call, b->h_call, sizeof(BatchCall), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return FMM_ERR_CUDA;
    cudaEventRecord(b->ev0, st);
    if (cudaGraphLaunch(b->exec, st) != cudaSuccess) return FMM_ERR_CUDA;
    cudaEventRecord(b->ev1, st);
    return FMM_OK;
}

// The autotuner's cache key: the device (name, SM count, driver version), the order, the precision,
// and the batch's shape (system count, total particles to the nearest power of two, systems per
// quadtree depth).  Spaces become underscores so the key is one token.
std::string tune_key(const fmm_batch_s* b) {
    cudaDeviceProp prop;
    memset(&prop, 0, sizeof(prop));
    cudaGetDeviceProperties(&prop, b->device);
    int drv = 0;
    cudaDriverGetVersion(&drv);
    int hist[FMM_MAX_LEVELS + 1] = {};
    for (const BatchSys& S : b->host_sys) ++hist[S.levels];
    int lg = 0;
    while ((1ll << (lg + 1)) <= b->nt) ++lg;
    std::string key = prop.name;
    for (char& c : key)
        if (c == ' ' || c == '|') c = '_';
    char buf[256];
    snprintf(buf, sizeof(buf), "|sm%d|drv%d|p%d|prec%d|nsys%d|N2^%d|depths", prop.multiProcessorCount, drv, b->p,
             b->precision, b->nsys, lg);
    key += buf;
    for (int k = 0; k <= FMM_MAX_LEVELS; ++k)
        if (hist[k]) {
            snprintf(buf, sizeof(buf), ":%dx%d", k, hist[k]);
            key += buf;
        }
    return key;
}

// device time of the current shape: one warm-up replay, then the sum of three
fmm_status time_shape(fmm_batch_s* b, const double* xy, const double* q, double* phi, double* ms_out) {
    fmm_status s = build_graph(b);
    if (s != FMM_OK) return s;
    double tot = 0.0;
    for (int rep = 0; rep < 4; ++rep) {
        double ms = 0.0;
        if ((s = batch_run(b, xy, q, phi)) != FMM_OK) return s;
        if ((s = fmm_batch_sync(b, &ms)) != FMM_OK) return s;
        if (rep > 0) tot += ms;
    }
    *ms_out = tot / 3.0;
    return FMM_OK;
}

}  // namespace

extern "C" {

fmm_status fmm_batch_plan(fmm_batch_t* out, int nsys, const int64_t* n, const int* levels, int p, double box,
                          int precision, void* stream) {
    // the per-system prefix arrays sit in shared memory next to the P2P staging buffers
    if (!out || nsys < 1 || nsys > 1536 || !n || !levels || p < 1 || p > FMM_MAX_P || !(box > 0.0) ||
        !(box < 1e300))
        return FMM_ERR_INVALID_ARG;
    if (precision != FMM_MIXED_FP32 && !fmm_tc_precision(precision)) return FMM_ERR_UNSUPPORTED;
    long long nt = 0;
    for (int i = 0; i < nsys; ++i) {
        if (n[i] < 1 || n[i] > 2147483647LL || levels[i] < 0 || levels[i] > FMM_MAX_LEVELS) return FMM_ERR_INVALID_ARG;
        nt += n[i];
    }
    if (nt > 2147483647LL) return FMM_ERR_INVALID_ARG;
    fmm_batch_s* b = new (std::nothrow) fmm_batch_s();
    if (!b) return FMM_ERR_OOM;
    cudaGetDevice(&b->device);
    b->nsys = nsys;
    b->p = p;
    b->box = box;
    b->stream = static_cast<cudaStream_t>(stream);
    b->precision = precision;
    b->grid_mult = 4;
    b->tc_rows = 0;
    b->p2p_block = FMM_P2P_BLOCK;
    const int m2l_kmax = fmm_tc_precision(precision) ? fmm_tc_kmin() - 1 : FMM_MAX_LEVELS;
    b->p1b = fmm_m2l_bucket(p + 1);
    if (b->p1b < 0) {
        delete b;
        return FMM_ERR_UNSUPPORTED;
    }
    const int p1 = p + 1;
    // system layout: particles, leaves, grid cells (all coarse regions first, then the fine ones)
    b->host_sys.resize(nsys);
    // prefix arrays 0..3, then the upward pass's parents of levels 2 .. FMM_MAX_LEVELS - 1
    constexpr int kPreArrays = 4 + (FMM_MAX_LEVELS - 2);
    std::vector<long long> pre(kPreArrays * (size_t)(nsys + 1), 0);
    b->m2m_kmax = 1;
    long long nl = 0, coarse = 0, cells_fine = 0, bcells = 0;
    nt = 0;
    for (int i = 0; i < nsys; ++i) {
        BatchSys& S = b->host_sys[i];
        memset(&S, 0, sizeof(S));
        S.n = (int)n[i];
        S.levels = levels[i];
        S.p_off = nt;
        S.leaf_off = nl;
        int kf = S.levels;
        while (kf > 2 && ((long long)S.n >> (2 * (kf - 1))) <= kFineMean) --kf;
        S.kf = S.levels < 2 ? 2 : kf;
        for (int k = 2; k < S.kf && k <= S.levels; ++k) {
            S.a_off[k] = coarse;
            coarse += (long long)fmm_grid_width(k) * fmm_grid_width(k);
        }
        nt += S.n;
        nl += 1ll << (2 * S.levels);
    }
    for (int i = 0; i < nsys; ++i) {
        BatchSys& S = b->host_sys[i];
        for (int k = S.kf; k <= S.levels; ++k) {
            S.a_off[k] = coarse + cells_fine;
            cells_fine += (long long)fmm_grid_width(k) * fmm_grid_width(k);
        }
        for (int k = 2; k <= S.levels; ++k) {
            S.b_off[k] = bcells;
            bcells += 1ll << (2 * k);
        }
        const long long s1 = nsys + 1;
        pre[0 * s1 + i + 1] = pre[0 * s1 + i] + S.n;
        pre[1 * s1 + i + 1] = pre[1 * s1 + i] + (1ll << (2 * S.levels));
        long long fine = 0;
        for (int k = S.kf; k <= S.levels && S.levels >= 2; ++k) fine += 1ll << (2 * k);
        pre[2 * s1 + i + 1] = pre[2 * s1 + i] + fine;
        long long m2l = 0;
        for (int k = 2; k <= S.levels && k <= m2l_kmax; ++k) {
            const long long w2 = 1ll << (k - 1);
            m2l += 4 * ((w2 * w2 + kT - 1) / kT);
        }
        pre[3 * s1 + i + 1] = pre[3 * s1 + i] + m2l;
        // the upward pass's parents: level k of this system if k is one of its coarse levels
        for (int k = 2; k < FMM_MAX_LEVELS; ++k) {
            const bool coarse_k = S.levels >= 2 && k < S.kf;
            pre[(size_t)(4 + k - 2) * s1 + i + 1] = pre[(size_t)(4 + k - 2) * s1 + i] + (coarse_k ? (1ll << (2 * k)) : 0);
            if (coarse_k && k > b->m2m_kmax) b->m2m_kmax = k;
        }
    }
    b->nt = nt;
    b->nl = nl;
    b->coarse_cells = coarse;
    b->a_cells = coarse + cells_fine;
    b->b_cells = bcells;
    bool ok = balloc(b, &b->d_sys, sizeof(BatchSys) * nsys) && balloc(b, &b->d_pre, sizeof(long long) * pre.size()) &&
              balloc(b, &b->d_call, sizeof(BatchCall)) && balloc(b, &b->keys, 4 * nt) && balloc(b, &b->rank, 4 * nt) &&
              balloc(b, &b->counts, 4 * nl) && balloc(b, &b->leaf_start, 4 * (nl + 1)) &&
              balloc(b, &b->block_sums, 4 * ((size_t)fmm_scan_blocks(nl) + 1)) && balloc(b, &b->sorted_key, 4 * nt) &&
              balloc(b, &b->leaf_nb, 4 * nl) && balloc(b, &b->bstart, 4 * (nl + 1)) &&
              balloc(b, &b->bmap, sizeof(uint2) * ((size_t)nl + (size_t)nt / kP2PBlockMin + 1)) &&
              balloc(b, &b->sorted32, 16 * nt) &&
              balloc(b, &b->a32, sizeof(float2) * b->a_cells * p1) && balloc(b, &b->b32, sizeof(float2) * bcells * p1) &&
              balloc(b, &b->acc, sizeof(double) * nt) && balloc(b, &b->d_status, sizeof(unsigned int));
    if (!ok) {
        batch_free(b);
        return FMM_ERR_OOM;
    }
    // operators and the upward pass's tables: the plan's FP64 builds, rounded to FP32 in the padded
    // layouts of the FP32 kernels
    {
        fmm_plan_t tmp = nullptr;
        fmm_status s = fmm_plan(&tmp, 1, 2, p, box, FMM_MIXED_FP32, stream);
        if (s != FMM_OK) {
            batch_free(b);
            return s;
        }
        const size_t tsz = (size_t)49 * b->p1b * b->p1b, usz = (size_t)4 * b->p1b * b->p1b;
        ok = balloc(b, &b->T32, sizeof(float2) * tsz) &&
             cudaMemcpy(b->T32, tmp->T32, sizeof(float2) * tsz, cudaMemcpyDeviceToDevice) == cudaSuccess &&
             balloc(b, &b->U32, sizeof(float2) * usz) &&
             cudaMemcpy(b->U32, tmp->U32, sizeof(float2) * usz, cudaMemcpyDeviceToDevice) == cudaSuccess;
        fmm_plan_destroy(tmp);
        if (!ok) {
            batch_free(b);
            return FMM_ERR_CUDA;
        }
    }
    // the tensor-core M2L: every system's levels 6 and finer, one segment each
    if (fmm_tc_precision(precision)) {
        std::vector<double> tre, tim;
        fmm_build_operators_f64(p, tre, tim);
        int err = 0;
        uint64_t bytes = 0;
        b->tc = fmm_tc_new(p, precision, tre, tim, &err, &bytes);
        if (!b->tc) {
            batch_free(b);
            return err == -2 ? FMM_ERR_UNSUPPORTED : FMM_ERR_CUDA;
        }
        std::vector<FmmTcLevel> lev;
        for (int i = 0; i < nsys; ++i) {
            const BatchSys& S = b->host_sys[i];
            for (int k = S.levels; k >= fmm_tc_kmin(); --k)
                lev.push_back({b->a32 + S.a_off[k] * p1, b->b32 + S.b_off[k] * p1, k});
        }
        const int r = fmm_tc_set_levels(b->tc, lev, &bytes);
        b->workspace_bytes += bytes;
        if (r < 0) {
            batch_free(b);
            return FMM_ERR_OOM;
        }
    }
    if (cudaMemcpy(b->d_sys, b->host_sys.data(), sizeof(BatchSys) * nsys, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_pre, pre.data(), sizeof(long long) * pre.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->a32, 0, sizeof(float2) * b->a_cells * p1) != cudaSuccess ||
        cudaMemset(b->d_status, 0, sizeof(unsigned int)) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&b->h_call), sizeof(BatchCall)) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&b->h_status), sizeof(unsigned int)) != cudaSuccess ||
        cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess) {
        batch_free(b);
        return FMM_ERR_CUDA;
    }
    const fmm_status gs = build_graph(b);
    if (gs != FMM_OK) {
        batch_free(b);
        return gs;
    }
    *out = b;
    return FMM_OK;
}

fmm_status fmm_batch_potential(fmm_batch_t b, const double* xy, const double* q, double* phi) {
    if (!b || !xy || !q || !phi) return FMM_ERR_INVALID_ARG;
    return batch_run(b, xy, q, phi);
}

fmm_status fmm_batch_sync(fmm_batch_t b, double* ms) {
    if (!b) return FMM_ERR_INVALID_ARG;
    cudaStream_t st = b->stream;
    if (cudaMemcpyAsync(b->h_status, b->d_status, sizeof(unsigned int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemsetAsync(b->d_status, 0, sizeof(unsigned int), st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return FMM_ERR_CUDA;
    if (ms) {
        float t = 0.f;
        *ms = cudaEventElapsedTime(&t, b->ev0, b->ev1) == cudaSuccess ? (double)t : -1.0;
    }
    const unsigned f = *b->h_status;
    if (f & FMM_FLAG_NONFINITE) return FMM_ERR_NONFINITE;
    if (f & FMM_FLAG_OUT_OF_BOX) return FMM_ERR_OUT_OF_BOX;
    if (f & FMM_FLAG_TIMEOUT) return FMM_ERR_TIMEOUT;
    return FMM_OK;
}

fmm_status fmm_batch_autotune(fmm_batch_t b, const double* xy, const double* q, double* phi, int* grid_mult_out) {
    const fmm_status s = fmm_batch_autotune_cached(b, xy, q, phi, nullptr);
    if (s == FMM_OK && grid_mult_out) *grid_mult_out = b->grid_mult;
    return s;
}

fmm_status fmm_batch_autotune_cached(fmm_batch_t b, const double* xy, const double* q, double* phi,
                                     const char* cache_path) {
    if (!b || !xy || !q || !phi) return FMM_ERR_INVALID_ARG;
    const std::string key = tune_key(b);
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "r")) {
            char line[1024];
            bool hit = false;
            while (!hit && fgets(line, sizeof(line), f)) {
                char k[768];
                int gm = 0, rows = 0, blk = 0;
                double ms = 0.0;
                if (sscanf(line, "%767s %d %d %d %lf", k, &gm, &rows, &blk, &ms) == 5 && key == k && gm >= 1 &&
                    gm <= 16 && rows >= 0 && rows <= 8 && (blk == 16 || blk == 24)) {
                    b->grid_mult = gm;
                    b->tc_rows = rows;
                    b->p2p_block = blk;
                    b->tuned_ms = ms;
                    hit = true;
                }
            }
            fclose(f);
            if (hit) return build_graph(b);
        }
    }
    const int gms[] = {2, 4, 8};
    const int rows_tc[] = {0, 2, 4};
    const int blks[] = {16, 24};
    int best_gm = b->grid_mult, best_rows = b->tc_rows, best_blk = b->p2p_block;
    double best_ms = 1e30;
    for (int gm : gms)
        for (int rows : rows_tc) {
            if (!b->tc && rows != 0) continue;
            for (int blk : blks) {
                b->grid_mult = gm;
                b->tc_rows = rows;
                b->p2p_block = blk;
                double ms = 0.0;
                const fmm_status s = time_shape(b, xy, q, phi, &ms);
                if (s != FMM_OK) return s;
                if (ms < best_ms) {
                    best_ms = ms;
                    best_gm = gm;
                    best_rows = rows;
                    best_blk = blk;
                }
            }
        }
    b->grid_mult = best_gm;
    b->tc_rows = best_rows;
    b->p2p_block = best_blk;
    b->tuned_ms = best_ms;
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "a")) {
            fprintf(f, "%s %d %d %d %.6f\n", key.c_str(), best_gm, best_rows, best_blk, best_ms);
            fclose(f);
        }
    }
    return build_graph(b);
}

fmm_status fmm_batch_tuning(fmm_batch_t b, int* grid_mult, int* tc_rows, int* p2p_block, double* ms) {
    if (!b) return FMM_ERR_INVALID_ARG;
    if (grid_mult) *grid_mult = b->grid_mult;
    if (tc_rows) *tc_rows = b->tc_rows;
    if (p2p_block) *p2p_block = b->p2p_block;
    if (ms) *ms = b->tuned_ms;
    return FMM_OK;
}

int fmm_batch_launches(fmm_batch_t b) { return b ? b->launches : -1; }

void fmm_batch_destroy(fmm_batch_t b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    batch_free(b);
}

}  // extern "C"
