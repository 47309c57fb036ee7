// Shift-free FMM with charges at Lagrange nodes (arXiv 2009.00767, Appendix STEP1-STEP5, Eq. 1-2;
// the summation scheme of Sec. 2.2.1), 2D log and 3D Coulomb kernels, on sm_103a.
//
// Data layout in device memory:
//   * the charges sorted by finest cell in Morton order, so that the charges of any cell at any
//     level are one contiguous range: FP32 forms keep (x, y, z, q) as a float4 "hi" and the
//     residues x - hi as a float4 "lo"; FP64 forms keep (x, y, z, q) as a Pos64;
//   * per level k, the cells in Morton order with d = 4^D node values each (node index
//     i + 4j + 16k): node charges Q_k and node potentials psi_k (node forms), or the vectors
//     v_k and dual vectors u_k (literal form);
//   * node forms: per level a 7^D table of d x d node-to-node matrices, indexed by the offset
//     between source and target cell, laid out [offset][source node i][target node j];
//   * literal form: per level the interaction-list pairs in CSR order by target cell, and one
//     d x d FP64 matrix B = M_{m_i}^T M_b M_m per pair (row a: the root-node coordinate of the
//     source's vector, column l: that of the target's).
//
// Work items of the particle kernels are chunks of up to 128 consecutive sorted charges within
// one finest cell; a persistent grid walks the chunk list, so crowded cells are split over
// blocks and any distribution keeps every SM busy.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "fmm.h"
#include "fmm_lagrange.h"

namespace {

constexpr int kChunk = 128;      // charges per work item
constexpr int kWarpChunk = 64;   // targets per near-field warp work item (two per lane)
constexpr int kMaxLevels = 8;
constexpr double kLn2 = 0.69314718055994530942;

__host__ __device__ constexpr int nodes_of(int D) { return D == 2 ? 16 : 64; }
__host__ __device__ constexpr int offsets_of(int D) { return D == 2 ? 49 : 343; }   // 7^D table

// Eq. 1 on the nodes {-2, -1, 1, 2}: f_i(x) = prod_{j != i} (x - a_j) / (a_i - a_j), written as
// products of the two node pairs' quadratics.
template <typename T>
__host__ __device__ __forceinline__ void lag_basis(T x, T* w) {
    const T a = (x + T(1)) * (x - T(1));   // (x + 1)(x - 1)
    const T b = (x + T(2)) * (x - T(2));   // (x + 2)(x - 2)
    w[0] = a * (x - T(2)) * T(-1.0 / 12.0);
    w[1] = b * (x - T(1)) * T(1.0 / 6.0);
    w[2] = b * (x + T(1)) * T(-1.0 / 6.0);
    w[3] = a * (x + T(2)) * T(1.0 / 12.0);
}

__host__ __device__ __forceinline__ uint32_t morton_enc(int D, const int* c) {
    uint32_t m = 0;
    for (int b = 0; b < 10; ++b)
        for (int a = 0; a < D; ++a) m |= (uint32_t)((c[a] >> b) & 1) << (b * D + a);
    return m;
}

__host__ __device__ __forceinline__ void morton_dec(int D, uint32_t m, int* c) {
    for (int a = 0; a < 3; ++a) c[a] = 0;
    for (int b = 0; b < 10; ++b)
        for (int a = 0; a < D; ++a) c[a] |= (int)((m >> (b * D + a)) & 1u) << b;
}

// The pairwise interaction of a unit charge seen at distance vector r (0 for r = 0).
__host__ __device__ inline double kernel64(int D, double r2) {
    if (r2 == 0.0) return 0.0;
    return D == 2 ? 0.5 * log(r2) : 1.0 / sqrt(r2);
}

constexpr unsigned kFlagOutOfBox = 1u, kFlagNonFinite = 2u;

// The MUFU reciprocal square root and base-2 logarithm with subnormal inputs flushed to zero:
// a near-field r^2 is never subnormal (coincident pairs give exactly 0, which both map to an
// infinity that the own cell's mask removes), so the subnormal handling of rsqrtf / __log2f is
// dead weight in the pair loop.
__device__ __forceinline__ float mufu_rsqrt(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float mufu_lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

}  // namespace

// A sorted charge of the FP64 forms: position and charge, one 32-byte load.
struct __align__(32) Pos64 {
    double x, y, z, w;
};

struct fmm_lag_plan_s {
    int dev = 0, dim = 2, levels = 0, form = 0, d = 16;
    double box = 5.0;
    int64_t n_max = 0, nleaf = 1, last_n = 0;
    cudaStream_t st = nullptr, st2 = nullptr;
    cudaEvent_t ev[9] = {};   // 0 start, 1 far field start, 2 up done, 3 down done, 4 end, 5/6 p2p, 7 sorted
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    uint32_t* key = nullptr;       // [n_max] finest Morton key, input order
    uint32_t* rank = nullptr;      // [n_max] rank within the cell
    uint32_t* skey = nullptr;      // [n_max] key, sorted order
    int* count = nullptr;          // [nleaf]
    int* start = nullptr;          // [nleaf + 1]
    int* chunk_start = nullptr;    // [nleaf + 1]
    int* wchunk_start = nullptr;   // [nleaf + 1] near-field warp chunks
    int* order = nullptr;          // [n_max] sorted -> input index
    float4* hi = nullptr;          // FP32 forms
    float4* lo = nullptr;
    Pos64* p64 = nullptr;        // FP64 forms
    double* nearf = nullptr;       // [n_max] near field, sorted order
    unsigned* status = nullptr;
    unsigned long long* pairs = nullptr;   // near-field pair counter
    int* next_item = nullptr;              // near-field work counter
    void* node[kMaxLevels + 1] = {};       // Q_k (node) or v_k (literal), d values per cell
    void* pot[kMaxLevels + 1] = {};        // psi_k (node) or u_k (literal)
    void* K = nullptr;                     // node forms: operators of levels 2..levels
    int* pair_start[kMaxLevels + 1] = {};  // literal: CSR by target cell
    int* pair_src[kMaxLevels + 1] = {};
    double* B[kMaxLevels + 1] = {};
    int64_t npairs[kMaxLevels + 1] = {};
    int64_t m2l_pairs = 0;
    uint64_t bytes = 0;
    int launches = 0;
    int grid_particles = 0;
    bool serial = false;   // every kernel in turn on the plan's stream (per-kernel timing)
    int grid_p2p = 0;      // resident blocks of the FP32 near-field kernel, all SMs
};

namespace {

// ------------------------------------------------------------------------------ binning

// Finest cell per charge with the FP64 floor/clamp rule, its Morton key and its rank within
// the cell (atomic), plus the input checks.
template <int D>
__global__ void k_bin(const double* __restrict__ pos, const double* __restrict__ q, int64_t n, int L,
                      double box, uint32_t* __restrict__ key, uint32_t* __restrict__ rank, int* __restrict__ count,
                      unsigned* __restrict__ status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int side = 1 << L;
    int c[3] = {0, 0, 0};
    unsigned bad = 0;
    if (!isfinite(q[i])) bad |= kFlagNonFinite;
    for (int a = 0; a < D; ++a) {
        const double x = pos[i * D + a];
        if (!isfinite(x)) bad |= kFlagNonFinite;
        else if (!(x >= 0.0 && x <= box)) bad |= kFlagOutOfBox;
        const double f = floor(x * (double)side / box);
        c[a] = f < 0.0 ? 0 : (f > (double)(side - 1) ? side - 1 : (int)f);
    }
    if (bad) atomicOr(status, bad);
    const uint32_t k = morton_enc(D, c);
    key[i] = k;
    rank[i] = (uint32_t)atomicAdd(count + k, 1);
}

// Exclusive scans of the populations and of the chunk counts, one block.
__global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ count, int nleaf, int* __restrict__ start,
                                               int* __restrict__ chunk_start, int* __restrict__ wchunk_start) {
    __shared__ int s_n[1024], s_c[1024], s_w[1024];
    const int t = threadIdx.x;
    const int per = (nleaf + 1023) / 1024;
    const int b0 = min(nleaf, t * per), b1 = min(nleaf, b0 + per);
    int sn = 0, sc = 0, sw = 0;
    for (int b = b0; b < b1; ++b) {
        sn += count[b];
        sc += (count[b] + kChunk - 1) / kChunk;
        sw += (count[b] + kWarpChunk - 1) / kWarpChunk;
    }
    s_n[t] = sn;
    s_c[t] = sc;
    s_w[t] = sw;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {   // Hillis-Steele inclusive scan
        const int vn = t >= off ? s_n[t - off] : 0, vc = t >= off ? s_c[t - off] : 0;
        const int vw = t >= off ? s_w[t - off] : 0;
        __syncthreads();
        s_n[t] += vn;
        s_c[t] += vc;
        s_w[t] += vw;
        __syncthreads();
    }
    int rn = s_n[t] - sn, rc = s_c[t] - sc, rw = s_w[t] - sw;
    for (int b = b0; b < b1; ++b) {
        start[b] = rn;
        chunk_start[b] = rc;
        wchunk_start[b] = rw;
        rn += count[b];
        rc += (count[b] + kChunk - 1) / kChunk;
        rw += (count[b] + kWarpChunk - 1) / kWarpChunk;
    }
    if (t == 1023) {
        start[nleaf] = s_n[1023];
        chunk_start[nleaf] = s_c[1023];
        wchunk_start[nleaf] = s_w[1023];
    }
}

template <int D, bool k64>
__global__ void k_scatter(const double* __restrict__ pos, const double* __restrict__ q, int64_t n,
                          const uint32_t* __restrict__ key, const uint32_t* __restrict__ rank,
                          const int* __restrict__ start, uint32_t* __restrict__ skey, int* __restrict__ order,
                          float4* __restrict__ hi, float4* __restrict__ lo, Pos64* __restrict__ p64) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t k = key[i];
    const int64_t s = (int64_t)start[k] + rank[i];
    const double x = pos[i * D], y = pos[i * D + 1], z = D == 3 ? pos[i * D + 2] : 0.0;
    skey[s] = k;
    order[s] = (int)i;
    if constexpr (k64) {
        p64[s] = Pos64{x, y, z, q[i]};
    } else {
        const float hx = (float)x, hy = (float)y, hz = (float)z;
        hi[s] = make_float4(hx, hy, hz, (float)q[i]);
        lo[s] = make_float4((float)(x - (double)hx), (float)(y - (double)hy), (float)(z - (double)hz), 0.f);
    }
}

// The finest cell of chunk work item w: the last b with chunk_start[b] <= w.
__device__ __forceinline__ int chunk_leaf(const int* __restrict__ chunk_start, int nleaf, int w) {
    int lo = 0, hi = nleaf;   // chunk_start[lo] <= w < chunk_start[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(chunk_start + mid) <= w) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------------------------ near field

// Sec. 2.1 E-2 in FP32, each pair of adjacent cells evaluated once for both sides.  A warp work
// item is one chunk of up to 64 targets of a finest cell A, two per lane (i and i + 32), against a
// group of A's "forward" cells: A itself and the neighbours B whose offset is positive in (z, y, x)
// order (13 in 3D, 4 in 2D), so that every unordered pair of adjacent cells is met once.  For B != A
// each 1/r (or log r) feeds the target, q_b / r, and the source, q_a / r: the lanes' source terms of
// a 32-source tile are summed across the warp by a transposing butterfly (31 shuffles leave lane j
// with source j's sum), then added to the source in FP64.  A itself is evaluated one-sided with the
// r > 0 mask (only there can a pair sit at distance 0).  The two targets of a lane run in packed
// FP32x2 against one source, staged negated and duplicated, (-x, -x, -y, -y), so that every
// difference is one FADD2; differences come from two-word coordinates, (hi_t - hi_s) + (lo_t - lo_s),
// so a close pair's distance keeps about 48 bits.  Empty slots hold far zero charges.  Sums are FP32
// within a tile and FP64 across tiles, and meet in FP64 atomics.
template <int D, bool kMask>
__device__ __forceinline__ float2 p2p_tile(const float4* __restrict__ s_a, const float4* __restrict__ s_b,
                                           const float4* __restrict__ s_c, const float2* __restrict__ s_d, int m,
                                           float2 tx, float2 ty, float2 tz, float2 ux, float2 uy, float2 uz) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int j = 0; j < m; ++j) {
        const float4 A = s_a[j], B = s_b[j], C = s_c[j];
        const float2 dx = __fadd2_rn(__fadd2_rn(tx, make_float2(A.x, A.y)), __fadd2_rn(ux, make_float2(C.x, C.y)));
        const float2 dy = __fadd2_rn(__fadd2_rn(ty, make_float2(A.z, A.w)), __fadd2_rn(uy, make_float2(C.z, C.w)));
        float2 r2 = __ffma2_rn(dy, dy, __fmul2_rn(dx, dx));
        if constexpr (D == 3) {
            const float2 E = s_d[j];
            const float2 dz = __fadd2_rn(__fadd2_rn(tz, make_float2(B.x, B.y)), __fadd2_rn(uz, E));
            r2 = __ffma2_rn(dz, dz, r2);
        }
        float2 k;
        if constexpr (D == 3) {
            k = make_float2(mufu_rsqrt(r2.x), mufu_rsqrt(r2.y));
        } else {
            k = make_float2(mufu_lg2(r2.x), mufu_lg2(r2.y));
        }
        if constexpr (kMask) {
            k.x = r2.x > 0.f ? k.x : 0.f;
            k.y = r2.y > 0.f ? k.y : 0.f;
        }
        acc = __ffma2_rn(make_float2(B.z, B.w), k, acc);
    }
    return acc;
}

constexpr int kSymTile = 32;     // sources per staged tile (one per lane for the butterfly)
constexpr int kP2PWarps = 8;     // warps per block, each on its own work items
template <int D>
__host__ __device__ constexpr int fwd_group() { return D == 3 ? 4 : 5; }   // forward cells per work item

// Forward cell f of a cell: f = 0 the cell itself, then the offsets o > 0 in (z, y, x) order.
template <int D>
__device__ __forceinline__ void fwd_offset(int f, int* o) {
    o[0] = o[1] = o[2] = 0;
    if (f == 0) return;
    const int e = f - 1;
    if constexpr (D == 3) {
        if (e < 9) { o[0] = e % 3 - 1; o[1] = e / 3 - 1; o[2] = 1; }
        else if (e < 12) { o[0] = e - 10; o[1] = 1; }
        else { o[0] = 1; }
    } else {
        if (e < 3) { o[0] = e - 1; o[1] = 1; }
        else { o[0] = 1; }
    }
}

// v[j] on every lane in, lane j holds the sum over the warp of v[j] out.
__device__ __forceinline__ float warp_transpose_sum(float (&v)[32], int lane) {
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const bool upper = (lane & w) != 0;
#pragma unroll
        for (int i = 0; i < w; ++i) {
            const float send = upper ? v[i] : v[i + w];
            const float keep = upper ? v[i + w] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
        }
    }
    return v[0];
}

template <int D>
__global__ void __launch_bounds__(kP2PWarps * 32) k_p2p32(const float4* __restrict__ hi, const float4* __restrict__ lo,
                                                          const int* __restrict__ start,
                                                          const int* __restrict__ wchunk_start, int nleaf, int L,
                                                          double* __restrict__ nearf,
                                                          unsigned long long* __restrict__ pairs,
                                                          int* __restrict__ next_item) {
    constexpr int F = D == 3 ? 14 : 5, FG = fwd_group<D>(), G = (F + FG - 1) / FG;
    __shared__ float4 s_a[kP2PWarps][kSymTile], s_b[kP2PWarps][kSymTile], s_c[kP2PWarps][kSymTile];
    __shared__ float2 s_d[kP2PWarps][kSymTile];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int side = 1 << L;
    const double scale = D == 2 ? 0.5 * kLn2 : 1.0;
    const int64_t total = (int64_t)wchunk_start[nleaf] * G;
    unsigned long long my_pairs = 0;
    // items are taken from a shared counter, so that the warps finish within one item of each other
    for (;;) {
        int64_t w = 0;
        if (lane == 0) w = atomicAdd(next_item, 1);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= total) break;
        const int cidx = (int)(w / G), g = (int)(w % G);
        const int b = chunk_leaf(wchunk_start, nleaf, cidx);
        const int t0 = start[b] + (cidx - wchunk_start[b]) * kWarpChunk, t1 = min(t0 + kWarpChunk, start[b + 1]);
        const int ia = t0 + lane, ib = ia + 32;
        const bool va = ia < t1, vb = ib < t1;
        // an empty target slot is a zero charge far outside the box
        const float4 far_t = make_float4(-1.0e4f, -1.0e4f, -1.0e4f, 0.f), z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 ha = va ? hi[ia] : far_t, hb = vb ? hi[ib] : far_t;
        const float4 la = va ? lo[ia] : z4, lb = vb ? lo[ib] : z4;
        const float2 tx = make_float2(ha.x, hb.x), ty = make_float2(ha.y, hb.y), tz = make_float2(ha.z, hb.z);
        const float2 ux = make_float2(la.x, lb.x), uy = make_float2(la.y, lb.y), uz = make_float2(la.z, lb.z);
        const float2 qa = make_float2(ha.w, hb.w);
        int c[3];
        morton_dec(D, (uint32_t)b, c);
        double acc_a = 0.0, acc_b = 0.0;
#pragma unroll 1
        for (int f = g * FG; f < min(F, (g + 1) * FG); ++f) {
            int o[3];
            fwd_offset<D>(f, o);
            const int nc[3] = {c[0] + o[0], c[1] + o[1], c[2] + o[2]};
            if (nc[0] < 0 || nc[0] >= side || nc[1] < 0 || nc[1] >= side) continue;
            if (D == 3 && (nc[2] < 0 || nc[2] >= side)) continue;
            const bool own = f == 0;
            const uint32_t nb = morton_enc(D, nc);
            const int s0 = start[nb], s1 = start[nb + 1];
            if (lane == 0) my_pairs += (own ? 1ull : 2ull) * (unsigned long long)(s1 - s0) * (unsigned long long)(t1 - t0);
            for (int s = s0; s < s1; s += kSymTile) {
                const int m = min(kSymTile, s1 - s);
                __syncwarp();
                {
                    const bool have = lane < m;
                    const float4 h = have ? hi[s + lane] : make_float4(1.0e4f, 1.0e4f, 1.0e4f, 0.f);
                    const float4 l = have ? lo[s + lane] : z4;
                    s_a[wid][lane] = make_float4(-h.x, -h.x, -h.y, -h.y);
                    s_b[wid][lane] = make_float4(-h.z, -h.z, h.w, h.w);
                    s_c[wid][lane] = make_float4(-l.x, -l.x, -l.y, -l.y);
                    s_d[wid][lane] = make_float2(-l.z, -l.z);
                }
                __syncwarp();
                if (own) {
                    const float2 a2 = p2p_tile<D, true>(s_a[wid], s_b[wid], s_c[wid], s_d[wid], m, tx, ty, tz, ux, uy, uz);
                    acc_a += (double)a2.x;
                    acc_b += (double)a2.y;
                    continue;
                }
                float cs[kSymTile];
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < kSymTile; ++j) {
                    const float4 A = s_a[wid][j], B = s_b[wid][j], C = s_c[wid][j];
                    const float2 dx = __fadd2_rn(__fadd2_rn(tx, make_float2(A.x, A.y)), __fadd2_rn(ux, make_float2(C.x, C.y)));
                    const float2 dy = __fadd2_rn(__fadd2_rn(ty, make_float2(A.z, A.w)), __fadd2_rn(uy, make_float2(C.z, C.w)));
                    float2 r2 = __ffma2_rn(dy, dy, __fmul2_rn(dx, dx));
                    if constexpr (D == 3) {
                        const float2 E = s_d[wid][j];
                        const float2 dz = __fadd2_rn(__fadd2_rn(tz, make_float2(B.x, B.y)), __fadd2_rn(uz, E));
                        r2 = __ffma2_rn(dz, dz, r2);
                    }
                    const float2 k = D == 3 ? make_float2(mufu_rsqrt(r2.x), mufu_rsqrt(r2.y))
                                            : make_float2(mufu_lg2(r2.x), mufu_lg2(r2.y));
                    acc = __ffma2_rn(make_float2(B.z, B.w), k, acc);
                    const float2 t = __fmul2_rn(qa, k);
                    cs[j] = t.x + t.y;
                }
                acc_a += (double)acc.x;
                acc_b += (double)acc.y;
                const float v = warp_transpose_sum(cs, lane);
                if (lane < m) atomicAdd(nearf + s + lane, (double)v * scale);
            }
        }
        if (va) atomicAdd(nearf + ia, acc_a * scale);
        if (vb) atomicAdd(nearf + ib, acc_b * scale);
    }
    if (lane == 0 && my_pairs) atomicAdd(pairs, my_pairs);
}

// The near field in FP64 (node and literal FP64 forms), same walk.
template <int D>
__global__ void __launch_bounds__(kChunk) k_p2p64(const Pos64* __restrict__ p, const int* __restrict__ start,
                                                  const int* __restrict__ chunk_start, int nleaf, int L,
                                                  double* __restrict__ nearf, unsigned long long* __restrict__ pairs) {
    __shared__ Pos64 s_p[kChunk];
    const int total = chunk_start[nleaf];
    const int side = 1 << L;
    unsigned long long my_pairs = 0;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int b = chunk_leaf(chunk_start, nleaf, w);
        const int t0 = start[b] + (w - chunk_start[b]) * kChunk, t1 = min(t0 + kChunk, start[b + 1]);
        const int i = t0 + (int)threadIdx.x;
        const bool act = i < t1;
        const Pos64 t = act ? p[i] : Pos64{0.0, 0.0, 0.0, 0.0};
        int c[3];
        morton_dec(D, (uint32_t)b, c);
        double acc = 0.0;
        for (int oz = (D == 3 ? -1 : 0); oz <= (D == 3 ? 1 : 0); ++oz)
            for (int oy = -1; oy <= 1; ++oy)
                for (int ox = -1; ox <= 1; ++ox) {
                    const int nc[3] = {c[0] + ox, c[1] + oy, c[2] + oz};
                    if (nc[0] < 0 || nc[0] >= side || nc[1] < 0 || nc[1] >= side) continue;
                    if (D == 3 && (nc[2] < 0 || nc[2] >= side)) continue;
                    const uint32_t nb = morton_enc(D, nc);
                    const int s0 = start[nb], s1 = start[nb + 1];
                    if (threadIdx.x == 0) my_pairs += (unsigned long long)(s1 - s0) * (unsigned long long)(t1 - t0);
                    for (int s = s0; s < s1; s += kChunk) {
                        __syncthreads();
                        if (s + (int)threadIdx.x < s1) s_p[threadIdx.x] = p[s + threadIdx.x];
                        __syncthreads();
                        const int m = min(kChunk, s1 - s);
                        for (int j = 0; j < m; ++j) {
                            const Pos64 sp = s_p[j];
                            const double dx = t.x - sp.x, dy = t.y - sp.y, dz = t.z - sp.z;
                            const double r2 = dx * dx + dy * dy + dz * dz;
                            if (r2 > 0.0) acc += sp.w * (D == 2 ? 0.5 * log(r2) : 1.0 / sqrt(r2));
                        }
                    }
                }
        if (act) nearf[i] = acc;
    }
    if (threadIdx.x == 0 && my_pairs) atomicAdd(pairs, my_pairs);
}

// ------------------------------------------------------------------------------ node charges

template <typename T>
__device__ __forceinline__ void atomic_add(T* a, T v) {
    atomicAdd(a, v);
}

// Local coordinate (position - centre) / (s/5) of a sorted charge on axis a.
template <typename T>
struct PosReader;
template <>
struct PosReader<float> {
    const float4* hi;
    const float4* lo;
    __device__ float local(int i, int a, double centre, double inv) const {
        const float4 h = hi[i], l = lo[i];
        const float hv = a == 0 ? h.x : (a == 1 ? h.y : h.z), lv = a == 0 ? l.x : (a == 1 ? l.y : l.z);
        return ((hv - (float)centre) + lv) * (float)inv;
    }
    __device__ float charge(int i) const { return hi[i].w; }
};
template <>
struct PosReader<double> {
    const Pos64* p;
    __device__ double local(int i, int a, double centre, double inv) const {
        const Pos64 v = p[i];
        return ((a == 0 ? v.x : (a == 1 ? v.y : v.z)) - centre) * inv;
    }
    __device__ double charge(int i) const { return p[i].w; }
};

struct LevelPtrs {
    void* p[kMaxLevels + 1];
};

// STEP2 summed per cell: for each level k in [k0, k1] add sum_c q_c h(c) over the chunk's
// charges into the node values of the accumulation cell.  Node forms: weights and accumulation
// at level k (the node charges M_m v_m of every level straight from the charges, no shift).
// Literal U-bar-1: weights of the root box (wlevel0) accumulated into the finest cell.
template <int D, typename T>
__global__ void __launch_bounds__(kChunk) k_p2m(PosReader<T> rd, const int* __restrict__ start,
                                                const int* __restrict__ chunk_start, int nleaf, int L, double box,
                                                int k0, int k1, bool wlevel0, LevelPtrs out) {
    constexpr int d = nodes_of(D), PL = kChunk / d;
    __shared__ T s_w[kChunk][D][4];
    __shared__ T s_q[kChunk];
    __shared__ T s_red[kChunk];
    const int total = chunk_start[nleaf];
    const int tid = threadIdx.x, j = tid % d, pl = tid / d;
    const int ji[3] = {j & 3, (j >> 2) & 3, j >> 4};
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int b = chunk_leaf(chunk_start, nleaf, w);
        const int t0 = start[b] + (w - chunk_start[b]) * kChunk, t1 = min(t0 + kChunk, start[b + 1]);
        const int m = t1 - t0;
        for (int k = k0; k <= k1; ++k) {
            const int kw = wlevel0 ? 0 : k;               // level whose nodes the weights refer to
            const uint32_t cell = (uint32_t)b >> (D * (L - k));
            int cc[3];
            morton_dec(D, (uint32_t)b >> (D * (L - kw)), cc);
            const double s = box / (double)(1 << kw), inv = 5.0 / s;
            __syncthreads();
            if (tid < m) {
                for (int a = 0; a < D; ++a) lag_basis<T>(rd.local(t0 + tid, a, ((double)cc[a] + 0.5) * s, inv), s_w[tid][a]);
                s_q[tid] = rd.charge(t0 + tid);
            }
            __syncthreads();
            T acc = T(0);
            for (int c = pl; c < m; c += PL) {
                T v = s_q[c] * s_w[c][0][ji[0]] * s_w[c][1][ji[1]];
                if constexpr (D == 3) v *= s_w[c][2][ji[2]];
                acc += v;
            }
            s_red[tid] = acc;
            __syncthreads();
            if (pl == 0) {
                for (int r = 1; r < PL; ++r) acc += s_red[r * d + j];
                atomic_add(static_cast<T*>(out.p[k]) + (size_t)cell * d + j, acc);
            }
        }
    }
}

// ------------------------------------------------------------------------------ node potentials

// psi_m[j] += sum_{o in IL} sum_i K_k[o][i][j] Q_{m+o}[i] for one level.  Targets are grouped by
// the parity of their coordinates: within a parity class the interaction list is the same set of
// offsets (o_a in [-2 - p_a, 3 - p_a], Chebyshev distance >= 2), so a block takes 32 targets of
// one class and a group of offsets, and applies each offset's d x d matrix to 32 source columns
// (a small dense product with the matrix in shared memory).
template <int D, typename T>
constexpr size_t m2l_smem_bytes() {
    return ((size_t)nodes_of(D) * nodes_of(D) + (size_t)nodes_of(D) * 33) * sizeof(T);
}

template <int D, typename T>
__global__ void __launch_bounds__(256) k_m2l(const T* __restrict__ K, const T* __restrict__ Q, T* __restrict__ psi,
                                             int k, int ngroups) {
    constexpr int d = nodes_of(D), TT = 32, NT = 256, NTG = NT / d, RT = TT / NTG;
    constexpr int NOFF = D == 2 ? 27 : 189;
    extern __shared__ __align__(16) unsigned char m2l_smem[];
    T* s_K = reinterpret_cast<T*>(m2l_smem);                              // [d][d]
    T(*s_Q)[TT + 1] = reinterpret_cast<T(*)[TT + 1]>(s_K + d * d);        // [d][TT + 1]
    const int side = 1 << k, pside = side >> 1;
    const int nparent = D == 2 ? pside * pside : pside * pside * pside;
    const int ntiles = (nparent + TT - 1) / TT;
    int blk = blockIdx.x;
    const int g = blk % ngroups;
    blk /= ngroups;
    const int tile = blk % ntiles, par = blk / ntiles;
    const int p[3] = {par & 1, (par >> 1) & 1, (par >> 2) & 1};
    const int tid = threadIdx.x, j = tid % d, tg = tid / d;
    // this group's offsets among the class's NOFF
    const int per = (NOFF + ngroups - 1) / ngroups, e0 = g * per, e1 = min(NOFF, e0 + per);
    T acc[RT], comp[RT];
#pragma unroll
    for (int r = 0; r < RT; ++r) acc[r] = comp[r] = T(0);
    int e = 0;   // running index of the class's offsets
    for (int oz = (D == 3 ? -2 - p[2] : 0); oz <= (D == 3 ? 3 - p[2] : 0); ++oz)
        for (int oy = -2 - p[1]; oy <= 3 - p[1]; ++oy)
            for (int ox = -2 - p[0]; ox <= 3 - p[0]; ++ox) {
                const int cheb = max(abs(ox), max(abs(oy), abs(oz)));
                if (cheb < 2) continue;
                const int my = e++;
                if (my < e0 || my >= e1) continue;
                const int oidx = (ox + 3) + 7 * (oy + 3) + (D == 3 ? 49 * (oz + 3) : 0);
                __syncthreads();
                const float4* Ko = reinterpret_cast<const float4*>(K + (size_t)oidx * d * d);
                for (int x = tid; x < d * d * (int)sizeof(T) / 16; x += NT) reinterpret_cast<float4*>(s_K)[x] = Ko[x];
                for (int x = tid; x < d * TT; x += NT) {
                    const int tt = x / d, i = x % d;
                    const int P = tile * TT + tt;
                    T v = T(0);
                    if (P < nparent) {
                        const int pc[3] = {P % pside, (P / pside) % pside, D == 3 ? P / (pside * pside) : 0};
                        const int sc[3] = {2 * pc[0] + p[0] + ox, 2 * pc[1] + p[1] + oy, 2 * pc[2] + p[2] + oz};
                        bool in = sc[0] >= 0 && sc[0] < side && sc[1] >= 0 && sc[1] < side;
                        if (D == 3) in = in && sc[2] >= 0 && sc[2] < side;
                        if (in) v = Q[(size_t)morton_enc(D, sc) * d + i];
                    }
                    s_Q[i][tt] = v;
                }
                __syncthreads();
                T t[RT];
#pragma unroll
                for (int r = 0; r < RT; ++r) t[r] = T(0);
#pragma unroll 8
                for (int i = 0; i < d; ++i) {
                    const T kv = s_K[i * d + j];
#pragma unroll
                    for (int r = 0; r < RT; ++r) t[r] += kv * s_Q[i][tg * RT + r];
                }
                // one offset's d-term product is added to the running sum with Kahan's compensation
                // in FP32: a plain running sum over a group's offsets (up to 21 x 64 terms in 3D)
                // would leave about 1e-6 of the far field in rounding
#pragma unroll
                for (int r = 0; r < RT; ++r) {
                    if constexpr (sizeof(T) == 4) {
                        const T y = t[r] - comp[r];
                        const T sum = acc[r] + y;
                        comp[r] = (sum - acc[r]) - y;
                        acc[r] = sum;
                    } else {
                        acc[r] += t[r];
                    }
                }
            }
#pragma unroll
    for (int r = 0; r < RT; ++r) {
        const int P = tile * TT + tg * RT + r;
        if (P >= nparent) continue;
        const int pc[3] = {P % pside, (P / pside) % pside, D == 3 ? P / (pside * pside) : 0};
        const int tc[3] = {2 * pc[0] + p[0], 2 * pc[1] + p[1], 2 * pc[2] + p[2]};
        atomic_add(psi + (size_t)morton_enc(D, tc) * d + j, acc[r]);
    }
}

// ------------------------------------------------------------------------------ evaluation

// Node forms: phi_far(c) = sum_{k=2..L} h_{m_k}(c) . psi_{m_k}, the tensor-product contraction
// done axis by axis; phi in input order = far + near, written only if the inputs passed.
template <int D, typename T>
__global__ void k_l2p(PosReader<T> rd, const uint32_t* __restrict__ skey, int64_t n, int L, double box,
                      LevelPtrs psi, const double* __restrict__ nearf, const int* __restrict__ order,
                      const unsigned* __restrict__ status, double* __restrict__ phi) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t key = skey[i];
    double far = 0.0;
    for (int k = 2; k <= L; ++k) {
        const uint32_t cell = key >> (D * (L - k));
        int cc[3];
        morton_dec(D, cell, cc);
        const double s = box / (double)(1 << k), inv = 5.0 / s;
        T f[3][4];
        for (int a = 0; a < D; ++a) lag_basis<T>(rd.local((int)i, a, ((double)cc[a] + 0.5) * s, inv), f[a]);
        const T* ps = static_cast<const T*>(psi.p[k]) + (size_t)cell * nodes_of(D);
        T v = T(0);
        if constexpr (D == 2) {
#pragma unroll
            for (int iy = 0; iy < 4; ++iy) {
                T r = T(0);
#pragma unroll
                for (int ix = 0; ix < 4; ++ix) r += f[0][ix] * __ldg(ps + ix + 4 * iy);
                v += f[1][iy] * r;
            }
        } else {
#pragma unroll
            for (int iz = 0; iz < 4; ++iz) {
                T u = T(0);
#pragma unroll
                for (int iy = 0; iy < 4; ++iy) {
                    T r = T(0);
#pragma unroll
                    for (int ix = 0; ix < 4; ++ix) r += f[0][ix] * __ldg(ps + ix + 4 * iy + 16 * iz);
                    u += f[1][iy] * r;
                }
                v += f[2][iz] * u;
            }
        }
        far += (double)v;
    }
    if (*(volatile const unsigned*)status != 0u) return;
    phi[order[i]] = far + nearf[i];
}

// ------------------------------------------------------------------------------ literal form

// U-bar-2: v_k of a cell = sum of its 2^D children's (contiguous in Morton order), no shift.
template <int D>
__global__ void k_lit_up(const double* __restrict__ child, double* __restrict__ parent, int64_t ncell) {
    constexpr int d = nodes_of(D);
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= ncell * d) return;
    const int64_t c = x / d, j = x % d;
    double s = 0.0;
    for (int ch = 0; ch < (1 << D); ++ch) s += child[((c << D) + ch) * d + j];
    parent[x] = s;
}

// D-bar-1 and D-bar-2 of one level: u_m = sum_{pairs (m_i, m)} B^T v_{m_i} + u_parent(m).
// Threads: d target coordinates l x (256 / d) pair lanes; B rows are read coalesced over l.
template <int D>
__global__ void __launch_bounds__(256) k_lit_down(const int* __restrict__ pstart, const int* __restrict__ psrc,
                                                  const double* __restrict__ B, const double* __restrict__ v,
                                                  const double* __restrict__ uparent, double* __restrict__ u,
                                                  int64_t ncell) {
    constexpr int d = nodes_of(D), PG = 256 / d;
    __shared__ double s_red[256];
    const int64_t m = blockIdx.x;
    if (m >= ncell) return;
    const int l = threadIdx.x % d, g = threadIdx.x / d;
    double acc = 0.0;
    for (int e = pstart[m] + g; e < pstart[m + 1]; e += PG) {
        const double* vs = v + (size_t)psrc[e] * d;
        const double* Be = B + (size_t)e * d * d;
        for (int a = 0; a < d; ++a) acc += __ldg(vs + a) * Be[(size_t)a * d + l];
    }
    s_red[threadIdx.x] = acc;
    __syncthreads();
    if (g == 0) {
        for (int r = 1; r < PG; ++r) acc += s_red[r * d + l];
        if (uparent) acc += uparent[(size_t)(m >> D) * d + l];
        u[(size_t)m * d + l] = acc;
    }
}

// F(v) = L_{m^l}(v) for each charge's own v (unit charge at the root box's nodes) + near field.
template <int D>
__global__ void k_lit_eval(const Pos64* __restrict__ p, const uint32_t* __restrict__ skey, int64_t n, double box,
                           const double* __restrict__ u, const double* __restrict__ nearf,
                           const int* __restrict__ order, const unsigned* __restrict__ status,
                           double* __restrict__ phi) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Pos64 c = p[i];
    const double inv = 5.0 / box, centre = 0.5 * box;
    double f[3][4];
    lag_basis<double>((c.x - centre) * inv, f[0]);
    lag_basis<double>((c.y - centre) * inv, f[1]);
    if (D == 3) lag_basis<double>((c.z - centre) * inv, f[2]);
    const double* ul = u + (size_t)skey[i] * nodes_of(D);
    double far = 0.0;
    for (int j = 0; j < nodes_of(D); ++j) {
        double w = f[0][j & 3] * f[1][(j >> 2) & 3];
        if (D == 3) w *= f[2][j >> 4];
        far += ul[j] * w;
    }
    if (*(volatile const unsigned*)status != 0u) return;
    phi[order[i]] = far + nearf[i];
}

// STEP3-STEP5 for one pair per block: M_m and M_{m_i} (columns h_m(p_l) of the root nodes),
// M_b[i][j] = K(node j of m - node i of m_i), T = M_b M_m, B = M_{m_i}^T T, all FP64.
template <int D>
__global__ void __launch_bounds__(256) k_lit_build(const int* __restrict__ ptgt, const int* __restrict__ psrc,
                                                   int64_t npairs, int k, double box, double* __restrict__ B) {
    constexpr int d = nodes_of(D);
    extern __shared__ double smem[];
    double* Mm = smem;             // [d][d]
    double* Mi = Mm + d * d;       // [d][d]
    double* T = Mi + d * d;        // [d][d], first M_b then M_b M_m
    double* Mb = T + d * d;        // [d][d]
    const int64_t e = blockIdx.x;
    if (e >= npairs) return;
    const double s = box / (double)(1 << k), h = s / 5.0;
    const double a_node[4] = {-2.0, -1.0, 1.0, 2.0};
    int cm[3], ci[3];
    morton_dec(D, (uint32_t)ptgt[e], cm);
    morton_dec(D, (uint32_t)psrc[e], ci);
    for (int x = threadIdx.x; x < d * d; x += blockDim.x) {
        const int row = x / d, col = x % d;   // row: cell node, col: root node
        const int rn[3] = {row & 3, (row >> 2) & 3, row >> 4};
        const int cn[3] = {col & 3, (col >> 2) & 3, col >> 4};
        double wm = 1.0, wi = 1.0;
        for (int a = 0; a < D; ++a) {
            const double pr = 0.5 * box + (box / 5.0) * a_node[cn[a]];   // root node coordinate
            double f[4];
            lag_basis<double>((pr - ((double)cm[a] + 0.5) * s) / h, f);
            wm *= f[rn[a]];
            lag_basis<double>((pr - ((double)ci[a] + 0.5) * s) / h, f);
            wi *= f[rn[a]];
        }
        Mm[x] = wm;
        Mi[x] = wi;
        // M_b[i = row][j = col]: source node i of m_i, target node j of m
        double r2 = 0.0;
        for (int a = 0; a < D; ++a) {
            const double pt = ((double)cm[a] + 0.5) * s + h * a_node[cn[a]];
            const double ps = ((double)ci[a] + 0.5) * s + h * a_node[rn[a]];
            r2 += (pt - ps) * (pt - ps);
        }
        Mb[x] = kernel64(D, r2);
    }
    __syncthreads();
    for (int x = threadIdx.x; x < d * d; x += blockDim.x) {
        const int i = x / d, l = x % d;
        double acc = 0.0;
        for (int j = 0; j < d; ++j) acc += Mb[i * d + j] * Mm[j * d + l];
        T[x] = acc;
    }
    __syncthreads();
    double* Be = B + (size_t)e * d * d;
    for (int x = threadIdx.x; x < d * d; x += blockDim.x) {
        const int a = x / d, l = x % d;
        double acc = 0.0;
        for (int i = 0; i < d; ++i) acc += Mi[i * d + a] * T[i * d + l];
        Be[x] = acc;
    }
}

// ------------------------------------------------------------------------------ direct sum

template <int D>
__global__ void k_direct_targets(const double* __restrict__ pos, const double* __restrict__ q, int64_t n,
                                 const int64_t* __restrict__ tgt, int64_t nt, double* __restrict__ phi) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const int64_t i = tgt[t];
    const double x = pos[i * D], y = pos[i * D + 1], z = D == 3 ? pos[i * D + 2] : 0.0;
    double acc = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        const double dx = x - pos[j * D], dy = y - pos[j * D + 1], dz = D == 3 ? z - pos[j * D + 2] : 0.0;
        acc += q[j] * kernel64(D, dx * dx + dy * dy + dz * dz);
    }
    phi[t] = acc;
}

// ------------------------------------------------------------------------------ host helpers

int64_t ipow(int64_t b, int e) {
    int64_t r = 1;
    while (e-- > 0) r *= b;
    return r;
}

// The interaction list of cell m (coords) at level k, as Morton indices.
int il_cells(int D, int k, const int* m, std::vector<uint32_t>& out) {
    const int side = 1 << k;
    out.clear();
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) {
        const int p = m[a] >> 1;
        lo[a] = std::max(0, 2 * (p - 1));
        hi[a] = std::min(side - 1, 2 * (p + 1) + 1);
    }
    int c[3] = {0, 0, 0};
    for (c[2] = (D == 3 ? lo[2] : 0); c[2] <= (D == 3 ? hi[2] : 0); ++c[2])
        for (c[1] = lo[1]; c[1] <= hi[1]; ++c[1])
            for (c[0] = lo[0]; c[0] <= hi[0]; ++c[0]) {
                int cheb = 0;
                for (int a = 0; a < D; ++a) cheb = std::max(cheb, std::abs(c[a] - m[a]));
                if (cheb >= 2) out.push_back(morton_enc(D, c));
            }
    return (int)out.size();
}

bool valid_form(int f) { return f == FMM_LAG_NODE_F32 || f == FMM_LAG_NODE_F64 || f == FMM_LAG_LITERAL_F64; }

fmm_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return FMM_OK;
    return e == cudaErrorMemoryAllocation ? FMM_ERR_OOM : FMM_ERR_CUDA;
}

template <typename T>
fmm_status alloc(fmm_lag_plan_s* pl, T** p, size_t count) {
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return cuda_status(e);
    }
    pl->bytes += bytes;
    return FMM_OK;
}

void plan_free(fmm_lag_plan_s* pl) {
    if (!pl) return;
    cudaFree(pl->key); cudaFree(pl->rank); cudaFree(pl->skey); cudaFree(pl->count); cudaFree(pl->start);
    cudaFree(pl->chunk_start); cudaFree(pl->wchunk_start); cudaFree(pl->order); cudaFree(pl->hi); cudaFree(pl->lo); cudaFree(pl->p64);
    cudaFree(pl->nearf); cudaFree(pl->status); cudaFree(pl->pairs); cudaFree(pl->next_item); cudaFree(pl->K);
    for (int k = 0; k <= kMaxLevels; ++k) {
        cudaFree(pl->node[k]); cudaFree(pl->pot[k]); cudaFree(pl->pair_start[k]); cudaFree(pl->pair_src[k]);
        cudaFree(pl->B[k]);
    }
    for (auto& e : pl->ev) if (e) cudaEventDestroy(e);
    if (pl->ev_fork) cudaEventDestroy(pl->ev_fork);
    if (pl->ev_join) cudaEventDestroy(pl->ev_join);
    if (pl->st2) cudaStreamDestroy(pl->st2);
    delete pl;
}

// Node-to-node operators of levels 2..L, FP64 on the host: K_k[o][i][j] = K(node j of the target
// - node i of the source at offset o), o over the 7^D table (the near offsets stay zero).
std::vector<double> build_operators(int D, int L, double box) {
    const int d = nodes_of(D), no = offsets_of(D);
    const double a_node[4] = {-2.0, -1.0, 1.0, 2.0};
    std::vector<double> K((size_t)std::max(0, L - 1) * no * d * d, 0.0);
    for (int k = 2; k <= L; ++k) {
        const double s = box / (double)(1 << k), h = s / 5.0;
        double* Kk = K.data() + (size_t)(k - 2) * no * d * d;
        for (int oi = 0; oi < no; ++oi) {
            const int o[3] = {oi % 7 - 3, (oi / 7) % 7 - 3, D == 3 ? oi / 49 - 3 : 0};
            if (std::max(std::abs(o[0]), std::max(std::abs(o[1]), std::abs(o[2]))) < 2) continue;
            for (int i = 0; i < d; ++i)
                for (int j = 0; j < d; ++j) {
                    const int ni[3] = {i & 3, (i >> 2) & 3, i >> 4}, nj[3] = {j & 3, (j >> 2) & 3, j >> 4};
                    double r2 = 0.0;
                    for (int a = 0; a < D; ++a) {
                        const double r = h * (a_node[nj[a]] - a_node[ni[a]]) - o[a] * s;
                        r2 += r * r;
                    }
                    Kk[((size_t)oi * d + i) * d + j] = kernel64(D, r2);
                }
        }
    }
    return K;
}

template <int D>
fmm_status enqueue(fmm_lag_plan_s* pl, const double* pos, const double* q, int64_t n, double* phi) {
    constexpr int d = nodes_of(D);
    const int L = pl->levels;
    const bool f64 = pl->form != FMM_LAG_NODE_F32, lit = pl->form == FMM_LAG_LITERAL_F64;
    cudaStream_t st = pl->st;
    int launches = 0;
    cudaEventRecord(pl->ev[0], st);
    cudaMemsetAsync(pl->count, 0, sizeof(int) * (size_t)pl->nleaf, st);
    cudaMemsetAsync(pl->pairs, 0, sizeof(unsigned long long), st);
    for (int k = (lit ? std::max(L, 2) : 2); k <= L; ++k) {
        const size_t cells = (size_t)ipow(1 << k, D) * d;
        cudaMemsetAsync(pl->node[k], 0, cells * (f64 ? 8 : 4), st);
        if (!lit) cudaMemsetAsync(pl->pot[k], 0, cells * (f64 ? 8 : 4), st);
    }
    const unsigned gb = (unsigned)((n + 255) / 256);
    k_bin<D><<<gb, 256, 0, st>>>(pos, q, n, L, pl->box, pl->key, pl->rank, pl->count, pl->status);
    k_scan<<<1, 1024, 0, st>>>(pl->count, (int)pl->nleaf, pl->start, pl->chunk_start, pl->wchunk_start);
    if (f64)
        k_scatter<D, true><<<gb, 256, 0, st>>>(pos, q, n, pl->key, pl->rank, pl->start, pl->skey, pl->order,
                                                nullptr, nullptr, pl->p64);
    else
        k_scatter<D, false><<<gb, 256, 0, st>>>(pos, q, n, pl->key, pl->rank, pl->start, pl->skey, pl->order,
                                                 pl->hi, pl->lo, nullptr);
    launches += 3;
    cudaEventRecord(pl->ev[7], st);
    cudaEventRecord(pl->ev[1], st);
    // near field on the second stream (or in turn on the plan's stream in serial mode)
    cudaStream_t p2p_st = pl->serial ? st : pl->st2;
    if (!pl->serial) {
        cudaEventRecord(pl->ev_fork, st);
        cudaStreamWaitEvent(pl->st2, pl->ev_fork, 0);
    }
    const unsigned gp = (unsigned)pl->grid_particles;
    if (!f64) {
        cudaMemsetAsync(pl->nearf, 0, sizeof(double) * (size_t)n, p2p_st);
        cudaMemsetAsync(pl->next_item, 0, sizeof(int), p2p_st);
    }
    cudaEventRecord(pl->ev[5], p2p_st);
    if (f64) {
        k_p2p64<D><<<gp, kChunk, 0, p2p_st>>>(pl->p64, pl->start, pl->chunk_start, (int)pl->nleaf, L, pl->nearf,
                                               pl->pairs);
    } else {
        k_p2p32<D><<<(unsigned)pl->grid_p2p, kP2PWarps * 32, 0, p2p_st>>>(
            pl->hi, pl->lo, pl->start, pl->wchunk_start, (int)pl->nleaf, L, pl->nearf, pl->pairs, pl->next_item);
    }
    ++launches;
    cudaEventRecord(pl->ev[6], p2p_st);
    cudaEventRecord(pl->ev_join, p2p_st);
    if (pl->serial) cudaEventRecord(pl->ev[1], st);   // the far-field stages start after the near field

    LevelPtrs nodes{}, pots{};
    for (int k = 0; k <= kMaxLevels; ++k) {
        nodes.p[k] = pl->node[k];
        pots.p[k] = pl->pot[k];
    }
    if (!lit) {
        if (L >= 2) {
            if (f64)
                k_p2m<D, double><<<gp, kChunk, 0, st>>>(PosReader<double>{pl->p64}, pl->start, pl->chunk_start,
                                                        (int)pl->nleaf, L, pl->box, 2, L, false, nodes);
            else
                k_p2m<D, float><<<gp, kChunk, 0, st>>>(PosReader<float>{pl->hi, pl->lo}, pl->start, pl->chunk_start,
                                                       (int)pl->nleaf, L, pl->box, 2, L, false, nodes);
            ++launches;
        }
        cudaEventRecord(pl->ev[2], st);
        const int ngroups = D == 2 ? 3 : 27;
        for (int k = 2; k <= L; ++k) {
            const int pside = 1 << (k - 1);
            const int64_t nparent = ipow(pside, D);
            const unsigned blocks = (unsigned)(((nparent + 31) / 32) * (1 << D) * ngroups);
            const size_t koff = (size_t)(k - 2) * offsets_of(D) * d * d;
            if (f64)
                k_m2l<D, double><<<blocks, 256, m2l_smem_bytes<D, double>(), st>>>(static_cast<const double*>(pl->K) + koff,
                                                         static_cast<const double*>(pl->node[k]),
                                                         static_cast<double*>(pl->pot[k]), k, ngroups);
            else
                k_m2l<D, float><<<blocks, 256, m2l_smem_bytes<D, float>(), st>>>(static_cast<const float*>(pl->K) + koff,
                                                        static_cast<const float*>(pl->node[k]),
                                                        static_cast<float*>(pl->pot[k]), k, ngroups);
            ++launches;
        }
        cudaEventRecord(pl->ev[3], st);
        cudaStreamWaitEvent(st, pl->ev_join, 0);
        if (f64)
            k_l2p<D, double><<<gb, 256, 0, st>>>(PosReader<double>{pl->p64}, pl->skey, n, L, pl->box, pots, pl->nearf,
                                                 pl->order, pl->status, phi);
        else
            k_l2p<D, float><<<gb, 256, 0, st>>>(PosReader<float>{pl->hi, pl->lo}, pl->skey, n, L, pl->box, pots,
                                                pl->nearf, pl->order, pl->status, phi);
        ++launches;
    } else if (L < 2) {
        // no interaction lists: phi is the near field (the node evaluation over no levels)
        cudaEventRecord(pl->ev[2], st);
        cudaEventRecord(pl->ev[3], st);
        cudaStreamWaitEvent(st, pl->ev_join, 0);
        k_l2p<D, double><<<gb, 256, 0, st>>>(PosReader<double>{pl->p64}, pl->skey, n, L, pl->box, pots, pl->nearf,
                                             pl->order, pl->status, phi);
        ++launches;
    } else {
        // U-bar-1: v of every finest cell from the charges' root-node images
        k_p2m<D, double><<<gp, kChunk, 0, st>>>(PosReader<double>{pl->p64}, pl->start, pl->chunk_start,
                                                (int)pl->nleaf, L, pl->box, L, L, true, nodes);
        ++launches;
        // U-bar-2: sums up the tree (levels below 2 are never read)
        for (int k = L - 1; k >= 2; --k) {
            const int64_t ncell = ipow(1 << k, D);
            k_lit_up<D><<<(unsigned)((ncell * d + 255) / 256), 256, 0, st>>>(
                static_cast<const double*>(pl->node[k + 1]), static_cast<double*>(pl->node[k]), ncell);
            ++launches;
        }
        cudaEventRecord(pl->ev[2], st);
        // D-bar-1 and D-bar-2 level by level, top down
        for (int k = 2; k <= L; ++k) {
            const int64_t ncell = ipow(1 << k, D);
            k_lit_down<D><<<(unsigned)ncell, 256, 0, st>>>(pl->pair_start[k], pl->pair_src[k], pl->B[k],
                                                           static_cast<const double*>(pl->node[k]),
                                                           k >= 3 ? static_cast<const double*>(pl->pot[k - 1]) : nullptr,
                                                           static_cast<double*>(pl->pot[k]), ncell);
            ++launches;
        }
        cudaEventRecord(pl->ev[3], st);
        cudaStreamWaitEvent(st, pl->ev_join, 0);
        k_lit_eval<D><<<gb, 256, 0, st>>>(pl->p64, pl->skey, n, pl->box, static_cast<const double*>(pl->pot[L]),
                                          pl->nearf, pl->order, pl->status, phi);
        ++launches;
    }
    cudaEventRecord(pl->ev[4], st);
    pl->launches = launches;
    pl->last_n = n;
    return cuda_status(cudaGetLastError());
}

}  // namespace

extern "C" {

fmm_status fmm_lag_plan(fmm_lag_plan_t* out, int dim, int64_t n_max, int levels, double box, int form,
                        void* stream) {
    if (!out || (dim != 2 && dim != 3) || n_max < 1 || n_max > (int64_t(1) << 30) || !valid_form(form) ||
        !(box > 0.0) || !std::isfinite(box) || levels < 0)
        return FMM_ERR_INVALID_ARG;
    const bool lit = form == FMM_LAG_LITERAL_F64;
    const int lmax = dim == 2 ? (lit ? 7 : 8) : (lit ? 3 : 5);
    if (levels > lmax) return FMM_ERR_INVALID_ARG;
    auto* pl = new (std::nothrow) fmm_lag_plan_s;
    if (!pl) return FMM_ERR_OOM;
    pl->dim = dim; pl->levels = levels; pl->form = form; pl->box = box; pl->n_max = n_max;
    pl->d = nodes_of(dim);
    pl->st = static_cast<cudaStream_t>(stream);
    pl->nleaf = ipow(1 << levels, dim);
    const int d = pl->d;
    const bool f64 = form != FMM_LAG_NODE_F32;
    fmm_status rc = cuda_status(cudaGetDevice(&pl->dev));
    int sms = 0;
    if (rc == FMM_OK) rc = cuda_status(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->dev));
    pl->grid_particles = std::max(1, sms) * 8;
    int per_sm = 0;
    if (rc == FMM_OK)
        rc = cuda_status(dim == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_p2p32<2>, kP2PWarps * 32, 0)
                                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_p2p32<3>, kP2PWarps * 32, 0));
    pl->grid_p2p = std::max(1, sms) * std::max(1, per_sm);
    if (rc == FMM_OK) rc = cuda_status(cudaStreamCreateWithFlags(&pl->st2, cudaStreamNonBlocking));
    for (auto& e : pl->ev)
        if (rc == FMM_OK) rc = cuda_status(cudaEventCreate(&e));
    if (rc == FMM_OK) rc = cuda_status(cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming));
    if (rc == FMM_OK) rc = cuda_status(cudaEventCreateWithFlags(&pl->ev_join, cudaEventDisableTiming));
    const size_t n = (size_t)n_max;
    if (rc == FMM_OK) rc = alloc(pl, &pl->key, n);
    if (rc == FMM_OK) rc = alloc(pl, &pl->rank, n);
    if (rc == FMM_OK) rc = alloc(pl, &pl->skey, n);
    if (rc == FMM_OK) rc = alloc(pl, &pl->order, n);
    if (rc == FMM_OK) rc = alloc(pl, &pl->nearf, n);
    if (rc == FMM_OK) rc = alloc(pl, &pl->count, (size_t)pl->nleaf);
    if (rc == FMM_OK) rc = alloc(pl, &pl->start, (size_t)pl->nleaf + 1);
    if (rc == FMM_OK) rc = alloc(pl, &pl->chunk_start, (size_t)pl->nleaf + 1);
    if (rc == FMM_OK) rc = alloc(pl, &pl->wchunk_start, (size_t)pl->nleaf + 1);
    if (rc == FMM_OK) rc = alloc(pl, &pl->status, 1);
    if (rc == FMM_OK) rc = alloc(pl, &pl->pairs, 1);
    if (rc == FMM_OK) rc = alloc(pl, &pl->next_item, 1);
    if (rc == FMM_OK && f64) rc = alloc(pl, &pl->p64, n);
    if (rc == FMM_OK && !f64) rc = alloc(pl, &pl->hi, n);
    if (rc == FMM_OK && !f64) rc = alloc(pl, &pl->lo, n);
    const size_t vb = f64 ? 8 : 4;
    for (int k = 2; k <= levels && rc == FMM_OK; ++k) {
        const size_t cells = (size_t)ipow(1 << k, dim) * d;
        void** a = &pl->node[k];
        void** b = &pl->pot[k];
        if (vb == 8) {
            rc = alloc(pl, reinterpret_cast<double**>(a), cells);
            if (rc == FMM_OK) rc = alloc(pl, reinterpret_cast<double**>(b), cells);
        } else {
            rc = alloc(pl, reinterpret_cast<float**>(a), cells);
            if (rc == FMM_OK) rc = alloc(pl, reinterpret_cast<float**>(b), cells);
        }
    }
    if (rc == FMM_OK) rc = cuda_status(cudaMemset(pl->status, 0, sizeof(unsigned)));
    if (rc == FMM_OK && dim == 3 && f64 && !lit)
        rc = cuda_status(cudaFuncSetAttribute(k_m2l<3, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)m2l_smem_bytes<3, double>()));
    if (rc == FMM_OK && !lit && levels >= 2) {
        const std::vector<double> K = build_operators(dim, levels, box);
        if (f64) {
            double* Kd = nullptr;
            rc = alloc(pl, &Kd, K.size());
            pl->K = Kd;
            if (rc == FMM_OK) rc = cuda_status(cudaMemcpy(Kd, K.data(), K.size() * 8, cudaMemcpyHostToDevice));
        } else {
            std::vector<float> Kf(K.begin(), K.end());
            float* Kd = nullptr;
            rc = alloc(pl, &Kd, Kf.size());
            pl->K = Kd;
            if (rc == FMM_OK) rc = cuda_status(cudaMemcpy(Kd, Kf.data(), Kf.size() * 4, cudaMemcpyHostToDevice));
        }
        for (int k = 2; k <= levels; ++k) {
            std::vector<uint32_t> il;
            for (int64_t c = 0; c < ipow(1 << k, dim); ++c) {
                int cc[3];
                morton_dec(dim, (uint32_t)c, cc);
                pl->m2l_pairs += il_cells(dim, k, cc, il);
            }
        }
    }
    if (rc == FMM_OK && lit && levels >= 2) {
        const size_t smem = 4 * (size_t)d * d * sizeof(double);
        cudaError_t e = dim == 2 ? cudaFuncSetAttribute(k_lit_build<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                                 : cudaFuncSetAttribute(k_lit_build<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        rc = cuda_status(e);
        for (int k = 2; k <= levels && rc == FMM_OK; ++k) {
            const int64_t ncell = ipow(1 << k, dim);
            std::vector<int> ps((size_t)ncell + 1, 0), src, tgt;
            std::vector<uint32_t> il;
            for (int64_t c = 0; c < ncell; ++c) {
                int cc[3];
                morton_dec(dim, (uint32_t)c, cc);
                il_cells(dim, k, cc, il);
                for (uint32_t s : il) {
                    src.push_back((int)s);
                    tgt.push_back((int)c);
                }
                ps[(size_t)c + 1] = (int)src.size();
            }
            pl->npairs[k] = (int64_t)src.size();
            pl->m2l_pairs += pl->npairs[k];
            int* dtgt = nullptr;
            rc = alloc(pl, &pl->pair_start[k], ps.size());
            if (rc == FMM_OK) rc = alloc(pl, &pl->pair_src[k], src.size());
            if (rc == FMM_OK) rc = alloc(pl, &pl->B[k], src.size() * (size_t)d * d);
            if (rc == FMM_OK) rc = cuda_status(cudaMalloc(&dtgt, std::max<size_t>(1, tgt.size()) * sizeof(int)));
            if (rc == FMM_OK)
                rc = cuda_status(cudaMemcpy(pl->pair_start[k], ps.data(), ps.size() * 4, cudaMemcpyHostToDevice));
            if (rc == FMM_OK && !src.empty())
                rc = cuda_status(cudaMemcpy(pl->pair_src[k], src.data(), src.size() * 4, cudaMemcpyHostToDevice));
            if (rc == FMM_OK && !tgt.empty())
                rc = cuda_status(cudaMemcpy(dtgt, tgt.data(), tgt.size() * 4, cudaMemcpyHostToDevice));
            if (rc == FMM_OK && !src.empty()) {
                if (dim == 2)
                    k_lit_build<2><<<(unsigned)src.size(), 256, smem>>>(dtgt, pl->pair_src[k], (int64_t)src.size(), k,
                                                                       box, pl->B[k]);
                else
                    k_lit_build<3><<<(unsigned)src.size(), 256, smem>>>(dtgt, pl->pair_src[k], (int64_t)src.size(), k,
                                                                       box, pl->B[k]);
                rc = cuda_status(cudaGetLastError());
                if (rc == FMM_OK) rc = cuda_status(cudaDeviceSynchronize());
            }
            if (dtgt) cudaFree(dtgt);
        }
    }
    if (rc != FMM_OK) {
        plan_free(pl);
        return rc;
    }
    *out = pl;
    return FMM_OK;
}

fmm_status fmm_lag_potential(fmm_lag_plan_t pl, const double* pos, const double* q, int64_t n, double* phi) {
    if (!pl || n < 0 || n > pl->n_max || (n > 0 && (!pos || !q || !phi))) return FMM_ERR_INVALID_ARG;
    if (n == 0) {
        pl->last_n = 0;
        return FMM_OK;
    }
    return pl->dim == 2 ? enqueue<2>(pl, pos, q, n, phi) : enqueue<3>(pl, pos, q, n, phi);
}

fmm_status fmm_lag_sync(fmm_lag_plan_t pl) {
    if (!pl) return FMM_ERR_INVALID_ARG;
    fmm_status rc = cuda_status(cudaStreamSynchronize(pl->st));
    if (rc == FMM_OK) rc = cuda_status(cudaStreamSynchronize(pl->st2));
    if (rc != FMM_OK) return rc;
    unsigned flags = 0;
    rc = cuda_status(cudaMemcpy(&flags, pl->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (rc != FMM_OK) return rc;
    if (flags) {
        cudaMemset(pl->status, 0, sizeof(unsigned));
        return (flags & kFlagNonFinite) ? FMM_ERR_NONFINITE : FMM_ERR_OUT_OF_BOX;
    }
    return FMM_OK;
}

fmm_status fmm_lag_stats_get(fmm_lag_plan_t pl, fmm_lag_stats* out) {
    if (!pl || !out) return FMM_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    out->n = pl->last_n;
    out->dim = pl->dim;
    out->levels = pl->levels;
    out->form = pl->form;
    out->workspace_bytes = pl->bytes;
    out->m2l_pairs = pl->m2l_pairs;
    if (pl->last_n == 0) return FMM_OK;
    auto span = [&](int a, int b) {
        float ms = 0.f;
        return cudaEventElapsedTime(&ms, pl->ev[a], pl->ev[b]) == cudaSuccess ? (double)ms : 0.0;
    };
    out->ms_total = span(0, 4);
    out->ms_sort = span(0, 7);
    out->ms_up = span(1, 2);
    out->ms_down = span(2, 3);
    out->ms_eval = span(3, 4);
    out->ms_p2p = span(5, 6);
    unsigned long long pairs = 0;
    if (cudaMemcpy(&pairs, pl->pairs, sizeof(pairs), cudaMemcpyDeviceToHost) != cudaSuccess) return FMM_ERR_CUDA;
    out->p2p_pairs = (int64_t)pairs;
    out->kernel_launches = pl->launches;
    return FMM_OK;
}

fmm_status fmm_lag_set_concurrency(fmm_lag_plan_t pl, int streams) {
    if (!pl || (streams != 1 && streams != 2)) return FMM_ERR_INVALID_ARG;
    pl->serial = streams == 1;
    return FMM_OK;
}

fmm_status fmm_lag_set_stream(fmm_lag_plan_t pl, void* stream) {
    if (!pl) return FMM_ERR_INVALID_ARG;
    pl->st = static_cast<cudaStream_t>(stream);
    return FMM_OK;
}

}  // extern "C"

namespace {
template <int D>
__global__ void k_cells(const uint32_t* __restrict__ key, int64_t n, int32_t* __restrict__ cells) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c[3];
    morton_dec(D, key[i], c);
    for (int a = 0; a < D; ++a) cells[i * D + a] = c[a];
}
}  // namespace

extern "C" {

fmm_status fmm_lag_cells(fmm_lag_plan_t pl, int32_t* cells) {
    if (!pl || (!cells && pl->last_n > 0)) return FMM_ERR_INVALID_ARG;
    if (pl->last_n == 0) return FMM_OK;
    const unsigned g = (unsigned)((pl->last_n + 255) / 256);
    if (pl->dim == 2) k_cells<2><<<g, 256, 0, pl->st>>>(pl->key, pl->last_n, cells);
    else k_cells<3><<<g, 256, 0, pl->st>>>(pl->key, pl->last_n, cells);
    return cuda_status(cudaGetLastError());
}

fmm_status fmm_lag_direct_targets(int dim, int64_t n, const double* pos, const double* q, int64_t nt,
                                  const int64_t* tgt, double* phi, void* stream) {
    if ((dim != 2 && dim != 3) || n < 0 || nt < 0 || (nt > 0 && (!pos || !q || !tgt || !phi))) return FMM_ERR_INVALID_ARG;
    if (nt == 0) return FMM_OK;
    const unsigned g = (unsigned)((nt + 127) / 128);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (dim == 2) k_direct_targets<2><<<g, 128, 0, st>>>(pos, q, n, tgt, nt, phi);
    else k_direct_targets<3><<<g, 128, 0, st>>>(pos, q, n, tgt, nt, phi);
    return cuda_status(cudaGetLastError());
}

void fmm_lag_plan_destroy(fmm_lag_plan_t pl) {
    if (!pl) return;
    cudaStreamSynchronize(pl->st);
    cudaStreamSynchronize(pl->st2);
    plan_free(pl);
}

}  // extern "C"
