// m2l_tc.cu -- M2L (D-bar-1 of Sec. 2.2.1) on the 5th-generation tensor cores (tcgen05) for every
// level, in TF32 or in split 3xTF32 with FP32 accumulation in tensor memory.
//
// For one level k and one parity class c = (px, py) of target squares, the conversion of the
// interaction list is a real GEMM
//     D[t][n] = sum_d sum_kk  S[t + d][kk] * Op_d[n][kk]
// with t the targets, n the outputs (N = 2H: Re b'_0..b'_p then Im b'_0..b'_p, each padded to H)
// and kk the inputs (K = 2H per offset: Re M_0..M_p then Im M_0..M_p).  The 27 offsets of the
// class fall into 12 groups that share one source window: the source parity (qx, qy) and the
// source row shift sy.  The source grid of a parity is a (w2 + 2) x (w2 + 2) array with a 1-cell
// zero halo, stored chunk-major ([parity][K/4 chunk][row][col][4 floats]); read as one flat array
// of cells, a tile is 128 consecutive cells starting at flat position P and its window for shift
// sy the 130 cells from P - 1 + sy (w2 + 2): each K-chunk of it is one contiguous run of 2080
// bytes.  Rows of at least 128 targets take tiles aligned to the row; narrower sub-grids (levels
// below 8) take consecutive runs of the flat array, and the outputs that fall on halo cells are
// dropped.  A window is KC bulk copies (cp.async.bulk) per part, issued by the producer warp's
// lanes in parallel, that land in the canonical no-swizzle K-major shared layout (16-byte
// core-matrix rows, K-chunk stride LBO = 130 x 16 B) and complete on the stage's mbarrier; the three column shifts of a group are the same window read from a
// descriptor start moved by 16 B per cell.  The operators are scale-free, so a CTA takes up to
// eight tiles of one class from any levels and loads each group's operators (one bulk copy) once
// for all of them.  Warp 0 issues the copies (running up to NSW windows ahead), one thread of
// warp 1 issues the MMAs into one tensor-memory accumulator per tile, all four warps run the
// epilogue, which reads the accumulators back with tcgen05.ld and stores them.
//
// 3xTF32 (Ootomo & Yokota, 2022): x = x_hi + x_lo with x_hi rounded to TF32, and
// D += A_hi B_hi + A_hi B_lo + A_lo B_hi, dropping A_lo B_lo, recovers about FP32 accuracy.
//
// The monopole-log term of b'_0, sum_d M_0 (log|w0| + ln s), carries the largest part of phi; it
// stays out of the GEMM (its (0, 0) operator entry is zero): k_m2l_mono sums it in float-float
// from the FP32 moment grid after the GEMM, in both TF32 modes; a TF32 product of a large M_0
// with the log would lose more than the error bound allows on clustered systems.  Every wait on
// an mbarrier is bounded and sets a status flag when it runs out.

#include <cmath>
#include <cstring>
#include <vector>

#include "mixed_common.cuh"

namespace {

constexpr int kTile = 128;        // targets per tile (MMA M)
constexpr int kWin = kTile + 2;   // source cells per window
constexpr int kThreads = 128;
constexpr int kMinLevel = 7;      // coarser levels stay on the CUDA cores (see fmm_tc_kmin)
constexpr int kMaxRows = 8;       // tiles per CTA: 8 accumulators of 64 columns fill tensor memory
constexpr int kSrcPad = 1024;     // cells after each source array: flat tiles past the last row read there
constexpr unsigned kSpin = 1u << 24;

struct TcGroup {
    int qx, qy, sy, nops, slot0;
    int sx[3];
    int d[3];
};

struct TcArgs {
    const float* src[2][FMM_MAX_LEVELS + 1];   // [part][level] -> [q][KC][w2+2][w2+2][4] (1-cell zero halo)
    const float* ops[2];                       // [part] -> [class][27 slots][KC][N][4], scale-free
    float2* B[FMM_MAX_LEVELS + 1];
    TcGroup groups[4][12];
    // the tiles of one class, finest level first: level seg_level[j] owns tiles
    // seg_start[j] .. seg_start[j + 1] - 1; CTA b takes tiles c * rows .. of class b % 4, c = b / 4
    int seg_start[FMM_MAX_LEVELS + 2];
    int seg_level[FMM_MAX_LEVELS + 1];
    int nseg, tiles, rows, tmem_cols;
    int levels, p;
    unsigned int* status;
};

// flat start (halo coordinates) of tile T of a parity sub-grid of width w2
__host__ __device__ __forceinline__ int tile_start(int w2, int T) {
    const int W2P = w2 + 2;
    if (w2 >= kTile) {
        const int per_row = w2 / kTile;
        return (T / per_row + 1) * W2P + 1 + (T % per_row) * kTile;
    }
    return W2P + 1 + T * kTile;
}

__host__ __device__ __forceinline__ int tiles_of_level(int k) {
    const int w2 = 1 << (k - 1);
    if (w2 >= kTile) return w2 * (w2 / kTile);
    return (w2 * (w2 + 2) - 2 + kTile - 1) / kTile;   // the flat run from (1, 1) to (w2, w2)
}

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity) {
    for (unsigned it = 0; it < kSpin; ++it) {
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

// Shared-memory matrix descriptor, no swizzle, K-major core matrices (8 rows x 16 B).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// A CTA takes up to kMaxRows tiles of one parity class (any levels), one TMEM accumulator each.
// For each of the 12 groups the operators are loaded once and serve all the CTA's tiles; the
// group's source windows, one per tile, stream through NSW buffers.
// Stages: ops buffers NSO (per group), window buffers NSW (per tile and group).

template <int KC, int NP, int NSO, int NSW>
__global__ void __launch_bounds__(kThreads, 1) k_m2l_tc(const __grid_constant__ TcArgs a) {
    constexpr int N = 4 * KC, H = 2 * KC;
    constexpr uint32_t A_BYTES = KC * kWin * 16;     // one window, one part
    constexpr uint32_t OP_BYTES = KC * N * 16;       // one offset's operator, one part
    constexpr uint32_t OPS_STAGE = NP * 3 * OP_BYTES;
    constexpr uint32_t WIN_STAGE = NP * A_BYTES;
    constexpr uint32_t ACC_COLS = 64;                // per tile (N <= 64)
    constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((128u >> 4) << 24);

    static_assert(NSW >= 2, "the window pipeline keeps one window in flight: it needs two window stages");
    extern __shared__ uint8_t smem_raw[];
    // no swizzled layouts are used: 128-byte alignment serves the copies and the descriptors
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    uint8_t* ops_buf = smem;                                   // NSO x OPS_STAGE
    uint8_t* win_buf = smem + NSO * OPS_STAGE;                 // NSW x WIN_STAGE
    uint64_t* bars = reinterpret_cast<uint64_t*>(win_buf + NSW * WIN_STAGE);
    uint64_t* ops_full = bars;                 // [NSO]
    uint64_t* ops_empty = bars + NSO;          // [NSO]
    uint64_t* win_full = bars + 2 * NSO;       // [NSW]
    uint64_t* win_empty = win_full + NSW;      // [NSW]
    uint64_t* done_bar = win_empty + NSW;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(done_bar + 1);
    int* tile_k = reinterpret_cast<int*>(tmem_holder + 1);   // [kMaxRows] level of each tile
    int* tile_P = tile_k + kMaxRows;                           // [kMaxRows] flat start of each tile

    // ---- which tiles
    const int cls = blockIdx.x & 3;
    const int t0 = (blockIdx.x >> 2) * a.rows;
    const int nrows = min(a.rows, a.tiles - t0);
    const int px = cls & 1, py = cls >> 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < nrows) {
        const int tau = t0 + threadIdx.x;
        int j = 0;
        while (j + 1 < a.nseg && tau >= a.seg_start[j + 1]) ++j;
        const int k = a.seg_level[j];
        tile_k[threadIdx.x] = k;
        tile_P[threadIdx.x] = tile_start(1 << (k - 1), tau - a.seg_start[j]);
    }
    const uint32_t TMEM_COLS = (uint32_t)a.tmem_cols;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_holder)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int b = 0; b < NSO; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&ops_full[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&ops_empty[b])) : "memory");
        }
        for (int b = 0; b < NSW; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&win_full[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&win_empty[b])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(done_bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_holder;

    bool ok = true;
    const int NWIN = 12 * nrows;
    if (warp == 0) {
        // producer warp: lane 0 waits for a free stage and posts its byte count, then the lanes
        // issue the stage's bulk copies in parallel (an operator part, or one K chunk of one part
        // of the window each); every copy completes on the stage's full barrier, so the producer
        // runs ahead of the MMAs
        for (int i = 0; i < NWIN; ++i) {
            const int g = i / nrows, t = i % nrows;
            const TcGroup& G = a.groups[cls][g];
            if (t == 0) {
                const int so = g % NSO, uso = g / NSO;
                const uint32_t bytes = (uint32_t)G.nops * OP_BYTES;
                if (lane == 0) {
                    if (g >= NSO && !wait_bar(su32(&ops_empty[so]), (uint32_t)((uso - 1) & 1))) ok = false;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&ops_full[so])),
                                 "r"(NP * bytes)
                                 : "memory");
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) break;
                if (lane < NP) {
                    const float* srcB = a.ops[lane] + ((size_t)cls * 27 + G.slot0) * (OP_BYTES / 4);
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            su32(ops_buf + so * OPS_STAGE + lane * 3 * OP_BYTES)),
                        "l"(srcB), "r"(bytes), "r"(su32(&ops_full[so]))
                        : "memory");
                }
            }
            const int sw = i % NSW, usw = i / NSW;
            if (lane == 0) {
                if (i >= NSW && !wait_bar(su32(&win_empty[sw]), (uint32_t)((usw - 1) & 1))) ok = false;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&win_full[sw])),
                             "r"((uint32_t)(NP * A_BYTES))
                             : "memory");
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            if (lane < NP * KC) {
                // chunk j of part `part` of the 130 cells from the window's flat start: 2080
                // contiguous bytes (past a chunk's end it reads the next chunk or the zero pad,
                // which only feed dropped outputs)
                const int part = lane / KC, j = lane % KC;
                const int q = G.qx + 2 * G.qy;
                const int k = tile_k[t];
                const size_t W2P = ((size_t)1 << (k - 1)) + 2;
                const size_t start = (size_t)(tile_P[t] - 1 + G.sy * (int)W2P);   // flat, >= 0
                const float* src = a.src[part][k] + (((size_t)q * KC + j) * W2P * W2P + start) * 4;
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        su32(win_buf + sw * WIN_STAGE + part * A_BYTES + j * (kWin * 16))),
                    "l"(src), "r"((uint32_t)(kWin * 16)), "r"(su32(&win_full[sw]))
                    : "memory");
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            for (int i = 0; i < NWIN; ++i) {
                const int g = i / nrows, t = i % nrows;
                const TcGroup& G = a.groups[cls][g];
                const int so = g % NSO, uso = g / NSO;
                const int sw = i % NSW, usw = i / NSW;
                if (t == 0 && !wait_bar(su32(&ops_full[so]), (uint32_t)(uso & 1))) ok = false;
                if (!wait_bar(su32(&win_full[sw]), (uint32_t)(usw & 1))) ok = false;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t aBase = su32(win_buf + sw * WIN_STAGE);
                const uint32_t bBase = su32(ops_buf + so * OPS_STAGE);
                const uint32_t acc_t = tmem + (uint32_t)t * ACC_COLS;
                for (int o = 0; o < G.nops && ok; ++o) {
                    const uint32_t aoff = (uint32_t)(1 + G.sx[o]) * 16u;
#pragma unroll
                    for (int ks = 0; ks < KC / 2; ++ks) {
                        const uint32_t acc = (g | o | ks) != 0;
                        const uint64_t ah = smem_desc(aBase + aoff + ks * 2 * (kWin * 16), kWin * 16, 128);
                        const uint64_t bh = smem_desc(bBase + o * OP_BYTES + ks * 2 * (N * 16), N * 16, 128);
                        mma_tf32(acc_t, ah, bh, IDESC, acc);
                        if (NP == 2) {
                            const uint64_t al =
                                smem_desc(aBase + A_BYTES + aoff + ks * 2 * (kWin * 16), kWin * 16, 128);
                            const uint64_t bl =
                                smem_desc(bBase + 3 * OP_BYTES + o * OP_BYTES + ks * 2 * (N * 16), N * 16, 128);
                            mma_tf32(acc_t, ah, bl, IDESC, 1u);
                            mma_tf32(acc_t, al, bh, IDESC, 1u);
                        }
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 su32(&win_empty[sw]))
                             : "memory");
                if (t == nrows - 1)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     su32(&ops_empty[so]))
                                 : "memory");
            }
            // the final commit tracks every MMA issued above
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             su32(done_bar))
                         : "memory");
        }
        __syncwarp();
    }
    if (!ok) atomicOr(a.status, FMM_FLAG_TIMEOUT);
    const bool done = wait_bar(su32(done_bar), 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // ---- epilogue: warp w holds accumulator rows (targets) 32w..32w+31 of every tile
    const int p1 = a.p + 1;
    for (int t = 0; t < nrows; ++t) {
        float v[N];
#pragma unroll
        for (int c = 0; c < N; c += 16)
            tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(t * ACC_COLS + c), v + c);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int k = tile_k[t];
        const int w2 = 1 << (k - 1), W2P = w2 + 2;
        const int pos = tile_P[t] + 32 * warp + lane;
        const int x = pos % W2P - 1, y = pos / W2P - 1;   // sub-grid cell; halo cells are dropped
        if (done && x >= 0 && x < w2 && y < w2) {
            const int tx = 2 * x + px, ty = 2 * y + py;
            // Re b'_0 without the monopole-log term, which k_m2l_mono adds in float-float
            float2* B = a.B[k] + ((size_t)ty * (1u << k) + tx) * p1;
            B[0] = make_float2(v[0], 0.f);
#pragma unroll
            for (int l = 1; l < H; ++l)
                if (l < p1) B[l] = make_float2(v[l], v[H + l]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// FP32 moment grid (3-cell halo) -> the GEMM's source layout, one thread per cell of a parity
// sub-grid: out[part][q][KC][w2][w2][4] with the K index Re M_0..M_p, pad, Im M_0..M_p, pad.
__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

struct PrepArgs {
    const float2* a32[FMM_MAX_LEVELS + 1];
    float4* hi[FMM_MAX_LEVELS + 1];
    float4* lo[FMM_MAX_LEVELS + 1];
    long long base[FMM_MAX_LEVELS + 2];   // first cell (over all four parities) of each level
    int kmin, levels, p1;
};

template <int KC, int NP>
__global__ void k_prep_tc(const __grid_constant__ PrepArgs a) {
    constexpr int H = 2 * KC;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.base[a.levels + 1]) return;
    int k = a.kmin;
    while (g >= a.base[k + 1]) ++k;
    const int64_t e = g - a.base[k];
    const int w2 = 1 << (k - 1), W2P = w2 + 2, p1 = a.p1;
    const int col = (int)(e % w2), row = (int)((e / w2) % w2), q = (int)(e / ((int64_t)w2 * w2));
    const int x = 2 * col + (q & 1), y = 2 * row + (q >> 1);
    const int W = fmm_grid_width(k);
    const float2* src = a.a32[k] + ((size_t)(y + FMM_HALO) * W + (x + FMM_HALO)) * p1;
    float vals[2 * H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
        const float2 m = (j < p1) ? src[j] : make_float2(0.f, 0.f);
        vals[j] = m.x;                     // coefficient 0 holds M_0's high word: M_0 is real
        vals[H + j] = (j == 0) ? 0.f : m.y;
    }
    // chunk-major source layout [q][chunk][row][col][4] (1-cell zero halo): the chunk of a run of
    // consecutive cells of the flat array is one contiguous block
    float4* hi = a.hi[k];
    float4* lo = a.lo[k];
#pragma unroll
    for (int c = 0; c < KC; ++c) {
        float h[4], l[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float v = vals[4 * c + t];
            h[t] = tf32_rna(v);
            l[t] = v - h[t];
        }
        const size_t at = (((size_t)q * KC + c) * W2P + (size_t)(row + 1)) * W2P + (size_t)(col + 1);
        hi[at] = make_float4(h[0], h[1], h[2], h[3]);
        if (NP == 2) lo[at] = make_float4(l[0], l[1], l[2], l[3]);
    }
}

// The monopole-log term of b'_0 for the tensor-core levels, sum_d M_0[t + d] (log|w0_d| + ln s_k)
// over the target's interaction list, summed in float-float (in the order dy, then dx) and added to
// the GEMM's Re b'_0: one thread per target, the 27 loads of a target issued together.
struct MonoArgs {
    const float2* a32[FMM_MAX_LEVELS + 1];
    float2* B[FMM_MAX_LEVELS + 1];
    float2 logc[FMM_MAX_LEVELS + 1][49];
    long long base[FMM_MAX_LEVELS + 2];   // first target of each level
    int kmin, levels, p1;
};

// the 27 list offsets of targets of parity (PX, PY), loads first, then the float-float sum
template <int PX, int PY>
__device__ __forceinline__ float2 mono_sum(const float2* __restrict__ A32, const float2 (&logc)[49], size_t c0, int W,
                                           int p1) {
    float2 m0[49];
#pragma unroll
    for (int dy = -3; dy <= 3; ++dy)
#pragma unroll
        for (int dx = -3; dx <= 3; ++dx) {
            const bool adj = dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1;
            const bool in = dx >= -2 - PX && dx <= 3 - PX && dy >= -2 - PY && dy <= 3 - PY;
            if (in && !adj) m0[(dy + 3) * 7 + dx + 3] = A32[(c0 + (ptrdiff_t)dy * W + dx) * p1];
        }
    float2 mono = make_float2(0.f, 0.f);
#pragma unroll
    for (int dy = -3; dy <= 3; ++dy)
#pragma unroll
        for (int dx = -3; dx <= 3; ++dx) {
            const bool adj = dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1;
            const bool in = dx >= -2 - PX && dx <= 3 - PX && dy >= -2 - PY && dy <= 3 - PY;
            if (in && !adj) mono = ff_add(mono, ff_mul(m0[(dy + 3) * 7 + dx + 3], logc[(dx + 3) + 7 * (dy + 3)]));
        }
    return mono;
}

__global__ void k_m2l_mono(const __grid_constant__ MonoArgs a) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.base[a.levels + 1]) return;
    int k = a.kmin;
    while (g >= a.base[k + 1]) ++k;
    const int64_t t = g - a.base[k];
    const int side = 1 << k, W = fmm_grid_width(k), p1 = a.p1;
    const int tx = (int)(t % side), ty = (int)(t / side);
    const size_t c0 = (size_t)(ty + FMM_HALO) * W + (tx + FMM_HALO);
    float2 mono;
    switch ((tx & 1) + 2 * (ty & 1)) {
        case 0: mono = mono_sum<0, 0>(a.a32[k], a.logc[k], c0, W, p1); break;
        case 1: mono = mono_sum<1, 0>(a.a32[k], a.logc[k], c0, W, p1); break;
        case 2: mono = mono_sum<0, 1>(a.a32[k], a.logc[k], c0, W, p1); break;
        default: mono = mono_sum<1, 1>(a.a32[k], a.logc[k], c0, W, p1); break;
    }
    float2* B = a.B[k] + (size_t)t * p1;
    B[0] = ff_add_f(mono, B[0].x);   // Re b'_0 as float-float
}

// host-side round to nearest TF32 (ties away), the rounding cvt.rna.tf32.f32 does on the device
float host_tf32(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return x;
    u = (u + 0x1000u) & 0xffffe000u;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

// shared-memory plan: (ops stages, window stages) = (2, 2), else (1, 2); 128 bytes of alignment
// slack and 256 bytes of barriers
template <int KC, int NP>
constexpr size_t tc_bytes(int nso, int nsw) {
    return (size_t)nso * NP * 3 * (KC * (4 * KC) * 16) + (size_t)nsw * NP * (KC * kWin * 16) + 128 + 256;
}
template <int KC, int NP>
constexpr int tc_nso() {
    return tc_bytes<KC, NP>(2, 2) <= 227 * 1024 ? 2 : 1;
}
template <int KC, int NP>
constexpr int tc_nsw() {
    static_assert(tc_bytes<KC, NP>(1, 2) <= 227 * 1024, "two window stages must fit");
    return 2;
}

}  // namespace

// ---------------------------------------------------------------- plan-side state
struct FmmTc {
    int kc, np, sms;
    float* ops[2];                              // one scale-free copy per part
    float4* src[2][FMM_MAX_LEVELS + 1];
    TcArgs args;   // tables, filled at plan time
};

// The tensor cores take levels kMinLevel and finer.  The coarse levels carry most of the far
// field's amplitude, and the tensor core's FP32 accumulation (product alignment and rounding inside
// each MMA) loses more there than FP32 FMAs; they hold few targets, so the CUDA cores take them.
int fmm_tc_kmin() { return kMinLevel; }

// Allocate and build the tensor-core M2L state.  Returns 0, or a negative value on failure
// (-1 CUDA error, -2 unsupported p).
int fmm_tc_create(fmm_plan_s* pl, const std::vector<double>& Tre, const std::vector<double>& Tim) {
    const int p1 = pl->p + 1;
    const int H = ((p1 + 7) / 8) * 8;
    const int kc = H / 2;
    if (kc != 4 && kc != 8 && kc != 12 && kc != 16) return -2;
    const int np = pl->precision == FMM_MIXED_3XTF32 ? 2 : 1;
    FmmTc* tc = new FmmTc();
    memset(tc, 0, sizeof(FmmTc));
    tc->kc = kc;
    tc->np = np;
    pl->tc = tc;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&tc->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -1;
    const int N = 4 * kc, K = 4 * kc;

    // class tables: 12 groups (source parity qx, qy and row shift sy) of 1..3 offsets each
    int slots[4] = {0, 0, 0, 0};
    for (int cls = 0; cls < 4; ++cls) {
        const int px = cls & 1, py = cls >> 1;
        int g = 0;
        for (int qy = 0; qy < 2; ++qy)
            for (int qx = 0; qx < 2; ++qx)
                for (int sy = -1; sy <= 1; ++sy, ++g) {
                    TcGroup& G = tc->args.groups[cls][g];
                    G.qx = qx;
                    G.qy = qy;
                    G.sy = sy;
                    G.nops = 0;
                    G.slot0 = slots[cls];
                    const int dy = 2 * sy + qy - py;
                    for (int sx = -1; sx <= 1; ++sx) {
                        const int dx = 2 * sx + qx - px;
                        if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
                        G.sx[G.nops] = sx;
                        G.d[G.nops] = (dx + 3) + 7 * (dy + 3);
                        ++G.nops;
                    }
                    slots[cls] += G.nops;
                }
        if (slots[cls] != 27) return -1;
    }
    // operators, real block form, [part][class][slot][KC][N][4]: scale-free, so one copy serves
    // every level; the monopole-log entry (0, 0) is left out (summed in float-float by k_m2l_mono)
    const size_t opsz = (size_t)4 * 27 * kc * N * 4;
    {
        std::vector<float> hostops[2];
        for (int part = 0; part < np; ++part) hostops[part].assign(opsz, 0.f);
        for (int cls = 0; cls < 4; ++cls)
            for (int g = 0; g < 12; ++g) {
                const TcGroup& G = tc->args.groups[cls][g];
                for (int o = 0; o < G.nops; ++o) {
                    const int d = G.d[o];
                    const size_t base = ((size_t)cls * 27 + G.slot0 + o) * kc * N * 4;
                    for (int n = 0; n < N; ++n)
                        for (int kk = 0; kk < K; ++kk) {
                            // input kk: Re M_j (kk < H) or Im M_j; output n: Re b_l (n < H) or Im b_l
                            const int j = kk < H ? kk : kk - H, l = n < H ? n : n - H;
                            double val = 0.0;
                            const bool mono = j == 0 && l == 0;   // summed in float-float instead
                            if (j < p1 && l < p1 && !mono) {
                                const double tr = Tre[((size_t)d * p1 + j) * p1 + l];
                                const double ti = Tim[((size_t)d * p1 + j) * p1 + l];
                                if (n < H && kk < H) val = tr;
                                else if (n < H) val = -ti;
                                else if (kk < H) val = ti;
                                else val = tr;
                            }
                            const float v = (float)val;
                            const float h = host_tf32(v);
                            const size_t at = base + ((size_t)(kk / 4) * N + n) * 4 + (kk % 4);
                            hostops[0][at] = h;
                            if (np == 2) hostops[1][at] = v - h;
                        }
                }
            }
        for (int part = 0; part < np; ++part) {
            if (cudaMalloc(&tc->ops[part], opsz * 4) != cudaSuccess) return -1;
            pl->workspace_bytes += opsz * 4;
            if (cudaMemcpy(tc->ops[part], hostops[part].data(), opsz * 4, cudaMemcpyHostToDevice) != cudaSuccess)
                return -1;
            tc->args.ops[part] = tc->ops[part];
        }
    }
    // source buffers (chunk-major, 1-cell zero halo, kSrcPad zero cells after), levels kMinLevel..L
    for (int k = kMinLevel; k <= pl->levels; ++k) {
        const size_t w2p = ((size_t)1 << (k - 1)) + 2;
        const size_t bytes = ((size_t)4 * w2p * w2p * kc + kSrcPad) * 16;
        for (int part = 0; part < np; ++part) {
            if (cudaMalloc(&tc->src[part][k], bytes) != cudaSuccess) return -1;
            pl->workspace_bytes += bytes;
            if (cudaMemset(tc->src[part][k], 0, bytes) != cudaSuccess) return -1;
            tc->args.src[part][k] = reinterpret_cast<const float*>(tc->src[part][k]);
        }
    }
    return 0;
}

void fmm_tc_destroy(fmm_plan_s* pl) {
    FmmTc* tc = pl->tc;
    if (!tc) return;
    for (int part = 0; part < 2; ++part) {
        if (tc->ops[part]) cudaFree(tc->ops[part]);
        for (int k = 0; k <= FMM_MAX_LEVELS; ++k)
            if (tc->src[part][k]) cudaFree(tc->src[part][k]);
    }
    delete tc;
    pl->tc = nullptr;
}

template <int KC, int NP>
static int launch_tc_kc(fmm_plan_s* pl, const MixedLevels& lv) {
    FmmTc* tc = pl->tc;
    cudaStream_t st = pl->stream;
    const int L = pl->levels, p1 = pl->p + 1;
    {
        PrepArgs pa{};
        long long acc = 0;
        for (int k = kMinLevel; k <= L; ++k) {
            pa.a32[k] = reinterpret_cast<const float2*>(pl->grids.A32[k]);
            pa.hi[k] = tc->src[0][k];
            pa.lo[k] = tc->src[1][k];
            pa.base[k] = acc;
            acc += 4ll << (2 * (k - 1));
        }
        pa.base[L + 1] = acc;
        pa.kmin = kMinLevel;
        pa.levels = L;
        pa.p1 = p1;
        k_prep_tc<KC, NP><<<(unsigned)((acc + 255) / 256), 256, 0, st>>>(pa);
    }
    TcArgs& a = tc->args;
    for (int k = 0; k <= FMM_MAX_LEVELS; ++k) a.B[k] = reinterpret_cast<float2*>(pl->grids.B[k]);
    a.levels = L;
    a.p = pl->p;
    a.status = pl->d_status;
    // the tiles of a class, finest level first; rows per CTA so that the four classes fill the
    // SMs about once (at most kMaxRows: more tiles make more waves)
    int tiles = 0, nseg = 0;
    for (int k = L; k >= kMinLevel; --k) {
        a.seg_start[nseg] = tiles;
        a.seg_level[nseg] = k;
        ++nseg;
        tiles += tiles_of_level(k);
    }
    a.seg_start[nseg] = tiles;
    a.nseg = nseg;
    a.tiles = tiles;
    const int per_class_ctas = tc->sms / 4 > 0 ? tc->sms / 4 : 1;
    a.rows = (tiles + per_class_ctas - 1) / per_class_ctas;
    if (a.rows > kMaxRows) a.rows = kMaxRows;
    if (a.rows < 1) a.rows = 1;
    int cols = 32;
    while (cols < a.rows * 64) cols <<= 1;
    a.tmem_cols = cols;
    const int items = (tiles + a.rows - 1) / a.rows;
    constexpr int NSO = tc_nso<KC, NP>(), NSW = tc_nsw<KC, NP>();
    const size_t shm = tc_bytes<KC, NP>(NSO, NSW);
    auto kern = k_m2l_tc<KC, NP, NSO, NSW>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) != cudaSuccess) return -1;
    kern<<<4 * items, kThreads, shm, st>>>(a);
    {
        MonoArgs ma{};
        long long acc = 0;
        for (int k = kMinLevel; k <= L; ++k) {
            ma.a32[k] = reinterpret_cast<const float2*>(pl->grids.A32[k]);
            ma.B[k] = reinterpret_cast<float2*>(pl->grids.B[k]);
            ma.base[k] = acc;
            acc += 1ll << (2 * k);
        }
        ma.base[L + 1] = acc;
        memcpy(ma.logc, lv.logc, sizeof(ma.logc));
        ma.kmin = kMinLevel;
        ma.levels = L;
        ma.p1 = p1;
        k_m2l_mono<<<(unsigned)((acc + 255) / 256), 256, 0, st>>>(ma);
    }
    return 3;
}

// Launch prep + tensor-core M2L for levels 2..L; returns kernels launched or -1.
int fmm_launch_m2l_tc(fmm_plan_s* pl, const MixedLevels& lv) {
    const FmmTc* tc = pl->tc;
    if (!tc || pl->levels < kMinLevel) return 0;
    const bool x3 = tc->np == 2;
    switch (tc->kc) {
        case 4: return x3 ? launch_tc_kc<4, 2>(pl, lv) : launch_tc_kc<4, 1>(pl, lv);
        case 8: return x3 ? launch_tc_kc<8, 2>(pl, lv) : launch_tc_kc<8, 1>(pl, lv);
        case 12: return x3 ? launch_tc_kc<12, 2>(pl, lv) : launch_tc_kc<12, 1>(pl, lv);
        case 16: return x3 ? launch_tc_kc<16, 2>(pl, lv) : launch_tc_kc<16, 1>(pl, lv);
        default: return -1;
    }
}
