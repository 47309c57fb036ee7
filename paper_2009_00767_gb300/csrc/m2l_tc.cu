// m2l_tc.cu -- M2L (D-bar-1 of Sec. 2.2.1) on the 5th-generation tensor cores (tcgen05) for the
// levels from 6 down, in TF32 or BF16, unsplit or split (3xTF32, BF16x2, BF16x3), with FP32 accumulation
// in tensor memory.
//
// For one level k and one parity class c = (px, py) of target squares, the conversion of the
// interaction list is a real GEMM
//     D[t][n] = sum_d sum_kk  S[t + d][kk] * Op_d[n][kk]
// with t the targets, n the outputs (N = 2H: Re b'_0..b'_p then Im b'_0..b'_p, each padded to H)
// and kk the inputs (K = 2H per offset: Re M_0..M_p then Im M_0..M_p).  The 27 offsets of the
// class fall into 12 groups that share one source window: the source parity (qx, qy) and the
// source row shift sy.  The source grid of a parity is a (w2 + 2) x (w2 + 2) array with a 1-cell
// zero halo, stored chunk-major ([parity][K chunk][row][col][16 bytes]); read as one flat array
// of cells, a tile is 128 consecutive cells starting at flat position P and its window for shift
// sy the 130 cells from P - 1 + sy (w2 + 2): each K-chunk of it is one contiguous run of 2080
// bytes.  Rows of at least 128 targets take tiles aligned to the row; narrower sub-grids (levels
// below 8) take consecutive runs of the flat array, and the outputs that fall on halo cells are
// dropped.
//
// A CTA takes up to eight tiles of one class from any levels (the operators are scale-free) and
// one tensor-memory accumulator per tile.  Warp 0 streams the windows (one 2080-byte bulk copy per
// K chunk and part, issued by its lanes in parallel, up to NSW windows ahead) into the canonical
// no-swizzle K-major shared layout (16-byte core-matrix rows, K-chunk stride LBO = 130 x 16 B);
// warp 2 loads each group's operators, once for all the CTA's tiles; warp 1, converged, runs the
// issuing loop and one elected lane issues the MMAs (the three column shifts of a group read the
// same window through a descriptor start moved by 16 B per cell); all four warps run the epilogue,
// which reads the accumulators back with tcgen05.ld and stores them.  Every copy completes on its
// stage's mbarrier, and every wait on an mbarrier is bounded and sets a status flag when it runs
// out.
//
// Split products: 3xTF32 (Ootomo & Yokota, 2022) writes x = x_hi + x_lo with x_hi rounded to TF32
// and keeps A_hi B_hi + A_hi B_lo + A_lo B_hi, about FP32 accuracy; BF16x2 does the same with two
// BF16 parts (16 significant bits, the dropped lo lo term at 2^-16 of the product) at twice the
// TF32 rate; BF16x3 writes x = hi + mid + lo in BF16 and keeps the six products down to 2^-16.
//
// The monopole-log term of b'_0, sum_d M_0 (log|w0| + ln s), carries the largest part of phi; it
// stays out of the GEMM (its (0, 0) operator entry is zero): k_prep_tc sums it in float-float
// from the FP32 moment grid before the GEMM, in every mode, and the epilogue adds the GEMM's part
// to it; a TF32 or BF16 product of a large M_0 with the log would lose more than the error bound
// allows on clustered systems.

#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "mixed_common.cuh"

namespace {

constexpr int kTile = 128;        // targets per tile (MMA M)
constexpr int kWin = kTile + 2;   // source cells per window
constexpr int kThreads = 128;
constexpr int kMinLevel = 6;      // coarser levels stay on the CUDA cores (see fmm_tc_kmin)
constexpr int kMaxRows = 8;       // tiles per CTA at most (also bounded by the 512 tensor-memory columns)
constexpr int kSrcPad = 1024;     // cells after each source array: flat tiles past the last row read there
constexpr unsigned kSpin = 1u << 24;      // polls of a bounded wait (each poll may suspend briefly)
constexpr unsigned kTestSpin = 1u << 12;  // the error-path test's limit

struct TcGroup {
    int qx, qy, sy, nops, slot0;
    int sx[3];
    int d[3];
};

constexpr int kMaxParts = 3;     // split parts of an operand: TF32 x2 (hi, lo), BF16 x3 (hi, mid, lo)

// One segment = the grids of one level of one system (a plan has one system; a batch many).  The
// tiles of a class are the segments' tiles one after the other (the same list in every class):
// segment j owns tiles tile0 .. segs[j + 1].tile0 - 1, and the prep kernel's cells
// cell0 .. cell0 + 4 w2^2 - 1 (w2 = 2^(k-1), four parity sub-grids).
struct TcSeg {
    const float2* a32;                // FP32 moment grid of the level, (2^k + 6)^2 cells (3-cell halo)
    uint8_t* src[kMaxParts];          // split sources [q][KC][w2+2][w2+2][16 bytes] (1-cell zero halo)
    float2* B;                        // local coefficients of the level, (2^k)^2 cells
    long long cell0;                  // first prep cell
    int k;                            // level
    int tile0;                        // first tile
};

struct TcArgs {
    const TcSeg* segs;                // [nseg] in device memory, tile0 increasing
    // [class][27 slots][KC][NP * N rows][16 bytes], scale-free: within a K chunk the operator's parts
    // are stacked along N (rows part * N + n), so one MMA can take several parts at once
    const uint8_t* ops;
    TcGroup groups[4][12];
    // CTA b takes tiles c * rows .. of class b % 4, c = b / 4
    int nseg, tiles, rows, tmem_cols;
    int p;
    unsigned int* status;
    unsigned spin;    // polls of a bounded mbarrier wait before it gives up
    int stall;        // error-path test: the producers issue nothing, so the first wait runs out
};

// the segment holding item x (a tile or a prep cell) of an increasing start table: binary search
template <typename F>
__device__ __forceinline__ int find_seg(int nseg, long long x, F start) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start(mid) <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

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

__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, unsigned spin) {
    for (unsigned it = 0; it < spin; ++it) {
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

// One MMA, D (+)= A B^T (kind::f16 with BF16 operands, or kind::tf32), issued by the lane that
// elect.sync picks in a converged warp: the whole warp runs the issuing loop, so its descriptors
// stay warp-uniform values, and the leader (the lowest lane, the same one every time) issues.
template <bool BF>
__device__ __forceinline__ void mma_issue(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    if constexpr (BF)
        asm volatile(
            "{\n\t.reg .pred p, e;\n\t"
            "elect.sync _|e, 0xffffffff;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p, e;\n\t"
            "elect.sync _|e, 0xffffffff;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "@e tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
}

// tcgen05.commit by the elected lane (the one that issued the MMAs): the barrier's arrival
// tracks the completion of every MMA that lane has issued so far
__device__ __forceinline__ void commit_elect(uint32_t bar) {
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(bar)
        : "memory");
}

// The split products kept: TF32 x2 drops lo lo; BF16 x3 keeps every term down to 2^-16 of the
// product (hi hi, hi mid, mid hi, hi lo, lo hi, mid mid).  Products that share an A part go in one
// MMA over stacked B parts, whose columns land side by side in the accumulator (column block j
// holds the products with B part (first part + j)); the epilogue adds the blocks.  As (A part,
// first B part, B parts) in issue order, the widest first (it initialises every column block):
//   TF32 x2: (hi, hi, 2) = hi hi | hi lo, then (lo, hi, 1) = lo hi;
//   BF16 x3: (hi, hi, 2), (mid, hi, 2), (hi, lo, 1), (lo, hi, 1).
__device__ constexpr int kMmaA[4] = {0, 1, 0, 2};
__device__ constexpr int kMmaB[4] = {0, 0, 2, 0};
__host__ __device__ constexpr int num_mmas(int np) { return np == 1 ? 1 : (np == 2 ? 2 : 4); }
__host__ __device__ constexpr int mma_width(int np, int mm) {
    return np == 1 ? 1 : (np == 2 ? (mm == 0 ? 2 : 1) : (mm < 2 ? 2 : 1));
}
__host__ __device__ constexpr int stack_width(int np) { return np == 1 ? 1 : 2; }   // column blocks
// accumulator columns per tile: the stacked width rounded up to a multiple of 32
__host__ __device__ constexpr int acc_cols(int n, int np) { return (stack_width(np) * n + 31) / 32 * 32; }

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

// H: coefficients per real half, padded to a multiple of 8 (N = K per offset = 2H); BF: BF16
// operands (else TF32); NP: split parts per operand.
template <int H, bool BF, int NP, int NSO, int NSW>
__global__ void __launch_bounds__(kThreads, 1) k_m2l_tc(const __grid_constant__ TcArgs a) {
    constexpr int N = 2 * H;
    constexpr int KC = BF ? H / 4 : H / 2;           // 16-byte K chunks per offset
    constexpr uint32_t A_BYTES = KC * kWin * 16;     // one window, one part
    constexpr uint32_t ROWS = NP * N;                // stacked operator rows per K chunk
    constexpr uint32_t OP_BYTES = KC * ROWS * 16;    // one offset's operator, all parts
    constexpr uint32_t OPS_STAGE = 3 * OP_BYTES;
    constexpr uint32_t WIN_STAGE = NP * A_BYTES;
    constexpr uint32_t ACC_COLS = acc_cols(N, NP);   // per tile
    constexpr uint32_t FMT = BF ? 1u : 2u;           // operand format: BF16 (kind::f16) or TF32
    constexpr uint32_t IDESC_BASE = (1u << 4) | (FMT << 7) | (FMT << 10) | ((128u >> 4) << 24);
    constexpr int NMMA = num_mmas(NP);
    static_assert(stack_width(NP) * N <= 256 && N % 16 == 0, "MMA N of 16..256 in steps of 16");
    static_assert(KC % 2 == 0 && NP * KC <= 32, "an MMA takes two K chunks; one producer lane per chunk");

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
    // [kMaxRows][kMaxParts + 1]: each tile's source arrays and its level's local grid
    uint8_t** tile_ptr = reinterpret_cast<uint8_t**>(((uintptr_t)(tile_P + kMaxRows) + 7) & ~(uintptr_t)7);
    static_assert(8 * (2 * NSO + 2 * NSW + 1) + 4 + 8 * kMaxRows + 8 + 8 * kMaxRows * (kMaxParts + 1) <= 512,
                  "barriers and tile tables fit the 512 bytes tc_bytes reserves");

    // ---- which tiles
    const int cls = blockIdx.x & 3;
    const int t0 = (blockIdx.x >> 2) * a.rows;
    const int nrows = min(a.rows, a.tiles - t0);
    const int px = cls & 1, py = cls >> 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < nrows) {
        const int tau = t0 + threadIdx.x;
        const TcSeg& S = a.segs[find_seg(a.nseg, tau, [&](int j) { return (long long)a.segs[j].tile0; })];
        const int k = S.k;
        tile_k[threadIdx.x] = k;
        tile_P[threadIdx.x] = tile_start(1 << (k - 1), tau - S.tile0);
#pragma unroll
        for (int part = 0; part < kMaxParts; ++part) tile_ptr[threadIdx.x * (kMaxParts + 1) + part] = S.src[part];
        tile_ptr[threadIdx.x * (kMaxParts + 1) + kMaxParts] = reinterpret_cast<uint8_t*>(S.B);
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
    if (warp == 2) {
        // operator producer: each group's operators (its offsets are consecutive slots) as soon
        // as the stage's previous group has been consumed; lane 0 posts the byte count, then the
        // lanes copy 16-byte-aligned slices in parallel
        int posted = 0;   // groups whose copies were issued
        for (int g = 0; g < 12 && !a.stall; ++g) {
            const TcGroup& G = a.groups[cls][g];
            const int so = g % NSO, uso = g / NSO;
            const uint32_t bytes = (uint32_t)G.nops * OP_BYTES;
            if (lane == 0) {
                // a stage's arrival is posted only together with its copies
                if (g >= NSO && !wait_bar(su32(&ops_empty[so]), (uint32_t)((uso - 1) & 1), a.spin))
                    ok = false;
                else
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                                     su32(&ops_full[so])),
                                 "r"(bytes)
                                 : "memory");
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            posted = g + 1;
            const uint32_t units = bytes / 16u, per = (units + 31u) / 32u;
            const uint32_t u0 = min(units, (uint32_t)lane * per), u1 = min(units, u0 + per);
            if (u1 > u0) {
                const uint8_t* srcB = a.ops + ((size_t)cls * 27 + G.slot0) * OP_BYTES + (size_t)u0 * 16u;
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        su32(ops_buf + so * OPS_STAGE + u0 * 16u)),
                    "l"(srcB), "r"((u1 - u0) * 16u), "r"(su32(&ops_full[so]))
                    : "memory");
            }
        }
        // before the CTA may exit: every copy issued has landed (each stage's last posted phase
        // completes only after its earlier ones)
        if (lane == 0)
            for (int g = posted - NSO > 0 ? posted - NSO : 0; g < posted; ++g)
                if (!wait_bar(su32(&ops_full[g % NSO]), (uint32_t)((g / NSO) & 1), a.spin)) ok = false;
        ok = __shfl_sync(0xffffffffu, ok, 0);
    } else if (warp == 0) {
        // window producer: lane 0 waits for a free stage and posts its byte count, then the lanes
        // issue the window's bulk copies in parallel (one K chunk of one part each); every copy
        // completes on the stage's full barrier, so the producer runs ahead of the MMAs
        int posted = 0;   // windows whose copies were issued
        for (int i = 0; i < NWIN && !a.stall; ++i) {
            const int g = i / nrows, t = i % nrows;
            const TcGroup& G = a.groups[cls][g];
            const int sw = i % NSW, usw = i / NSW;
            if (lane == 0) {
                if (i >= NSW && !wait_bar(su32(&win_empty[sw]), (uint32_t)((usw - 1) & 1), a.spin))
                    ok = false;
                else
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                                     su32(&win_full[sw])),
                                 "r"((uint32_t)(NP * A_BYTES))
                                 : "memory");
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            posted = i + 1;
            if (lane < NP * KC) {
                // chunk j of part `part` of the 130 cells from the window's flat start: 2080
                // contiguous bytes (past a chunk's end it reads the next chunk or the zero pad,
                // which only feed dropped outputs)
                const int part = lane / KC, j = lane % KC;
                const int q = G.qx + 2 * G.qy;
                const int k = tile_k[t];
                const size_t W2P = ((size_t)1 << (k - 1)) + 2;
                const size_t start = (size_t)(tile_P[t] - 1 + G.sy * (int)W2P);   // flat, >= 0
                const uint8_t* src = tile_ptr[t * (kMaxParts + 1) + part] + (((size_t)q * KC + j) * W2P * W2P + start) * 16;
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        su32(win_buf + sw * WIN_STAGE + part * A_BYTES + j * (kWin * 16))),
                    "l"(src), "r"((uint32_t)(kWin * 16)), "r"(su32(&win_full[sw]))
                    : "memory");
            }
        }
        if (lane == 0)
            for (int i = posted - NSW > 0 ? posted - NSW : 0; i < posted; ++i)
                if (!wait_bar(su32(&win_full[i % NSW]), (uint32_t)((i / NSW) & 1), a.spin)) ok = false;
        ok = __shfl_sync(0xffffffffu, ok, 0);
    } else if (warp == 1) {
        // MMA issuer: the whole warp runs the loop (waits, descriptors) in step, one elected lane
        // issues the MMAs and commits
        for (int i = 0; i < NWIN; ++i) {
            const int g = i / nrows, t = i % nrows;
            const TcGroup& G = a.groups[cls][g];
            const int so = g % NSO, uso = g / NSO;
            const int sw = i % NSW, usw = i / NSW;
            if (t == 0 && !wait_bar(su32(&ops_full[so]), (uint32_t)(uso & 1), a.spin)) ok = false;
            if (ok && !wait_bar(su32(&win_full[sw]), (uint32_t)(usw & 1), a.spin)) ok = false;
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;   // nothing more is issued; the producers' own waits then run out
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // descriptors: the window's and the group's base descriptors once, then constant
            // offsets in 16-byte units on the start-address field (shared addresses stay below
            // 2^18 bytes, so the 14-bit field never carries)
            const uint64_t aDesc = smem_desc(su32(win_buf + sw * WIN_STAGE), kWin * 16, 128);
            const uint64_t bDesc = smem_desc(su32(ops_buf + so * OPS_STAGE), ROWS * 16, 128);
            const uint32_t acc_t = tmem + (uint32_t)t * ACC_COLS;
            const int nops = G.nops;
            for (int o = 0; o < nops; ++o) {
                const uint64_t ad0 = aDesc + (uint64_t)(1 + G.sx[o]);   // column shift: one 16-byte cell
                const uint64_t bd0 = bDesc + (uint64_t)(o * (OP_BYTES / 16));
                const uint32_t acc0 = (g | o) != 0;
#pragma unroll
                for (int ks = 0; ks < KC / 2; ++ks) {
#pragma unroll
                    for (int mm = 0; mm < NMMA; ++mm) {
                        const uint64_t ad = ad0 + (uint64_t)((kMmaA[mm] * A_BYTES + ks * 2 * (kWin * 16)) / 16);
                        const uint64_t bd = bd0 + (uint64_t)((kMmaB[mm] * N * 16 + ks * 2 * (ROWS * 16)) / 16);
                        const uint32_t width = (uint32_t)mma_width(NP, mm);
                        mma_issue<BF>(acc_t, ad, bd, IDESC_BASE | ((width * N) >> 3) << 17,
                                      (ks | mm) != 0 ? 1u : acc0);
                    }
                }
            }
            commit_elect(su32(&win_empty[sw]));
            if (t == nrows - 1) commit_elect(su32(&ops_empty[so]));
        }
        // the final commit tracks every MMA issued above (it arrives at once if none was)
        commit_elect(su32(done_bar));
        __syncwarp();
    }
    // warp w holds accumulator rows (targets) 32w..32w+31 of every tile: each thread's targets,
    // and the monopole-log part of their Re b'_0 that k_prep_tc left in B, loaded while the MMAs
    // run (kept in registers: the tile loops are unrolled over kMaxRows)
    const int p1 = a.p + 1;
    float2* bt[kMaxRows];
    float2 b0[kMaxRows];
#pragma unroll
    for (int t = 0; t < kMaxRows; ++t) {
        bt[t] = nullptr;
        b0[t] = make_float2(0.f, 0.f);
        if (t < nrows) {
            const int k = tile_k[t];
            const int w2 = 1 << (k - 1), W2P = w2 + 2;
            const int pos = tile_P[t] + 32 * warp + lane;
            const int x = pos % W2P - 1, y = pos / W2P - 1;   // sub-grid cell; halo cells are dropped
            if (x >= 0 && x < w2 && y < w2) {
                bt[t] = reinterpret_cast<float2*>(tile_ptr[t * (kMaxParts + 1) + kMaxParts]) +
                        ((size_t)(2 * y + py) * (1u << k) + (2 * x + px)) * p1;
                b0[t] = bt[t][0];
            }
        }
    }
    // Every issued copy has landed (the producers waited for them); the MMAs are done once
    // done_bar completes.  If any wait of the CTA ran out, nothing is read back or stored.
    const bool done = wait_bar(su32(done_bar), 0, a.spin);
    const bool fail = __syncthreads_or(!ok || !done) != 0;
    if (fail && threadIdx.x == 0) atomicOr(a.status, FMM_FLAG_TIMEOUT);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // ---- epilogue: each thread's target row (p + 1 complex values, slot 0 the float-float Re b'_0)
    // goes through a per-warp staging area in the window buffers (idle once the MMAs are done), then
    // each row is stored by the lanes over its coefficients: 168 contiguous bytes per store at p = 20
    // instead of one row per thread at a stride of two cells
    const int RS = 2 * p1 + 1;   // staging row stride in floats (odd: no bank conflicts on the row writes)
    static_assert((size_t)(kThreads / 32) * 32 * (2 * H + 1) * 4 <= (size_t)NSW * WIN_STAGE,
                  "the epilogue's staging rows fit the window buffers");
    float* stage = reinterpret_cast<float*>(win_buf) + (size_t)warp * 32 * RS;
#pragma unroll
    for (int t = 0; t < kMaxRows; ++t) {
        if (t >= nrows || fail) break;
        constexpr int SW = stack_width(NP);
        float v[SW * N];
#pragma unroll
        for (int c = 0; c < SW * N; c += 16)
            tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(t * ACC_COLS + c), v + c);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (SW == 2) {
#pragma unroll
            for (int c = 0; c < N; ++c) v[c] += v[N + c];   // the column blocks of the stacked products
        }
        float* row = stage + lane * RS;
        const float2 r0 = ff_add_f(b0[t], v[0]);   // Re b'_0: the GEMM's part added to the monopole-log term
        row[0] = r0.x;
        row[1] = r0.y;
#pragma unroll
        for (int l = 1; l < H; ++l)
            if (l < p1) {
                row[2 * l] = v[l];
                row[2 * l + 1] = v[H + l];
            }
        __syncwarp();
        const unsigned long long mine = reinterpret_cast<unsigned long long>(bt[t]);
        for (int r = 0; r < 32; ++r) {
            float2* B = reinterpret_cast<float2*>(__shfl_sync(0xffffffffu, mine, r));
            if (B != nullptr && lane < p1) B[lane] = make_float2(stage[r * RS + 2 * lane], stage[r * RS + 2 * lane + 1]);
        }
        __syncwarp();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        // MMAs still in flight after a wait that ran out: one more bounded wait before the
        // tensor memory they write is freed
        if (fail) wait_bar(su32(done_bar), 0, a.spin);
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ uint32_t bf16_rn_bits(float x) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
}

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

struct PrepArgs {
    const TcSeg* segs;
    int nseg;
    long long cells;                      // cells of all segments
    float2 logc[FMM_MAX_LEVELS + 1][49];
    int p1;
};

// FP32 moment grid (3-cell halo) -> the GEMM's source layout, one thread per cell of a parity
// sub-grid: out[part][q][KC][w2][w2][16 bytes] with the K index Re M_0..M_p, pad, Im M_0..M_p,
// pad, each value split into NP parts: TF32 x2 hi = rna(x), lo = x - hi; BF16 x3 hi = rn(x),
// mid = rn(x - hi), lo = rn(x - hi - mid) (each difference exact in FP32).
// The same thread, as the target square of that cell, also writes the monopole-log term of b'_0,
// sum_d M_0[t + d] (log|w0_d| + ln s_k) over its interaction list, summed in float-float (in the
// order dy, then dx, the 27 loads issued together) into B's slot 0, where the tensor-core kernel's
// epilogue adds the GEMM's part: it stays out of the GEMM (its operator entry (0, 0) is zero), as
// a TF32 or BF16 product of a large M_0 with the log would lose more than the error bound allows.
template <int H, bool BF, int NP>
__global__ void k_prep_tc(const __grid_constant__ PrepArgs a) {
    constexpr int KC = BF ? H / 4 : H / 2, PER = BF ? 8 : 4;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.cells) return;
    const TcSeg& S = a.segs[find_seg(a.nseg, g, [&](int j) { return a.segs[j].cell0; })];
    const int k = S.k;
    const int64_t e = g - S.cell0;
    const int w2 = 1 << (k - 1), W2P = w2 + 2, p1 = a.p1;
    const int col = (int)(e % w2), row = (int)((e / w2) % w2), q = (int)(e / ((int64_t)w2 * w2));
    const int x = 2 * col + (q & 1), y = 2 * row + (q >> 1);
    const int W = fmm_grid_width(k);
    const float2* src = S.a32 + ((size_t)(y + FMM_HALO) * W + (x + FMM_HALO)) * p1;
    float vals[2 * H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
        const float2 m = (j < p1) ? src[j] : make_float2(0.f, 0.f);
        vals[j] = m.x;                     // coefficient 0 holds M_0's high word: M_0 is real
        vals[H + j] = (j == 0) ? 0.f : m.y;
    }
    // chunk-major source layout [q][chunk][row][col] (1-cell zero halo): the chunk of a run of
    // consecutive cells of the flat array is one contiguous block
    const size_t cell = (size_t)(row + 1) * W2P + (size_t)(col + 1);
#pragma unroll
    for (int c = 0; c < KC; ++c) {
        uint32_t w[NP][4];
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            float r = vals[PER * c + t];
#pragma unroll
            for (int part = 0; part < NP; ++part) {
                if constexpr (BF) {
                    const uint32_t b = bf16_rn_bits(r);
                    r -= __uint_as_float(b << 16);
                    if (t & 1) w[part][t >> 1] |= b << 16;
                    else w[part][t >> 1] = b;
                } else {
                    const float h = (part + 1 < NP || NP == 1) ? tf32_rna(r) : r;   // x2: lo stays FP32
                    r -= h;
                    w[part][t] = __float_as_uint(h);
                }
            }
        }
        const size_t at = ((size_t)q * KC + c) * (size_t)W2P * W2P + cell;
#pragma unroll
        for (int part = 0; part < NP; ++part)
            reinterpret_cast<uint4*>(S.src[part])[at] = make_uint4(w[part][0], w[part][1], w[part][2], w[part][3]);
    }
    const size_t c0 = (size_t)(y + FMM_HALO) * W + (x + FMM_HALO);
    float2 mono;
    switch (q) {
        case 0: mono = mono_sum<0, 0>(S.a32, a.logc[k], c0, W, p1); break;
        case 1: mono = mono_sum<1, 0>(S.a32, a.logc[k], c0, W, p1); break;
        case 2: mono = mono_sum<0, 1>(S.a32, a.logc[k], c0, W, p1); break;
        default: mono = mono_sum<1, 1>(S.a32, a.logc[k], c0, W, p1); break;
    }
    S.B[((size_t)y * (1u << k) + x) * p1] = mono;   // Re b'_0 as float-float, the GEMM's part to come
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

// host-side round to nearest even BF16 (finite inputs), returned as its 16 bits
uint16_t host_bf16_bits(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
float bf16_bits_to_float(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

// shared-memory plan: two operator stages and as many window stages (2 to 5) as fit, else one
// operator stage and two window stages; 128 bytes of alignment slack and 512 bytes of barriers
// and per-tile tables
template <int H, bool BF, int NP>
constexpr size_t tc_bytes(int nso, int nsw) {
    constexpr int KC = BF ? H / 4 : H / 2;
    return (size_t)nso * NP * 3 * (KC * (2 * H) * 16) + (size_t)nsw * NP * (KC * kWin * 16) + 128 + 512;
}
template <int H, bool BF, int NP>
constexpr int tc_nso() {
    return tc_bytes<H, BF, NP>(2, 2) <= 227 * 1024 ? 2 : 1;
}
template <int H, bool BF, int NP>
constexpr int tc_nsw() {
    static_assert(tc_bytes<H, BF, NP>(1, 2) <= 227 * 1024, "two window stages must fit");
    constexpr int nso = tc_nso<H, BF, NP>();
    // five window stages where they fit (BF16x2 at p <= 23: 177 KB): a window ring one stage deeper
    // than four cut the issuing loop's waits (59.4 -> 57.3 us at 2^20 particles, levels 8, p = 20);
    // a sixth stage gained nothing more
    return tc_bytes<H, BF, NP>(nso, 5) <= 227 * 1024
               ? 5
               : (tc_bytes<H, BF, NP>(nso, 4) <= 227 * 1024 ? 4 : (tc_bytes<H, BF, NP>(nso, 3) <= 227 * 1024 ? 3 : 2));
}

}  // namespace

// ---------------------------------------------------------------- plan-side state
struct FmmTc {
    int h, kc, np, sms, p, precision;
    bool bf;                       // BF16 operands (else TF32)
    uint8_t* ops;                  // one scale-free copy, the parts stacked
    uint8_t* src_all;              // every segment's split source arrays
    TcSeg* d_segs;                 // the segment table in device memory
    std::vector<TcSeg> segs;       // host copy
    long long cells;               // prep cells of all segments
    TcArgs args;                   // tables, filled at plan time
};

// The tensor cores take levels kMinLevel and finer.  The coarse levels carry most of the far
// field's amplitude, and the tensor core's FP32 accumulation (product alignment and rounding inside
// each MMA) loses more there than FP32 FMAs; they hold few targets, so the CUDA cores take them.
int fmm_tc_kmin() { return kMinLevel; }

bool fmm_tc_precision(int precision) {
    return precision == FMM_MIXED_TF32 || precision == FMM_MIXED_3XTF32 || precision == FMM_MIXED_BF16 ||
           precision == FMM_MIXED_BF16X2 || precision == FMM_MIXED_BF16X3;
}

void fmm_tc_free(FmmTc* tc) {
    if (!tc) return;
    if (tc->ops) cudaFree(tc->ops);
    if (tc->src_all) cudaFree(tc->src_all);
    if (tc->d_segs) cudaFree(tc->d_segs);
    delete tc;
}

// The operators and class tables of a tensor-core precision (TF32, 3xTF32, BF16, BF16x2 or BF16x3)
// at order p, from the FP64 operators Tre/Tim ([49][p+1][p+1]).  *err: 0, -1 (CUDA error) or -2
// (unsupported p); *bytes grows by the device memory taken.
FmmTc* fmm_tc_new(int p, int precision, const std::vector<double>& Tre, const std::vector<double>& Tim, int* err,
                  uint64_t* bytes) {
    *err = 0;
    const int p1 = p + 1;
    const int H = ((p1 + 7) / 8) * 8;
    if (!fmm_tc_precision(precision) || (H != 8 && H != 16 && H != 24 && H != 32)) {
        *err = -2;
        return nullptr;
    }
    const bool bf = precision == FMM_MIXED_BF16 || precision == FMM_MIXED_BF16X2 || precision == FMM_MIXED_BF16X3;
    const int kc = bf ? H / 4 : H / 2;
    const int per = bf ? 8 : 4, elem = bf ? 2 : 4;
    const int np = (precision == FMM_MIXED_3XTF32 || precision == FMM_MIXED_BF16X2)
                       ? 2
                       : (precision == FMM_MIXED_BF16X3 ? 3 : 1);
    FmmTc* tc = new FmmTc();
    tc->h = H;
    tc->kc = kc;
    tc->np = np;
    tc->bf = bf;
    tc->p = p;
    tc->precision = precision;
    tc->ops = nullptr;
    tc->src_all = nullptr;
    tc->d_segs = nullptr;
    tc->cells = 0;
    memset(&tc->args, 0, sizeof(TcArgs));
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&tc->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        *err = -1;
        fmm_tc_free(tc);
        return nullptr;
    }
    const int N = 2 * H, K = 2 * H;

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
        if (slots[cls] != 27) {
            *err = -1;
            fmm_tc_free(tc);
            return nullptr;
        }
    }
    // operators, real block form, [part][class][slot][KC][N][16 bytes]: scale-free, so one copy
    // serves every level; the monopole-log entry (0, 0) is left out (summed in float-float by
    // k_prep_tc).  Each value is split into np parts as the sources are (TF32 x2: hi, FP32 lo;
    // BF16 x3: hi, mid, lo, the differences taken in FP64).
    const size_t opsz = (size_t)4 * 27 * kc * np * N * 16;   // bytes, all parts
    {
        std::vector<uint8_t> hostops(opsz, 0);
        for (int cls = 0; cls < 4; ++cls)
            for (int g = 0; g < 12; ++g) {
                const TcGroup& G = tc->args.groups[cls][g];
                for (int o = 0; o < G.nops; ++o) {
                    const int d = G.d[o];
                    const size_t base = ((size_t)cls * 27 + G.slot0 + o) * kc * np * N * 16;
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
                            // row part * N + n of K chunk kk / per
                            const size_t at0 = base + (size_t)(kk / per) * np * N * 16 + (size_t)n * 16 +
                                               (size_t)(kk % per) * elem;
                            if (bf) {
                                double r = val;
                                for (int part = 0; part < np; ++part) {
                                    const uint16_t b = host_bf16_bits((float)r);
                                    r -= (double)bf16_bits_to_float(b);
                                    memcpy(&hostops[at0 + (size_t)part * N * 16], &b, 2);
                                }
                            } else {
                                const float v = (float)val;
                                const float h = host_tf32(v);
                                const float parts[2] = {h, v - h};
                                for (int part = 0; part < np; ++part)
                                    memcpy(&hostops[at0 + (size_t)part * N * 16], &parts[part], 4);
                            }
                        }
                }
            }
        if (cudaMalloc(&tc->ops, opsz) != cudaSuccess ||
            cudaMemcpy(tc->ops, hostops.data(), opsz, cudaMemcpyHostToDevice) != cudaSuccess) {
            *err = -1;
            fmm_tc_free(tc);
            return nullptr;
        }
        *bytes += opsz;
        tc->args.ops = tc->ops;
    }
    tc->args.p = p;
    return tc;
}

// The levels the tensor cores convert, one segment each (kMinLevel <= k): their FP32 moment grids
// and local grids.  Allocates the split source arrays (chunk-major, 1-cell zero halo, kSrcPad zero
// cells after each: flat tiles past a sub-grid's last row read there) and uploads the segment
// table.  Returns 0 or -1.
int fmm_tc_set_levels(FmmTc* tc, const std::vector<FmmTcLevel>& levels, uint64_t* bytes) {
    tc->segs.clear();
    size_t total = 0;
    std::vector<size_t> part_bytes;
    for (const FmmTcLevel& L : levels) {
        if (L.k < kMinLevel || L.k > FMM_MAX_LEVELS) return -1;
        const size_t w2p = ((size_t)1 << (L.k - 1)) + 2;
        part_bytes.push_back(((size_t)4 * w2p * w2p * tc->kc + kSrcPad) * 16);
        total += part_bytes.back() * tc->np;
    }
    if (total > 0) {
        if (cudaMalloc(&tc->src_all, total) != cudaSuccess || cudaMemset(tc->src_all, 0, total) != cudaSuccess)
            return -1;
        *bytes += total;
    }
    size_t off = 0;
    long long cells = 0;
    int tiles = 0;
    for (size_t i = 0; i < levels.size(); ++i) {
        TcSeg S;
        memset(&S, 0, sizeof(S));
        S.a32 = levels[i].a32;
        S.B = levels[i].B;
        S.k = levels[i].k;
        for (int part = 0; part < tc->np; ++part) {
            S.src[part] = tc->src_all + off;
            off += part_bytes[i];
        }
        S.cell0 = cells;
        S.tile0 = tiles;
        cells += 4ll << (2 * (S.k - 1));
        tiles += tiles_of_level(S.k);
        tc->segs.push_back(S);
    }
    tc->cells = cells;
    tc->args.nseg = (int)tc->segs.size();
    tc->args.tiles = tiles;
    if (!tc->segs.empty()) {
        if (cudaMalloc(&tc->d_segs, sizeof(TcSeg) * tc->segs.size()) != cudaSuccess ||
            cudaMemcpy(tc->d_segs, tc->segs.data(), sizeof(TcSeg) * tc->segs.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess)
            return -1;
        *bytes += sizeof(TcSeg) * tc->segs.size();
    }
    tc->args.segs = tc->d_segs;
    return 0;
}

namespace {

template <int H, bool BF, int NP>
int launch_tc(FmmTc* tc, const MixedLevels& lv, cudaStream_t st, unsigned int* status, int stall, int rows_max,
              cudaEvent_t e0, cudaEvent_t e1) {
    if (tc->args.nseg == 0) return 0;
    {
        PrepArgs pa;
        memset(&pa, 0, sizeof(pa));
        pa.segs = tc->d_segs;
        pa.nseg = tc->args.nseg;
        pa.cells = tc->cells;
        pa.p1 = tc->p + 1;
        memcpy(pa.logc, lv.logc, sizeof(pa.logc));
        k_prep_tc<H, BF, NP><<<(unsigned)((tc->cells + 255) / 256), 256, 0, st>>>(pa);
    }
    TcArgs& a = tc->args;
    a.status = status;
    a.spin = stall ? kTestSpin : kSpin;
    a.stall = stall;
    // rows (tiles) per CTA so that the four classes fill the SMs about once (at most kMaxRows or
    // rows_max: more tiles make more waves)
    const int per_class_ctas = tc->sms / 4 > 0 ? tc->sms / 4 : 1;
    constexpr int ACC = acc_cols(2 * H, NP);
    int max_rows = 512 / ACC < kMaxRows ? 512 / ACC : kMaxRows;   // accumulators fit tensor memory
    if (rows_max > 0 && rows_max < max_rows) max_rows = rows_max;
    a.rows = (a.tiles + per_class_ctas - 1) / per_class_ctas;
    if (a.rows > max_rows) a.rows = max_rows;
    if (a.rows < 1) a.rows = 1;
    int cols = 32;
    while (cols < a.rows * ACC) cols <<= 1;
    a.tmem_cols = cols;
    const int items = (a.tiles + a.rows - 1) / a.rows;
    constexpr int NSO = tc_nso<H, BF, NP>(), NSW = tc_nsw<H, BF, NP>();
    const size_t shm = tc_bytes<H, BF, NP>(NSO, NSW);
    auto kern = k_m2l_tc<H, BF, NP, NSO, NSW>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) != cudaSuccess) return -1;
    if (e0) cudaEventRecord(e0, st);
    kern<<<4 * items, kThreads, shm, st>>>(a);
    if (e1) cudaEventRecord(e1, st);
    return cudaGetLastError() == cudaSuccess ? 2 : -1;
}

}  // namespace

// Prep + tensor-core M2L of every segment on stream st; returns the kernels launched or -1.
// rows_max (> 0) caps the tiles per CTA (an autotuned shape; 0: the default).
int fmm_tc_enqueue(FmmTc* tc, const MixedLevels& lv, cudaStream_t st, unsigned int* status, int stall, int rows_max,
                   cudaEvent_t e0, cudaEvent_t e1) {
    if (!tc) return 0;
#define FMM_TC_CASES(H)                                                                                     \
    case H:                                                                                                 \
        if (tc->bf)                                                                                         \
            return tc->np == 3 ? launch_tc<H, true, 3>(tc, lv, st, status, stall, rows_max, e0, e1)         \
                               : (tc->np == 2 ? launch_tc<H, true, 2>(tc, lv, st, status, stall, rows_max, e0, e1) \
                                              : launch_tc<H, true, 1>(tc, lv, st, status, stall, rows_max, e0, e1)); \
        return tc->np == 2 ? launch_tc<H, false, 2>(tc, lv, st, status, stall, rows_max, e0, e1)           \
                           : launch_tc<H, false, 1>(tc, lv, st, status, stall, rows_max, e0, e1);
    switch (tc->h) {
        FMM_TC_CASES(8)
        FMM_TC_CASES(16)
        FMM_TC_CASES(24)
        FMM_TC_CASES(32)
        default: return -1;
    }
#undef FMM_TC_CASES
}

// ---------------------------------------------------------------- the single-system plan
// Allocate and build the tensor-core M2L state for the plan's precision, its levels kMinLevel..L
// finest first.  Returns 0, or a negative value on failure (-1 CUDA error, -2 unsupported p).
int fmm_tc_create(fmm_plan_s* pl, const std::vector<double>& Tre, const std::vector<double>& Tim) {
    int err = 0;
    uint64_t bytes = 0;
    FmmTc* tc = fmm_tc_new(pl->p, pl->precision, Tre, Tim, &err, &bytes);
    pl->workspace_bytes += bytes;
    if (!tc) return err;
    pl->tc = tc;
    std::vector<FmmTcLevel> lev;
    for (int k = pl->levels; k >= kMinLevel; --k)
        lev.push_back({reinterpret_cast<const float2*>(pl->grids.A32[k]), reinterpret_cast<float2*>(pl->grids.B[k]), k});
    bytes = 0;
    const int r = fmm_tc_set_levels(tc, lev, &bytes);
    pl->workspace_bytes += bytes;
    return r;
}

void fmm_tc_destroy(fmm_plan_s* pl) {
    fmm_tc_free(pl->tc);
    pl->tc = nullptr;
}

// Launch prep + tensor-core M2L for levels kMinLevel..L; returns kernels launched or -1.
int fmm_launch_m2l_tc(fmm_plan_s* pl, const MixedLevels& lv) {
    if (!pl->tc || pl->levels < kMinLevel) return 0;
    const int r = fmm_tc_enqueue(pl->tc, lv, pl->stream, pl->d_status, pl->test_stall, 0, pl->ev[6], pl->ev[7]);
    if (r > 0) pl->ev_kernels |= 1;
    return r;
}
