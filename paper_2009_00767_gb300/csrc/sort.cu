// sort.cu -- binning of the particles into the finest squares and the box-sorted copy.
//
// The tree is the uniform quadtree of Sec. 2.1 items 1-4: the square [0, box]^2 at level 0,
// each level-k square split into four at level k+1, down to `levels`.  A particle's finest
// square is (floor(x 2^l / box), floor(y 2^l / box)) in FP64, clamped to [0, 2^l - 1]; its
// level-k square is the finest one shifted right by l - k.  Keys are Morton-interleaved, so
// after a counting sort the particles of any square at any level form one contiguous range.
//
// Stages (HBM-bound gathers and scatters):
//   k_bin      key + rank-in-square (atomic histogram) + device-side input checks
//   k_scan_*   exclusive scan of the 4^l square populations -> CSR leaf_start
//   k_scatter  box-sorted copy (FP64 absolute, or FP32 relative to the square centre)
#include "fmm_internal.cuh"

namespace {

constexpr int kScanThreads = 256;

constexpr int kScanItems = 2;   // small tiles: 128 blocks for 4^8 squares, each with little serial work
constexpr int kScanTile = kScanThreads * kScanItems;

// particles [i0, n)
__global__ void k_bin(const double2* __restrict__ xy, const double* __restrict__ q, int64_t i0, int64_t n, int levels,
                      double box, float scale_over_box32, uint32_t* __restrict__ keys, uint32_t* __restrict__ rank,
                      uint32_t* __restrict__ counts, unsigned int* __restrict__ status) {
    int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 p = xy[i];
    double qq = q[i];
    const double scale = (double)(1 << levels);
    const int side = 1 << levels;
    uint32_t key = 0;
    if (!(finite_bits(p.x) && finite_bits(p.y) && finite_bits(qq))) {
        atomicOr(status, FMM_FLAG_NONFINITE);
    } else {
        const long long bb = __double_as_longlong(box);
        if (!(in_box_bits(p.x, bb) && in_box_bits(p.y, bb))) atomicOr(status, FMM_FLAG_OUT_OF_BOX);
        const int ix = finest_coord(p.x, scale, scale_over_box32, box, side);
        const int iy = finest_coord(p.y, scale, scale_over_box32, box, side);
        key = fmm_morton((uint32_t)ix, (uint32_t)iy);
    }
    keys[i] = key;
    rank[i] = atomicAdd(&counts[key], 1u);
}

// block-wide exclusive scan of kScanItems values per thread; returns the block total
template <typename T>
__device__ T block_exclusive_scan(T (&v)[kScanItems], T* warp_tot) {
    T s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) { T t = v[j]; v[j] = s; s += t; }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < (kScanThreads / 32) ? warp_tot[lane] : T(0);
        T wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < (kScanThreads / 32)) warp_tot[lane] = wi - w;   // exclusive warp offsets
        if (lane == (kScanThreads / 32) - 1) warp_tot[kScanThreads / 32] = wi;
    }
    __syncthreads();
    T base = warp_tot[warp] + inc - s;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) v[j] += base;
    T total = warp_tot[kScanThreads / 32];
    __syncthreads();
    return total;
}

__global__ void k_scan_reduce(const uint32_t* __restrict__ in, int64_t m, uint32_t* __restrict__ sums) {
    __shared__ uint32_t wt[kScanThreads / 32 + 1];
    uint32_t v[kScanItems];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) v[j] = (base + j < m) ? in[base + j] : 0u;
    uint32_t tot = block_exclusive_scan(v, wt);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_top(uint32_t* __restrict__ sums, int nb) {
    // one block of kScanThreads scans up to kScanTile block sums; larger counts loop in tiles
    __shared__ uint32_t wt[kScanThreads / 32 + 1];
    uint32_t carry = 0;
    for (int t0 = 0; t0 < nb; t0 += kScanTile) {
        uint32_t v[kScanItems];
        int base = t0 + threadIdx.x * kScanItems;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) v[j] = (base + j < nb) ? sums[base + j] : 0u;
        uint32_t tot = block_exclusive_scan(v, wt);
#pragma unroll
        for (int j = 0; j < kScanItems; ++j)
            if (base + j < nb) sums[base + j] = v[j] + carry;
        carry += tot;
    }
    if (threadIdx.x == 0) sums[nb] = carry;   // the grand total, for scans whose total is not known
}

__global__ void k_scan_down(const uint32_t* __restrict__ in, int64_t m, const uint32_t* __restrict__ sums,
                            uint32_t* __restrict__ out, uint32_t n_total) {
    __shared__ uint32_t wt[kScanThreads / 32 + 1];
    uint32_t v[kScanItems];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) v[j] = (base + j < m) ? in[base + j] : 0u;
    block_exclusive_scan(v, wt);
    uint32_t off = sums[blockIdx.x];
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
        if (base + j < m) out[base + j] = v[j] + off;
    if (blockIdx.x == 0 && threadIdx.x == 0) out[m] = (n_total == 0xffffffffu) ? sums[gridDim.x] : n_total;
}

// Mixed path: one scan of (population, near-field blocks) pairs packed in 64 bits (the low word
// never carries: n < 2^32) gives leaf_start and the block starts at once; the down-sweep also
// writes the block -> (square, block inside it) map and zeroes the populations it has read.
__device__ __forceinline__ unsigned long long pop_blocks(uint32_t c) {
    return (unsigned long long)c | ((unsigned long long)((c + FMM_P2P_BLOCK - 1u) / FMM_P2P_BLOCK) << 32);
}

__global__ void k_scan2_reduce(const uint32_t* __restrict__ in, int64_t m, unsigned long long* __restrict__ sums) {
    __shared__ unsigned long long wt[kScanThreads / 32 + 1];
    unsigned long long v[kScanItems];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) v[j] = (base + j < m) ? pop_blocks(in[base + j]) : 0ull;
    unsigned long long tot = block_exclusive_scan(v, wt);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan2_top(unsigned long long* __restrict__ sums, int nb) {
    __shared__ unsigned long long wt[kScanThreads / 32 + 1];
    unsigned long long carry = 0;
    for (int t0 = 0; t0 < nb; t0 += kScanTile) {
        unsigned long long v[kScanItems];
        int base = t0 + threadIdx.x * kScanItems;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) v[j] = (base + j < nb) ? sums[base + j] : 0ull;
        unsigned long long tot = block_exclusive_scan(v, wt);
#pragma unroll
        for (int j = 0; j < kScanItems; ++j)
            if (base + j < nb) sums[base + j] = v[j] + carry;
        carry += tot;
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

// sum over the CTA's threads (every thread gets it)
__device__ unsigned long long block_sum_u64(unsigned long long x, unsigned long long* wt) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) wt[warp] = x;
    __syncthreads();
    unsigned long long t = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) t += wt[w];
    __syncthreads();
    return t;
}

// few scan blocks (at most kLocalTopMax): each CTA of the down-sweep sums the partials before it
// itself, which spares the separate top-level pass
constexpr int kLocalTopMax = 1024;

template <bool kLocalTop>
__global__ void k_scan2_down(uint32_t* __restrict__ in, int64_t m, const unsigned long long* __restrict__ sums,
                             uint32_t* __restrict__ leaf_start, uint32_t* __restrict__ bstart,
                             uint2* __restrict__ map, int* __restrict__ crowd_hint) {
    __shared__ unsigned long long wt[kScanThreads / 32 + 1];
    unsigned long long v[kScanItems];
    uint32_t nbk[kScanItems];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    bool crowded = false;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = (base + j < m) ? pop_blocks(in[base + j]) : 0ull;
        nbk[j] = (uint32_t)(v[j] >> 32);
        crowded |= (uint32_t)v[j] > (uint32_t)FMM_LANE_MAX;
        if (base + j < m) in[base + j] = 0u;   // the populations start the next call at zero
    }
    if (crowded && crowd_hint) *(volatile int*)crowd_hint = 1;
    block_exclusive_scan(v, wt);
    unsigned long long off;
    if (kLocalTop) {
        unsigned long long part = 0;
        for (int b = threadIdx.x; b < (int)blockIdx.x; b += kScanThreads) part += sums[b];
        off = block_sum_u64(part, wt);
    } else {
        off = sums[blockIdx.x];
    }
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
        if (base + j < m) {
            const unsigned long long e = v[j] + off;
            const uint32_t b0 = (uint32_t)(e >> 32);
            leaf_start[base + j] = (uint32_t)e;
            bstart[base + j] = b0;
            for (uint32_t b = 0; b < nbk[j]; ++b) map[b0 + b] = make_uint2((uint32_t)(base + j), b);
        }
    if (blockIdx.x == gridDim.x - 1) {
        unsigned long long tot;
        if (kLocalTop) {
            // this CTA's offset plus its own partial
            tot = off + sums[blockIdx.x];
        } else {
            tot = sums[gridDim.x];
        }
        if (threadIdx.x == 0) {
            leaf_start[m] = (uint32_t)tot;
            bstart[m] = (uint32_t)(tot >> 32);
        }
    }
}

template <bool kMixed>
__global__ void k_scatter(const double2* __restrict__ xy, const double* __restrict__ q, int64_t n, int levels,
                          float2 s_ff, const uint32_t* __restrict__ keys, const uint32_t* __restrict__ rank,
                          const uint32_t* __restrict__ leaf_start, uint32_t* __restrict__ sorted_key,
                          fmm_p64* __restrict__ s64, float4* __restrict__ s32, float2* __restrict__ s32_lo) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t key = keys[i];
    uint32_t pos = leaf_start[key] + rank[i];
    double2 p = xy[i];
    double qq = q[i];
    sorted_key[pos] = key;
    if (kMixed) {
        // coordinates relative to the finest-square centre (ix + 1/2) s, formed in float-float
        // (s = box / 2^l as an FP32 pair), so FP32 keeps about 1e-7 of the square side
        const float2 cx = scatter_mul((float)fmm_compact2(key) + 0.5f, s_ff);
        const float2 cy = scatter_mul((float)fmm_compact2(key >> 1) + 0.5f, s_ff);
        const float2 xf = fmm_d2ff_bits(p.x), yf = fmm_d2ff_bits(p.y), qf = fmm_d2ff_bits(qq);
        const float hx = xf.x - cx.x, hy = yf.x - cy.x;   // exact: the high words are close
        const float lx = xf.y - cx.y, ly = yf.y - cy.y;
        const float dx = hx + lx, dy = hy + ly;
        s32[pos] = make_float4(dx, dy, qf.x + qf.y, __int_as_float((int)i));
        // the rounding residue of the local coordinates, for the field's near pairs (TwoSum)
        if (s32_lo) s32_lo[pos] = make_float2(two_sum_err(hx, lx, dx), two_sum_err(hy, ly, dy));
    } else {
        s64[pos] = fmm_p64{p.x, p.y, qq, (double)i};
    }
}

}  // namespace

// Bin particles [i0, i1) on stream s (key, rank in its square, device checks); the populations
// must start at zero.
int fmm_launch_bin_range(fmm_plan_s* pl, const double* xy, const double* q, int64_t i0, int64_t i1, cudaStream_t s) {
    if (i1 <= i0) return 0;
    const int tb = 256;
    const unsigned nblk = (unsigned)((i1 - i0 + tb - 1) / tb);
    const float scale_over_box32 = (float)((double)(1 << pl->levels) / pl->box);
    k_bin<<<nblk, tb, 0, s>>>(reinterpret_cast<const double2*>(xy), q, i0, i1, pl->levels, pl->box, scale_over_box32,
                              pl->keys, pl->rank, pl->counts, pl->d_status);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int fmm_launch_sort(fmm_plan_s* pl, const double* xy, const double* q, bool with_lo, bool binned) {
    const int64_t n = pl->n;
    const int64_t m = (int64_t)1 << (2 * pl->levels);
    cudaStream_t st = pl->stream;
    int launches = 0;
    const int tb = 256;
    const unsigned nblk = (unsigned)((n + tb - 1) / tb);
    if (!binned) {
        // the mixed path's scan returns counts to zero for the next call
        if (pl->precision == FMM_FP64 && cudaMemsetAsync(pl->counts, 0, sizeof(uint32_t) * m, st) != cudaSuccess)
            return -1;
        if (fmm_launch_bin_range(pl, xy, q, 0, n, st) < 0) return -1;
        ++launches;
    }
    const int nb = pl->scan_blocks;
    if (pl->precision == FMM_FP64) {
        k_scan_reduce<<<nb, kScanThreads, 0, st>>>(pl->counts, m, pl->block_sums);
        k_scan_top<<<1, kScanThreads, 0, st>>>(pl->block_sums, nb);
        k_scan_down<<<nb, kScanThreads, 0, st>>>(pl->counts, m, pl->block_sums, pl->leaf_start, (uint32_t)n);
    } else {
        // the near-field blocks come with the same scan (block_sums holds 64-bit partials here)
        unsigned long long* sums = reinterpret_cast<unsigned long long*>(pl->block_sums);
        k_scan2_reduce<<<nb, kScanThreads, 0, st>>>(pl->counts, m, sums);
        if (nb <= kLocalTopMax) {
            k_scan2_down<true><<<nb, kScanThreads, 0, st>>>(pl->counts, m, sums, pl->leaf_start, pl->leaf_bstart,
                                                            pl->blk_map, pl->crowd_hint_d);
            launches -= 1;
        } else {
            k_scan2_top<<<1, kScanThreads, 0, st>>>(sums, nb);
            k_scan2_down<false><<<nb, kScanThreads, 0, st>>>(pl->counts, m, sums, pl->leaf_start, pl->leaf_bstart,
                                                             pl->blk_map, pl->crowd_hint_d);
        }
    }
    launches += 3;
    const double sd = pl->box / (double)(1 << pl->levels);
    const float s_hi = (float)sd;
    const float2 s_ff = make_float2(s_hi, (float)(sd - (double)s_hi));
    if (pl->precision == FMM_FP64)
        k_scatter<false><<<nblk, tb, 0, st>>>(reinterpret_cast<const double2*>(xy), q, n, pl->levels, s_ff,
                                              pl->keys, pl->rank, pl->leaf_start, pl->sorted_key, pl->sorted64,
                                              pl->sorted32, nullptr);
    else
        k_scatter<true><<<nblk, tb, 0, st>>>(reinterpret_cast<const double2*>(xy), q, n, pl->levels, s_ff,
                                             pl->keys, pl->rank, pl->leaf_start, pl->sorted_key, pl->sorted64,
                                             pl->sorted32, with_lo ? pl->sorted_lo : nullptr);
    ++launches;
    if (cudaGetLastError() != cudaSuccess) return -1;
    return launches;
}

int fmm_scan_blocks(int64_t m) { return (int)((m + kScanTile - 1) / kScanTile); }

// target blocks of up to `block` particles per finest square, for the near-field work split
__global__ void k_leaf_blocks(const uint32_t* __restrict__ leaf_start, int64_t m, uint32_t block,
                              uint32_t* __restrict__ nb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) nb[i] = (leaf_start[i + 1] - leaf_start[i] + block - 1u) / block;
}

// block -> (square, block index inside the square), one thread per square
__global__ void k_block_map(const uint32_t* __restrict__ bstart, int64_t m, uint2* __restrict__ map) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const uint32_t b0 = bstart[i], b1 = bstart[i + 1];
    for (uint32_t b = b0; b < b1; ++b) map[b] = make_uint2((uint32_t)i, b - b0);
}

int fmm_launch_scan(const uint32_t* counts, int64_t m, uint32_t* block_sums, uint32_t* leaf_start, uint32_t n_total,
                    cudaStream_t st) {
    const int nb = fmm_scan_blocks(m);
    k_scan_reduce<<<nb, kScanThreads, 0, st>>>(counts, m, block_sums);
    k_scan_top<<<1, kScanThreads, 0, st>>>(block_sums, nb);
    k_scan_down<<<nb, kScanThreads, 0, st>>>(counts, m, block_sums, leaf_start, n_total);
    return cudaGetLastError() == cudaSuccess ? 3 : -1;
}

int fmm_launch_leaf_blocks(const uint32_t* leaf_start, int64_t m, uint32_t block, uint32_t* nb, uint32_t* block_sums,
                           uint32_t* bstart, uint2* map, cudaStream_t st) {
    const unsigned g = (unsigned)((m + 255) / 256);
    k_leaf_blocks<<<g, 256, 0, st>>>(leaf_start, m, block, nb);
    const int r = fmm_launch_scan(nb, m, block_sums, bstart, 0xffffffffu, st);
    if (r < 0) return -1;
    if (map == nullptr) return r + 1;
    k_block_map<<<g, 256, 0, st>>>(bstart, m, map);
    return cudaGetLastError() == cudaSuccess ? r + 2 : -1;
}
