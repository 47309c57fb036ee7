// p2p_block.cuh -- the near field (E-2 of Sec. 2.1) of one block of targets, shared by the
// single-system kernel (mixed.cu) and the batched one (batch.cu).
#pragma once

#include "mixed_common.cuh"

namespace {

// Near field (E-2 of Sec. 2.1): every particle of a finest square against the particles of that
// square and its (up to) eight neighbours, in FP32 on square-local coordinates.
//
// One warp takes a block of up to 24 targets of one finest square.  The lanes walk the sources 32
// at a time (the own square's first, then the neighbours'), each lane holding one source moved into the target square's
// frame, and keep one FP32 partial sum per target in registers; the targets' coordinates are
// shared-memory broadcasts, two targets per load.  The arithmetic of two targets runs in packed
// FP32x2 instructions, so a pair costs one lg2 on the MUFU unit and two to three FP32 slots.
// Coincidence (r^2 = 0: the target itself, duplicate points) only arises within the own square,
// whose chunks test r^2 > 0; a neighbour's pair adds 2^-100 to r^2 instead, which keeps the
// logarithm finite should two particles of adjacent squares round to the same FP32 point and
// changes no other pair.  After each run of kP2PRun chunks the partials of each target are
// combined across the warp by a shuffle reduce-scatter (lane t ends with target t's sum) and
// added in float-float, so crowded squares keep their accuracy.
constexpr int kP2PRun = 16;   // chunks of 32 sources summed in FP32 before the float-float add

__device__ __forceinline__ float mufu_lg2(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// 1 / x on the MUFU unit (within one ulp)
__device__ __forceinline__ float mufu_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Sum of v[l & (W - 1)] over the warp's lanes, returned in lane l (v[t] = p[t / 2].x or .y for
// t < 2 NP, 0 beyond).  The low log2(W) lane bits scatter (at the step with mask m a lane keeps
// the half of its live entries whose bit m matches its own and sends the other half to its
// partner), the remaining bits add by butterfly.
template <int W, int NP>
__device__ __forceinline__ float warp_reduce_scatter(const float2 (&p)[NP], int lane) {
    float v[W];
#pragma unroll
    for (int i = 0; i < W; ++i) v[i] = i < 2 * NP ? ((i & 1) ? p[i >> 1].y : p[i >> 1].x) : 0.f;
#pragma unroll
    for (int m = W / 2; m >= 1; m >>= 1) {
        const bool up = (lane & m) != 0;
#pragma unroll
        for (int i = 0; i < m; ++i) {
            const float send = up ? v[i] : v[i + m];
            const float keep = up ? v[i + m] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
        }
    }
    float s = v[0];
#pragma unroll
    for (int m = W; m < 32; m <<= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    return s;
}

// one chunk: the lane's source (sx, sy, q) against the NP target pairs of the block (the
// coordinates of targets past the block's end are zero and their sums are dropped)
template <bool kOwn, int NP>
__device__ __forceinline__ void p2p_chunk(float2 (&part)[NP], const float4* __restrict__ tg, float4 src) {
    const float2 nsx = make_float2(-src.x, -src.x), nsy = make_float2(-src.y, -src.y);
    const float2 q2 = make_float2(src.z, src.z);
    const float2 tiny = make_float2(0x1p-100f, 0x1p-100f);
#pragma unroll
    for (int tp = 0; tp < NP; ++tp) {
        const float4 t = tg[tp];   // {x of target 2tp, x of 2tp + 1, y of 2tp, y of 2tp + 1}
        const float2 dx = __fadd2_rn(make_float2(t.x, t.y), nsx);
        const float2 dy = __fadd2_rn(make_float2(t.z, t.w), nsy);
        float2 r2, lg;
        if (kOwn) {
            r2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
            lg = make_float2(mufu_lg2(r2.x), mufu_lg2(r2.y));
            lg.x = r2.x > 0.f ? lg.x : 0.f;
            lg.y = r2.y > 0.f ? lg.y : 0.f;
        } else {
            r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, tiny));
            lg = make_float2(mufu_lg2(r2.x), mufu_lg2(r2.y));
        }
        part[tp] = __ffma2_rn(q2, lg, part[tp]);
    }
}

// The block's sources: the own square's particles [t0, t0 + n_own) in nch_own chunks, then the
// eight neighbours' in slot order (seg: sorted index minus slot and the frame shift per
// neighbour, thr: first slot of neighbours 1..7).
struct P2PSources {
    const float4* sp;
    const int4* seg;
    uint32_t thr[7];
    uint32_t t0, n_own, nch_own, n_nb;

    // source of chunk c for this lane, in the target square's frame; slots past a part's end
    // carry q = 0
    __device__ __forceinline__ float4 load(uint32_t c, int lane) const {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c < nch_own) {
            const uint32_t s = 32u * c + (uint32_t)lane;
            if (s < n_own) v = sp[t0 + s];
        } else {
            const uint32_t s = 32u * (c - nch_own) + (uint32_t)lane;
            if (s < n_nb) {
                int b = 0;
#pragma unroll
                for (int i = 0; i < 7; ++i) b += s >= thr[i] ? 1 : 0;
                const int4 g = seg[b];
                v = sp[s + (uint32_t)g.x];
                v.x += __int_as_float(g.y);
                v.y += __int_as_float(g.z);
            }
        }
        return v;
    }
};

// the near-field sum (log2 r^2 units, float-float) of target `lane` of a block of at most 2 NP
// targets
template <int NP>
__device__ __forceinline__ float2 p2p_block(const P2PSources& S, const float4* __restrict__ tg, int lane) {
    constexpr int W = NP <= 2 ? 4 : (NP <= 4 ? 8 : (NP <= 8 ? 16 : 32));
    const uint32_t nch = S.nch_own + (S.n_nb + 31u) / 32u;
    float2 near = make_float2(0.f, 0.f);
    for (uint32_t r0 = 0; r0 < nch; r0 += kP2PRun) {
        const uint32_t r1 = min(nch, r0 + (uint32_t)kP2PRun);
        float2 part[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) part[i] = make_float2(0.f, 0.f);
        // the next chunk's loads are in flight while one is summed (a deeper ring, unrolled, made
        // the kernel's code outgrow the instruction cache)
        float4 cur = S.load(r0, lane);
        for (uint32_t c = r0; c < r1; ++c) {
            const float4 nxt = (c + 1 < r1) ? S.load(c + 1, lane) : cur;
            if (c < S.nch_own)
                p2p_chunk<true, NP>(part, tg, cur);
            else
                p2p_chunk<false, NP>(part, tg, cur);
            cur = nxt;
        }
        near = ff_add_f(near, warp_reduce_scatter<W, NP>(part, lane));
    }
    return near;
}

// Neighbour b = (dx + 1) + 3 (dy + 1) of finest square `leaf` (lane b < 9, b != 4; other lanes
// and squares outside the domain give an empty range): its first sorted particle and count.
__device__ __forceinline__ uint2 p2p_neighbour(const uint32_t* __restrict__ ls, uint32_t leaf, int levels, int lane) {
    uint32_t first = 0, cnt = 0;
    if (lane < 9 && lane != 4) {
        const int side = 1 << levels;
        const int jx = (int)fmm_compact2(leaf) + lane % 3 - 1, jy = (int)fmm_compact2(leaf >> 1) + lane / 3 - 1;
        if (jx >= 0 && jy >= 0 && jx < side && jy < side) {
            const uint32_t nl = fmm_morton((uint32_t)jx, (uint32_t)jy);
            first = ls[nl];
            cnt = ls[nl + 1] - first;
        }
    }
    return make_uint2(first, cnt);
}

// The near field of the targets [b0, b0 + T) (T <= 24) of a finest square with particles
// [t0, t1), whose neighbours' ranges nb came from p2p_neighbour; s_leaf is the square's side.
// Returns target `lane`'s sum in log2 r^2 units as a float-float pair and the block's source
// count in *nsrc.  tgt (16 float4) and seg (8 int4) are the warp's shared memory.
__device__ __forceinline__ float2 p2p_near_nb(const float4* __restrict__ sp, uint32_t t0, uint32_t t1, uint32_t b0,
                                              int T, uint2 nb, float s_leaf, float4* tgt, int4* seg, int lane,
                                              uint32_t* nsrc) {
    const uint32_t n_own = t1 - t0;
    // the eight neighbours' sources take consecutive slots of the neighbour chunks
    const uint32_t first = nb.x, cnt = nb.y;
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t excl = incl - cnt;
    const uint32_t n_nb = __shfl_sync(0xffffffffu, incl, 8);
    if (lane < 9 && lane != 4)
        seg[lane - (lane > 4)] = make_int4((int)(first - excl), __float_as_int((float)(lane % 3 - 1) * s_leaf),
                                           __float_as_int((float)(lane / 3 - 1) * s_leaf), 0);
    P2PSources S;
    S.sp = sp;
    S.seg = seg;
#pragma unroll
    for (int i = 1; i < 8; ++i) S.thr[i - 1] = __shfl_sync(0xffffffffu, excl, i + (i >= 4));
    S.t0 = t0;
    S.n_own = n_own;
    S.nch_own = (n_own + 31u) / 32u;
    S.n_nb = n_nb;
    *nsrc = n_own + n_nb;
    {
        float x = 0.f, y = 0.f;
        if (lane < T) {
            const float4 P = sp[b0 + lane];
            x = P.x;
            y = P.y;
        }
        float* t = reinterpret_cast<float*>(&tgt[lane >> 1]);
        t[lane & 1] = x;
        t[2 + (lane & 1)] = y;
    }
    __syncwarp();
    // the block's target pairs, rounded up to an even count, fix the unrolled width
    switch ((T + 3) >> 2) {
        case 1: return p2p_block<2>(S, tgt, lane);
        case 2: return p2p_block<4>(S, tgt, lane);
        case 3: return p2p_block<6>(S, tgt, lane);
        case 4: return p2p_block<8>(S, tgt, lane);
        case 5: return p2p_block<10>(S, tgt, lane);
        default: return p2p_block<12>(S, tgt, lane);
    }
}

// p2p_near_nb with the neighbours looked up first (square `leaf` of a quadtree of depth `levels`
// whose CSR over the sorted array is ls)
__device__ __forceinline__ float2 p2p_near(const float4* __restrict__ sp, const uint32_t* __restrict__ ls,
                                           uint32_t leaf, uint32_t t0, uint32_t t1, uint32_t b0, int T, int levels,
                                           float s_leaf, float4* tgt, int4* seg, int lane, uint32_t* nsrc) {
    return p2p_near_nb(sp, t0, t1, b0, T, p2p_neighbour(ls, leaf, levels, lane), s_leaf, tgt, seg, lane, nsrc);
}

// ---------------------------------------------------------------- symmetric near field
// The pair term log r^2 is symmetric, so each pair of adjacent squares is evaluated once: the
// block's targets take their own square in full (both orders, as above) and only the four
// "forward" neighbours E (+1, 0), NE (+1, +1), N (0, +1) and NW (-1, +1); the other four
// neighbours are covered by the squares that have this one as their forward neighbour.  For a
// forward pair the logarithm serves both sides: q_s L goes to the target (register partials, as
// above) and q_t L to the source, summed over the block's targets in the lane that holds the
// source and added to the source's accumulator with one FP64 atomic per lane and chunk.

// Forward neighbour `lane` (< 4: E, NE, N, NW) of finest square `leaf`: its first sorted particle
// and count (an empty range outside the domain and on the other lanes).
__device__ __forceinline__ uint2 p2p_forward(const uint32_t* __restrict__ ls, uint32_t leaf, int levels, int lane) {
    uint32_t first = 0, cnt = 0;
    if (lane < 4) {
        const int side = 1 << levels;
        const int jx = (int)fmm_compact2(leaf) + (lane == 3 ? -1 : (lane == 2 ? 0 : 1));
        const int jy = (int)fmm_compact2(leaf >> 1) + (lane == 0 ? 0 : 1);
        if (jx >= 0 && jy >= 0 && jx < side && jy < side) {
            const uint32_t nl = fmm_morton((uint32_t)jx, (uint32_t)jy);
            first = ls[nl];
            cnt = ls[nl + 1] - first;
        }
    }
    return make_uint2(first, cnt);
}

// The block's sources: the own square's particles [t0, t0 + n_own) in nch_own chunks, then the
// four forward neighbours' in lane order (seg[b]: sorted index minus slot, frame shift; thr:
// first slot of forward neighbours 1..3).
struct P2PSymSources {
    const float4* sp;
    const int4* seg;
    uint32_t thr[3];
    uint32_t t0, n_own, nch_own, n_fw;

    // source of chunk c for this lane in the target square's frame, and for a forward chunk its
    // sorted index (0xffffffff past the end, where q = 0)
    __device__ __forceinline__ float4 load(uint32_t c, int lane, uint32_t* idx) const {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        *idx = 0xffffffffu;
        if (c < nch_own) {
            const uint32_t s = 32u * c + (uint32_t)lane;
            if (s < n_own) v = sp[t0 + s];
        } else {
            const uint32_t s = 32u * (c - nch_own) + (uint32_t)lane;
            if (s < n_fw) {
                const int b = (s >= thr[0] ? 1 : 0) + (s >= thr[1] ? 1 : 0) + (s >= thr[2] ? 1 : 0);
                const int4 g = seg[b];
                *idx = s + (uint32_t)g.x;
                v = sp[*idx];
                v.x += __int_as_float(g.y);
                v.y += __int_as_float(g.z);
            }
        }
        return v;
    }
};

// one forward chunk: the lane's source against the NP target pairs, both sides; returns the
// source's sum over the block's targets (targets past the block's end have q = 0)
template <int NP>
__device__ __forceinline__ float p2p_chunk_sym(float2 (&part)[NP], const float4* __restrict__ tg,
                                               const float2* __restrict__ tq, float4 src) {
    const float2 nsx = make_float2(-src.x, -src.x), nsy = make_float2(-src.y, -src.y);
    const float2 q2 = make_float2(src.z, src.z);
    const float2 tiny = make_float2(0x1p-100f, 0x1p-100f);
    float2 sacc = make_float2(0.f, 0.f);
#pragma unroll
    for (int tp = 0; tp < NP; ++tp) {
        const float4 t = tg[tp];
        const float2 dx = __fadd2_rn(make_float2(t.x, t.y), nsx);
        const float2 dy = __fadd2_rn(make_float2(t.z, t.w), nsy);
        const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, tiny));
        const float2 lg = make_float2(mufu_lg2(r2.x), mufu_lg2(r2.y));
        part[tp] = __ffma2_rn(q2, lg, part[tp]);
        sacc = __ffma2_rn(tq[tp], lg, sacc);
    }
    return sacc.x + sacc.y;
}

// the block's own-square and forward-neighbour sums: returns target `lane`'s sum (log2 r^2 units,
// float-float) and adds each forward source's sum to acc[its sorted index]
template <int NP>
__device__ __forceinline__ float2 p2p_block_sym(const P2PSymSources& S, const float4* __restrict__ tg,
                                                const float2* __restrict__ tq, int lane, double* __restrict__ acc) {
    constexpr int W = NP <= 2 ? 4 : (NP <= 4 ? 8 : (NP <= 8 ? 16 : 32));
    const uint32_t nch = S.nch_own + (S.n_fw + 31u) / 32u;
    float2 near = make_float2(0.f, 0.f);
    for (uint32_t r0 = 0; r0 < nch; r0 += kP2PRun) {
        const uint32_t r1 = min(nch, r0 + (uint32_t)kP2PRun);
        float2 part[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) part[i] = make_float2(0.f, 0.f);
        uint32_t idx;
        float4 cur = S.load(r0, lane, &idx);
        for (uint32_t c = r0; c < r1; ++c) {
            uint32_t nidx = idx;
            const float4 nxt = (c + 1 < r1) ? S.load(c + 1, lane, &nidx) : cur;
            if (c < S.nch_own) {
                p2p_chunk<true, NP>(part, tg, cur);
            } else {
                const float ssum = p2p_chunk_sym<NP>(part, tg, tq, cur);
                if (idx != 0xffffffffu) atomicAdd(acc + idx, fmm_f2d_bits(ssum));
            }
            cur = nxt;
            idx = nidx;
        }
        near = ff_add_f(near, warp_reduce_scatter<W, NP>(part, lane));
    }
    return near;
}

// Symmetric near field of the targets [b0, b0 + T) (T <= 24) of finest square `leaf` with
// particles [t0, t1): target `lane`'s own-square and forward sum (log2 r^2 units, float-float) is
// returned, the forward sources' shares go to acc.  *pairs receives the ordered pairs covered
// (both directions of every forward pair).  tgt (16 float4), tq (16 float2) and seg (4 int4) are
// the warp's shared memory.
__device__ __forceinline__ float2 p2p_near_sym(const float4* __restrict__ sp, const uint32_t* __restrict__ ls,
                                               uint32_t leaf, uint32_t t0, uint32_t t1, uint32_t b0, int T,
                                               int levels, float s_leaf, float4* tgt, float2* tq, int4* seg,
                                               int lane, double* __restrict__ acc, uint32_t* pairs) {
    const uint2 nb = p2p_forward(ls, leaf, levels, lane);
    const uint32_t n_own = t1 - t0;
    uint32_t incl = nb.y;
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t excl = incl - nb.y;
    const uint32_t n_fw = __shfl_sync(0xffffffffu, incl, 3);
    if (lane < 4) {
        const float ox = (float)(lane == 3 ? -1 : (lane == 2 ? 0 : 1)) * s_leaf;
        const float oy = (float)(lane == 0 ? 0 : 1) * s_leaf;
        seg[lane] = make_int4((int)(nb.x - excl), __float_as_int(ox), __float_as_int(oy), 0);
    }
    P2PSymSources S;
    S.sp = sp;
    S.seg = seg;
#pragma unroll
    for (int i = 0; i < 3; ++i) S.thr[i] = __shfl_sync(0xffffffffu, excl, i + 1);
    S.t0 = t0;
    S.n_own = n_own;
    S.nch_own = (n_own + 31u) / 32u;
    S.n_fw = n_fw;
    *pairs = (uint32_t)T * (n_own + 2u * n_fw) - (uint32_t)T;
    {
        float x = 0.f, y = 0.f, q = 0.f;
        if (lane < T) {
            const float4 P = sp[b0 + lane];
            x = P.x;
            y = P.y;
            q = P.z;
        }
        float* t = reinterpret_cast<float*>(&tgt[lane >> 1]);
        t[lane & 1] = x;
        t[2 + (lane & 1)] = y;
        reinterpret_cast<float*>(&tq[lane >> 1])[lane & 1] = q;
    }
    __syncwarp();
    switch ((T + 3) >> 2) {
        case 1: return p2p_block_sym<2>(S, tgt, tq, lane, acc);
        case 2: return p2p_block_sym<4>(S, tgt, tq, lane, acc);
        case 3: return p2p_block_sym<6>(S, tgt, tq, lane, acc);
        case 4: return p2p_block_sym<8>(S, tgt, tq, lane, acc);
        case 5: return p2p_block_sym<10>(S, tgt, tq, lane, acc);
        default: return p2p_block_sym<12>(S, tgt, tq, lane, acc);
    }
}

// ---------------------------------------------------------------- near field with the field
// The same symmetric scheme with grad phi beside phi: a pair adds q_s log2 r^2 to the target's
// phi and q_s (dx, dy) / r^2 to its gradient (dx, dy = target - source), and for a forward pair q_t
// log2 r^2 and -q_t (dx, dy) / r^2 to the source's; 1 / r^2 comes from the MUFU reciprocal.  A
// coincident own-square pair (r^2 = 0) gives 0 to both.  The field of a close pair goes as 1 / r,
// so FP32 square-local coordinates alone (about 1e-9 of the box) would limit it; each coordinate
// also carries its FP32 rounding residue (written by the sort for field calls), and a pair's
// difference takes the high words (exact for close pairs) plus the residues' difference.
struct NearField {
    float2 phi, gx, gy;   // float-float sums of target `lane`
};

template <bool kOwn, int NP>
__device__ __forceinline__ float3 p2p_chunk_field(float2 (&pp)[NP], float2 (&px)[NP], float2 (&py)[NP],
                                                  const float4* __restrict__ tg, const float4* __restrict__ tl,
                                                  const float2* __restrict__ tq, float4 src, float2 slo) {
    const float2 nsx = make_float2(-src.x, -src.x), nsy = make_float2(-src.y, -src.y);
    const float2 nlx = make_float2(-slo.x, -slo.x), nly = make_float2(-slo.y, -slo.y);
    const float2 q2 = make_float2(src.z, src.z);
    const float2 tiny = make_float2(0x1p-100f, 0x1p-100f);
    float2 sp = make_float2(0.f, 0.f), sx = make_float2(0.f, 0.f), sy = make_float2(0.f, 0.f);
#pragma unroll
    for (int tp = 0; tp < NP; ++tp) {
        const float4 t = tg[tp], u = tl[tp];
        // the coordinates' high words differ exactly for close pairs; the low words carry the rest
        const float2 dx = __fadd2_rn(__fadd2_rn(make_float2(t.x, t.y), nsx), __fadd2_rn(make_float2(u.x, u.y), nlx));
        const float2 dy = __fadd2_rn(__fadd2_rn(make_float2(t.z, t.w), nsy), __fadd2_rn(make_float2(u.z, u.w), nly));
        float2 r2, lg, iv;
        if (kOwn) {
            r2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
            lg = make_float2(mufu_lg2(r2.x), mufu_lg2(r2.y));
            iv = make_float2(mufu_rcp(r2.x), mufu_rcp(r2.y));
            lg.x = r2.x > 0.f ? lg.x : 0.f;
            lg.y = r2.y > 0.f ? lg.y : 0.f;
            iv.x = r2.x > 0.f ? iv.x : 0.f;
            iv.y = r2.y > 0.f ? iv.y : 0.f;
        } else {
            r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, tiny));
            lg = make_float2(mufu_lg2(r2.x), mufu_lg2(r2.y));
            iv = make_float2(mufu_rcp(r2.x), mufu_rcp(r2.y));
        }
        const float2 wx = __fmul2_rn(dx, iv), wy = __fmul2_rn(dy, iv);   // (dx, dy) / r^2
        pp[tp] = __ffma2_rn(q2, lg, pp[tp]);
        px[tp] = __ffma2_rn(q2, wx, px[tp]);
        py[tp] = __ffma2_rn(q2, wy, py[tp]);
        if (!kOwn) {
            const float2 qt = tq[tp];
            sp = __ffma2_rn(qt, lg, sp);
            sx = __ffma2_rn(qt, wx, sx);
            sy = __ffma2_rn(qt, wy, sy);
        }
    }
    return make_float3(sp.x + sp.y, -(sx.x + sx.y), -(sy.x + sy.y));   // the source's phi and gradient
}

// the source of chunk c with its coordinates' low words (frame shift by TwoSum), for the field
__device__ __forceinline__ float4 load_lo(const P2PSymSources& S, const float2* __restrict__ lo, uint32_t c, int lane,
                                          uint32_t* idx, float2* vlo) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    *vlo = make_float2(0.f, 0.f);
    *idx = 0xffffffffu;
    if (c < S.nch_own) {
        const uint32_t s = 32u * c + (uint32_t)lane;
        if (s < S.n_own) {
            v = S.sp[S.t0 + s];
            *vlo = lo[S.t0 + s];
        }
    } else {
        const uint32_t s = 32u * (c - S.nch_own) + (uint32_t)lane;
        if (s < S.n_fw) {
            const int b = (s >= S.thr[0] ? 1 : 0) + (s >= S.thr[1] ? 1 : 0) + (s >= S.thr[2] ? 1 : 0);
            const int4 g = S.seg[b];
            *idx = s + (uint32_t)g.x;
            v = S.sp[*idx];
            float2 l = lo[*idx];
            const float ox = __int_as_float(g.y), oy = __int_as_float(g.z);
            const float sx = v.x + ox, sy = v.y + oy;
            l.x += two_sum_err(v.x, ox, sx);
            l.y += two_sum_err(v.y, oy, sy);
            v.x = sx;
            v.y = sy;
            *vlo = l;
        }
    }
    return v;
}

template <int NP>
__device__ __forceinline__ NearField p2p_block_sym_field(const P2PSymSources& S, const float2* __restrict__ lo,
                                                         const float4* __restrict__ tg, const float4* __restrict__ tl,
                                                         const float2* __restrict__ tq, int lane,
                                                         double* __restrict__ acc, double2* __restrict__ accg) {
    constexpr int W = NP <= 2 ? 4 : (NP <= 4 ? 8 : (NP <= 8 ? 16 : 32));
    const uint32_t nch = S.nch_own + (S.n_fw + 31u) / 32u;
    NearField out;
    out.phi = out.gx = out.gy = make_float2(0.f, 0.f);
    for (uint32_t r0 = 0; r0 < nch; r0 += kP2PRun) {
        const uint32_t r1 = min(nch, r0 + (uint32_t)kP2PRun);
        float2 pp[NP], px[NP], py[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) pp[i] = px[i] = py[i] = make_float2(0.f, 0.f);
        uint32_t idx;
        float2 clo;
        float4 cur = load_lo(S, lo, r0, lane, &idx, &clo);
        for (uint32_t c = r0; c < r1; ++c) {
            uint32_t nidx = idx;
            float2 nlo = clo;
            const float4 nxt = (c + 1 < r1) ? load_lo(S, lo, c + 1, lane, &nidx, &nlo) : cur;
            if (c < S.nch_own) {
                p2p_chunk_field<true, NP>(pp, px, py, tg, tl, tq, cur, clo);
            } else {
                const float3 sv = p2p_chunk_field<false, NP>(pp, px, py, tg, tl, tq, cur, clo);
                if (idx != 0xffffffffu) {
                    atomicAdd(acc + idx, fmm_f2d_bits(sv.x));
                    atomicAdd(&accg[idx].x, fmm_f2d_bits(sv.y));
                    atomicAdd(&accg[idx].y, fmm_f2d_bits(sv.z));
                }
            }
            cur = nxt;
            idx = nidx;
            clo = nlo;
        }
        out.phi = ff_add_f(out.phi, warp_reduce_scatter<W, NP>(pp, lane));
        out.gx = ff_add_f(out.gx, warp_reduce_scatter<W, NP>(px, lane));
        out.gy = ff_add_f(out.gy, warp_reduce_scatter<W, NP>(py, lane));
    }
    return out;
}

// p2p_near_sym with the gradient: target `lane`'s phi (log2 r^2 units) and grad phi sums; the
// forward sources' shares go to acc and accg.
__device__ __forceinline__ NearField p2p_near_sym_field(const float4* __restrict__ sp, const float2* __restrict__ lo,
                                                        const uint32_t* __restrict__ ls, uint32_t leaf, uint32_t t0,
                                                        uint32_t t1, uint32_t b0, int T, int levels, float s_leaf,
                                                        float4* tgt, float4* tlo, float2* tq, int4* seg, int lane,
                                                        double* __restrict__ acc, double2* __restrict__ accg,
                                                        uint32_t* pairs) {
    const uint2 nb = p2p_forward(ls, leaf, levels, lane);
    const uint32_t n_own = t1 - t0;
    uint32_t incl = nb.y;
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t excl = incl - nb.y;
    const uint32_t n_fw = __shfl_sync(0xffffffffu, incl, 3);
    if (lane < 4) {
        const float ox = (float)(lane == 3 ? -1 : (lane == 2 ? 0 : 1)) * s_leaf;
        const float oy = (float)(lane == 0 ? 0 : 1) * s_leaf;
        seg[lane] = make_int4((int)(nb.x - excl), __float_as_int(ox), __float_as_int(oy), 0);
    }
    P2PSymSources S;
    S.sp = sp;
    S.seg = seg;
#pragma unroll
    for (int i = 0; i < 3; ++i) S.thr[i] = __shfl_sync(0xffffffffu, excl, i + 1);
    S.t0 = t0;
    S.n_own = n_own;
    S.nch_own = (n_own + 31u) / 32u;
    S.n_fw = n_fw;
    *pairs = (uint32_t)T * (n_own + 2u * n_fw) - (uint32_t)T;
    {
        float x = 0.f, y = 0.f, q = 0.f;
        float2 l = make_float2(0.f, 0.f);
        if (lane < T) {
            const float4 P = sp[b0 + lane];
            x = P.x;
            y = P.y;
            q = P.z;
            l = lo[b0 + lane];
        }
        float* t = reinterpret_cast<float*>(&tgt[lane >> 1]);
        t[lane & 1] = x;
        t[2 + (lane & 1)] = y;
        float* u = reinterpret_cast<float*>(&tlo[lane >> 1]);
        u[lane & 1] = l.x;
        u[2 + (lane & 1)] = l.y;
        reinterpret_cast<float*>(&tq[lane >> 1])[lane & 1] = q;
    }
    __syncwarp();
    switch ((T + 3) >> 2) {
        case 1: return p2p_block_sym_field<2>(S, lo, tgt, tlo, tq, lane, acc, accg);
        case 2: return p2p_block_sym_field<4>(S, lo, tgt, tlo, tq, lane, acc, accg);
        case 3: return p2p_block_sym_field<6>(S, lo, tgt, tlo, tq, lane, acc, accg);
        case 4: return p2p_block_sym_field<8>(S, lo, tgt, tlo, tq, lane, acc, accg);
        case 5: return p2p_block_sym_field<10>(S, lo, tgt, tlo, tq, lane, acc, accg);
        default: return p2p_block_sym_field<12>(S, lo, tgt, tlo, tq, lane, acc, accg);
    }
}

// phi = far + near x ln2 / 2 (the float-float factor turns sum q log2 r^2 into sum q ln r)
__device__ __forceinline__ double p2p_phi(float2 far, float2 near) {
    const float2 v = ff_add(far, ff_mul(near, make_float2(0.3465736f, -9.523271e-10f)));
    return fmm_f2d_bits(v.x) + fmm_f2d_bits(v.y);
}

}  // namespace
