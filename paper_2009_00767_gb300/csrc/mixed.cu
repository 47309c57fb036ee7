// mixed.cu -- the mixed-precision path: FP32 particle stages, FP32 M2L on the CUDA cores,
// FP64 where magnitudes are large (moment accumulation, the monopole-log part of b'_0, the
// cross-level sum of phi).
//
// Scaled form as in fp64.cu (w = (z - c) / s, power-sum moments M_m = sum q w^m):
//   P2M  every level straight from the particles (U-bar of Sec. 2.2.1): w is formed in FP32
//        from the particle's offset to its finest-square centre (exact dyadic square offsets
//        plus an FP32 product), q w^m in FP32, warp-segmented FP32 sums of at most 32 terms,
//        then FP64 atomics into the level's grid.
//   M2L  (D-bar-1) per target: b'_l = sum_d sum_k T_d[k][l] M[t+d][k] in FP32 (k, l = 0..p),
//        except the monopole-log term M_0 (log|w0| + ln s) of b'_0, which is summed in FP64
//        (it dominates the magnitude of phi for random-sign charges).
//   L2P  (D-bar-2 by linearity) per particle and level: Re sum_{l>=1} b'_l w^l by Horner in
//        FP32, plus the FP64 b'_0; levels summed in FP64.
//   P2P  (E-2 of Sec. 2.1) in FP32 on square-local coordinates; log via the MUFU lg2 unit.
#include "fmm_internal.cuh"

namespace {

constexpr int kWarpsPerBlock = 4;
constexpr int kM2LThreads = 128;

// w of a particle in its level-k square, from its offset (dx, dy) to the centre of its finest
// square (ix, iy): w = ((i_local + 1/2) 2^-(l-k) - 1/2) + d 2^k / box.  The first part is an
// exact dyadic number in FP32.
__device__ __forceinline__ float2 level_w(float dx, float dy, uint32_t ix, uint32_t iy, int sh, float inv_s) {
    const uint32_t mask = (1u << sh) - 1u;
    const float sc = __int_as_float((127 - sh) << 23);   // 2^-sh
    const float ox = fmaf((float)(ix & mask) + 0.5f, sc, -0.5f);
    const float oy = fmaf((float)(iy & mask) + 0.5f, sc, -0.5f);
    return make_float2(fmaf(dx, inv_s, ox), fmaf(dy, inv_s, oy));
}

// -------------------------------------------------------------------------------- P2M
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_p2m_mixed(const float4* __restrict__ sp, const uint32_t* __restrict__ skey, int64_t n, int levels, int p,
            double box, FmmLevelPtrs g) {
    extern __shared__ float smf[];
    __shared__ uint32_t bid[kWarpsPerBlock][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ncol = 2 * (p + 1), stride = ncol + 1;
    float* rows = smf + (size_t)warp * 32 * stride;
    const int64_t w0 = ((int64_t)blockIdx.x * kWarpsPerBlock + warp) * 32;
    if (w0 >= n) return;
    const int64_t i = w0 + lane;
    const bool valid = i < n;
    const float4 P = valid ? sp[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const uint32_t key = valid ? skey[i] : 0u;
    const uint32_t ix = fmm_compact2(key), iy = fmm_compact2(key >> 1);
    for (int k = 2; k <= levels; ++k) {
        const int sh = levels - k;
        const uint32_t kk = key >> (2 * sh);
        const float inv_s = (float)((double)(1 << k) / box);
        const float2 w = level_w(P.x, P.y, ix, iy, sh, inv_s);
        float* r = rows + lane * stride;
        float pr = P.z, pi = 0.f;
        r[0] = pr;
        r[1] = 0.f;
        for (int m = 1; m <= p; ++m) {
            const float nr = fmaf(pr, w.x, -pi * w.y);
            const float ni = fmaf(pr, w.y, pi * w.x);
            pr = nr;
            pi = ni;
            r[2 * m] = pr;
            r[2 * m + 1] = pi;
        }
        bid[warp][lane] = valid ? kk : 0xffffffffu;
        __syncwarp();
        const int W = fmm_grid_width(k);
        double* A = reinterpret_cast<double*>(g.A[k]);
        for (int col = lane; col < ncol; col += 32) {
            uint32_t cur = bid[warp][0];
            float run = 0.f;
            for (int rr = 0; rr < 32; ++rr) {
                const uint32_t b = bid[warp][rr];
                if (b == 0xffffffffu) break;
                if (b != cur) {
                    const size_t cell = (size_t)(fmm_compact2(cur >> 1) + FMM_HALO) * W + fmm_compact2(cur) + FMM_HALO;
                    atomicAdd(A + cell * ncol + col, (double)run);
                    run = 0.f;
                    cur = b;
                }
                run += rows[rr * stride + col];
            }
            const size_t cell = (size_t)(fmm_compact2(cur >> 1) + FMM_HALO) * W + fmm_compact2(cur) + FMM_HALO;
            atomicAdd(A + cell * ncol + col, (double)run);
        }
        __syncwarp();
    }
}

// -------------------------------------------------------------------------------- M2L (FP32 SIMT)
struct M2LMixedArgs {
    FmmLevelPtrs g;
    const float2* T;                    // [49][P1B][P1B] FP32, zero beyond p and at [d][0][0]
    double logw0[49];                   // log|w0| per offset (FP64 monopole term)
    double ln_s[FMM_MAX_LEVELS + 1];
    int cta_base[FMM_MAX_LEVELS + 2];   // first CTA of each level
    int levels, p;
};

// One thread per target square; the CTA's 128 targets share one parity class (so one list of
// 27 offsets) and stage each offset's operator in shared memory, read as broadcasts.
template <int P1B>
__global__ void __launch_bounds__(kM2LThreads) k_m2l_f32(M2LMixedArgs a) {
    __shared__ float2 Ts[P1B * P1B];
    const int cta = blockIdx.x;
    int k = 2;
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
    const double2* A = reinterpret_cast<const double2*>(a.g.A[k]);
    float2 acc[P1B];
#pragma unroll
    for (int l = 0; l < P1B; ++l) acc[l] = make_float2(0.f, 0.f);
    double mono = 0.0;
    for (int dy = -2 - py; dy <= 3 - py; ++dy) {
        for (int dx = -2 - px; dx <= 3 - px; ++dx) {
            if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
            const int d = (dx + 3) + 7 * (dy + 3);
            __syncthreads();
            const float2* Td = a.T + (size_t)d * P1B * P1B;
            for (int e = threadIdx.x; e < P1B * P1B; e += kM2LThreads) Ts[e] = Td[e];
            __syncthreads();
            // sources outside the domain read the zero halo
            const double2* src = A + ((size_t)(ty + dy + FMM_HALO) * W + (tx + dx + FMM_HALO)) * p1;
            float2 m[P1B];
#pragma unroll
            for (int kk = 0; kk < P1B; ++kk) {
                if (kk < p1) {
                    const double2 v = src[kk];
                    m[kk] = make_float2((float)v.x, (float)v.y);
                    if (kk == 0) mono = fma(v.x, a.logw0[d] + a.ln_s[k], mono);   // M_0 (log|w0| + ln s)
                } else {
                    m[kk] = make_float2(0.f, 0.f);
                }
            }
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
    double* B0 = reinterpret_cast<double*>(a.g.B0[k]);
    for (int l = 0; l < p1 && l < P1B; ++l) B[t * p1 + l] = acc[l];
    B0[t] = mono + (double)acc[0].x;
}

// -------------------------------------------------------------------------------- L2P
__global__ void k_l2p_mixed(const float4* __restrict__ sp, const uint32_t* __restrict__ skey, int64_t n,
                            int levels, int p, double box, FmmLevelPtrs g, double* __restrict__ phi_far) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 P = sp[i];
    const uint32_t key = skey[i];
    const uint32_t ix = fmm_compact2(key), iy = fmm_compact2(key >> 1);
    const int p1 = p + 1;
    double far = 0.0;
    for (int k = 2; k <= levels; ++k) {
        const int sh = levels - k;
        const float inv_s = (float)((double)(1 << k) / box);
        const float2 w = level_w(P.x, P.y, ix, iy, sh, inv_s);
        const size_t t = (size_t)(iy >> sh) * (1u << k) + (ix >> sh);
        const float2* Bt = reinterpret_cast<const float2*>(g.B[k]) + t * p1;
        float2 u = Bt[p];
        for (int l = p - 1; l >= 1; --l) {
            const float2 b = Bt[l];
            const float ur = fmaf(u.x, w.x, fmaf(-u.y, w.y, b.x));
            const float ui = fmaf(u.x, w.y, fmaf(u.y, w.x, b.y));
            u.x = ur;
            u.y = ui;
        }
        const float v = fmaf(u.x, w.x, -u.y * w.y);   // Re(u w)
        far += reinterpret_cast<const double*>(g.B0[k])[t] + (double)v;
    }
    phi_far[i] = far;
}

// -------------------------------------------------------------------------------- P2P + final phi
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_p2p_mixed(const float4* __restrict__ sp, const uint32_t* __restrict__ leaf_start, int levels, double box,
            const double* __restrict__ phi_far, double* __restrict__ phi, const unsigned int* __restrict__ status,
            unsigned long long* __restrict__ counters) {
    const int lane = threadIdx.x & 31;
    const uint32_t leaf = (uint32_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const uint32_t nleaf = 1u << (2 * levels);
    if (leaf >= nleaf) return;
    if (*(volatile const unsigned int*)status != 0u) return;
    const uint32_t t0 = leaf_start[leaf], t1 = leaf_start[leaf + 1];
    const int T = (int)(t1 - t0);
    if (T == 0) return;
    const int side = 1 << levels;
    const float s = (float)(box / (double)side);
    const int ix = (int)fmm_compact2(leaf), iy = (int)fmm_compact2(leaf >> 1);
    uint32_t ns0[9], ns1[9];
    float offx[9], offy[9];
    uint64_t nsrc = 0;
    int nn = 0;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            const int jx = ix + dx, jy = iy + dy;
            if (jx < 0 || jy < 0 || jx >= side || jy >= side) continue;
            const uint32_t nl = fmm_morton((uint32_t)jx, (uint32_t)jy);
            ns0[nn] = leaf_start[nl];
            ns1[nn] = leaf_start[nl + 1];
            offx[nn] = (float)(-dx) * s;   // target-centre minus source-centre, exact
            offy[nn] = (float)(-dy) * s;
            nsrc += ns1[nn] - ns0[nn];
            ++nn;
        }
    if (lane == 0) {
        atomicAdd(&counters[0], (unsigned long long)T * nsrc - (unsigned long long)T);
        atomicMax(&counters[1], (unsigned long long)T);
    }
    int tp = 1;
    while (tp < T && tp < 32) tp <<= 1;
    const int groups = 32 / tp;
    const int slot = lane & (tp - 1), grp = lane / tp;
    for (int tb = 0; tb < T; tb += tp) {
        const int ti = tb + slot;
        const bool active = ti < T;
        const uint32_t gi = t0 + (active ? ti : 0);
        const float4 Pi = sp[gi];
        float acc = 0.f;
        for (int b = 0; b < nn; ++b) {
            const float bx = Pi.x + offx[b], by = Pi.y + offy[b];
            for (uint32_t j = ns0[b] + grp; j < ns1[b]; j += groups) {
                const float4 Pj = sp[j];
                const float ddx = bx - Pj.x, ddy = by - Pj.y;
                const float r2 = fmaf(ddx, ddx, ddy * ddy);
                if (j != gi && r2 > 0.f) acc = fmaf(Pj.z, __log2f(r2), acc);
            }
        }
        for (int o = tp; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (active && grp == 0)
            phi[__float_as_int(Pi.w)] = phi_far[gi] + (double)acc * 0.34657359027997264;   // ln2 / 2
    }
}

template <int P1B>
void launch_m2l(const M2LMixedArgs& a, int blocks, cudaStream_t st) {
    k_m2l_f32<P1B><<<blocks, kM2LThreads, 0, st>>>(a);
}

}  // namespace

int fmm_m2l_bucket(int p1) {
    const int b[] = {9, 13, 17, 21, 25, 33, 41};
    for (int v : b)
        if (p1 <= v) return v;
    return -1;
}

int fmm_launch_mixed(fmm_plan_s* pl, double* phi) {
    if (pl->precision != FMM_MIXED_FP32) return -2;
    cudaStream_t st = pl->stream;
    const int64_t n = pl->n;
    const int L = pl->levels, p = pl->p;
    int launches = 0;
    cudaEventRecord(pl->ev[1], st);
    if (L >= 2) {
        for (int k = 2; k <= L; ++k)
            if (cudaMemsetAsync(pl->grids.A[k], 0, pl->a_bytes[k], st) != cudaSuccess) return -1;
        const int64_t warps = (n + 31) / 32;
        const unsigned blocks = (unsigned)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock);
        const size_t shm = sizeof(float) * kWarpsPerBlock * 32 * (2 * (p + 1) + 1);
        k_p2m_mixed<<<blocks, kWarpsPerBlock * 32, shm, st>>>(pl->sorted32, pl->sorted_key, n, L, p, pl->box,
                                                              pl->grids);
        ++launches;
    }
    cudaEventRecord(pl->ev[2], st);
    if (L >= 2) {
        M2LMixedArgs a;
        a.g = pl->grids;
        a.T = pl->T32;
        a.levels = L;
        a.p = p;
        for (int d = 0; d < 49; ++d) {
            const int dx = d % 7 - 3, dy = d / 7 - 3;
            a.logw0[d] = (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) ? 0.0 : 0.5 * log((double)(dx * dx + dy * dy));
        }
        for (int k = 0; k <= FMM_MAX_LEVELS; ++k) a.ln_s[k] = log(pl->box / (double)(1 << k));
        int acc = 0;
        for (int k = 0; k <= FMM_MAX_LEVELS + 1; ++k) a.cta_base[k] = 0;
        for (int k = 2; k <= L; ++k) {
            a.cta_base[k] = acc;
            const int w2 = 1 << (k - 1);
            acc += 4 * ((w2 * w2 + kM2LThreads - 1) / kM2LThreads);
        }
        a.cta_base[L + 1] = acc;
        switch (pl->p1b) {
            case 9: launch_m2l<9>(a, acc, st); break;
            case 13: launch_m2l<13>(a, acc, st); break;
            case 17: launch_m2l<17>(a, acc, st); break;
            case 21: launch_m2l<21>(a, acc, st); break;
            case 25: launch_m2l<25>(a, acc, st); break;
            case 33: launch_m2l<33>(a, acc, st); break;
            case 41: launch_m2l<41>(a, acc, st); break;
            default: return -2;
        }
        ++launches;
    }
    cudaEventRecord(pl->ev[3], st);
    {
        const unsigned blocks = (unsigned)((n + 127) / 128);
        k_l2p_mixed<<<blocks, 128, 0, st>>>(pl->sorted32, pl->sorted_key, n, L, p, pl->box, pl->grids, pl->phi_far);
        ++launches;
    }
    cudaEventRecord(pl->ev[4], st);
    {
        const uint32_t nleaf = 1u << (2 * L);
        const unsigned blocks = (nleaf + kWarpsPerBlock - 1) / kWarpsPerBlock;
        k_p2p_mixed<<<blocks, kWarpsPerBlock * 32, 0, st>>>(pl->sorted32, pl->leaf_start, L, pl->box, pl->phi_far,
                                                            phi, pl->d_status, pl->d_counters);
        ++launches;
    }
    cudaEventRecord(pl->ev[5], st);
    if (cudaGetLastError() != cudaSuccess) return -1;
    return launches;
}
