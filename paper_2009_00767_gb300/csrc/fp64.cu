// fp64.cu -- the plain FP64 path of the shift-free FMM on the CUDA cores.
//
// Scaled, box-centred form (w = (z - c) / s for a square of side s and centre c):
//   P2M (U-bar of Sec. 2.2.1, every level straight from the particles, no M2M):
//       M_0 = sum q,   M_m = sum q w^m  (m = 1..p)           -- pure power sums
//   M2L (D-bar-1): b'[t] = sum_{d in IL offsets} T_d M[t + d]  (+ M_0 ln s on b'_0), where the
//       40 scale-free operators T_d fold in Greengard's 2D conversion and the -1/m of the
//       moments, built once per plan in FP64
//   L2P (D-bar-2 by linearity, no L2L): phi_far += Re sum_l b'_l w^l for every level
//   P2P (E-2 of Sec. 2.1): own + eight adjacent finest squares, j != i, r > 0
// Everything is FP64; GB300's FP64 pipe is narrow, so these kernels are DFMA-bound.
#include "fmm_internal.cuh"

namespace {

constexpr int kWarpsPerBlock = 4;

// -------------------------------------------------------------------------------- P2M
// One warp per 32 consecutive box-sorted particles; for each level the per-particle power
// sums are written to shared memory and reduced column-wise over runs of equal square key
// (a segmented reduction); each run head adds its sums into the level's grid atomically.
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_p2m_f64(const fmm_p64* __restrict__ sp, const uint32_t* __restrict__ skey, int64_t n, int levels, int p,
          double box, FmmLevelPtrs g) {
    extern __shared__ double smem[];
    __shared__ uint32_t bid[kWarpsPerBlock][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ncol = 2 * (p + 1), stride = ncol + 1;
    double* rows = smem + (size_t)warp * 32 * stride;
    const int64_t i = ((int64_t)blockIdx.x * kWarpsPerBlock + warp) * 32 + lane;
    if (((int64_t)blockIdx.x * kWarpsPerBlock + warp) * 32 >= n) return;   // whole warp idle
    const bool valid = i < n;
    fmm_p64 P = valid ? sp[i] : fmm_p64{0.0, 0.0, 0.0, 0.0};
    uint32_t key = valid ? skey[i] : 0u;
    for (int k = 2; k <= levels; ++k) {
        const uint32_t kk = key >> (2 * (levels - k));
        const double s = box / (double)(1 << k);
        const double inv_s = (double)(1 << k) / box;
        const uint32_t bx = fmm_compact2(kk), by = fmm_compact2(kk >> 1);
        const double wx = (P.x - ((double)bx + 0.5) * s) * inv_s;
        const double wy = (P.y - ((double)by + 0.5) * s) * inv_s;
        double* r = rows + lane * stride;
        double pr = P.q, pi = 0.0;   // q w^m
        r[0] = pr;
        r[1] = 0.0;
        for (int m = 1; m <= p; ++m) {
            double nr = pr * wx - pi * wy;
            double ni = pr * wy + pi * wx;
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
            double run = 0.0;
            for (int rr = 0; rr < 32; ++rr) {
                uint32_t b = bid[warp][rr];
                if (b == 0xffffffffu) break;
                if (b != cur) {
                    size_t cell = (size_t)(fmm_compact2(cur >> 1) + FMM_HALO) * W + fmm_compact2(cur) + FMM_HALO;
                    atomicAdd(A + cell * ncol + col, run);
                    run = 0.0;
                    cur = b;
                }
                run += rows[rr * stride + col];
            }
            size_t cell = (size_t)(fmm_compact2(cur >> 1) + FMM_HALO) * W + fmm_compact2(cur) + FMM_HALO;
            atomicAdd(A + cell * ncol + col, run);
        }
        __syncwarp();
    }
}

// -------------------------------------------------------------------------------- M2L
struct M2LArgs {
    FmmLevelPtrs g;
    const double2* T;              // [49][p+1][p+1], [d][k][l]
    int64_t base[FMM_MAX_LEVELS + 2];   // first flattened target of each level (levels 2..L)
    double ln_s[FMM_MAX_LEVELS + 1];
    int levels, p;
};

// One warp per target square of any level 2..L; lane l accumulates output coefficient l
// (and l + 32 when p >= 32) over the square's interaction list.
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_m2l_f64(M2LArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t gt = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (gt >= a.base[a.levels + 1]) return;
    int k = 2;
    while (gt >= a.base[k + 1]) ++k;
    const int64_t t = gt - a.base[k];
    const int side = 1 << k;
    const int tx = (int)(t % side), ty = (int)(t / side);
    const int px = tx & 1, py = ty & 1;
    const int p1 = a.p + 1, W = fmm_grid_width(k);
    const double2* A = reinterpret_cast<const double2*>(a.g.A[k]);
    double2* B = reinterpret_cast<double2*>(a.g.B[k]);
    for (int l0 = 0; l0 < p1; l0 += 32) {
        const int l = l0 + lane;
        double accr = 0.0, acci = 0.0;
        for (int dy = -2 - py; dy <= 3 - py; ++dy) {
            const int sy = ty + dy;
            if (sy < 0 || sy >= side) continue;
            for (int dx = -2 - px; dx <= 3 - px; ++dx) {
                const int sx = tx + dx;
                if (sx < 0 || sx >= side) continue;
                if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
                const double2* src = A + ((size_t)(sy + FMM_HALO) * W + (sx + FMM_HALO)) * p1;
                const double2* Td = a.T + (size_t)((dx + 3) + 7 * (dy + 3)) * p1 * p1;
                if (l < p1) {
                    for (int kk = 0; kk < p1; ++kk) {
                        const double2 m = src[kk];
                        const double2 tt = Td[(size_t)kk * p1 + l];
                        accr = fma(tt.x, m.x, accr);
                        accr = fma(-tt.y, m.y, accr);
                        acci = fma(tt.x, m.y, acci);
                        acci = fma(tt.y, m.x, acci);
                    }
                    if (l == 0) accr = fma(a.ln_s[k], src[0].x, accr);
                }
            }
        }
        if (l < p1) B[(size_t)t * p1 + l] = make_double2(accr, acci);
    }
}

// -------------------------------------------------------------------------------- L2P
// kField: also the far field's gradient, grad phi = (Re f', -Im f') with f'(z) = sum_l l b_l w^(l-1) / s
// (one Horner pass for the expansion and its derivative), per sorted particle into grad_far.
template <bool kField>
__global__ void k_l2p_f64(const fmm_p64* __restrict__ sp, const uint32_t* __restrict__ skey, int64_t n,
                          int levels, int p, double box, FmmLevelPtrs g, double* __restrict__ phi_far,
                          double2* __restrict__ grad_far) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const fmm_p64 P = sp[i];
    const uint32_t key = skey[i];
    const int p1 = p + 1;
    double far = 0.0, gx = 0.0, gy = 0.0;
    for (int k = 2; k <= levels; ++k) {
        const uint32_t kk = key >> (2 * (levels - k));
        const double s = box / (double)(1 << k);
        const double inv_s = (double)(1 << k) / box;
        const uint32_t bx = fmm_compact2(kk), by = fmm_compact2(kk >> 1);
        const double wx = (P.x - ((double)bx + 0.5) * s) * inv_s;
        const double wy = (P.y - ((double)by + 0.5) * s) * inv_s;
        const double2* Bt = reinterpret_cast<const double2*>(g.B[k]) + ((size_t)by * (1u << k) + bx) * p1;
        double2 acc = Bt[p], d = make_double2(0.0, 0.0);
        for (int l = p - 1; l >= 0; --l) {
            const double2 b = Bt[l];
            if (kField) {   // d <- d w + acc before acc moves on: d ends as the derivative
                const double dr = fma(d.x, wx, fma(-d.y, wy, acc.x));
                const double di = fma(d.x, wy, fma(d.y, wx, acc.y));
                d.x = dr;
                d.y = di;
            }
            const double r = fma(acc.x, wx, fma(-acc.y, wy, b.x));
            const double im = fma(acc.x, wy, fma(acc.y, wx, b.y));
            acc.x = r;
            acc.y = im;
        }
        far += acc.x;
        if (kField) {
            gx += d.x * inv_s;
            gy -= d.y * inv_s;
        }
    }
    phi_far[i] = far;
    if (kField) grad_far[i] = make_double2(gx, gy);
}

// -------------------------------------------------------------------------------- P2P + final phi
// One warp per finest square.  With T targets (T <= 32) the warp is split into 32 / T' groups
// (T' = T rounded up to a power of two) that take interleaved sources, then combine by shuffles.
// kField: also the near field's gradient q_j (z_i - z_j) / r^2, added to grad_far; the field
// E = -grad phi goes to field[2 i], field[2 i + 1] in input order.
template <bool kField>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_p2p_f64(const fmm_p64* __restrict__ sp, const uint32_t* __restrict__ leaf_start, int levels,
          const double* __restrict__ phi_far, double* __restrict__ phi, const unsigned int* __restrict__ status,
          unsigned long long* __restrict__ counters, const double2* __restrict__ grad_far,
          double* __restrict__ field) {
    const int lane = threadIdx.x & 31;
    const uint32_t leaf = (uint32_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const uint32_t nleaf = 1u << (2 * levels);
    if (leaf >= nleaf) return;
    if (*(volatile const unsigned int*)status != 0u) return;   // inputs failed the device checks
    const uint32_t t0 = leaf_start[leaf], t1 = leaf_start[leaf + 1];
    const int T = (int)(t1 - t0);
    if (T == 0) return;
    const int side = 1 << levels;
    const int ix = (int)fmm_compact2(leaf), iy = (int)fmm_compact2(leaf >> 1);
    uint32_t ns0[9], ns1[9];
    uint64_t nsrc = 0;
    int nn = 0;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            const int jx = ix + dx, jy = iy + dy;
            if (jx < 0 || jy < 0 || jx >= side || jy >= side) continue;
            const uint32_t nl = fmm_morton((uint32_t)jx, (uint32_t)jy);
            ns0[nn] = leaf_start[nl];
            ns1[nn] = leaf_start[nl + 1];
            nsrc += ns1[nn] - ns0[nn];
            ++nn;
        }
    if (lane == 0) {
        const unsigned slot = blockIdx.x % FMM_COUNTER_SLOTS;
        atomicAdd(&counters[slot], (unsigned long long)T * nsrc - (unsigned long long)T);
        atomicMax(&counters[FMM_COUNTER_SLOTS + slot], (unsigned long long)T);
    }
    int tp = 1;
    while (tp < T && tp < 32) tp <<= 1;
    const int groups = 32 / tp;
    const int slot = lane & (tp - 1), grp = lane / tp;
    for (int tb = 0; tb < T; tb += tp) {
        const int ti = tb + slot;
        const bool active = ti < T;
        const uint32_t gi = t0 + (active ? ti : 0);
        const fmm_p64 Pi = sp[gi];
        double acc = 0.0, ax = 0.0, ay = 0.0;
        for (int b = 0; b < nn; ++b) {
            for (uint32_t j = ns0[b] + grp; j < ns1[b]; j += groups) {
                const fmm_p64 Pj = sp[j];
                const double dx = Pi.x - Pj.x, dy = Pi.y - Pj.y;
                const double r2 = fma(dx, dx, dy * dy);
                if (j != gi && r2 > 0.0) {
                    acc = fma(Pj.q, 0.5 * log(r2), acc);
                    if (kField) {
                        const double w = Pj.q / r2;
                        ax = fma(w, dx, ax);
                        ay = fma(w, dy, ay);
                    }
                }
            }
        }
        for (int o = tp; o < 32; o <<= 1) {
            acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (kField) {
                ax += __shfl_xor_sync(0xffffffffu, ax, o);
                ay += __shfl_xor_sync(0xffffffffu, ay, o);
            }
        }
        if (active && grp == 0) {
            phi[(int64_t)Pi.w] = phi_far[gi] + acc;
            if (kField) {
                const double2 gf = grad_far[gi];
                field[2 * (int64_t)Pi.w] = -(gf.x + ax);
                field[2 * (int64_t)Pi.w + 1] = -(gf.y + ay);
            }
        }
    }
}

// -------------------------------------------------------------------------------- FP64 direct sum
__global__ void k_direct_f64(int64_t n, const double2* __restrict__ xy, const double* __restrict__ q,
                             const int64_t* __restrict__ targets, double* __restrict__ out) {
    __shared__ double red[32];
    const int64_t it = targets[blockIdx.x];
    const double2 zi = xy[it];
    double acc = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        const double2 zj = xy[j];
        const double dx = zi.x - zj.x, dy = zi.y - zj.y;
        const double r2 = fma(dx, dx, dy * dy);
        if (j != it && r2 > 0.0) acc = fma(q[j], 0.5 * log(r2), acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) out[blockIdx.x] = v;
    }
}

}  // namespace

int fmm_launch_fp64(fmm_plan_s* pl, double* phi, double* field) {
    cudaStream_t st = pl->stream;
    const int64_t n = pl->n;
    const int L = pl->levels, p = pl->p;
    int launches = 0;
    // P2M
    cudaEventRecord(pl->ev[1], st);
    if (L >= 2) {
        for (int k = 2; k <= L; ++k)
            if (cudaMemsetAsync(pl->grids.A[k], 0, pl->a_bytes[k], st) != cudaSuccess) return -1;
        const int64_t warps = (n + 31) / 32;
        const unsigned blocks = (unsigned)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock);
        const size_t shm = sizeof(double) * kWarpsPerBlock * 32 * (2 * (p + 1) + 1);
        if (shm > 48 * 1024 &&
            cudaFuncSetAttribute(k_p2m_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) != cudaSuccess)
            return -1;
        k_p2m_f64<<<blocks, kWarpsPerBlock * 32, shm, st>>>(pl->sorted64, pl->sorted_key, n, L, p, pl->box,
                                                            pl->grids);
        ++launches;
    }
    cudaEventRecord(pl->ev[2], st);
    // M2L
    if (L >= 2) {
        M2LArgs a;
        a.g = pl->grids;
        a.T = pl->T64;
        a.levels = L;
        a.p = p;
        int64_t acc = 0;
        for (int k = 0; k <= FMM_MAX_LEVELS + 1; ++k) a.base[k] = 0;
        for (int k = 2; k <= L; ++k) {
            a.base[k] = acc;
            acc += (int64_t)1 << (2 * k);
        }
        a.base[L + 1] = acc;
        for (int k = 0; k <= FMM_MAX_LEVELS; ++k) a.ln_s[k] = log(pl->box / (double)(1 << k));
        const unsigned blocks = (unsigned)((acc + kWarpsPerBlock - 1) / kWarpsPerBlock);
        k_m2l_f64<<<blocks, kWarpsPerBlock * 32, 0, st>>>(a);
        ++launches;
    }
    cudaEventRecord(pl->ev[3], st);
    // L2P
    {
        const unsigned blocks = (unsigned)((n + 127) / 128);
        if (field)
            k_l2p_f64<true><<<blocks, 128, 0, st>>>(pl->sorted64, pl->sorted_key, n, L, p, pl->box, pl->grids,
                                                    pl->phi_far, pl->near_grad);
        else
            k_l2p_f64<false><<<blocks, 128, 0, st>>>(pl->sorted64, pl->sorted_key, n, L, p, pl->box, pl->grids,
                                                     pl->phi_far, nullptr);
        ++launches;
    }
    cudaEventRecord(pl->ev[4], st);
    // P2P + final phi in input order
    {
        const uint32_t nleaf = 1u << (2 * L);
        const unsigned blocks = (nleaf + kWarpsPerBlock - 1) / kWarpsPerBlock;
        if (field)
            k_p2p_f64<true><<<blocks, kWarpsPerBlock * 32, 0, st>>>(pl->sorted64, pl->leaf_start, L, pl->phi_far, phi,
                                                                    pl->d_status, pl->d_counters, pl->near_grad,
                                                                    field);
        else
            k_p2p_f64<false><<<blocks, kWarpsPerBlock * 32, 0, st>>>(pl->sorted64, pl->leaf_start, L, pl->phi_far,
                                                                     phi, pl->d_status, pl->d_counters, nullptr,
                                                                     nullptr);
        ++launches;
    }
    cudaEventRecord(pl->ev[5], st);
    if (cudaGetLastError() != cudaSuccess) return -1;
    return launches;
}

int fmm_launch_direct_f64(int64_t n, const double* xy, const double* q, int64_t nt, const int64_t* targets,
                          double* phi_t, cudaStream_t stream) {
    if (nt == 0) return 0;
    k_direct_f64<<<(unsigned)nt, 256, 0, stream>>>(n, reinterpret_cast<const double2*>(xy), q, targets, phi_t);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}
