// api.cu -- the C ABI of include/fmm.h: plans, the FP64 operator build, dispatch and status.
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "mixed_common.cuh"

namespace {

using cd = std::complex<double>;

// Scale-free M2L operators on power-sum moments (D-bar-1 of Sec. 2.2.1 realised with Greengard's
// 2D multipole-to-local conversion, the paper's ref. [101]).  For a source square at offset
// w0 = dx + i dy (in units of the side s) from the target, with moments M_0 = sum q,
// M_k = sum q w^k and local coefficients b'_l of (z - c_t)/s:
//   b'_0 = M_0 log(-w0)       + sum_k M_k (-1)^(k+1) / k  w0^-k                (+ M_0 ln s)
//   b'_l = -M_0 / (l w0^l)    + sum_k M_k (-1)^(k+1) / k  C(l+k-1, k-1) w0^-(l+k)
// Built in FP64 (Sec. 4, Discussion (3): the entries come from large binomials times small powers).
// Layout [d][k][l], d = (dx + 3) + 7 (dy + 3); the nine adjacent offsets stay zero.
void build_operators(int p, std::vector<cd>& T) {
    const int p1 = p + 1;
    T.assign((size_t)49 * p1 * p1, cd(0.0, 0.0));
    std::vector<std::vector<double>> C(2 * p + 2, std::vector<double>(2 * p + 2, 0.0));
    for (int nn = 0; nn < 2 * p + 2; ++nn) {
        C[nn][0] = 1.0;
        for (int r = 1; r <= nn; ++r) C[nn][r] = C[nn - 1][r - 1] + (r <= nn - 1 ? C[nn - 1][r] : 0.0);
    }
    for (int dy = -3; dy <= 3; ++dy)
        for (int dx = -3; dx <= 3; ++dx) {
            if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
            const cd w0((double)dx, (double)dy);
            const cd inv = 1.0 / w0;
            std::vector<cd> ip(2 * p + 2);
            ip[0] = 1.0;
            for (int m = 1; m < 2 * p + 2; ++m) ip[m] = ip[m - 1] * inv;
            cd* Td = &T[(size_t)((dx + 3) + 7 * (dy + 3)) * p1 * p1];
            auto at = [&](int k, int l) -> cd& { return Td[(size_t)k * p1 + l]; };
            at(0, 0) = std::log(-w0);
            for (int l = 1; l <= p; ++l) at(0, l) = -ip[l] / (double)l;
            for (int k = 1; k <= p; ++k) {
                const double sgn = (k & 1) ? 1.0 : -1.0;   // (-1)^(k+1)
                at(k, 0) = sgn / (double)k * ip[k];
                for (int l = 1; l <= p; ++l) at(k, l) = sgn / (double)k * C[l + k - 1][k - 1] * ip[l + k];
            }
        }
}

bool valid_precision(int v) { return v >= FMM_FP64 && v <= FMM_MIXED_BF16X2; }

// fmm_potential_host: inputs of at least kHostChunkMin particles go up in kHostChunks chunks
constexpr size_t kHostChunkMin = 1 << 16;
constexpr int kHostChunks = 4;

}  // namespace

void fmm_build_operators_f64(int p, std::vector<double>& re, std::vector<double>& im) {
    std::vector<cd> T;
    build_operators(p, T);
    re.resize(T.size());
    im.resize(T.size());
    for (size_t i = 0; i < T.size(); ++i) {
        re[i] = T[i].real();
        im[i] = T[i].imag();
    }
}

namespace {

template <class T>
fmm_status dev_alloc(fmm_plan_s* pl, T** ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? FMM_ERR_OOM : FMM_ERR_CUDA;
    }
    pl->workspace_bytes += bytes;
    return FMM_OK;
}

void free_plan(fmm_plan_s* pl) {
    if (!pl) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(pl->device);
    void* bufs[] = {pl->keys, pl->rank, pl->counts, pl->leaf_start, pl->block_sums, pl->leaf_bstart,
                    pl->blk_map, pl->sorted_key,
                    pl->sorted64, pl->sorted32, pl->sorted_lo, pl->phi_far, pl->near_grad, pl->far_part,
                    pl->T64, pl->T32, pl->U32,
                    pl->d_status,
                    pl->d_counters, pl->d_xy_stage[0], pl->d_q_stage[0], pl->d_phi_stage[0], pl->d_xy_stage[1],
                    pl->d_q_stage[1], pl->d_phi_stage[1]};
    for (void* b : bufs)
        if (b) cudaFree(b);
    for (int k = 0; k <= FMM_MAX_LEVELS; ++k) {
        if (pl->grids.A[k]) cudaFree(pl->grids.A[k]);
        if (pl->grids.B[k]) cudaFree(pl->grids.B[k]);
        if (pl->grids.A32[k]) cudaFree(pl->grids.A32[k]);
    }
    fmm_tc_destroy(pl);
    if (pl->h_status) cudaFreeHost(pl->h_status);
    if (pl->h_counters) cudaFreeHost(pl->h_counters);
    if (pl->crowd_hint_h) cudaFreeHost(pl->crowd_hint_h);
    for (int e = 0; e < fmm_plan_s::kEvents; ++e)
        if (pl->ev[e]) cudaEventDestroy(pl->ev[e]);
    if (pl->ev_fork) cudaEventDestroy(pl->ev_fork);
    if (pl->ev_join) cudaEventDestroy(pl->ev_join);
    if (pl->ev_join3) cudaEventDestroy(pl->ev_join3);
    if (pl->ev_a32) cudaEventDestroy(pl->ev_a32);
    if (pl->stream2) cudaStreamDestroy(pl->stream2);
    if (pl->stream3) cudaStreamDestroy(pl->stream3);
    if (pl->s_up) cudaStreamDestroy(pl->s_up);
    if (pl->s_down) cudaStreamDestroy(pl->s_down);
    cudaEvent_t evs[] = {pl->ev_sorted, pl->ev_stage_free[0], pl->ev_stage_free[1], pl->ev_up_done, pl->ev_l2p_done,
                         pl->ev_down_done[0], pl->ev_down_done[1]};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    cudaSetDevice(prev);
    delete pl;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// the mixed path's accumulator (the square populations) back to zero
fmm_status reset_accumulators(fmm_plan_s* pl, cudaStream_t st) {
    const size_t m = (size_t)1 << (2 * pl->levels);
    if (cudaMemsetAsync(pl->counts, 0, sizeof(uint32_t) * m, st) != cudaSuccess) return FMM_ERR_CUDA;
    pl->clean = 1;
    return FMM_OK;
}

// The call's first steps, up to the start event: counters and, after a call that failed to enqueue,
// the mixed path's accumulators back to zero.
fmm_status enqueue_prologue(fmm_plan_s* pl) {
    cudaStream_t st = pl->stream;
    if (cudaMemsetAsync(pl->d_counters, 0, 2 * FMM_COUNTER_SLOTS * sizeof(unsigned long long), st) != cudaSuccess)
        return FMM_ERR_CUDA;
    if (pl->precision != FMM_FP64) {
        if (!pl->clean && reset_accumulators(pl, st) != FMM_OK) return FMM_ERR_CUDA;
        pl->clean = 0;   // until the whole call is enqueued
    }
    pl->ev_kernels = 0;
    cudaEventRecord(pl->ev[0], st);
    return FMM_OK;
}

// binned: the prologue ran and the particles were binned already (fmm_potential_host)
fmm_status enqueue(fmm_plan_s* pl, const double* xy, const double* q, double* phi, double* field = nullptr,
                   bool binned = false) {
    if (!binned) {
        const fmm_status s = enqueue_prologue(pl);
        if (s != FMM_OK) return s;
    }
    int launches = fmm_launch_sort(pl, xy, q, field != nullptr && pl->precision != FMM_FP64, binned);
    if (launches < 0) return FMM_ERR_CUDA;
    if (pl->ev_sorted) {
        // the inputs, keys, ranks and populations are free for the next host call's uploads
        if (cudaEventRecord(pl->ev_sorted, pl->stream) != cudaSuccess ||
            cudaEventRecord(pl->ev_stage_free[pl->stage_next], pl->stream) != cudaSuccess)
            return FMM_ERR_CUDA;
    }
    if (binned) launches += pl->host_chunks;   // the binning kernels of the chunks
    int more = pl->precision == FMM_FP64 ? fmm_launch_fp64(pl, phi, field) : fmm_launch_mixed(pl, phi, field);
    if (more == -2) return FMM_ERR_UNSUPPORTED;
    if (more < 0) return FMM_ERR_CUDA;
    pl->launches = launches + more;
    pl->events_recorded = 1;
    if (pl->precision != FMM_FP64) pl->clean = 1;
    return FMM_OK;
}

}  // namespace

extern "C" {

const char* fmm_status_string(int status) {
    switch (status) {
        case FMM_OK: return "ok";
        case FMM_ERR_INVALID_ARG: return "invalid argument";
        case FMM_ERR_OUT_OF_BOX: return "a particle lies outside the computation box";
        case FMM_ERR_NONFINITE: return "a coordinate or charge is not finite";
        case FMM_ERR_CUDA: return "CUDA runtime error";
        case FMM_ERR_OOM: return "out of device memory";
        case FMM_ERR_TIMEOUT: return "a bounded device-side wait timed out";
        case FMM_ERR_UNSUPPORTED: return "unsupported configuration";
        default: return "unknown status";
    }
}

fmm_status fmm_plan(fmm_plan_t* out, int64_t n, int levels, int p, double box, int precision, void* stream) {
    if (!out) return FMM_ERR_INVALID_ARG;
    if (n < 1 || n > 2147483647LL || levels < 0 || levels > FMM_MAX_LEVELS || p < 1 || p > FMM_MAX_P ||
        !(box > 0.0) || !std::isfinite(box) || !valid_precision(precision))
        return FMM_ERR_INVALID_ARG;
    fmm_plan_s* pl = new (std::nothrow) fmm_plan_s();
    if (!pl) return FMM_ERR_OOM;
    if (cudaGetDevice(&pl->device) != cudaSuccess) {
        delete pl;
        return FMM_ERR_CUDA;
    }
    pl->n = n;
    pl->levels = levels;
    pl->p = p;
    pl->box = box;
    pl->precision = precision;
    pl->stream = static_cast<cudaStream_t>(stream);
    const int64_t m = (int64_t)1 << (2 * levels);
    const int p1 = p + 1;
    fmm_status s = FMM_OK;
#define FMM_TRY(expr)                \
    do {                             \
        s = (expr);                  \
        if (s != FMM_OK) {           \
            free_plan(pl);           \
            return s;                \
        }                            \
    } while (0)
    FMM_TRY(dev_alloc(pl, &pl->keys, sizeof(uint32_t) * n));
    FMM_TRY(dev_alloc(pl, &pl->rank, sizeof(uint32_t) * n));
    FMM_TRY(dev_alloc(pl, &pl->counts, sizeof(uint32_t) * m));
    FMM_TRY(dev_alloc(pl, &pl->leaf_start, sizeof(uint32_t) * (m + 1)));
    pl->scan_blocks = fmm_scan_blocks(m);
    // 64-bit partials in the mixed path (one scan of populations and near-field blocks)
    FMM_TRY(dev_alloc(pl, &pl->block_sums, sizeof(unsigned long long) * (pl->scan_blocks + 1)));
    if (precision != FMM_FP64) {
        FMM_TRY(dev_alloc(pl, &pl->leaf_bstart, sizeof(uint32_t) * (m + 1)));
        // near-field blocks: at most one partial block per square; the near-field grid has four warps
        // a CTA and every warp reads its entry, so the map is rounded up to four entries
        const size_t nblk = ((size_t)m + (size_t)n / FMM_P2P_BLOCK + 1 + 3) & ~(size_t)3;
        FMM_TRY(dev_alloc(pl, &pl->blk_map, sizeof(uint2) * nblk));
    }
    FMM_TRY(dev_alloc(pl, &pl->sorted_key, sizeof(uint32_t) * n));
    if (precision == FMM_FP64)
        FMM_TRY(dev_alloc(pl, &pl->sorted64, sizeof(fmm_p64) * n));
    else
        FMM_TRY(dev_alloc(pl, &pl->sorted32, sizeof(float4) * n));
    FMM_TRY(dev_alloc(pl, &pl->phi_far, sizeof(double) * n));
    // the field's gradient accumulator (near field in the mixed path, far field in the FP64 path)
    FMM_TRY(dev_alloc(pl, &pl->near_grad, sizeof(double2) * n));
    if (precision != FMM_FP64) {
        FMM_TRY(dev_alloc(pl, &pl->sorted_lo, sizeof(float2) * n));
        FMM_TRY(dev_alloc(pl, &pl->far_part, sizeof(float2) * n));
    }
    const size_t bcplx = precision == FMM_FP64 ? sizeof(double2) : sizeof(float2);
    for (int k = 2; k <= levels; ++k) {
        const size_t W = (size_t)fmm_grid_width(k);
        pl->a_bytes[k] = W * W * p1 * sizeof(double2);
        if (precision == FMM_FP64)   // the mixed path's moments live in the FP32 grids only
            FMM_TRY(dev_alloc(pl, reinterpret_cast<char**>(&pl->grids.A[k]), pl->a_bytes[k]));
        FMM_TRY(dev_alloc(pl, reinterpret_cast<char**>(&pl->grids.B[k]), ((size_t)1 << (2 * k)) * p1 * bcplx));
        if (precision != FMM_FP64) {
            // the 3-cell halo of the FP32 grid stays zero for the plan's lifetime
            FMM_TRY(dev_alloc(pl, reinterpret_cast<char**>(&pl->grids.A32[k]), W * W * p1 * sizeof(float2)));
            if (cudaMemset(pl->grids.A32[k], 0, W * W * p1 * sizeof(float2)) != cudaSuccess) FMM_TRY(FMM_ERR_CUDA);
        }
    }
    std::vector<cd> T;
    build_operators(p, T);
    FMM_TRY(dev_alloc(pl, &pl->T64, sizeof(double2) * T.size()));
    if (cudaMemcpy(pl->T64, T.data(), sizeof(double2) * T.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        FMM_TRY(FMM_ERR_CUDA);
    if (fmm_tc_precision(precision)) {
        std::vector<double> tre(T.size()), tim(T.size());
        for (size_t i = 0; i < T.size(); ++i) {
            tre[i] = T[i].real();
            tim[i] = T[i].imag();
        }
        const int r = fmm_tc_create(pl, tre, tim);
        if (r == -2) FMM_TRY(FMM_ERR_UNSUPPORTED);
        if (r < 0) FMM_TRY(FMM_ERR_CUDA);
    }
    if (precision != FMM_FP64) {
        pl->p1b = fmm_m2l_bucket(p1);
        if (pl->p1b < 0) FMM_TRY(FMM_ERR_UNSUPPORTED);
        const int pb = pl->p1b;
        std::vector<float2> T32((size_t)49 * pb * pb, make_float2(0.f, 0.f));
        for (int d = 0; d < 49; ++d)
            for (int k = 0; k < p1; ++k)
                for (int l = 0; l < p1; ++l) {
                    if (k == 0 && l == 0) continue;   // the monopole-log term runs in FP64
                    const cd v = T[((size_t)d * p1 + k) * p1 + l];
                    T32[((size_t)d * pb + k) * pb + l] = make_float2((float)v.real(), (float)v.imag());
                }
        FMM_TRY(dev_alloc(pl, &pl->T32, sizeof(float2) * T32.size()));
        if (cudaMemcpy(pl->T32, T32.data(), sizeof(float2) * T32.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            FMM_TRY(FMM_ERR_CUDA);
        // the upward pass's translations, one per child position c = cx + 2 cy: a child's moments
        // about its centre re-expanded about its parent's, M_m(parent) += sum_{j <= m} U_c[m][j] M_j
        // with U_c[m][j] = C(m, j) 2^-j d_c^(m-j), d_c = ((cx - 1/2) / 2, (cy - 1/2) / 2): w = w'/2 + d_c
        // between the parent's and the child's scaled offsets (FP64, rounded once to FP32); stored
        // [c][j][m], so that the threads over m read one j together
        std::vector<float2> U((size_t)4 * pb * pb, make_float2(0.f, 0.f));
        for (int c = 0; c < 4; ++c) {
            const cd d(((c & 1) - 0.5) * 0.5, ((c >> 1) - 0.5) * 0.5);
            for (int m = 0; m < p1; ++m) {
                double binom = 1.0;   // C(m, j)
                for (int j = 0; j <= m; ++j) {
                    const cd v = binom * std::ldexp(1.0, -j) * std::pow(d, m - j);
                    U[((size_t)c * pb + j) * pb + m] = make_float2((float)v.real(), (float)v.imag());
                    binom = binom * (double)(m - j) / (double)(j + 1);
                }
            }
        }
        FMM_TRY(dev_alloc(pl, &pl->U32, sizeof(float2) * U.size()));
        if (cudaMemcpy(pl->U32, U.data(), sizeof(float2) * U.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            FMM_TRY(FMM_ERR_CUDA);
    }
    FMM_TRY(dev_alloc(pl, &pl->d_status, sizeof(unsigned int)));
    FMM_TRY(dev_alloc(pl, &pl->d_counters, 2 * FMM_COUNTER_SLOTS * sizeof(unsigned long long)));
    if (cudaMemset(pl->d_status, 0, sizeof(unsigned int)) != cudaSuccess) FMM_TRY(FMM_ERR_CUDA);
    if (cudaHostAlloc(reinterpret_cast<void**>(&pl->crowd_hint_h), sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void**>(&pl->crowd_hint_d), pl->crowd_hint_h, 0) != cudaSuccess)
        FMM_TRY(FMM_ERR_CUDA);
    *pl->crowd_hint_h = 0;
    if (cudaMallocHost(reinterpret_cast<void**>(&pl->h_status), sizeof(unsigned int)) != cudaSuccess)
        FMM_TRY(FMM_ERR_OOM);
    if (cudaMallocHost(reinterpret_cast<void**>(&pl->h_counters), 2 * FMM_COUNTER_SLOTS * sizeof(unsigned long long)) !=
        cudaSuccess)
        FMM_TRY(FMM_ERR_OOM);
    for (int b = 0; b < 2; ++b) {
        FMM_TRY(dev_alloc(pl, &pl->d_xy_stage[b], sizeof(double) * 2 * n));
        FMM_TRY(dev_alloc(pl, &pl->d_q_stage[b], sizeof(double) * n));
        FMM_TRY(dev_alloc(pl, &pl->d_phi_stage[b], sizeof(double) * n));
    }
    for (int e = 0; e < fmm_plan_s::kEvents; ++e)
        if (cudaEventCreate(&pl->ev[e]) != cudaSuccess) FMM_TRY(FMM_ERR_CUDA);
    if (precision != FMM_FP64) {
        // the mixed path's near field and coarse levels run on streams of the plan's own
        if (cudaStreamCreateWithFlags(&pl->stream2, cudaStreamNonBlocking) != cudaSuccess ||

            cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&pl->ev_join, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&pl->ev_join3, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&pl->ev_a32, cudaEventDisableTiming) != cudaSuccess ||
            cudaStreamCreateWithFlags(&pl->s_up, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&pl->s_down, cudaStreamNonBlocking) != cudaSuccess)
            FMM_TRY(FMM_ERR_CUDA);
        // The coarse levels' chain (upward pass, coarse M2L and L2P) is a string of small launches
        // behind the fine P2M; at the device's highest priority its blocks go first whenever the
        // near field's blocks leave an SM, instead of after all of them.
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
            cudaStreamCreateWithPriority(&pl->stream3, cudaStreamNonBlocking, greatest) != cudaSuccess)
            FMM_TRY(FMM_ERR_CUDA);
        cudaEvent_t* evs[] = {&pl->ev_sorted, &pl->ev_stage_free[0], &pl->ev_stage_free[1], &pl->ev_up_done,
                              &pl->ev_l2p_done, &pl->ev_down_done[0], &pl->ev_down_done[1]};
        for (cudaEvent_t* e : evs)
            if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) FMM_TRY(FMM_ERR_CUDA);
    }
#undef FMM_TRY
    pl->last.n = n;
    pl->last.levels = levels;
    pl->last.p = p;
    pl->last.precision = precision;
    pl->last.workspace_bytes = pl->workspace_bytes;
    *out = pl;
    return FMM_OK;
}

fmm_status fmm_set_concurrency(fmm_plan_t plan, int streams) {
    if (!plan || (streams != 1 && streams != 3)) return FMM_ERR_INVALID_ARG;
    plan->serial = streams == 1;
    return FMM_OK;
}

fmm_status fmm_set_stream(fmm_plan_t plan, void* stream) {
    if (!plan) return FMM_ERR_INVALID_ARG;
    plan->stream = static_cast<cudaStream_t>(stream);
    return FMM_OK;
}

fmm_status fmm_potential(fmm_plan_t plan, const double* xy, const double* q, double* phi) {
    if (!plan || !xy || !q || !phi) return FMM_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    return enqueue(plan, xy, q, phi);
}

fmm_status fmm_potential_field(fmm_plan_t plan, const double* xy, const double* q, double* phi, double* field) {
    if (!plan || !xy || !q || !phi || !field) return FMM_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    return enqueue(plan, xy, q, phi, field);
}

fmm_status fmm_potential_host_async(fmm_plan_t plan, const double* xy_host, const double* q_host, double* phi_host) {
    if (!plan || !xy_host || !q_host || !phi_host) return FMM_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    cudaStream_t st = plan->stream;
    const size_t n = (size_t)plan->n;
    const int b = plan->stage_next;
    double *xy = plan->d_xy_stage[b], *q = plan->d_q_stage[b], *phi = plan->d_phi_stage[b];
    fmm_status s;
    if (plan->precision == FMM_FP64 || plan->serial) {
        // one stream: upload, method, download in turn
        if (cudaMemcpyAsync(xy, xy_host, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(q, q_host, sizeof(double) * n, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return FMM_ERR_CUDA;
        if ((s = enqueue(plan, xy, q, phi)) != FMM_OK) return s;
        if (cudaMemcpyAsync(phi_host, phi, sizeof(double) * n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return FMM_ERR_CUDA;
    } else {
        // Mixed path.  Upload stream: once this set's inputs are free (the call two back scattered
        // them) and the previous call's sort has released the keys, ranks and populations, the
        // inputs go up in chunks, each binned as it lands -- beside the previous call's compute.
        // Plan's stream: the rest of the method once the uploads are in (and, before L2P writes this
        // set's phi, once the call two back has downloaded it).  Download stream: phi, after L2P.
        cudaStream_t up = plan->s_up, down = plan->s_down;
        if (cudaStreamWaitEvent(up, plan->ev_stage_free[b], 0) != cudaSuccess ||
            cudaStreamWaitEvent(up, plan->ev_sorted, 0) != cudaSuccess)
            return FMM_ERR_CUDA;
        const bool reset = !plan->clean;   // a failed earlier call: the populations are reset first
        if ((s = enqueue_prologue(plan)) != FMM_OK) return s;
        if (reset && (cudaEventRecord(plan->ev_fork, st) != cudaSuccess ||
                      cudaStreamWaitEvent(up, plan->ev_fork, 0) != cudaSuccess))
            return FMM_ERR_CUDA;
        const int chunks = n >= kHostChunkMin ? kHostChunks : 1;
        for (int c = 0; c < chunks; ++c) {
            const size_t i0 = n * c / chunks, i1 = n * (c + 1) / chunks;
            if (cudaMemcpyAsync(xy + 2 * i0, xy_host + 2 * i0, sizeof(double) * 2 * (i1 - i0), cudaMemcpyHostToDevice,
                                up) != cudaSuccess ||
                cudaMemcpyAsync(q + i0, q_host + i0, sizeof(double) * (i1 - i0), cudaMemcpyHostToDevice, up) !=
                    cudaSuccess ||
                fmm_launch_bin_range(plan, xy, q, (int64_t)i0, (int64_t)i1, up) < 0)
                return FMM_ERR_CUDA;
        }
        if (cudaEventRecord(plan->ev_up_done, up) != cudaSuccess ||
            cudaStreamWaitEvent(st, plan->ev_up_done, 0) != cudaSuccess ||
            cudaStreamWaitEvent(st, plan->ev_down_done[b], 0) != cudaSuccess)
            return FMM_ERR_CUDA;
        plan->host_chunks = chunks;
        s = enqueue(plan, xy, q, phi, nullptr, true);
        plan->host_chunks = 0;
        if (s != FMM_OK) return s;
        if (cudaEventRecord(plan->ev_l2p_done, st) != cudaSuccess ||
            cudaStreamWaitEvent(down, plan->ev_l2p_done, 0) != cudaSuccess ||
            cudaMemcpyAsync(phi_host, phi, sizeof(double) * n, cudaMemcpyDeviceToHost, down) != cudaSuccess ||
            cudaEventRecord(plan->ev_down_done[b], down) != cudaSuccess)
            return FMM_ERR_CUDA;
    }
    plan->stage_next = b ^ 1;
    return FMM_OK;
}

fmm_status fmm_potential_host(fmm_plan_t plan, const double* xy_host, const double* q_host, double* phi_host) {
    const fmm_status s = fmm_potential_host_async(plan, xy_host, q_host, phi_host);
    if (s != FMM_OK) return s;
    return fmm_sync(plan);
}

fmm_status fmm_sync(fmm_plan_t plan) {
    if (!plan) return FMM_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    cudaStream_t st = plan->stream;
    if (cudaMemcpyAsync(plan->h_status, plan->d_status, sizeof(unsigned int), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(plan->h_counters, plan->d_counters, 2 * FMM_COUNTER_SLOTS * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemsetAsync(plan->d_status, 0, sizeof(unsigned int), st) != cudaSuccess)
        return FMM_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FMM_ERR_CUDA;
    if (plan->s_down && cudaStreamSynchronize(plan->s_down) != cudaSuccess) return FMM_ERR_CUDA;
    if (plan->events_recorded) {
        auto span = [&](int a, int b) -> double {
            float t = 0.f;
            return cudaEventElapsedTime(&t, plan->ev[a], plan->ev[b]) == cudaSuccess ? (double)t : 0.0;
        };
        const int kb = plan->ev_kernels;
        plan->last.ms_total = span(0, 5);
        plan->last.ms_sort = span(0, 1);
        plan->last.ms_m2l_tc = (kb & 1) ? span(6, 7) : 0.0;
        plan->last.ms_p2p_kernel = (kb & 2) ? span(8, 9) : 0.0;
        if (plan->precision == FMM_FP64) {
            plan->last.ms_p2m = span(1, 2);
            plan->last.ms_m2l = span(2, 3);
            plan->last.ms_l2p = span(3, 4);
            plan->last.ms_p2p = span(4, 5);
            plan->last.ms_p2m_fine = plan->last.ms_p2m_coarse = plan->last.ms_m2l_coarse = 0.0;
            plan->last.ms_m2l_fine = plan->last.ms_m2l;
        } else {
            // three streams overlap: each stage is the sum of its kernels' own spans
            plan->last.ms_p2m_fine = span(1, 2);
            plan->last.ms_p2m_coarse = (kb & 4) ? span(10, 11) : 0.0;
            plan->last.ms_m2l_fine = span(14, 3);
            plan->last.ms_m2l_coarse = (kb & 8) ? span(12, 13) : 0.0;
            plan->last.ms_p2m = plan->last.ms_p2m_fine + plan->last.ms_p2m_coarse;
            plan->last.ms_m2l = plan->last.ms_m2l_fine + plan->last.ms_m2l_coarse;
            plan->last.ms_l2p = span(4, 5) + ((kb & 16) ? span(15, 16) : 0.0);
            plan->last.ms_p2p = plan->last.ms_p2p_kernel;
        }
        plan->ev_kernels = 0;
        unsigned long long pairs = 0, mx = 0;
        for (int c = 0; c < FMM_COUNTER_SLOTS; ++c) {
            pairs += plan->h_counters[c];
            mx = plan->h_counters[FMM_COUNTER_SLOTS + c] > mx ? plan->h_counters[FMM_COUNTER_SLOTS + c] : mx;
        }
        plan->last.p2p_pairs = (int64_t)pairs;
        plan->last.max_leaf = (int64_t)mx;
        plan->last.kernel_launches = plan->launches;
        plan->events_recorded = 0;
    }
    const unsigned int f = *plan->h_status;
    if (f & FMM_FLAG_NONFINITE) return FMM_ERR_NONFINITE;
    if (f & FMM_FLAG_OUT_OF_BOX) return FMM_ERR_OUT_OF_BOX;
    if (f & FMM_FLAG_TIMEOUT) return FMM_ERR_TIMEOUT;
    return FMM_OK;
}

fmm_status fmm_leaf_keys(fmm_plan_t plan, uint32_t* keys) {
    if (!plan || !keys) return FMM_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    return cudaMemcpyAsync(keys, plan->keys, sizeof(uint32_t) * (size_t)plan->n, cudaMemcpyDeviceToDevice,
                           plan->stream) == cudaSuccess ? FMM_OK : FMM_ERR_CUDA;
}

fmm_status fmm_inject_timeout(fmm_plan_t plan, int enable) {
    if (!plan) return FMM_ERR_INVALID_ARG;
    if (plan->tc == nullptr || plan->levels < fmm_tc_kmin()) return FMM_ERR_UNSUPPORTED;
    plan->test_stall = enable != 0;
    return FMM_OK;
}

fmm_status fmm_plan_stats(fmm_plan_t plan, fmm_stats* out) {
    if (!plan || !out) return FMM_ERR_INVALID_ARG;
    *out = plan->last;
    return FMM_OK;
}

void fmm_plan_destroy(fmm_plan_t plan) {
    if (!plan) return;
    cudaStreamSynchronize(plan->stream);
    free_plan(plan);
}

fmm_status fmm_direct_targets(int64_t n, const double* xy, const double* q, int64_t n_targets,
                              const int64_t* targets, double* phi_t, void* stream) {
    if (n < 0 || n_targets < 0 || n_targets > 2147483647LL) return FMM_ERR_INVALID_ARG;
    if (n_targets > 0 && (!targets || !phi_t || n == 0 || !xy || !q)) return FMM_ERR_INVALID_ARG;
    int r = fmm_launch_direct_f64(n, xy, q, n_targets, targets, phi_t, static_cast<cudaStream_t>(stream));
    return r < 0 ? FMM_ERR_CUDA : FMM_OK;
}

}  // extern "C"
