// noalloc.cu -- fmm_potential_noalloc: the FP64 path with every workspace in a fixed,
// file-scope device array, for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs after an application has fixed its
// memory budget (a real-time or embedded loop that forbids allocation after start-up), code
// that shares a device with an allocator that owns all free memory (a framework's caching
// pool), or a plugin that may not create allocations of its own.  fmm_potential needs a plan,
// and fmm_plan allocates; this entry point needs none.  Its scratch is the static array below,
// which the CUDA runtime reserves on a device when the library's module is loaded there and
// keeps until the process exits.  With lazy module loading (the CUDA default) that happens at
// the first use of the library on the device -- this entry point's first call, or the first
// library kernel -- so a caller whose allocator claims the free memory later should make one
// call first.
//
// Host code sees `g_noalloc_scratch` only as a host-side stand-in symbol, not as a device
// address: a kernel handed that name faults or, where the GPU can reach host memory, uses the
// wrong memory.  The device address is therefore looked up once per device, with that device
// current, by cudaGetSymbolAddress, and passed to the kernels.
#include <mutex>

#include "fmm_internal.cuh"

namespace {

// Limits of the no-allocation path and the scratch they need (each sub-buffer 256-byte aligned):
// particles <= 65536, levels <= 6, p <= 20.  Worst case about 8.0 MB; the array holds 8.5 MB.
constexpr int64_t kMaxN = 65536;
constexpr int kMaxLevels = 6;
constexpr int kMaxP = 20;
constexpr size_t kScratchBytes = (size_t)8704 * 1024;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};
cudaEvent_t g_events[kMaxDevices][6] = {};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Scale-free FP64 M2L operators on power-sum moments, built on the device so that the call
// needs neither a host buffer nor a host-to-device copy; the same formulas as the plan's
// host-side build (Greengard's 2D conversion, ref. [101] of the paper):
//   T[d][k][l], d = (dx + 3) + 7 (dy + 3), w0 = dx + i dy:
//   T[0][0] = log(-w0), T[0][l] = -w0^-l / l, T[k][0] = (-1)^(k+1) w0^-k / k,
//   T[k][l] = (-1)^(k+1) C(l+k-1, k-1) w0^-(l+k) / k;  zero for the nine adjacent offsets.
__global__ void k_build_ops_f64(int p, double2* __restrict__ T) {
    const int p1 = p + 1;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 49 * p1 * p1) return;
    const int d = e / (p1 * p1), k = (e / p1) % p1, l = e % p1;
    const int dx = d % 7 - 3, dy = d / 7 - 3;
    if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) {
        T[e] = make_double2(0.0, 0.0);
        return;
    }
    const double r2 = (double)(dx * dx + dy * dy);
    const double ivr = (double)dx / r2, ivi = -(double)dy / r2;   // 1 / w0
    if (k == 0 && l == 0) {
        T[e] = make_double2(0.5 * log(r2), atan2(-(double)dy, -(double)dx));
        return;
    }
    double pr = 1.0, pi = 0.0;   // w0^-(l+k)
    for (int m = 0; m < l + k; ++m) {
        const double nr = pr * ivr - pi * ivi;
        const double ni = pr * ivi + pi * ivr;
        pr = nr;
        pi = ni;
    }
    double c;
    if (k == 0) {
        c = -1.0 / (double)l;
    } else {
        double b = 1.0;   // C(l+k-1, k-1) by the multiplicative formula (exact for these sizes)
        for (int i = 1; i <= k - 1; ++i) b = b * (double)(l + i) / (double)i;
        c = ((k & 1) ? 1.0 : -1.0) * b / (double)k;
    }
    T[e] = make_double2(c * pr, c * pi);
}

// Carve the plan's workspaces out of the scratch block; returns the bytes used.
size_t carve(fmm_plan_s* pl, unsigned char* base) {
    const int64_t n = pl->n;
    const int L = pl->levels, p1 = pl->p + 1;
    const int64_t m = (int64_t)1 << (2 * L);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char* ptr = base ? base + off : nullptr;
        off = align256(off + bytes);
        return ptr;
    };
    pl->keys = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * n));
    pl->rank = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * n));
    pl->counts = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * m));
    pl->leaf_start = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (m + 1)));
    pl->scan_blocks = fmm_scan_blocks(m);
    pl->block_sums = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (pl->scan_blocks + 1)));
    pl->sorted_key = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * n));
    pl->sorted64 = reinterpret_cast<fmm_p64*>(take(sizeof(fmm_p64) * n));
    pl->phi_far = reinterpret_cast<double*>(take(sizeof(double) * n));
    for (int k = 2; k <= L; ++k) {
        const size_t W = (size_t)fmm_grid_width(k);
        pl->a_bytes[k] = W * W * p1 * sizeof(double2);
        pl->grids.A[k] = take(pl->a_bytes[k]);
        pl->grids.B[k] = take(((size_t)1 << (2 * k)) * p1 * sizeof(double2));
    }
    pl->T64 = reinterpret_cast<double2*>(take(sizeof(double2) * 49 * p1 * p1));
    pl->d_status = reinterpret_cast<unsigned int*>(take(sizeof(unsigned int)));
    pl->d_counters = reinterpret_cast<unsigned long long*>(take(2 * FMM_COUNTER_SLOTS * sizeof(unsigned long long)));
    return off;
}

// Once per device, with that device current: the scratch block's device address and the
// (memory-free) events the stage launchers record.
fmm_status setup(int dev, void** scratch, cudaEvent_t** events) {
    if (dev < 0 || dev >= kMaxDevices) return FMM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        const cudaError_t r = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (r != cudaSuccess || !ptr) {
            // the module (and with it the array) could not be loaded on this device
            return r == cudaErrorMemoryAllocation ? FMM_ERR_OOM : FMM_ERR_CUDA;
        }
        for (int e = 0; e < 6; ++e)
            if (cudaEventCreate(&g_events[dev][e]) != cudaSuccess) {
                for (int f = 0; f < e; ++f) {   // a later call starts the set-up again
                    cudaEventDestroy(g_events[dev][f]);
                    g_events[dev][f] = nullptr;
                }
                return FMM_ERR_CUDA;
            }
        g_scratch_ptr[dev] = ptr;
    }
    *scratch = g_scratch_ptr[dev];
    *events = g_events[dev];
    return FMM_OK;
}

}  // namespace

extern "C" fmm_status fmm_potential_noalloc(int64_t n, int levels, int p, double box, const double* xy,
                                            const double* q, double* phi, void* stream) {
    if (n < 1 || n > kMaxN || levels < 0 || levels > kMaxLevels || p < 1 || p > kMaxP || !(box > 0.0) ||
        !(box < 1e300) || !xy || !q || !phi)
        return FMM_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FMM_ERR_CUDA;
    void* scratch = nullptr;
    cudaEvent_t* events = nullptr;
    fmm_status s = setup(dev, &scratch, &events);
    if (s != FMM_OK) return s;

    fmm_plan_s pl{};
    pl.device = dev;
    pl.n = n;
    pl.levels = levels;
    pl.p = p;
    pl.box = box;
    pl.precision = FMM_FP64;
    pl.stream = static_cast<cudaStream_t>(stream);
    if (carve(&pl, nullptr) > kScratchBytes) return FMM_ERR_INVALID_ARG;   // cannot happen within the limits
    carve(&pl, static_cast<unsigned char*>(scratch));
    for (int e = 0; e < 6; ++e) pl.ev[e] = events[e];

    // The array keeps the previous call's contents: clear what must start at zero.
    cudaStream_t st = pl.stream;
    if (cudaMemsetAsync(pl.d_status, 0, sizeof(unsigned int), st) != cudaSuccess ||
        cudaMemsetAsync(pl.d_counters, 0, 2 * FMM_COUNTER_SLOTS * sizeof(unsigned long long), st) != cudaSuccess)
        return FMM_ERR_CUDA;
    const int nops = 49 * (p + 1) * (p + 1);
    // an error left pending by the caller's own earlier work is not this call's to report or clear
    if (cudaPeekAtLastError() != cudaSuccess) return FMM_ERR_CUDA;
    k_build_ops_f64<<<(nops + 255) / 256, 256, 0, st>>>(p, pl.T64);
    if (cudaPeekAtLastError() != cudaSuccess) return FMM_ERR_CUDA;
    cudaEventRecord(pl.ev[0], st);
    if (fmm_launch_sort(&pl, xy, q) < 0 || fmm_launch_fp64(&pl, phi) < 0) return FMM_ERR_CUDA;

    // Wait for the stream and report what the device checks found (phi is unwritten then).
    unsigned int flags = 0;
    if (cudaMemcpyAsync(&flags, pl.d_status, sizeof(unsigned int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return FMM_ERR_CUDA;
    if (flags & FMM_FLAG_NONFINITE) return FMM_ERR_NONFINITE;
    if (flags & FMM_FLAG_OUT_OF_BOX) return FMM_ERR_OUT_OF_BOX;
    return FMM_OK;
}
