// selector.cu -- the learned (levels, p) selector: occupancy statistics and a small MLP with
// hand-written forward, backward and Adam kernels.
//
// Features of a particle system (computed on the device from xy): for every level k = 3..11 of
// the uniform quadtree over [0, box]^2, the fraction of squares whose population c falls in bin
// floor(log2(c + 1)) (12 bins, the last one open), plus log2 N / 22.  The network reads these
// features and one candidate (levels, p) and predicts (log10 error / 8, log time in ms) of the
// method at that candidate.  fmm_select evaluates every candidate of a small grid around
// levels = log4(N / 16) and p = 8..32 and returns the cheapest one whose predicted error meets
// the requested accuracy with a margin, or the fixed fallback (8, 20).
//
// Network: IN -> H -> H -> 2, ReLU, FP32; loss = mean over rows of sum_j (y_j - t_j)^2.
// Parameters are one contiguous buffer [W1 (IN x H) | b1 (H) | W2 (H x H) | b2 (H) | W3 (H x 2) | b3 (2)].
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "fmm_internal.cuh"

namespace {

constexpr int kLevMin = 3, kLevMax = 11, kBins = 12;
constexpr int kHistLevels = kLevMax - kLevMin + 1;
constexpr int kFeat = kHistLevels * kBins + 1;   // 109
constexpr int kIn = kFeat + 2;                   // + candidate levels / 12, p / 32
constexpr int kOut = 2;

// ---------------------------------------------------------------- occupancy statistics
__global__ void k_occ_count(const double2* __restrict__ xy, int64_t n, double box, uint32_t* __restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 p = xy[i];
    const float sob = (float)((double)(1 << kLevMax) / box);
    const int side = 1 << kLevMax;
    const int ix = finest_coord(p.x, (double)side, sob, box, side);
    const int iy = finest_coord(p.y, (double)side, sob, box, side);
    size_t off = 0;
    for (int k = kLevMin; k <= kLevMax; ++k) {
        const int sh = kLevMax - k;
        atomicAdd(&cnt[off + ((size_t)(iy >> sh) << k) + (ix >> sh)], 1u);
        off += (size_t)1 << (2 * k);
    }
}

__global__ void k_occ_hist(const uint32_t* __restrict__ cnt, size_t total, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[kHistLevels * kBins];
    for (int i = threadIdx.x; i < kHistLevels * kBins; i += blockDim.x) h[i] = 0u;
    __syncthreads();
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        int k = kLevMin;
        size_t off = 0;
        while (e >= off + ((size_t)1 << (2 * k))) {
            off += (size_t)1 << (2 * k);
            ++k;
        }
        const uint32_t c = cnt[e];
        const int bin = min(kBins - 1, 31 - __clz(c + 1u));   // floor(log2(c + 1))
        atomicAdd(&h[(k - kLevMin) * kBins + bin], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kHistLevels * kBins; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// ---------------------------------------------------------------- dense layers
// Y[r][o] = b[o] + sum_i X[r][i] W[i][o], optional ReLU
__global__ void k_dense_fwd(const float* __restrict__ X, const float* __restrict__ W, const float* __restrict__ b,
                            float* __restrict__ Y, int rows, int in, int out, int relu) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * out) return;
    const int r = e / out, o = e - r * out;
    float acc = b[o];
    for (int i = 0; i < in; ++i) acc = fmaf(X[(size_t)r * in + i], W[(size_t)i * out + o], acc);
    Y[e] = (relu && acc < 0.f) ? 0.f : acc;
}

// dX[r][i] = (sum_o dY[r][o] W[i][o]) * (Xact[r][i] > 0), the mask of the ReLU that produced X
__global__ void k_dense_bwd_data(const float* __restrict__ dY, const float* __restrict__ W,
                                 const float* __restrict__ Xact, float* __restrict__ dX, int rows, int in, int out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * in) return;
    const int r = e / in, i = e - r * in;
    float acc = 0.f;
    for (int o = 0; o < out; ++o) acc = fmaf(dY[(size_t)r * out + o], W[(size_t)i * out + o], acc);
    dX[e] = Xact[e] > 0.f ? acc : 0.f;
}

// dW[i][o] = sum_r X[r][i] dY[r][o]; db[o] = sum_r dY[r][o] (threads i == in hold db)
__global__ void k_dense_bwd_weight(const float* __restrict__ X, const float* __restrict__ dY, float* __restrict__ dW,
                                   float* __restrict__ db, int rows, int in, int out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (in + 1) * out) return;
    const int i = e / out, o = e - i * out;
    float acc = 0.f;
    if (i < in) {
        for (int r = 0; r < rows; ++r) acc = fmaf(X[(size_t)r * in + i], dY[(size_t)r * out + o], acc);
        dW[(size_t)i * out + o] = acc;
    } else {
        for (int r = 0; r < rows; ++r) acc += dY[(size_t)r * out + o];
        db[o] = acc;
    }
}

// loss rows and dL/dY for L = (1 / rows) sum_r sum_j (Y - T)^2
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ dY,
                      float* __restrict__ lrow, int rows) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    float l = 0.f;
    for (int j = 0; j < kOut; ++j) {
        const float d = Y[r * kOut + j] - T[r * kOut + j];
        l = fmaf(d, d, l);
        dY[r * kOut + j] = 2.f * d / (float)rows;
    }
    lrow[r] = l;
}

// Adam (Kingma & Ba, 2015) with bias correction
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int np, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

unsigned nblk(int64_t n, int t = 128) { return (unsigned)((n + t - 1) / t); }

}  // namespace

struct fmm_selector_s {
    int device, hidden, np;
    cudaStream_t stream;
    float *w, *g, *m, *v;            // parameters, gradients, Adam moments
    int adam_t;
    // activations for a batch of up to cap rows
    int cap;
    float *x, *h1, *h2, *y, *t, *dy, *dh2, *dh1, *lrow;
    uint32_t* cnt;                   // occupancy counters of levels 3..11
    uint32_t* hist;
    size_t ncnt;
};

namespace {

int offW1(const fmm_selector_s* s) { return 0; }
int offb1(const fmm_selector_s* s) { return kIn * s->hidden; }
int offW2(const fmm_selector_s* s) { return offb1(s) + s->hidden; }
int offb2(const fmm_selector_s* s) { return offW2(s) + s->hidden * s->hidden; }
int offW3(const fmm_selector_s* s) { return offb2(s) + s->hidden; }
int offb3(const fmm_selector_s* s) { return offW3(s) + s->hidden * kOut; }

void sel_free_acts(fmm_selector_s* s) {
    float* bufs[] = {s->x, s->h1, s->h2, s->y, s->t, s->dy, s->dh2, s->dh1, s->lrow};
    for (float* b : bufs)
        if (b) cudaFree(b);
    s->x = s->h1 = s->h2 = s->y = s->t = s->dy = s->dh2 = s->dh1 = s->lrow = nullptr;
    s->cap = 0;
}

fmm_status sel_reserve(fmm_selector_s* s, int rows) {
    if (rows <= s->cap) return FMM_OK;
    sel_free_acts(s);
    const size_t H = s->hidden;
    bool ok = cudaMalloc(&s->x, sizeof(float) * rows * kIn) == cudaSuccess &&
              cudaMalloc(&s->h1, sizeof(float) * rows * H) == cudaSuccess &&
              cudaMalloc(&s->h2, sizeof(float) * rows * H) == cudaSuccess &&
              cudaMalloc(&s->y, sizeof(float) * rows * kOut) == cudaSuccess &&
              cudaMalloc(&s->t, sizeof(float) * rows * kOut) == cudaSuccess &&
              cudaMalloc(&s->dy, sizeof(float) * rows * kOut) == cudaSuccess &&
              cudaMalloc(&s->dh2, sizeof(float) * rows * H) == cudaSuccess &&
              cudaMalloc(&s->dh1, sizeof(float) * rows * H) == cudaSuccess &&
              cudaMalloc(&s->lrow, sizeof(float) * rows) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        sel_free_acts(s);
        return FMM_ERR_OOM;
    }
    s->cap = rows;
    return FMM_OK;
}

void forward(fmm_selector_s* s, int rows) {
    const int H = s->hidden;
    cudaStream_t st = s->stream;
    k_dense_fwd<<<nblk((int64_t)rows * H), 128, 0, st>>>(s->x, s->w + offW1(s), s->w + offb1(s), s->h1, rows, kIn, H, 1);
    k_dense_fwd<<<nblk((int64_t)rows * H), 128, 0, st>>>(s->h1, s->w + offW2(s), s->w + offb2(s), s->h2, rows, H, H, 1);
    k_dense_fwd<<<nblk((int64_t)rows * kOut), 128, 0, st>>>(s->h2, s->w + offW3(s), s->w + offb3(s), s->y, rows, H,
                                                            kOut, 0);
}

void backward(fmm_selector_s* s, int rows) {
    const int H = s->hidden;
    cudaStream_t st = s->stream;
    k_mse<<<nblk(rows), 128, 0, st>>>(s->y, s->t, s->dy, s->lrow, rows);
    k_dense_bwd_weight<<<nblk((int64_t)(H + 1) * kOut), 128, 0, st>>>(s->h2, s->dy, s->g + offW3(s), s->g + offb3(s),
                                                                     rows, H, kOut);
    k_dense_bwd_data<<<nblk((int64_t)rows * H), 128, 0, st>>>(s->dy, s->w + offW3(s), s->h2, s->dh2, rows, H, kOut);
    k_dense_bwd_weight<<<nblk((int64_t)(H + 1) * H), 128, 0, st>>>(s->h1, s->dh2, s->g + offW2(s), s->g + offb2(s),
                                                                  rows, H, H);
    k_dense_bwd_data<<<nblk((int64_t)rows * H), 128, 0, st>>>(s->dh2, s->w + offW2(s), s->h1, s->dh1, rows, H, H);
    k_dense_bwd_weight<<<nblk((int64_t)(kIn + 1) * H), 128, 0, st>>>(s->x, s->dh1, s->g + offW1(s), s->g + offb1(s),
                                                                    rows, kIn, H);
}

// deterministic host-side initialisation (He-uniform) from a SplitMix64 stream
void init_weights(const fmm_selector_s* s, uint64_t seed, std::vector<float>& w) {
    w.assign(s->np, 0.f);
    uint64_t st = seed;
    auto next = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    auto fill = [&](int off, int fan_in, int count) {
        const double a = std::sqrt(6.0 / fan_in);
        for (int i = 0; i < count; ++i) w[off + i] = (float)((2.0 * next() - 1.0) * a);
    };
    fill(offW1(s), kIn, kIn * s->hidden);
    fill(offW2(s), s->hidden, s->hidden * s->hidden);
    fill(offW3(s), s->hidden, s->hidden * kOut);
}

void candidate_row(const float* feat, int levels, int p, float* row) {
    memcpy(row, feat, sizeof(float) * kFeat);
    row[kFeat] = (float)levels / 12.f;
    row[kFeat + 1] = (float)p / 32.f;
}

}  // namespace

extern "C" {

int fmm_selector_dims(int* in, int* out, int* feat) {
    if (in) *in = kIn;
    if (out) *out = kOut;
    if (feat) *feat = kFeat;
    return 0;
}

fmm_status fmm_selector_create(fmm_selector_t* out, int hidden, uint64_t seed, void* stream) {
    if (!out || hidden < 1 || hidden > 1024) return FMM_ERR_INVALID_ARG;
    fmm_selector_s* s = new (std::nothrow) fmm_selector_s();
    if (!s) return FMM_ERR_OOM;
    cudaGetDevice(&s->device);
    s->hidden = hidden;
    s->stream = static_cast<cudaStream_t>(stream);
    s->np = kIn * hidden + hidden + hidden * hidden + hidden + hidden * kOut + kOut;
    s->ncnt = 0;
    for (int k = kLevMin; k <= kLevMax; ++k) s->ncnt += (size_t)1 << (2 * k);
    bool ok = cudaMalloc(&s->w, sizeof(float) * s->np) == cudaSuccess &&
              cudaMalloc(&s->g, sizeof(float) * s->np) == cudaSuccess &&
              cudaMalloc(&s->m, sizeof(float) * s->np) == cudaSuccess &&
              cudaMalloc(&s->v, sizeof(float) * s->np) == cudaSuccess &&
              cudaMalloc(&s->cnt, sizeof(uint32_t) * s->ncnt) == cudaSuccess &&
              cudaMalloc(&s->hist, sizeof(uint32_t) * kHistLevels * kBins) == cudaSuccess;
    std::vector<float> w;
    init_weights(s, seed, w);
    ok = ok && cudaMemcpy(s->w, w.data(), sizeof(float) * s->np, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(s->m, 0, sizeof(float) * s->np) == cudaSuccess &&
         cudaMemset(s->v, 0, sizeof(float) * s->np) == cudaSuccess;
    if (!ok) {
        fmm_selector_destroy(s);
        return FMM_ERR_OOM;
    }
    *out = s;
    return FMM_OK;
}

void fmm_selector_destroy(fmm_selector_t s) {
    if (!s) return;
    sel_free_acts(s);
    void* bufs[] = {s->w, s->g, s->m, s->v, s->cnt, s->hist};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete s;
}

int fmm_selector_num_params(fmm_selector_t s) { return s ? s->np : -1; }

// Features of the system xy (device, [n][2]) into feat_host[kFeat]; waits for the stream.
fmm_status fmm_selector_features(fmm_selector_t s, const double* xy, int64_t n, double box, float* feat_host) {
    if (!s || !xy || n < 1 || !feat_host || !(box > 0.0)) return FMM_ERR_INVALID_ARG;
    cudaStream_t st = s->stream;
    if (cudaMemsetAsync(s->cnt, 0, sizeof(uint32_t) * s->ncnt, st) != cudaSuccess ||
        cudaMemsetAsync(s->hist, 0, sizeof(uint32_t) * kHistLevels * kBins, st) != cudaSuccess)
        return FMM_ERR_CUDA;
    k_occ_count<<<nblk(n, 256), 256, 0, st>>>(reinterpret_cast<const double2*>(xy), n, box, s->cnt);
    k_occ_hist<<<1024, 256, 0, st>>>(s->cnt, s->ncnt, s->hist);
    uint32_t h[kHistLevels * kBins];
    if (cudaMemcpyAsync(h, s->hist, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return FMM_ERR_CUDA;
    for (int k = kLevMin; k <= kLevMax; ++k)
        for (int b = 0; b < kBins; ++b)
            feat_host[(k - kLevMin) * kBins + b] = (float)((double)h[(k - kLevMin) * kBins + b] / (double)(1ull << (2 * k)));
    feat_host[kFeat - 1] = (float)(std::log2((double)n) / 22.0);
    return FMM_OK;
}

// Copy parameters in or out (host arrays of fmm_selector_num_params floats).
fmm_status fmm_selector_get_params(fmm_selector_t s, float* host) {
    if (!s || !host) return FMM_ERR_INVALID_ARG;
    return cudaMemcpy(host, s->w, sizeof(float) * s->np, cudaMemcpyDeviceToHost) == cudaSuccess ? FMM_OK : FMM_ERR_CUDA;
}
fmm_status fmm_selector_set_params(fmm_selector_t s, const float* host) {
    if (!s || !host) return FMM_ERR_INVALID_ARG;
    return cudaMemcpy(s->w, host, sizeof(float) * s->np, cudaMemcpyHostToDevice) == cudaSuccess ? FMM_OK : FMM_ERR_CUDA;
}

// Forward pass on rows x [rows][kIn] (host) -> y [rows][kOut] (host).
fmm_status fmm_selector_predict(fmm_selector_t s, const float* x_host, int rows, float* y_host) {
    if (!s || !x_host || !y_host || rows < 1) return FMM_ERR_INVALID_ARG;
    if (sel_reserve(s, rows) != FMM_OK) return FMM_ERR_OOM;
    cudaStream_t st = s->stream;
    if (cudaMemcpyAsync(s->x, x_host, sizeof(float) * rows * kIn, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return FMM_ERR_CUDA;
    forward(s, rows);
    if (cudaMemcpyAsync(y_host, s->y, sizeof(float) * rows * kOut, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return FMM_ERR_CUDA;
    return FMM_OK;
}

// Loss and gradient on (x, t) host arrays; grad_host (may be NULL) receives dL/dparams.
fmm_status fmm_selector_loss_grad(fmm_selector_t s, const float* x_host, const float* t_host, int rows, float* loss,
                                  float* grad_host) {
    if (!s || !x_host || !t_host || rows < 1) return FMM_ERR_INVALID_ARG;
    if (sel_reserve(s, rows) != FMM_OK) return FMM_ERR_OOM;
    cudaStream_t st = s->stream;
    if (cudaMemcpyAsync(s->x, x_host, sizeof(float) * rows * kIn, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(s->t, t_host, sizeof(float) * rows * kOut, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return FMM_ERR_CUDA;
    forward(s, rows);
    backward(s, rows);
    std::vector<float> lr(rows);
    if (cudaMemcpyAsync(lr.data(), s->lrow, sizeof(float) * rows, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return FMM_ERR_CUDA;
    if (grad_host && cudaMemcpyAsync(grad_host, s->g, sizeof(float) * s->np, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return FMM_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FMM_ERR_CUDA;
    if (loss) {
        double a = 0.0;
        for (float l : lr) a += l;
        *loss = (float)(a / rows);
    }
    return FMM_OK;
}

// Full-batch Adam training for `epochs` steps on (x, t) host arrays; loss_out receives the
// final loss.  The Adam step counter persists across calls (training resumes).
fmm_status fmm_selector_train(fmm_selector_t s, const float* x_host, const float* t_host, int rows, int epochs,
                              float lr, float* loss_out) {
    if (!s || !x_host || !t_host || rows < 1 || epochs < 0) return FMM_ERR_INVALID_ARG;
    if (sel_reserve(s, rows) != FMM_OK) return FMM_ERR_OOM;
    cudaStream_t st = s->stream;
    if (cudaMemcpyAsync(s->x, x_host, sizeof(float) * rows * kIn, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(s->t, t_host, sizeof(float) * rows * kOut, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return FMM_ERR_CUDA;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int e = 0; e < epochs; ++e) {
        forward(s, rows);
        backward(s, rows);
        ++s->adam_t;
        const float c1 = 1.f - std::pow(b1, (float)s->adam_t), c2 = 1.f - std::pow(b2, (float)s->adam_t);
        k_adam<<<nblk(s->np), 128, 0, st>>>(s->w, s->g, s->m, s->v, s->np, lr, b1, b2, eps, c1, c2);
    }
    if (cudaGetLastError() != cudaSuccess) return FMM_ERR_CUDA;
    if (loss_out) {
        forward(s, rows);
        k_mse<<<nblk(rows), 128, 0, st>>>(s->y, s->t, s->dy, s->lrow, rows);
        std::vector<float> lr_rows(rows);
        if (cudaMemcpyAsync(lr_rows.data(), s->lrow, sizeof(float) * rows, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return FMM_ERR_CUDA;
        double a = 0.0;
        for (float l : lr_rows) a += l;
        *loss_out = (float)(a / rows);
    }
    return cudaStreamSynchronize(st) == cudaSuccess ? FMM_OK : FMM_ERR_CUDA;
}

// Save / load parameters, Adam moments and step (a small versioned binary file).
fmm_status fmm_selector_save(fmm_selector_t s, const char* path) {
    if (!s || !path) return FMM_ERR_INVALID_ARG;
    std::vector<float> w(s->np), m(s->np), v(s->np);
    if (cudaMemcpy(w.data(), s->w, sizeof(float) * s->np, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(m.data(), s->m, sizeof(float) * s->np, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(v.data(), s->v, sizeof(float) * s->np, cudaMemcpyDeviceToHost) != cudaSuccess)
        return FMM_ERR_CUDA;
    FILE* f = fopen(path, "wb");
    if (!f) return FMM_ERR_INVALID_ARG;
    const int hdr[4] = {0x46534C31 /* "FSL1" */, kIn, s->hidden, s->adam_t};
    bool ok = fwrite(hdr, sizeof(int), 4, f) == 4 && fwrite(w.data(), sizeof(float), s->np, f) == (size_t)s->np &&
              fwrite(m.data(), sizeof(float), s->np, f) == (size_t)s->np &&
              fwrite(v.data(), sizeof(float), s->np, f) == (size_t)s->np;
    fclose(f);
    return ok ? FMM_OK : FMM_ERR_INVALID_ARG;
}

fmm_status fmm_selector_load(fmm_selector_t s, const char* path) {
    if (!s || !path) return FMM_ERR_INVALID_ARG;
    FILE* f = fopen(path, "rb");
    if (!f) return FMM_ERR_INVALID_ARG;
    int hdr[4];
    std::vector<float> w(s->np), m(s->np), v(s->np);
    bool ok = fread(hdr, sizeof(int), 4, f) == 4 && hdr[0] == 0x46534C31 && hdr[1] == kIn && hdr[2] == s->hidden &&
              fread(w.data(), sizeof(float), s->np, f) == (size_t)s->np &&
              fread(m.data(), sizeof(float), s->np, f) == (size_t)s->np &&
              fread(v.data(), sizeof(float), s->np, f) == (size_t)s->np;
    fclose(f);
    if (!ok) return FMM_ERR_INVALID_ARG;
    s->adam_t = hdr[3];
    if (cudaMemcpy(s->w, w.data(), sizeof(float) * s->np, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(s->m, m.data(), sizeof(float) * s->np, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(s->v, v.data(), sizeof(float) * s->np, cudaMemcpyHostToDevice) != cudaSuccess)
        return FMM_ERR_CUDA;
    return FMM_OK;
}

// Pick (levels, p) for the system xy: candidates levels = l0 - 2 .. l0 + 2 (l0 = round(log4(n / 16)),
// clamped to 2..11) x p = 8, 12, ..., 28; the cheapest predicted time among those whose predicted
// log10 error is at most log10(target_err) - margin_decades; else the fallback (8, 20).
fmm_status fmm_select(fmm_selector_t s, const double* xy, int64_t n, double box, double target_err,
                      double margin_decades, int* levels_out, int* p_out, int* used_fallback) {
    if (!s || !xy || n < 1 || !(target_err > 0.0) || !levels_out || !p_out) return FMM_ERR_INVALID_ARG;
    float feat[kFeat];
    fmm_status st = fmm_selector_features(s, xy, n, box, feat);
    if (st != FMM_OK) return st;
    const int l0 = (int)std::lround(std::log((double)n / 16.0) / std::log(4.0));
    std::vector<int> cl, cp;
    for (int l = l0 - 2; l <= l0 + 2; ++l) {
        if (l < 2 || l > 11) continue;
        for (int p = 8; p <= 28; p += 4) {
            cl.push_back(l);
            cp.push_back(p);
        }
    }
    const int rows = (int)cl.size();
    std::vector<float> x((size_t)rows * kIn), y((size_t)rows * kOut);
    for (int r = 0; r < rows; ++r) candidate_row(feat, cl[r], cp[r], &x[(size_t)r * kIn]);
    st = fmm_selector_predict(s, x.data(), rows, y.data());
    if (st != FMM_OK) return st;
    const double lim = (std::log10(target_err) - margin_decades) / 8.0;
    int best = -1;
    for (int r = 0; r < rows; ++r)
        if (y[(size_t)r * kOut] <= lim && (best < 0 || y[(size_t)r * kOut + 1] < y[(size_t)best * kOut + 1])) best = r;
    if (best < 0) {
        *levels_out = 8;
        *p_out = 20;
        if (used_fallback) *used_fallback = 1;
    } else {
        *levels_out = cl[best];
        *p_out = cp[best];
        if (used_fallback) *used_fallback = 0;
    }
    return FMM_OK;
}

}  // extern "C"
