// closure_api.cu -- C ABI of the MLP closure: parameters, normalisation,
// GPU training (mini-batch Adam over a shuffled data set), gradients for
// checking, prediction, and the feature / target kernels on packed coarse
// states.  The lattice-side calls (mhd_set_closure, mhd_closure_filter) are
// in api.cu.  Not part of the paper.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/mhd.h"
#include "closure_internal.h"

namespace {

mhd_status cfail(mhd_status s, const std::string& m) {
    mhd::set_last_error(m);
    return s;
}
mhd_status ccuda(cudaError_t e, const char* what) {
    return cfail(e == cudaErrorMemoryAllocation ? MHD_ENOMEM : MHD_ECUDA,
                 std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}
#define CCK(call, what)                                \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return ccuda(e_, what); \
    } while (0)

unsigned long long splitmix(unsigned long long& s) {
    s += 0x9E3779B97F4A7C15ULL;
    unsigned long long z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
double uniform01(unsigned long long& s) { return (double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0); }

constexpr int kStatBlocks = 256;

}  // namespace

struct mhd_mlp {
    int dev = 0;
    cudaStream_t stream = nullptr;
    int max_rows = 0;
    float *prm = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    double* statp = nullptr;
    float* tpart = nullptr;      // per-block gradient partials of a training step
    double* tlossp = nullptr;    // per-block loss sums of a training step
    long long* t_d = nullptr;    // Adam step count while a training graph runs
    double* loss_acc = nullptr;  // the epoch's loss, summed on the device
    cudaStream_t cap = nullptr;  // private stream for graph capture
    mhd::MlpDev d{};
    std::vector<void*> allocs;
    long long t = 0;
};

namespace {

template <typename T> mhd_status alloc(mhd_mlp* m, T** p, size_t count) {
    void* q = nullptr;
    CCK(cudaMalloc(&q, sizeof(T) * count), "cudaMalloc(mlp)");
    CCK(cudaMemset(q, 0, sizeof(T) * count), "cudaMemset(mlp)");
    m->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return MHD_OK;
}

#define CALLOC(ptr, count)                        \
    do {                                          \
        mhd_status s_ = alloc(m, &(ptr), (count)); \
        if (s_ != MHD_OK) return s_;              \
    } while (0)

mhd_status mlp_buffers(mhd_mlp* m) {
    using namespace mhd;
    const size_t R = (size_t)m->max_rows;
    CALLOC(m->prm, kBlob); CALLOC(m->m, kBlob); CALLOC(m->v, kBlob); CALLOC(m->grad, kBlob);
    CALLOC(m->t_d, 1);
    CALLOC(m->loss_acc, 1);
    CALLOC(m->statp, (size_t)kStatBlocks * 2 * (kIn + kOut));
    CALLOC(m->tpart, (size_t)train_blocks(m->max_rows) * kBlob);
    CALLOC(m->tlossp, (size_t)train_blocks(m->max_rows));
    MlpDev& d = m->d;
    CALLOC(d.Wt1, kHid * kInPad); CALLOC(d.W1, kInPad * kHid);
    CALLOC(d.Wt2, kHid * kHid); CALLOC(d.W2, kHid * kHid);
    CALLOC(d.Wt3, kOutPad * kHid); CALLOC(d.W3, kHid * kOutPadK);
    CALLOC(d.b1, kHid); CALLOC(d.b2, kHid); CALLOC(d.b3, kOutPad);
    CALLOC(d.xb, R * kInPad); CALLOC(d.tb, R * kOut);
    CALLOC(d.Z1, R * kHid); CALLOC(d.H1, R * kHid);
    CALLOC(d.Z2, R * kHid); CALLOC(d.H2, R * kHid);
    CALLOC(d.Y, R * kOutPad);
    return MHD_OK;
}

// He-normal initial weights (Box-Muller on SplitMix64), zero biases, unit
// normalisation.
std::vector<float> initial_params(unsigned long long seed) {
    using namespace mhd;
    std::vector<float> p(kBlob, 0.f);
    for (int c = 0; c < kIn; ++c) p[kOffScale + c] = 1.f;
    for (int c = 0; c < kOut; ++c) p[kOffOutScale + c] = 1.f;
    unsigned long long s = seed;
    auto normal = [&]() {
        const double u1 = std::max(uniform01(s), 1e-300), u2 = uniform01(s);
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    };
    for (int i = 0; i < kIn * kHid; ++i) p[kOffW1 + i] = (float)(normal() * std::sqrt(2.0 / kIn));
    for (int i = 0; i < kHid * kHid; ++i) p[kOffW2 + i] = (float)(normal() * std::sqrt(2.0 / kHid));
    for (int i = 0; i < kHid * kOut; ++i) p[kOffW3 + i] = (float)(normal() * std::sqrt(2.0 / kHid));
    return p;
}

int rows_of(long long n) { return (int)((n + 15) / 16 * 16); }

}  // namespace

void mhd_internal_closure_params(const mhd_mlp* m, mhd::ClosureParamsDev* cp) {
    cp->Wt1 = m->d.Wt1; cp->Wt2 = m->d.Wt2; cp->Wt3 = m->d.Wt3;
    cp->b1 = m->d.b1; cp->b2 = m->d.b2; cp->b3 = m->d.b3;
    cp->mean = m->prm + mhd::kOffMean; cp->scale = m->prm + mhd::kOffScale;
    cp->out_scale = m->prm + mhd::kOffOutScale;
}

extern "C" {

mhd_status mhd_mlp_create(unsigned long long seed, int max_batch, void* stream, mhd_mlp** out) {
    if (!out) return cfail(MHD_EINVAL, "out is NULL");
    *out = nullptr;
    if (max_batch < 16 || max_batch > (1 << 24)) return cfail(MHD_EINVAL, "max_batch must be in [16, 2^24]");
    auto* m = new (std::nothrow) mhd_mlp();
    if (!m) return cfail(MHD_ENOMEM, "host allocation failed");
    m->stream = static_cast<cudaStream_t>(stream);
    m->max_rows = rows_of(max_batch);
    cudaError_t e = cudaGetDevice(&m->dev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = mhd::prepare_train_kernels();
    mhd_status s = e == cudaSuccess ? mlp_buffers(m) : ccuda(e, "mhd_mlp_create");
    if (s == MHD_OK) {
        std::vector<float> p = initial_params(seed);
        e = cudaMemcpy(m->prm, p.data(), sizeof(float) * p.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = mhd::launch_refresh(m->prm, m->d, m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) s = ccuda(e, "mhd_mlp_create");
    }
    if (s != MHD_OK) {
        mhd_mlp_destroy(m);
        return s;
    }
    *out = m;
    return MHD_OK;
}

mhd_status mhd_mlp_destroy(mhd_mlp* m) {
    if (!m) return cfail(MHD_EINVAL, "mlp is NULL");
    cudaSetDevice(m->dev);
    cudaStreamSynchronize(m->stream);
    for (void* p : m->allocs) cudaFree(p);
    if (m->cap) cudaStreamDestroy(m->cap);
    delete m;
    return MHD_OK;
}

mhd_status mhd_mlp_get_params(const mhd_mlp* m, float* host, size_t count) {
    if (!m || !host) return cfail(MHD_EINVAL, "NULL argument");
    if (count != (size_t)mhd::kBlob) return cfail(MHD_EINVAL, "count must be MHD_MLP_PARAMS");
    CCK(cudaSetDevice(m->dev), "cudaSetDevice");
    CCK(cudaMemcpyAsync(host, m->prm, sizeof(float) * count, cudaMemcpyDeviceToHost, m->stream), "D2H params");
    CCK(cudaStreamSynchronize(m->stream), "mhd_mlp_get_params");
    return MHD_OK;
}

mhd_status mhd_mlp_set_params(mhd_mlp* m, const float* host, size_t count) {
    if (!m || !host) return cfail(MHD_EINVAL, "NULL argument");
    if (count != (size_t)mhd::kBlob) return cfail(MHD_EINVAL, "count must be MHD_MLP_PARAMS");
    for (size_t i = 0; i < count; ++i)
        if (!std::isfinite(host[i])) return cfail(MHD_EINVAL, "non-finite parameter");
    CCK(cudaSetDevice(m->dev), "cudaSetDevice");
    CCK(cudaMemcpyAsync(m->prm, host, sizeof(float) * count, cudaMemcpyHostToDevice, m->stream), "H2D params");
    CCK(mhd::launch_refresh(m->prm, m->d, m->stream), "refresh weights");
    CCK(cudaMemsetAsync(m->m, 0, sizeof(float) * count, m->stream), "reset Adam");
    CCK(cudaMemsetAsync(m->v, 0, sizeof(float) * count, m->stream), "reset Adam");
    CCK(cudaStreamSynchronize(m->stream), "mhd_mlp_set_params");
    m->t = 0;
    return MHD_OK;
}

mhd_status mhd_mlp_fit_normalisation(mhd_mlp* m, const float* X, const float* T, long long n) {
    if (!m || !X || !T || n < 2) return cfail(MHD_EINVAL, "bad argument");
    CCK(cudaSetDevice(m->dev), "cudaSetDevice");
    CCK(mhd::launch_stats(X, T, n, m->statp, kStatBlocks, m->prm, m->stream), "statistics kernels");
    CCK(cudaStreamSynchronize(m->stream), "mhd_mlp_fit_normalisation");
    return MHD_OK;
}

mhd_status mhd_mlp_gradients(mhd_mlp* m, const float* X, const float* T, long long n, float* grad_host,
                             double* loss) {
    if (!m || !X || !T || !grad_host) return cfail(MHD_EINVAL, "NULL argument");
    if (n < 1 || n > m->max_rows) return cfail(MHD_EINVAL, "n must be in [1, max_batch]");
    CCK(cudaSetDevice(m->dev), "cudaSetDevice");
    const int rows = rows_of(n), nblk = mhd::train_blocks(rows);
    CCK(mhd::launch_train_step(X, T, nullptr, (int)n, rows, m->prm, m->d, m->tpart, m->tlossp, nullptr, m->grad,
                               m->m, m->v, 0.f, nullptr, false, m->stream),
        "forward / backward");
    CCK(cudaMemcpyAsync(grad_host, m->grad, sizeof(float) * mhd::kBlob, cudaMemcpyDeviceToHost, m->stream), "D2H");
    std::vector<double> lp((size_t)nblk);
    CCK(cudaMemcpyAsync(lp.data(), m->tlossp, sizeof(double) * nblk, cudaMemcpyDeviceToHost, m->stream), "D2H loss");
    CCK(cudaStreamSynchronize(m->stream), "mhd_mlp_gradients");
    double s = 0;
    for (double v : lp) s += v;
    if (loss) *loss = s / (double)(n * mhd::kOut);
    return MHD_OK;
}

// One epoch -- the sample order (a keyed permutation computed on the GPU),
// then two kernels per batch: the fused forward / backward / weight-gradient
// pass and the Adam update with the weight refresh and the loss
// accumulation (step count on the device) -- recorded once as a CUDA graph
// and replayed every epoch.
static cudaError_t capture_epoch(mhd_mlp* m, const float* X, const float* T, int* idx, long long n, int batch,
                                 float lr, unsigned long long seed, cudaGraphExec_t* exec) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(m->loss_acc, 0, sizeof(double), m->cap);
    if (e == cudaSuccess) e = mhd::launch_epoch_permutation(idx, n, seed, m->t_d, m->cap);
    for (long long b0 = 0; b0 < n && e == cudaSuccess; b0 += batch) {
        const int nb = (int)std::min<long long>(batch, n - b0), rows = rows_of(nb);
        e = mhd::launch_train_step(X, T, idx + b0, nb, rows, m->prm, m->d, m->tpart, m->tlossp, m->t_d, m->grad,
                                   m->m, m->v, lr, m->loss_acc, true, m->cap);
    }
    const cudaError_t ee = cudaStreamEndCapture(m->cap, &g);
    if (e == cudaSuccess) e = ee;
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

mhd_status mhd_mlp_train(mhd_mlp* m, const float* X, const float* T, long long n, int epochs, int batch,
                         float lr, unsigned long long seed, double* last_epoch_loss) {
    if (!m || !X || !T) return cfail(MHD_EINVAL, "NULL argument");
    if (n < 1 || epochs < 1 || batch < 16 || batch > m->max_rows || !(lr > 0))
        return cfail(MHD_EINVAL, "bad n / epochs / batch / lr");
    if (n > (1LL << 31) - 1) return cfail(MHD_EINVAL, "n too large");
    CCK(cudaSetDevice(m->dev), "cudaSetDevice");
    int* idx = nullptr;
    CCK(cudaMalloc(&idx, sizeof(int) * n), "cudaMalloc(index)");
    // the work so far on the caller's stream comes first; the step count
    // continues from the host copy
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e == cudaSuccess) e = cudaMemcpy(m->t_d, &m->t, sizeof(long long), cudaMemcpyHostToDevice);
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = capture_epoch(m, X, T, idx, n, batch, lr, seed, &exec);
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) e = cudaGraphLaunch(exec, m->stream);
    double acc = 0;
    long long t = m->t;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&acc, m->loss_acc, sizeof(double), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&t, m->t_d, sizeof(long long), cudaMemcpyDeviceToHost, m->stream);
    const cudaError_t e2 = cudaStreamSynchronize(m->stream);
    if (exec) cudaGraphExecDestroy(exec);
    cudaFree(idx);
    if (e != cudaSuccess) return ccuda(e, "mhd_mlp_train");
    if (e2 != cudaSuccess) return ccuda(e2, "mhd_mlp_train");
    m->t = t;
    const double epoch_loss = acc / (double)(n * mhd::kOut);
    if (last_epoch_loss) *last_epoch_loss = epoch_loss;
    if (!std::isfinite(epoch_loss)) return cfail(MHD_EUNSTABLE, "training loss is not finite");
    return MHD_OK;
}

mhd_status mhd_mlp_predict(mhd_mlp* m, const float* X, long long n, float* Y) {
    if (!m || !X || !Y || n < 1) return cfail(MHD_EINVAL, "bad argument");
    CCK(cudaSetDevice(m->dev), "cudaSetDevice");
    for (long long b0 = 0; b0 < n; b0 += m->max_rows) {
        const int nb = (int)std::min<long long>(m->max_rows, n - b0), rows = rows_of(nb);
        CCK(mhd::launch_gather_batch(X + b0 * mhd::kIn, nullptr, nullptr, nb, rows, m->prm, m->d, m->stream),
            "gather");
        CCK(mhd::launch_mlp_predict(m->d, rows, nb, m->prm, Y + b0 * mhd::kOut, m->stream), "predict");
    }
    CCK(cudaStreamSynchronize(m->stream), "mhd_mlp_predict");
    return MHD_OK;
}

mhd_status mhd_closure_features(const float* state, int nx, int ny, double rho0, float* X, void* stream) {
    if (!state || !X || nx < 2 || ny < 2) return cfail(MHD_EINVAL, "bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CCK(mhd::launch_features(state, nx, ny, (float)rho0, X, st), "features kernel");
    CCK(cudaStreamSynchronize(st), "mhd_closure_features");
    return MHD_OK;
}

mhd_status mhd_closure_targets(const float* state_t, const float* state_t1, int nx, int ny, double rho0,
                               double tau_f, float* T, void* stream) {
    if (!state_t || !state_t1 || !T || nx < 2 || ny < 2 || !(tau_f > 0.5)) return cfail(MHD_EINVAL, "bad argument");
    if (std::fabs(1.0 - 1.0 / tau_f) < 1e-12) return cfail(MHD_EINVAL, "tau_f = 1 leaves a1^(2) unrecoverable");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CCK(mhd::launch_targets(state_t, state_t1, nx, ny, rho0, 1.0 / tau_f, T, st), "targets kernel");
    CCK(cudaStreamSynchronize(st), "mhd_closure_targets");
    return MHD_OK;
}

}  // extern "C"
