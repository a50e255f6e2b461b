// The learned short-range factor: training on the GPU and validation.
//
// Samples: x_k (24 random bits from a counter-based splitmix64 stream),
// r = x_k rcut, target = the exact factor at r as the PP kernel evaluates it
// (SFU ex2 times the fitted polynomial).  Network input z0 = 2 x_k - 1.
// Each training step draws `batch` sample indices from a second stream,
// computes the mean relative squared error and its gradient (forward and
// backward by hand, FP32), and applies one Adam update with a cosine
// learning-rate schedule.  The step counter lives in device memory, so a run
// of steps is captured once in a CUDA graph and replayed.
//
// Validation evaluates the trained network exactly as the learned PP kernel
// does (warp-level BF16 tensor-core MMAs) on a dense grid of r in [0, rcut)
// and records the largest relative deviation from the exact factor.
#include <cstdio>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "factor.cuh"
#include "handles.cuh"
#include "mlp_handle.cuh"

namespace phpp {

int pp_learned_setup();   // the learned PP kernels' shared-memory opt-in (pp.cu)

void fit_factor_poly(double U, int deg, float *coef);

namespace {

constexpr int kTrainThreads = 128;
constexpr int kTrainWarps = kTrainThreads / 32;
constexpr int kGraphSteps = 64;
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t stream, uint64_t k)
{
    uint64_t z = stream + (k + 1) * kGamma;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ float uniform24(uint64_t stream, uint64_t k)
{
    return (float)(splitmix64(stream, k) >> 40) * (1.0f / 16777216.0f);
}

struct FactorConsts {
    float poly[kMaxPoly + 1];
    int npoly;
    float c_e, rcut;
};

__global__ void k_samples(int64_t n, uint64_t stream, FactorConsts fc, float *z0, float *tgt)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const float x = uniform24(stream, (uint64_t)k);
        const float r = x * fc.rcut;
        const float t = 2.f * x - 1.f;
        z0[k] = t;
        tgt[k] = exact_factor(r * r, t, fc.poly, fc.npoly, fc.c_e);
    }
}

__device__ __forceinline__ float silu_f(float a) { return a / (1.f + __expf(-a)); }
__device__ __forceinline__ float silu_grad_f(float a)
{
    const float s = 1.f / (1.f + __expf(-a));
    return s * (1.f + a * (1.f - s));
}

struct TrainArgs {
    const float *theta;      // [321]
    const float *z0, *tgt;   // samples
    int64_t n_samples;
    uint64_t batch_stream;   // index stream; ~0 = samples 0..batch-1 in order
    const int32_t *step;     // device step counter
    int batch;
    float *partial;          // [gridDim.x][kMlpParams + 1]
};

// Forward + backward over the batch: every lane one sample at a time; the
// warp's per-sample activations go through shared memory so that each lane
// sums ~10 gradient entries over the warp's 32 samples (no atomics: the
// summation order is fixed).
__global__ void __launch_bounds__(kTrainThreads) k_grad(TrainArgs a)
{
    __shared__ float th[kMlpParams];
    __shared__ float s_h1[kTrainWarps][32][17];
    __shared__ float s_h2[kTrainWarps][32][17];
    __shared__ float s_da1[kTrainWarps][32][17];
    __shared__ float s_da2[kTrainWarps][32][17];
    __shared__ float s_z0[kTrainWarps][32];
    __shared__ float s_dy[kTrainWarps][32];
    __shared__ float s_red[kTrainWarps][kMlpParams + 1];   // per-warp gradient sums, then loss
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < kMlpParams; e += kTrainThreads) th[e] = a.theta[e];
    for (int e = lane; e <= kMlpParams; e += 32) s_red[w][e] = 0.f;
    __syncthreads();
    const float *W1 = th, *b1 = th + 16, *W2 = th + 32, *b2 = th + 288, *W3 = th + 304;
    const float b3 = th[320];
    const int step = *a.step;
    float loss = 0.f;
    const int per_block = (a.batch + gridDim.x - 1) / gridDim.x;
    const int lo = blockIdx.x * per_block;
    const int hi = min(a.batch, lo + per_block);
    for (int base = lo + w * 32; base < hi; base += kTrainWarps * 32) {
        const int s = base + lane;
        float z = 0.f, dy = 0.f, tg = 1.f;
        bool ok = s < hi;
        if (ok) {
            int64_t idx = s;
            if (a.batch_stream != ~0ull)
                idx = (int64_t)(splitmix64(a.batch_stream, (uint64_t)step * (uint64_t)a.batch + (uint64_t)s) %
                                (uint64_t)a.n_samples);
            z = a.z0[idx];
            tg = a.tgt[idx];
        }
        // forward; a1 and a2 are parked in the da1 / da2 rows until backward
        float h1[16];
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const float a1 = fmaf(W1[j], z, b1[j]);
            s_da1[w][lane][j] = a1;
            h1[j] = silu_f(a1);
            s_h1[w][lane][j] = h1[j];
        }
        float y = b3;
#pragma unroll 1
        for (int k = 0; k < 16; k++) {
            float t = b2[k];
#pragma unroll
            for (int j = 0; j < 16; j++) t = fmaf(W2[16 * k + j], h1[j], t);
            s_da2[w][lane][k] = t;
            const float h2 = silu_f(t);
            s_h2[w][lane][k] = ok ? h2 : 0.f;
            y = fmaf(W3[k], h2, y);
        }
        if (ok) {
            const float rel = (y - tg) / tg;
            loss += rel * rel;
            dy = 2.f * rel / tg / (float)a.batch;
        }
        // backward
#pragma unroll 1
        for (int k = 0; k < 16; k++) s_da2[w][lane][k] = dy * W3[k] * silu_grad_f(s_da2[w][lane][k]);
#pragma unroll 1
        for (int j = 0; j < 16; j++) {
            float t = 0.f;
#pragma unroll
            for (int k = 0; k < 16; k++) t = fmaf(W2[16 * k + j], s_da2[w][lane][k], t);
            s_da1[w][lane][j] = t * silu_grad_f(s_da1[w][lane][j]);
        }
        s_z0[w][lane] = z;
        s_dy[w][lane] = dy;
        __syncwarp();
        // entry e = lane + 32 q of the flat gradient
#pragma unroll 1
        for (int e = lane; e < kMlpParams; e += 32) {
            float t = 0.f;
            if (e < 16) {
                for (int s2 = 0; s2 < 32; s2++) t = fmaf(s_da1[w][s2][e], s_z0[w][s2], t);
            } else if (e < 32) {
                for (int s2 = 0; s2 < 32; s2++) t += s_da1[w][s2][e - 16];
            } else if (e < 288) {
                const int k = (e - 32) >> 4, j = (e - 32) & 15;
                for (int s2 = 0; s2 < 32; s2++) t = fmaf(s_da2[w][s2][k], s_h1[w][s2][j], t);
            } else if (e < 304) {
                for (int s2 = 0; s2 < 32; s2++) t += s_da2[w][s2][e - 288];
            } else if (e < 320) {
                for (int s2 = 0; s2 < 32; s2++) t = fmaf(s_dy[w][s2], s_h2[w][s2][e - 304], t);
            } else {
                for (int s2 = 0; s2 < 32; s2++) t += s_dy[w][s2];
            }
            s_red[w][e] += t;
        }
        __syncwarp();
    }
    // fixed-order reduction over lanes (loss) and warps
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if (lane == 0) s_red[w][kMlpParams] = loss;
    __syncthreads();
    for (int e = threadIdx.x; e <= kMlpParams; e += kTrainThreads) {
        float t = 0.f;
        for (int ww = 0; ww < kTrainWarps; ww++) t += s_red[ww][e];
        a.partial[(size_t)blockIdx.x * (kMlpParams + 1) + e] = t;
    }
}

struct AdamArgs {
    float *theta, *m, *v;
    const float *partial;
    int nblocks;
    int32_t *step;
    int steps;
    float lr0, lr_min, b1, b2, eps;
    int batch;
    float *loss_hist;        // [steps] (may be null)
};

__global__ void k_adam(AdamArgs a)
{
    const int e = threadIdx.x;
    const int step = *a.step;
    if (e <= kMlpParams) {
        float g = 0.f;
        for (int b = 0; b < a.nblocks; b++) g += a.partial[(size_t)b * (kMlpParams + 1) + e];
        if (e < kMlpParams) {
            const float lr = a.lr_min + 0.5f * (a.lr0 - a.lr_min) *
                                            (1.f + cosf(3.14159265358979f * (float)step / (float)max(a.steps, 1)));
            const float m = a.b1 * a.m[e] + (1.f - a.b1) * g;
            const float v = a.b2 * a.v[e] + (1.f - a.b2) * g * g;
            a.m[e] = m;
            a.v[e] = v;
            const float t = (float)(step + 1);
            const float mh = m / (1.f - powf(a.b1, t));
            const float vh = v / (1.f - powf(a.b2, t));
            a.theta[e] -= lr * mh / (sqrtf(vh) + a.eps);
        } else if (a.loss_hist && step < a.steps) {
            a.loss_hist[step] = g / (float)a.batch;
        }
    }
    __syncthreads();
    if (e == 0) *a.step = step + 1;
}

// Largest |g_hat / g - 1| over n_grid points r in [0, rcut), g_hat evaluated
// by the warp-level tensor-core path of the learned PP kernel.
__global__ void k_validate(const float *theta, FactorConsts fc, int n_grid, unsigned int *max_err_bits)
{
    __shared__ float w[kMlpParams];
    __shared__ float4 tab[4 * kL1Nodes];
    for (int e = threadIdx.x; e < kMlpParams; e += blockDim.x) w[e] = theta[e];
    __syncthreads();
    l1_table_fill(w, tab);
    __syncthreads();
    MlpLane L;
    mlp_lane_load(w, L);
    const int warps = (gridDim.x * blockDim.x) >> 5;
    float worst = 0.f;
    for (int base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < n_grid; base += warps * 32) {
        const int k = base + (threadIdx.x & 31);
        const float x = (float)min(k, n_grid - 1) / (float)n_grid;
        const float t = 2.f * x - 1.f;
        const float r = x * fc.rcut;
        const float gh = mlp_warp_eval(t, L, tab);
        const float g = exact_factor(r * r, t, fc.poly, fc.npoly, fc.c_e);
        const float err = fabsf(gh / g - 1.f);
        if (k < n_grid) worst = fmaxf(worst, isfinite(err) ? err : 3.0e38f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    if ((threadIdx.x & 31) == 0) atomicMax(max_err_bits, __float_as_uint(worst));
}

// g_hat at caller-given inputs z0 (device array), by the same warp-level
// evaluation as the learned PP kernel (layer-1 table, BF16 tensor cores).
__global__ void k_eval(const float *theta, const float *z0, int64_t n, float *out)
{
    __shared__ float w[kMlpParams];
    __shared__ float4 tab[4 * kL1Nodes];
    for (int e = threadIdx.x; e < kMlpParams; e += blockDim.x) w[e] = theta[e];
    __syncthreads();
    l1_table_fill(w, tab);
    __syncthreads();
    MlpLane L;
    mlp_lane_load(w, L);
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < n; base += warps * 32) {
        const int64_t k = base + (threadIdx.x & 31);
        const float t = k < n ? z0[k] : -1.f;   // (the evaluation is warp-wide: idle lanes take t = -1)
        const float gh = mlp_warp_eval(t, L, tab);
        if (k < n) out[k] = gh;
    }
}

FactorConsts factor_consts(double rs, double rcut)
{
    FactorConsts fc;
    memset(&fc, 0, sizeof fc);
    const double U = rcut / (2.0 * rs);
    fc.npoly = U <= 2.3 ? 10 : (U <= 3.05 ? 12 : (U <= 4.05 ? 14 : 16));
    fit_factor_poly(U, fc.npoly, fc.poly);
    fc.c_e = (float)(-1.4426950408889634 / (4.0 * rs * rs));
    fc.rcut = (float)rcut;
    return fc;
}

void host_init_params(uint64_t seed, float *w)
{
    for (int e = 0; e < kMlpParams; e++) {
        const double fan = (e < 32) ? 1.0 : 16.0;
        const double u = (double)(splitmix64(seed, (uint64_t)e) >> 40) * (1.0 / 16777216.0);
        w[e] = (float)((2.0 * u - 1.0) / std::sqrt(fan));
    }
}

void free_mlp(ph_mlp *h)
{
    DevBuf *bufs[] = {&h->theta, &h->m, &h->v, &h->z0, &h->tgt, &h->partial, &h->work, &h->loss_hist};
    for (DevBuf *b : bufs) release(*b);
}

int validate(ph_mlp *h, cudaStream_t s)
{
    const FactorConsts fc = factor_consts(h->rs, h->rcut);
    unsigned int *bits = static_cast<unsigned int *>(h->work.p) + 2;
    int rc = cuda_check(cudaMemsetAsync(bits, 0, 4, s), "clear validation");
    if (rc) return rc;
    k_validate<<<152, 256, 0, s>>>(static_cast<const float *>(h->theta.p), fc, 1 << 16, bits);
    count_launch();
    unsigned int b = 0;
    rc = cuda_check(cudaMemcpyAsync(&b, bits, 4, cudaMemcpyDeviceToHost, s), "read validation");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "validation sync");
    if (rc) return rc;
    float e;
    memcpy(&e, &b, 4);
    h->max_rel_err = e;
    return PH_OK;
}

int new_mlp(double rs, double rcut, float tol, ph_mlp **out)
{
    if (!(rs > 0) || !(rcut > 0) || !std::isfinite(rs) || !std::isfinite(rcut))
        return fail(PH_ERR_ARG, "rs and rcut must be finite and > 0");
    const double U = rcut / (2.0 * rs);
    if (U > 4.6) return fail(PH_ERR_ARG, "rcut/rs = %g above the supported 9.2", rcut / rs);
    int rc0 = pp_learned_setup();
    if (rc0) return rc0;
    ph_mlp *h = new (std::nothrow) ph_mlp();
    if (!h) return fail(PH_ERR_OOM, "host allocation failed");
    h->rs = rs;
    h->rcut = rcut;
    h->tol = tol > 0 ? tol : 1e-3f;
    int rc = ensure(h->theta, kMlpParams * 4);
    if (!rc) rc = ensure(h->work, 64);
    if (rc) {
        free_mlp(h);
        delete h;
        return rc;
    }
    *out = h;
    return PH_OK;
}

}  // namespace

void mlp_free(ph_mlp *h)
{
    free_mlp(h);
    delete h;
}

}  // namespace phpp

using namespace phpp;

// ---- the network file (layout in phpp.h): fixed little-endian fields
// written byte by byte, so the file is the same on every host.
namespace {
constexpr size_t kMlpFileBytes = 1348, kMlpHashed = 1332;
const unsigned char kMlpMagic[8] = {'P', 'H', 'M', 'L', 'P', 0, 0, 1};

void put_le(unsigned char *b, uint64_t v, int nbytes)
{
    for (int i = 0; i < nbytes; i++) b[i] = (unsigned char)(v >> (8 * i));
}

uint64_t get_le(const unsigned char *b, int nbytes)
{
    uint64_t v = 0;
    for (int i = 0; i < nbytes; i++) v |= (uint64_t)b[i] << (8 * i);
    return v;
}

template <typename T, typename U>
U bits_of(T x)
{
    static_assert(sizeof(T) == sizeof(U), "size");
    U u;
    memcpy(&u, &x, sizeof u);
    return u;
}

uint64_t fnv1a(const unsigned char *b, size_t n)
{
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; i++) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}
}  // namespace

extern "C" {

int ph_mlp_create(const float *weights, double rs, double rcut, float tol, void *stream, ph_mlp **mlp)
{
    TraceRange trace_("ph_mlp_create");
    if (!weights || !mlp) return fail(PH_ERR_ARG, "weights and mlp must not be NULL");
    ph_mlp *h = nullptr;
    int rc = new_mlp(rs, rcut, tol, &h);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = cuda_check(cudaMemcpyAsync(h->theta.p, weights, kMlpParams * 4,
                                    is_device_ptr(weights) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s),
                    "copy weights");
    if (!rc) rc = validate(h, s);
    if (rc) {
        mlp_free(h);
        return rc;
    }
    *mlp = h;
    return PH_OK;
}

int ph_mlp_train(const ph_train_params *tp, double rs, double rcut, const float *init_weights, void *stream,
                 ph_mlp **mlp)
{
    TraceRange trace_("ph_mlp_train");
    if (!tp || !mlp) return fail(PH_ERR_ARG, "train params and mlp must not be NULL");
    if (tp->n_samples < 1 || tp->batch < 1 || tp->steps < 0 || !(tp->lr0 > 0) || tp->lr_min < 0)
        return fail(PH_ERR_ARG, "bad training parameters");
    ph_mlp *h = nullptr;
    int rc = new_mlp(rs, rcut, tp->tol, &h);
    if (rc) return rc;
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    const int nblocks = (tp->batch + kTrainThreads - 1) / kTrainThreads < 152
                            ? (tp->batch + kTrainThreads - 1) / kTrainThreads
                            : 152;
    if (!rc) rc = ensure(h->m, kMlpParams * 4);
    if (!rc) rc = ensure(h->v, kMlpParams * 4);
    if (!rc) rc = ensure(h->z0, (size_t)tp->n_samples * 4);
    if (!rc) rc = ensure(h->tgt, (size_t)tp->n_samples * 4);
    if (!rc) rc = ensure(h->partial, (size_t)nblocks * (kMlpParams + 1) * 4);
    if (!rc) rc = ensure(h->loss_hist, (size_t)(tp->steps > 0 ? tp->steps : 1) * 4);
    float w0[kMlpParams];
    if (init_weights) {
        memcpy(w0, init_weights, sizeof w0);
    } else {
        host_init_params(tp->seed, w0);
    }
    // training runs on a private stream (graph capture is not allowed on the
    // legacy default stream), ordered after the caller's work
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    if (!rc) rc = cuda_check(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "create stream");
    if (!rc) rc = cuda_check(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "create event");
    if (!rc) rc = cuda_check(cudaEventRecord(ev, caller), "record");
    if (!rc) rc = cuda_check(cudaStreamWaitEvent(s, ev, 0), "wait");
    if (!rc) rc = cuda_check(cudaMemcpyAsync(h->theta.p, w0, sizeof w0, cudaMemcpyHostToDevice, s), "copy init");
    if (!rc) rc = cuda_check(cudaMemsetAsync(h->m.p, 0, kMlpParams * 4, s), "clear m");
    if (!rc) rc = cuda_check(cudaMemsetAsync(h->v.p, 0, kMlpParams * 4, s), "clear v");
    if (!rc) rc = cuda_check(cudaMemsetAsync(h->work.p, 0, 64, s), "clear step");
    const FactorConsts fc = factor_consts(rs, rcut);
    if (!rc) {
        k_samples<<<152 * 8, 256, 0, s>>>(tp->n_samples, tp->seed + 1, fc, static_cast<float *>(h->z0.p),
                                          static_cast<float *>(h->tgt.p));
        count_launch();
        rc = cuda_check(cudaGetLastError(), "samples");
    }
    TrainArgs ta;
    ta.theta = static_cast<const float *>(h->theta.p);
    ta.z0 = static_cast<const float *>(h->z0.p);
    ta.tgt = static_cast<const float *>(h->tgt.p);
    ta.n_samples = tp->n_samples;
    ta.batch_stream = tp->seed + 2;
    ta.step = static_cast<const int32_t *>(h->work.p);
    ta.batch = tp->batch;
    ta.partial = static_cast<float *>(h->partial.p);
    AdamArgs aa;
    aa.theta = static_cast<float *>(h->theta.p);
    aa.m = static_cast<float *>(h->m.p);
    aa.v = static_cast<float *>(h->v.p);
    aa.partial = static_cast<const float *>(h->partial.p);
    aa.nblocks = nblocks;
    aa.step = static_cast<int32_t *>(h->work.p);
    aa.steps = tp->steps;
    aa.lr0 = tp->lr0;
    aa.lr_min = tp->lr_min;
    aa.b1 = 0.9f;
    aa.b2 = 0.999f;
    aa.eps = 1e-8f;
    aa.batch = tp->batch;
    aa.loss_hist = static_cast<float *>(h->loss_hist.p);
    // a graph of kGraphSteps steps, replayed; the remainder launched directly
    const int full = tp->steps / kGraphSteps, rest = tp->steps % kGraphSteps;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (!rc && full > 0) {
        rc = cuda_check(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
        if (!rc) {
            for (int k = 0; k < kGraphSteps; k++) {
                k_grad<<<nblocks, kTrainThreads, 0, s>>>(ta);
                k_adam<<<1, 352, 0, s>>>(aa);
            }
            rc = cuda_check(cudaStreamEndCapture(s, &graph), "end capture");
        }
        if (!rc) rc = cuda_check(cudaGraphInstantiate(&exec, graph, 0), "instantiate");
        for (int r = 0; !rc && r < full; r++) {
            rc = cuda_check(cudaGraphLaunch(exec, s), "graph launch");
            count_launch(2 * kGraphSteps);
        }
    }
    for (int k = 0; !rc && k < rest; k++) {
        k_grad<<<nblocks, kTrainThreads, 0, s>>>(ta);
        k_adam<<<1, 352, 0, s>>>(aa);
        count_launch(2);
        rc = cuda_check(cudaGetLastError(), "train step");
    }
    if (!rc) rc = validate(h, s);
    if (!rc && tp->steps > 0) {
        float last = 0.f;
        rc = cuda_check(cudaMemcpyAsync(&last, static_cast<float *>(h->loss_hist.p) + tp->steps - 1, 4,
                                        cudaMemcpyDeviceToHost, s),
                        "read loss");
        if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "train sync");
        h->last_loss = last;
    }
    if (!rc) rc = cuda_check(cudaEventRecord(ev, s), "record");
    if (!rc) rc = cuda_check(cudaStreamWaitEvent(caller, ev, 0), "wait");
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (ev) cudaEventDestroy(ev);
    if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    if (rc) {
        mlp_free(h);
        return rc;
    }
    h->steps_done = tp->steps;
    *mlp = h;
    return PH_OK;
}

int ph_mlp_eval(const ph_mlp *h, const float *d_z0, int64_t n, float *d_out, void *stream)
{
    TraceRange trace_("ph_mlp_eval");
    if (!h || h->kind != KIND_MLP) return fail(PH_ERR_ARG, "not a ph_mlp handle");
    if (n < 0 || (n > 0 && (!d_z0 || !d_out))) return fail(PH_ERR_ARG, "bad arguments");
    if (n > 0 && (!is_device_ptr(d_z0) || !is_device_ptr(d_out))) return fail(PH_ERR_ARG, "device buffers only");
    if (n == 0) return PH_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t warps = (n + 31) / 32;
    const int grid = (int)std::min<int64_t>((warps + 7) / 8, 152 * 8);
    k_eval<<<grid, 256, 0, s>>>(static_cast<const float *>(h->theta.p), d_z0, n, d_out);
    count_launch();
    return cuda_check(cudaGetLastError(), "network evaluation");
}

int ph_mlp_get(const ph_mlp *h, float *weights, float *max_rel_err, float *last_loss)
{
    if (!h || h->kind != KIND_MLP) return fail(PH_ERR_ARG, "not a ph_mlp handle");
    if (weights) {
        int rc = cuda_check(cudaMemcpy(weights, h->theta.p, kMlpParams * 4, cudaMemcpyDeviceToHost), "read weights");
        if (rc) return rc;
    }
    if (max_rel_err) *max_rel_err = h->max_rel_err;
    if (last_loss) *last_loss = h->last_loss;
    return PH_OK;
}


int ph_mlp_file_write(const char *path, const float *weights, double rs, double rcut, float max_rel_err,
                      float last_loss, int32_t steps)
{
    if (!path || !weights) return fail(PH_ERR_ARG, "path and weights must not be NULL");
    unsigned char b[kMlpFileBytes];
    memset(b, 0, sizeof b);
    memcpy(b, kMlpMagic, 8);
    put_le(b + 8, 1, 4);
    put_le(b + 12, kMlpParams, 4);
    put_le(b + 16, bits_of<double, uint64_t>(rs), 8);
    put_le(b + 24, bits_of<double, uint64_t>(rcut), 8);
    put_le(b + 32, bits_of<float, uint32_t>(max_rel_err), 4);
    put_le(b + 36, bits_of<float, uint32_t>(last_loss), 4);
    put_le(b + 40, (uint32_t)steps, 4);
    for (int e = 0; e < kMlpParams; e++) put_le(b + 48 + 4 * e, bits_of<float, uint32_t>(weights[e]), 4);
    put_le(b + kMlpHashed, fnv1a(b, kMlpHashed), 8);
    FILE *f = fopen(path, "wb");
    if (!f) return fail(PH_ERR_ARG, "cannot open %s for writing", path);
    const size_t w = fwrite(b, 1, sizeof b, f);
    const int closed = fclose(f);
    if (w != sizeof b || closed != 0) return fail(PH_ERR_ARG, "cannot write %s", path);
    return PH_OK;
}

int ph_mlp_file_read(const char *path, float *weights, double *rs, double *rcut, float *max_rel_err, float *last_loss,
                     int32_t *steps)
{
    if (!path || !weights) return fail(PH_ERR_ARG, "path and weights must not be NULL");
    unsigned char b[kMlpFileBytes + 1];
    FILE *f = fopen(path, "rb");
    if (!f) return fail(PH_ERR_ARG, "cannot open %s", path);
    const size_t got = fread(b, 1, sizeof b, f);
    fclose(f);
    if (got != kMlpFileBytes) return fail(PH_ERR_ARG, "%s: %zu bytes, a network file has %zu", path, got, kMlpFileBytes);
    if (memcmp(b, kMlpMagic, 8) != 0) return fail(PH_ERR_ARG, "%s is not a network file (magic)", path);
    if (get_le(b + 8, 4) != 1) return fail(PH_ERR_ARG, "%s: unknown format version %u", path, (unsigned)get_le(b + 8, 4));
    if (get_le(b + 12, 4) != (uint64_t)kMlpParams) return fail(PH_ERR_ARG, "%s: parameter count is not 321", path);
    if (get_le(b + kMlpHashed, 8) != fnv1a(b, kMlpHashed)) return fail(PH_ERR_ARG, "%s: damaged (hash mismatch)", path);
    for (int e = 0; e < kMlpParams; e++) weights[e] = bits_of<uint32_t, float>((uint32_t)get_le(b + 48 + 4 * e, 4));
    if (rs) *rs = bits_of<uint64_t, double>(get_le(b + 16, 8));
    if (rcut) *rcut = bits_of<uint64_t, double>(get_le(b + 24, 8));
    if (max_rel_err) *max_rel_err = bits_of<uint32_t, float>((uint32_t)get_le(b + 32, 4));
    if (last_loss) *last_loss = bits_of<uint32_t, float>((uint32_t)get_le(b + 36, 4));
    if (steps) *steps = (int32_t)(uint32_t)get_le(b + 40, 4);
    return PH_OK;
}

int ph_mlp_save(const ph_mlp *h, const char *path)
{
    if (!h || h->kind != KIND_MLP) return fail(PH_ERR_ARG, "not a ph_mlp handle");
    float w[kMlpParams];
    int rc = cuda_check(cudaMemcpy(w, h->theta.p, sizeof w, cudaMemcpyDeviceToHost), "read weights");
    if (rc) return rc;
    return ph_mlp_file_write(path, w, h->rs, h->rcut, h->max_rel_err, h->last_loss, h->steps_done);
}

int ph_mlp_load(const char *path, float tol, void *stream, ph_mlp **mlp)
{
    if (!mlp) return fail(PH_ERR_ARG, "mlp must not be NULL");
    float w[kMlpParams];
    double rs = 0, rcut = 0;
    float err = 0, loss = 0;
    int32_t steps = 0;
    int rc = ph_mlp_file_read(path, w, &rs, &rcut, &err, &loss, &steps);
    if (rc) return rc;
    ph_mlp *h = nullptr;
    rc = ph_mlp_create(w, rs, rcut, tol, stream, &h);
    if (rc) return rc;
    h->last_loss = loss;
    h->steps_done = steps;
    *mlp = h;
    return PH_OK;
}

int ph_mlp_loss_grad(const float *weights, const float *z0, const float *target, int64_t n, float *grad, float *loss,
                     void *stream)
{
    TraceRange trace_("ph_mlp_loss_grad");
    if (!weights || !z0 || !target || !grad || n < 1 || n > (1 << 24)) return fail(PH_ERR_ARG, "bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevBuf th, zz, tt, part, st;
    const int nblocks = (int)((n + kTrainThreads - 1) / kTrainThreads < 152 ? (n + kTrainThreads - 1) / kTrainThreads
                                                                             : 152);
    int rc = ensure(th, kMlpParams * 4);
    if (!rc) rc = ensure(zz, (size_t)n * 4);
    if (!rc) rc = ensure(tt, (size_t)n * 4);
    if (!rc) rc = ensure(part, (size_t)nblocks * (kMlpParams + 1) * 4);
    if (!rc) rc = ensure(st, 16);
    if (!rc) rc = cuda_check(cudaMemcpyAsync(th.p, weights, kMlpParams * 4, cudaMemcpyDefault, s), "copy");
    if (!rc) rc = cuda_check(cudaMemcpyAsync(zz.p, z0, (size_t)n * 4, cudaMemcpyDefault, s), "copy");
    if (!rc) rc = cuda_check(cudaMemcpyAsync(tt.p, target, (size_t)n * 4, cudaMemcpyDefault, s), "copy");
    if (!rc) rc = cuda_check(cudaMemsetAsync(st.p, 0, 16, s), "clear");
    std::vector<float> hp((size_t)nblocks * (kMlpParams + 1));
    if (!rc) {
        TrainArgs ta;
        ta.theta = static_cast<const float *>(th.p);
        ta.z0 = static_cast<const float *>(zz.p);
        ta.tgt = static_cast<const float *>(tt.p);
        ta.n_samples = n;
        ta.batch_stream = ~0ull;
        ta.step = static_cast<const int32_t *>(st.p);
        ta.batch = (int)n;
        ta.partial = static_cast<float *>(part.p);
        k_grad<<<nblocks, kTrainThreads, 0, s>>>(ta);
        count_launch();
        rc = cuda_check(cudaGetLastError(), "grad");
    }
    if (!rc)
        rc = cuda_check(cudaMemcpyAsync(hp.data(), part.p, hp.size() * 4, cudaMemcpyDeviceToHost, s), "read grad");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(s), "grad sync");
    if (!rc) {
        for (int e = 0; e <= kMlpParams; e++) {
            float t = 0.f;
            for (int b = 0; b < nblocks; b++) t += hp[(size_t)b * (kMlpParams + 1) + e];
            if (e < kMlpParams) grad[e] = t;
            else if (loss) *loss = t / (float)n;
        }
    }
    release(th);
    release(zz);
    release(tt);
    release(part);
    release(st);
    return rc;
}

}  // extern "C"
