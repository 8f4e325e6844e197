// Learned ACA-rank predictor: a two-hidden-layer tanh MLP with hand-written
// forward, backward, gradient-reduction and Adam kernels (FP32), and the block
// features it reads.  The paper has no learned component; the network only
// preallocates and orders the ACA of admissible blocks (Sec. III), and plain
// adaptive ACA re-runs every block whose prediction was too low, so the H-matrix
// never depends on it.
//
// Network (nin inputs, nh hidden units):
//   h1 = tanh(W1 x + b1),  h2 = tanh(W2 h1 + b2),  y = w3 . h2 + b3
// Packed parameters: W1 [nh][nin] row-major, b1 [nh], W2 [nh][nh], b2 [nh], w3 [nh], b3.
// Loss: L = (1/n) sum_s (y_s - t_s)^2.  Adam (Kingma & Ba 2015) with bias correction.
#include <cmath>
#include <cstring>

#include "hm_internal.h"

#define MLP_NH_MAX 64
#define MLP_NIN_MAX 16
#define MLP_T 128

struct hm_mlp_s {
    cudaStream_t stream = nullptr;
    int nin = 0, nh = 0, np = 0;
    float *d_par = nullptr, *d_m = nullptr, *d_v = nullptr, *d_grad = nullptr;
    float *d_work = nullptr;  // activations and deltas, 4 * nh * cap
    double *d_loss = nullptr;
    int cap = 0;              // samples the work buffer holds
    int adam_t = 0;
    std::string err;
    long long launches = 0;
};

static int mlp_nparams(int nin, int nh) { return nh * nin + nh + nh * nh + nh + nh + 1; }

struct MlpView {
    const float *W1, *b1, *W2, *b2, *w3, *b3;
};

__device__ __forceinline__ MlpView mlp_view(const float *p, int nin, int nh)
{
    MlpView v;
    v.W1 = p;
    v.b1 = v.W1 + nh * nin;
    v.W2 = v.b1 + nh;
    v.b2 = v.W2 + nh * nh;
    v.w3 = v.b2 + nh;
    v.b3 = v.w3 + nh;
    return v;
}

// One thread per sample.  Stores h1, h2 ([n][nh] each) when H1/H2 are non-null.
__global__ void __launch_bounds__(MLP_T) k_mlp_forward(const float *__restrict__ par, int nin, int nh, int n,
                                                        const float *__restrict__ X, float *__restrict__ Y,
                                                        float *__restrict__ H1, float *__restrict__ H2)
{
    __shared__ float sp[MLP_NH_MAX * MLP_NIN_MAX + 3 * MLP_NH_MAX + MLP_NH_MAX * MLP_NH_MAX + 1];
    const int np = nh * nin + nh + nh * nh + nh + nh + 1;
    for (int i = threadIdx.x; i < np; i += blockDim.x) sp[i] = par[i];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    MlpView w = mlp_view(sp, nin, nh);
    float x[MLP_NIN_MAX], h1[MLP_NH_MAX];
    for (int i = 0; i < nin; ++i) x[i] = X[(size_t)s * nin + i];
    for (int j = 0; j < nh; ++j) {
        float a = w.b1[j];
        for (int i = 0; i < nin; ++i) a = fmaf(w.W1[j * nin + i], x[i], a);
        h1[j] = tanhf(a);
        if (H1) H1[(size_t)s * nh + j] = h1[j];
    }
    float y = w.b3[0];
    for (int j = 0; j < nh; ++j) {
        float a = w.b2[j];
        for (int i = 0; i < nh; ++i) a = fmaf(w.W2[j * nh + i], h1[i], a);
        float h2 = tanhf(a);
        if (H2) H2[(size_t)s * nh + j] = h2;
        y = fmaf(w.w3[j], h2, y);
    }
    Y[s] = y;
}

// Per-sample deltas: e = 2 (y - t) / n;  D2 = e w3 (1 - h2^2);  D1 = (W2^T D2) (1 - h1^2).
// E[s] = e.  Also accumulates the loss sum in FP64 (one atomic per CTA).
__global__ void __launch_bounds__(MLP_T) k_mlp_backward(const float *__restrict__ par, int nin, int nh, int n,
                                                         const float *__restrict__ Y, const float *__restrict__ T,
                                                         const float *__restrict__ H1, const float *__restrict__ H2,
                                                         float *__restrict__ E, float *__restrict__ D1,
                                                         float *__restrict__ D2, double *__restrict__ loss)
{
    __shared__ float sp[MLP_NH_MAX * MLP_NIN_MAX + 3 * MLP_NH_MAX + MLP_NH_MAX * MLP_NH_MAX + 1];
    __shared__ double sl[MLP_T / 32];
    const int np = nh * nin + nh + nh * nh + nh + nh + 1;
    for (int i = threadIdx.x; i < np; i += blockDim.x) sp[i] = par[i];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (s < n) {
        MlpView w = mlp_view(sp, nin, nh);
        float r = Y[s] - T[s];
        l = (double)r * r;
        float e = 2.0f * r / (float)n;
        E[s] = e;
        float d2[MLP_NH_MAX];
        for (int j = 0; j < nh; ++j) {
            float h = H2[(size_t)s * nh + j];
            d2[j] = e * w.w3[j] * (1.0f - h * h);
            D2[(size_t)s * nh + j] = d2[j];
        }
        for (int i = 0; i < nh; ++i) {
            float a = 0.0f;
            for (int j = 0; j < nh; ++j) a = fmaf(w.W2[j * nh + i], d2[j], a);
            float h = H1[(size_t)s * nh + i];
            D1[(size_t)s * nh + i] = a * (1.0f - h * h);
        }
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffff, l, o);
    if ((threadIdx.x & 31) == 0) sl[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int i = 0; i < MLP_T / 32; ++i) t += sl[i];
        atomicAdd(loss, t);
    }
}

// One CTA per parameter: the gradient is a sum over samples of (delta x input),
// reduced in a fixed order (deterministic).
__global__ void __launch_bounds__(MLP_T) k_mlp_grad(int nin, int nh, int n, const float *__restrict__ X,
                                                     const float *__restrict__ H1, const float *__restrict__ H2,
                                                     const float *__restrict__ E, const float *__restrict__ D1,
                                                     const float *__restrict__ D2, float *__restrict__ grad)
{
    const int p = blockIdx.x;
    // which parameter: (delta array, delta index, input array, input index, input width)
    const float *dl, *in = nullptr;
    int dj, ii = 0, dw, iw = 0;
    int q = p;
    if (q < nh * nin) {
        dl = D1; dw = nh; dj = q / nin; in = X; iw = nin; ii = q % nin;
    } else if ((q -= nh * nin) < nh) {
        dl = D1; dw = nh; dj = q;
    } else if ((q -= nh) < nh * nh) {
        dl = D2; dw = nh; dj = q / nh; in = H1; iw = nh; ii = q % nh;
    } else if ((q -= nh * nh) < nh) {
        dl = D2; dw = nh; dj = q;
    } else if ((q -= nh) < nh) {
        dl = E; dw = 1; dj = 0; in = H2; iw = nh; ii = q;
    } else {
        dl = E; dw = 1; dj = 0;
    }
    float acc = 0.0f;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        float d = dl[(size_t)s * dw + dj];
        acc = fmaf(d, in ? in[(size_t)s * iw + ii] : 1.0f, acc);
    }
    __shared__ float sh[MLP_T / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffff, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0;
        for (int i = 0; i < MLP_T / 32; ++i) t += sh[i];
        grad[p] = t;
    }
}

// Adam step t (1-based): bias-corrected first and second moments.
__global__ void k_mlp_adam(int np, float *__restrict__ par, float *__restrict__ m, float *__restrict__ v,
                           const float *__restrict__ g, float lr, float b1, float b2, float eps, int t)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float mh = mi / (1.0f - powf(b1, (float)t));
    float vh = vi / (1.0f - powf(b2, (float)t));
    par[i] -= lr * mh / (sqrtf(vh) + eps);
}

namespace {

template <class F>
hm_status mlp_guard(hm_mlp m, F &&f)
{
    if (!m) return HM_ERR_ARG;
    try {
        f();
        m->err.clear();
        return HM_OK;
    } catch (const HmError &e) {
        m->err = e.msg;
        return e.st;
    } catch (...) {
        m->err = "unknown error";
        return HM_ERR_CUDA;
    }
}

void mlp_reserve(hm_mlp m, int n)
{
    if (n <= m->cap) return;
    if (m->d_work) HM_CUDA(cudaFree(m->d_work));
    m->d_work = nullptr;
    m->cap = 0;
    HM_CUDA(cudaMalloc(&m->d_work, sizeof(float) * ((size_t)4 * m->nh + 2) * n));
    m->cap = n;
}

// forward + backward + gradient reduction; loss sum left in d_loss (FP64)
void mlp_loss_grad(hm_mlp m, int n, const float *X, const float *T)
{
    mlp_reserve(m, n);
    float *H1 = m->d_work, *H2 = H1 + (size_t)m->nh * n, *D1 = H2 + (size_t)m->nh * n;
    float *D2 = D1 + (size_t)m->nh * n, *Y = D2 + (size_t)m->nh * n, *E = Y + n;
    unsigned g = (unsigned)((n + MLP_T - 1) / MLP_T);
    HM_CUDA(cudaMemsetAsync(m->d_loss, 0, sizeof(double), m->stream));
    k_mlp_forward<<<g, MLP_T, 0, m->stream>>>(m->d_par, m->nin, m->nh, n, X, Y, H1, H2);
    HM_CHECK_LAUNCH();
    k_mlp_backward<<<g, MLP_T, 0, m->stream>>>(m->d_par, m->nin, m->nh, n, Y, T, H1, H2, E, D1, D2, m->d_loss);
    HM_CHECK_LAUNCH();
    k_mlp_grad<<<m->np, MLP_T, 0, m->stream>>>(m->nin, m->nh, n, X, H1, H2, E, D1, D2, m->d_grad);
    HM_CHECK_LAUNCH();
    m->launches += 3;
}

}  // namespace

// Host-side helpers used by the fill (hm_api.cu): predictions for a feature batch.
void mlp_predict_host(hm_mlp m, int n, const float *feat_host, float *pred_host)
{
    if (n <= 0) return;
    float *d = nullptr;
    HM_CUDA(cudaMallocAsync(&d, sizeof(float) * (size_t)(m->nin + 1) * n, m->stream));
    HM_CUDA(cudaMemcpyAsync(d, feat_host, sizeof(float) * (size_t)m->nin * n, cudaMemcpyHostToDevice, m->stream));
    k_mlp_forward<<<(unsigned)((n + MLP_T - 1) / MLP_T), MLP_T, 0, m->stream>>>(
        m->d_par, m->nin, m->nh, n, d, d + (size_t)m->nin * n, nullptr, nullptr);
    HM_CHECK_LAUNCH();
    m->launches += 1;
    HM_CUDA(cudaMemcpyAsync(pred_host, d + (size_t)m->nin * n, sizeof(float) * n, cudaMemcpyDeviceToHost, m->stream));
    HM_CUDA(cudaFreeAsync(d, m->stream));
    HM_CUDA(cudaStreamSynchronize(m->stream));
}

int mlp_nin(hm_mlp m) { return m ? m->nin : 0; }

extern "C" {

hm_status hm_mlp_create(hm_mlp *out, int nin, int nh, void *stream)
{
    if (!out) return HM_ERR_ARG;
    *out = nullptr;
    if (nin < 1 || nin > MLP_NIN_MAX || nh < 1 || nh > MLP_NH_MAX) return HM_ERR_ARG;
    hm_mlp m = new (std::nothrow) hm_mlp_s();
    if (!m) return HM_ERR_OOM;
    m->stream = (cudaStream_t)stream;
    m->nin = nin;
    m->nh = nh;
    m->np = mlp_nparams(nin, nh);
    size_t b = sizeof(float) * m->np;
    if (cudaMalloc(&m->d_par, b) != cudaSuccess || cudaMalloc(&m->d_m, b) != cudaSuccess ||
        cudaMalloc(&m->d_v, b) != cudaSuccess || cudaMalloc(&m->d_grad, b) != cudaSuccess ||
        cudaMalloc(&m->d_loss, sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        hm_mlp_destroy(m);
        return HM_ERR_OOM;
    }
    cudaMemset(m->d_par, 0, b);
    cudaMemset(m->d_m, 0, b);
    cudaMemset(m->d_v, 0, b);
    *out = m;
    return HM_OK;
}

int hm_mlp_num_params(hm_mlp m) { return m ? m->np : 0; }

hm_status hm_mlp_set_params(hm_mlp m, const float *par)
{
    return mlp_guard(m, [&] {
        if (!par) throw HmError{HM_ERR_ARG, "null params"};
        HM_CUDA(cudaMemcpyAsync(m->d_par, par, sizeof(float) * m->np, cudaMemcpyHostToDevice, m->stream));
        HM_CUDA(cudaMemsetAsync(m->d_m, 0, sizeof(float) * m->np, m->stream));
        HM_CUDA(cudaMemsetAsync(m->d_v, 0, sizeof(float) * m->np, m->stream));
        HM_CUDA(cudaStreamSynchronize(m->stream));
        m->adam_t = 0;
    });
}

hm_status hm_mlp_get_params(hm_mlp m, float *par)
{
    return mlp_guard(m, [&] {
        if (!par) throw HmError{HM_ERR_ARG, "null params"};
        HM_CUDA(cudaMemcpyAsync(par, m->d_par, sizeof(float) * m->np, cudaMemcpyDeviceToHost, m->stream));
        HM_CUDA(cudaStreamSynchronize(m->stream));
    });
}

hm_status hm_mlp_forward(hm_mlp m, int n, const float *x_dev, float *y_dev)
{
    return mlp_guard(m, [&] {
        if (n < 0 || (n > 0 && (!x_dev || !y_dev))) throw HmError{HM_ERR_ARG, "bad forward arguments"};
        if (n == 0) return;
        k_mlp_forward<<<(unsigned)((n + MLP_T - 1) / MLP_T), MLP_T, 0, m->stream>>>(m->d_par, m->nin, m->nh, n, x_dev,
                                                                                    y_dev, nullptr, nullptr);
        HM_CHECK_LAUNCH();
        m->launches += 1;
    });
}

hm_status hm_mlp_loss_grad(hm_mlp m, int n, const float *x_dev, const float *t_dev, double *loss_host,
                           float *grad_host)
{
    return mlp_guard(m, [&] {
        if (n <= 0 || !x_dev || !t_dev) throw HmError{HM_ERR_ARG, "bad loss arguments"};
        mlp_loss_grad(m, n, x_dev, t_dev);
        if (grad_host)
            HM_CUDA(cudaMemcpyAsync(grad_host, m->d_grad, sizeof(float) * m->np, cudaMemcpyDeviceToHost, m->stream));
        double l = 0;
        HM_CUDA(cudaMemcpyAsync(&l, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
        HM_CUDA(cudaStreamSynchronize(m->stream));
        if (loss_host) *loss_host = l / n;
    });
}

hm_status hm_mlp_train(hm_mlp m, int n, const float *x_dev, const float *t_dev, int steps, float lr,
                       double *loss_host)
{
    return mlp_guard(m, [&] {
        if (n <= 0 || !x_dev || !t_dev || steps < 0 || !(lr > 0.0f)) throw HmError{HM_ERR_ARG, "bad train arguments"};
        unsigned ga = (unsigned)((m->np + 255) / 256);
        for (int it = 0; it < steps; ++it) {
            mlp_loss_grad(m, n, x_dev, t_dev);
            ++m->adam_t;
            k_mlp_adam<<<ga, 256, 0, m->stream>>>(m->np, m->d_par, m->d_m, m->d_v, m->d_grad, lr, 0.9f, 0.999f,
                                                  1e-8f, m->adam_t);
            HM_CHECK_LAUNCH();
            m->launches += 1;
        }
        if (loss_host) {
            mlp_loss_grad(m, n, x_dev, t_dev);
            double l = 0;
            HM_CUDA(cudaMemcpyAsync(&l, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
            HM_CUDA(cudaStreamSynchronize(m->stream));
            *loss_host = l / n;
        }
    });
}

const char *hm_mlp_last_error(hm_mlp m) { return m ? m->err.c_str() : "null model"; }

void hm_mlp_destroy(hm_mlp m)
{
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    cudaFree(m->d_par);
    cudaFree(m->d_m);
    cudaFree(m->d_v);
    cudaFree(m->d_grad);
    cudaFree(m->d_work);
    cudaFree(m->d_loss);
    delete m;
}

}  // extern "C"
