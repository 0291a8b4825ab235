// Learned preconditioner (SE_PRECOND_LEARNED): a network that reads every particle's
// radius and its neighbours inside rc and sets the long-wavelength correction of the
// block-diagonal far-field preconditioner of Sec. 4.2.
//
// Per particle i the network reads rotation- and permutation-invariant features of
// its radius and of its neighbours inside rc, and one feature of the whole box,
//   f = [ sum_j b_k(h_ij) (k < 7),  sum_j b_k(h_ij) a_j/a_i (k < 7),  a_i / <a>,  ln(L / <a>) / 5 ],
//   h_ij = r_ij / (a_i + a_j),  b_k(h) = exp(-((h - c_k)/0.35)^2),  c = 1, 1.25, 1.5, 2, 2.5, 3, 4.
// Its outputs, averaged over the particles (a permutation-invariant set function of
// the configuration), are the damping theta, the cutoff k_c <a> and the norm cap c_max of
// the spectral correction P^-1 = B - S C S (se_solve.cu): they decide how far the
// long-wavelength collective modes, which set the GMRES iteration count, are corrected.
// The network is trained on the iteration counts of solves the method itself runs over
// a grid of (theta, k_c <a>, c_max) on generated configurations (train_pc.py).  Output 3
// is unused (trained to zero).  theta is clamped to [0.5, 0.985], k_c <a> to [0.4, 1.5]
// and c_max to [0.85, 0.985]; the plain block preconditioner stays the fallback (no
// weights, sheared cells), and a corrected cycle that fails to halve the residual is
// retried with less damping.
//
// Network: 16 -> 64 -> 64 -> 4, tanh, FP32, standardised inputs and outputs.
// Packed parameters (float): W1[64][16] b1[64] W2[64][64] b2[64] W3[4][64] b3[4]
// (5508 trained values), then mu[16] sd[16] (input standardisation) and os[4]
// (output scale), 5544 floats in all.
#include <algorithm>
#include <cmath>
#include <vector>

#include "se_internal.cuh"

namespace se {

constexpr int kF = 16, kH = 64, kO = 4;
constexpr int kNTrain = kH * kF + kH + kH * kH + kH + kO * kH + kO;   // 5508
constexpr int kNW = kNTrain + 2 * kF + kO;                              // 5544
constexpr int kSampleStride = kF + 4 * kH + kO;                         // per-sample scratch

namespace {

struct WOff {
    static constexpr int W1 = 0, b1 = W1 + kH * kF, W2 = b1 + kH, b2 = W2 + kH * kH, W3 = b2 + kH,
                         b3 = W3 + kO * kH, mu = b3 + kO, sd = mu + kF, os = sd + kF;
};

// features of every particle (written in caller order) from the stored pair lists
__global__ void features_kernel(int N, double amean, double L, const int *off, size_t np, const int *pj,
                                const float *px, const double *px64, const double *rad, const int *perm, float *feat)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float c[7] = {1.0f, 1.25f, 1.5f, 2.0f, 2.5f, 3.0f, 4.0f};
    float f[kF] = {0};
    const double ai = rad[i];
    for (int k = off[i]; k < off[i + 1]; ++k) {
        const int j = pj[k];
        double x0, x1, x2;
        if (px) { x0 = px[k]; x1 = px[np + k]; x2 = px[2 * np + k]; }
        else { x0 = px64[k]; x1 = px64[np + k]; x2 = px64[2 * np + k]; }
        const float h = (float)(sqrt(x0 * x0 + x1 * x1 + x2 * x2) / (ai + rad[j]));
        const float ra = (float)(rad[j] / ai);
        for (int q = 0; q < 7; ++q) {
            const float t = (h - c[q]) / 0.35f;
            const float b = expf(-t * t);
            f[q] += b;
            f[7 + q] += b * ra;
        }
    }
    f[14] = (float)(ai / amean);
    f[15] = (float)(log(L / amean) / 5.0);
    float *o = feat + (size_t)perm[i] * kF;
    for (int q = 0; q < kF; ++q) o[q] = f[q];
}

// forward pass, one thread per sample; weights staged in shared memory
__device__ __forceinline__ void mlp_forward_one(const float *w, const float *x, float *xs, float *h1, float *h2,
                                                float *y)
{
    for (int d = 0; d < kF; ++d) xs[d] = (x[d] - w[WOff::mu + d]) / w[WOff::sd + d];
    for (int a = 0; a < kH; ++a) {
        float z = w[WOff::b1 + a];
        for (int d = 0; d < kF; ++d) z += w[WOff::W1 + a * kF + d] * xs[d];
        h1[a] = tanhf(z);
    }
    for (int a = 0; a < kH; ++a) {
        float z = w[WOff::b2 + a];
        for (int b = 0; b < kH; ++b) z += w[WOff::W2 + a * kH + b] * h1[b];
        h2[a] = tanhf(z);
    }
    for (int o = 0; o < kO; ++o) {
        float z = w[WOff::b3 + o];
        for (int b = 0; b < kH; ++b) z += w[WOff::W3 + o * kH + b] * h2[b];
        y[o] = z;
    }
}

__global__ void __launch_bounds__(128) mlp_forward_kernel(const float *wg, const float *X, int n, float *Y)
{
    __shared__ float w[kNW];
    for (int e = threadIdx.x; e < kNW; e += blockDim.x) w[e] = wg[e];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float xs[kF], h1[kH], h2[kH], y[kO];
    mlp_forward_one(w, X + (size_t)s * kF, xs, h1, h2, y);
    for (int o = 0; o < kO; ++o) Y[(size_t)s * kO + o] = y[o] * w[WOff::os + o];
}

// forward + per-sample backward of the mean squared error on standardised outputs;
// stores x, z1' (dL/dpre1), h1, z2' (dL/dpre2), h2... per sample for the reduction
__global__ void __launch_bounds__(128) mlp_sample_grad_kernel(const float *wg, const float *X, const float *Yt, int n,
                                                              float *S, float *loss)
{
    __shared__ float w[kNW];
    __shared__ float red[128];
    for (int e = threadIdx.x; e < kNW; e += blockDim.x) w[e] = wg[e];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (s < n) {
        float xs[kF], h1[kH], h2[kH], y[kO], dy[kO], d2[kH];
        mlp_forward_one(w, X + (size_t)s * kF, xs, h1, h2, y);
        for (int o = 0; o < kO; ++o) {
            const float e = y[o] - Yt[(size_t)s * kO + o] / w[WOff::os + o];
            l += e * e;
            dy[o] = 2.f * e / (float)(n * kO);
        }
        for (int a = 0; a < kH; ++a) {
            float g = 0.f;
            for (int o = 0; o < kO; ++o) g += w[WOff::W3 + o * kH + a] * dy[o];
            d2[a] = g * (1.f - h2[a] * h2[a]);
        }
        float *so = S + (size_t)s * kSampleStride;
        for (int d = 0; d < kF; ++d) so[d] = xs[d];
        for (int a = 0; a < kH; ++a) {
            float g = 0.f;
            for (int b = 0; b < kH; ++b) g += w[WOff::W2 + b * kH + a] * d2[b];
            so[kF + a] = g * (1.f - h1[a] * h1[a]);       // d1
            so[kF + kH + a] = h1[a];
            so[kF + 2 * kH + a] = d2[a];
            so[kF + 3 * kH + a] = h2[a];
        }
        for (int o = 0; o < kO; ++o) so[kF + 4 * kH + o] = dy[o];
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] / (float)(n * kO));
}

// gradient of every trained parameter: sums over samples of the per-sample factors
__global__ void mlp_reduce_grad_kernel(const float *S, int n, float *grad)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kNTrain) return;
    int ua, ub;     // offsets of the two per-sample factors (ub < 0: bias)
    if (p < WOff::b1) { ua = kF + (p / kF); ub = p % kF; }                               // d1 x
    else if (p < WOff::W2) { ua = kF + (p - WOff::b1); ub = -1; }                          // d1
    else if (p < WOff::b2) { const int q = p - WOff::W2; ua = kF + 2 * kH + q / kH; ub = kF + kH + q % kH; }  // d2 h1
    else if (p < WOff::W3) { ua = kF + 2 * kH + (p - WOff::b2); ub = -1; }                 // d2
    else if (p < WOff::b3) { const int q = p - WOff::W3; ua = kF + 4 * kH + q / kH; ub = kF + 3 * kH + q % kH; }  // dy h2
    else { ua = kF + 4 * kH + (p - WOff::b3); ub = -1; }                                   // dy
    double g = 0.0;
    for (int s = 0; s < n; ++s) {
        const float *so = S + (size_t)s * kSampleStride;
        g += (double)so[ua] * (ub >= 0 ? so[ub] : 1.f);
    }
    grad[p] = (float)g;
}

__global__ void adam_kernel(float *w, float *m, float *v, const float *g, int step, float lr)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kNTrain) return;
    const float b1 = 0.9f, b2 = 0.999f;
    m[p] = b1 * m[p] + (1 - b1) * g[p];
    v[p] = b2 * v[p] + (1 - b2) * g[p] * g[p];
    const float mh = m[p] / (1 - powf(b1, (float)step)), vh = v[p] / (1 - powf(b2, (float)step));
    w[p] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

}  // namespace

// ---- used by se_solve: the spectral correction's damping and cutoff for the configuration
int learned_spectral_params(se_ctx *c, double *theta, double *ka, double *cmax)
{
    if (c->lp_ready) {
        *theta = c->lp_theta;
        *ka = c->lp_ka;
        *cmax = c->lp_cmax;
        return SE_OK;
    }
    cudaStream_t s = c->stream;
    const int N = (int)c->N;
    if (!c->b.pair_off || (!c->pairs_ok[0] && !c->pairs_ok[1])) {
        const int r = c->precision == 1 ? build_pair_table<double>(c) : build_pair_table<float>(c);
        if (r != SE_OK) return r;
    }
    float *feat = nullptr, *y = nullptr;
    if (cudaMalloc(&feat, (size_t)N * kF * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&y, (size_t)N * kO * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        if (feat) cudaFree(feat);
        c->err = "learned preconditioner allocation failed";
        return SE_ERR_NOMEM;
    }
    std::vector<double> r(N);
    cudaMemcpy(r.data(), c->b.rad, N * sizeof(double), cudaMemcpyDeviceToHost);
    double am = 0;
    for (double v : r) am += v;
    am /= N;
    features_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, am, c->L, c->b.pair_off, c->npairs, c->b.pair_j,
                                                    c->pairs_ok[0] ? (const float *)c->b.pair_x[0] : nullptr,
                                                    c->pairs_ok[0] ? nullptr : (const double *)c->b.pair_x[1],
                                                    c->b.rad, c->b.perm, feat);
    mlp_forward_kernel<<<(N + 127) / 128, 128, 0, s>>>(c->b.mlp_w, feat, N, y);
    c->launches += 2;
    std::vector<float> yh((size_t)N * kO);
    cudaError_t e = cudaMemcpyAsync(yh.data(), y, yh.size() * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(feat);
    cudaFree(y);
    if (e != cudaSuccess) {
        c->err = std::string("learned preconditioner: ") + cudaGetErrorString(e);
        return SE_ERR_CUDA;
    }
    double t = 0, k = 0, m = 0;
    for (int i = 0; i < N; ++i) {
        t += yh[(size_t)i * kO];
        k += yh[(size_t)i * kO + 1];
        m += yh[(size_t)i * kO + 2];
    }
    t /= N;
    k /= N;
    m /= N;
    if (!std::isfinite(t)) t = 0.5;
    if (!std::isfinite(k)) k = 0.9;
    if (!std::isfinite(m)) m = 0.85;
    c->lp_theta = std::min(0.985, std::max(0.5, t));
    c->lp_ka = std::min(1.5, std::max(0.4, k));
    c->lp_cmax = std::min(0.985, std::max(0.85, m));
    c->lp_ready = true;
    *theta = c->lp_theta;
    *ka = c->lp_ka;
    *cmax = c->lp_cmax;
    return SE_OK;
}

}  // namespace se

using namespace se;

extern "C" int se_set_learned_weights(se_ctx *c, const float *w, int nw)
{
    if (!c) return SE_ERR_ARG;
    if (!w || nw != kNW) {
        c->err = "learned weights: expected " + std::to_string(kNW) + " floats";
        return SE_ERR_ARG;
    }
    for (int q = 0; q < nw; ++q)
        if (!std::isfinite(w[q])) {
            c->err = "learned weights: non-finite value";
            return SE_ERR_NONFINITE;
        }
    cudaSetDevice(c->device);
    if (!c->b.mlp_w && cudaMalloc(&c->b.mlp_w, kNW * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        c->err = "learned weights: allocation failed";
        return SE_ERR_NOMEM;
    }
    SE_CUDA_CHECK(c, cudaMemcpy(c->b.mlp_w, w, kNW * sizeof(float), cudaMemcpyHostToDevice));
    c->have_mlp = true;
    c->lp_ready = false;
    return SE_OK;
}

extern "C" int se_learned_features(se_ctx *c, float *feat)
{
    if (!c || !feat) return SE_ERR_ARG;
    if (!c->have_config) { c->err = "se_set_config must be called first"; return SE_ERR_STATE; }
    cudaSetDevice(c->device);
    const int N = (int)c->N;
    if (!c->pairs_ok[0] && !c->pairs_ok[1]) {
        const int r = c->precision == 1 ? build_pair_table<double>(c) : build_pair_table<float>(c);
        if (r != SE_OK) return r;
    }
    std::vector<double> r(N);
    cudaMemcpy(r.data(), c->b.rad, N * sizeof(double), cudaMemcpyDeviceToHost);
    double am = 0;
    for (double v : r) am += v;
    am /= N;
    features_kernel<<<(N + 127) / 128, 128, 0, c->stream>>>(N, am, c->L, c->b.pair_off, c->npairs, c->b.pair_j,
                                                             c->pairs_ok[0] ? (const float *)c->b.pair_x[0] : nullptr,
                                                             c->pairs_ok[0] ? nullptr : (const double *)c->b.pair_x[1],
                                                             c->b.rad, c->b.perm, feat);
    c->launches++;
    SE_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    return SE_OK;
}

extern "C" int se_mlp_forward(const float *w, const float *X, int n, float *Y, void *stream)
{
    if (!w || !X || !Y || n < 1) return SE_ERR_ARG;
    mlp_forward_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(w, X, n, Y);
    return cudaGetLastError() == cudaSuccess ? SE_OK : SE_ERR_CUDA;
}

extern "C" int se_mlp_grad(const float *w, const float *X, const float *Yt, int n, float *grad, float *loss,
                           float *scratch, size_t scratch_floats, void *stream)
{
    if (!w || !X || !Yt || !grad || !loss || !scratch || n < 1) return SE_ERR_ARG;
    if (scratch_floats < (size_t)n * kSampleStride) return SE_ERR_TOO_LARGE;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return SE_ERR_CUDA;
    mlp_sample_grad_kernel<<<(n + 127) / 128, 128, 0, s>>>(w, X, Yt, n, scratch, loss);
    mlp_reduce_grad_kernel<<<(kNTrain + 127) / 128, 128, 0, s>>>(scratch, n, grad);
    return cudaGetLastError() == cudaSuccess ? SE_OK : SE_ERR_CUDA;
}

extern "C" int se_mlp_adam_step(float *w, float *m, float *v, const float *grad, int step, float lr, void *stream)
{
    if (!w || !m || !v || !grad || step < 1) return SE_ERR_ARG;
    adam_kernel<<<(kNTrain + 127) / 128, 128, 0, (cudaStream_t)stream>>>(w, m, v, grad, step, lr);
    return cudaGetLastError() == cudaSuccess ? SE_OK : SE_ERR_CUDA;
}
