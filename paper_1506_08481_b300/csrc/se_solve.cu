// se_solve: M_inf . x = b by right-preconditioned restarted flexible GMRES (Sec. 4.1;
// the preconditioned vectors are stored, so a preconditioner evaluated in FP32 need
// not be exactly linear) with the block-diagonal far-field preconditioner of Sec. 4.2.
//
// Far-field-only reading of Sec. 4.2: with no lubrication (R^nf = 0) the
// preconditioner is the inverse of the block diagonal of M_inf, each block being
// the sphere's self mobility plus the interaction with its own periodic images
// (Eq. rfu-approx with the near-field blocks set to zero).  ILU0 of a dense block
// is its exact LU, so each block is inverted exactly.  Because the block depends
// only on the radius a (and the box), it is a polynomial of degree 2 in a^2 plus
// the isolated-sphere terms; the polynomial is sampled with single-sphere Spectral
// Ewald products (the same operator the solver inverts) at three radii.
//
// Precision: Krylov vectors, Gram-Schmidt (CGS2) and the true residual b - M x are
// FP64; Krylov products run at the context's compute precision.  Each restart
// starts from the FP64 true residual, which is the iterative-refinement step when
// products are FP32.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "se_internal.cuh"

namespace se {

namespace {

constexpr int kRedBlocks = 296;

// part[i * kRedBlocks + blk] = partial sum of V_i . w (V_i = V + i * ld)
__global__ void mdot_partial(const double *V, size_t ld, size_t n, const double *w, double *part)
{
    const int i = blockIdx.y;
    const double *v = V + (size_t)i * ld;
    double s = 0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        s += v[e] * w[e];
    __shared__ double sm[32];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (threadIdx.x == 0) part[(size_t)i * gridDim.x + blockIdx.x] = s;
    }
}

__global__ void mdot_final(const double *part, int nblk, double *out)
{
    const int i = blockIdx.x;
    double s = 0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[(size_t)i * nblk + b];
    __shared__ double sm[32];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (threadIdx.x == 0) out[i] = s;
    }
}

// w -= sum_i h[i] V_i   (h on the device)
__global__ void maxpy_kernel(const double *V, size_t ld, size_t n, int k, const double *h, double *w)
{
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double s = w[e];
        for (int i = 0; i < k; ++i) s -= h[i] * V[(size_t)i * ld + e];
        w[e] = s;
    }
}

// out = sum_i y[i] V_i
__global__ void combine_kernel(const double *V, size_t ld, size_t n, int k, const double *y, double *out)
{
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double s = 0;
        for (int i = 0; i < k; ++i) s += y[i] * V[(size_t)i * ld + e];
        out[e] = s;
    }
}

__global__ void axpby_kernel(size_t n, double a, const double *x, double b, const double *y, double *out)
{
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        out[e] = a * x[e] + b * y[e];
}

// the rigid-particle operator (11 components per particle): ms = v with the force and
// torque slots zeroed; out -= the force and torque slots of v
__global__ void mixed_mask_kernel(int N, const double *v, double *ms)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int c = 0; c < 11; ++c) ms[(size_t)i * 11 + c] = c < 6 ? 0.0 : v[(size_t)i * 11 + c];
}
__global__ void mixed_fix_kernel(int N, const double *v, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int c = 0; c < 6; ++c) out[(size_t)i * 11 + c] -= v[(size_t)i * 11 + c];
}

template <typename TI, typename TO>
__global__ void convert_kernel(size_t n, const TI *x, TO *y)
{
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        y[e] = (TO)x[e];
}

// z_p = B_p^{-1} v_p for every particle p (blocks nc x nc, caller order)
__global__ void block_apply_kernel(int N, int nc, const double *Binv, const double *v, double *z)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const double *B = Binv + (size_t)p * nc * nc;
    const double *vp = v + (size_t)p * nc;
    double *zp = z + (size_t)p * nc;
    for (int a = 0; a < nc; ++a) {
        double s = 0;
        for (int b = 0; b < nc; ++b) s += B[a * nc + b] * vp[b];
        zp[a] = s;
    }
}

// Block of particle with radius a: isolated-sphere self terms + C0 + a^2 C1 + a^4 C2
// (the diagonal block M_ii), shifted to alpha I + beta M_ii (the diagonal block of the
// operator alpha I + beta M; alpha = 0, beta = 1 for M itself), inverted by Gauss-Jordan
// elimination with partial pivoting.  Sorted particle k is stored at caller index
// perm[k].  Singular blocks fall back to the shifted isolated-sphere inverse (counted in
// *fallbacks).  mixed = 1 (the rigid-particle system of se_rigid_solve, nc = 11): the
// columns of the force and torque unknowns are replaced by -I (they hold U, Omega there).
__global__ void block_build_kernel(int N, int nc, double eta, const double *rad, const int *perm,
                                   const double *C /*[3][12][12]*/, double alpha, double beta, int mixed,
                                   double *Binv, int *fallbacks)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const double a = rad[k], a2 = a * a;
    double A[kNC][2 * kNC];
    const double pi = kPi;
    for (int r = 0; r < nc; ++r) {
        for (int q = 0; q < nc; ++q) {
            A[r][q] = C[r * kNC + q] + a2 * C[kNC * kNC + r * kNC + q] + a2 * a2 * C[2 * kNC * kNC + r * kNC + q];
            A[r][nc + q] = r == q ? 1.0 : 0.0;
        }
        const double iso = r < 3 ? 1.0 / (6 * pi * eta * a)
                         : r < 6 ? 1.0 / (8 * pi * eta * a * a2)
                         : r < 11 ? 3.0 / (20 * pi * eta * a * a2) : 3.0 / (16 * pi * eta * a * a2);
        A[r][r] += iso;
        for (int q = 0; q < nc; ++q) A[r][q] *= beta;
        A[r][r] += alpha;
        if (mixed)
            for (int q = 0; q < 6; ++q) A[r][q] = r == q ? -1.0 : 0.0;
    }
    bool ok = true;
    for (int col = 0; col < nc && ok; ++col) {
        int piv = col;
        for (int r = col + 1; r < nc; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (!(fabs(A[piv][col]) > 1e-300)) { ok = false; break; }
        if (piv != col)
            for (int q = 0; q < 2 * nc; ++q) { double t = A[col][q]; A[col][q] = A[piv][q]; A[piv][q] = t; }
        const double inv = 1.0 / A[col][col];
        for (int q = 0; q < 2 * nc; ++q) A[col][q] *= inv;
        for (int r = 0; r < nc; ++r) {
            if (r == col) continue;
            const double f = A[r][col];
            if (f != 0.0)
                for (int q = 0; q < 2 * nc; ++q) A[r][q] -= f * A[col][q];
        }
    }
    double *out = Binv + (size_t)perm[k] * nc * nc;
    bool fell_back = false;
    for (int r = 0; r < nc; ++r)
        for (int q = 0; q < nc; ++q) {
            double v = A[r][nc + q];
            if (!ok || !isfinite(v)) {
                const double mob = r < 3 ? 1.0 / (6 * pi * eta * a) : r < 6 ? 1.0 / (8 * pi * eta * a * a2)
                                 : r < 11 ? 3.0 / (20 * pi * eta * a * a2) : 3.0 / (16 * pi * eta * a * a2);
                v = r == q ? (mixed && r < 6 ? -1.0 : 1.0 / (alpha + beta * mob)) : 0.0;
                fell_back = true;
            }
            out[r * nc + q] = v;
        }
    if (fell_back) atomicAdd(fallbacks, 1);
}

}  // namespace

void convert_f2d(int n, const float *x, double *y, cudaStream_t s)
{
    convert_kernel<float, double><<<(n + 255) / 256, 256, 0, s>>>((size_t)n, x, y);
}

static int grid_for(size_t n) { size_t g = (n + 255) / 256; return (int)(g > 4096 ? 4096 : (g < 1 ? 1 : g)); }

// ---------------------------------------------------------------- preconditioner

static int build_blocks(se_ctx *c, int ncomp, bool learned, double alpha, double beta, int mixed = 0);

static int build_precond(se_ctx *c, int ncomp, bool learned)
{
    cudaStream_t s = c->stream;
    const int N = (int)c->N;
    // radii range (sorted copy)
    std::vector<double> rad(N);
    SE_CUDA_CHECK(c, cudaMemcpy(rad.data(), c->b.rad, N * sizeof(double), cudaMemcpyDeviceToHost));
    double amin = rad[0], amax = rad[0], asum = 0;
    for (double a : rad) { amin = a < amin ? a : amin; amax = a > amax ? a : amax; asum += a; }
    const bool mono = amax - amin <= 1e-12 * amax;
    const double aref = asum / N;
    const double samples[3] = {0.5 * aref, aref, 1.5 * aref};
    const int nsamp = mono ? 1 : 3;

    // single-sphere Spectral Ewald products in FP64 with the same parameters
    se_ctx *sc = nullptr;
    int rc = se_create(&sc, c->device, (void *)s);
    if (rc != SE_OK) { c->err = "preconditioner: se_create failed"; return rc; }
    rc = se_set_params(sc, c->xi, c->M, c->P, c->rc);
    if (rc == SE_OK) rc = se_set_option(sc, SE_OPT_PRECISION, 1);
    if (rc == SE_OK) rc = se_set_option(sc, SE_OPT_SIZE_MODE, c->size_mode);
    if (rc == SE_OK) rc = se_set_option(sc, SE_OPT_SHEAR, c->shear);
    if (rc == SE_OK) rc = se_set_option(sc, SE_OPT_ETA, c->eta);
    if (rc == SE_OK && c->m_user) rc = se_set_option(sc, SE_OPT_SHAPE_M, c->m_shape);
    if (rc == SE_OK) rc = se_set_option(sc, SE_OPT_PARTS, 2);   // wave space only (no real-space neighbours)
    double *d = nullptr;                                         // pos(3) rad(1) x(12) y(12)
    if (rc == SE_OK && cudaMalloc(&d, 28 * sizeof(double)) != cudaSuccess) rc = SE_ERR_NOMEM;
    std::vector<double> blocks(3 * kNC * kNC, 0.0);
    for (int si = 0; si < nsamp && rc == SE_OK; ++si) {
        const double a = mono ? aref : samples[si];
        double h[4] = {0.5 * c->L, 0.5 * c->L, 0.5 * c->L, a};
        cudaMemcpy(d, h, 4 * sizeof(double), cudaMemcpyHostToDevice);
        rc = se_set_config(sc, 1, c->L, d, d + 3);
        for (int col = 0; col < ncomp && rc == SE_OK; ++col) {
            double e[kNC] = {0};
            e[col] = 1.0;
            cudaMemcpyAsync(d + 4, e, kNC * sizeof(double), cudaMemcpyHostToDevice, s);
            rc = se_mobility_apply(sc, kNC, d + 4, d + 16, SE_F64);
            double y[kNC];
            cudaMemcpyAsync(y, d + 16, kNC * sizeof(double), cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
            for (int r = 0; r < kNC; ++r) blocks[(size_t)si * kNC * kNC + r * kNC + col] = y[r];
        }
    }
    if (rc != SE_OK) c->err = std::string("preconditioner: ") + se_last_error(sc);
    se_destroy(sc);
    if (d) cudaFree(d);
    if (rc != SE_OK) return rc;

    // self-image blocks minus nothing (wave + wave-self only): fit C0 + C1 a^2 + C2 a^4
    std::vector<double> C(3 * kNC * kNC, 0.0);
    // subtract the wave self term? No: the wave-only product of a single sphere is exactly the
    // image interaction plus the wave sum's own self interaction; the self removal is added below.
    for (int e = 0; e < kNC * kNC; ++e) {
        if (mono) { C[e] = blocks[e]; continue; }
        const double x0 = samples[0] * samples[0], x1 = samples[1] * samples[1], x2 = samples[2] * samples[2];
        const double y0 = blocks[e], y1 = blocks[kNC * kNC + e], y2 = blocks[2 * kNC * kNC + e];
        // quadratic through (x_i, y_i) in the variable a^2
        const double l0 = y0 / ((x0 - x1) * (x0 - x2)), l1 = y1 / ((x1 - x0) * (x1 - x2)),
                     l2 = y2 / ((x2 - x0) * (x2 - x1));
        C[2 * kNC * kNC + e] = l0 + l1 + l2;
        C[kNC * kNC + e] = -(l0 * (x1 + x2) + l1 * (x0 + x2) + l2 * (x0 + x1));
        C[e] = l0 * x1 * x2 + l1 * x0 * x2 + l2 * x0 * x1;
    }
    // wave-space self removal (Eq. uf-self and its rotation / strain analogues)
    {
        const double xi = c->xi, eta = c->eta, x2 = xi * xi, pi32 = kPi * std::sqrt(kPi);
        for (int r = 0; r < kNC; ++r) {
            double c0 = 0, c1 = 0, c2 = 0;
            if (r < 3) { c0 = 9 * xi; c1 = -10 * xi * x2; c2 = 7 * xi * x2 * x2; c0 /= 18 * pi32 * eta; c1 /= 18 * pi32 * eta; c2 /= 18 * pi32 * eta; }
            else if (r < 6) { c0 = 5 * xi * x2 / (12 * pi32 * eta); }
            else if (r < 11) { c0 = 25 * xi * x2 / (50 * pi32 * eta); c1 = -42 * xi * x2 * x2 / (50 * pi32 * eta); c2 = 27 * xi * x2 * x2 * x2 / (50 * pi32 * eta); }
            if (mono) {
                const double a2 = aref * aref;
                C[r * kNC + r] -= c0 + c1 * a2 + c2 * a2 * a2;
            } else {
                C[r * kNC + r] -= c0;
                C[kNC * kNC + r * kNC + r] -= c1;
                C[2 * kNC * kNC + r * kNC + r] -= c2;
            }
        }
    }
    // the fitted coefficients stay with the configuration: shifted blocks (alpha I +
    // beta M_ii, the Brownian IVP's systems) are rebuilt from them without new products
    if (!c->b.pc_C) SE_CUDA_CHECK(c, cudaMalloc(&c->b.pc_C, C.size() * sizeof(double)));
    SE_CUDA_CHECK(c, cudaMemcpyAsync(c->b.pc_C, C.data(), C.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    c->pc_ready = false;
    return build_blocks(c, ncomp, learned, 0.0, 1.0);
}

// the inverse blocks of alpha I + beta M_ii from the fitted coefficients
static int build_blocks(se_ctx *c, int ncomp, bool learned, double alpha, double beta, int mixed)
{
    (void)learned;
    cudaStream_t s = c->stream;
    const int N = (int)c->N;
    if (c->b.pc_inv) cudaFree(c->b.pc_inv);
    c->b.pc_inv = nullptr;
    c->pc_ready = false;
    if (cudaMalloc(&c->b.pc_inv, (size_t)N * ncomp * ncomp * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->err = "preconditioner allocation failed";
        return SE_ERR_NOMEM;
    }
    int *dfb = nullptr;
    if (cudaMalloc(&dfb, sizeof(int)) != cudaSuccess) { cudaGetLastError(); return SE_ERR_NOMEM; }
    cudaMemsetAsync(dfb, 0, sizeof(int), s);
    block_build_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, ncomp, c->eta, c->b.rad, c->b.perm, c->b.pc_C, alpha,
                                                       beta, mixed, c->b.pc_inv, dfb);
    c->launches++;
    int fb = 0;
    cudaMemcpyAsync(&fb, dfb, sizeof(int), cudaMemcpyDeviceToHost, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(dfb);
    if (e != cudaSuccess) {
        c->err = std::string("preconditioner blocks: ") + cudaGetErrorString(e);
        return SE_ERR_CUDA;
    }
    c->pc_fallbacks = fb;
    c->pc_ready = true;
    c->pc_ncomp = ncomp;
    c->pc_kind = SE_PRECOND_BLOCK;
    c->pc_alpha = alpha;
    c->pc_beta = beta;
    c->pc_mixed = mixed;
    return SE_OK;
}

// ---------------------------------------------------------------- GMRES

struct Gm {
    se_ctx *c;
    size_t n;
    double *part, *hd;
    int dots(const double *V, size_t ld, int k, const double *w, double *h_host)
    {
        cudaStream_t s = c->stream;
        mdot_partial<<<dim3(kRedBlocks, k), 256, 0, s>>>(V, ld, n, w, part);
        mdot_final<<<k, 256, 0, s>>>(part, kRedBlocks, hd);
        c->launches += 2;
        SE_CUDA_CHECK(c, cudaMemcpyAsync(h_host, hd, k * sizeof(double), cudaMemcpyDeviceToHost, s));
        SE_CUDA_CHECK(c, cudaStreamSynchronize(s));
        return SE_OK;
    }
    int axpy_multi(const double *V, size_t ld, int k, const double *h_host, double *w)
    {
        cudaStream_t s = c->stream;
        SE_CUDA_CHECK(c, cudaMemcpyAsync(hd, h_host, k * sizeof(double), cudaMemcpyHostToDevice, s));
        maxpy_kernel<<<grid_for(n), 256, 0, s>>>(V, ld, n, k, hd, w);
        c->launches++;
        return SE_OK;
    }
};


// ---------------------------------------------------------------- spectral correction
//
// SE_PRECOND_SPECTRAL = block preconditioner minus a correction of the long-wavelength
// force modes.  For a transverse plane wave of the forces, f_j = e^{i k.r_j} u (u . k = 0),
// M f is close to lambda(k) f with lambda(k) = A/k^2 + l0: the collective Stokes mobility
// n/(eta k^2) of the suspension (A comes out near n/eta) plus a bulk term.  These modes
// carry the largest eigenvalues of the preconditioned operator (cond(M) grows like L^2).
// With S = diag(s_i), s_i^2 the force diagonal of particle i's block, the preconditioner
// is P^-1 = B - S C S on the force components, C = sum over 0 < |k| <= k_c of
// (1/N) e^{i k.r_i} h(k) P_T(k) e^{-i k.r_j}, h(k) = theta (1 - 1/lambda(k))^+, lambda(k)
// the Rayleigh quotient of S M S on the mode: the scaled mode goes to (1 - theta) lambda
// + theta times itself, and P^-1 stays positive definite for any size mix (h < 1).
// The cutoff k_c is where the fitted lambda falls to 1.2, so h decays to zero there.  C is a forces-only wave-space product on a coarse grid whose k-space kernel
// is the table h(|k|)/N; A and l0 come from three probe shells (one product each);
// k_c a = 0.9 stays below the structure peak of the suspension.

__global__ void unpermute_pos_kernel(int N, const double *pos_cell, const int *perm, double *pos_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int j = perm[i];
    for (int d = 0; d < 3; ++d) pos_out[3 * j + d] = pos_cell[3 * i + d];
}

__global__ void fill_kernel(int n, double v, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = v;
}

// z[i][0..2] = Re sum_m (ar_m + i ai_m) e^{i k_m . r_i}, other components 0
__global__ void probe_kernel(int N, int ncomp, int nmode, const double *pos, const double *modes /*[nmode][9]*/,
                             double *z)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double f[3] = {0, 0, 0};
    for (int m = 0; m < nmode; ++m) {
        const double *md = modes + 9 * m;
        const double ph = md[0] * pos[3 * i] + md[1] * pos[3 * i + 1] + md[2] * pos[3 * i + 2];
        const double cs = cos(ph), sn = sin(ph);
        for (int d = 0; d < 3; ++d) f[d] += md[3 + d] * cs - md[6 + d] * sn;
    }
    for (int c = 0; c < ncomp; ++c) z[(size_t)i * ncomp + c] = c < 3 ? f[c] : 0.0;
}

// s_i = sqrt of the mean force diagonal of particle i's preconditioner block
__global__ void force_scale_kernel(int N, int ncomp, const double *Binv, double *s)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double *B = Binv + (size_t)i * ncomp * ncomp;
    const double d = (B[0] + B[ncomp + 1] + B[2 * ncomp + 2]) / 3.0;
    s[i] = sqrt(d > 0 ? d : 0.0);
}

// f = s v_F (the force components of v, scaled)
__global__ void take_forces_kernel(int N, int ncomp, const double *s, const double *v, double *f)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int d = 0; d < 3; ++d) f[3 * i + d] = s[i] * v[(size_t)i * ncomp + d];
}

// z_F -= s u
__global__ void sub_forces_kernel(int N, int ncomp, const double *s, const double *u, double *z)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int d = 0; d < 3; ++d) z[(size_t)i * ncomp + d] -= s[i] * u[3 * i + d];
}

// v[i] = uniform(-1, 1) from a counter hash (start vector of the power iteration)
__global__ void hash_fill_kernel(size_t n, unsigned seed, double *v)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long x = (unsigned long long)i * 0x9E3779B97F4A7C15ull + seed;
    x ^= x >> 33; x *= 0xFF51AFD7ED558CCDull; x ^= x >> 33; x *= 0xC4CEB9FE1A85EC53ull; x ^= x >> 33;
    v[i] = (double)(x >> 11) / 4503599627370496.0 - 1.0;
}

// z_F *= s (in place)
__global__ void scale_forces_kernel(int N, int ncomp, const double *s, double *z)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int d = 0; d < 3; ++d) z[(size_t)i * ncomp + d] *= s[i];
}

void free_spectral(se_ctx *c)
{
    if (c->spc) se_destroy(c->spc);
    c->spc = nullptr;
    if (c->sp_f) cudaFree(c->sp_f);
    if (c->sp_u) cudaFree(c->sp_u);
    if (c->sp_s) cudaFree(c->sp_s);
    c->sp_f = c->sp_u = c->sp_s = nullptr;
}

// Lanczos steps of the estimate of the largest eigenvalue of the correction C
constexpr int kLanczos = 48;

// theta_in, ka_in, cmax_in: the damping, the cutoff k_c <a> and the cap of the largest
// eigenvalue of C (<= 0: the options SE_OPT_PC_THETA / _KA / _CMAX and their defaults)
static int build_spectral(se_ctx *c, int ncomp, Gm &gm, double *z, double *w, double theta_in = 0,
                          double ka_in = 0, double cmax_in = 0)
{
    cudaStream_t s = c->stream;
    const int N = (int)c->N;
    free_spectral(c);
    std::vector<double> rad(N);
    SE_CUDA_CHECK(c, cudaMemcpy(rad.data(), c->b.rad, N * sizeof(double), cudaMemcpyDeviceToHost));
    double asum = 0;
    for (double a : rad) asum += a;
    // damping: 0.9 unless given (the best single value over 160 generated mono-, bi- and
    // polydisperse configurations; the best per configuration ranges from 0.8 to 0.98),
    // at most the cap left by earlier stalls on this configuration
    const double theta = std::min(c->sp_theta_cap, theta_in > 0 ? theta_in : (c->sp_theta > 0 ? c->sp_theta : 0.9));
    c->sp_theta_used = theta;
    const double ka = ka_in > 0 ? ka_in : c->sp_ka;
    c->sp_cmax_used = cmax_in > 0 ? cmax_in : c->sp_cmax;
    c->spc_theta = theta_in;
    c->spc_ka = ka_in;
    c->spc_cmax = cmax_in;
    const double aref = asum / N, L = c->L, k1 = 2 * kPi / L;
    double kc = ka / aref;
    if (kc <= 1.5 * k1) return SE_OK;                       // box too small: no long waves to correct
    // coarse grid with Nyquist wave number >= 2.5 k_c
    int Mc = 16;
    const int sizes[] = {16, 24, 32, 48, 64, 72, 96, 128, 144, 192, 216, 256};
    for (int q : sizes) { Mc = q; if (kPi * q / L >= 2.5 * kc) break; }
    // probe shells: |n|^2 = 1, about (n_c/2)^2 and n_c^2 (n_c = k_c / k1)
    const double nc = kc / k1;
    const int targets[3] = {1, std::max(2, (int)std::lround(0.25 * nc * nc)), std::max(3, (int)std::floor(nc * nc))};
    double lamT[3], lamB[3], kk[3];
    double *modes_d = nullptr;
    SE_CUDA_CHECK(c, cudaMalloc(&modes_d, 9 * 64 * sizeof(double)));
    unsigned long long rng = 0x9e3779b97f4a7c15ull;
    auto urand = [&]() { rng ^= rng << 13; rng ^= rng >> 7; rng ^= rng << 17; return (double)(rng >> 11) / 9007199254740992.0; };
    auto gauss = [&]() { const double u1 = std::max(urand(), 1e-300), u2 = urand(); return std::sqrt(-2 * std::log(u1)) * std::cos(2 * kPi * u2); };
    double *posc = nullptr;
    SE_CUDA_CHECK(c, cudaMalloc(&posc, 3 * (size_t)N * sizeof(double)));
    SE_CUDA_CHECK(c, cudaMalloc(&c->sp_s, (size_t)N * sizeof(double)));
    unpermute_pos_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, c->b.pos, c->b.perm, posc);
    force_scale_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, ncomp, c->b.pc_inv, c->sp_s);
    int rc = SE_OK;
    for (int t = 0; t < 3 && rc == SE_OK; ++t) {
        // modes with |n|^2 = target (nearest populated shell above it), at most 64
        std::vector<double> md;
        double k2sum = 0;
        int r2 = targets[t];
        for (; md.empty() && r2 < targets[t] + 64; ++r2) {
            const int R = (int)std::ceil(std::sqrt((double)r2));
            for (int a = -R; a <= R && md.size() < 9 * 64; ++a)
                for (int b2 = -R; b2 <= R && md.size() < 9 * 64; ++b2)
                    for (int cc = -R; cc <= R && md.size() < 9 * 64; ++cc) {
                        if (a * a + b2 * b2 + cc * cc != r2) continue;
                        // the reciprocal lattice of the (sheared) cell: k = k1 (a, b - gamma a, c)
                        const double kv[3] = {k1 * a, k1 * (b2 - c->shear * a), k1 * cc};
                        const double kn = std::sqrt(kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2]);
                        k2sum += kn * kn;
                        double ar[3], ai[3];
                        for (int d = 0; d < 3; ++d) { ar[d] = gauss(); ai[d] = gauss(); }
                        double pr = 0, pi_ = 0;
                        for (int d = 0; d < 3; ++d) { pr += ar[d] * kv[d] / kn; pi_ += ai[d] * kv[d] / kn; }
                        for (int d = 0; d < 3; ++d) { ar[d] -= pr * kv[d] / kn; ai[d] -= pi_ * kv[d] / kn; }
                        md.insert(md.end(), {kv[0], kv[1], kv[2], ar[0], ar[1], ar[2], ai[0], ai[1], ai[2]});
                    }
        }
        const int nm = (int)(md.size() / 9);
        kk[t] = std::sqrt(k2sum / std::max(nm, 1));     // the shell's rms |k| (k1 sqrt(n^2) in the cube)
        cudaMemcpyAsync(modes_d, md.data(), md.size() * sizeof(double), cudaMemcpyHostToDevice, s);
        probe_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, ncomp, nm, posc, modes_d, z);
        c->launches++;
        double zz, zMz;
        if ((rc = gm.dots(z, 0, 1, z, &zz)) != SE_OK) break;
        // Rayleigh quotient of S M S on the plane-wave combination
        scale_forces_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, ncomp, c->sp_s, z);
        c->launches++;
        rc = se_apply_internal(c, ncomp, z, w, SE_F64, c->precision);
        if (rc != SE_OK) break;
        if ((rc = gm.dots(z, 0, 1, w, &zMz)) != SE_OK) break;
        lamT[t] = zMz / zz;
        lamB[t] = 1.0;
    }
    cudaFree(modes_d);
    if (rc != SE_OK) { cudaFree(posc); return rc; }
    // least squares lambda = A / k^2 + l0 over the three shells
    double sxx = 0, sx = 0, sy = 0, sxy = 0;
    for (int t = 0; t < 3; ++t) {
        const double xk = 1.0 / (kk[t] * kk[t]);
        sxx += xk * xk; sx += xk; sy += lamT[t]; sxy += xk * lamT[t];
    }
    const double A = (3 * sxy - sx * sy) / (3 * sxx - sx * sx), l0 = (sy - A * sx) / 3;
    const double lB = (lamB[0] + lamB[1] + lamB[2]) / 3;
    if (A > 0 && 1.2 * lB - l0 > 0) kc = std::min(2.0 / aref, std::max(kc, std::sqrt(A / (1.2 * lB - l0))));
    {
        int q = 16;
        for (int s2 : sizes) { q = s2; if (kPi * s2 / L >= 2.5 * kc) break; }
        Mc = q;
    }
    c->sp_fit[0] = A;
    c->sp_fit[1] = l0;
    c->sp_fit[2] = lB;
    // table h(k)/N on [0, k_c]
    const int ntab = 512;
    std::vector<float> tab(ntab);
    for (int i = 0; i < ntab; ++i) {
        const double k = kc * i / (ntab - 1);
        // h = theta (1 - 1/lambda): a mode with the fitted lambda goes to
        // (1 - theta) lambda + theta; zero where the fit reaches 1 (at k_c, see above)
        double h = 0;
        const double lam = i > 0 ? A / (k * k) + l0 : 1e300;
        if (lam > lB) h = theta * (1.0 - lB / lam);
        tab[i] = (float)(h / N);
    }
    // coarse forces-only context with a tabulated kernel (wave part only, point forces)
    se_ctx *sc = nullptr;
    rc = se_create(&sc, c->device, (void *)s);
    if (rc != SE_OK) { cudaFree(posc); c->err = "spectral preconditioner: se_create failed"; return rc; }
    c->spc = sc;
    const int Pc = 8;
    sc->point_forces = true;                     // radii 1e-6 <a>: a sheared cell keeps size mode 1
    if (rc == SE_OK) rc = se_set_params(sc, 1.0, Mc, Pc, std::min(0.25 * L, 1.0));
    if (rc == SE_OK) rc = se_set_option(sc, SE_OPT_PRECISION, 0);
    if (rc == SE_OK) rc = se_set_option(sc, SE_OPT_SIZE_MODE, 1);
    if (rc == SE_OK) rc = se_set_option(sc, SE_OPT_SHEAR, c->shear);
    if (rc == SE_OK) rc = se_set_option(sc, SE_OPT_PARTS, 2);
    double *rtiny = nullptr;
    if (rc == SE_OK && cudaMalloc(&rtiny, (size_t)N * sizeof(double)) != cudaSuccess) rc = SE_ERR_NOMEM;
    if (rc == SE_OK) {
        fill_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, 1e-6 * aref, rtiny);
        rc = se_set_config(sc, N, L, posc, rtiny);
    }
    if (rtiny) cudaFree(rtiny);
    cudaFree(posc);
    if (rc == SE_OK) {
        if (cudaMalloc(&sc->ktab[0], ntab * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&c->sp_f, 3 * (size_t)N * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&c->sp_u, 3 * (size_t)N * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            rc = SE_ERR_NOMEM;
        }
    }
    if (rc == SE_OK) {
        cudaMemcpyAsync(sc->ktab[0], tab.data(), ntab * sizeof(float), cudaMemcpyHostToDevice, s);
        sc->ktab_n = ntab;
        sc->ktab_kmax = kc;
        sc->ktab_on = true;
        // On particle positions the plane waves are only nearly orthogonal, so |C| can
        // exceed max h (measured up to 1.11 at theta 0.98): C is symmetric positive
        // semi-definite, and its largest eigenvalue is estimated by kLanczos steps of
        // Lanczos (the largest Ritz value of the tridiagonal matrix, by Sturm bisection)
        // times 1.01; if that passes the cap c_max the table is scaled down to c_max,
        // which keeps I - C, and P^-1, positive definite.  (A 12-step power iteration
        // underestimated |C| by up to 10%: corrected cycles stalled on an indefinite P^-1.)
        const size_t n3 = 3 * (size_t)N;
        Gm g3{c, n3, gm.part, gm.hd};
        double *vp = z, *v = c->sp_f, *wv = c->sp_u;
        hash_fill_kernel<<<(unsigned)((n3 + 255) / 256), 256, 0, s>>>(n3, 12345u, v);
        SE_CUDA_CHECK(c, cudaMemsetAsync(vp, 0, n3 * sizeof(double), s));
        c->launches++;
        std::vector<double> al, be;           // diagonal alpha_j and off-diagonal beta_{j+1}
        double vv = 0;
        if ((rc = g3.dots(v, 0, 1, v, &vv)) == SE_OK && vv > 0) {
            axpby_kernel<<<grid_for(n3), 256, 0, s>>>(n3, 1.0 / std::sqrt(vv), v, 0.0, v, v);
            c->launches++;
        }
        double bprev = 0;
        for (int j = 0; j < kLanczos && rc == SE_OK; ++j) {
            rc = se_apply_internal(sc, 3, v, wv, SE_F64, 0);
            double a = 0, ww = 0;
            if (rc == SE_OK) rc = g3.dots(v, 0, 1, wv, &a);
            if (rc != SE_OK) break;
            axpby_kernel<<<grid_for(n3), 256, 0, s>>>(n3, -a, v, 1.0, wv, wv);
            axpby_kernel<<<grid_for(n3), 256, 0, s>>>(n3, -bprev, vp, 1.0, wv, wv);
            c->launches += 2;
            al.push_back(a);
            if ((rc = g3.dots(wv, 0, 1, wv, &ww)) != SE_OK) break;
            const double b = std::sqrt(std::max(ww, 0.0));
            if (!(b > 1e-12 * std::fabs(a)) || j + 1 == kLanczos) break;
            be.push_back(b);
            axpby_kernel<<<grid_for(n3), 256, 0, s>>>(n3, 1.0, v, 0.0, v, vp);
            axpby_kernel<<<grid_for(n3), 256, 0, s>>>(n3, 1.0 / b, wv, 0.0, wv, v);
            c->launches += 2;
            bprev = b;
        }
        // the largest eigenvalue of the tridiagonal matrix: bisection on the Sturm count
        double rho = 0;
        if (rc == SE_OK && !al.empty()) {
            const int K = (int)al.size();
            double lo = 1e300, hi = -1e300;
            for (int i = 0; i < K; ++i) {
                const double r = (i > 0 ? std::fabs(be[i - 1]) : 0.0) + (i + 1 < K ? std::fabs(be[i]) : 0.0);
                lo = std::min(lo, al[i] - r);
                hi = std::max(hi, al[i] + r);
            }
            auto below = [&](double x) {      // eigenvalues smaller than x
                int cnt = 0;
                double d = 1.0;
                for (int i = 0; i < K; ++i) {
                    const double b2 = i > 0 ? be[i - 1] * be[i - 1] : 0.0;
                    d = al[i] - x - (i > 0 ? b2 / (d != 0.0 ? d : 1e-300) : 0.0);
                    if (d < 0) ++cnt;
                }
                return cnt;
            };
            for (int it = 0; it < 100; ++it) {
                const double mid = 0.5 * (lo + hi);
                if (below(mid) >= K) hi = mid; else lo = mid;
            }
            rho = 1.01 * hi;
        }
        c->sp_rho = rho;
        const double cmax = c->sp_cmax_used;
        if (rc == SE_OK && rho > cmax) {
            for (float &v : tab) v = (float)(v * (cmax / rho));
            cudaMemcpyAsync(sc->ktab[0], tab.data(), ntab * sizeof(float), cudaMemcpyHostToDevice, s);
        }
        c->launches += sc->launches;
        sc->launches = 0;
        SE_CUDA_CHECK(c, cudaStreamSynchronize(s));
    }
    if (rc != SE_OK) {
        if (c->err.empty()) c->err = std::string("spectral preconditioner: ") + se_last_error(sc);
        free_spectral(c);
    }
    return rc;
}

// z = P^-1 v for the spectral preconditioner: block part, then minus the correction
static int spectral_apply(se_ctx *c, int ncomp, const double *v, double *z)
{
    cudaStream_t s = c->stream;
    const int N = (int)c->N;
    block_apply_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, ncomp, c->b.pc_inv, v, z);
    c->launches++;
    if (!c->spc) return SE_OK;
    take_forces_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, ncomp, c->sp_s, v, c->sp_f);
    c->launches++;
    const int rc = se_apply_internal(c->spc, 3, c->sp_f, c->sp_u, SE_F64, 0);
    if (rc != SE_OK) {
        c->err = std::string("spectral preconditioner: ") + c->spc->err;
        return rc;
    }
    c->launches += c->spc->launches;
    c->spc->launches = 0;
    sub_forces_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, ncomp, c->sp_s, c->sp_u, z);
    c->launches++;
    return SE_OK;
}

}  // namespace se

using namespace se;

// working-precision restart residuals are used while rel > kFp64Switch * rtol and they
// still fall by 2x per cycle
constexpr double kFp64Switch = 30.0;
// products after which a cycle of the spectral correction must have halved the residual
constexpr int kStallIts = 30;

// Krylov basis, preconditioned vectors, work vectors and reduction scratch for the
// context's restart length and n unknowns (kept between solves of the same size)
static int ensure_solver_work(se_ctx *c, size_t n)
{
    const int m = c->restart;
    if (c->b.kry && c->b.kry_n == n && c->b.kry_m == m) return SE_OK;
    if (c->b.kry) cudaFree(c->b.kry);
    if (c->b.work64) cudaFree(c->b.work64);
    if (c->b.red) cudaFree(c->b.red);
    c->b.kry = c->b.work64 = c->b.red = nullptr;
    c->b.kry_n = 0;
    // flexible GMRES: Krylov basis V [m + 1][n] and the preconditioned vectors Z [m][n]
    if (cudaMalloc(&c->b.kry, (size_t)(2 * m + 1) * n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->b.work64, 6 * n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->b.red, ((size_t)kRedBlocks * (m + 1) + 2 * (m + 1)) * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->err = "solver allocation failed";
        return SE_ERR_NOMEM;
    }
    c->b.kry_n = n;
    c->b.kry_m = m;
    return SE_OK;
}

// Right-preconditioned flexible GMRES(restart) on (alpha I + beta M) x = b, with M the
// grand mobility of the ncomp-prefix; bd and xd are FP64 device arrays [N][ncomp] (xd:
// initial guess in, solution out; neither may alias the work vectors).  The block
// preconditioner inverts the blocks of alpha I + beta M_ii; the learned and spectral
// corrections apply to M itself (alpha = 0, beta = 1) only, shifted systems take the
// block preconditioner.
//
// mixed = 1 (ncomp 11, alpha = 0, beta = 1): the rigid-particle system of se_rigid_solve,
// K w = M (P_S w) - P_FT w, whose unknowns w hold (U, Omega) in the force and torque
// slots and S in the stresslet slots (P_S, P_FT: the stresslet and force-torque parts).
static int solve_core(se_ctx *c, int ncomp, const double *bd, double *xd, double rtol, int maxit, int precond,
                      double alpha, double beta, int *iters, double *relres, int mixed = 0)
{
    cudaStream_t s = c->stream;
    const int m = c->restart;
    const size_t n = (size_t)c->N * ncomp;
    int rc = ensure_solver_work(c, n);
    if (rc != SE_OK) return rc;
    double *V = c->b.kry, *Zb = c->b.kry + (size_t)(m + 1) * n;
    double *r = c->b.work64, *w = r + n, *z = w + n;
    Gm gm{c, n, c->b.red, c->b.red + (size_t)kRedBlocks * (m + 1)};
    double *yd = gm.hd + (m + 1);
    const bool shifted = !(alpha == 0.0 && beta == 1.0);
    if ((shifted || mixed) && precond != SE_PRECOND_NONE) precond = SE_PRECOND_BLOCK;
    double *ms = c->b.work64 + 5 * n;     // the masked vector P_S v of the mixed operator

    // the learned preconditioner: the spectral correction with the damping and cutoff
    // the network predicts for this configuration; without weights (or where the
    // spectral correction does not apply) it is the plain block preconditioner
    double l_theta = 0, l_ka = 0, l_cmax = 0;
    if (precond == SE_PRECOND_LEARNED) {
        if (c->have_mlp && !shifted && !mixed) {
            rc = learned_spectral_params(c, &l_theta, &l_ka, &l_cmax);
            if (rc != SE_OK) return rc;
            precond = SE_PRECOND_SPECTRAL;
        } else {
            precond = SE_PRECOND_BLOCK;
        }
    }
    if (precond != SE_PRECOND_NONE) {
        if (!c->pc_ready || c->pc_ncomp != ncomp) {
            rc = build_precond(c, ncomp, false);
            if (rc != SE_OK) return rc;
            free_spectral(c);
        }
        if (c->pc_kind != SE_PRECOND_BLOCK || c->pc_alpha != alpha || c->pc_beta != beta || c->pc_mixed != mixed) {
            rc = build_blocks(c, ncomp, false, alpha, beta, mixed);
            if (rc != SE_OK) return rc;
            free_spectral(c);
        }
    }
    if (precond == SE_PRECOND_SPECTRAL &&
        (!c->spc || c->spc_theta != l_theta || c->spc_ka != l_ka || c->spc_cmax != l_cmax)) {
        rc = build_spectral(c, ncomp, gm, z, w, l_theta, l_ka, l_cmax);
        if (rc != SE_OK) return rc;
    }
    auto Pinv = [&](const double *v, double *out) -> int {
        if (precond == SE_PRECOND_NONE) {
            SE_CUDA_CHECK(c, cudaMemcpyAsync(out, v, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        } else if (precond == SE_PRECOND_SPECTRAL) {
            return spectral_apply(c, ncomp, v, out);
        } else {
            block_apply_kernel<<<((int)c->N + 127) / 128, 128, 0, s>>>((int)c->N, ncomp, c->b.pc_inv, v, out);
            c->launches++;
        }
        return SE_OK;
    };
    // out = (alpha I + beta M) v at product precision prec
    auto op = [&](const double *v, double *out, int prec) -> int {
        if (mixed) {
            mixed_mask_kernel<<<((int)c->N + 127) / 128, 128, 0, s>>>((int)c->N, v, ms);
            const int e = se_apply_internal(c, ncomp, ms, out, SE_F64, prec);
            if (e != SE_OK) return e;
            mixed_fix_kernel<<<((int)c->N + 127) / 128, 128, 0, s>>>((int)c->N, v, out);
            c->launches += 2;
            return SE_OK;
        }
        const int e = se_apply_internal(c, ncomp, v, out, SE_F64, prec);
        if (e != SE_OK || !shifted) return e;
        axpby_kernel<<<grid_for(n), 256, 0, s>>>(n, alpha, v, beta, out, out);
        c->launches++;
        return SE_OK;
    };

    double bn2, xn2;
    rc = gm.dots(bd, 0, 1, bd, &bn2);
    if (rc != SE_OK) return rc;
    if ((rc = gm.dots(xd, 0, 1, xd, &xn2)) != SE_OK) return rc;
    const double bnorm = std::sqrt(bn2);
    bool x_zero = xn2 == 0.0;          // a zero initial guess: the first residual is b itself
    int prods = 0;
    double rel = 0.0;
    std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), h(m + 1), h2(m + 1), yv(m);
    if (bnorm == 0.0) {
        SE_CUDA_CHECK(c, cudaMemsetAsync(xd, 0, n * sizeof(double), s));
    } else {
        // Residuals at the restarts: while the working-precision residual b - M x is well
        // above rtol (kFp64Switch rtol) it is formed with working-precision products
        // (accumulated in FP64): its FP32 rounding, a few 1e-7 of |M| |x|, is then small
        // against the residual itself.  Below that every restart uses the FP64 residual
        // (an FP64 product), so each further cycle is a step of iterative refinement on
        // the FP64 residual, and convergence is decided by it.
        bool fp64_res = c->precision >= 1;
        // the precision of the "FP64" residual products: FP64 or double-float (the same
        // accuracy; SE_OPT_RESIDUAL) when the Krylov products run in FP32
        const int res_prec = c->precision == 0 ? c->res_precision : c->precision;
        double rel_wp = 1.0;                  // the previous working-precision restart residual
        // A restart cycle of the spectral preconditioner that fails to halve the residual
        // (a damping too strong for this configuration makes the corrected operator nearly
        // singular on some modes) switches the remaining cycles to the plain block
        // preconditioner; flexible GMRES allows the change between cycles.
        double rel_cycle = -1.0;              // residual at the start of the last cycle
        int prods_cycle = 0;
        bool stalled = false;                 // the last cycle was cut short by a stall
        // A stall (the spectral correction's damping too strong for this configuration):
        // lower the damping by 0.05 for the rest of this solve and the next solves on the
        // configuration, and rebuild the correction; below 0.6 use the block preconditioner.
        auto relax_damping = [&]() -> int {
            c->pc_stalls++;
            const double th = c->sp_theta_used - 0.05;
            if (th < 0.6 || !c->spc) {
                precond = SE_PRECOND_BLOCK;
                return SE_OK;
            }
            c->sp_theta_cap = th;
            return build_spectral(c, ncomp, gm, z, w, l_theta, l_ka, l_cmax);
        };
        for (;;) {
            bool exact = fp64_res;            // r is the FP64 residual (or b itself)
            if (x_zero) {
                SE_CUDA_CHECK(c, cudaMemcpyAsync(r, bd, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
                x_zero = false;
                exact = true;
            } else {
                rc = op(xd, w, fp64_res ? res_prec : c->precision);
                if (rc != SE_OK) return rc;
                axpby_kernel<<<grid_for(n), 256, 0, s>>>(n, 1.0, bd, -1.0, w, r);
                c->launches++;
            }
            double rn2;
            rc = gm.dots(r, 0, 1, r, &rn2);
            if (rc != SE_OK) return rc;
            const double beta = std::sqrt(rn2);
            rel = beta / bnorm;
            if (!std::isfinite(rel)) { c->err = "non-finite residual"; return SE_ERR_NONFINITE; }
            // from here on the FP64 residual decides: near rtol, at maxit, or when the
            // working-precision residual stopped falling (its rounding floor lies above
            // rtol, so only refinement on the FP64 residual gets further)
            if (!exact && (rel <= kFp64Switch * rtol || prods >= maxit || rel > 0.5 * rel_wp)) {
                fp64_res = true;
                continue;
            }
            if (!exact) rel_wp = rel;
            if (rel <= rtol || prods >= maxit) break;
            if (precond == SE_PRECOND_SPECTRAL && rel > 10 * rtol &&
                (stalled || (rel_cycle > 0 && prods - prods_cycle >= std::min(m, kStallIts) && rel > 0.5 * rel_cycle))) {
                if ((rc = relax_damping()) != SE_OK) return rc;
            }
            stalled = false;
            rel_cycle = rel;
            prods_cycle = prods;
            axpby_kernel<<<grid_for(n), 256, 0, s>>>(n, 1.0 / beta, r, 0.0, r, V);
            c->launches++;
            std::fill(g.begin(), g.end(), 0.0);
            g[0] = beta;
            int k = 0;
            for (int j = 0; j < m && prods < maxit; ++j) {
                double *zj = Zb + (size_t)j * n;
                if ((rc = Pinv(V + (size_t)j * n, zj)) != SE_OK) return rc;
                rc = op(zj, w, c->precision);
                if (rc != SE_OK) return rc;
                ++prods;
                // classical Gram-Schmidt with selective reorthogonalisation (Daniel, Gragg,
                // Kaufman & Stewart 1976): a second pass only when the first one cancelled,
                // |w - V h|^2 < |w|^2 / 2 with |w|^2 = |h|^2 + |w - V h|^2
                if ((rc = gm.dots(V, n, j + 1, w, h.data())) != SE_OK) return rc;
                if ((rc = gm.axpy_multi(V, n, j + 1, h.data(), w)) != SE_OK) return rc;
                double wn2;
                if ((rc = gm.dots(w, 0, 1, w, &wn2)) != SE_OK) return rc;
                double hn2 = 0;
                for (int i = 0; i <= j; ++i) hn2 += h[i] * h[i];
                std::fill(h2.begin(), h2.begin() + (j + 1), 0.0);
                if (wn2 < 0.5 * (hn2 + wn2)) {
                    if ((rc = gm.dots(V, n, j + 1, w, h2.data())) != SE_OK) return rc;
                    if ((rc = gm.axpy_multi(V, n, j + 1, h2.data(), w)) != SE_OK) return rc;
                    if ((rc = gm.dots(w, 0, 1, w, &wn2)) != SE_OK) return rc;
                }
                const double hn = std::sqrt(wn2);
                for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h[i] + h2[i];
                H[(size_t)(j + 1) * m + j] = hn;
                // apply the previous Givens rotations to column j, then a new one
                for (int i = 0; i < j; ++i) {
                    const double a0 = H[(size_t)i * m + j], a1 = H[(size_t)(i + 1) * m + j];
                    H[(size_t)i * m + j] = cs[i] * a0 + sn[i] * a1;
                    H[(size_t)(i + 1) * m + j] = -sn[i] * a0 + cs[i] * a1;
                }
                const double a0 = H[(size_t)j * m + j], a1 = H[(size_t)(j + 1) * m + j];
                const double den = std::hypot(a0, a1);
                cs[j] = den > 0 ? a0 / den : 1.0;
                sn[j] = den > 0 ? a1 / den : 0.0;
                H[(size_t)j * m + j] = den;
                H[(size_t)(j + 1) * m + j] = 0.0;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                k = j + 1;
                if (hn > 0 && j + 1 < m + 1) {
                    axpby_kernel<<<grid_for(n), 256, 0, s>>>(n, 1.0 / hn, w, 0.0, w, V + (size_t)(j + 1) * n);
                    c->launches++;
                }
                if (std::fabs(g[j + 1]) <= 0.3 * rtol * bnorm || hn == 0.0) break;
                // a spectral cycle that has not halved the residual after kStallIts products
                // is cut short (the correction is rebuilt with less damping at the restart)
                if (precond == SE_PRECOND_SPECTRAL && j + 1 == kStallIts && j + 1 < m &&
                    std::fabs(g[j + 1]) > 0.5 * beta && std::fabs(g[j + 1]) > 10 * rtol * bnorm) {
                    stalled = true;
                    break;
                }
            }
            // y = H^{-1} g (upper triangular), x += Z y (flexible GMRES: the stored
            // preconditioned vectors, so an FP32-rounded preconditioner stays consistent)
            for (int i = k - 1; i >= 0; --i) {
                double sacc = g[i];
                for (int q = i + 1; q < k; ++q) sacc -= H[(size_t)i * m + q] * yv[q];
                yv[i] = sacc / H[(size_t)i * m + i];
            }
            SE_CUDA_CHECK(c, cudaMemcpyAsync(yd, yv.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
            combine_kernel<<<grid_for(n), 256, 0, s>>>(Zb, n, n, k, yd, w);
            c->launches++;
            axpby_kernel<<<grid_for(n), 256, 0, s>>>(n, 1.0, xd, 1.0, w, xd);
            c->launches++;
        }
    }
    SE_CUDA_CHECK(c, cudaStreamSynchronize(s));
    if (iters) *iters = prods;
    if (relres) *relres = rel;
    if (rel > rtol) {
        c->err = "GMRES did not reach rtol within maxit products";
        return SE_ERR_NOT_CONVERGED;
    }
    return SE_OK;
}

extern "C" int se_solve(se_ctx *c, int ncomp, const void *b, void *x, int dtype, double rtol, int maxit,
                        int precond, int *iters, double *relres)
{
    if (!c) return SE_ERR_ARG;
    if (!b || !x) { c->err = "null b or x"; return SE_ERR_ARG; }
    if (ncomp != 3 && ncomp != 6 && ncomp != 11 && ncomp != 12) { c->err = "ncomp must be 3, 6, 11 or 12"; return SE_ERR_ARG; }
    if (dtype != SE_F32 && dtype != SE_F64) { c->err = "bad dtype"; return SE_ERR_ARG; }
    if (!(rtol > 0) || maxit < 1) { c->err = "rtol must be > 0 and maxit >= 1"; return SE_ERR_ARG; }
    if (precond < SE_PRECOND_NONE || precond > SE_PRECOND_SPECTRAL) { c->err = "bad preconditioner"; return SE_ERR_ARG; }
    if (!c->have_config) { c->err = "se_set_config must be called first"; return SE_ERR_STATE; }
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    const size_t n = (size_t)c->N * ncomp;
    int rc = ensure_solver_work(c, n);
    if (rc != SE_OK) return rc;
    double *bd = c->b.work64 + 3 * n, *xd = bd + n;      // work vectors 3 and 4: b, x in FP64
    if (dtype == SE_F64) {
        SE_CUDA_CHECK(c, cudaMemcpyAsync(bd, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        SE_CUDA_CHECK(c, cudaMemcpyAsync(xd, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else {
        convert_kernel<float, double><<<grid_for(n), 256, 0, s>>>(n, (const float *)b, bd);
        convert_kernel<float, double><<<grid_for(n), 256, 0, s>>>(n, (const float *)x, xd);
        c->launches += 2;
    }
    rc = solve_core(c, ncomp, bd, xd, rtol, maxit, precond, 0.0, 1.0, iters, relres);
    if (rc != SE_OK && rc != SE_ERR_NOT_CONVERGED) return rc;
    if (dtype == SE_F64) {
        SE_CUDA_CHECK(c, cudaMemcpyAsync(x, xd, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else {
        convert_kernel<double, float><<<grid_for(n), 256, 0, s>>>(n, xd, (float *)x);
        c->launches++;
    }
    SE_CUDA_CHECK(c, cudaStreamSynchronize(s));
    return rc;
}

// ---------------------------------------------------------------- Brownian IVP
//
// x = M^{-1/2} c by the initial value problem of Sec. 4.3 (Eq. ivp-1): with A = s M
// (s a scale that brings A's self blocks near the identity), x(tau) solves
//   dx/dtau = -1/2 [tau I + (1 - tau) A]^{-1} (A - I) x,  x(0) = c,
// and x(1) = A^{-1/2} c, so M^{-1/2} c = sqrt(s) x(1).  n steps of size dtau = 1/n, each
// an explicit Euler half-step (Eq. ivp-forward) and an implicit one (Eq. ivp-backward):
//   [tau_i I + (1 - tau_i) A] y = (A - I) x_i,            x_{i+1/2} = x_i - (dtau/4) y,
//   [(tau_{i+1} - dtau/4) I + (1 - tau_{i+1} + dtau/4) A] x_{i+1}
//                                = [tau_{i+1} I + (1 - tau_{i+1}) A] x_{i+1/2},
// the second written with the operator multiplied through by tau_{i+1} I + (1 - tau_{i+1}) A.
// Both systems are solved by the GMRES above (block preconditioner of the shifted
// operator), the right-hand sides formed with one product each.
extern "C" int se_brownian_ivp(se_ctx *c, int ncomp, double scale, int nsteps, double rtol, int maxit,
                               const double *cvec, double *xout, int *products)
{
    if (!c) return SE_ERR_ARG;
    if (!cvec || !xout) { c->err = "null c or x"; return SE_ERR_ARG; }
    if (ncomp != 3 && ncomp != 6 && ncomp != 11) {
        c->err = "ncomp must be 3, 6 or 11 (the F, T, S block is symmetric positive definite)";
        return SE_ERR_ARG;
    }
    if (nsteps < 1 || nsteps > 10000 || !(rtol > 0) || maxit < 1) { c->err = "bad nsteps, rtol or maxit"; return SE_ERR_ARG; }
    if (!c->have_config) { c->err = "se_set_config must be called first"; return SE_ERR_STATE; }
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    const size_t n = (size_t)c->N * ncomp;
    if (!(scale > 0)) {
        // default: 6 pi eta <a>, so the translational self block of A is near the identity
        std::vector<double> rad(c->N);
        SE_CUDA_CHECK(c, cudaMemcpy(rad.data(), c->b.rad, c->N * sizeof(double), cudaMemcpyDeviceToHost));
        double am = 0;
        for (double a : rad) am += a;
        scale = 6 * kPi * c->eta * am / (double)c->N;
    }
    double *xv = nullptr, *yv = nullptr, *tv = nullptr;
    if (cudaMalloc(&xv, 3 * n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->err = "IVP allocation failed";
        return SE_ERR_NOMEM;
    }
    yv = xv + n;
    tv = yv + n;
    int total = 0, status = SE_OK;
    auto fail = [&](int rc) {
        cudaFree(xv);
        if (products) *products = total;
        return rc;
    };
    if (cudaMemcpyAsync(xv, cvec, n * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(yv, 0, n * sizeof(double), s) != cudaSuccess) {
        c->err = "IVP: copy of c failed";
        return fail(SE_ERR_CUDA);
    }
    const double dt = 1.0 / nsteps;
    for (int i = 0; i < nsteps; ++i) {
        const double t0 = i * dt, t1 = (i + 1) * dt;
        // forward half-step: t = (A - I) x, then [t0 I + (1 - t0) A] y = t
        int rc = se_apply_internal(c, ncomp, xv, tv, SE_F64, c->precision);
        if (rc != SE_OK) return fail(rc);
        axpby_kernel<<<grid_for(n), 256, 0, s>>>(n, -1.0, xv, scale, tv, tv);
        c->launches++;
        ++total;
        int it = 0;
        rc = solve_core(c, ncomp, tv, yv, rtol, maxit, SE_PRECOND_BLOCK, t0, (1 - t0) * scale, &it, nullptr);
        total += it;
        if (rc == SE_ERR_NOT_CONVERGED) status = rc;
        else if (rc != SE_OK) return fail(rc);
        axpby_kernel<<<grid_for(n), 256, 0, s>>>(n, 1.0, xv, -0.25 * dt, yv, xv);      // x_{i+1/2}
        c->launches++;
        // backward half-step: t = [t1 I + (1 - t1) A] x_{i+1/2}; x_{i+1} starts from x_{i+1/2}
        rc = se_apply_internal(c, ncomp, xv, tv, SE_F64, c->precision);
        if (rc != SE_OK) return fail(rc);
        axpby_kernel<<<grid_for(n), 256, 0, s>>>(n, t1, xv, (1 - t1) * scale, tv, tv);
        c->launches++;
        ++total;
        rc = solve_core(c, ncomp, tv, xv, rtol, maxit, SE_PRECOND_BLOCK, t1 - 0.25 * dt, (1 - t1 + 0.25 * dt) * scale,
                        &it, nullptr);
        total += it;
        if (rc == SE_ERR_NOT_CONVERGED) status = rc;
        else if (rc != SE_OK) return fail(rc);
    }
    axpby_kernel<<<grid_for(n), 256, 0, s>>>(n, std::sqrt(scale), xv, 0.0, xv, xout);
    c->launches++;
    const cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(xv);
    if (e != cudaSuccess) {
        c->err = std::string("IVP: ") + cudaGetErrorString(e);
        if (products) *products = total;
        return SE_ERR_CUDA;
    }
    if (products) *products = total;
    if (status != SE_OK) c->err = "a GMRES solve of the IVP did not reach rtol within maxit products";
    return status;
}

// ---------------------------------------------------------------- rigid particles and the
// far-field self-diffusivities
//
// Force- and torque-driven rigid spheres in the quiescent fluid (E = 0): from the grand
// mobility, [U; Omega; 0] = M [F; T; S] with S unknown, i.e. U = mu (F, T) with
// mu = M_UF - M_US M_ES^{-1} M_EF, the inverse of the FU block of the far-field resistance
// M^{-1} (Sec. 6.1, Eq. dstr-def: mu_ii are the diagonal blocks of R_FU^{-1}).  Written as
// one system for w = (U, Omega, S): M (P_S w) - P_FT w = -M [F; T; 0].

namespace se {
namespace {

// x11 = (F, T, 0) of particle i from ft [N][6] (ft may be null: zero forces and torques)
__global__ void embed_ft_kernel(int N, const double *ft, double *x11)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int c = 0; c < 11; ++c) x11[(size_t)i * 11 + c] = c < 6 && ft ? ft[(size_t)i * 6 + c] : 0.0;
}
// the right-hand side of the rigid-particle system: out = (0, 0, E_inf) - w11 (w11 = M (F, T, 0))
__global__ void rigid_rhs_kernel(int N, const double *w11, double e0, double e1, double e2, double e3, double e4,
                                 double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double e[5] = {e0, e1, e2, e3, e4};
    for (int c = 0; c < 11; ++c) out[(size_t)i * 11 + c] = (c < 6 ? 0.0 : e[c - 6]) - w11[(size_t)i * 11 + c];
}
__global__ void split_w_kernel(int N, const double *w, double *uw, double *sv)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int c = 0; c < 6; ++c) uw[(size_t)i * 6 + c] = w[(size_t)i * 11 + c];
    if (sv)
        for (int c = 0; c < 5; ++c) sv[(size_t)i * 5 + c] = w[(size_t)i * 11 + 6 + c];
}
// d[i] += ((U . F) / 3, (Omega . T) / 3) of one sample
__global__ void diffusivity_accum_kernel(int N, const double *ft, const double *uw, double *d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double t = 0, r = 0;
    for (int c = 0; c < 3; ++c) {
        t += uw[(size_t)i * 6 + c] * ft[(size_t)i * 6 + c];
        r += uw[(size_t)i * 6 + 3 + c] * ft[(size_t)i * 6 + 3 + c];
    }
    d[2 * i] += t / 3.0;
    d[2 * i + 1] += r / 3.0;
}

// one rigid-particle solve with device work arrays x11, w11 [N][11]; einf: the imposed
// strain rate on the orthonormal basis (5 host doubles) or null
int rigid_core(se_ctx *c, const double *ft, const double *einf, double *x11, double *w11, double rtol, int maxit,
               int *iters, double *relres)
{
    cudaStream_t s = c->stream;
    const int N = (int)c->N;
    const size_t n = (size_t)N * 11;
    const double z[5] = {0, 0, 0, 0, 0};
    const double *e = einf ? einf : z;
    embed_ft_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, ft, x11);
    c->launches++;
    // M [F; T; 0] at FP64 accuracy (FP64 or double-float products)
    int rc = se_apply_internal(c, 11, x11, w11, SE_F64, c->precision == 0 ? c->res_precision : c->precision);
    if (rc != SE_OK) return rc;
    rigid_rhs_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, w11, e[0], e[1], e[2], e[3], e[4], x11);
    c->launches++;
    SE_CUDA_CHECK(c, cudaMemsetAsync(w11, 0, n * sizeof(double), s));
    return solve_core(c, 11, x11, w11, rtol, maxit, SE_PRECOND_BLOCK, 0.0, 1.0, iters, relres, 1);
}

}  // namespace
}  // namespace se

extern "C" int se_rigid_solve(se_ctx *c, const double *ft, const double *einf, double *uw, double *sv, double rtol,
                              int maxit, int *iters, double *relres)
{
    if (!c) return SE_ERR_ARG;
    if (!uw) { c->err = "null U"; return SE_ERR_ARG; }
    if (!(rtol > 0) || maxit < 1) { c->err = "rtol must be > 0 and maxit >= 1"; return SE_ERR_ARG; }
    if (!c->have_config) { c->err = "se_set_config must be called first"; return SE_ERR_STATE; }
    cudaSetDevice(c->device);
    const int N = (int)c->N;
    const size_t n = (size_t)N * 11;
    double *x11 = nullptr;
    if (cudaMalloc(&x11, 2 * n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->err = "rigid solve allocation failed";
        return SE_ERR_NOMEM;
    }
    double *w11 = x11 + n;
    int rc = rigid_core(c, ft, einf, x11, w11, rtol, maxit, iters, relres);
    if (rc == SE_OK || rc == SE_ERR_NOT_CONVERGED) {
        split_w_kernel<<<(N + 127) / 128, 128, 0, c->stream>>>(N, w11, uw, sv);
        c->launches++;
        const cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            c->err = std::string("rigid solve: ") + cudaGetErrorString(e);
            rc = SE_ERR_CUDA;
        }
    }
    cudaFree(x11);
    return rc;
}

extern "C" int se_far_field_diffusivity(se_ctx *c, int nsamples, const double *fr, double *d, double rtol,
                                        int maxit, int *products)
{
    if (!c) return SE_ERR_ARG;
    if (!fr || !d || nsamples < 1) { c->err = "null F^R or d, or nsamples < 1"; return SE_ERR_ARG; }
    if (!(rtol > 0) || maxit < 1) { c->err = "rtol must be > 0 and maxit >= 1"; return SE_ERR_ARG; }
    if (!c->have_config) { c->err = "se_set_config must be called first"; return SE_ERR_STATE; }
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    const int N = (int)c->N;
    const size_t n = (size_t)N * 11;
    double *x11 = nullptr;
    if (cudaMalloc(&x11, (2 * n + (size_t)N * 6 + (size_t)N * 2) * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->err = "diffusivity allocation failed";
        return SE_ERR_NOMEM;
    }
    double *w11 = x11 + n, *uw = w11 + n, *acc = uw + (size_t)N * 6;
    int total = 0, status = SE_OK;
    cudaMemsetAsync(acc, 0, (size_t)N * 2 * sizeof(double), s);
    for (int k = 0; k < nsamples; ++k) {
        const double *ft = fr + (size_t)k * N * 6;
        int it = 0;
        int rc = rigid_core(c, ft, nullptr, x11, w11, rtol, maxit, &it, nullptr);
        total += it + 1;
        if (rc == SE_ERR_NOT_CONVERGED) status = rc;
        else if (rc != SE_OK) {
            cudaFree(x11);
            if (products) *products = total;
            return rc;
        }
        split_w_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, w11, uw, nullptr);
        diffusivity_accum_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, ft, uw, acc);
        c->launches += 2;
    }
    axpby_kernel<<<grid_for((size_t)N * 2), 256, 0, s>>>((size_t)N * 2, 1.0 / nsamples, acc, 0.0, acc, d);
    c->launches++;
    const cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(x11);
    if (products) *products = total;
    if (e != cudaSuccess) {
        c->err = std::string("diffusivity: ") + cudaGetErrorString(e);
        return SE_ERR_CUDA;
    }
    if (status != SE_OK) c->err = "a rigid-particle solve did not reach rtol within maxit products";
    return status;
}

// High-frequency shear viscosity of the far-field suspension (the eta_s of Eq. dst-corr):
// force- and torque-free rigid spheres in the imposed strain E_inf = e_k (each of the five
// orthonormal basis tensors in turn); the particle stress is n <S>, so along e_k
// eta_s / eta - 1 = (sum_i S_i . e_k) / (2 eta V), averaged over k (an isotropic
// suspension gives five equal values).  The isolated sphere's S = (20/3) pi eta a^3 E_inf
// gives Einstein's 1 + 5 phi / 2.
extern "C" int se_high_frequency_viscosity(se_ctx *c, double rtol, int maxit, double *eta_ratio, int *products)
{
    if (!c || !eta_ratio) return SE_ERR_ARG;
    if (!(rtol > 0) || maxit < 1) { c->err = "rtol must be > 0 and maxit >= 1"; return SE_ERR_ARG; }
    if (!c->have_config) { c->err = "se_set_config must be called first"; return SE_ERR_STATE; }
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    const int N = (int)c->N;
    const size_t n = (size_t)N * 11;
    double *x11 = nullptr;
    if (cudaMalloc(&x11, 2 * n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->err = "viscosity allocation failed";
        return SE_ERR_NOMEM;
    }
    double *w11 = x11 + n;
    std::vector<double> h(n);
    int total = 0, status = SE_OK;
    double acc = 0;
    for (int k = 0; k < 5; ++k) {
        double e[5] = {0, 0, 0, 0, 0};
        e[k] = 1.0;
        int it = 0;
        const int rc = rigid_core(c, nullptr, e, x11, w11, rtol, maxit, &it, nullptr);
        total += it + 1;
        if (rc == SE_ERR_NOT_CONVERGED) status = rc;
        else if (rc != SE_OK) {
            cudaFree(x11);
            return rc;
        }
        if (cudaMemcpyAsync(h.data(), w11, n * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaFree(x11);
            c->err = "viscosity: copy of the stresslets failed";
            return SE_ERR_CUDA;
        }
        double sk = 0;
        for (int i = 0; i < N; ++i) sk += h[(size_t)i * 11 + 6 + k];
        acc += sk / (2.0 * c->eta * c->L * c->L * c->L);
    }
    cudaFree(x11);
    *eta_ratio = 1.0 + acc / 5.0;
    if (products) *products = total;
    if (status != SE_OK) c->err = "a rigid-particle solve did not reach rtol within maxit products";
    return status;
}
