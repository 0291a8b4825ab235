// Per-configuration setup: positions wrapped into the box, particles ordered by
// real-space cell (counting sort; cells of side >= rc, Sec. 3.3 linked-list /
// chaining-mesh search), Spectral Ewald support of every particle, and the
// particle bins the spreading tiles read.
#include <cmath>
#include <cstdio>

#include "se_internal.cuh"

namespace se {

SeParams make_params(const se_ctx *c)
{
    SeParams p{};
    p.M = c->M;
    p.P = c->P;
    p.Mh = c->M / 2 + 1;
    p.ntile = c->M / kTile;
    p.L = c->L;
    p.xi = c->xi;
    p.rc = c->rc;
    p.eta = c->eta;
    const double m = c->m_user ? c->m_shape : std::sqrt(kPi * c->P);
    p.alpha = 2.0 * m * m / ((double)c->P * c->P);
    p.kappa = c->L > 0 ? c->M / c->L : 0.0;
    p.hybrid = c->size_mode != 1 ? 1 : 0;
    p.wsrc = c->size_mode == 2 ? 1 : 0;
    p.gamma = c->shear;
    return p;
}

namespace {

// Wraps positions into the periodic cell and keys them by real-space cell.  The cell is
// spanned by a1 = (L, 0, 0), a2 = (gamma L, L, 0), a3 = (0, 0, L) (gamma = 0: the cube);
// in the fractional coordinates L t = (x - gamma y, y, z) it is [0, L)^3, and the cells
// and the Spectral Ewald grid are uniform in t.  The stored position is x = L B t.
__global__ void wrap_key_kernel(int N, double L, double gamma, int nc, const double *pos_in, const double *rad_in,
                                double *posw, int *key, int *bad)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int k[3];
    bool ok = isfinite(rad_in[i]) && rad_in[i] > 0;
    double v[3];
    for (int d = 0; d < 3; ++d) {
        v[d] = pos_in[3 * i + d];
        ok = ok && isfinite(v[d]);
    }
    if (!ok) v[0] = v[1] = v[2] = 0.0;
    double t[3] = {v[0] - gamma * v[1], v[1], v[2]};      // L t
    for (int d = 0; d < 3; ++d) {
        t[d] -= L * floor(t[d] / L);
        if (t[d] >= L) t[d] -= L;                  // rounding of the wrap
        int kk = (int)(t[d] / (L / nc));
        k[d] = kk >= nc ? nc - 1 : kk;
    }
    posw[3 * i] = t[0] + gamma * t[1];
    posw[3 * i + 1] = t[1];
    posw[3 * i + 2] = t[2];
    key[i] = (k[2] * nc + k[1]) * nc + k[0];
    if (!ok) atomicOr(bad, 1);
    // bit 2: a radius differs from the first one (the configuration is not monodisperse)
    const unsigned act = __activemask();
    if (__ballot_sync(act, rad_in[i] != rad_in[0]) && (int)(threadIdx.x & 31) == __ffs(act) - 1) atomicOr(bad, 2);
}

__global__ void histogram_kernel(int N, const int *key, int *count)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) atomicAdd(&count[key[i]], 1);
}

// exclusive scan of n counts into start[0..n] by one CTA of 1024 threads
__global__ void scan_kernel(int n, const int *count, int *start)
{
    __shared__ int warp_sums[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < n ? count[i] : 0;
        int x = v;
        for (int off = 1; off < 32; off <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
            for (int off = 1; off < 32; off <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, w, off);
                if (lane >= off) w += y;
            }
            warp_sums[lane] = w;
        }
        __syncthreads();
        const int incl = x + (warp > 0 ? warp_sums[warp - 1] : 0) + carry;
        if (i < n) start[i] = incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[n] = carry;
}

__global__ void scatter_kernel(int N, const int *key, const int *start, int *cursor, int *perm)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int k = key[i];
    perm[start[k] + atomicAdd(&cursor[k], 1)] = i;
}

// order each bin by original index so that the layout is deterministic
__global__ void sort_bins_kernel(int nbins, const int *start, int *perm)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    const int s = start[b], e = start[b + 1];
    for (int i = s + 1; i < e; ++i) {
        const int v = perm[i];
        int j = i - 1;
        while (j >= s && perm[j] > v) {
            perm[j + 1] = perm[j];
            --j;
        }
        perm[j + 1] = v;
    }
}

__global__ void gather_sorted_kernel(int N, const int *perm, const double *posw, const double *rad_in,
                                     double *pos, double *rad)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int i = perm[k];
    pos[3 * k] = posw[3 * i];
    pos[3 * k + 1] = posw[3 * i + 1];
    pos[3 * k + 2] = posw[3 * i + 2];
    rad[k] = rad_in[i];
}

__global__ void tile_key_kernel(int N, int nt, const int *base, int *key)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    key[i] = ((base[3 * i + 2] / kTile) * nt + base[3 * i + 1] / kTile) * nt + base[3 * i] / kTile;
}

}  // namespace

void launch_scan(se_ctx *c, int n, const int *in, int *out, cudaStream_t s)
{
    scan_kernel<<<1, 1024, 0, s>>>(n, in, out);
    c->launches++;
}

// counting sort of keys[0..N) into perm / start[0..nbins]; scratch: count (nbins)
static int counting_sort(se_ctx *c, int N, int nbins, const int *key, int *count, int *start, int *perm,
                         bool sort_bins)
{
    cudaStream_t s = c->stream;
    SE_CUDA_CHECK(c, cudaMemsetAsync(count, 0, sizeof(int) * nbins, s));
    histogram_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, key, count);
    scan_kernel<<<1, 1024, 0, s>>>(nbins, count, start);
    SE_CUDA_CHECK(c, cudaMemsetAsync(count, 0, sizeof(int) * nbins, s));
    scatter_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, key, start, count, perm);
    c->launches += 3;
    if (sort_bins) {
        sort_bins_kernel<<<(nbins + 127) / 128, 128, 0, s>>>(nbins, start, perm);
        c->launches++;
    }
    SE_CUDA_CHECK(c, cudaGetLastError());
    return SE_OK;
}

int build_cells(se_ctx *c, const double *pos_in, const double *rad_in)
{
    const int N = (int)c->N;
    cudaStream_t s = c->stream;
    const int nc = c->nc;
    const int ncell = nc * nc * nc;
    double *posw = nullptr;
    int *key = nullptr, *count = nullptr, *bad = nullptr;
    SE_CUDA_CHECK(c, cudaMalloc(&posw, sizeof(double) * 3 * N));
    SE_CUDA_CHECK(c, cudaMalloc(&key, sizeof(int) * N));
    SE_CUDA_CHECK(c, cudaMalloc(&count, sizeof(int) * (ncell + 1)));
    SE_CUDA_CHECK(c, cudaMalloc(&bad, sizeof(int)));
    SE_CUDA_CHECK(c, cudaMemsetAsync(bad, 0, sizeof(int), s));
    wrap_key_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, c->L, c->shear, nc, pos_in, rad_in, posw, key, bad);
    c->launches++;
    int rc = counting_sort(c, N, ncell, key, count, c->b.cell_start, c->b.perm, true);
    if (rc == SE_OK) {
        gather_sorted_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, c->b.perm, posw, rad_in, c->b.pos, c->b.rad);
        c->launches++;
    }
    int hbad = 0;
    cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(posw);
    cudaFree(key);
    cudaFree(count);
    cudaFree(bad);
    if (rc != SE_OK) return rc;
    if (e != cudaSuccess) {
        c->err = std::string("cell list: ") + cudaGetErrorString(e);
        return SE_ERR_CUDA;
    }
    if (hbad & 1) {
        c->err = "non-finite position or non-positive radius";
        return SE_ERR_NONFINITE;
    }
    c->mono = (hbad & 2) == 0;
    return SE_OK;
}

// Spectral Ewald support at compute precision `prec` and (once) the spreading bins.
int build_support(se_ctx *c, int prec)
{
    const int N = (int)c->N;
    cudaStream_t s = c->stream;
    const int nt = c->M / kTile, ntile = nt * nt * nt;
    if (prec == 1) setup_support<double>(c, s);
    else setup_support<float>(c, s);
    if (!c->tiles_ok) {
        int *key = nullptr, *count = nullptr;
        SE_CUDA_CHECK(c, cudaMalloc(&key, sizeof(int) * N));
        SE_CUDA_CHECK(c, cudaMalloc(&count, sizeof(int) * (ntile + 1)));
        tile_key_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, nt, c->b.sup_base, key);
        c->launches++;
        int rc = counting_sort(c, N, ntile, key, count, c->b.tile_start, c->b.tile_perm, true);
        cudaError_t e = cudaStreamSynchronize(s);
        cudaFree(key);
        cudaFree(count);
        if (rc != SE_OK) return rc;
        if (e != cudaSuccess) {
            c->err = std::string("support setup: ") + cudaGetErrorString(e);
            return SE_ERR_CUDA;
        }
        c->tiles_ok = true;
    }
    SE_CUDA_CHECK(c, cudaStreamSynchronize(s));
    c->support_ok[prec] = true;
    return SE_OK;
}

}  // namespace se
