// C ABI entry points (include/se_mobility.h): context lifecycle, parameters,
// configuration, and the grand-mobility product y = M_inf . x.
//
// Product schedule (one call, all on the device, no host round trip):
//   permute x into cell order -> real-space pair sum -> spread -> FFT x -> FFT y
//   -> FFT z + k-space scaling + inverse z -> inverse y -> inverse x
//   -> gather + real + self, written in caller order.
// SE_OPT_OVERLAP can move the real-space sum onto a second, high-priority stream
// beside the spread or the FFT chain (forked and joined with events).
#include <cmath>
#include <cstdio>
#include <cstring>

#include "se_internal.cuh"

using namespace se;

static std::string g_create_error;

namespace se {

namespace {

template <typename T, typename TI>
__global__ void permute_in_kernel(int N, int ncomp, const int *perm, const TI *x, T *xs)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const TI *src = x + (size_t)perm[k] * ncomp;
    T *dst = xs + (size_t)k * kNC;
#pragma unroll
    for (int c = 0; c < kNC; ++c) dst[c] = c < ncomp ? (T)src[c] : (T)0;
}

}  // namespace

template <typename T, typename TI>
void launch_permute_in(se_ctx *c, const TI *x, T *xs, int ncomp, cudaStream_t s)
{
    const int N = (int)c->N;
    permute_in_kernel<T, TI><<<(N + 255) / 256, 256, 0, s>>>(N, ncomp, c->b.perm, x, xs);
    c->launches++;
}

template void launch_permute_in<float, float>(se_ctx *, const float *, float *, int, cudaStream_t);
template void launch_permute_in<float, double>(se_ctx *, const double *, float *, int, cudaStream_t);
template void launch_permute_in<double, float>(se_ctx *, const float *, double *, int, cudaStream_t);
template void launch_permute_in<double, double>(se_ctx *, const double *, double *, int, cudaStream_t);

void stage_mark(se_ctx *c, int stage, cudaStream_t s, bool end)
{
    if (!c->timing) return;
    const size_t need = (size_t)(c->tprod + 1) * 2 * SE_NSTAGE;
    while (c->tev.size() < need) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->tev.push_back(e);
    }
    cudaEventRecord(c->tev[(size_t)c->tprod * 2 * SE_NSTAGE + 2 * stage + (end ? 1 : 0)], s);
}

}  // namespace se

// ---------------------------------------------------------------- helpers

static bool grid_size_ok(int M)
{
    if (M < 8 || M > 512 || M % kTile != 0) return false;
    int m = M;
    while (m % 2 == 0) m /= 2;
    while (m % 3 == 0) m /= 3;
    return m == 1;
}

static void make_plan(int M, FftPlan &plan)
{
    plan.M = M;
    plan.nst = 0;
    int m = M;
    // radix 8 and 9 first, then at most two of 6, 4, 3, 2 (M = 2^a 3^b, 8 | M):
    // every admissible M up to 512 takes at most three passes
    while (m % 8 == 0) { plan.rad[plan.nst++] = 8; m /= 8; }
    while (m % 9 == 0) { plan.rad[plan.nst++] = 9; m /= 9; }
    if (m == 6) { plan.rad[plan.nst++] = 6; m = 1; }
    if (m % 4 == 0) { plan.rad[plan.nst++] = 4; m /= 4; }
    if (m % 2 == 0) { plan.rad[plan.nst++] = 2; m /= 2; }
    if (m % 3 == 0) { plan.rad[plan.nst++] = 3; m /= 3; }
}

static void dfree(void *&p)
{
    if (p) cudaFree(p);
    p = nullptr;
}
template <typename P>
static void dfree_t(P *&p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

static void free_grids(se_ctx *c)
{
    for (int q = 0; q < 3; ++q) {
        dfree(c->b.grid_f[q]);
        dfree(c->b.grid_part[q]);
        dfree(c->b.spec_f[q]);
        dfree(c->b.spec_o[q]);
        dfree(c->b.grid_o[q]);
        dfree(c->b.tw[q]);
        c->grid_M[q] = 0;
    }
    for (int q = 0; q < 2; ++q) {
        dfree(c->b.ws_grid[q]);
        dfree(c->b.ws_spec_a[q]);
        dfree(c->b.ws_spec_b[q]);
        c->b.ws_M[q] = 0;
    }
}

// keep_pairs: the pair table's buffers stay allocated for the next configuration (set_config
// overwrites them in place), only the table's validity is dropped
static void free_config(se_ctx *c, bool keep_pairs = false)
{
    free_spectral(c);
    c->lp_ready = false;
    c->sp_theta_cap = 1.0;
    dfree_t(c->b.pos);
    dfree_t(c->b.rad);
    dfree_t(c->b.perm);
    dfree_t(c->b.cell_start);
    dfree_t(c->b.tile_perm);
    dfree_t(c->b.tile_start);
    dfree_t(c->b.sup_base);
    for (int q = 0; q < 3; ++q) {
        dfree(c->b.sup_s0[q]);
        dfree(c->b.sup_w[q]);
        dfree(c->b.self_c[q]);
        dfree(c->b.xs[q]);
        dfree(c->b.yreal[q]);
        dfree(c->b.rel[q]);
        c->support_ok[q] = false;
    }
    c->lists_ok = false;
    if (!keep_pairs) {
        dfree_t(c->b.pair_off);
        dfree_t(c->b.pair_j);
        c->pair_off_n = 0;
        c->pairj_cap = 0;
    }
    for (int q = 0; q < 3; ++q) {
        if (!keep_pairs || q == 2) {
            dfree(c->b.pair_x[q]);
            dfree(c->b.pair_c[q]);
            c->pair_cap[q] = 0;
        }
        c->pairs_ok[q] = false;
    }
    c->npairs = 0;
    dfree_t(c->b.pc_inv);
    dfree_t(c->b.pc_C);
    dfree_t(c->b.kry);
    dfree_t(c->b.work64);
    c->b.kry_n = 0;
    c->b.kry_m = 0;
    dfree_t(c->b.red);
    dfree_t(c->b.stage);
    c->alloc_N = 0;
    c->tiles_ok = false;
    c->pc_ready = false;
}

#define SE_ALLOC(ctx, ptr, bytes)                                                     \
    do {                                                                              \
        if (cudaMalloc((void **)&(ptr), (bytes)) != cudaSuccess) {                    \
            cudaGetLastError();                                                       \
            (ctx)->err = "device allocation of " + std::to_string((size_t)(bytes)) + " bytes failed"; \
            return SE_ERR_NOMEM;                                                      \
        }                                                                             \
    } while (0)

template <typename TI, typename TO>
__global__ void cvt_kernel(size_t n, const TI *in, TO *out)
{
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        out[e] = (TO)in[e];
}
template <typename TI, typename TO>
static void launch_cvt(se_ctx *c, size_t n, const void *in, void *out, cudaStream_t s)
{
    const size_t g = std::min<size_t>((n + 255) / 256, 8192);
    cvt_kernel<TI, TO><<<(unsigned)std::max<size_t>(g, 1), 256, 0, s>>>(n, (const TI *)in, (TO *)out);
    c->launches++;
}

static int ensure_grids(se_ctx *c, int prec);

// the double-float (precision 2) grids: spread and gathered grids in double-float, the
// spectra, twiddles and the FFT's own grids those of FP64
static int ensure_grids_ff(se_ctx *c)
{
    int rc = ensure_grids(c, 1);
    if (rc != SE_OK) return rc;
    if (c->grid_M[2] == (size_t)c->M && c->b.grid_f[2]) return SE_OK;
    dfree(c->b.grid_f[2]);
    dfree(c->b.grid_part[2]);
    dfree(c->b.grid_o[2]);
    const size_t M = c->M;
    SE_ALLOC(c, c->b.grid_f[2], M * M * M * 8 * sizeof(ff));
    {
        const size_t ntiles = (M / kTile) * (M / kTile) * (M / kTile);
        c->nsplit[2] = (int)std::min<size_t>(16, std::max<size_t>(1, (2 * (size_t)c->sms * 11 + ntiles - 1) / ntiles));
        if (c->nsplit[2] > 1) SE_ALLOC(c, c->b.grid_part[2], (size_t)c->nsplit[2] * M * M * M * 8 * sizeof(ff));
    }
    SE_ALLOC(c, c->b.grid_o[2], M * M * M * 8 * sizeof(ff));
    c->grid_M[2] = c->M;
    return SE_OK;
}

// grids for (M, precision prec)
static int ensure_grids(se_ctx *c, int prec)
{
    if (prec == 2) return ensure_grids_ff(c);
    const size_t es = prec == 1 ? sizeof(double) : sizeof(float);
    if (c->grid_M[prec] == (size_t)c->M && c->b.grid_f[prec]) return SE_OK;
    dfree(c->b.grid_f[prec]);
    dfree(c->b.grid_part[prec]);
    dfree(c->b.spec_f[prec]);
    dfree(c->b.spec_o[prec]);
    dfree(c->b.grid_o[prec]);
    dfree(c->b.tw[prec]);
    const size_t M = c->M, Mh = M / 2 + 1;
    // 8 components: the wave-space approach spreads 7 grids (4 otherwise)
    SE_ALLOC(c, c->b.grid_f[prec], M * M * M * 8 * es);
    // With few spreading tiles (small M) several CTAs share a tile, each summing part
    // of its particles into its own partial grid: about two waves of CTAs on the SMs.
    {
        const size_t ntiles = (M / kTile) * (M / kTile) * (M / kTile);
        int ns = (int)std::min<size_t>(16, std::max<size_t>(1, (2 * (size_t)c->sms * 11 + ntiles - 1) / ntiles));
        // the FP32 16-plane tiles may split too, to fill the last wave of CTAs
        const int nt = (int)(M / kTile);
        if (prec == 0) ns = std::max(ns, spread16_split(c->sms, nt * nt * ((nt + 1) / 2), 4));
        c->nsplit[prec] = ns;
        if (ns > 1) SE_ALLOC(c, c->b.grid_part[prec], (size_t)ns * M * M * M * 8 * es);
    }
    SE_ALLOC(c, c->b.spec_f[prec], M * M * Mh * 8 * 2 * es);
    SE_ALLOC(c, c->b.spec_o[prec], M * M * Mh * 8 * 2 * es);
    SE_ALLOC(c, c->b.grid_o[prec], M * M * M * 8 * es);
    SE_ALLOC(c, c->b.tw[prec], M * 2 * es);
    c->grid_M[prec] = c->M;
    make_twiddles(c, prec);
    return SE_OK;
}

static int ensure_support(se_ctx *c, int prec);

// the wave-space approach's 20-component grids and spectra (SE_OPT_SIZE_MODE 3)
static int ensure_ws_grids(se_ctx *c, int prec)
{
    if (c->b.ws_M[prec] == (size_t)c->M && c->b.ws_grid[prec]) return SE_OK;
    dfree(c->b.ws_grid[prec]);
    dfree(c->b.ws_spec_a[prec]);
    dfree(c->b.ws_spec_b[prec]);
    const size_t es = prec == 1 ? sizeof(double) : sizeof(float);
    const size_t M = c->M, Mh = M / 2 + 1;
    SE_ALLOC(c, c->b.ws_grid[prec], M * M * M * 20 * es);
    SE_ALLOC(c, c->b.ws_spec_a[prec], M * M * Mh * 20 * 2 * es);
    SE_ALLOC(c, c->b.ws_spec_b[prec], M * M * Mh * 20 * 2 * es);
    c->b.ws_M[prec] = c->M;
    return SE_OK;
}

// double-float support: the FP64 tables and the FP64 pair table of the real-space sum
// converted once per configuration
static int ensure_support_ff(se_ctx *c)
{
    int rc = ensure_support(c, 1);
    if (rc != SE_OK) return rc;
    const size_t N = c->N;
    if (!c->b.xs[2]) SE_ALLOC(c, c->b.xs[2], N * kNC * sizeof(ff));
    if (!c->b.yreal[2]) SE_ALLOC(c, c->b.yreal[2], N * kNC * sizeof(ff));
    if (!c->support_ok[2]) {
        dfree(c->b.sup_w[2]);
        if (!c->b.sup_s0[2]) SE_ALLOC(c, c->b.sup_s0[2], N * 3 * sizeof(ff));
        if (!c->b.self_c[2]) SE_ALLOC(c, c->b.self_c[2], N * 4 * sizeof(ff));
        SE_ALLOC(c, c->b.sup_w[2], N * 3 * c->P * sizeof(ff));
        cudaStream_t s = c->stream;
        launch_cvt<double, ff>(c, N * 3, c->b.sup_s0[1], c->b.sup_s0[2], s);
        launch_cvt<double, ff>(c, N * 3 * c->P, c->b.sup_w[1], c->b.sup_w[2], s);
        launch_cvt<double, ff>(c, N * 4, c->b.self_c[1], c->b.self_c[2], s);
        SE_CUDA_CHECK(c, cudaStreamSynchronize(s));
        c->support_ok[2] = true;
    }
    return build_pair_table_ff(c);
}

// support tables and work vectors at precision prec
static int ensure_support(se_ctx *c, int prec)
{
    if (prec == 2) return ensure_support_ff(c);
    if (c->alloc_N == 0 || !c->b.pos) {
        c->err = "se_set_config must be called first";
        return SE_ERR_STATE;
    }
    const size_t es = prec == 1 ? sizeof(double) : sizeof(float);
    const size_t N = c->N;
    if (!c->b.sup_s0[prec]) SE_ALLOC(c, c->b.sup_s0[prec], N * 3 * es);
    if (!c->b.xs[prec]) SE_ALLOC(c, c->b.xs[prec], N * kNC * es);
    if (!c->b.yreal[prec]) SE_ALLOC(c, c->b.yreal[prec], N * kNC * es);
    if (!c->b.rel[prec]) {
        SE_ALLOC(c, c->b.rel[prec], N * 4 * es);
        if (prec == 1) setup_rel<double>(c, c->stream);
        else setup_rel<float>(c, c->stream);
    }
    if (!c->pairs_ok[prec]) {
        // the stored pair table is an optimisation: without memory for it the
        // real-space kernel recomputes the pairs from the cell list
        const int r = prec == 1 ? build_pair_table<double>(c) : build_pair_table<float>(c);
        if (r == SE_ERR_OVERLAP) return r;
        if (r != SE_OK && c->shear != 0) return r;      // the cell-list fallback is for the cube only
        if (r != SE_OK) {
            cudaGetLastError();
            dfree(c->b.pair_x[prec]);
            dfree(c->b.pair_c[prec]);
            c->pair_cap[prec] = 0;
            c->err.clear();
        }
    }
    if (!c->support_ok[prec]) {
        dfree(c->b.sup_w[prec]);
        SE_ALLOC(c, c->b.sup_w[prec], N * 3 * c->P * es);
        if (!c->b.self_c[prec]) SE_ALLOC(c, c->b.self_c[prec], N * 4 * es);
        return build_support(c, prec);
    }
    return SE_OK;
}

static int set_error(se_ctx *c, int code, const std::string &msg)
{
    c->err = msg;
    return code;
}

// ---------------------------------------------------------------- ABI

extern "C" int se_create(se_ctx **out, int device, void *stream)
{
    if (!out) return SE_ERR_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) {
        g_create_error = "cudaSetDevice failed";
        return SE_ERR_CUDA;
    }
    se_ctx *c = new se_ctx();
    c->device = device;
    c->stream = (cudaStream_t)stream;
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || c->sms < 1) {
        g_create_error = "cudaDeviceGetAttribute(MultiProcessorCount) failed";
        delete c;
        return SE_ERR_CUDA;
    }
    int prio_least = 0, prio_greatest = 0;
    cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
    if (cudaStreamCreateWithPriority(&c->aux, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        g_create_error = "stream/event creation failed";
        delete c;
        return SE_ERR_CUDA;
    }
    *out = c;
    return SE_OK;
}

extern "C" int se_destroy(se_ctx *c)
{
    if (!c) return SE_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    cudaStreamSynchronize(c->aux);
    free_grids(c);
    free_config(c);
    dfree_t(c->b.mlp_w);
    for (int q = 0; q < 2; ++q) dfree(c->ktab[q]);
    cudaEventDestroy(c->ev_fork);
    cudaEventDestroy(c->ev_join);
    for (cudaEvent_t e : c->tev) cudaEventDestroy(e);
    cudaStreamDestroy(c->aux);
    delete c;
    return SE_OK;
}

extern "C" const char *se_last_error(const se_ctx *c)
{
    return c ? c->err.c_str() : g_create_error.c_str();
}

extern "C" int64_t se_kernel_launches(const se_ctx *c) { return c ? c->launches : 0; }

extern "C" int se_stage_times(se_ctx *c, double *ms, int nstage)
{
    if (!c || !ms || nstage < 1 || nstage > SE_NSTAGE) return SE_ERR_ARG;
    for (int st = 0; st < nstage; ++st) ms[st] = 0.0;
    const int n = c->tprod;
    for (int q = 0; q < n; ++q)
        for (int st = 0; st < nstage; ++st) {
            cudaEvent_t b = c->tev[(size_t)q * 2 * SE_NSTAGE + 2 * st], e = c->tev[(size_t)q * 2 * SE_NSTAGE + 2 * st + 1];
            SE_CUDA_CHECK(c, cudaEventSynchronize(e));
            float t = 0.f;
            SE_CUDA_CHECK(c, cudaEventElapsedTime(&t, b, e));
            ms[st] += t;
        }
    c->tprod = 0;
    return n;
}

extern "C" int se_set_params(se_ctx *c, double xi, int M, int P, double rc)
{
    if (!c) return SE_ERR_ARG;
    if (!(xi > 0) || !std::isfinite(xi)) return set_error(c, SE_ERR_ARG, "xi must be positive");
    if (!grid_size_ok(M)) return set_error(c, SE_ERR_GRID, "M must be 2^a 3^b, a multiple of 8, in [8, 512]");
    if (P < 2 || P > 32 || P > M - kTile) return set_error(c, SE_ERR_GRID, "P must satisfy 2 <= P <= min(32, M - 8)");
    if (!(rc > 0) || !std::isfinite(rc)) return set_error(c, SE_ERR_CUTOFF, "rc must be positive");
    cudaSetDevice(c->device);
    c->xi = xi;
    c->M = M;
    c->P = P;
    c->rc = rc;
    make_plan(M, c->plan);
    c->have_params = true;
    c->have_config = false;            // configuration-dependent setup must be rebuilt
    c->pc_ready = false;
    c->err.clear();
    return SE_OK;
}

extern "C" int se_set_option(se_ctx *c, int key, double value)
{
    if (!c) return SE_ERR_ARG;
    switch (key) {
    case SE_OPT_PRECISION:
        if (value != 0 && value != 1 && value != 2)
            return set_error(c, SE_ERR_ARG, "precision must be 0 (FP32), 1 (FP64) or 2 (FP64-equivalent double-float)");
        c->precision = (int)value;
        return SE_OK;
    case SE_OPT_SIZE_MODE:
        if (value != 0 && value != 1 && value != 2 && value != 3)
            return set_error(c, SE_ERR_ARG, "size mode must be 0 (hybrid), 1 (real-space), 2 (wave-space, "
                                            "gradients in the spread) or 3 (wave-space, all derivatives in k-space)");
        if (c->shear != 0 && value != 2 && value != 3 && !c->point_forces)
            return set_error(c, SE_ERR_ARG, "a sheared cell needs a wave-space size approach (SE_OPT_SIZE_MODE 2 or 3)");
        c->size_mode = (int)value;
        c->pc_ready = false;
        return SE_OK;
    case SE_OPT_ETA:
        if (!(value > 0)) return set_error(c, SE_ERR_ARG, "eta must be positive");
        if (value != c->eta) {
            // the stored pair coefficients and the self coefficients carry 1/eta
            c->eta = value;
            for (int q = 0; q < 3; ++q) {
                dfree(c->b.pair_x[q]);
                dfree(c->b.pair_c[q]);
                c->pair_cap[q] = 0;
                c->pairs_ok[q] = false;
                c->support_ok[q] = false;
            }
        }
        c->pc_ready = false;
        return SE_OK;
    case SE_OPT_SHAPE_M:
        if (!(value > 0)) return set_error(c, SE_ERR_ARG, "m must be positive");
        c->m_shape = value;
        c->m_user = true;
        c->support_ok[0] = c->support_ok[1] = c->support_ok[2] = false;
        c->pc_ready = false;
        return SE_OK;
    case SE_OPT_RESTART:
        if (value < 1 || value > 1000) return set_error(c, SE_ERR_ARG, "restart must be in [1, 1000]");
        c->restart = (int)value;
        return SE_OK;
    case SE_OPT_PARTS:
        if (value < 0 || value > 7) return set_error(c, SE_ERR_ARG, "parts must be a mask in [0, 7]");
        c->parts = (int)value;
        return SE_OK;
    case SE_OPT_OVERLAP:
        if (value != 0 && value != 1 && value != 2 && value != 3)
            return set_error(c, SE_ERR_ARG, "overlap must be 0, 1, 2 or 3");
        c->overlap = (int)value;
        return SE_OK;
    case SE_OPT_PC_THETA:
        if (!(value >= 0 && value <= 1)) return set_error(c, SE_ERR_ARG, "theta must be in [0, 1]");
        if (value != c->sp_theta) free_spectral(c);
        c->sp_theta = value;
        c->sp_theta_cap = 1.0;
        return SE_OK;
    case SE_OPT_PC_CMAX:
        if (!(value >= 0.5 && value <= 0.99)) return set_error(c, SE_ERR_ARG, "c_max must be in [0.5, 0.99]");
        if (value != c->sp_cmax) free_spectral(c);
        c->sp_cmax = value;
        return SE_OK;
    case SE_OPT_PC_KA:
        if (!(value > 0 && value <= 3)) return set_error(c, SE_ERR_ARG, "k_c a must be in (0, 3]");
        if (value != c->sp_ka) free_spectral(c);
        c->sp_ka = value;
        return SE_OK;
    case SE_OPT_GATHER:
        if (value != 0 && value != 1 && value != 2) return set_error(c, SE_ERR_ARG, "gather must be 0, 1 or 2");
        c->gather = (int)value;
        return SE_OK;
    case SE_OPT_SPREAD:
        if (value != 0 && value != 1 && value != 2) return set_error(c, SE_ERR_ARG, "spread must be 0, 1 or 2");
        c->spread = (int)value;
        return SE_OK;
    case SE_OPT_FF_TABLE:
        if (value != 0 && value != 1) return set_error(c, SE_ERR_ARG, "ff table must be 0 or 1");
        c->ff_table = (int)value;
        if (!c->ff_table && c->pairs_ok[2]) {
            dfree(c->b.pair_x[2]);
            dfree(c->b.pair_c[2]);
            c->pairs_ok[2] = false;
        }
        return SE_OK;
    case SE_OPT_RESIDUAL:
        if (value != 1 && value != 2) return set_error(c, SE_ERR_ARG, "residual precision must be 1 or 2");
        c->res_precision = (int)value;
        return SE_OK;
    case SE_OPT_SHEAR:
        if (!(std::fabs(value) <= 0.5)) return set_error(c, SE_ERR_ARG, "shear strain must be in [-0.5, 0.5]");
        if (value != 0 && c->size_mode != 2 && c->size_mode != 3 && !c->point_forces)
            return set_error(c, SE_ERR_ARG, "a sheared cell needs a wave-space size approach (SE_OPT_SIZE_MODE 2 or 3)");
        if (value != c->shear) {
            c->shear = value;
            c->have_config = false;        // the configuration must be set again
            c->pc_ready = false;
        }
        return SE_OK;
    case SE_OPT_PAIR_FILL:
        if (value != 0 && value != 1) return set_error(c, SE_ERR_ARG, "pair fill must be 0 or 1");
        if ((int)value != c->pair_fill_fp64) {
            c->pair_fill_fp64 = (int)value;
            c->pairs_ok[0] = false;         // the FP32 table is evaluated again when next needed
        }
        return SE_OK;
    case SE_OPT_OVERLAP_CHECK:
        if (value != 0 && value != 1) return set_error(c, SE_ERR_ARG, "overlap check must be 0 or 1");
        c->overlap_check = (int)value;
        return SE_OK;
    case SE_OPT_TIMING:
        if (value != 0 && value != 1) return set_error(c, SE_ERR_ARG, "timing must be 0 or 1");
        c->timing = value != 0;
        c->tprod = 0;
        return SE_OK;
    default:
        return set_error(c, SE_ERR_ARG, "unknown option");
    }
}

extern "C" int se_set_config(se_ctx *c, int64_t N, double L, const double *pos, const double *radius)
{
    if (!c || !pos || !radius || N <= 0 || N > (1 << 28)) return c ? set_error(c, SE_ERR_ARG, "bad N or null pointer") : SE_ERR_ARG;
    if (!c->have_params) return set_error(c, SE_ERR_STATE, "se_set_params must be called first");
    if (!(L > 0) || !std::isfinite(L)) return set_error(c, SE_ERR_ARG, "L must be positive");
    if (c->rc >= 0.5 * L) return set_error(c, SE_ERR_CUTOFF, "rc must be smaller than L/2");
    if (c->shear != 0 && c->size_mode != 2 && c->size_mode != 3 && !c->point_forces)
        return set_error(c, SE_ERR_ARG, "a sheared cell needs a wave-space size approach (SE_OPT_SIZE_MODE 2 or 3)");
    cudaSetDevice(c->device);
    // the pair table is overwritten in place: work of this context in flight on any stream
    // (its own two, a batch's stream pool or graph) must finish first, as a cudaFree would wait
    SE_CUDA_CHECK(c, cudaDeviceSynchronize());
    free_config(c, true);
    c->N = N;
    c->L = L;
    // cells uniform in the fractional coordinates: the rc ball reaches (1 + |gamma|) rc along t_x
    int nc = (int)std::floor(L / ((1 + std::fabs(c->shear)) * c->rc));
    if (nc < 3) nc = 1;
    if (nc > 256) nc = 256;
    c->nc = nc;
    const size_t nt = c->M / kTile;
    SE_ALLOC(c, c->b.pos, N * 3 * sizeof(double));
    SE_ALLOC(c, c->b.rad, N * sizeof(double));
    SE_ALLOC(c, c->b.perm, N * sizeof(int));
    SE_ALLOC(c, c->b.cell_start, ((size_t)nc * nc * nc + 1) * sizeof(int));
    SE_ALLOC(c, c->b.tile_perm, N * sizeof(int));
    SE_ALLOC(c, c->b.tile_start, (nt * nt * nt + 1) * sizeof(int));
    SE_ALLOC(c, c->b.sup_base, N * 3 * sizeof(int));
    c->alloc_N = N;
    int rc = build_cells(c, pos, radius);
    if (rc == SE_OK) rc = ensure_support(c, c->precision);
    if (rc != SE_OK) {
        c->have_config = false;
        free_config(c);
        return rc;
    }
    c->have_config = true;
    c->pc_ready = false;
    c->err.clear();
    return SE_OK;
}

template <typename T, typename TO>
static int apply_t(se_ctx *c, int ncomp, const TO *x, TO *y)
{
    cudaStream_t s = c->stream;
    T *xs = (T *)c->b.xs[pix<T>()], *yr = (T *)c->b.yreal[pix<T>()];
    stage_mark(c, SE_STAGE_PERMUTE, s, false);
    launch_permute_in<T, TO>(c, x, xs, ncomp, s);
    stage_mark(c, SE_STAGE_PERMUTE, s, true);
    const int with_wave = (c->parts & 2) ? 1 : 0;
    // the real-space sum runs inside the gather kernel where fused_real_gather applies
    // (overlap 3, the default), else in line before the spread (2, and 3 where the fused
    // kernel does not apply), or on the auxiliary high-priority stream beside the spread (0)
    // or the FFT chain (1)
    auto real_part = [&](cudaStream_t rs) -> int {
        stage_mark(c, SE_STAGE_REAL, rs, false);
        if (c->parts & 1) launch_real<T>(c, xs, yr, rs, ncomp);
        else SE_CUDA_CHECK(c, cudaMemsetAsync(yr, 0, c->N * kNC * sizeof(T), rs));
        stage_mark(c, SE_STAGE_REAL, rs, true);
        return SE_OK;
    };
    auto fork_real = [&]() -> int {
        SE_CUDA_CHECK(c, cudaEventRecord(c->ev_fork, s));
        SE_CUDA_CHECK(c, cudaStreamWaitEvent(c->aux, c->ev_fork, 0));
        const int r = real_part(c->aux);
        if (r != SE_OK) return r;
        SE_CUDA_CHECK(c, cudaEventRecord(c->ev_join, c->aux));
        return SE_OK;
    };
    int rc;
    if (c->size_mode == 3) {
        // the wave-space approach: its own 20-component chain after the real-space sum
        if ((rc = real_part(s)) != SE_OK) return rc;
        launch_wave_ws<T, TO>(c, xs, yr, y, ncomp, with_wave, s);
        if (c->timing) c->tprod++;
        SE_CUDA_CHECK(c, cudaGetLastError());
        return SE_OK;
    }
    const bool fused = std::is_same<T, float>::value && fused_real_gather(c, ncomp, with_wave);
    if (fused) {
        stage_mark(c, SE_STAGE_REAL, s, false);
        stage_mark(c, SE_STAGE_REAL, s, true);
    } else if (c->overlap >= 2 && (rc = real_part(s)) != SE_OK) return rc;
    if (c->overlap == 0 && (rc = fork_real()) != SE_OK) return rc;
    if (with_wave) launch_wave_spread<T>(c, xs, s, ncomp);
    else {
        stage_mark(c, SE_STAGE_SPREAD, s, false);
        stage_mark(c, SE_STAGE_SPREAD, s, true);
    }
    if (c->overlap == 1 && (rc = fork_real()) != SE_OK) return rc;
    if (with_wave) launch_wave_fft<T>(c, s);
    else
        for (int st = SE_STAGE_FFT_XF; st <= SE_STAGE_FFT_XI; ++st) {
            stage_mark(c, st, s, false);
            stage_mark(c, st, s, true);
        }
    if (c->overlap <= 1) SE_CUDA_CHECK(c, cudaStreamWaitEvent(s, c->ev_join, 0));
    stage_mark(c, SE_STAGE_GATHER, s, false);
    launch_gather_combine<T, TO>(c, xs, yr, y, ncomp, with_wave, s);
    stage_mark(c, SE_STAGE_GATHER, s, true);
    if (c->timing) c->tprod++;
    SE_CUDA_CHECK(c, cudaGetLastError());
    return SE_OK;
}

// FP64-equivalent product (precision 2): the FFT and the k-space scaling in FP64, the
// real-space sum (from the FP64 pair table), the spread and the gather (the stages bound
// by B300's FP64 pipe) in double-float
template <typename TO>
static int apply_ff(se_ctx *c, int ncomp, const TO *x, TO *y)
{
    cudaStream_t s = c->stream;
    const size_t N = c->N;
    double *xs1 = (double *)c->b.xs[1], *yr1 = (double *)c->b.yreal[1];
    ff *xs2 = (ff *)c->b.xs[2], *yr2 = (ff *)c->b.yreal[2];
    const int with_wave = (c->parts & 2) ? 1 : 0;
    stage_mark(c, SE_STAGE_PERMUTE, s, false);
    launch_permute_in<double, TO>(c, x, xs1, ncomp, s);
    launch_cvt<double, ff>(c, N * kNC, xs1, xs2, s);
    stage_mark(c, SE_STAGE_PERMUTE, s, true);
    stage_mark(c, SE_STAGE_REAL, s, false);
    if (!(c->parts & 1) || !launch_real_ff(c, xs2, yr2, s, ncomp)) {
        if (c->parts & 1) launch_real<double>(c, xs1, yr1, s, ncomp);
        else SE_CUDA_CHECK(c, cudaMemsetAsync(yr1, 0, N * kNC * sizeof(double), s));
        launch_cvt<double, ff>(c, N * kNC, yr1, yr2, s);
    }
    stage_mark(c, SE_STAGE_REAL, s, true);
    const size_t M3 = (size_t)c->M * c->M * c->M;
    if (with_wave) {
        launch_wave_spread<ff>(c, xs2, s, ncomp);
        launch_cvt<ff, double>(c, M3 * (c->size_mode == 2 ? 8 : 4), c->b.grid_f[2], c->b.grid_f[1], s);
        launch_wave_fft<double>(c, s);
        launch_cvt<double, ff>(c, M3 * (c->size_mode != 1 ? 8 : 4), c->b.grid_o[1], c->b.grid_o[2], s);
    } else {
        for (int st = SE_STAGE_SPREAD; st <= SE_STAGE_FFT_XI; ++st) {
            stage_mark(c, st, s, false);
            stage_mark(c, st, s, true);
        }
    }
    stage_mark(c, SE_STAGE_GATHER, s, false);
    launch_gather_combine<ff, TO>(c, xs2, yr2, y, ncomp, with_wave, s);
    stage_mark(c, SE_STAGE_GATHER, s, true);
    if (c->timing) c->tprod++;
    SE_CUDA_CHECK(c, cudaGetLastError());
    return SE_OK;
}

int se::se_apply_internal(se_ctx *c, int ncomp, const void *x, void *y, int dtype, int prec)
{
    if (!c->have_config) return set_error(c, SE_ERR_STATE, "se_set_config must be called first");
    if (c->size_mode == 3 && prec == 2) prec = 1;     // the wave-space approach runs in FP32 or FP64
    int rc = ensure_support(c, prec);
    if (rc != SE_OK) return rc;
    rc = ensure_grids(c, prec);
    if (rc != SE_OK) return rc;
    if (c->size_mode == 3 && (rc = ensure_ws_grids(c, prec)) != SE_OK) return rc;
    if (prec == 2) {
        return dtype == SE_F64 ? apply_ff<double>(c, ncomp, (const double *)x, (double *)y)
                               : apply_ff<float>(c, ncomp, (const float *)x, (float *)y);
    }
    if (prec == 1) {
        return dtype == SE_F64 ? apply_t<double, double>(c, ncomp, (const double *)x, (double *)y)
                               : apply_t<double, float>(c, ncomp, (const float *)x, (float *)y);
    }
    return dtype == SE_F64 ? apply_t<float, double>(c, ncomp, (const double *)x, (double *)y)
                           : apply_t<float, float>(c, ncomp, (const float *)x, (float *)y);
}

static int check_apply_args(se_ctx *c, int ncomp, const void *x, const void *y, int dtype)
{
    if (!c) return SE_ERR_ARG;
    if (!x || !y) return set_error(c, SE_ERR_ARG, "null x or y");
    if (ncomp != 3 && ncomp != 6 && ncomp != 11 && ncomp != 12) return set_error(c, SE_ERR_ARG, "ncomp must be 3, 6, 11 or 12");
    if (dtype != SE_F32 && dtype != SE_F64) return set_error(c, SE_ERR_ARG, "dtype must be SE_F32 or SE_F64");
    if (!c->have_params) return set_error(c, SE_ERR_STATE, "se_set_params must be called first");
    if (c->alloc_N == 0) return set_error(c, SE_ERR_STATE, "se_set_config must be called first");
    return SE_OK;
}

extern "C" int se_mobility_apply(se_ctx *c, int ncomp, const void *x, void *y, int dtype)
{
    int rc = check_apply_args(c, ncomp, x, y, dtype);
    if (rc != SE_OK) return rc;
    cudaSetDevice(c->device);
    return se_apply_internal(c, ncomp, x, y, dtype, c->precision);
}

extern "C" int se_mobility_apply_host(se_ctx *c, int ncomp, const double *x, double *y)
{
    int rc = check_apply_args(c, ncomp, x, y, SE_F64);
    if (rc != SE_OK) return rc;
    cudaSetDevice(c->device);
    const size_t bytes = (size_t)c->N * ncomp * sizeof(double);
    if (!c->b.stage) SE_ALLOC(c, c->b.stage, (size_t)c->N * kNC * sizeof(double) * 2);
    double *dx = c->b.stage, *dy = c->b.stage + (size_t)c->N * kNC;
    SE_CUDA_CHECK(c, cudaMemcpyAsync(dx, x, bytes, cudaMemcpyHostToDevice, c->stream));
    rc = se_apply_internal(c, ncomp, dx, dy, SE_F64, c->precision);
    if (rc != SE_OK) return rc;
    SE_CUDA_CHECK(c, cudaMemcpyAsync(y, dy, bytes, cudaMemcpyDeviceToHost, c->stream));
    SE_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    return SE_OK;
}
