// Internal declarations of the B300 Spectral Ewald mobility library.
// Not part of the C ABI (include/se_mobility.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include <type_traits>

#include "../../include/se_mobility.h"
#include "se_ff.cuh"

namespace se {

constexpr double kPi = 3.14159265358979323846;
constexpr int kNC = 12;          // components per particle, internal layout
constexpr int kTile = 8;         // spreading tile edge (grid points)

template <typename T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };
// index of the per-precision buffers: FP32, FP64, double-float (SE_OPT_PRECISION 0, 1, 2)
template <typename T> constexpr int pix()
{
    return std::is_same<T, float>::value ? 0 : (std::is_same<T, double>::value ? 1 : 2);
}

// radices of a mixed-radix Stockham FFT of length M = 2^a 3^b
struct FftPlan {
    int M;
    int nst;
    int rad[16];
};

// Spectral Ewald parameters as used on the device (grid units: u = x M / L).
struct SeParams {
    int M, P, Mh;                // grid, support, M/2 + 1
    int ntile;                   // M / kTile
    double L, xi, rc, eta;
    double alpha;                // Gaussian exp(-alpha s^2) in grid units, alpha = 2 m^2 / P^2
    double kappa;                // M / L  (d/dx = kappa d/ds)
    int hybrid;                  // 1: target Faxen terms in wave space (hybrid and wave-space approaches)
    int wsrc;                    // 1: source Faxen terms in wave space too (wave-space approach)
    double gamma;                // strain of the sheared cell a2 = (gamma L, L, 0)
};

// Cell list for the real-space sum (cells of side >= rc).
struct CellGrid {
    int nc;                      // cells per dimension (1 if fewer than 3 fit)
};

struct Buffers {
    // configuration (sorted by cell)
    double *pos = nullptr;       // [N][3] wrapped positions, cell order
    double *rad = nullptr;       // [N]
    int *perm = nullptr;         // sorted index -> caller index
    int *cell_start = nullptr;   // [nc^3 + 1]
    int *tile_perm = nullptr;    // tile order -> sorted index
    int *tile_start = nullptr;   // [ntile^3 + 1]
    int *sup_base = nullptr;     // [N][3] first support point (wrapped)
    // per compute precision (index 0: FP32, 1: FP64)
    void *sup_s0[3] = {};        // [N][3] T: offset of the first support point from the particle
    void *sup_w[3] = {};         // [N][3][P] T: Gaussian weights along each axis
    void *self_c[3] = {};        // [N][4] T: self coefficients of U, Omega, E, E_tr (computed in FP64)
    void *rel[3] = {};           // [N][4] T offset from the cell origin (3) and radius
    void *xs[3] = {};            // [N][12] T inputs in cell order
    void *yreal[3] = {};         // [N][12] T real-space result
    void *grid_f[3] = {};        // [M^3][4] T spread grids
    void *grid_part[3] = {};     // [nsplit][M^3][4] T partial spread grids (small grids only)
    void *spec_f[3] = {};        // [M][M][Mh][4] complex T
    void *spec_o[3] = {};        // [M][M][Mh][8] complex T
    void *grid_o[3] = {};        // [M^3][8] T gathered grids
    void *tw[3] = {};            // [M] complex T twiddles
    // the wave-space approach of SE_OPT_SIZE_MODE 3 (FP32 and FP64 only)
    void *ws_grid[2] = {};       // [5][M^3][4] T spread grids, then the gathered grids
    void *ws_spec_a[2] = {};     // [5][M][M][Mh][4] complex T forward spectra
    void *ws_spec_b[2] = {};     // [5][M][M][Mh][4] complex T output spectra
    size_t ws_M[2] = {0, 0};
    // stored real-space pairs (Sec. 3.3): CSR over targets in cell order
    int *pair_off = nullptr;     // [N + 1]
    int *pair_j = nullptr;       // [npairs]
    void *pair_x[3] = {};        // [3][npairs] T separations (SoA)
    void *pair_c[3] = {};        // [19][npairs] T radial coefficients (SoA)
    // host-API staging (device side)
    double *stage = nullptr;     // [2][N][12]
    // solver
    double *pc_inv = nullptr;    // [N][nc][nc] inverse preconditioner blocks (caller order)
    double *pc_C = nullptr;      // [3][12][12] fitted self-image block coefficients (C0, C1, C2)
    float *mlp_w = nullptr;      // learned correction network (packed parameters)
    double *kry = nullptr;       // Krylov basis [restart + 1][n] and preconditioned vectors [restart][n]
    double *work64 = nullptr;    // FP64 work vectors [6][n]
    size_t kry_n = 0;            // n and restart the Krylov arrays were sized for
    int kry_m = 0;
    double *red = nullptr;       // reduction scratch
};

}  // namespace se

struct se_ctx {
    int device = 0;
    int sms = 1;                       // streaming multiprocessors of the device (grid sizing)
    cudaStream_t stream = nullptr;     // borrowed
    cudaStream_t aux = nullptr;        // owned: real space overlaps the wave chain
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // parameters
    bool have_params = false;
    double xi = 0, rc = 0, m_shape = 0, eta = 1.0;
    bool m_user = false;
    int M = 0, P = 0;
    int precision = 0;                 // 0 FP32, 1 FP64, 2 FP64-equivalent (double-float spread/gather)
    int res_precision = 2;             // true residuals of the solver (SE_OPT_RESIDUAL): 1 FP64, 2 double-float
    int size_mode = 0;                 // 0 hybrid, 1 real-space approach, 2 wave-space approach
    int restart = 30;
    int parts = 7;
    int overlap = 3;             // SE_OPT_OVERLAP
    int gather = 0;              // SE_OPT_GATHER
    int spread = 0;              // SE_OPT_SPREAD
    int overlap_check = 1;       // SE_OPT_OVERLAP_CHECK
    int pair_fill_fp64 = 0;      // SE_OPT_PAIR_FILL
    int ff_table = 1;            // SE_OPT_FF_TABLE
    double shear = 0.0;          // SE_OPT_SHEAR: strain gamma of the periodic cell
    int nsplit[3] = {1, 1, 1};   // partial spread grids allocated per precision (CTAs sharing a tile)
    int split_cap = 16;          // upper bound on the parts a launch uses (1 while boxes run concurrently)
    // configuration
    bool have_config = false;
    bool support_ok[3] = {false, false, false};
    bool tiles_ok = false;
    bool pairs_ok[3] = {false, false, false};
    size_t npairs = 0;
    // the pair table's buffers outlive a configuration: set_config overwrites them in place
    // (same N for the offsets, the neighbour indices and coefficients while they fit)
    bool lists_ok = false;       // neighbour lists of the current configuration built
    int64_t pair_off_n = 0;      // N of the allocated offsets
    size_t pairj_cap = 0;        // allocated neighbour indices
    size_t pair_cap[3] = {};     // pairs the coefficient buffers of precision q hold (0, 1)
    bool mono = false;           // every radius of the configuration equal
    // internal contexts of point forces only (the spectral correction's coarse product: radii
    // negligible, wave part): no window gradient enters, so a sheared cell runs with the
    // real-space size approach
    bool point_forces = false;
    bool pair_mono[3] = {};      // table q stores the 13 coefficients of a monodisperse configuration
    size_t grid_M[3] = {0, 0, 0};
    int64_t N = 0;
    double L = 0;
    int nc = 1;
    // preconditioner state
    bool pc_ready = false;
    int pc_ncomp = 0, pc_prec = -1, pc_kind = -1;
    double pc_alpha = 0, pc_beta = 1;  // the blocks invert alpha I + beta M_ii
    int pc_mixed = 0;                  // ... or the rigid-particle block (se_rigid_solve)
    bool have_mlp = false;
    int pc_fallbacks = 0;              // particles whose learned block fell back to the plain one
    // spectral correction (SE_PRECOND_SPECTRAL): a coarse forces-only context whose
    // k-space kernel is the radial table ktab (transverse modes, |k| <= ktab_kmax)
    se_ctx *spc = nullptr;
    double *sp_f = nullptr, *sp_u = nullptr;   // [N][3] FP64 force part of a vector / correction
    double *sp_s = nullptr;             // [N] sqrt of the block preconditioner's force diagonal
    double sp_theta = 0, sp_ka = 0.9;    // theta 0: 0.98 (monodisperse) or 0.9
    bool ktab_on = false;
    void *ktab[2] = {};                 // [ktab_n] T: h(k) at k = i ktab_kmax / (ktab_n - 1)
    int ktab_n = 0;
    double ktab_kmax = 0;
    double sp_fit[3] = {0, 0, 0};       // fitted lambda_T(k) = A / k^2 + l0, and lambda_B
    double sp_rho = 0;                  // largest eigenvalue of the correction before capping
    double sp_cmax = 0.97;              // cap of the largest eigenvalue of the correction (SE_OPT_PC_CMAX)
    double sp_cmax_used = 0.97;
    double spc_theta = 0, spc_ka = 0, spc_cmax = 0;   // what spc was requested with (0: the options)
    double sp_theta_used = 0;           // the damping spc was built with
    double sp_theta_cap = 1.0;          // at most this damping on this configuration (lowered by stalls)
    int pc_stalls = 0;                  // solves whose spectral correction stalled and fell back to the block
    bool lp_ready = false;              // the learned damping and cutoff for this configuration and weights
    double lp_theta = 0, lp_ka = 0, lp_cmax = 0;
    se::FftPlan plan{};
    se::Buffers b;
    size_t alloc_N = 0;
    int64_t launches = 0;
    std::string err;
    // stage timing (SE_OPT_TIMING): one pair of events per stage per product
    bool timing = false;
    std::vector<cudaEvent_t> tev;      // pool, 2 * SE_NSTAGE per product
    int tprod = 0;                     // products recorded since the last read
};

// ---- launchers implemented in the .cu files ----
namespace se {

// Record the begin (end = false) or end (end = true) event of `stage` of the current product.
void stage_mark(se_ctx *c, int stage, cudaStream_t s, bool end);

SeParams make_params(const se_ctx *c);

// se_config.cu
int build_cells(se_ctx *c, const double *pos_dev, const double *rad_dev);
int build_support(se_ctx *c, int prec);

// se_real.cu
template <typename T>
void launch_real(se_ctx *c, const T *xs, T *yreal, cudaStream_t s, int ncomp);
template <typename T>
void setup_rel(se_ctx *c, cudaStream_t s);
template <typename T>
int build_pair_table(se_ctx *c);
bool launch_real_ff(se_ctx *c, const ff *xs, ff *yreal, cudaStream_t s, int ncomp);
int build_pair_table_ff(se_ctx *c);
// se_learned.cu: the damping theta and cutoff k_c <a> of the spectral correction that the
// learned network predicts for the configuration (mean of its per-particle outputs)
int learned_spectral_params(se_ctx *c, double *theta, double *ka, double *cmax);
// se_solve.cu
void convert_f2d(int n, const float *x, double *y, cudaStream_t s);
// exclusive scan of n ints into out[0..n] on stream s
void launch_scan(se_ctx *c, int n, const int *in, int *out, cudaStream_t s);

// se_wave.cu
template <typename T>
void launch_wave_spread(se_ctx *c, const T *xs, cudaStream_t s, int ncomp);
// CTAs per 16-plane spreading tile (partial grids) for ntiles tiles, at most maxparts
int spread16_split(int sms, int ntiles, int maxparts);
template <typename T>
void launch_wave_fft(se_ctx *c, cudaStream_t s);
// releases the spectral-correction sub-context (se_solve.cu)
void free_spectral(se_ctx *c);
bool fused_real_gather(const se_ctx *c, int ncomp, int with_wave);
template <typename T, typename TO>
void launch_gather_combine(se_ctx *c, const T *xs, const T *yreal, TO *y, int ncomp, int with_wave,
                           cudaStream_t s);
// the wave-space approach (SE_OPT_SIZE_MODE 3): spread, transforms, k-space step, gather + combine
template <typename T, typename TO>
void launch_wave_ws(se_ctx *c, const T *xs, const T *yreal, TO *y, int ncomp, int with_wave, cudaStream_t s);
template <typename T>
void setup_support(se_ctx *c, cudaStream_t s);
void make_twiddles(se_ctx *c, int prec);

// se_wave.cu: one persistent launch for the products of a batch of boxes (FP32)
struct PersistPlan {
    void *desc = nullptr;        // device BoxDesc[nbox]
    int *pref = nullptr;         // device [nbox][kPersistPhases] work items per phase
    unsigned *ctl = nullptr;     // device: abort flag, per-box claimed / finished counters, failure flag
    int ctl_words = 0;
    long long wait_ns = 2000000000ll;   // limit of every wait in the launch
    int stall_box = -1;          // test hook: this box's phase 1 never finishes (waits run out)
    int nbox = 0, ncomp = 0, dtype = -1, grid = 0;
    size_t smem = 0;
    const void *kernel = nullptr;
};
int persist_prepare(se_ctx *const *box, int nbox, int ncomp, const void *const *x, void *const *y, int dtype,
                    PersistPlan &pl, std::string &err);
int persist_launch(const PersistPlan &pl, cudaStream_t s, std::string &err);
// 1 if a persistent launch since the last call gave up at a grid barrier (synchronises)
int persist_failed(const PersistPlan &pl, cudaStream_t s);
void persist_free(PersistPlan &pl);

// se_api.cu
template <typename T, typename TI>
void launch_permute_in(se_ctx *c, const TI *x, T *xs, int ncomp, cudaStream_t s);
int se_apply_internal(se_ctx *c, int ncomp, const void *x, void *y, int dtype, int prec);

}  // namespace se

#define SE_CUDA_CHECK(ctx, call)                                                     \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);         \
            return SE_ERR_CUDA;                                                      \
        }                                                                            \
    } while (0)
