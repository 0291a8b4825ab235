// The wave-space approach to the particle sizes of Sec. 3.2 (SE_OPT_SIZE_MODE 3):
// every derivative of the Faxen laws and of the multipole expansion is taken in k-space.
//
// Source side (Eq. wave-only-f-assign and its torque / stresslet analogues): the moments
// F, T, S (5 coordinates), S_tr and a^2 F, a^2 S are spread with the plain window h, 20
// grid components in five groups of four.  After the forward transform the force density
// of the mobility is (this FFT's forward transform carries exp(-i q.n), so a real-space
// gradient of the window is a factor +i k)
//   H = F + (1/2) i k x T - i S.k - k^2 [ (1/6) a^2F - (1/10) i (a^2 S).k ]
// (Eqs. wave-only-compute-1/2 with the torque and stresslet terms), and the source
// density is S_tr.  The k-space kernel of Eq. wave-result (the one of the other size
// approaches) gives the velocity and pressure spectra v, p; the target derivatives are
// again factors of i k: v'' = -k^2 v, Omega = (1/2) i k x v, E = sym(i k v) on the
// orthonormal basis and E'' = -k^2 E, so that 20 grids come back (Eq. parseval-sum-2
// and its rotation / strain analogues) and the gather is the plain window:
//   U = sum h (v + a^2/6 v''),  Omega = sum h Omega,  E = sum h (E + a^2/10 E''),
//   E_tr = sum h p.
// The five groups reuse the 4-component FFT passes; a separate z pass (forward and
// inverse) runs on either side of the k-space kernel.  Spreading is grid-point centric
// (one thread per grid point over the particles of the spreading bins that reach it),
// the gather one warp per particle over its P^3 support.  This approach is for accuracy:
// it moves 40 grids through the FFT instead of 8.
//
// Included by se_wave.cu after its own kernels (same translation unit).

namespace se {
namespace {

constexpr int kWsGroups = 5;     // 20 real grid components in groups of 4

// z pass (forward or inverse) in place on half spectra [z][y][q][C]: a CTA takes the
// NL / C wave numbers q0.. of one y row, lines along z
template <typename T, int C, bool INV>
__global__ void __launch_bounds__(kFftThreads, 4) fft_z_plain(FftPlan plan, const typename C2<T>::t *twg,
                                                              typename C2<T>::t *data)
{
    using T2 = typename C2<T>::t;
    constexpr int NL = fft_nl<T>(), LB = NL / C, CPE = sizeof(T) == 4 ? 2 : 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int M = plan.M, Mh = M / 2 + 1;
    T2 *tw, *A, *B;
    fft_smem(smraw, M, NL, tw, A, B);
    for (int e = threadIdx.x; e < M; e += blockDim.x) tw[e] = twg[e];
    const int q0 = blockIdx.x * LB, nv = min(LB, Mh - q0) * C;
    const size_t base = ((size_t)blockIdx.y * Mh + q0) * C, es = (size_t)M * Mh * C;
    for (int e = threadIdx.x; e < (NL / CPE) * M; e += blockDim.x) {
        const int k = e % (NL / CPE), z = e / (NL / CPE);
        T2 *d = A + z * NL + k * CPE;
        if (k * CPE < nv) cp_async16(d, data + base + z * es + k * CPE);
        else
            for (int u = 0; u < CPE; ++u) d[u] = T2{0, 0};
    }
    cp_async_wait_all();
    __syncthreads();
    const T2 *Z = fft_run_dir<NL, INV>(A, B, plan, tw);
    for (int e = threadIdx.x; e < NL * M; e += blockDim.x) {
        const int l = e % NL, z = e / NL;
        if (l < nv) data[base + z * es + l] = Z[z * NL + l];
    }
}

// One thread per grid point: the plain window times the 20 moments of every particle
// whose support (P points from its first support point in each direction) contains the
// point, over the spreading bins (particles binned by first support point into tiles
// of 8^3) that can hold such a particle.  grid: [5][M^3][4].
template <typename T>
__global__ void __launch_bounds__(128) ws_spread_kernel(SeParams p, const int *tile_start, const int *tile_perm,
                                                        const int *base, const T *wg, const double *rad,
                                                        const T *xs, T *grid)
{
    const int M = p.M, P = p.P, nt = p.ntile;
    const size_t M3 = (size_t)M * M * M;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= M3) return;
    const int pt[3] = {(int)(n % M), (int)((n / M) % M), (int)(n / ((size_t)M * M))};
    // tiles holding a first support point b with (pt - b) mod M in [0, P)
    int tb0[3], ntb[3];
    for (int d = 0; d < 3; ++d) {
        const int lo = wrapi(pt[d] - P + 1 + M, M) % M;        // first admissible b
        tb0[d] = lo / kTile;
        ntb[d] = min(nt, (lo % kTile + P - 1) / kTile + 1);
    }
    T acc[4 * kWsGroups];
#pragma unroll
    for (int c = 0; c < 4 * kWsGroups; ++c) acc[c] = 0;
    for (int bz = 0; bz < ntb[2]; ++bz)
        for (int by = 0; by < ntb[1]; ++by)
            for (int bx = 0; bx < ntb[0]; ++bx) {
                const int bin = ((tb0[2] + bz) % nt * nt + (tb0[1] + by) % nt) * nt + (tb0[0] + bx) % nt;
                for (int e = tile_start[bin]; e < tile_start[bin + 1]; ++e) {
                    const int i = tile_perm[e];
                    int o[3];
                    bool in = true;
                    for (int d = 0; d < 3; ++d) {
                        o[d] = wrapi(pt[d] - base[3 * i + d], M);
                        in &= o[d] < P;
                    }
                    if (!in) continue;
                    const T *w = wg + (size_t)i * 3 * P;
                    const T h = w[o[0]] * w[P + o[1]] * w[2 * P + o[2]];
                    const T *x = xs + (size_t)i * kNC;
                    const T a2 = (T)(rad[i] * rad[i]);
                    // groups: F0 F1 F2 Str | T0 T1 T2 S0 | S1 S2 S3 S4 | a2F0 a2F1 a2F2 a2S0 | a2S1..a2S4
                    acc[0] += h * x[0];
                    acc[1] += h * x[1];
                    acc[2] += h * x[2];
                    acc[3] += h * x[11];
                    acc[4] += h * x[3];
                    acc[5] += h * x[4];
                    acc[6] += h * x[5];
                    acc[7] += h * x[6];
                    acc[8] += h * x[7];
                    acc[9] += h * x[8];
                    acc[10] += h * x[9];
                    acc[11] += h * x[10];
                    const T ha = h * a2;
                    acc[12] += ha * x[0];
                    acc[13] += ha * x[1];
                    acc[14] += ha * x[2];
                    acc[15] += ha * x[6];
                    acc[16] += ha * x[7];
                    acc[17] += ha * x[8];
                    acc[18] += ha * x[9];
                    acc[19] += ha * x[10];
                }
            }
#pragma unroll
    for (int g = 0; g < kWsGroups; ++g) {
        T *o = grid + ((size_t)g * M3 + n) * 4;
#pragma unroll
        for (int c = 0; c < 4; ++c) o[c] = acc[4 * g + c];
    }
}

template <typename T2>
__device__ __forceinline__ T2 cmul_i(T2 a) { return T2{-a.y, a.x}; }         // i a

// The k-space step of the wave-space approach on the full half spectrum: 20 input
// spectra (five groups [M][M][Mh][4]) to 20 output spectra (five groups), see the file
// header.  E, cnorm, the exponent and the Green's function are those of fft_z_scale.
template <typename T>
__global__ void __launch_bounds__(256) ws_kspace_kernel(int M, const typename C2<T>::t *in,
                                                        typename C2<T>::t *out, T cnorm, T twopiL, T i4x2,
                                                        T ecoef, T gam)
{
    using T2 = typename C2<T>::t;
    const int Mh = M / 2 + 1;
    const size_t nsp = (size_t)M * M * Mh;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nsp) return;
    const int qx = (int)(e % Mh), y = (int)((e / Mh) % M), z = (int)(e / ((size_t)Mh * M));
    const int ys = y <= M / 2 ? y : y - M, zsn = z <= M / 2 ? z : z - M;
    T2 o[4 * kWsGroups];
#pragma unroll
    for (int c = 0; c < 4 * kWsGroups; ++c) o[c] = T2{0, 0};
    const bool zero = (qx == 0 && ys == 0 && zsn == 0) || 2 * qx == M || 2 * ys == M || 2 * zsn == M;
    if (!zero) {
        T2 h[4 * kWsGroups];
#pragma unroll
        for (int g = 0; g < kWsGroups; ++g)
#pragma unroll
            for (int c = 0; c < 4; ++c) h[4 * g + c] = in[((size_t)g * nsp + e) * 4 + c];
        const T kx = twopiL * qx, ky = twopiL * ((T)ys - gam * (T)qx), kz = twopiL * zsn;
        const T kv[3] = {kx, ky, kz};
        const T k2 = kx * kx + ky * ky + kz * kz;
        const T q2 = (T)(qx * qx + ys * ys + zsn * zsn);
        const T ex = -k2 * i4x2 + ecoef * q2;
        T E;
        if constexpr (sizeof(T) == 4) E = expf(ex) * cnorm;
        else E = exp(ex) * cnorm;
        const T ik2 = 1 / k2;
        const T Phi = E * (1 + k2 * i4x2) * ik2;
        // moments: F (3), S_tr, T (3), S and a^2 S as tensors (xx yy zz xy xz yz), a^2 F (3)
        const T2 F[3] = {h[0], h[1], h[2]}, Hs = h[3], Tq[3] = {h[4], h[5], h[6]};
        const T2 sc[5] = {h[7], h[8], h[9], h[10], h[11]}, asc[5] = {h[15], h[16], h[17], h[18], h[19]};
        const T2 aF[3] = {h[12], h[13], h[14]};
        T Sr[6], Si[6], aSr[6], aSi[6];
        {
            const T a[5] = {sc[0].x, sc[1].x, sc[2].x, sc[3].x, sc[4].x}, b[5] = {sc[0].y, sc[1].y, sc[2].y, sc[3].y, sc[4].y};
            const T c[5] = {asc[0].x, asc[1].x, asc[2].x, asc[3].x, asc[4].x};
            const T d[5] = {asc[0].y, asc[1].y, asc[2].y, asc[3].y, asc[4].y};
            stresslet_tensor(a, Sr);
            stresslet_tensor(b, Si);
            stresslet_tensor(c, aSr);
            stresslet_tensor(d, aSi);
        }
        // (S.k)_a for a symmetric tensor stored (xx yy zz xy xz yz)
        auto sdot = [&](const T *S, int a) {
            const int ix[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
            return S[ix[a][0]] * kv[0] + S[ix[a][1]] * kv[1] + S[ix[a][2]] * kv[2];
        };
        T2 H[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int b = (a + 1) % 3, c = (a + 2) % 3;
            // (k x T)_a
            const T2 kT = T2{kv[b] * Tq[c].x - kv[c] * Tq[b].x, kv[b] * Tq[c].y - kv[c] * Tq[b].y};
            const T2 Sk = T2{sdot(Sr, a), sdot(Si, a)}, aSk = T2{sdot(aSr, a), sdot(aSi, a)};
            const T2 t1 = cmul_i(kT), t2 = cmul_i(Sk), t3 = cmul_i(aSk);
            // F + (1/2) i k x T - i S.k - k^2 [ a^2 F / 6 - (1/10) i a^2 S.k ]
            H[a] = T2{F[a].x + (T)0.5 * t1.x - t2.x - k2 * (aF[a].x / 6 - (T)0.1 * t3.x),
                      F[a].y + (T)0.5 * t1.y - t2.y - k2 * (aF[a].y / 6 - (T)0.1 * t3.y)};
        }
        const T2 kH = T2{kx * H[0].x + ky * H[1].x + kz * H[2].x, kx * H[0].y + ky * H[1].y + kz * H[2].y};
        const T2 pr = T2{kH.x * ik2, kH.y * ik2};
        const T sq = -E * (T)0.25 * ik2;
        const T2 iHs = T2{-Hs.y * sq, Hs.x * sq};
        T2 v[3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            v[a] = T2{Phi * (H[a].x - kv[a] * pr.x) + kv[a] * iHs.x, Phi * (H[a].y - kv[a] * pr.y) + kv[a] * iHs.y};
        const T cp = (T)-0.75 * E;
        const T2 op = T2{-cp * pr.y, cp * pr.x};
        // Omega = (1/2) i k x v
        T2 Om[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int b = (a + 1) % 3, c = (a + 2) % 3;
            const T2 kv_ = T2{kv[b] * v[c].x - kv[c] * v[b].x, kv[b] * v[c].y - kv[c] * v[b].y};
            const T2 t = cmul_i(kv_);
            Om[a] = T2{(T)0.5 * t.x, (T)0.5 * t.y};
        }
        // G_ab = i k_a v_b (the gradient), E on the orthonormal basis of its symmetric part
        auto G = [&](int a, int b) { return cmul_i(T2{kv[a] * v[b].x, kv[a] * v[b].y}); };
        const T r2 = (T)0.70710678118654752440, r6 = (T)0.40824829046386301637;
        const T2 gxx = G(0, 0), gyy = G(1, 1), gzz = G(2, 2);
        const T2 gxy = G(0, 1), gyx = G(1, 0), gxz = G(0, 2), gzx = G(2, 0), gyz = G(1, 2), gzy = G(2, 1);
        T2 Em[5];
        Em[0] = T2{r2 * (gxx.x - gyy.x), r2 * (gxx.y - gyy.y)};
        Em[1] = T2{r6 * (2 * gzz.x - gxx.x - gyy.x), r6 * (2 * gzz.y - gxx.y - gyy.y)};
        Em[2] = T2{r2 * (gxy.x + gyx.x), r2 * (gxy.y + gyx.y)};
        Em[3] = T2{r2 * (gxz.x + gzx.x), r2 * (gxz.y + gzx.y)};
        Em[4] = T2{r2 * (gyz.x + gzy.x), r2 * (gyz.y + gzy.y)};
        // outputs: v0 v1 v2 p | v''0 v''1 v''2 Om0 | Om1 Om2 E0 E1 | E2 E3 E4 E''0 | E''1..E''4
        o[0] = v[0];
        o[1] = v[1];
        o[2] = v[2];
        o[3] = op;
        o[4] = T2{-k2 * v[0].x, -k2 * v[0].y};
        o[5] = T2{-k2 * v[1].x, -k2 * v[1].y};
        o[6] = T2{-k2 * v[2].x, -k2 * v[2].y};
        o[7] = Om[0];
        o[8] = Om[1];
        o[9] = Om[2];
        o[10] = Em[0];
        o[11] = Em[1];
        o[12] = Em[2];
        o[13] = Em[3];
        o[14] = Em[4];
#pragma unroll
        for (int m = 0; m < 5; ++m) o[15 + m] = T2{-k2 * Em[m].x, -k2 * Em[m].y};
    }
#pragma unroll
    for (int g = 0; g < kWsGroups; ++g)
#pragma unroll
        for (int c = 0; c < 4; ++c) out[((size_t)g * nsp + e) * 4 + c] = o[4 * g + c];
}

// One warp per particle (internal order): plain-window sums of the 20 gathered grids over
// the P^3 support (lanes on points, compensated), then the outputs, the real-space part
// and the self terms, written in the caller's order and dtype.
template <typename T, typename TO>
__global__ void __launch_bounds__(256) ws_gather_kernel(SeParams p, int N, const int *base, const T *wg,
                                                        const double *rad, const T *selfc, const int *perm,
                                                        const T *grid, const T *xs, const T *yreal, TO *y,
                                                        int ncomp_out, int with_wave, int with_self)
{
    const int i = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (i >= N) return;
    const int M = p.M, P = p.P;
    const size_t M3 = (size_t)M * M * M;
    T acc[4 * kWsGroups], cmp[4 * kWsGroups];
#pragma unroll
    for (int c = 0; c < 4 * kWsGroups; ++c) acc[c] = cmp[c] = 0;
    if (with_wave) {
        const int bx = base[3 * i], by = base[3 * i + 1], bz = base[3 * i + 2];
        const T *w = wg + (size_t)i * 3 * P;
        const int P3 = P * P * P;
        for (int e = lane; e < P3; e += 32) {
            const int ox = e % P, oy = (e / P) % P, oz = e / (P * P);
            const T h = w[ox] * w[P + oy] * w[2 * P + oz];
            const size_t n = ((size_t)wrapi(bz + oz, M) * M + wrapi(by + oy, M)) * M + wrapi(bx + ox, M);
#pragma unroll
            for (int g = 0; g < kWsGroups; ++g) {
                const T *gp = grid + ((size_t)g * M3 + n) * 4;
#pragma unroll
                for (int c = 0; c < 4; ++c) kahan_add(acc[4 * g + c], cmp[4 * g + c], h * gp[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < 4 * kWsGroups; ++c) {
            T v = acc[c] - cmp[c];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            acc[c] = v;
        }
    }
    if (lane != 0) return;
    const T a2 = (T)(rad[i] * rad[i]);
    T out[kNC];
    for (int a = 0; a < 3; ++a) out[a] = acc[a] + a2 / 6 * acc[4 + a];
    out[3] = acc[7];
    out[4] = acc[8];
    out[5] = acc[9];
    for (int m = 0; m < 5; ++m) out[6 + m] = acc[10 + m] + a2 / 10 * acc[15 + m];
    out[11] = acc[3];
    const T *xi_ = xs + (size_t)i * kNC;
    const T *yr = yreal + (size_t)i * kNC;
    T sc[4] = {0, 0, 0, 0};
    if (with_self)
        for (int k = 0; k < 4; ++k) sc[k] = selfc[4 * i + k];
    TO *yo = y + (size_t)perm[i] * ncomp_out;
    for (int c = 0; c < kNC; ++c)
        if (c < ncomp_out) yo[c] = (TO)(out[c] + yr[c] + sc[c < 3 ? 0 : (c < 6 ? 1 : (c < 11 ? 2 : 3))] * xi_[c]);
}

}  // namespace

// the whole wave-space-approach chain after the real-space part: spread, five forward
// 3D transforms, the k-space step, five inverse transforms, gather + combine
template <typename T, typename TO>
void launch_wave_ws(se_ctx *c, const T *xs, const T *yreal, TO *y, int ncomp, int with_wave, cudaStream_t s)
{
    using T2 = typename C2<T>::t;
    const int P = pix<T>();
    const SeParams p = make_params(c);
    const int M = c->M, Mh = M / 2 + 1;
    const size_t M3 = (size_t)M * M * M, nsp = (size_t)M * M * Mh;
    T *grid = (T *)c->b.ws_grid[P];
    T2 *sa = (T2 *)c->b.ws_spec_a[P], *sb = (T2 *)c->b.ws_spec_b[P];
    const T2 *tw = (const T2 *)c->b.tw[P];
    const int N = (int)c->N;
    if (with_wave) {
        stage_mark(c, SE_STAGE_SPREAD, s, false);
        ws_spread_kernel<T><<<(unsigned)((M3 + 127) / 128), 128, 0, s>>>(
            p, c->b.tile_start, c->b.tile_perm, c->b.sup_base, (const T *)c->b.sup_w[P], c->b.rad, xs, grid);
        c->launches++;
        stage_mark(c, SE_STAGE_SPREAD, s, true);
        constexpr int NL = fft_nl<T>();
        const size_t smem = fft_smem_bytes<T2>(M, NL);
        cudaFuncSetAttribute(fft_x_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(fft_z_plain<T, 4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(fft_z_plain<T, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(fft_x_inv<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const dim3 zg((Mh + NL / 4 - 1) / (NL / 4), M);
        stage_mark(c, SE_STAGE_FFT_XF, s, false);
        for (int g = 0; g < kWsGroups; ++g)
            fft_x_fwd<T><<<M * M / (NL / 2), kFftThreads, smem, s>>>(c->plan, tw, grid + (size_t)g * M3 * 4,
                                                                      sa + (size_t)g * nsp * 4);
        stage_mark(c, SE_STAGE_FFT_XF, s, true);
        stage_mark(c, SE_STAGE_FFT_YF, s, false);
        for (int g = 0; g < kWsGroups; ++g) launch_y<T, 4, false>(c, tw, sa + (size_t)g * nsp * 4, s);
        stage_mark(c, SE_STAGE_FFT_YF, s, true);
        stage_mark(c, SE_STAGE_FFT_Z, s, false);
        for (int g = 0; g < kWsGroups; ++g)
            fft_z_plain<T, 4, false><<<zg, kFftThreads, smem, s>>>(c->plan, tw, sa + (size_t)g * nsp * 4);
        const T cnorm = (T)(pow(p.alpha / kPi, 3.0) / (p.eta * p.L * p.L * p.L));
        const T twopiL = (T)(2.0 * kPi / p.L), i4x2 = (T)(0.25 / (p.xi * p.xi));
        const T ecoef = (T)(2.0 * kPi * kPi / (p.alpha * (double)M * M));
        ws_kspace_kernel<T><<<(unsigned)((nsp + 255) / 256), 256, 0, s>>>(M, sa, sb, cnorm, twopiL, i4x2, ecoef,
                                                                          (T)p.gamma);
        for (int g = 0; g < kWsGroups; ++g)
            fft_z_plain<T, 4, true><<<zg, kFftThreads, smem, s>>>(c->plan, tw, sb + (size_t)g * nsp * 4);
        stage_mark(c, SE_STAGE_FFT_Z, s, true);
        stage_mark(c, SE_STAGE_FFT_YI, s, false);
        for (int g = 0; g < kWsGroups; ++g) launch_y<T, 4, true>(c, tw, sb + (size_t)g * nsp * 4, s);
        stage_mark(c, SE_STAGE_FFT_YI, s, true);
        stage_mark(c, SE_STAGE_FFT_XI, s, false);
        for (int g = 0; g < kWsGroups; ++g)
            fft_x_inv<T, 4><<<M * M / (NL / 2), kFftThreads, smem, s>>>(c->plan, tw, sb + (size_t)g * nsp * 4,
                                                                         grid + (size_t)g * M3 * 4);
        stage_mark(c, SE_STAGE_FFT_XI, s, true);
        c->launches += 6 * kWsGroups + 2;
    }
    stage_mark(c, SE_STAGE_GATHER, s, false);
    ws_gather_kernel<T, TO><<<(unsigned)((N + 7) / 8), 256, 0, s>>>(
        p, N, c->b.sup_base, (const T *)c->b.sup_w[P], c->b.rad, (const T *)c->b.self_c[P], c->b.perm, grid, xs,
        yreal, y, ncomp, with_wave, (c->parts & 4) ? 1 : 0);
    c->launches++;
    stage_mark(c, SE_STAGE_GATHER, s, true);
}

template void launch_wave_ws<float, float>(se_ctx *, const float *, const float *, float *, int, int, cudaStream_t);
template void launch_wave_ws<float, double>(se_ctx *, const float *, const float *, double *, int, int, cudaStream_t);
template void launch_wave_ws<double, float>(se_ctx *, const double *, const double *, float *, int, int, cudaStream_t);
template void launch_wave_ws<double, double>(se_ctx *, const double *, const double *, double *, int, int,
                                             cudaStream_t);

}  // namespace se
