// FP32 spreading over 8 x 4 x 16 blocks, one warp per block (included by se_wave.cu inside its
// anonymous namespace, after spread16_body).
//
// The same column scheme as spread16_body (column coefficients, packed plane-pair FMAs over 16
// planes), with the 8 x 8 x 16 tile split into two halves of 4 rows, each owned by one warp that
// stages its own candidates.  Against the two-warp tile: (1) no CTA barrier (a warp's __syncwarp
// ends a staging round), so a warp never waits for the other half of the tile, which in the
// two-warp form sat at the barrier whenever a particle covered only the other half's rows;
// (2) a particle that misses the half's 4 rows is dropped at staging instead of costing the
// warp an idle pass.  Each block takes the candidates of its 8 x 8 x 16 tile (the same spreading
// bins) and keeps those whose support reaches its rows.
constexpr int kTw = 4;     // rows of a warp block

#ifndef SE_SPREAD16W_CH
#define SE_SPREAD16W_CH 24
#endif
#ifndef SE_SPREAD16W_MINB
#define SE_SPREAD16W_MINB 16
#endif

struct Spread16wSmem {
    float sxy[SE_SPREAD16W_CH][2 * kTile];   // x weights (8), y weights of the 4 rows; entry e at e ^ sw
    float4 swz[SE_SPREAD16W_CH][kTz];        // as Spread16SmemT::swz
    float4 sp[SE_SPREAD16W_CH][7];           // as Spread16SmemT::sp
    int bin_beg[6 * 6 * 7], bin_off[6 * 6 * 7 + 1];
};

// block `blk` (x tile, row half, y tile, z tile) of the grid, part `part` of nsplit
template <int NCOMP, bool SPLIT>
__device__ __forceinline__ void spread16w_body(int blk, int part, int lane, Spread16wSmem &sm, SeParams p,
                                               const int *tile_start, const int *tile_perm, const int *base,
                                               const float *s0g, const float *wg, const double *rad,
                                               const float *xs, float *grid, int nsplit)
{
    constexpr int TT = kTile, TZ = kTz, CH = SE_SPREAD16W_CH;
    auto &sxy = sm.sxy;
    auto &swz = sm.swz;
    auto &sp = sm.sp;
    auto &bin_beg = sm.bin_beg;
    auto &bin_off = sm.bin_off;
    const int M = p.M, P = p.P, nt = p.ntile;
    const int bx0 = blk % nt, hy = (blk / nt) % (2 * nt), bzp = blk / (2 * nt * nt);
    const int by0 = hy >> 1, half = hy & 1;
    // origin of the warp's block: x, y (its 4 rows), z
    const int t0[3] = {bx0 * TT, by0 * TT + half * kTw, bzp * TZ};
    const int tz_planes = min(TZ, M - t0[2]);           // 16, or 8 for the last tile of an odd nt
    const int tx = lane & 7, ty = lane >> 3;            // column of the lane (ty < 4)
    const int nbin = (P - 1 + TT - 1) / TT + 1;
    const int nbz = nbin + (tz_planes > TT ? 1 : 0);
    const int bztop = 2 * bzp + (tz_planes > TT ? 1 : 0);
    const int nb3 = nbin * nbin * nbz;
    const float alpha = (float)p.alpha, kap = (float)p.kappa, akap = alpha * kap;
    u64 acc2[TZ / 2][4];
#pragma unroll
    for (int z = 0; z < TZ / 2; ++z)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc2[z][c] = 0ull;

    for (int bb = lane; bb < nb3; bb += 32) {
        const int bx = bb % nbin, by = (bb / nbin) % nbin, bz = bb / (nbin * nbin);
        const int bin = (wrapi(bztop - bz, nt) * nt + wrapi(by0 - by, nt)) * nt + wrapi(bx0 - bx, nt);
        bin_beg[bb] = tile_start[bin];
        bin_off[bb + 1] = tile_start[bin + 1] - tile_start[bin];
    }
    __syncwarp();
    if (lane == 0) {
        bin_off[0] = 0;
        for (int bb = 0; bb < nb3; ++bb) bin_off[bb + 1] += bin_off[bb];
    }
    __syncwarp();
    const int total = bin_off[nb3];

    int cbeg = 0, cstep = CH;
    if constexpr (SPLIT) {
        grid += (size_t)part * M * M * M * 4;
        cbeg = part * CH;
        cstep = nsplit * CH;
    }
    for (int c0 = cbeg; c0 < total; c0 += cstep) {
        const int cnt = min(CH, total - c0);
        __syncwarp();
        // candidate of this lane, kept if its support reaches the block (compacted by ballot)
        bool ok = false;
        int i = 0, od[3] = {0, 0, 0};
        if (lane < cnt) {
            const int idx = c0 + lane;
            int lo = 0, hi = nb3;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (bin_off[mid] <= idx) lo = mid; else hi = mid;
            }
            i = tile_perm[bin_beg[lo] + idx - bin_off[lo]];
            ok = true;
            for (int d = 0; d < 3; ++d) {
                int o = wrapi(t0[d] - base[3 * i + d], M);
                if (o >= P) o -= M;
                ok &= (o < P) && (o > -(d == 2 ? TZ : (d == 1 ? kTw : TT)));
                od[d] = o;
            }
        }
        const unsigned keep = __ballot_sync(0xffffffffu, ok);
        const int nk = __popc(keep);
        if (ok) {
            const int k = __popc(keep & ((1u << lane) - 1u));
            const float *w = wg + (size_t)i * 3 * P;
            const int sw_xy = (k >> 1) & 15, sw_z = k & 7;
#pragma unroll
            for (int t = 0; t < TT; ++t) {
                const int ix = od[0] + t;
                sxy[k][t ^ sw_xy] = (ix >= 0 && ix < P) ? w[ix] : 0.f;
            }
#pragma unroll
            for (int t = 0; t < kTw; ++t) {
                const int iy = od[1] + t;
                sxy[k][(TT + t) ^ sw_xy] = (iy >= 0 && iy < P) ? w[P + iy] : 0.f;
            }
            const float s0z = s0g[3 * i + 2];
#pragma unroll
            for (int zp = 0; zp < TZ / 2; ++zp) {
                float4 W[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int iz = od[2] + 2 * zp + h;
                    const float g = (iz >= 0 && iz < P) ? w[2 * P + iz] : 0.f;
                    const float sz = s0z + (float)iz;
                    W[h] = make_float4(g, g * sz, g * sz * sz, g * sz * sz * sz);
                }
                swz[k][(2 * zp) ^ sw_z] = make_float4(W[0].x, W[1].x, W[0].y, W[1].y);
                swz[k][(2 * zp + 1) ^ sw_z] = make_float4(W[0].z, W[1].z, W[0].w, W[1].w);
            }
            const float a = (float)rad[i], a2k2 = a * a * kap * kap;
            const float *xi = xs + (size_t)i * kNC;
            float S[6] = {0, 0, 0, 0, 0, 0}, Tq[3] = {0, 0, 0};
            if constexpr (NCOMP >= 6) { Tq[0] = xi[3]; Tq[1] = xi[4]; Tq[2] = xi[5]; }
            if constexpr (NCOMP >= 11) stresslet_tensor(xi + 6, S);
            const int zlo = max(0, -od[2]), zhi = min(tz_planes, P - od[2]);
            int quarters = 0;
#pragma unroll
            for (int qq = 0; qq < 4; ++qq)
                if (zlo < 4 * qq + 4 && zhi > 4 * qq) quarters |= 1 << qq;
            // column-polynomial coefficients of the particle, as in spread16_body
            const float A0 = 1 - a2k2 * alpha, A1 = (2.0f / 3.0f) * a2k2 * alpha * alpha;
            const float B0 = 2 * kap * alpha * (1 - a2k2 * alpha), B1 = 0.8f * kap * a2k2 * alpha * alpha * alpha;
            sp[k][0] = make_float4(s0g[3 * i] + (float)od[0], s0g[3 * i + 1] + (float)od[1], (float)quarters,
                                   NCOMP >= 12 ? xi[11] : 0.f);
            sp[k][1] = make_float4(A0, A1, B0, B1);
            sp[k][2] = make_float4(xi[0], xi[1], xi[2], akap * Tq[0]);
            sp[k][3] = make_float4(akap * Tq[1], akap * Tq[2], S[0], S[1]);
            sp[k][4] = make_float4(S[2], S[3], S[4], S[5]);
            sp[k][5] = make_float4(A1 * xi[0], A1 * xi[1], A1 * xi[2], B1 * S[4]);
            sp[k][6] = make_float4(B1 * S[5], B1 * S[2], 0.f, 0.f);
        }
        __syncwarp();
        for (int k = 0; k < nk; ++k) {
            const int sw_xy = (k >> 1) & 15, sw_z = k & 7;
            const float gxy = sxy[k][tx ^ sw_xy] * sxy[k][(TT + ty) ^ sw_xy];
            const float4 v0 = sp[k][0];
            const int quarters = (int)v0.z;
            if (gxy == 0.f || quarters == 0) continue;
            spread16_column<NCOMP>(k, sw_z, gxy, v0, tx, ty, sp, swz, acc2);
        }
    }
#pragma unroll
    for (int zp = 0; zp < TZ / 2; ++zp) {
        float lo[4], hi[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) unpack2(acc2[zp][q], lo[q], hi[q]);
        const int z = 2 * zp;
        if (z < tz_planes) {
            const size_t gi = (((size_t)(t0[2] + z) * M + (t0[1] + ty)) * M + (t0[0] + tx)) * 4;
            *reinterpret_cast<float4 *>(grid + gi) = make_float4(lo[0], lo[1], lo[2], NCOMP >= 12 ? lo[3] : 0.f);
            *reinterpret_cast<float4 *>(grid + gi + (size_t)M * M * 4) =
                make_float4(hi[0], hi[1], hi[2], NCOMP >= 12 ? hi[3] : 0.f);
        }
    }
}

template <int NCOMP, bool SPLIT>
__global__ void __launch_bounds__(32, SE_SPREAD16W_MINB) spread16w_kernel(SeParams p, const int *tile_start,
                                                                          const int *tile_perm, const int *base,
                                                                          const float *s0g, const float *wg,
                                                                          const double *rad, const float *xs,
                                                                          float *grid, int nsplit)
{
    __shared__ Spread16wSmem sm;
    spread16w_body<NCOMP, SPLIT>(blockIdx.x, blockIdx.y, threadIdx.x, sm, p, tile_start, tile_perm, base, s0g, wg,
                                 rad, xs, grid, nsplit);
}
