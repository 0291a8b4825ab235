/*
 * Direct-Ewald oracle for the periodic far-field grand mobility
 *   M_inf . [F, T, S, S_tr]  ->  [U, Omega, E, E_tr]
 * of Wang & Brady, "Spectral Ewald Acceleration of Stokesian Dynamics for
 * polydisperse suspensions" (arXiv 1506.08481).
 *
 * TEST INFRASTRUCTURE.  This file is the parity reference for the CUDA path.
 * Only the test-suite, the smoke check and the CPU-baseline leg of the bench
 * may load it.  It shares no code with the CUDA path.  It is plain FP64 and
 * deliberately slow: O(N^2) real space plus O(N K) wave space, no Spectral
 * Ewald, no FFT, no grids.
 *
 * ---------------------------------------------------------------------------
 * What is computed (all citations are to the paper's sections / equations)
 * ---------------------------------------------------------------------------
 * Per particle: 12 input components  [F(3), T(3), S(5), S_tr(1)]
 *               12 output components [U(3), Omega(3), E(5), E_tr(1)]
 * S and E are traceless symmetric tensors stored as coordinates on the
 * orthonormal basis Y^m (see stresslet_basis).  S_tr is the pressure moment
 * (trace of the stresslet, Eq. press-moment), E_tr its conjugate expansion rate.
 *
 * Inputs are moments exerted by the particles on the fluid, outputs the rigid
 * body motions / strain rates they induce, so that every self block is
 * positive and the F,T,S block is symmetric positive definite (Sec. 2.1).
 *
 * Velocity field of source j at x = r - r_j (Eq. mul-expand, Eq. compress-vel-disturb):
 *   v = 1/(8 pi eta) [ (1 + a_j^2 Lap/6) J.F + R.T - (1 + a_j^2 Lap/10) K:S ] + Q S_tr
 * with J = (I Lap - grad grad) psi, R_ab = 1/2 eps_agb d_g Lap psi,
 * K:S = (delta_ab d_g Lap psi - d_a d_b d_g psi) S_bg,  Q = -grad(phi)/(16 pi eta)
 * where psi is the Stokes generator (psi = r in free space, Eq. oseen) and
 * phi the Laplace generator (phi = 1/r; Eq. pres-vel-disturb, Eq. wave-dist-S).
 * Pressure (Eq. pres-multi-expans):  p = 1/(4 pi) [ P.F - grad P : S ],  P = -grad phi.
 *
 * Faxen laws at the target i (Eqs. faxen-f, faxen-t, faxen-s, faxen-p):
 *   U     = F_i/(6 pi eta a)         + (1 + a_i^2 Lap/6) v
 *   Omega = T_i/(8 pi eta a^3)       + 1/2 curl v
 *   E     = S_i/((20/3) pi eta a^3)  + (1 + a_i^2 Lap/10) sym grad v
 *   E_tr  = 3 S_tr,i/(16 pi eta a^3) + 3/(4 eta) p
 * (E_tr receives nothing from other particles' S_tr: pressure moments do not
 *  produce pressure disturbances, Sec. 2.3.)
 *
 * Periodic sums (Eq. oseen-peridoic, Eq. wave-dist-S) are split by Hasimoto's
 * integral (Eq. ewald-theta) into
 *   real space : psi_R(r) = r erfc(xi r) - exp(-xi^2 r^2)/(xi sqrt(pi))   (Eq. oseen-ewald-rs)
 *                phi_R(r) = erfc(xi r)/r                                  (Eq. source-split)
 *   wave space : psi^_k = -(8 pi/V) k^-4 (1 + k^2/(4 xi^2)) exp(-k^2/(4 xi^2))   (Eq. oseen-ewald-ws)
 *                phi^_k = (4 pi/V) k^-2 exp(-k^2/(4 xi^2))                     (Eq. source-split)
 *   with fields f(x) = sum_{k != 0} f^_k exp(-i k.x), so d/dx -> -i k, Lap -> -k^2.
 * The self interaction contained in the wave sum is removed (Eq. uf-self) by
 * subtracting the limit x -> 0 of the same operators applied to the smooth
 * functions  W_psi = psi_free - psi_R = r erf(xi r) + exp(-xi^2 r^2)/(xi sqrt(pi))
 *       and  W_phi = phi_free - phi_R = erf(xi r)/r.
 *
 * Radial machinery.  For a radial function g(r) let D = (1/r) d/dr.  Then
 *   d_a g = x_a Dg,  d_a d_b g = delta_ab Dg + x_a x_b D^2 g, ... (orders <= 4 below),
 *   D^k(Lap g) = (2k+3) D^{k+1} g + r^2 D^{k+2} g.
 * For psi_R:  D psi_R = B_0 = erfc(xi r)/r  and  D^k psi_R = (-1)^{k-1} B_{k-1};
 * for phi_R:  D^k phi_R = (-1)^k B_k, with the multipole-Ewald recurrence of
 * W. Smith (CCP5 Newsletter 46, 1998):
 *   B_n = [ (2n-1) B_{n-1} + (2 xi^2)^n exp(-xi^2 r^2)/(xi sqrt(pi)) ] / r^2.
 * At r = 0 an even analytic g = sum_m c_m r^{2m} has D^k g(0) = 2^k k! c_k.
 *
 * Cubic box of side L only (lattice vectors L e_1, L e_2, L e_3).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NC 12          /* components per particle */
#define ND 12          /* length of D-arrays */

static const double PI = 3.14159265358979323846;

/* Orthonormal basis of symmetric traceless 3x3 tensors. */
static void stresslet_basis(double Y[5][3][3])
{
    memset(Y, 0, sizeof(double) * 45);
    const double s2 = 1.0 / sqrt(2.0), s6 = 1.0 / sqrt(6.0);
    Y[0][0][0] = s2;  Y[0][1][1] = -s2;                       /* (xx - yy)/sqrt2      */
    Y[1][0][0] = -s6; Y[1][1][1] = -s6; Y[1][2][2] = 2 * s6;  /* (2zz - xx - yy)/sqrt6 */
    Y[2][0][1] = s2;  Y[2][1][0] = s2;                        /* (xy + yx)/sqrt2      */
    Y[3][0][2] = s2;  Y[3][2][0] = s2;                        /* (xz + zx)/sqrt2      */
    Y[4][1][2] = s2;  Y[4][2][1] = s2;                        /* (yz + zy)/sqrt2      */
}

static int eps3(int a, int b, int c)
{
    if (a == b || b == c || a == c) return 0;
    return ((a == 0 && b == 1) || (a == 1 && b == 2) || (a == 2 && b == 0)) ? 1 : -1;
}

/* ---------------- radial D-arrays ---------------- */

/* Real-space Ewald functions B_0..B_nmax at r > 0 (Smith's recurrence). */
static void ewald_B(double r, double xi, int nmax, double *B)
{
    double r2 = r * r;
    double ex = exp(-xi * xi * r2) / (xi * sqrt(PI));
    B[0] = erfc(xi * r) / r;
    double p = 1.0;
    for (int n = 1; n <= nmax; n++) {
        p *= 2 * xi * xi;
        B[n] = ((2 * n - 1) * B[n - 1] + p * ex) / r2;
    }
}

/* Free-space limit (xi -> 0) of B_n: (2n-1)!!/r^{2n+1}. */
static void free_B(double r, int nmax, double *B)
{
    B[0] = 1.0 / r;
    for (int n = 1; n <= nmax; n++) B[n] = (2 * n - 1) * B[n - 1] / (r * r);
}

/* D^k psi and D^k phi from B_n (index 0 unused: psi, phi never appear undifferentiated). */
static void dpsi_dphi_from_B(const double *B, double *dpsi, double *dphi)
{
    dpsi[0] = 0.0;
    for (int k = 1; k < ND; k++) dpsi[k] = ((k - 1) % 2 == 0 ? 1.0 : -1.0) * B[k - 1];
    for (int k = 0; k < ND; k++) dphi[k] = (k % 2 == 0 ? 1.0 : -1.0) * B[k];
}

/* D-arrays at r = 0 of the smooth wave-space remainders W_psi and W_phi. */
static void dW_at_origin(double xi, double *dpsi, double *dphi)
{
    double sp = sqrt(PI);
    double fact = 1.0, two_k = 1.0;
    for (int k = 0; k < ND; k++) {
        if (k > 0) { fact *= k; two_k *= 2.0; }
        /* W_psi = r erf(xi r) + exp(-xi^2 r^2)/(xi sqrt pi): c_0 = 1/(xi sqrt pi),
           c_m = (-1)^{m-1} xi^{2m-1} / (sqrt(pi) m! (2m-1)) */
        double cpsi = (k == 0) ? 1.0 / (xi * sp)
                               : ((k - 1) % 2 == 0 ? 1.0 : -1.0) * pow(xi, 2 * k - 1) / (sp * fact * (2 * k - 1));
        /* W_phi = erf(xi r)/r: c_m = 2 (-1)^m xi^{2m+1} / (sqrt(pi) m! (2m+1)) */
        double cphi = 2.0 * (k % 2 == 0 ? 1.0 : -1.0) * pow(xi, 2 * k + 1) / (sp * fact * (2 * k + 1));
        dpsi[k] = two_k * fact * cpsi;
        dphi[k] = two_k * fact * cphi;
    }
}

/* D^k (Lap g) = (2k+3) D^{k+1} g + r^2 D^{k+2} g, for k = 0 .. n-1. */
static void lap_D(const double *in, double r2, double *out, int n)
{
    for (int k = 0; k < n; k++) out[k] = (2 * k + 3) * in[k + 1] + r2 * in[k + 2];
    for (int k = n; k < ND; k++) out[k] = 0.0;
}

/* ---------------- Cartesian derivative tensors of a radial function ---------------- */

static inline double dl(int a, int b) { return a == b ? 1.0 : 0.0; }

static void tens1(const double *g, const double *x, double t[3])
{
    for (int a = 0; a < 3; a++) t[a] = x[a] * g[1];
}
static void tens2(const double *g, const double *x, double t[3][3])
{
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) t[a][b] = dl(a, b) * g[1] + x[a] * x[b] * g[2];
}
static void tens3(const double *g, const double *x, double t[3][3][3])
{
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            for (int c = 0; c < 3; c++)
                t[a][b][c] = (dl(a, b) * x[c] + dl(a, c) * x[b] + dl(b, c) * x[a]) * g[2]
                           + x[a] * x[b] * x[c] * g[3];
}
static void tens4(const double *g, const double *x, double t[3][3][3][3])
{
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            for (int c = 0; c < 3; c++)
                for (int d = 0; d < 3; d++)
                    t[a][b][c][d] =
                        (dl(a, b) * dl(c, d) + dl(a, c) * dl(b, d) + dl(a, d) * dl(b, c)) * g[2]
                      + (dl(a, b) * x[c] * x[d] + dl(a, c) * x[b] * x[d] + dl(a, d) * x[b] * x[c]
                       + dl(b, c) * x[a] * x[d] + dl(b, d) * x[a] * x[c] + dl(c, d) * x[a] * x[b]) * g[3]
                      + x[a] * x[b] * x[c] * x[d] * g[4];
}

/* ---------------- generator sets ---------------- */

/* D-arrays of psi, Lap psi, Lap^2 psi, Lap^3 psi, phi, Lap phi at one separation. */
typedef struct {
    double psi[ND], Lpsi[ND], L2psi[ND], L3psi[ND];
    double phi[ND], Lphi[ND];
} gens_t;

static void make_gens(const double *dpsi, const double *dphi, double r2, gens_t *g)
{
    memcpy(g->psi, dpsi, sizeof(double) * ND);
    lap_D(g->psi, r2, g->Lpsi, ND - 2);
    lap_D(g->Lpsi, r2, g->L2psi, ND - 4);
    lap_D(g->L2psi, r2, g->L3psi, ND - 6);
    memcpy(g->phi, dphi, sizeof(double) * ND);
    lap_D(g->phi, r2, g->Lphi, ND - 2);
}

/* D-array of (1 + c1 Lap + c2 Lap^2) psi  (out)  and of Lap of it (Lout). */
static void faxen_psi(const gens_t *g, double c1, double c2, double *out, double *Lout)
{
    for (int k = 0; k < ND; k++) {
        out[k] = g->psi[k] + c1 * g->Lpsi[k] + c2 * g->L2psi[k];
        Lout[k] = g->Lpsi[k] + c1 * g->L2psi[k] + c2 * g->L3psi[k];
    }
}

/* Faxen operator products as (c1, c2):  (1 + s Lap)(1 + t Lap) = 1 + (s+t) Lap + s t Lap^2. */
typedef struct { double c1, c2; } fx_t;
static fx_t fx(double s, double t) { fx_t f = { s + t, s * t }; return f; }

/* Velocity v_n at separation x from the source multipoles in[12] of particle j,
 * with the Faxen operator products fF (on F), fT (on T), fS (on S), and
 * Laplace factor fQ (on S_tr), all already including the target operator. */
static void velocity(const gens_t *g, const double *x, const double *in,
                     fx_t fF, fx_t fT, fx_t fS, double fQ, double eta, double v[3])
{
    double Y[5][3][3];
    stresslet_basis(Y);
    double S[3][3] = { { 0 } };
    for (int m = 0; m < 5; m++)
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) S[a][b] += in[6 + m] * Y[m][a][b];

    double G[ND], LG[ND];
    double LGs, G2[3][3], LG1[3], G3[3][3][3], Q1[3];
    double Qd[ND];
    const double c8 = 1.0 / (8 * PI * eta), c16 = 1.0 / (16 * PI * eta);
    for (int n = 0; n < 3; n++) v[n] = 0.0;

    /* force: (delta Lap G - d d G) F */
    faxen_psi(g, fF.c1, fF.c2, G, LG);
    LGs = 3 * G[1] + (x[0] * x[0] + x[1] * x[1] + x[2] * x[2]) * G[2];   /* Lap G itself */
    tens2(G, x, G2);
    for (int n = 0; n < 3; n++)
        for (int b = 0; b < 3; b++) v[n] += c8 * (dl(n, b) * LGs - G2[n][b]) * in[b];

    /* torque: 1/2 eps_ngb d_g Lap G T_b */
    faxen_psi(g, fT.c1, fT.c2, G, LG);
    tens1(LG, x, LG1);
    for (int n = 0; n < 3; n++)
        for (int gg = 0; gg < 3; gg++)
            for (int b = 0; b < 3; b++) v[n] += c8 * 0.5 * eps3(n, gg, b) * LG1[gg] * in[3 + b];

    /* stresslet: -(delta_nb d_g Lap G - d_n d_b d_g G) S_bg */
    faxen_psi(g, fS.c1, fS.c2, G, LG);
    tens1(LG, x, LG1);
    tens3(G, x, G3);
    for (int n = 0; n < 3; n++)
        for (int b = 0; b < 3; b++)
            for (int gg = 0; gg < 3; gg++)
                v[n] -= c8 * (dl(n, b) * LG1[gg] - G3[n][b][gg]) * S[b][gg];

    /* source: Q S_tr = -grad((1 + fQ Lap) phi)/(16 pi eta) S_tr */
    for (int k = 0; k < ND; k++) Qd[k] = g->phi[k] + fQ * g->Lphi[k];
    tens1(Qd, x, Q1);
    for (int n = 0; n < 3; n++) v[n] -= c16 * Q1[n] * in[11];
}

/* Velocity gradient gv[mu][n] = d_mu v_n, same arguments as velocity(). */
static void velocity_grad(const gens_t *g, const double *x, const double *in,
                          fx_t fF, fx_t fT, fx_t fS, double fQ, double eta, double gv[3][3])
{
    double Y[5][3][3];
    stresslet_basis(Y);
    double S[3][3] = { { 0 } };
    for (int m = 0; m < 5; m++)
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) S[a][b] += in[6 + m] * Y[m][a][b];

    double G[ND], LG[ND], Qd[ND];
    double LG1[3], LG2[3][3], G3[3][3][3], G4[3][3][3][3], Q2[3][3];
    const double c8 = 1.0 / (8 * PI * eta), c16 = 1.0 / (16 * PI * eta);
    memset(gv, 0, sizeof(double) * 9);

    faxen_psi(g, fF.c1, fF.c2, G, LG);
    tens1(LG, x, LG1);
    tens3(G, x, G3);
    for (int mu = 0; mu < 3; mu++)
        for (int n = 0; n < 3; n++)
            for (int b = 0; b < 3; b++) gv[mu][n] += c8 * (dl(n, b) * LG1[mu] - G3[mu][n][b]) * in[b];

    faxen_psi(g, fT.c1, fT.c2, G, LG);
    tens2(LG, x, LG2);
    for (int mu = 0; mu < 3; mu++)
        for (int n = 0; n < 3; n++)
            for (int gg = 0; gg < 3; gg++)
                for (int b = 0; b < 3; b++)
                    gv[mu][n] += c8 * 0.5 * eps3(n, gg, b) * LG2[mu][gg] * in[3 + b];

    faxen_psi(g, fS.c1, fS.c2, G, LG);
    tens2(LG, x, LG2);
    tens4(G, x, G4);
    for (int mu = 0; mu < 3; mu++)
        for (int n = 0; n < 3; n++)
            for (int b = 0; b < 3; b++)
                for (int gg = 0; gg < 3; gg++)
                    gv[mu][n] -= c8 * (dl(n, b) * LG2[mu][gg] - G4[mu][n][b][gg]) * S[b][gg];

    for (int k = 0; k < ND; k++) Qd[k] = g->phi[k] + fQ * g->Lphi[k];
    tens2(Qd, x, Q2);
    for (int mu = 0; mu < 3; mu++)
        for (int n = 0; n < 3; n++) gv[mu][n] -= c16 * Q2[mu][n] * in[11];
}

/* Adds to out[12] the contribution of source multipoles in[12] (radius aj)
 * to target (radius ai) at separation x = r_i - r_j, for generators g. */
static void pair_apply(const gens_t *g, const double *x, double ai, double aj,
                       const double *in, double eta, double *out)
{
    double Y[5][3][3];
    stresslet_basis(Y);
    const double ai2 = ai * ai, aj2 = aj * aj;
    double v[3], gv[3][3];

    /* U = (1 + ai^2 Lap/6) v */
    velocity(g, x, in, fx(ai2 / 6, aj2 / 6), fx(ai2 / 6, 0), fx(ai2 / 6, aj2 / 10), ai2 / 6, eta, v);
    for (int a = 0; a < 3; a++) out[a] += v[a];

    /* Omega = 1/2 curl v */
    velocity_grad(g, x, in, fx(0, aj2 / 6), fx(0, 0), fx(0, aj2 / 10), 0.0, eta, gv);
    for (int a = 0; a < 3; a++)
        for (int mu = 0; mu < 3; mu++)
            for (int n = 0; n < 3; n++) out[3 + a] += 0.5 * eps3(a, mu, n) * gv[mu][n];

    /* E = (1 + ai^2 Lap/10) sym grad v, projected on Y^m */
    velocity_grad(g, x, in, fx(ai2 / 10, aj2 / 6), fx(ai2 / 10, 0), fx(ai2 / 10, aj2 / 10), ai2 / 10, eta, gv);
    for (int m = 0; m < 5; m++)
        for (int mu = 0; mu < 3; mu++)
            for (int n = 0; n < 3; n++) out[6 + m] += Y[m][mu][n] * gv[mu][n];

    /* E_tr = 3/(4 eta) p,  p = 1/(4 pi) [ -d_b phi F_b + d_b d_g phi S_bg ] */
    {
        double P1[3], P2[3][3];
        tens1(g->phi, x, P1);
        tens2(g->phi, x, P2);
        double p = 0.0;
        for (int b = 0; b < 3; b++) p -= P1[b] * in[b];
        for (int m = 0; m < 5; m++)
            for (int b = 0; b < 3; b++)
                for (int gg = 0; gg < 3; gg++) p += P2[b][gg] * Y[m][b][gg] * in[6 + m];
        out[11] += 3.0 / (4.0 * eta) * p / (4 * PI);
    }
}

/* Isolated-sphere self mobilities (Eqs. faxen-f, faxen-t, faxen-s, faxen-p). */
static void isolated_self(double a, const double *in, double eta, double *out)
{
    for (int c = 0; c < 3; c++) out[c] += in[c] / (6 * PI * eta * a);
    for (int c = 0; c < 3; c++) out[3 + c] += in[3 + c] / (8 * PI * eta * a * a * a);
    for (int c = 0; c < 5; c++) out[6 + c] += in[6 + c] * 3.0 / (20 * PI * eta * a * a * a);
    out[11] += in[11] * 3.0 / (16 * PI * eta * a * a * a);
}

/* ---------------- wave space ---------------- */

typedef struct { double re, im; } cplx;
static inline cplx cmul(cplx a, cplx b) { cplx c = { a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re }; return c; }

/* Number of raw moment structure factors per k:
   F(3), a^2 F(3), T(3), S(5), a^2 S(5), S_tr(1). */
#define NSF 20

/* For one wave vector k (|k|^2 = k2): given the structure factors
 *   sf[c] = sum_j exp(i k.r_j) w_c(j)
 * of the raw source moments, form the velocity symbol  V^(k) (3 complex) and
 * the pressure symbol P^(k) (1 complex), literally from the source operators
 * with d -> -i k, Lap -> -k^2  (source Faxen factors only). */
static void wave_source_symbols(const double *k, double k2, double xi, double V, double eta,
                                const cplx *sf, cplx vh[3], cplx *ph)
{
    double Y[5][3][3];
    stresslet_basis(Y);
    const double e = exp(-k2 / (4 * xi * xi));
    const double psih = -(8 * PI / V) * (1 + k2 / (4 * xi * xi)) * e / (k2 * k2);
    const double phih = (4 * PI / V) * e / k2;
    const double c8 = 1.0 / (8 * PI * eta), c16 = 1.0 / (16 * PI * eta);

    /* effective moments with the source Faxen factors (1 - a^2 k^2/6), (1 - a^2 k^2/10) */
    cplx F[3], T[3], S[3][3];
    for (int a = 0; a < 3; a++) {
        F[a].re = sf[a].re - k2 / 6 * sf[3 + a].re;
        F[a].im = sf[a].im - k2 / 6 * sf[3 + a].im;
        T[a] = sf[6 + a];
    }
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            S[a][b].re = S[a][b].im = 0;
            for (int m = 0; m < 5; m++) {
                S[a][b].re += Y[m][a][b] * (sf[9 + m].re - k2 / 10 * sf[14 + m].re);
                S[a][b].im += Y[m][a][b] * (sf[9 + m].im - k2 / 10 * sf[14 + m].im);
            }
        }
    cplx Str = sf[19];

    for (int n = 0; n < 3; n++) {
        cplx acc = { 0, 0 };
        /* (delta_nb Lap - d_n d_b) psi F_b  ->  (-k^2 delta_nb + k_n k_b) psih F_b */
        for (int b = 0; b < 3; b++) {
            double s = c8 * (-(k2) * dl(n, b) + k[n] * k[b]) * psih;
            acc.re += s * F[b].re; acc.im += s * F[b].im;
        }
        /* 1/2 eps_ngb d_g Lap psi T_b -> 1/2 eps_ngb (-i k_g)(-k^2) psih T_b = i/2 eps k_g k^2 psih T_b */
        for (int gg = 0; gg < 3; gg++)
            for (int b = 0; b < 3; b++) {
                double s = c8 * 0.5 * eps3(n, gg, b) * k[gg] * k2 * psih;
                acc.re += -s * T[b].im; acc.im += s * T[b].re;
            }
        /* -(delta_nb d_g Lap psi - d_n d_b d_g psi) S_bg
           -> -(delta_nb (-i k_g)(-k^2) - (-i)^3 k_n k_b k_g) psih S_bg = -i (k^2 delta_nb k_g - k_n k_b k_g) psih S_bg */
        for (int b = 0; b < 3; b++)
            for (int gg = 0; gg < 3; gg++) {
                double s = -c8 * (k2 * dl(n, b) * k[gg] - k[n] * k[b] * k[gg]) * psih;
                acc.re += -s * S[b][gg].im; acc.im += s * S[b][gg].re;
            }
        /* -grad phi/(16 pi eta) S_tr -> -(-i k_n) phih/(16 pi eta) S_tr = i k_n phih c16 S_tr */
        {
            double s = c16 * k[n] * phih;
            acc.re += -s * Str.im; acc.im += s * Str.re;
        }
        vh[n] = acc;
    }

    /* p = 1/(4 pi)[ -d_b phi F_b + d_b d_g phi S_bg ] with the UNfactored moments
       -> 1/(4 pi)[ i k_b phih F_b - k_b k_g phih S_bg ] */
    {
        cplx acc = { 0, 0 };
        for (int b = 0; b < 3; b++) {
            double s = k[b] * phih / (4 * PI);
            acc.re += -s * sf[b].im; acc.im += s * sf[b].re;
        }
        for (int m = 0; m < 5; m++) {
            double kyk = 0;
            for (int b = 0; b < 3; b++)
                for (int gg = 0; gg < 3; gg++) kyk += k[b] * Y[m][b][gg] * k[gg];
            double s = -kyk * phih / (4 * PI);
            acc.re += s * sf[9 + m].re; acc.im += s * sf[9 + m].im;
        }
        *ph = acc;
    }
}

/* Target operators in wave space applied to exp(-i k.r_i) times the symbols:
 * returns 2 Re[...] (the +/- k pair) added to out[12]. */
static void wave_target_add(const double *k, double k2, double ai, cplx phase,
                            const cplx vh[3], cplx ph, double eta, double *out)
{
    double Y[5][3][3];
    stresslet_basis(Y);
    cplx w[3];
    for (int n = 0; n < 3; n++) w[n] = cmul(phase, vh[n]);
    cplx p = cmul(phase, ph);
    const double f6 = 1 - ai * ai * k2 / 6, f10 = 1 - ai * ai * k2 / 10;
    /* U = (1 - a^2 k^2/6) v */
    for (int a = 0; a < 3; a++) out[a] += 2 * f6 * w[a].re;
    /* Omega = 1/2 eps_amn (-i k_m) v_n ;  Re(-i z) = Im z */
    for (int a = 0; a < 3; a++)
        for (int m = 0; m < 3; m++)
            for (int n = 0; n < 3; n++) out[3 + a] += 2 * 0.5 * eps3(a, m, n) * k[m] * w[n].im;
    /* E_m = (1 - a^2 k^2/10) Y_mn (-i k_m) v_n */
    for (int q = 0; q < 5; q++)
        for (int m = 0; m < 3; m++)
            for (int n = 0; n < 3; n++) out[6 + q] += 2 * f10 * Y[q][m][n] * k[m] * w[n].im;
    /* E_tr = 3/(4 eta) p */
    out[11] += 2 * 3.0 / (4.0 * eta) * p.re;
}

/* ---------------- public entry points ---------------- */

/* Minimum image for the lattice a1 = (L, 0, 0), a2 = (gamma L, L, 0), a3 = (0, 0, L)
 * (a cubic box sheared by the strain gamma in x along y, Sec. 3.2; gamma = 0: the cube):
 * first the multiple of a2 that brings d_y into [-L/2, L/2), then a1 and a3. */
static void minimum_shift(double *d, double L, double gamma)
{
    const double ny = floor(d[1] / L + 0.5);
    d[1] -= ny * L;
    d[0] -= ny * gamma * L;
    d[0] -= L * floor(d[0] / L + 0.5);
    d[2] -= L * floor(d[2] / L + 0.5);
}

/*
 * Periodic grand-mobility product by direct Ewald summation.
 *   N, L          : particles, cubic box side
 *   pos  [N*3]    : positions;  rad [N] : radii
 *   x    [N*12]   : input multipoles (F, T, S(5), S_tr)
 *   rows [nrows]  : target particle indices (all if rows == NULL)
 *   y    [nrows*12] : outputs, for the listed targets in order
 *   xi            : Ewald splitting parameter (result independent of it)
 *   rc            : real-space cutoff (absolute)
 *   kc            : wave-space cutoff on |k| (absolute)
 *   parts         : bit 1 real space, bit 2 wave space, bit 4 self (wave-self removal
 *                   and isolated sphere); 7 = full product
 *   eta           : viscosity
 * Returns 0 on success, negative on bad arguments.
 */
int se_oracle_mobility_sheared(long N, double L, double gamma, const double *pos, const double *rad,
                               const double *x, const long *rows, long nrows, double *y, double xi, double rc,
                               double kc, int parts, double eta);

int se_oracle_mobility(long N, double L, const double *pos, const double *rad, const double *x,
                       const long *rows, long nrows, double *y, double xi, double rc, double kc,
                       int parts, double eta)
{
    return se_oracle_mobility_sheared(N, L, 0.0, pos, rad, x, rows, nrows, y, xi, rc, kc, parts, eta);
}

/*
 * The same on the sheared lattice a1 = (L, 0, 0), a2 = (gamma L, L, 0), a3 = (0, 0, L):
 * real-space images d + p1 a1 + p2 a2 + p3 a3, wave vectors k = (2 pi / L)(q1, q2 - gamma q1, q3)
 * (the reciprocal lattice), cell volume L^3.
 */
int se_oracle_mobility_sheared(long N, double L, double gamma, const double *pos, const double *rad,
                               const double *x, const long *rows, long nrows, double *y, double xi, double rc,
                               double kc, int parts, double eta)
{
    if (N <= 0 || L <= 0 || xi <= 0 || !pos || !rad || !x || !y || !(fabs(gamma) <= 1.0)) return -1;
    if (!rows) nrows = N;
    memset(y, 0, sizeof(double) * nrows * NC);
    const double V = L * L * L;

    /* real space: all images with |x| < rc, excluding (i = j, p = 0) */
    if (parts & 1) {
        int pmax = (int)ceil(rc / L) + 2;
#pragma omp parallel for schedule(dynamic, 1)
        for (long ii = 0; ii < nrows; ii++) {
            long i = rows ? rows[ii] : ii;
            double *out = y + ii * NC;
            double B[ND + 1], dpsi[ND], dphi[ND];
            gens_t g;
            for (long j = 0; j < N; j++) {
                double d0[3] = { pos[3 * i] - pos[3 * j], pos[3 * i + 1] - pos[3 * j + 1], pos[3 * i + 2] - pos[3 * j + 2] };
                minimum_shift(d0, L, gamma);
                for (int px = -pmax; px <= pmax; px++)
                    for (int py = -pmax; py <= pmax; py++)
                        for (int pz = -pmax; pz <= pmax; pz++) {
                            double d[3] = { d0[0] + px * L + py * gamma * L, d0[1] + py * L, d0[2] + pz * L };
                            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                            if (r2 >= rc * rc) continue;
                            if (i == j && px == 0 && py == 0 && pz == 0) continue;
                            double r = sqrt(r2);
                            ewald_B(r, xi, ND, B);
                            dpsi_dphi_from_B(B, dpsi, dphi);
                            make_gens(dpsi, dphi, r2, &g);
                            pair_apply(&g, d, rad[i], rad[j], x + j * NC, eta, out);
                        }
            }
        }
    }

    /* wave space: half space of integer vectors q != 0 with |k| < kc,
     * k = (2 pi / L)(q1, q2 - gamma q1, q3) */
    if (parts & 2) {
        int qmax = (int)floor(kc * L / (2 * PI));
        int qmy = qmax + (int)ceil(fabs(gamma) * qmax);
        int ncol = (2 * qmax + 1) * (2 * qmy + 1);
        int nthreads = 1;
#ifdef _OPENMP
        nthreads = omp_get_max_threads();
#endif
        double *acc = (double *)calloc((size_t)nthreads * nrows * NC, sizeof(double));
        if (!acc) return -2;
#pragma omp parallel
        {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            double *myacc = acc + (size_t)tid * nrows * NC;
            cplx *sf = (cplx *)malloc(sizeof(cplx) * (size_t)(qmax + 1) * NSF);
#pragma omp for schedule(dynamic, 1)
            for (int col = 0; col < ncol; col++) {
                int qx = col % (2 * qmax + 1) - qmax, qy = col / (2 * qmax + 1) - qmy;
                const double ky_q = qy - gamma * qx;       /* k_y L / (2 pi) */
                double kxy2 = (2 * PI / L) * (2 * PI / L) * ((double)(qx * qx) + ky_q * ky_q);
                if (kxy2 >= kc * kc) continue;
                int qz0 = (qy > 0 || (qy == 0 && qx > 0)) ? 0 : 1;
                int qz1 = (int)floor(sqrt(fmax(0.0, kc * kc - kxy2)) * L / (2 * PI));
                while (qz1 >= 0 && kxy2 + pow(2 * PI * qz1 / L, 2) >= kc * kc) qz1--;
                if (qz1 < qz0) continue;
                int nq = qz1 - qz0 + 1;
                memset(sf, 0, sizeof(cplx) * (size_t)nq * NSF);
                /* structure factors of raw moments, exp(i k.r_j) by recurrence along qz */
                for (long j = 0; j < N; j++) {
                    double th = 2 * PI / L * (qx * pos[3 * j] + ky_q * pos[3 * j + 1] + qz0 * pos[3 * j + 2]);
                    cplx ph = { cos(th), sin(th) };
                    double tz = 2 * PI / L * pos[3 * j + 2];
                    cplx st = { cos(tz), sin(tz) };
                    double a2 = rad[j] * rad[j];
                    const double *xj = x + j * NC;
                    double w[NSF];
                    for (int c = 0; c < 3; c++) { w[c] = xj[c]; w[3 + c] = a2 * xj[c]; w[6 + c] = xj[3 + c]; }
                    for (int m = 0; m < 5; m++) { w[9 + m] = xj[6 + m]; w[14 + m] = a2 * xj[6 + m]; }
                    w[19] = xj[11];
                    for (int iq = 0; iq < nq; iq++) {
                        cplx *s = sf + (size_t)iq * NSF;
                        for (int c = 0; c < NSF; c++) { s[c].re += w[c] * ph.re; s[c].im += w[c] * ph.im; }
                        ph = cmul(ph, st);
                    }
                }
                /* symbols and targets */
                cplx vh[64][3], phh[64];
                for (int iq0 = 0; iq0 < nq; iq0 += 64) {
                    int nb = nq - iq0 < 64 ? nq - iq0 : 64;
                    for (int b = 0; b < nb; b++) {
                        int qz = qz0 + iq0 + b;
                        double k[3] = { 2 * PI * qx / L, 2 * PI * ky_q / L, 2 * PI * qz / L };
                        double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                        wave_source_symbols(k, k2, xi, V, eta, sf + (size_t)(iq0 + b) * NSF, vh[b], &phh[b]);
                    }
                    for (long ii = 0; ii < nrows; ii++) {
                        long i = rows ? rows[ii] : ii;
                        int qz = qz0 + iq0;
                        double th = -2 * PI / L * (qx * pos[3 * i] + ky_q * pos[3 * i + 1] + qz * pos[3 * i + 2]);
                        cplx ph = { cos(th), sin(th) };
                        double tz = -2 * PI / L * pos[3 * i + 2];
                        cplx st = { cos(tz), sin(tz) };
                        for (int b = 0; b < nb; b++) {
                            double k[3] = { 2 * PI * qx / L, 2 * PI * ky_q / L, 2 * PI * (qz + b) / L };
                            double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                            wave_target_add(k, k2, rad[i], ph, vh[b], phh[b], eta, myacc + ii * NC);
                            ph = cmul(ph, st);
                        }
                    }
                }
            }
            free(sf);
        }
        for (int t = 0; t < nthreads; t++)
            for (long c = 0; c < nrows * NC; c++) y[c] += acc[(size_t)t * nrows * NC + c];
        free(acc);
    }

    /* self: isolated sphere minus the self interaction inside the wave sum */
    if (parts & 4) {
        double dpsi[ND], dphi[ND];
        gens_t g;
        dW_at_origin(xi, dpsi, dphi);
        make_gens(dpsi, dphi, 0.0, &g);
        const double zero[3] = { 0, 0, 0 };
        for (long ii = 0; ii < nrows; ii++) {
            long i = rows ? rows[ii] : ii;
            double w[NC] = { 0 };
            pair_apply(&g, zero, rad[i], rad[i], x + i * NC, eta, w);
            for (int c = 0; c < NC; c++) y[ii * NC + c] -= w[c];
            isolated_self(rad[i], x + i * NC, eta, y + ii * NC);
        }
    }
    return 0;
}

/*
 * One pair block (12 x 12, row-major out[r*12 + c]: output r from input c) at
 * separation x = r_i - r_j for radii ai, aj.
 *   kind 0: real-space Ewald part at xi;  kind 1: free space (psi = r, phi = 1/r);
 *   kind 2: the wave-space self remainder at x = 0 (xi), i.e. what is subtracted.
 */
int se_oracle_pair_block(const double *x, double ai, double aj, double xi, int kind, double eta, double *out)
{
    double B[ND + 1], dpsi[ND], dphi[ND];
    gens_t g;
    double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    double r = sqrt(r2);
    if (kind == 0) { if (r <= 0 || xi <= 0) return -1; ewald_B(r, xi, ND, B); dpsi_dphi_from_B(B, dpsi, dphi); }
    else if (kind == 1) { if (r <= 0) return -1; free_B(r, ND, B); dpsi_dphi_from_B(B, dpsi, dphi); }
    else if (kind == 2) { if (xi <= 0) return -1; dW_at_origin(xi, dpsi, dphi); r2 = 0; }
    else return -1;
    make_gens(dpsi, dphi, r2, &g);
    const double zero[3] = { 0, 0, 0 };
    for (int c = 0; c < NC; c++) {
        double in[NC] = { 0 }, o[NC] = { 0 };
        in[c] = 1.0;
        pair_apply(&g, kind == 2 ? zero : x, ai, aj, in, eta, o);
        for (int rr = 0; rr < NC; rr++) out[rr * NC + c] = o[rr];
    }
    return 0;
}

/* The orthonormal stresslet basis, for the test-suite (out[m*9 + a*3 + b]). */
void se_oracle_stresslet_basis(double *out)
{
    double Y[5][3][3];
    stresslet_basis(Y);
    memcpy(out, Y, sizeof(Y));
}

int se_oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
