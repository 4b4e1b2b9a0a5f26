/* ORACLE (test infrastructure only; only tests, the smoke check and the benchmark's CPU-baseline leg may
 * load it). A plain sequential CPU restatement of one UGKWP-LTS steady-iteration step, checked against
 * the paper's fixed points by the `-m "not gpu"` tests. It shares no code with the CUDA library.
 *
 * Paper sections cited: Sec. II (kinetic model, Eqs. 1-8), Sec. III (UGKWP, Eqs. 9-32), Sec. III C (algorithm
 * steps 1-4), Sec. IV (LTS: Eqs. 33-34 time steps; Eq. 41 proportional scaling; Eqs. 47-53 LTS form).
 *
 * Readings of points the paper leaves open (each is a reading, not a statement of the paper):
 *  - units rho_inf = T_inf = 1, R = 1/2; monatomic, three velocity components, D = 0;
 *  - mu_inf from Kn by the VHS mean-free-path relation; mu = mu_inf T^omega; tau = mu / p (Sec. II);
 *  - tau_i from the total W^n_i at the start of the step;
 *  - reconstruction is first order (piecewise constant) by default: the initial distribution has no slope;
 *    the equilibrium g_0 has normal slopes a^L = (W_0 - W_L)/d_L on u.n > 0 and a^R = (W_R - W_0)/d_R on
 *    u.n < 0, no tangential slope; A from the compatibility condition with both half slopes (Sec. III A);
 *    order 2 (Eq. 12) reconstructs the face states from limited cell gradients and adds the normal slope
 *    term of g^h, the slopes of g_0 still taken against the cell states;
 *  - Prandtl fix applied to a through d(lambda)/Pr; wave fluxes use the Maxwellian g_0 (Sec. III A);
 *  - wall faces: incoming half from the fluid cell (first order), outgoing half a wall Maxwellian at T_w
 *    whose density zeroes the wave mass flux, or with accommodation alpha < 1 the fraction 1 - alpha
 *    mirrored; far-field / fixed ghosts are virtual cells of the ghost state whose collisionless part
 *    enters as particles (ghost particle sources), so their wave keeps dbar_d - e^{-x};
 *  - the particle w-momentum (and in 1-D the v-momentum) is not part of W;
 *  - unstructured meshes (the paper's, Sec. V): convex cells, faces numbered by first appearance over the
 *    cells and their edges with the first cell as L, a triangle stored as the quadrilateral (v0, v1, v2, v2).
 *
 * Pinned by checks independent of this file (tests/): the wall wave flux by velocity quadrature of its
 * definition (wall_flux), the ghost particle sources by the half-range flux of the ghost Maxwellian
 * (inject_params, inject), the vacuum floor's reset and count (update), the Shakhov weights by the heat flux
 * of Eq. 5 evaluated directly (shakhov_weights). Parity unpinned (the CUDA library is compared with it as
 * written): the limiter constant K = 5 (gradients), a choice the paper does not make.
 */
#include "oracle_internal.h"
#include <stdio.h>
#include <string.h>

static const double OR_PI = 3.14159265358979323846;

void or_set_error(or_ctx* cx, int code, const char* msg)
{
    if (cx->err == OR_OK) {
        cx->err = code;
        snprintf(cx->msg, sizeof cx->msg, "%s", msg);
    }
}

static void* zalloc(size_t n, size_t sz)
{
    void* p = calloc(n ? n : 1, sz);
    return p;
}

static void find_stagnation(or_ctx* cx);

/* ---------------------------------------------------------------- kinetic model helpers (Sec. II) */

/* conservative (rho, rho U, rho V, rho E) of a primitive state; E = |U|^2/2 + (3/2) R T */
static void prim_to_cons(double rho, double U, double V, double T, double W[4])
{
    W[0] = rho;
    W[1] = rho * U;
    W[2] = rho * V;
    W[3] = rho * (0.5 * (U * U + V * V) + 1.5 * OR_R * T);
}

double oracle_mu_inf(double Kn, double omega)
{
    /* VHS: lambda = 2 (5 - 2w)(7 - 2w) / 15 * mu / (rho sqrt(2 pi R T)), solved for mu at rho = T = 1 */
    return (15.0 * sqrt(2.0 * OR_PI * OR_R) * Kn) / (2.0 * (5.0 - 2.0 * omega) * (7.0 - 2.0 * omega));
}

static double tau_of(const or_ctx* cx, const double W[4])
{
    /* primitive variables through r = 1 / rho */
    const double rho = W[0], r = 1.0 / rho, U = W[1] * r, V = W[2] * r;
    const double RT = (W[3] * r - 0.5 * (U * U + V * V)) * (2.0 / 3.0);
    const double T = RT / OR_R;
    const double mu = cx->mu_inf * or_powd(T, cx->omega);
    return mu / (rho * RT);
}

/* the same in float (production precision, cells without a wall face) */
static float tau_of_f32(const or_ctx* cx, const double W[4])
{
    const float rho = (float)W[0], r = 1.0f / rho, U = (float)W[1] * r, V = (float)W[2] * r;
    const float RT = ((float)W[3] * r - 0.5f * (U * U + V * V)) * (2.0f / 3.0f);
    const float T = 2.0f * RT;   /* RT / R, R = 1/2 */
    const float mu = (float)cx->mu_inf * or_expf((float)cx->omega * or_logf(T));
    return mu / (rho * RT);
}

/* ---------------------------------------------- time-integration coefficients (Eq. 16, Eqs. 47-48) */

/* out = (dbar_a, dbar_b, dbar_c, dbar_d, dbar_e, dbar_d - e^{-x}, dbar_e + dt/2 e^{-x}),
 * the coefficients of Eq. 16 evaluated with (dt, tau) and divided by dt (Eq. 48). With x = dt/tau and the
 * entire functions phi1 = (1-e^-x)/x, psi2 = (e^-x - 1 + x)/x^2, psi3 = (x^2/2 - x + 1 - e^-x)/x^3,
 * chi = (phi1 - e^-x)/x, beta = (1 + e^-x - 2 phi1)/x^2, kappa = (chi - e^-x/2)/x:
 *   dbar_a = x psi2, dbar_b = -dt x beta, dbar_c = dt x psi3, dbar_d = phi1, dbar_e = -dt chi,
 *   dbar_d - e^-x = x chi, dbar_e + dt e^-x / 2 = -dt x kappa.
 * Each function is summed from its Taylor series for x < 1 (no cancellation) and from the closed form
 * otherwise. */
static void lts_coeffs(double dt, double tau, double e, double out[7])
{
    const double x = dt / tau;
    double phi1, psi2, psi3, chi, beta, kappa;
    if (x < 1.0) {
        /* term k of each series carries (-x)^k / (k + j)! with a polynomial weight in k */
        phi1 = psi2 = psi3 = chi = beta = kappa = 0.0;
        double pw = 1.0;               /* (-x)^k */
        double f1 = 1.0, f2 = 2.0, f3 = 6.0;   /* (k+1)!, (k+2)!, (k+3)! */
        for (int k = 0; k <= 24; ++k) {
            phi1 += pw / f1;
            psi2 += pw / f2;
            psi3 += pw / f3;
            chi += pw * (double)(k + 1) / f2;
            beta += pw * (double)(k + 1) / f3;
            kappa += pw * (double)((k + 1) * (k + 2)) / (2.0 * f3);
            pw *= -x;
            f1 *= (double)(k + 2);
            f2 *= (double)(k + 3);
            f3 *= (double)(k + 4);
        }
    } else {
        phi1 = (1.0 - e) / x;
        psi2 = (e - 1.0 + x) / (x * x);
        psi3 = (0.5 * x * x - x + 1.0 - e) / (x * x * x);
        chi = (phi1 - e) / x;
        beta = (1.0 + e - 2.0 * phi1) / (x * x);
        kappa = (chi - 0.5 * e) / x;
    }
    out[0] = x * psi2;
    out[1] = -dt * x * beta;
    out[2] = dt * x * psi3;
    out[3] = phi1;
    out[4] = -dt * chi;
    out[5] = x * chi;
    out[6] = -dt * x * kappa;
}

void oracle_coeffs(double dt, double tau, double* out)
{
    lts_coeffs(dt, tau, or_expd(-dt / tau), out);
}

/* ------------------------------------------------------- Maxwellian moments (Sec. III A, Eqs. 17-22) */

typedef struct { double rho, U, V, lam; } or_prim;          /* face frame: U normal, V tangential */
typedef struct { double uf[9], up[9], um[9], v[7], xi2, xi4; } or_mom;

/* W in the face frame -> primitive; lambda = 1 / (2 R T); returns 0 if not physical */
static int frame_prim(const double W[4], or_prim* p)
{
    p->rho = W[0];
    if (!(W[0] > 0.0)) return 0;
    p->U = W[1] / W[0];
    p->V = W[2] / W[0];
    const double e = W[3] / W[0] - 0.5 * (p->U * p->U + p->V * p->V);   /* (3/2) R T */
    if (!(e > 0.0)) return 0;
    p->lam = 0.75 / e;
    return 1;
}

/* <u^k> over all u, over u > 0 and over u < 0, per unit density; <v^k>; <w^2>, <w^4> (w: the
 * out-of-plane component, which enters only through |u|^2 like one internal degree of freedom) */
static void moments(const or_prim* p, or_mom* M)
{
    const double U = p->U, V = p->V, lam = p->lam, th = 0.5 / lam;
    const double ex = or_expd(-lam * U * U) / (2.0 * sqrt(OR_PI * lam));
    M->uf[0] = 1.0;
    M->uf[1] = U;
    M->up[0] = 0.5 * or_erfcd(-sqrt(lam) * U);
    M->up[1] = U * M->up[0] + ex;
    M->um[0] = 0.5 * or_erfcd(sqrt(lam) * U);
    M->um[1] = U * M->um[0] - ex;
    for (int k = 2; k < 9; ++k) {
        M->uf[k] = U * M->uf[k - 1] + (double)(k - 1) * th * M->uf[k - 2];
        M->up[k] = U * M->up[k - 1] + (double)(k - 1) * th * M->up[k - 2];
        M->um[k] = U * M->um[k - 1] + (double)(k - 1) * th * M->um[k - 2];
    }
    M->v[0] = 1.0;
    M->v[1] = V;
    for (int k = 2; k < 7; ++k) M->v[k] = V * M->v[k - 1] + (double)(k - 1) * th * M->v[k - 2];
    M->xi2 = th;
    M->xi4 = 3.0 * th * th;
}

/* <psi u^a v^b w^(2c)> with psi = (1, u, v, (u^2 + v^2 + w^2)/2); Mu selects the u range */
static void psi_mom(const double* Mu, const or_mom* M, int a, int b, int c, double out[4])
{
    const double w0 = c == 0 ? 1.0 : M->xi2, w2 = c == 0 ? M->xi2 : M->xi4;
    out[0] = Mu[a] * M->v[b] * w0;
    out[1] = Mu[a + 1] * M->v[b] * w0;
    out[2] = Mu[a] * M->v[b + 1] * w0;
    out[3] = 0.5 * (Mu[a + 2] * M->v[b] * w0 + Mu[a] * M->v[b + 2] * w0 + Mu[a] * M->v[b] * w2);
}

/* <psi u^a v^b (c0 + c1 u + c2 v + c3 (u^2+v^2+w^2)/2)> */
static void psi_poly_mom(const double* Mu, const or_mom* M, int a, int b, const double cf[4], double out[4])
{
    double t0[4], t1[4], t2[4], t3[4], t4[4], t5[4];
    psi_mom(Mu, M, a, b, 0, t0);
    psi_mom(Mu, M, a + 1, b, 0, t1);
    psi_mom(Mu, M, a, b + 1, 0, t2);
    psi_mom(Mu, M, a + 2, b, 0, t3);
    psi_mom(Mu, M, a, b + 2, 0, t4);
    psi_mom(Mu, M, a, b, 1, t5);
    for (int k = 0; k < 4; ++k)
        out[k] = cf[0] * t0[k] + cf[1] * t1[k] + cf[2] * t2[k] + cf[3] * 0.5 * (t3[k] + t4[k] + t5[k]);
}

/* Solve <psi (a0 + a1 u + a2 v + a3 (u^2+v^2+w^2)/2)> = dw for the Maxwellian p (Eq. 20 / Eq. 22),
 * closed form of the 4 x 4 moment system (three velocity dimensions). */
static void micro_slope(const or_prim* p, const double dw[4], double a[4])
{
    const double U = p->U, V = p->V, lam = p->lam;
    const double R4 = 2.0 * dw[3] - 2.0 * U * dw[1] - 2.0 * V * dw[2] + (U * U + V * V) * dw[0]
                      - (1.5 / lam) * dw[0];
    a[3] = (4.0 * lam * lam / 3.0) * R4;
    a[1] = 2.0 * lam * (dw[1] - U * dw[0]) - a[3] * U;
    a[2] = 2.0 * lam * (dw[2] - V * dw[0]) - a[3] * V;
    a[0] = dw[0] - a[3] * 0.75 / lam - a[1] * U - a[2] * V - a[3] * 0.5 * (U * U + V * V);
}

/* Prandtl correction (Sec. III A): d(lambda)/dx -> d(lambda)/dx / Pr inside a */
static void pr_fix(const or_prim* p, double a[4], double Pr)
{
    if (Pr == 1.0) return;
    const double U = p->U, V = p->V, lam = p->lam;
    const double dlam = -0.5 * a[3];
    const double dU = (a[1] + U * a[3]) / (2.0 * lam), dV = (a[2] + V * a[3]) / (2.0 * lam);
    const double drho = a[0] - 1.5 * dlam / lam + dlam * (U * U + V * V) + 2.0 * lam * (U * dU + V * dV);
    const double dl = dlam / Pr;
    a[3] = -2.0 * dl;
    a[1] = 2.0 * lam * dU + 2.0 * U * dl;
    a[2] = 2.0 * lam * dV + 2.0 * V * dl;
    a[0] = drho + 1.5 * dl / lam - dl * (U * U + V * V) - 2.0 * lam * (U * dU + V * dV);
}

/* Time-averaged wave flux through one face in the face frame (normal from L to R):
 * equilibrium part (Eq. 49) from g_0 and its slopes, plus the analytic free-transport part of the
 * hydrodynamic wave (Eq. 50). cL/cR are the 7 normalised coefficients of each side; frL/frR the weight of
 * each side's sampled-from part of g^h (dbar_d - e^{-x}, or the full dbar_d where no particles were sampled
 * or without particles), fdL/fdR the weight of its never-sampled remainder (dbar_d). Returns W_0 and the
 * slopes for the pins. */
static void face_flux(const double WL[4], const double WR[4], const double WhL[4], const double WhR[4],
                      double fdL, double fdR, const double cL[7], const double cR[7], double frL, double frR,
                      double dL, double dR, double Pr, const double WLc[4], const double WRc[4],
                      const double dhL[4], const double dhR[4], double csL, double csR, double F[4],
                      double W0o[4], double aLo[4], double aRo[4], double Ao[4])
{
    /* WL, WR: the states at the face (the cell states in first order); WLc, WRc: the cell states the
     * normal slopes of g_0 are taken against (S7), NULL for WL, WR */
    if (!WLc) WLc = WL;
    if (!WRc) WRc = WR;
    or_prim pL, pR, p0;
    or_mom mL, mR, m0;
    frame_prim(WL, &pL);
    frame_prim(WR, &pR);
    moments(&pL, &mL);
    moments(&pR, &mR);
    double t1[4], t2[4], W0[4];
    psi_mom(mL.up, &mL, 0, 0, 0, t1);
    psi_mom(mR.um, &mR, 0, 0, 0, t2);
    for (int k = 0; k < 4; ++k) W0[k] = pL.rho * t1[k] + pR.rho * t2[k];      /* Eq. 17 */
    for (int k = 0; k < 4; ++k) F[k] = 0.0;
    if (!frame_prim(W0, &p0)) {
        /* vacuum interface (reading): no molecule of either side reaches the face (the half-range masses
         * underflow), so there is no equilibrium state and no equilibrium flux */
        goto free_transport;
    }
    moments(&p0, &m0);
    double dwL[4], dwR[4], aL[4], aR[4], dA[4], A[4];
    for (int k = 0; k < 4; ++k) {
        dwL[k] = (W0[k] - WLc[k]) / (dL * p0.rho);
        dwR[k] = (WRc[k] - W0[k]) / (dR * p0.rho);
    }
    micro_slope(&p0, dwL, aL);
    micro_slope(&p0, dwR, aR);
    pr_fix(&p0, aL, Pr);
    pr_fix(&p0, aR, Pr);
    psi_poly_mom(m0.up, &m0, 1, 0, aL, t1);
    psi_poly_mom(m0.um, &m0, 1, 0, aR, t2);
    for (int k = 0; k < 4; ++k) dA[k] = -(t1[k] + t2[k]);                    /* Eq. 22 */
    micro_slope(&p0, dA, A);
    double fa_p[4], fa_m[4], fb_p[4], fb_m[4], fc_p[4], fc_m[4];
    psi_mom(m0.up, &m0, 1, 0, 0, fa_p);
    psi_mom(m0.um, &m0, 1, 0, 0, fa_m);
    psi_poly_mom(m0.up, &m0, 2, 0, aL, fb_p);
    psi_poly_mom(m0.um, &m0, 2, 0, aR, fb_m);
    psi_poly_mom(m0.up, &m0, 1, 0, A, fc_p);
    psi_poly_mom(m0.um, &m0, 1, 0, A, fc_m);
    for (int k = 0; k < 4; ++k)
        F[k] = p0.rho * (cL[0] * fa_p[k] + cL[1] * fb_p[k] + cL[2] * fc_p[k]
                         + cR[0] * fa_m[k] + cR[1] * fb_m[k] + cR[2] * fc_m[k]);
    if (W0o) for (int k = 0; k < 4; ++k) W0o[k] = W0[k];
    if (aLo) for (int k = 0; k < 4; ++k) aLo[k] = aL[k];
    if (aRo) for (int k = 0; k < 4; ++k) aRo[k] = aR[k];
    if (Ao) for (int k = 0; k < 4; ++k) Ao[k] = A[k];
free_transport:
    /* free transport of the hydrodynamic wave (Eq. 50), reading of Sec. III B: the wave W^h of a side is the
     * local (equilibrium) distribution of the side's total state, carrying the hydrodynamic density rho^h,
     * plus the remainder dW = W^h - (rho^h / rho) W, which has no mass, represented to first order about the
     * same Maxwellian, g (a . psi) with <psi g (a . psi)> = dW (Eq. 20 form). The first part is what the new
     * particles are sampled from (e^{-x} of it, Eq. 26), so its free-transport weight is frL / frR (dbar_d -
     * e^{-x} when particles were sampled, else dbar_d); the remainder is never sampled and keeps the whole
     * dbar_d (fdL / fdR). Both parts are linear in W^h, so particle noise in W^h = W - W^p leaves no bias.
     * Order 2 (Eq. 12): the normal slope term of W^h (dhL, dhR, NULL for none) about the same Maxwellian,
     * weighted with csL / csR. */
    {
        double dw[4], a[4];
        psi_mom(mL.up, &mL, 1, 0, 0, t1);
        for (int k = 0; k < 4; ++k) {
            F[k] += frL * WhL[0] * t1[k];
            dw[k] = (WhL[k] - (WhL[0] / pL.rho) * WL[k]) / pL.rho;
        }
        micro_slope(&pL, dw, a);
        psi_poly_mom(mL.up, &mL, 1, 0, a, t1);
        for (int k = 0; k < 4; ++k) F[k] += fdL * pL.rho * t1[k];
        if (dhL) {
            for (int k = 0; k < 4; ++k) dw[k] = dhL[k] / pL.rho;
            micro_slope(&pL, dw, a);
            psi_poly_mom(mL.up, &mL, 2, 0, a, t1);
            for (int k = 0; k < 4; ++k) F[k] += csL * pL.rho * t1[k];
        }
        psi_mom(mR.um, &mR, 1, 0, 0, t2);
        for (int k = 0; k < 4; ++k) {
            F[k] += frR * WhR[0] * t2[k];
            dw[k] = (WhR[k] - (WhR[0] / pR.rho) * WR[k]) / pR.rho;
        }
        micro_slope(&pR, dw, a);
        psi_poly_mom(mR.um, &mR, 1, 0, a, t2);
        for (int k = 0; k < 4; ++k) F[k] += fdR * pR.rho * t2[k];
        if (dhR) {
            for (int k = 0; k < 4; ++k) dw[k] = dhR[k] / pR.rho;
            micro_slope(&pR, dw, a);
            psi_poly_mom(mR.um, &mR, 2, 0, a, t2);
            for (int k = 0; k < 4; ++k) F[k] += csR * pR.rho * t2[k];
        }
    }
}

void oracle_face_flux_test(const double* WL, const double* WR, const double* WhL, const double* WhR,
                           const double* cL, const double* cR, double dL, double dR, double Pr,
                           double* F, double* W0, double* aL, double* aR, double* A)
{
    face_flux(WL, WR, WhL ? WhL : WL, WhR ? WhR : WR, WhL ? cL[3] : 0.0, WhR ? cR[3] : 0.0, cL, cR,
              WhL ? cL[5] : 0.0, WhR ? cR[5] : 0.0, dL, dR, Pr, NULL, NULL, NULL, NULL, 0.0, 0.0, F, W0, aL, aR, A);
}

/* diffuse isothermal wall (reading): incoming half of the fluid cell's g and its hydrodynamic wave (as in
 * face_flux: rho^h times the cell's local distribution with weight frL, the massless remainder with fdL),
 * outgoing wall Maxwellian at T_w with the density that makes the wave mass flux zero */
static void wall_flux(const or_ctx* cx, const double WL[4], const double WhL[4], double fdL, const double cL[7],
                      double frL, double F[4])
{
    or_prim pL, pw;
    or_mom mL, mw;
    double t[4], o[4], dw[4], sl[4];
    frame_prim(WL, &pL);
    moments(&pL, &mL);
    psi_mom(mL.up, &mL, 1, 0, 0, t);
    for (int k = 0; k < 4; ++k) {
        F[k] = cL[0] * pL.rho * t[k];
        F[k] += frL * WhL[0] * t[k];
        dw[k] = (WhL[k] - (WhL[0] / pL.rho) * WL[k]) / pL.rho;
    }
    micro_slope(&pL, dw, sl);
    psi_poly_mom(mL.up, &mL, 1, 0, sl, t);
    for (int k = 0; k < 4; ++k) F[k] += fdL * pL.rho * t[k];
    pw.rho = 1.0; pw.U = 0.0; pw.V = 0.0; pw.lam = 0.5 / (OR_R * cx->Tw);
    moments(&pw, &mw);
    psi_mom(mw.um, &mw, 1, 0, 0, o);
    const double rw = -F[0] / o[0];
    if (cx->ws == 0.0) {
        for (int k = 0; k < 4; ++k) F[k] += rw * o[k];
        return;
    }
    /* Maxwell wall (reading, §8f f3): the fraction ws of the incoming half is reflected specularly (u_n -> -u_n:
     * in the face frame the mass, tangential momentum and energy fluxes change sign, the normal momentum flux
     * keeps it), the rest re-emitted diffusely at T_w with zero net mass */
    const double sg[4] = {-1.0, 1.0, -1.0, -1.0}, a = 1.0 - cx->ws;
    for (int k = 0; k < 4; ++k) F[k] = (F[k] + cx->ws * (sg[k] * F[k])) + a * (rw * o[k]);
}

/* exported for the quadrature pin of the wall flux (face frame: normal from the fluid cell into the wall) */
void oracle_wall_flux_test(double Tw, double ws, const double* WL, const double* WhL, const double* cL, double frL,
                           double* F)
{
    static or_ctx cx;   /* only Tw and ws are read */
    cx.Tw = Tw;
    cx.ws = ws;
    wall_flux(&cx, WL, WhL ? WhL : WL, WhL ? cL[3] : 0.0, cL, WhL ? frL : 0.0, F);
}

static void to_frame(const double W[4], double nx, double ny, double out[4])
{
    out[0] = W[0];
    out[1] = W[1] * nx + W[2] * ny;
    out[2] = -W[1] * ny + W[2] * nx;
    out[3] = W[3];
}

/* ------------------------------------------------------------------------------- set-up (a0) */

static int boundary_lists(or_ctx* cx);

static int build_geometry(or_ctx* cx, const oracle_mesh* m)
{
    const int ni = m->ni, nj = m->nj, C = ni * nj;
    cx->ni = ni; cx->nj = nj; cx->C = C; cx->dim = m->dim; cx->periodic_j = m->periodic_j;
    int periodic_i = m->dim == 1 && m->bc_imin[0] == OR_BC_PERIODIC;
    if (m->dim == 1) {
        if (nj != 1) return OR_EINVAL;
        if ((m->bc_imin[0] == OR_BC_PERIODIC) != (m->bc_imax[0] == OR_BC_PERIODIC)) return OR_EINVAL;
        cx->F = periodic_i ? ni : ni + 1;
    } else {
        cx->F = (ni + 1) * nj + ni * (m->periodic_j ? nj : nj + 1);
    }
    const int F = cx->F;
    cx->vol = zalloc(C, 8); cx->inv_vol = zalloc(C, 8); cx->xc = zalloc(C, 8); cx->yc = zalloc(C, 8);
    cx->nfc = zalloc(C, 4);
    cx->cface = zalloc(4 * C, 4); cx->csgn = zalloc(4 * C, 4); cx->cnbr = zalloc(4 * C, 4);
    cx->cnk = zalloc(4 * C, 4); cx->cbc = zalloc(4 * C, 4);
    cx->cnx = zalloc(4 * C, 8); cx->cny = zalloc(4 * C, 8); cx->cd = zalloc(4 * C, 8);
    cx->cshift = zalloc(4 * C, 8); cx->cvx = zalloc(4 * C, 8); cx->cvy = zalloc(4 * C, 8);
    cx->xl = zalloc(C, 8); cx->xr = zalloc(C, 8);
    cx->fL = zalloc(F, 4); cx->fR = zalloc(F, 4); cx->fbc = zalloc(F, 4); cx->fwall = zalloc(F, 4);
    cx->fnx = zalloc(F, 8); cx->fny = zalloc(F, 8); cx->fs = zalloc(F, 8); cx->fdL = zalloc(F, 8);
    cx->fdR = zalloc(F, 8); cx->finv_s = zalloc(F, 8);
    cx->fax = zalloc(F, 8); cx->fay = zalloc(F, 8); cx->fex = zalloc(F, 8); cx->fey = zalloc(F, 8);
    double* fd = zalloc(F, 8);
    if (m->dim == 1) {
        const double* xs = m->xv;
        for (int i = 0; i < ni; ++i) {
            cx->xl[i] = xs[i];
            cx->xr[i] = xs[i + 1];
            cx->vol[i] = xs[i + 1] - xs[i];
            cx->xc[i] = 0.5 * (xs[i] + xs[i + 1]);
            cx->nfc[i] = 2;
        }
        for (int f = 0; f < F; ++f) {
            cx->fnx[f] = 1.0; cx->fny[f] = 0.0; cx->fs[f] = 1.0;
            cx->fax[f] = xs[f];
            if (f == 0 && periodic_i) {
                cx->fL[f] = ni - 1; cx->fR[f] = 0; cx->fbc[f] = OR_BC_PERIODIC;
                cx->fdL[f] = xs[ni] - cx->xc[ni - 1]; cx->fdR[f] = cx->xc[0] - xs[0];
            } else if (f == 0) {
                cx->fL[f] = 0; cx->fR[f] = -1; cx->fbc[f] = m->bc_imin[0]; cx->fnx[f] = -1.0;
                cx->fdL[f] = cx->fdR[f] = cx->xc[0] - xs[0];
            } else if (f == ni) {
                cx->fL[f] = ni - 1; cx->fR[f] = -1; cx->fbc[f] = m->bc_imax[0];
                cx->fdL[f] = cx->fdR[f] = xs[ni] - cx->xc[ni - 1];
            } else {
                cx->fL[f] = f - 1; cx->fR[f] = f; cx->fbc[f] = 0;
                cx->fdL[f] = xs[f] - cx->xc[f - 1]; cx->fdR[f] = cx->xc[f] - xs[f];
            }
        }
        for (int i = 0; i < ni; ++i) {
            /* local face 0: left end (outward -x), local face 1: right end (outward +x) */
            const int fl = (i == 0 && periodic_i) ? 0 : i;
            const int fr = (i == ni - 1 && periodic_i) ? 0 : i + 1;
            const int q0 = 4 * i, q1 = 4 * i + 1;
            cx->cface[q0] = fl; cx->cface[q1] = fr;
            cx->cnx[q0] = -1.0; cx->cny[q0] = 0.0; cx->cd[q0] = -xs[i];
            cx->cnx[q1] = 1.0; cx->cny[q1] = 0.0; cx->cd[q1] = xs[i + 1];
            /* left face */
            if (i > 0) { cx->cnbr[q0] = i - 1; cx->cnk[q0] = 1; cx->csgn[q0] = -1; cx->cbc[q0] = 0; }
            else if (periodic_i) {
                cx->cnbr[q0] = ni - 1; cx->cnk[q0] = 1; cx->csgn[q0] = -1; cx->cbc[q0] = OR_BC_PERIODIC;
                cx->cshift[q0] = xs[ni] - xs[0];
            } else { cx->cnbr[q0] = -1; cx->cnk[q0] = -1; cx->csgn[q0] = 1; cx->cbc[q0] = m->bc_imin[0]; }
            /* right face */
            if (i < ni - 1) { cx->cnbr[q1] = i + 1; cx->cnk[q1] = 0; cx->csgn[q1] = 1; cx->cbc[q1] = 0; }
            else if (periodic_i) {
                cx->cnbr[q1] = 0; cx->cnk[q1] = 0; cx->csgn[q1] = 1; cx->cbc[q1] = OR_BC_PERIODIC;
                cx->cshift[q1] = xs[0] - xs[ni];
            } else { cx->cnbr[q1] = -1; cx->cnk[q1] = -1; cx->csgn[q1] = 1; cx->cbc[q1] = m->bc_imax[0]; }
        }
    } else {
        const int nvi = ni + 1;
#define VID(i, j) ((i) + nvi * ((m->periodic_j && (j) == nj) ? 0 : (j)))
        const int njf = m->periodic_j ? nj : nj + 1;
        const int joff = (ni + 1) * nj;
        /* i-faces: from vertex (i, j) to (i, j+1), normal toward +i */
        for (int j = 0; j < nj; ++j) {
            for (int i = 0; i <= ni; ++i) {
                const int f = i + (ni + 1) * j;
                const int a = VID(i, j), b = VID(i, j + 1);
                const double ex = m->xv[b] - m->xv[a], ey = m->yv[b] - m->yv[a];
                cx->fax[f] = m->xv[a]; cx->fay[f] = m->yv[a]; cx->fex[f] = ex; cx->fey[f] = ey;
                const double len = sqrt(ex * ex + ey * ey);
                double nx = ey / len, ny = -ex / len;
                cx->fs[f] = len;
                if (i == 0) {
                    nx = -nx; ny = -ny;
                    cx->fL[f] = i + ni * j; cx->fR[f] = -1; cx->fbc[f] = m->bc_imin[j];
                } else if (i == ni) {
                    cx->fL[f] = (i - 1) + ni * j; cx->fR[f] = -1; cx->fbc[f] = m->bc_imax[j];
                } else {
                    cx->fL[f] = (i - 1) + ni * j; cx->fR[f] = i + ni * j; cx->fbc[f] = 0;
                }
                cx->fnx[f] = nx; cx->fny[f] = ny;
                fd[f] = nx * m->xv[a] + ny * m->yv[a];
            }
        }
        /* j-faces: from vertex (i, j) to (i+1, j), normal toward +j */
        for (int j = 0; j < njf; ++j) {
            for (int i = 0; i < ni; ++i) {
                const int f = joff + i + ni * j;
                const int a = VID(i, j), b = VID(i + 1, j);
                const double ex = m->xv[b] - m->xv[a], ey = m->yv[b] - m->yv[a];
                cx->fax[f] = m->xv[a]; cx->fay[f] = m->yv[a]; cx->fex[f] = ex; cx->fey[f] = ey;
                const double len = sqrt(ex * ex + ey * ey);
                double nx = -ey / len, ny = ex / len;
                cx->fs[f] = len;
                if (m->periodic_j) {
                    cx->fL[f] = i + ni * ((j + nj - 1) % nj); cx->fR[f] = i + ni * j; cx->fbc[f] = 0;
                } else if (j == 0) {
                    nx = -nx; ny = -ny;
                    cx->fL[f] = i; cx->fR[f] = -1; cx->fbc[f] = m->bc_jmin[i];
                } else if (j == nj) {
                    cx->fL[f] = i + ni * (nj - 1); cx->fR[f] = -1; cx->fbc[f] = m->bc_jmax[i];
                } else {
                    cx->fL[f] = i + ni * (j - 1); cx->fR[f] = i + ni * j; cx->fbc[f] = 0;
                }
                cx->fnx[f] = nx; cx->fny[f] = ny;
                fd[f] = nx * m->xv[a] + ny * m->yv[a];
            }
        }
        for (int j = 0; j < nj; ++j) {
            for (int i = 0; i < ni; ++i) {
                const int c = i + ni * j;
                const int v[4] = {VID(i, j), VID(i + 1, j), VID(i + 1, j + 1), VID(i, j + 1)};
                double X[4], Y[4];
                for (int q = 0; q < 4; ++q) {
                    X[q] = m->xv[v[q]]; Y[q] = m->yv[v[q]];
                    cx->cvx[4 * c + q] = X[q]; cx->cvy[4 * c + q] = Y[q];
                }
                cx->vol[c] = 0.5 * ((X[2] - X[0]) * (Y[3] - Y[1]) - (X[3] - X[1]) * (Y[2] - Y[0]));
                const double A1 = 0.5 * ((X[1] - X[0]) * (Y[2] - Y[0]) - (X[2] - X[0]) * (Y[1] - Y[0]));
                const double A2 = 0.5 * ((X[2] - X[0]) * (Y[3] - Y[0]) - (X[3] - X[0]) * (Y[2] - Y[0]));
                cx->xc[c] = (A1 * (X[0] + X[1] + X[2]) + A2 * (X[0] + X[2] + X[3])) / (3.0 * (A1 + A2));
                cx->yc[c] = (A1 * (Y[0] + Y[1] + Y[2]) + A2 * (Y[0] + Y[2] + Y[3])) / (3.0 * (A1 + A2));
                cx->nfc[c] = 4;
                const int jm = m->periodic_j ? j : j;
                const int fq[4] = {i + (ni + 1) * j, (i + 1) + (ni + 1) * j, joff + i + ni * jm,
                                   joff + i + ni * ((m->periodic_j && j + 1 == nj) ? 0 : j + 1)};
                for (int k = 0; k < 4; ++k) {
                    const int f = fq[k], q = 4 * c + k;
                    const int isL = cx->fL[f] == c && !(cx->fR[f] == c && (k == 0 || k == 2));
                    cx->cface[q] = f;
                    cx->csgn[q] = isL ? 1 : -1;
                    cx->cnx[q] = isL ? cx->fnx[f] : -cx->fnx[f];
                    cx->cny[q] = isL ? cx->fny[f] : -cx->fny[f];
                    cx->cd[q] = isL ? fd[f] : -fd[f];
                    if (cx->fR[f] < 0) {
                        cx->cnbr[q] = -1; cx->cnk[q] = -1; cx->cbc[q] = cx->fbc[f];
                    } else {
                        cx->cnbr[q] = isL ? cx->fR[f] : cx->fL[f];
                        cx->cbc[q] = 0;
                        /* local index of the same face in the neighbour: -i <-> +i, -j <-> +j */
                        cx->cnk[q] = k ^ 1;
                    }
                }
            }
        }
        for (int f = 0; f < F; ++f) {
            const int L = cx->fL[f], R = cx->fR[f];
            cx->fdL[f] = fd[f] - (cx->fnx[f] * cx->xc[L] + cx->fny[f] * cx->yc[L]);
            cx->fdR[f] = R >= 0 ? (cx->fnx[f] * cx->xc[R] + cx->fny[f] * cx->yc[R]) - fd[f] : cx->fdL[f];
        }
#undef VID
    }
    free(fd);
    return boundary_lists(cx);
}

/* areas, wall numbering and ghost sources of a built geometry (both mesh kinds) */
static int boundary_lists(or_ctx* cx)
{
    const int C = cx->C, F = cx->F;
    for (int c = 0; c < C; ++c) {
        if (!(cx->vol[c] > 0.0)) return OR_EINVAL;
        cx->inv_vol[c] = 1.0 / cx->vol[c];
    }
    cx->nwall = 0;
    for (int f = 0; f < F; ++f) {
        cx->finv_s[f] = 1.0 / cx->fs[f];
        cx->fwall[f] = -1;
        if (cx->fbc[f] == OR_BC_WALL) cx->fwall[f] = cx->nwall++;
    }
    cx->wall_face = zalloc(cx->nwall, 4);
    for (int f = 0; f < F; ++f) if (cx->fwall[f] >= 0) cx->wall_face[cx->fwall[f]] = f;
    /* far-field and fixed faces: ghost particle sources */
    cx->n_inj = 0;
    for (int f = 0; f < F; ++f) if (cx->fbc[f] == OR_BC_FARFIELD || cx->fbc[f] == OR_BC_FIXED) cx->n_inj++;
    const int ni1 = cx->n_inj > 0 ? cx->n_inj : 1;
    cx->inj_face = zalloc(ni1, 4); cx->inj_k = zalloc(ni1, 4); cx->inj_n = zalloc(ni1, 4);
    cx->inj_m = zalloc(ni1, 8); cx->inj_u = zalloc(ni1, 8); cx->inj_v = zalloc(ni1, 8);
    cx->inj_sig = zalloc(ni1, 8); cx->inj_D = zalloc(ni1, 8);
    for (int f = 0, j = 0; f < F; ++f) {
        if (cx->fbc[f] != OR_BC_FARFIELD && cx->fbc[f] != OR_BC_FIXED) continue;
        const int L = cx->fL[f];
        int kk = -1;
        for (int k = 0; k < cx->nfc[L]; ++k) if (cx->cface[4 * L + k] == f) kk = k;
        cx->inj_face[j] = f;
        cx->inj_k[j] = kk;
        j++;
    }
    return OR_OK;
}

/* Unstructured mesh of triangles and convex quadrilaterals (Sec. V: the paper's meshes are unstructured).
 * Local face k of a cell is its edge from vertex k to vertex k + 1 (mod the vertex count). Faces are numbered
 * in order of first appearance, walking the cells in order and each cell's edges in order; the cell that
 * first names an edge is its L side and the edge keeps that cell's direction a -> b, so that the unit normal
 * (e_y, -e_x) / |e| of a counter-clockwise cell points from L to R. A triangle is stored as the degenerate
 * quadrilateral (v0, v1, v2, v2): the area and centroid formulas and the position sampling of the
 * quadrilateral then reduce to the triangle's. */
static int build_geometry_u(or_ctx* cx, const oracle_umesh* m)
{
    const int C = m->n_cells, NV = m->n_vertices;
    cx->ni = C; cx->nj = 1; cx->C = C; cx->dim = 2; cx->periodic_j = 0;
    /* cells: vertex indices in range and distinct, counter-clockwise and strictly convex */
    for (int c = 0; c < C; ++c) {
        const int32_t* v = m->cells + 4 * (size_t)c;
        const int n = v[3] < 0 ? 3 : 4;
        for (int q = 0; q < n; ++q) {
            if (v[q] < 0 || v[q] >= NV) return OR_EINVAL;
            for (int r = 0; r < q; ++r) if (v[r] == v[q]) return OR_EINVAL;
        }
        for (int q = 0; q < n; ++q) {
            const int a = v[q], b = v[(q + 1) % n], e = v[(q + 2) % n];
            const double cr = (m->xv[b] - m->xv[a]) * (m->yv[e] - m->yv[b]) - (m->yv[b] - m->yv[a]) * (m->xv[e] - m->xv[b]);
            if (!(cr > 0.0)) return OR_EINVAL;
        }
    }
    /* faces: an edge list per lower vertex index, searched linearly */
    int* fa = zalloc(4 * (size_t)C + 1, 4);
    int* fb = zalloc(4 * (size_t)C + 1, 4);
    int* fkL = zalloc(4 * (size_t)C + 1, 4);
    int* fkR = zalloc(4 * (size_t)C + 1, 4);
    int* fLt = zalloc(4 * (size_t)C + 1, 4);
    int* fRt = zalloc(4 * (size_t)C + 1, 4);
    int* fbct = zalloc(4 * (size_t)C + 1, 4);
    int* nxt = zalloc(4 * (size_t)C + 1, 4);
    int* head = zalloc(NV > 0 ? NV : 1, 4);
    int* cf = zalloc(4 * (size_t)C, 4);
    int st = OR_OK, F = 0;
    for (int v = 0; v < NV; ++v) head[v] = -1;
    for (int c = 0; c < C && !st; ++c) {
        const int32_t* v = m->cells + 4 * (size_t)c;
        const int n = v[3] < 0 ? 3 : 4;
        for (int k = 0; k < n && !st; ++k) {
            const int a = v[k], b = v[(k + 1) % n];
            const int lo = a < b ? a : b, hi = a < b ? b : a;
            int f = -1;
            for (int g = head[lo]; g >= 0; g = nxt[g])
                if ((fa[g] < fb[g] ? fb[g] : fa[g]) == hi) { f = g; break; }
            if (f < 0) {
                f = F++;
                fa[f] = a; fb[f] = b; fLt[f] = c; fkL[f] = k; fRt[f] = -1; fkR[f] = -1; fbct[f] = 0;
                nxt[f] = head[lo]; head[lo] = f;
            } else if (fRt[f] >= 0 || fa[f] != b) {
                st = OR_EINVAL;   /* an edge of three cells, or two cells that overlap along it */
            } else {
                fRt[f] = c; fkR[f] = k;
            }
            cf[4 * (size_t)c + k] = f;
        }
    }
    /* boundary tags: every edge of one cell gets exactly one */
    for (int e = 0; e < m->n_boundary && !st; ++e) {
        const int a = m->boundary[3 * e], b = m->boundary[3 * e + 1], tag = m->boundary[3 * e + 2];
        if (a < 0 || a >= NV || b < 0 || b >= NV) { st = OR_EINVAL; break; }
        if (tag != OR_BC_WALL && tag != OR_BC_FARFIELD && tag != OR_BC_FIXED && tag != OR_BC_SYMMETRY) { st = OR_EINVAL; break; }
        const int lo = a < b ? a : b, hi = a < b ? b : a;
        int f = -1;
        for (int g = head[lo]; g >= 0; g = nxt[g])
            if ((fa[g] < fb[g] ? fb[g] : fa[g]) == hi) { f = g; break; }
        if (f < 0 || fRt[f] >= 0 || fbct[f] != 0) { st = OR_EINVAL; break; }
        fbct[f] = tag;
    }
    for (int f = 0; f < F && !st; ++f) if (fRt[f] < 0 && fbct[f] == 0) st = OR_EINVAL;
    if (!st) {
        cx->F = F;
        cx->vol = zalloc(C, 8); cx->inv_vol = zalloc(C, 8); cx->xc = zalloc(C, 8); cx->yc = zalloc(C, 8);
        cx->nfc = zalloc(C, 4);
        cx->cface = zalloc(4 * C, 4); cx->csgn = zalloc(4 * C, 4); cx->cnbr = zalloc(4 * C, 4);
        cx->cnk = zalloc(4 * C, 4); cx->cbc = zalloc(4 * C, 4);
        cx->cnx = zalloc(4 * C, 8); cx->cny = zalloc(4 * C, 8); cx->cd = zalloc(4 * C, 8);
        cx->cshift = zalloc(4 * C, 8); cx->cvx = zalloc(4 * C, 8); cx->cvy = zalloc(4 * C, 8);
        cx->xl = zalloc(C, 8); cx->xr = zalloc(C, 8);
        cx->fL = zalloc(F, 4); cx->fR = zalloc(F, 4); cx->fbc = zalloc(F, 4); cx->fwall = zalloc(F, 4);
        cx->fnx = zalloc(F, 8); cx->fny = zalloc(F, 8); cx->fs = zalloc(F, 8); cx->fdL = zalloc(F, 8);
        cx->fdR = zalloc(F, 8); cx->finv_s = zalloc(F, 8);
        cx->fax = zalloc(F, 8); cx->fay = zalloc(F, 8); cx->fex = zalloc(F, 8); cx->fey = zalloc(F, 8);
        double* fd = zalloc(F, 8);
        for (int f = 0; f < F; ++f) {
            const int a = fa[f], b = fb[f];
            const double ex = m->xv[b] - m->xv[a], ey = m->yv[b] - m->yv[a];
            const double len = sqrt(ex * ex + ey * ey);
            cx->fax[f] = m->xv[a]; cx->fay[f] = m->yv[a]; cx->fex[f] = ex; cx->fey[f] = ey;
            cx->fs[f] = len;
            cx->fnx[f] = ey / len; cx->fny[f] = -ex / len;
            cx->fL[f] = fLt[f]; cx->fR[f] = fRt[f]; cx->fbc[f] = fRt[f] < 0 ? fbct[f] : 0;
            fd[f] = cx->fnx[f] * m->xv[a] + cx->fny[f] * m->yv[a];
        }
        for (int c = 0; c < C; ++c) {
            const int32_t* v = m->cells + 4 * (size_t)c;
            const int n = v[3] < 0 ? 3 : 4;
            double X[4], Y[4];
            for (int q = 0; q < 4; ++q) {
                const int vq = q < n ? v[q] : v[2];
                X[q] = m->xv[vq]; Y[q] = m->yv[vq];
                cx->cvx[4 * c + q] = X[q]; cx->cvy[4 * c + q] = Y[q];
            }
            cx->vol[c] = 0.5 * ((X[2] - X[0]) * (Y[3] - Y[1]) - (X[3] - X[1]) * (Y[2] - Y[0]));
            const double A1 = 0.5 * ((X[1] - X[0]) * (Y[2] - Y[0]) - (X[2] - X[0]) * (Y[1] - Y[0]));
            const double A2 = 0.5 * ((X[2] - X[0]) * (Y[3] - Y[0]) - (X[3] - X[0]) * (Y[2] - Y[0]));
            cx->xc[c] = (A1 * (X[0] + X[1] + X[2]) + A2 * (X[0] + X[2] + X[3])) / (3.0 * (A1 + A2));
            cx->yc[c] = (A1 * (Y[0] + Y[1] + Y[2]) + A2 * (Y[0] + Y[2] + Y[3])) / (3.0 * (A1 + A2));
            cx->nfc[c] = n;
            for (int k = 0; k < 4; ++k) {
                const int q = 4 * c + k;
                if (k >= n) { cx->cnbr[q] = -1; cx->cnk[q] = -1; cx->csgn[q] = 1; continue; }
                const int f = cf[q];
                const int isL = fLt[f] == c;
                cx->cface[q] = f;
                cx->csgn[q] = isL ? 1 : -1;
                cx->cnx[q] = isL ? cx->fnx[f] : -cx->fnx[f];
                cx->cny[q] = isL ? cx->fny[f] : -cx->fny[f];
                cx->cd[q] = isL ? fd[f] : -fd[f];
                if (fRt[f] < 0) { cx->cnbr[q] = -1; cx->cnk[q] = -1; cx->cbc[q] = fbct[f]; }
                else { cx->cnbr[q] = isL ? fRt[f] : fLt[f]; cx->cnk[q] = isL ? fkR[f] : fkL[f]; cx->cbc[q] = 0; }
            }
        }
        for (int f = 0; f < F; ++f) {
            const int L = cx->fL[f], R = cx->fR[f];
            cx->fdL[f] = fd[f] - (cx->fnx[f] * cx->xc[L] + cx->fny[f] * cx->yc[L]);
            cx->fdR[f] = R >= 0 ? (cx->fnx[f] * cx->xc[R] + cx->fny[f] * cx->yc[R]) - fd[f] : cx->fdL[f];
        }
        free(fd);
    }
    free(fa); free(fb); free(fkL); free(fkR); free(fLt); free(fRt); free(fbct); free(nxt); free(head); free(cf);
    if (st) return st;
    return boundary_lists(cx);
}

/* mass and remaining-time scaling of a crossing from cell c through its local face k: dt_R / dt_L (Eq. 41) */
static void set_ratios(or_ctx* cx)
{
    for (int c = 0; c < cx->C; ++c)
        for (int k = 0; k < cx->nfc[c]; ++k) {
            const int q = 4 * c + k;
            cx->ratio[q] = cx->cnbr[q] >= 0 ? cx->dt[cx->cnbr[q]] / cx->dt[c] : 1.0;
        }
}

/* local time steps (Eq. 33) from the initial freestream field, then the global one (Eq. 34) */
static void init_time_steps(or_ctx* cx)
{
    const double cs = cx->U_inf + 3.0 * sqrt(OR_R * 1.0);
    cx->dtG = 0.0;
    for (int c = 0; c < cx->C; ++c) {
        double perim = 0.0;
        for (int k = 0; k < cx->nfc[c]; ++k) perim += cx->fs[cx->cface[4 * c + k]];
        cx->dt[c] = (cx->cfl * cx->vol[c]) / (cs * perim);
        if (c == 0 || cx->dt[c] < cx->dtG) cx->dtG = cx->dt[c];
    }
    if (cx->gts)
        for (int c = 0; c < cx->C; ++c) cx->dt[c] = cx->dtG;
    set_ratios(cx);
}

/* ceil(log2(x)) for x > 0, exact through frexp */
static int ceil_log2(double x)
{
    int e;
    const double m = frexp(x, &e);
    return m == 0.5 ? e - 1 : e;
}

/* Fixed-point exponents of the particle tallies (a build choice, not the paper's): a cell may hold up to
 * 1024 times the freestream density in the largest cell, particles move at most U_inf + 10 sqrt(R T_max);
 * each per-cell sum then stays below 2^61. */
static void fixed_exponents(or_ctx* cx, double T_fix)
{
    double vmax = 0.0;
    for (int c = 0; c < cx->C; ++c) if (cx->vol[c] > vmax) vmax = cx->vol[c];
    double Tmax = 1.0;
    if (cx->Tw > Tmax) Tmax = cx->Tw;
    if (T_fix > Tmax) Tmax = T_fix;
    const double speed = cx->U_inf + 10.0 * sqrt(OR_R * Tmax);
    const double b0 = 1024.0 * vmax;
    cx->fx[0] = 61 - ceil_log2(b0);
    cx->fx[1] = 61 - ceil_log2(b0 * speed);
    cx->fx[2] = 61 - ceil_log2(b0 * (0.5 * (speed * speed)));
    cx->fx[3] = 61 - ceil_log2(b0 * (speed * speed));
    cx->fx[4] = 61 - ceil_log2(b0 * (speed * speed * speed));
}

int oracle_fixed_exponents(oracle_ctx* cx, int32_t* out)
{
    out[0] = cx->fx[0]; out[1] = cx->fx[1]; out[2] = cx->fx[2];
    return OR_OK;
}

static int finish_create(or_ctx* cx, const oracle_gas* gas, double Kn, double Ma, double Tw, double cfl,
                         int32_t gts, const oracle_opts* opts, oracle_ctx** out);

int oracle_create(const oracle_mesh* mesh, const oracle_gas* gas, double Kn, double Ma, double Tw,
                  double cfl, int32_t gts, const oracle_opts* opts, oracle_ctx** out)
{
    if (!mesh || !gas || !opts || !out || mesh->ni <= 0 || mesh->nj <= 0) return OR_EINVAL;
    if (mesh->ni * (int64_t)mesh->nj >= (1 << 21)) return OR_EINVAL;
    if (!(gas->wall_specular >= 0.0 && gas->wall_specular <= 1.0)) return OR_EINVAL;
    if (!(opts->emx_cutoff >= 0.0 && opts->emx_cutoff < 1.0)) return OR_EINVAL;
    or_ctx* cx = zalloc(1, sizeof(or_ctx));
    int st = build_geometry(cx, mesh);
    if (st) { oracle_destroy(cx); return st; }
    return finish_create(cx, gas, Kn, Ma, Tw, cfl, gts, opts, out);
}

int oracle_create_unstructured(const oracle_umesh* mesh, const oracle_gas* gas, double Kn, double Ma, double Tw,
                               double cfl, int32_t gts, const oracle_opts* opts, oracle_ctx** out)
{
    if (!mesh || !gas || !opts || !out || mesh->n_cells <= 0 || mesh->n_vertices <= 0 || !mesh->xv || !mesh->yv ||
        !mesh->cells || mesh->n_boundary < 0 || (mesh->n_boundary > 0 && !mesh->boundary))
        return OR_EINVAL;
    if (mesh->n_cells >= (1 << 21)) return OR_EINVAL;
    if (!(gas->wall_specular >= 0.0 && gas->wall_specular <= 1.0)) return OR_EINVAL;
    if (!(opts->emx_cutoff >= 0.0 && opts->emx_cutoff < 1.0)) return OR_EINVAL;
    or_ctx* cx = zalloc(1, sizeof(or_ctx));
    int st = build_geometry_u(cx, mesh);
    if (st) { oracle_destroy(cx); return st; }
    return finish_create(cx, gas, Kn, Ma, Tw, cfl, gts, opts, out);
}

/* everything after the geometry: time steps, bounds, state arrays, the freestream start */
static int finish_create(or_ctx* cx, const oracle_gas* gas, double Kn, double Ma, double Tw, double cfl,
                         int32_t gts, const oracle_opts* opts, oracle_ctx** out)
{
    const int C = cx->C, F = cx->F;
    cx->prec = opts->precision; cx->wave_only = opts->wave_only; cx->record_faces = opts->record_faces;
    cx->order = opts->order == 2 ? 2 : 1;
    cx->emx_cutoff = opts->emx_cutoff;
    cx->gts = gts; cx->n_ref = opts->n_ref; cx->seed = opts->seed; cx->case_id = opts->case_id;
    cx->Kn = Kn; cx->Ma = Ma; cx->Tw = Tw; cx->cfl = cfl; cx->omega = gas->omega; cx->Pr = gas->Pr;
    cx->ws = gas->wall_specular;
    cx->mu_inf = oracle_mu_inf(Kn, gas->omega);
    cx->U_inf = Ma * sqrt((5.0 / 3.0) * OR_R * 1.0);
    cx->m2RTw = -2.0 * OR_R * Tw;
    cx->sig_w = sqrt(OR_R * Tw);
    prim_to_cons(1.0, cx->U_inf, 0.0, 1.0, cx->W_inf);
    prim_to_cons(opts->ghost_state[0], opts->ghost_state[1], opts->ghost_state[2], opts->ghost_state[3], cx->W_fix);
    cx->dt = zalloc(C, 8); cx->ratio = zalloc(4 * C, 8);
    init_time_steps(cx);
    fixed_exponents(cx, opts->ghost_state[3]);
    {
        double Tc = 1.0 + Ma * Ma / 3.0;
        if (Tw > Tc) Tc = Tw;
        if (opts->ghost_state[3] > Tc) Tc = opts->ghost_state[3];
        cx->T_cap = 10.0 * Tc;
        double Tm = 1.0;
        if (Tw < Tm) Tm = Tw;
        if (opts->ghost_state[3] > 0.0 && opts->ghost_state[3] < Tm) Tm = opts->ghost_state[3];
        cx->T_min = 0.01 * Tm;
        cx->U_cap = cx->U_inf + 10.0 * sqrt(OR_R * cx->T_cap);
    }
    cx->W = zalloc(4 * C, 8); cx->wret_prev = zalloc(5 * C, 8);
    cx->tau = zalloc(C, 8); cx->xr_t = zalloc(C, 8); cx->emx = zalloc(C, 8);
    cx->Wp = zalloc(4 * C, 8); cx->Wh = zalloc(4 * C, 8); cx->mnew = zalloc(C, 8); cx->co = zalloc(7 * C, 8);
    cx->samp = zalloc(3 * C, 8); cx->grad = zalloc(16 * (size_t)C, 8);
    cx->whq = zalloc(9 * C, 8); cx->hq = zalloc(3 * C, 8);
    cx->nhp = zalloc(C, 4); cx->nhp_off = zalloc(C + 1, 8);
    cx->wm = zalloc(5 * C, 8); cx->wpl = zalloc(5 * C, 8); cx->wrt = zalloc(5 * C, 8);
    cx->cross = zalloc(2 * F, 8); cx->wallt = zalloc(3 * cx->nwall, 8); cx->frec = zalloc(4 * F, 8);
    cx->flux = zalloc(4 * F, 8);
    cx->chi_ema = zalloc(C, 8);
    cx->surf_sum = zalloc(3 * cx->nwall, 8); cx->surf_last = zalloc(3 * cx->nwall, 8);
    find_stagnation(cx);
    for (int k = 0; k < 8; ++k) cx->mon[k] = NAN;
    cx->cap = 1024;
    cx->p = zalloc(cx->cap, sizeof(or_particle));
    for (int c = 0; c < C; ++c)
        for (int k = 0; k < 4; ++k) cx->W[4 * c + k] = cx->W_inf[k];
    *out = cx;
    return OR_OK;
}

void oracle_destroy(oracle_ctx* cx)
{
    if (!cx) return;
    void* ptrs[] = {cx->vol, cx->inv_vol, cx->xc, cx->yc, cx->nfc, cx->cface, cx->csgn, cx->cnbr, cx->cnk,
                    cx->cbc, cx->cnx, cx->cny, cx->cd, cx->cshift, cx->cvx, cx->cvy, cx->xl, cx->xr, cx->fL,
                    cx->fR, cx->fbc, cx->fwall, cx->fnx, cx->fny, cx->fs, cx->fdL, cx->fdR, cx->finv_s,
                    cx->wall_face, cx->dt, cx->ratio, cx->W, cx->wret_prev, cx->tau, cx->xr_t, cx->emx, cx->Wp,
                    cx->Wh, cx->mnew, cx->co, cx->samp, cx->grad, cx->nhp, cx->nhp_off, cx->wm, cx->wpl,
                    cx->wrt, cx->cross, cx->wallt, cx->frec, cx->flux, cx->chi_ema, cx->surf_sum,
                    cx->surf_last, cx->p, cx->whq, cx->hq, cx->fax, cx->fay, cx->fex, cx->fey,
                    cx->inj_face, cx->inj_k, cx->inj_n, cx->inj_m, cx->inj_u, cx->inj_v, cx->inj_sig,
                    cx->inj_D};
    for (size_t i = 0; i < sizeof ptrs / sizeof ptrs[0]; ++i) free(ptrs[i]);
    free(cx);
}

/* Realizability of a cell state (reading): density above the vacuum floor, temperature between
 * T_min = 0.01 min(1, T_w, T_fix) and T_cap = 10 max(T_0, T_w, T_fix) with T_0 = 1 + Ma^2 / 3 the
 * freestream stagnation temperature, speed at most U_inf + 10 sqrt(R T_cap). States outside arise only
 * from statistical noise in cells that have (nearly) no gas. */
static int realizable(const or_ctx* cx, const double W[4])
{
    if (!(W[0] > OR_RHO_FLOOR)) return 0;
    const double r = 1.0 / W[0];
    const double U = W[1] * r, V = W[2] * r;
    const double q = U * U + V * V;
    const double e = W[3] * r - 0.5 * q;
    if (!(e > 0.0)) return 0;
    const double T = (e * (2.0 / 3.0)) * (1.0 / OR_R);
    return T >= cx->T_min && T <= cx->T_cap && q <= cx->U_cap * cx->U_cap;
}

/* ------------------------------------------------------------------ a1: decomposition (Sec. IV B) */

/* Shakhov acceptance-rejection weights of cell c (Eqs. 4-5; reading): the heat flux Q_i of the particles
 * retained in the cell at the start of the step, about the cell velocity U_i, from their raw moments: the
 * new particles follow the cell's g^S (Eq. 4 at U_i, T_i, Q_i): accept a proposal c = sqrt(RT_i) z from the
 * Maxwellian with probability (1 + psi) / M, psi = (a . z) (|z|^2 - 5), a = (1 - Pr) Q_i / (5 rho_i
 * (RT_i)^(3/2)), M = 1 + 6 * 31 |a| (|z| <= 6 enforced by rejection). W has no z-momentum, so Q_z = 0; in
 * 1-D also Q_y = 0. */
static void shakhov_weights(or_ctx* cx, int c)
{
    const int64_t* h = cx->whq + 9 * c;
    const double s0 = ldexp(1.0, -cx->fx[0]), s1 = ldexp(1.0, -cx->fx[1]), s2 = ldexp(1.0, -cx->fx[3]);
    const double s3 = ldexp(1.0, -cx->fx[4]);
    const double Sm = (double)h[0] * s0, Su = (double)h[1] * s1, Sv = (double)h[2] * s1;
    const double Suu = (double)h[3] * s2, Suv = (double)h[4] * s2, Svv = (double)h[5] * s2, Sq = (double)h[6] * s2;
    const double Suq = (double)h[7] * s3, Svq = (double)h[8] * s3;
    const double* W = cx->W + 4 * c;
    const double U = W[1] / W[0], V = cx->dim == 1 ? 0.0 : W[2] / W[0];
    const double UU = U * U + V * V;
    const double Ud = U * Su + V * Sv;
    /* sum m c_a |c|^2 with c = u - U_i, expanded in the raw moments */
    const double cx3 = ((((Suq - 2.0 * (U * Suu + V * Suv)) + UU * Su) - U * Sq) + 2.0 * U * Ud) - U * UU * Sm;
    const double cy3 = ((((Svq - 2.0 * (U * Suv + V * Svv)) + UU * Sv) - V * Sq) + 2.0 * V * Ud) - V * UU * Sm;
    const double Qx = cx3 / (2.0 * cx->vol[c]);
    const double Qy = cx->dim == 1 ? 0.0 : cy3 / (2.0 * cx->vol[c]);
    const double RTi = cx->samp[3 * c + 2];
    const double den = 5.0 * W[0] * (RTi * sqrt(RTi));
    const double ax = ((1.0 - cx->Pr) * Qx) / den, ay = ((1.0 - cx->Pr) * Qy) / den;
    cx->hq[3 * c] = ax;
    cx->hq[3 * c + 1] = ay;
    cx->hq[3 * c + 2] = 1.0 + 186.0 * sqrt(ax * ax + ay * ay);
}

static void decompose(or_ctx* cx)
{
    const double s0 = ldexp(1.0, -cx->fx[0]), s1 = ldexp(1.0, -cx->fx[1]), s4 = ldexp(1.0, -cx->fx[2]);
    const int shakhov = cx->Pr != 1.0 && !cx->wave_only;
    if (shakhov) {
        memset(cx->whq, 0, 9 * (size_t)cx->C * 8);
        if (cx->prec == 0) or_heat_tally_f32(cx); else or_heat_tally_f64(cx);
    }
    for (int c = 0; c < cx->C; ++c) {
        const double* W = cx->W + 4 * c;
        const int64_t* r = cx->wret_prev + 5 * c;
        double* Wp = cx->Wp + 4 * c;
        double* Wh = cx->Wh + 4 * c;
        /* production precision: tau, x = dt / tau and e^{-x} in float, except in cells with a wall face
         * (stretched, where the wave-flux time integrals need FP64) and at order 2 */
        int wallcell = 0;
        for (int k = 0; k < cx->nfc[c]; ++k) if (cx->cbc[4 * c + k] == OR_BC_WALL) wallcell = 1;
        const int f32 = cx->prec == 0 && !wallcell && cx->order != 2;
        double tau, x, e;
        if (f32) {
            const float t32 = tau_of_f32(cx, W);
            const float x32 = (float)cx->dt[c] / t32;
            tau = t32;
            x = x32;
            e = or_expf(-x32);
        } else {
            tau = tau_of(cx, W);
            x = cx->dt[c] / tau;
            e = or_expd(-x);
        }
        /* W^p from the particles retained at the end of the previous step, the factor 1 / Omega_i of Eq. 30
         * applied to the tally sums; W^h = W - W^p (Eq. 24) */
        Wp[0] = ((double)r[0] * s0) * cx->inv_vol[c];
        Wp[1] = ((double)r[1] * s1) * cx->inv_vol[c];
        Wp[2] = cx->dim == 1 ? 0.0 : ((double)r[2] * s1) * cx->inv_vol[c];
        Wp[3] = ((double)r[4] * s4) * cx->inv_vol[c];
        for (int k = 0; k < 4; ++k) Wh[k] = W[k] - Wp[k];
        cx->tau[c] = tau;
        cx->xr_t[c] = x;
        cx->emx[c] = e;
        lts_coeffs(cx->dt[c], tau, e, cx->co + 7 * c);
        cx->nhp[c] = 0;
        cx->mnew[c] = 0.0;
        cx->samp[3 * c] = cx->samp[3 * c + 1] = cx->samp[3 * c + 2] = 0.0;
        /* W^hp = W^h e^{-dt_i / tau_i}; for rho^hp > 0: N^hp = ceil(rho^hp / rho N_ref), m = rho^hp Omega / N^hp
         * (Eqs. 25-26). Reading of Sec. III B: the new particles' velocities follow the local distribution of
         * the cell, at the cell velocity U_i and temperature T_i (not those of W^h, which is a small difference
         * of noisy tallies where particles dominate); the rest of W^h is transported by the wave (face_flux).
         * Particle cutoff (reading of Sec. V A's cost discussion): a cell with e^{-x} below emx_cutoff samples
         * nothing, and all of its W^h travels with the wave */
        const double rho_hp = Wh[0] * e;
        if (!cx->wave_only && rho_hp > 0.0 && !(e < cx->emx_cutoff)) {
            const double q = ceil((rho_hp / W[0]) * (double)cx->n_ref);
            if (q > (double)OR_MAX_NEW) {
                or_set_error(cx, OR_ELIMIT, "more than 2047 new particles in one cell");
                continue;
            }
            cx->nhp[c] = (int)q;
            cx->mnew[c] = (rho_hp * cx->vol[c]) / q;
            const double rw = 1.0 / W[0], Ui = W[1] * rw, Vi = cx->dim == 1 ? 0.0 : W[2] * rw;
            cx->samp[3 * c] = Ui;
            cx->samp[3 * c + 1] = Vi;
            cx->samp[3 * c + 2] = (W[3] * rw - 0.5 * (Ui * Ui + Vi * Vi)) * (2.0 / 3.0);
            if (shakhov) shakhov_weights(cx, c);
        }
    }
}

/* ---------------------------------------------------------------------------- a9: wave fluxes */

/* Ghost state behind a far-field / fixed face (S19): the fixed state, or the freestream where it flows in
 * (U_inf . n < 0, n outward from the fluid cell), else the fluid cell's own state (zero gradient). */
static void ghost_state(const or_ctx* cx, int f, double Wg[4])
{
    const double* src;
    if (cx->fbc[f] == OR_BC_FIXED) {
        src = cx->W_fix;
    } else {
        const double un_inf = cx->W_inf[1] * cx->fnx[f] + cx->W_inf[2] * cx->fny[f];
        src = un_inf < 0.0 ? cx->W_inf : cx->W + 4 * cx->fL[f];
    }
    for (int k = 0; k < 4; ++k) Wg[k] = src[k];
}

/* Ghost particle sources (reading; the paper is silent on boundaries): the virtual ghost cell behind a
 * far-field / fixed face holds the ghost state with the fluid cell's time step dt_L; its collisionless part
 * e^{-x}, x = dt_L / tau_g, is sampled as particles in a slab of depth D = (max(W_0, 0) + 6 sqrt(RT_g)) dt_L
 * behind the face (W_0 the ghost's inflow speed), and those that reach the face within dt_L enter the fluid
 * cell (Sec. III B: collisionless particles fly the whole step). Per face: N = ceil(M / m_ref) particles
 * (at most 2047) of mass M / N, M = rho_g e^{-x} s D, m_ref = rho_g Omega_L / N_ref. FP64. */
static void inject_params(or_ctx* cx)
{
    for (int j = 0; j < cx->n_inj; ++j) {
        const int f = cx->inj_face[j], L = cx->fL[f];
        double Wg[4];
        ghost_state(cx, f, Wg);
        const double rho = Wg[0], r = 1.0 / rho, U = Wg[1] * r, V = Wg[2] * r;
        const double RT = (Wg[3] * r - 0.5 * (U * U + V * V)) * (2.0 / 3.0);
        const double x = cx->dt[L] / tau_of(cx, Wg);
        const double e = or_expd(-x);
        const double sig = sqrt(RT);
        const double W0 = -(U * cx->fnx[f] + V * cx->fny[f]);
        const double D = ((W0 > 0.0 ? W0 : 0.0) + 6.0 * sig) * cx->dt[L];
        const double M = ((rho * e) * cx->fs[f]) * D;
        int n = 0;
        if (!cx->wave_only && M > 0.0) {
            const double q = ceil(M / ((rho * cx->vol[L]) / (double)cx->n_ref));
            n = q > (double)OR_MAX_NEW ? OR_MAX_NEW : (q < 1.0 ? 1 : (int)q);
        }
        cx->inj_n[j] = n;
        cx->inj_m[j] = n > 0 ? M / (double)n : 0.0;
        cx->inj_u[j] = U; cx->inj_v[j] = V; cx->inj_sig[j] = sig; cx->inj_D[j] = D;
    }
}

/* ----------------------------------------------------------- a8: reconstruction (order 2, S6 reading) */

/* smooth (van Albada type) limited slope from the one-sided slopes a, b: ((b^2 + e2) a + (a^2 + e2) b) /
 * (a^2 + b^2 + 2 e2); exact for a = b, zero for a = -b, and differentiable, so that steady runs converge */
static double smooth_slope(double a, double b, double e2) { return ((b * b + e2) * a + (a * a + e2) * b) / ((a * a + b * b) + 2.0 * e2); }

/* Limited gradients (d/dx, d/dy) of the four components of W (v = 0..3) and of W^h (v = 4..7) per cell.
 * 1-D: a smooth limiter of the one-sided slopes a, b to the two neighbours (zero next to a boundary face),
 * ((b^2 + e2) a + (a^2 + e2) b) / (a^2 + b^2 + 2 e2) with e2 = K^3 h s^2 (the slope form of Venkatakrishnan's
 * epsilon below: K = 5, h the cell length, s the component's freestream scale).
 * 2-D: least-squares gradient over the neighbours across interior and periodic faces, weights 1 / |dx|^2
 * (zero with fewer than two neighbours), then Venkatakrishnan's limiter (a smooth form of keeping the
 * reconstruction at every face midpoint within the values of the cell and those neighbours): one factor per
 * component, the smallest over the faces and at most 1, with epsilon^2 = (K h)^3 s^2, K = 5, h = sqrt(Omega)
 * and s the freestream scale of the component (rho_inf; rho_inf (U_inf + sqrt(R T_inf)) for the momenta;
 * (rho E)_inf), which makes it independent of the units of each component. */
static void gradients(or_ctx* cx)
{
    for (int c = 0; c < cx->C; ++c) {
        double* g = cx->grad + 16 * (size_t)c;
        for (int v = 0; v < 8; ++v) {
            const double* A = v < 4 ? cx->W : cx->Wh;
            const int comp = v & 3;
            const double vc = A[4 * c + comp];
            double gx = 0.0, gy = 0.0;
            if (cx->dim == 1) {
                const int ql = 4 * c, qr = 4 * c + 1, nl = cx->cnbr[ql], nr = cx->cnbr[qr];
                if (nl >= 0 && nr >= 0) {
                    /* a neighbour across a periodic face, in this cell's frame */
                    const double xl = cx->xc[nl] - cx->cshift[ql], xr = cx->xc[nr] - cx->cshift[qr];
                    const double sc = comp == 0 ? cx->W_inf[0]
                                    : comp == 3 ? cx->W_inf[3] : cx->W_inf[0] * (cx->U_inf + sqrt(OR_R));
                    gx = smooth_slope((vc - A[4 * nl + comp]) / (cx->xc[c] - xl), (A[4 * nr + comp] - vc) / (xr - cx->xc[c]),
                                      (125.0 * cx->vol[c]) * (sc * sc));
                }
            } else {
                double a11 = 0.0, a12 = 0.0, a22 = 0.0, b1 = 0.0, b2 = 0.0, vmax = vc, vmin = vc;
                int nn = 0;
                for (int k = 0; k < cx->nfc[c]; ++k) {
                    const int nb = cx->cnbr[4 * c + k];
                    if (nb < 0) continue;
                    const double dx = cx->xc[nb] - cx->xc[c], dy = cx->yc[nb] - cx->yc[c];
                    const double w = 1.0 / (dx * dx + dy * dy), dv = A[4 * nb + comp] - vc;
                    a11 += w * dx * dx; a12 += w * dx * dy; a22 += w * dy * dy;
                    b1 += w * dx * dv; b2 += w * dy * dv;
                    if (A[4 * nb + comp] > vmax) vmax = A[4 * nb + comp];
                    if (A[4 * nb + comp] < vmin) vmin = A[4 * nb + comp];
                    nn++;
                }
                const double det = a11 * a22 - a12 * a12;
                if (nn >= 2 && det > 1e-12 * (a11 * a22)) {
                    gx = (a22 * b1 - a12 * b2) / det;
                    gy = (a11 * b2 - a12 * b1) / det;
                    const double sc = comp == 0 ? cx->W_inf[0]
                                    : comp == 3 ? cx->W_inf[3] : cx->W_inf[0] * (cx->U_inf + sqrt(OR_R));
                    const double kh = 5.0 * sqrt(cx->vol[c]);
                    const double eps2 = ((kh * kh) * kh) * (sc * sc);
                    double phi = 1.0;
                    for (int k = 0; k < cx->nfc[c]; ++k) {
                        const int f = cx->cface[4 * c + k];
                        const double mx = cx->fax[f] + 0.5 * cx->fex[f], my = cx->fay[f] + 0.5 * cx->fey[f];
                        const double d2 = gx * (mx - cx->xc[c]) + gy * (my - cx->yc[c]);
                        if (d2 == 0.0) continue;
                        const double d1 = d2 > 0.0 ? vmax - vc : vmin - vc;
                        const double r = ((d1 * d1 + eps2) * d2 + (2.0 * d2) * (d2 * d1)) /
                                         (d2 * (((d1 * d1 + 2.0 * (d2 * d2)) + d1 * d2) + eps2));
                        if (r < phi) phi = r;
                    }
                    gx *= phi;
                    gy *= phi;
                }
            }
            g[2 * v] = gx;
            g[2 * v + 1] = gy;
        }
    }
}

/* Order 2: the state of cell c's W (which = 0) or W^h (which = 1) at face f (its local face k), W_c + grad .
 * (x_f - x_c) with x_f the face point (1-D) or midpoint (2-D), and the normal derivative n . grad, both in
 * the face frame (n, t). Returns 0 when the reconstructed state is not a positive density and internal
 * energy (for W: that side stays first order). */
static int face_side(const or_ctx* cx, int c, int k, int f, int which, double Wf[4], double dn[4])
{
    const double* g = cx->grad + 16 * (size_t)c + 8 * which;
    const double* Wc = (which ? cx->Wh : cx->W) + 4 * c;
    double ddx, ddy;
    if (cx->dim == 1) {
        ddx = (k == 0 ? cx->xl[c] : cx->xr[c]) - cx->xc[c];   /* local face 0: left end, 1: right end */
        ddy = 0.0;
    } else {
        ddx = (cx->fax[f] + 0.5 * cx->fex[f]) - cx->xc[c];
        ddy = (cx->fay[f] + 0.5 * cx->fey[f]) - cx->yc[c];
    }
    double W[4], d[4];
    for (int q = 0; q < 4; ++q) {
        W[q] = Wc[q] + (g[2 * q] * ddx + g[2 * q + 1] * ddy);
        d[q] = g[2 * q] * cx->fnx[f] + g[2 * q + 1] * cx->fny[f];
    }
    to_frame(W, cx->fnx[f], cx->fny[f], Wf);
    to_frame(d, cx->fnx[f], cx->fny[f], dn);
    return W[0] > 0.0 && W[3] - 0.5 * (W[1] * W[1] + W[2] * W[2]) / W[0] > 0.0;
}

static int local_face(const or_ctx* cx, int c, int f)
{
    for (int k = 0; k < cx->nfc[c]; ++k)
        if (cx->cface[4 * c + k] == f) return k;
    return -1;
}

static void wave_fluxes(or_ctx* cx)
{
    for (int f = 0; f < cx->F; ++f) {
        const int L = cx->fL[f], R = cx->fR[f], bc = cx->fbc[f];
        const double nx = cx->fnx[f], ny = cx->fny[f];
        double WL[4], WhL[4], WR[4], WhR[4], F[4];
        to_frame(cx->W + 4 * L, nx, ny, WL);
        to_frame(cx->Wh + 4 * L, nx, ny, WhL);
        const double* cL = cx->co + 7 * L;
        /* the sampled-from part of g^h keeps dbar_d - e^{-x} where this step's particles carry e^{-x} of it */
        const double frL = (cx->wave_only || cx->nhp[L] == 0) ? cL[3] : cL[5];
        /* order 2 (S6): reconstructed face states of W (equilibrium part) and W^h (free-transport wave, with
         * its normal slope term weighted with dbar_e, or dbar_e + dt e^{-x} / 2 when the collisionless part is
         * carried by particles, Eq. 50) on interior, periodic and far-field / fixed faces */
        const int o2 = cx->order == 2 && (bc == 0 || bc == OR_BC_PERIODIC || bc == OR_BC_FARFIELD || bc == OR_BC_FIXED);
        double dhL[4], dhR[4], dtmp[4], WLc[4], WRc[4];
        int sL = 0, sR = 0;
        for (int q = 0; q < 4; ++q) WLc[q] = WL[q];
        const double csL = cx->wave_only ? cL[4] : cL[6];
        if (o2) {
            /* W and W^h are reconstructed together (the remainder of W^h is taken against W at the same
             * point); a side whose reconstructed W is not a positive density and internal energy stays first
             * order */
            const int kL = local_face(cx, L, f);
            double Wf[4], Whf[4];
            if (face_side(cx, L, kL, f, 0, Wf, dtmp)) {
                face_side(cx, L, kL, f, 1, Whf, dhL);
                for (int q = 0; q < 4; ++q) { WL[q] = Wf[q]; WhL[q] = Whf[q]; }
                sL = 1;
            }
        }
        if (bc == 0 || bc == OR_BC_PERIODIC) {
            to_frame(cx->W + 4 * R, nx, ny, WR);
            to_frame(cx->Wh + 4 * R, nx, ny, WhR);
            for (int q = 0; q < 4; ++q) WRc[q] = WR[q];
            const double* cR = cx->co + 7 * R;
            const double frR = (cx->wave_only || cx->nhp[R] == 0) ? cR[3] : cR[5];
            if (o2) {
                const int kR = local_face(cx, R, f);
                double Wf[4], Whf[4];
                if (face_side(cx, R, kR, f, 0, Wf, dtmp)) {
                    face_side(cx, R, kR, f, 1, Whf, dhR);
                    for (int q = 0; q < 4; ++q) { WR[q] = Wf[q]; WhR[q] = Whf[q]; }
                    sR = 1;
                }
            }
            face_flux(WL, WR, WhL, WhR, cL[3], cR[3], cL, cR, frL, frR, cx->fdL[f], cx->fdR[f],
                      cx->Pr, WLc, WRc, sL ? dhL : NULL, sR ? dhR : NULL, csL, cx->wave_only ? cR[4] : cR[6], F,
                      NULL, NULL, NULL, NULL);
        } else if (bc == OR_BC_WALL) {
            wall_flux(cx, WL, WhL, cL[3], cL, frL, F);
        } else if (bc == OR_BC_SYMMETRY) {
            /* mirror ghost: same state with the normal velocity reversed, same coefficients */
            double Wm[4] = {WL[0], -WL[1], WL[2], WL[3]}, Whm[4] = {WhL[0], -WhL[1], WhL[2], WhL[3]};
            face_flux(WL, Wm, WhL, Whm, cL[3], cL[3], cL, cL, frL, frL, cx->fdL[f], cx->fdL[f],
                      cx->Pr, NULL, NULL, NULL, NULL, 0.0, 0.0, F, NULL, NULL, NULL, NULL);
        } else {
            /* far-field / fixed ghost: a virtual cell of the ghost state with the fluid cell's time step
             * (Sec. IV B). Its collisionless part e^{-x} enters as particles (ghost sources, see the particle
             * stage), so its wave free-transport weight is dbar_d - e^{-x}, as for an interior side; without
             * particles (wave-only mode) the whole free-transport part stays in the wave */
            double Wg[4];
            ghost_state(cx, f, Wg);
            to_frame(Wg, nx, ny, WR);
            double cR[7];
            lts_coeffs(cx->dt[L], tau_of(cx, Wg), or_expd(-cx->dt[L] / tau_of(cx, Wg)), cR);
            face_flux(WL, WR, WhL, WR, cL[3], cR[3], cL, cR, frL, cx->wave_only ? cR[3] : cR[5], cx->fdL[f],
                      cx->fdL[f], cx->Pr, WLc, NULL, sL ? dhL : NULL, NULL, csL, 0.0, F, NULL, NULL, NULL, NULL);
        }
        /* non-finite flux (reading): extreme near-vacuum neighbours can make the interface density underflow
         * against its neighbours' and the slopes overflow; such a face carries no wave flux */
        if (!isfinite(F[0]) || !isfinite(F[1]) || !isfinite(F[2]) || !isfinite(F[3])) F[0] = F[1] = F[2] = F[3] = 0.0;
        /* back to the global frame: momentum = F_n n + F_t t, t = (-n_y, n_x) */
        cx->flux[4 * f + 0] = F[0];
        cx->flux[4 * f + 1] = F[1] * nx - F[2] * ny;
        cx->flux[4 * f + 2] = F[1] * ny + F[2] * nx;
        cx->flux[4 * f + 3] = F[3];
    }
}

/* -------------------------------------------------------------------- a10: update (Eq. 53) */

static void update(or_ctx* cx)
{
    const double sc[4] = {ldexp(1.0, -cx->fx[0]), ldexp(1.0, -cx->fx[1]), ldexp(1.0, -cx->fx[1]),
                          ldexp(1.0, -cx->fx[2])};
    const int tk[4] = {0, 1, 2, 4};
    double rs[4] = {0, 0, 0, 0};
    const double alpha = 2.0 / 1001.0;
    for (int c = 0; c < cx->C; ++c) {
        double acc[4] = {0, 0, 0, 0};
        for (int k = 0; k < cx->nfc[c]; ++k) {
            const int f = cx->cface[4 * c + k];
            for (int q = 0; q < 4; ++q) {
                const double t = cx->flux[4 * f + q] * cx->fs[f];
                acc[q] += cx->csgn[4 * c + k] > 0 ? t : -t;
            }
        }
        const double coef = cx->dt[c] / cx->vol[c];
        double* W = cx->W + 4 * c;
        double Wn[4];
        for (int q = 0; q < 4; ++q) {
            const int64_t d = cx->wpl[5 * c + tk[q]] - cx->wm[5 * c + tk[q]];
            Wn[q] = (W[q] - coef * acc[q]) + ((double)d * sc[q]) / cx->vol[c];
        }
        if (cx->dim == 1) Wn[2] = 0.0;
        if (!isfinite(Wn[0]) || !isfinite(Wn[1]) || !isfinite(Wn[2]) || !isfinite(Wn[3]))
            or_set_error(cx, OR_ENONPHYS, "non-finite cell state after the update");
        /* realizability floor (reading): statistical noise can leave the wave's share W - W^p of a cell
         * negative and drive the updated state out of the realizable set. Such a cell restarts from its
         * particle content W^{p,+} / Omega_i (so that the next step's W^h = W - W^p, the mass of the collided
         * particles, is not negative), its speed limited to U_cap and its temperature clamped to
         * [T_min, T_cap]; a cell without particles restarts from the near-vacuum state at rest at T_inf.
         * (Restarting a cell that holds particles from vacuum instead leaves W^h = -W^p, whose wave flux
         * drives the neighbours out of the realizable set in turn.) */
        if (!realizable(cx, Wn)) {
            double P[4];
            for (int q = 0; q < 4; ++q) P[q] = ((double)cx->wpl[5 * c + tk[q]] * sc[q]) / cx->vol[c];
            if (cx->dim == 1) P[2] = 0.0;
            if (P[0] > OR_RHO_FLOOR) {
                const double r = 1.0 / P[0];
                double U = P[1] * r, V = P[2] * r;
                double q2 = U * U + V * V;
                if (q2 > cx->U_cap * cx->U_cap) {
                    const double f = cx->U_cap / sqrt(q2);
                    U = U * f;
                    V = V * f;
                    q2 = U * U + V * V;
                }
                double e = P[3] * r - 0.5 * q2;
                const double emin = (1.5 * OR_R) * cx->T_min, emax = (1.5 * OR_R) * cx->T_cap;
                if (!(e >= emin)) e = emin;
                if (e > emax) e = emax;
                Wn[0] = P[0]; Wn[1] = P[0] * U; Wn[2] = P[0] * V; Wn[3] = P[0] * (e + 0.5 * q2);
            } else {
                Wn[0] = OR_RHO_FLOOR; Wn[1] = 0.0; Wn[2] = 0.0; Wn[3] = OR_RHO_FLOOR * (1.5 * OR_R);
            }
            cx->stats[8] += 1;
        }
        for (int q = 0; q < 4; ++q) {
            const double r = (Wn[q] - W[q]) / cx->dt[c];
            rs[q] += cx->vol[c] * (r * r);
            W[q] = Wn[q];
        }
        const double chi = (((double)cx->wpl[5 * c] * sc[0]) / cx->vol[c]) / W[0];
        cx->chi_ema[c] = cx->step == 0 ? chi : cx->chi_ema[c] + alpha * (chi - cx->chi_ema[c]);
    }
    for (int q = 0; q < 4; ++q) cx->res[q] = sqrt(rs[q]);
}

/* ------------------------------------------------------------ a11: surface quantities (Sec. V A) */

static void monitors(or_ctx* cx);

static void surface(or_ctx* cx)
{
    const double s1 = ldexp(1.0, -cx->fx[1]), s4 = ldexp(1.0, -cx->fx[2]);
    for (int iw = 0; iw < cx->nwall; ++iw) {
        const int f = cx->wall_face[iw], c = cx->fL[f];
        const double nx = cx->fnx[f], ny = cx->fny[f], tx = -ny, ty = nx;
        const double* F = cx->flux + 4 * f;
        const double sdt = cx->fs[f] * cx->dt[c];
        const double px = ((double)cx->wallt[3 * iw] * s1) / sdt;
        const double py = ((double)cx->wallt[3 * iw + 1] * s1) / sdt;
        const double pe = ((double)cx->wallt[3 * iw + 2] * s4) / sdt;
        const double p = (F[1] + px) * nx + (F[2] + py) * ny;
        const double tw = (F[1] + px) * tx + (F[2] + py) * ty;
        const double q = F[3] + pe;
        cx->surf_last[3 * iw] = p; cx->surf_last[3 * iw + 1] = tw; cx->surf_last[3 * iw + 2] = q;
        cx->surf_sum[3 * iw] += p; cx->surf_sum[3 * iw + 1] += tw; cx->surf_sum[3 * iw + 2] += q;
    }
    monitors(cx);
    cx->nsurf += 1;
}

/* Monitored wall loads (Sec. V A, V B; reading of their definitions, L_ref = 1): drag coefficient
 * C_d = F_x / (rho_inf U_inf^2 / 2) and heat-load coefficient C_H = Q / (rho_inf U_inf^3 / 2), with
 * F = sum_j s_j (p_j n_j + tau_j t_j), t = (-n_y, n_x), Q = sum_j s_j q_j over the wall faces in order (n: the
 * fluid cell's outward normal); at the stagnation point, the mean of the two wall faces adjacent to it (S29),
 * C_p = (p - p_inf) / (rho_inf U_inf^2 / 2) and C_Q = q / (rho_inf U_inf^3 / 2); each followed by its EMA
 * (alpha = 2/1001, the monitor of Sec. V A) from the first surface sample on. */
static void monitors(or_ctx* cx)
{
    const double U = cx->W_inf[1] / cx->W_inf[0];
    const double qd = 0.5 * cx->W_inf[0] * (U * U), qh = 0.5 * cx->W_inf[0] * ((U * U) * U);
    const double p_inf = cx->W_inf[0] * OR_R;   /* T_inf = 1 */
    double fx = 0.0, Q = 0.0;
    for (int iw = 0; iw < cx->nwall; ++iw) {
        const int f = cx->wall_face[iw];
        const double* sv = cx->surf_last + 3 * iw;
        fx += cx->fs[f] * (sv[0] * cx->fnx[f] - sv[1] * cx->fny[f]);
        Q += cx->fs[f] * sv[2];
    }
    double v[4] = {fx / qd, Q / qh, NAN, NAN};
    if (cx->stag[0] >= 0) {
        const double ps = 0.5 * (cx->surf_last[3 * cx->stag[0]] + cx->surf_last[3 * cx->stag[1]]);
        const double qs = 0.5 * (cx->surf_last[3 * cx->stag[0] + 2] + cx->surf_last[3 * cx->stag[1] + 2]);
        v[2] = (ps - p_inf) / qd;
        v[3] = qs / qh;
    }
    const double alpha = 2.0 / 1001.0;
    for (int k = 0; k < 4; ++k) {
        cx->mon[k] = v[k];
        cx->mon[4 + k] = cx->nsurf == 0 ? v[k] : cx->mon[4 + k] + alpha * (v[k] - cx->mon[4 + k]);
    }
}

/* the stagnation point's two wall faces (reading): the two whose fluid-cell normals face the freestream
 * (+x) most, ties to the lower index, when the best of them is within 60 degrees of it (a blunt body);
 * none otherwise (e.g. a flat plate along the flow) */
static void find_stagnation(or_ctx* cx)
{
    int a = -1, b = -1;
    for (int iw = 0; iw < cx->nwall; ++iw) {
        const double nx = cx->fnx[cx->wall_face[iw]];
        if (a < 0 || nx > cx->fnx[cx->wall_face[a]]) { b = a; a = iw; }
        else if (b < 0 || nx > cx->fnx[cx->wall_face[b]]) b = iw;
    }
    cx->stag[0] = cx->stag[1] = -1;
    if (a >= 0 && b >= 0 && cx->fnx[cx->wall_face[a]] > 0.5) {
        cx->stag[0] = a < b ? a : b;
        cx->stag[1] = a < b ? b : a;
    }
}

/* restart the surface averages (and the monitors' EMAs) at the next step */
int oracle_reset_surface(oracle_ctx* cx)
{
    memset(cx->surf_sum, 0, 3 * (size_t)cx->nwall * sizeof(double));
    cx->nsurf = 0;
    return cx->err;
}

int oracle_monitors(oracle_ctx* cx, double* out)
{
    for (int k = 0; k < 8; ++k) out[k] = cx->mon[k];
    return cx->err;
}

/* ----------------------------------------------------------------------------------- one step */

static int one_step(or_ctx* cx)
{
    const int C = cx->C;
    memset(cx->wm, 0, 5 * (size_t)C * 8);
    memset(cx->wpl, 0, 5 * (size_t)C * 8);
    memset(cx->wrt, 0, 5 * (size_t)C * 8);
    memset(cx->cross, 0, 2 * (size_t)cx->F * 8);
    memset(cx->frec, 0, 4 * (size_t)cx->F * 8);
    memset(cx->wallt, 0, 3 * (size_t)cx->nwall * 8);
    for (int k = 2; k < 11; ++k) cx->stats[k] = 0;
    /* step 1: decomposition and sampling; step 2: free transport and tallies (Sec. III C, Sec. IV B) */
    decompose(cx);
    if (cx->err) return cx->err;
    inject_params(cx);
    if (cx->prec == 0) or_particles_step_f32(cx); else or_particles_step_f64(cx);
    /* step 3: wave fluxes from the step-start W and W^h (order 2: reconstructed, S6), then the conservative
     * update (Eq. 53) */
    if (cx->order == 2) gradients(cx);
    wave_fluxes(cx);
    update(cx);
    surface(cx);
    memcpy(cx->wret_prev, cx->wrt, 5 * (size_t)C * 8);
    cx->step += 1;
    cx->stats[0] = cx->step;
    cx->stats[1] = cx->np;
    return cx->err;
}

int oracle_step(oracle_ctx* cx, int32_t n)
{
    if (!cx || n < 0) return OR_EINVAL;
    if (cx->err) return cx->err;
    for (int32_t s = 0; s < n; ++s) {
        int st = one_step(cx);
        if (st) return st;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------------------- accessors */

int oracle_set_field(oracle_ctx* cx, const double* prim)
{
    for (int c = 0; c < cx->C; ++c) {
        const double* p = prim + 4 * c;
        if (!(p[0] > 0.0) || !(p[3] > 0.0)) return OR_EINVAL;
        prim_to_cons(p[0], p[1], p[2], p[3], cx->W + 4 * c);
    }
    memset(cx->wret_prev, 0, 5 * (size_t)cx->C * 8);
    cx->np = 0;
    return OR_OK;
}

int oracle_get_field(oracle_ctx* cx, double* W, double* Wp)
{
    memcpy(W, cx->W, 4 * (size_t)cx->C * 8);
    if (Wp) {
        for (int c = 0; c < cx->C; ++c) {
            const int64_t* r = cx->wret_prev + 5 * c;
            Wp[4 * c] = ((double)r[0] * ldexp(1.0, -cx->fx[0])) / cx->vol[c];
            Wp[4 * c + 1] = ((double)r[1] * ldexp(1.0, -cx->fx[1])) / cx->vol[c];
            Wp[4 * c + 2] = ((double)r[2] * ldexp(1.0, -cx->fx[1])) / cx->vol[c];
            Wp[4 * c + 3] = ((double)r[4] * ldexp(1.0, -cx->fx[2])) / cx->vol[c];
        }
    }
    return OR_OK;
}

/* The paper judges steady state by monitored histories and defines no residual (Sec. V A). Normalised
 * residual of this library: the raw residual of each component divided by a freestream scale that cannot
 * vanish, S_c sqrt(sum_i Omega_i) / L_ref with L_ref = 1 and S = (rho c, rho c^2, rho c^2, rho c^3 / 2) at
 * rho_inf = 1, c = U_inf + sqrt(gamma R T_inf) (the freestream's largest signal speed): an O(1) imbalance of
 * the freestream fluxes over the whole domain reads about 1, whatever the first step changed. */
static void residual_scale(const or_ctx* cx, double S[4])
{
    double area = 0.0;
    for (int c = 0; c < cx->C; ++c) area += cx->vol[c];
    const double cs = cx->U_inf + sqrt((5.0 / 3.0) * OR_R * 1.0);
    const double ra = sqrt(area);
    S[0] = cs * ra;
    S[1] = (cs * cs) * ra;
    S[2] = S[1];
    S[3] = (0.5 * ((cs * cs) * cs)) * ra;
}

int oracle_residual(oracle_ctx* cx, double* out)
{
    double S[4];
    residual_scale(cx, S);
    for (int q = 0; q < 4; ++q) {
        out[q] = cx->res[q] / S[q];
        out[4 + q] = cx->res[q];
    }
    return OR_OK;
}

int oracle_surface(oracle_ctx* cx, double* p, double* tau, double* q, int32_t n_wall, int32_t averaged)
{
    if (n_wall != cx->nwall) return OR_EINVAL;
    const double* src = averaged ? cx->surf_sum : cx->surf_last;
    const double d = averaged ? (cx->nsurf > 0 ? (double)cx->nsurf : 1.0) : 1.0;
    for (int i = 0; i < n_wall; ++i) {
        p[i] = src[3 * i] / d;
        tau[i] = src[3 * i + 1] / d;
        q[i] = src[3 * i + 2] / d;
    }
    return OR_OK;
}

int64_t oracle_ar_sample(int32_t precision, uint64_t seed, uint32_t case_id, int64_t step, uint64_t pid0, int32_t n,
                         double ax, double ay, double M, double* z)
{
    or_ctx cx;
    memset(&cx, 0, sizeof cx);
    cx.seed = seed; cx.case_id = case_id; cx.step = step;
    int64_t fb = 0;
    for (int32_t k = 0; k < n; ++k) {
        if (precision == 0) {
            float zf[3];
            fb += or_new_velocity_f32(&cx, pid0 + (uint64_t)k, 1, (float)ax, (float)ay, (float)M, zf);
            for (int q = 0; q < 3; ++q) z[3 * (int64_t)k + q] = (double)zf[q];
        } else {
            fb += or_new_velocity_f64(&cx, pid0 + (uint64_t)k, 1, ax, ay, M, z + 3 * (int64_t)k);
        }
    }
    return fb;
}

int oracle_stats(oracle_ctx* cx, int64_t* out)
{
    memcpy(out, cx->stats, sizeof cx->stats);
    return OR_OK;
}

int64_t oracle_num_particles(oracle_ctx* cx) { return cx->np; }

int oracle_get_particles(oracle_ctx* cx, int64_t cap, uint64_t* pid, int32_t* cell, double* x, double* y,
                         double* u, double* v, double* w, double* m)
{
    if (cap < cx->np) return OR_EINVAL;
    for (int64_t i = 0; i < cx->np; ++i) {
        const or_particle* P = &cx->p[i];
        pid[i] = P->pid; cell[i] = P->cell;
        x[i] = P->x; y[i] = P->y; u[i] = P->u; v[i] = P->v; w[i] = P->w; m[i] = P->m;
    }
    return OR_OK;
}

int oracle_set_state(oracle_ctx* cx, int64_t step, const double* W, const int64_t* wret, int64_t np,
                     const uint64_t* pid, const int32_t* cell, const double* x, const double* y,
                     const double* u, const double* v, const double* w, const double* m)
{
    cx->step = step;
    memcpy(cx->W, W, 4 * (size_t)cx->C * 8);
    memcpy(cx->wret_prev, wret, 5 * (size_t)cx->C * 8);
    if (np > cx->cap) {
        cx->cap = np;
        cx->p = (or_particle*)realloc(cx->p, (size_t)np * sizeof(or_particle));
    }
    for (int64_t i = 0; i < np; ++i) {
        or_particle* P = &cx->p[i];
        memset(P, 0, sizeof *P);
        P->pid = pid[i]; P->cell = cell[i];
        P->x = x[i]; P->y = y[i]; P->u = u[i]; P->v = v[i]; P->w = w[i]; P->m = m[i];
    }
    cx->np = np;
    return OR_OK;
}

/* Time-varying steps (Sec. IV A, Eqs. 44-46; a study tool, the method keeps its steps fixed): replace the
 * local time steps from the next step on; the crossing scaling follows the current steps. */
int oracle_set_time_steps(oracle_ctx* cx, const double* dt)
{
    if (!cx || !dt) return OR_EINVAL;
    for (int c = 0; c < cx->C; ++c)
        if (!(dt[c] > 0.0) || !isfinite(dt[c])) return OR_EINVAL;
    for (int c = 0; c < cx->C; ++c) cx->dt[c] = dt[c];
    set_ratios(cx);
    return OR_OK;
}

int oracle_get_tallies(oracle_ctx* cx, int64_t* wm, int64_t* wpl, int64_t* wret, int64_t* cross, int64_t* wall,
                       int64_t* frec)
{
    const size_t C = (size_t)cx->C;
    if (wm) memcpy(wm, cx->wm, 5 * C * 8);
    if (wpl) memcpy(wpl, cx->wpl, 5 * C * 8);
    if (wret) memcpy(wret, cx->wrt, 5 * C * 8);
    if (cross) memcpy(cross, cx->cross, 2 * (size_t)cx->F * 8);
    if (wall) memcpy(wall, cx->wallt, 3 * (size_t)cx->nwall * 8);
    if (frec) memcpy(frec, cx->frec, 4 * (size_t)cx->F * 8);
    return OR_OK;
}

/* per cell: tau, x = dt/tau, e^{-x}, N^hp, m_new, U^h, V^h, R T^h of the last decomposition */
int oracle_get_cell_data(oracle_ctx* cx, double* out)
{
    for (int c = 0; c < cx->C; ++c) {
        double* o = out + 8 * c;
        o[0] = cx->tau[c]; o[1] = cx->xr_t[c]; o[2] = cx->emx[c]; o[3] = (double)cx->nhp[c];
        o[4] = cx->mnew[c]; o[5] = cx->samp[3 * c]; o[6] = cx->samp[3 * c + 1]; o[7] = cx->samp[3 * c + 2];
    }
    return OR_OK;
}

int oracle_get_shakhov(oracle_ctx* cx, double* out)
{
    if (!cx || !out) return OR_EINVAL;
    memcpy(out, cx->hq, 3 * (size_t)cx->C * 8);
    return OR_OK;
}

int oracle_get_gradients(oracle_ctx* cx, double* out)
{
    if (!cx || !out) return OR_EINVAL;
    memcpy(out, cx->grad, 16 * (size_t)cx->C * 8);
    return OR_OK;
}

int oracle_get_flux(oracle_ctx* cx, double* flux)
{
    memcpy(flux, cx->flux, 4 * (size_t)cx->F * 8);
    return OR_OK;
}

int oracle_get_geometry(oracle_ctx* cx, double* dt, double* vol, int32_t* nfaces, int32_t* nwall)
{
    if (dt) memcpy(dt, cx->dt, (size_t)cx->C * 8);
    if (vol) memcpy(vol, cx->vol, (size_t)cx->C * 8);
    if (nfaces) *nfaces = cx->F;
    if (nwall) *nwall = cx->nwall;
    return OR_OK;
}

int oracle_get_mesh(oracle_ctx* cx, double* cells, int32_t* faces, double* fgeo)
{
    if (!cx) return OR_EINVAL;
    for (int c = 0; cells && c < cx->C; ++c) {
        cells[3 * c] = cx->xc[c]; cells[3 * c + 1] = cx->yc[c]; cells[3 * c + 2] = cx->vol[c];
    }
    for (int f = 0; f < cx->F; ++f) {
        if (faces) { faces[3 * f] = cx->fL[f]; faces[3 * f + 1] = cx->fR[f]; faces[3 * f + 2] = cx->fbc[f]; }
        if (fgeo) {
            double* g = fgeo + 5 * f;
            g[0] = cx->fnx[f]; g[1] = cx->fny[f]; g[2] = cx->fs[f]; g[3] = cx->fdL[f]; g[4] = cx->fdR[f];
        }
    }
    return OR_OK;
}

const char* oracle_last_error(oracle_ctx* cx) { return cx->msg; }

/* Sec. IV A, Eq. 46 with constant transported mass: left- and right-hand sides of the balance condition
 * sum(dt_R) / sum(dt_L) and (1/M) sum(dt_R / dt_L) for a sequence of M step pairs. */
void oracle_balance_condition(int32_t M, const double* dtL, const double* dtR, double* out)
{
    double sL = 0.0, sR = 0.0, q = 0.0;
    for (int32_t l = 0; l < M; ++l) {
        sL += dtL[l];
        sR += dtR[l];
        q += dtR[l] / dtL[l];
    }
    out[0] = sR / sL;
    out[1] = q / (double)M;
}
