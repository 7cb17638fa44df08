/*
 * teuk_oracle.c -- the ORACLE: a plain, slow, obviously-correct FP64 CPU
 * implementation of the time-domain Teukolsky solver of McKennon, Forrester &
 * Khanna, "High Accuracy Gravitational Waveforms from Black Hole Binary
 * Inspirals Using OpenCL" (arXiv:1206.0270).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test-suite, the package smoke check
 * and the benchmark's CPU-baseline / reference legs may load it.  It shares no
 * code, header, table or helper with the CUDA path, and the CUDA path never
 * calls it.
 *
 * What it computes (paper section "Teukolsky Code"):
 *   - Eq. (1): the Teukolsky master equation for spin weight s on Kerr, M = 1.
 *   - Eq. (2): Psi = e^{i m phi} r^3 Phi_m(t, r, theta), Boyer-Lindquist phi.
 *   - the first-order-in-time form with the auxiliary momentum Pi,
 *     u = {Phi_R, Phi_I, Pi_R, Pi_I}, written here as u_t + D u_{r*} = S;
 *   - Eq. (3) (predictor at radial mid-points, half time step) and Eq. (4)
 *     (corrector to the full step) of the two-step Lax-Wendroff scheme, with
 *     angular derivatives inside S by second-order centred differences;
 *   - the angular boundary rule (even |m|: dPhi/dtheta = 0 at the poles, odd
 *     |m|: Phi = 0) and Phi = Pi = 0 on the inner and outer radial boundary;
 *   - a point particle modelled as a narrow Gaussian ("Mathematical
 *     Advances", item 1) on a circular equatorial orbit.
 *
 * The paper does not print D, S, Pi, the source, the time-step rule or the
 * grid; the readings used here (each marked READING below) are:
 *   - Pi = d_t Phi + b d_{r*} Phi with b = (r^2+a^2)/Sigma_hat; then
 *     D = [[b, 0], [-d, -b]] and S = (Pi, -c_t Pi - W Phi + kappa L_theta Phi + F).
 *   - grid r*_i = r*_min + i h (i < nr), mid-points r*_{i+1/2};
 *     theta_j = (j + 1/2) pi / nth (cell-centred; the poles are never nodes);
 *     ghosts Phi_{-1} = p Phi_0, Phi_nth = p Phi_{nth-1}, p = +1 (even |m|),
 *     -1 (odd |m|).  Coefficients are evaluated analytically at mid-points.
 *   - S at a mid-point (predictor) and at a node (corrector) is evaluated on
 *     the average of the two neighbouring values of u.
 *   - tortoise coordinate r* = r + 2 r+/(r+ - r-) ln((r - r+)/2)
 *                                 - 2 r-/(r+ - r-) ln((r - r-)/2).
 *   - source F = A G(r*, theta) e^{-i m Omega t} added to the Pi row, G a
 *     Gaussian of width sigma in r* and sigma/r0 in theta around
 *     (r*(r0), pi/2), cut to zero where its exponent exceeds 50, normalised
 *     so that sum_ij G(r*_i, theta_j) h dtheta = 1; Omega = +-1/(r0^{3/2} +- a).
 *   - t_n = n dt; the predictor uses the source at t_n, the corrector at
 *     t_n + dt/2.
 *   - time step: dt = min(C_r h / max b, C_theta / omega_max), omega_max^2 the
 *     Gershgorin bound of the discrete angular-plus-potential operator.
 *   - angular dissipation (Kreiss & Oliger 1973, the sixth-order member of
 *     their family), optional with strength eps (0 = the bare scheme): the
 *     corrector subtracts (eps/64) D6 u^n from u^{n+1} on every interior row,
 *     D6 u_j = -(u_{j-3} + u_{j+3}) + 6 (u_{j-2} + u_{j+2})
 *              - 15 (u_{j-1} + u_{j+1}) + 20 u_j,
 *     for Phi and Pi alike, with the ghosts u_{-1-q} = p u_q and
 *     u_{nth+q} = p u_{nth-1-q} of the pole rule (reflection across the pole,
 *     applied again where a short row needs it).  On cos(k theta_j) (p = +1)
 *     and sin(k theta_j) (p = -1) it multiplies by 1 - eps sin^6(k dtheta/2).
 *     It damps the stiff pole modes of the source terms, so that C_theta can
 *     be 0.8 with eps = 1 instead of 0.1 with eps = 0.
 *   - time-symmetric initial data: Pi_i = b_i (Phi_{i+1} - Phi_{i-1}) / (2h).
 *
 * Parity unpinned: the amplitude and phase of the waveform relative to a
 * physical h_22.  The paper does not give the true source T or its
 * normalisation, so the Gaussian's strength A is a reading.  It is pinned
 * only through its discrete normalisation, linearity and the forced
 * frequency m Omega.  Everything else above is pinned by the tests against
 * Eq. (1), exact amplification factors, convergence and published
 * quasinormal frequencies.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA contraction,
 * so every product is rounded on its own).  Arrays of complex numbers are
 * interleaved (re, im) doubles, row-major [i][j] with theta (j) fastest.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI 3.14159265358979323846

typedef double complex cplx;

/* ------------------------------------------------------------------------ */
/* Kerr background (M = 1)                                                   */
/* ------------------------------------------------------------------------ */

/* Horizons r_{+-} = 1 +- sqrt(1 - a^2) (roots of Delta = r^2 - 2r + a^2). */
static void horizons(double a, double *rp, double *rm)
{
    double q = sqrt(1.0 - a * a);
    *rp = 1.0 + q;
    *rm = 1.0 - q;
}

/* Tortoise coordinate r*(r), with d(r*)/dr = (r^2 + a^2)/Delta  (READING: constant). */
double oracle_rstar_of_r(double r, double a)
{
    double rp, rm;
    horizons(a, &rp, &rm);
    double kp = 2.0 * rp / (rp - rm);
    double km = 2.0 * rm / (rp - rm);
    return r + kp * log((r - rp) / 2.0) - km * log((r - rm) / 2.0);
}

/* r*(y) with y = ln(r - r+): monotone increasing in y. */
static double rstar_of_y(double y, double a)
{
    double rp, rm;
    horizons(a, &rp, &rm);
    double kp = 2.0 * rp / (rp - rm);
    double km = 2.0 * rm / (rp - rm);
    double x = exp(y);
    return rp + x + kp * (y - log(2.0)) - km * log((x + rp - rm) / 2.0);
}

/* Inverse tortoise map by bisection on y = ln(r - r+).  Delta is formed as
 * x (x + r+ - r-) with x = r - r+, which keeps it accurate near the horizon. */
void oracle_r_of_rstar(double rstar, double a, double *r_out, double *Delta_out)
{
    double lo = -1500.0, hi = 30.0;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (rstar_of_y(mid, a) < rstar) lo = mid; else hi = mid;
    }
    double rp, rm;
    horizons(a, &rp, &rm);
    double x = exp(0.5 * (lo + hi));
    *r_out = rp + x;
    *Delta_out = x * (x + rp - rm);
}

/* Coefficients of the first-order system at (r, theta).
 *
 * From Eq. (1) with Psi = e^{i m phi} psi (d_phi -> i m), multiplied by
 * -Delta/Sigma_hat^2, where Sigma_hat^2 = (r^2+a^2)^2 - a^2 Delta sin^2(theta):
 *   psi_tt + c_t psi_t - b^2 psi_{r*r*} - c_1 psi_{r*}
 *          - kappa (psi_thth + cot(theta) psi_th) + c_0 psi = F,
 *   b = (r^2+a^2)/Sigma_hat, kappa = Delta/Sigma_hat^2,
 *   c_t = [4 i a m r + 2 s (r Delta - (r^2 - a^2)) + 2 i s a Delta cos(theta)] / Sigma_hat^2,
 *   c_1 = [2 r Delta + 2 s (r - 1)(r^2 + a^2)] / Sigma_hat^2,
 *   c_0 = [Delta ((m + s cos(theta))^2 / sin^2(theta) - s) - m^2 a^2
 *          - 2 i s m a (r - 1)] / Sigma_hat^2.
 * With psi = r^3 Phi (Eq. 2) and rho = dr/dr* = Delta/(r^2+a^2):
 *   Phi_tt + c_t Phi_t - b^2 Phi_{r*r*} - e Phi_{r*} - kappa L_theta Phi + W Phi = F/r^3,
 *   e = 6 b^2 rho / r + c_1,
 *   W = c_0 - b^2 rho (3 r^2 rho)' / r^3 - 3 c_1 rho / r,  ' = d/dr.
 * With Pi = Phi_t + b Phi_{r*}:  Pi_t - b Pi_{r*} - d Phi_{r*} = -c_t Pi - W Phi + kappa L_theta Phi,
 *   d = c_t b + e - b d_{r*} b.
 *
 * out[0] = b, out[1..2] = d, out[3..4] = c_t, out[5..6] = W, out[7] = kappa.
 */
void oracle_coefficients(double r, double Delta, double theta, double a, int s, int m,
                         double *out)
{
    double w2 = r * r + a * a;                      /* r^2 + a^2 */
    double sn = sin(theta), cs = cos(theta);
    double Sig2 = w2 * w2 - a * a * Delta * sn * sn; /* Sigma_hat^2 */
    double Sig = sqrt(Sig2);
    double b = w2 / Sig;
    double rho = Delta / w2;
    double kappa = Delta / Sig2;

    cplx c_t = (4.0 * I * a * m * r + 2.0 * s * (r * Delta - (r * r - a * a))
                + 2.0 * I * s * a * Delta * cs) / Sig2;
    double c_1 = (2.0 * r * Delta + 2.0 * s * (r - 1.0) * w2) / Sig2;
    double msc = m + s * cs;
    cplx c_0 = (Delta * (msc * msc / (sn * sn) - s) - (double)(m * m) * a * a
                - 2.0 * I * s * m * a * (r - 1.0)) / Sig2;

    double e = 6.0 * b * b * rho / r + c_1;
    /* (3 r^2 rho)' = 3 [2 r Delta / w2 + r^2 Delta' / w2 - r^2 Delta 2r / w2^2], Delta' = 2r - 2 */
    double d3r2rho = 3.0 * (2.0 * r * Delta / w2 + r * r * (2.0 * r - 2.0) / w2
                            - 2.0 * r * r * r * Delta / (w2 * w2));
    cplx W = c_0 - b * b * rho * d3r2rho / (r * r * r) - 3.0 * c_1 * rho / r;

    /* d_r b = (2 r Sigma_hat - w2 d_r Sigma_hat) / Sigma_hat^2,
     * d_r Sigma_hat = [4 r w2 - a^2 sin^2 (2r - 2)] / (2 Sigma_hat) */
    double dSig = (4.0 * r * w2 - a * a * sn * sn * (2.0 * r - 2.0)) / (2.0 * Sig);
    double db_dr = (2.0 * r * Sig - w2 * dSig) / Sig2;
    double db_drs = rho * db_dr;
    cplx d = c_t * b + e - b * db_drs;

    out[0] = b;
    out[1] = creal(d);  out[2] = cimag(d);
    out[3] = creal(c_t); out[4] = cimag(c_t);
    out[5] = creal(W);  out[6] = cimag(W);
    out[7] = kappa;
}

/* Circular equatorial orbit frequency (Bardeen-Press-Teukolsky), M = 1. */
double oracle_orbit_omega(double r0, double a, int prograde)
{
    double r32 = r0 * sqrt(r0);
    return prograde ? 1.0 / (r32 + a) : -1.0 / (r32 - a);
}

/* ------------------------------------------------------------------------ */
/* Angular operator: L_theta Phi = Phi_thth + cot(theta) Phi_th               */
/* ------------------------------------------------------------------------ */

/* Second-order centred differences on theta_j = (j + 1/2) dth, with the
 * ghost values Phi_{-1} = parity Phi_0 and Phi_{nth} = parity Phi_{nth-1}
 * that encode the pole conditions of the paper (even |m|: parity = +1 gives
 * dPhi/dtheta = 0 at the pole; odd |m|: parity = -1 gives Phi = 0). */
static cplx angular_op_at(const cplx *row, int j, int nth, int parity, double dth, double cotj)
{
    cplx pm = (j > 0) ? row[j - 1] : parity * row[0];
    cplx pp = (j < nth - 1) ? row[j + 1] : parity * row[nth - 1];
    cplx p0 = row[j];
    return (pp - 2.0 * p0 + pm) / (dth * dth) + cotj * (pp - pm) / (2.0 * dth);
}

/* Value of a row at theta index j, extended past the poles by the ghost
 * rule: reflection across theta = 0 maps j < 0 to -1 - j, reflection across
 * theta = pi maps j >= nth to 2 nth - 1 - j, each with the factor parity.
 * Reflections repeat until j lies on the grid (rows shorter than the
 * stencil). */
static cplx ghost_value(const cplx *row, int j, int nth, int parity)
{
    int sign = 1;
    while (j < 0 || j >= nth) {
        j = (j < 0) ? -1 - j : 2 * nth - 1 - j;
        sign *= parity;
    }
    return sign * row[j];
}

/* Sixth-order Kreiss-Oliger difference D6 u_j along theta (minus the third
 * power of the second difference): its Fourier symbol is 64 sin^6(k dth/2). */
static cplx ko6_at(const cplx *row, int j, int nth, int parity)
{
    cplx s1 = ghost_value(row, j - 1, nth, parity) + ghost_value(row, j + 1, nth, parity);
    cplx s2 = ghost_value(row, j - 2, nth, parity) + ghost_value(row, j + 2, nth, parity);
    cplx s3 = ghost_value(row, j - 3, nth, parity) + ghost_value(row, j + 3, nth, parity);
    return -s3 + 6.0 * s2 - 15.0 * s1 + 20.0 * row[j];
}

void oracle_angular_op(int nth, int parity, const double *phi_row, double *out_row)
{
    double dth = ORACLE_PI / nth;
    const cplx *row = (const cplx *)phi_row;
    cplx *out = (cplx *)out_row;
    for (int j = 0; j < nth; ++j) {
        double th = (j + 0.5) * dth;
        out[j] = angular_op_at(row, j, nth, parity, dth, cos(th) / sin(th));
    }
}

/* ------------------------------------------------------------------------ */
/* One two-step Lax-Wendroff step of u_t + D u_{r*} = S  (Eqs. 3 and 4)       */
/* ------------------------------------------------------------------------ */

/* Coefficient fields of the system on an nr x nth grid.  Node fields have nr
 * rows, mid-point fields nr - 1 rows (row i is r*_{i+1/2}); each row holds nth
 * values.  G_* is the source profile (amplitude and normalisation included),
 * or NULL for no source. */
typedef struct {
    int nr, nth, parity;
    double h, dth, dt;
    const double *b_node, *b_mid, *kap_node, *kap_mid;
    const cplx *d_node, *d_mid, *ct_node, *ct_mid, *W_node, *W_mid;
    const double *cot;            /* [nth] */
    const double *G_node, *G_mid; /* [nr][nth], [nr-1][nth] or NULL */
    double eps;                   /* Kreiss-Oliger strength (0: none) */
} lw_system;

/* S(u) at one point (Pi row gets the source F):
 * S_Phi = Pi,  S_Pi = -c_t Pi - W Phi + kappa L_theta Phi + F. */
static void eval_S(const cplx *phi_row, const cplx *pi_row, int j, const lw_system *sys,
                   double kap, cplx ct, cplx W, cplx F, cplx *S_phi, cplx *S_pi)
{
    cplx Lphi = angular_op_at(phi_row, j, sys->nth, sys->parity, sys->dth, sys->cot[j]);
    *S_phi = pi_row[j];
    *S_pi = -ct * pi_row[j] - W * phi_row[j] + kap * Lphi + F;
}

static void lw_step(const lw_system *sys, cplx phase_n, cplx phase_half,
                    const cplx *Phi, const cplx *Pi, cplx *Phi_out, cplx *Pi_out,
                    cplx *Phi_h, cplx *Pi_h)
{
    const int nr = sys->nr, nth = sys->nth;
    const double h = sys->h, dt = sys->dt;

    /* Eq. (3): u^{n+1/2}_{i+1/2} = (u_{i+1} + u_i)/2
     *          - dt/2 [ D_{i+1/2} (u_{i+1} - u_i)/h - S^n_{i+1/2} ],
     * S^n_{i+1/2} evaluated on the average (u_i + u_{i+1})/2 and source at t_n. */
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nr - 1; ++i) {
        cplx avg_phi[nth], avg_pi[nth];
        for (int j = 0; j < nth; ++j) {
            avg_phi[j] = 0.5 * (Phi[(i + 1) * nth + j] + Phi[i * nth + j]);
            avg_pi[j] = 0.5 * (Pi[(i + 1) * nth + j] + Pi[i * nth + j]);
        }
        for (int j = 0; j < nth; ++j) {
            int k = i * nth + j;
            cplx dphi = Phi[(i + 1) * nth + j] - Phi[i * nth + j];
            cplx dpi = Pi[(i + 1) * nth + j] - Pi[i * nth + j];
            double b = sys->b_mid[k];
            cplx dd = sys->d_mid[k];
            cplx Dphi = b * dphi / h;                  /* row 1 of D (u_{i+1} - u_i)/h */
            cplx Dpi = (-dd * dphi - b * dpi) / h;     /* row 2 */
            cplx F = sys->G_mid ? sys->G_mid[k] * phase_n : 0.0;
            cplx S_phi, S_pi;
            eval_S(avg_phi, avg_pi, j, sys, sys->kap_mid[k], sys->ct_mid[k], sys->W_mid[k], F,
                   &S_phi, &S_pi);
            Phi_h[k] = avg_phi[j] - 0.5 * dt * (Dphi - S_phi);
            Pi_h[k] = avg_pi[j] - 0.5 * dt * (Dpi - S_pi);
        }
    }

    /* Eq. (4): u^{n+1}_i = u_i - dt [ D_i (u^{n+1/2}_{i+1/2} - u^{n+1/2}_{i-1/2})/h
     *                                 - S^{n+1/2}_i ],
     * S^{n+1/2}_i evaluated on the average of the two half-step values and
     * source at t_n + dt/2.  Rows 0 and nr-1 are the radial boundary: 0. */
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nr; ++i) {
        if (i == 0 || i == nr - 1) {
            for (int j = 0; j < nth; ++j) {
                Phi_out[i * nth + j] = 0.0;
                Pi_out[i * nth + j] = 0.0;
            }
            continue;
        }
        cplx avg_phi[nth], avg_pi[nth];
        for (int j = 0; j < nth; ++j) {
            avg_phi[j] = 0.5 * (Phi_h[i * nth + j] + Phi_h[(i - 1) * nth + j]);
            avg_pi[j] = 0.5 * (Pi_h[i * nth + j] + Pi_h[(i - 1) * nth + j]);
        }
        for (int j = 0; j < nth; ++j) {
            int k = i * nth + j;
            cplx dphi = Phi_h[i * nth + j] - Phi_h[(i - 1) * nth + j];
            cplx dpi = Pi_h[i * nth + j] - Pi_h[(i - 1) * nth + j];
            double b = sys->b_node[k];
            cplx dd = sys->d_node[k];
            cplx Dphi = b * dphi / h;
            cplx Dpi = (-dd * dphi - b * dpi) / h;
            cplx F = sys->G_node ? sys->G_node[k] * phase_half : 0.0;
            cplx S_phi, S_pi;
            eval_S(avg_phi, avg_pi, j, sys, sys->kap_node[k], sys->ct_node[k], sys->W_node[k], F,
                   &S_phi, &S_pi);
            Phi_out[k] = Phi[k] - dt * (Dphi - S_phi);
            Pi_out[k] = Pi[k] - dt * (Dpi - S_pi);
            /* angular Kreiss-Oliger dissipation on u^n of this row */
            if (sys->eps != 0.0) {
                Phi_out[k] -= sys->eps / 64.0 * ko6_at(Phi + i * nth, j, nth, sys->parity);
                Pi_out[k] -= sys->eps / 64.0 * ko6_at(Pi + i * nth, j, nth, sys->parity);
            }
        }
    }
}

/* Exported generic step: every coefficient field is supplied by the caller
 * (complex fields as interleaved re/im), and eps is the Kreiss-Oliger
 * strength.  Used by tests that drive the scheme with constant coefficients,
 * where its result has a closed form. */
void oracle_lw_step_generic(int nr, int nth, int parity, double h, double dt,
                            const double *b_node, const double *b_mid,
                            const double *d_node, const double *d_mid,
                            const double *ct_node, const double *ct_mid,
                            const double *W_node, const double *W_mid,
                            const double *kap_node, const double *kap_mid,
                            const double *cot,
                            const double *G_node, const double *G_mid,
                            double phase_n_re, double phase_n_im,
                            double phase_half_re, double phase_half_im,
                            double eps,
                            const double *Phi, const double *Pi,
                            double *Phi_out, double *Pi_out)
{
    lw_system sys = {nr, nth, parity, h, ORACLE_PI / nth, dt,
                     b_node, b_mid, kap_node, kap_mid,
                     (const cplx *)d_node, (const cplx *)d_mid,
                     (const cplx *)ct_node, (const cplx *)ct_mid,
                     (const cplx *)W_node, (const cplx *)W_mid,
                     cot, G_node, G_mid, eps};
    cplx *Phi_h = malloc(sizeof(cplx) * (size_t)(nr - 1) * nth);
    cplx *Pi_h = malloc(sizeof(cplx) * (size_t)(nr - 1) * nth);
    lw_step(&sys, phase_n_re + I * phase_n_im, phase_half_re + I * phase_half_im,
            (const cplx *)Phi, (const cplx *)Pi, (cplx *)Phi_out, (cplx *)Pi_out, Phi_h, Pi_h);
    free(Phi_h);
    free(Pi_h);
}

/* ------------------------------------------------------------------------ */
/* The Teukolsky solver: grid, coefficients, source, extraction               */
/* ------------------------------------------------------------------------ */

typedef struct {
    int nr, nth, s, m, parity;
    double rstar_min, rstar_max, h, dth, dt, a;
    double *r_node, *Delta_node, *r_mid, *Delta_mid;
    double *b_node, *b_mid, *kap_node, *kap_mid, *cot;
    cplx *d_node, *d_mid, *ct_node, *ct_mid, *W_node, *W_mid;
    double *G_node, *G_mid; /* NULL: no source */
    double Omega;
    double eps;             /* Kreiss-Oliger strength, 0 unless set */
    cplx *Phi, *Pi, *Phi_n, *Pi_n, *Phi_h, *Pi_h;
    long nstep;
    /* extraction */
    int i_ext, every;
    long nsamp, cap;
    double *samp_t;
    cplx *samp_phi;
} oracle_solver;

static double rstar_node(const oracle_solver *o, int i) { return o->rstar_min + i * o->h; }
static double rstar_mid(const oracle_solver *o, int i) { return o->rstar_min + (i + 0.5) * o->h; }
static double theta_node(const oracle_solver *o, int j) { return (j + 0.5) * o->dth; }

static void fill_coefficients(const double *r, const double *Delta, int rows, const oracle_solver *o,
                              double *b, cplx *d, cplx *ct, cplx *W, double *kap)
{
    for (int i = 0; i < rows; ++i)
        for (int j = 0; j < o->nth; ++j) {
            double c[8];
            oracle_coefficients(r[i], Delta[i], theta_node(o, j), o->a, o->s, o->m, c);
            int k = i * o->nth + j;
            b[k] = c[0];
            d[k] = c[1] + I * c[2];
            ct[k] = c[3] + I * c[4];
            W[k] = c[5] + I * c[6];
            kap[k] = c[7];
        }
}

void oracle_destroy(oracle_solver *o)
{
    if (!o) return;
    free(o->r_node); free(o->Delta_node); free(o->r_mid); free(o->Delta_mid);
    free(o->b_node); free(o->b_mid); free(o->kap_node); free(o->kap_mid); free(o->cot);
    free(o->d_node); free(o->d_mid); free(o->ct_node); free(o->ct_mid);
    free(o->W_node); free(o->W_mid); free(o->G_node); free(o->G_mid);
    free(o->Phi); free(o->Pi); free(o->Phi_n); free(o->Pi_n); free(o->Phi_h); free(o->Pi_h);
    free(o->samp_t); free(o->samp_phi);
    free(o);
}

/* Returns NULL on a bad argument. */
oracle_solver *oracle_create(int nr, int nth, double rstar_min, double rstar_max, double dt,
                             double a, int s, int m)
{
    if (nr < 4 || nth < 2 || !(rstar_max > rstar_min) || !(dt > 0) || !(fabs(a) < 1.0)
        || !(s == -2 || s == 0 || s == 2))
        return NULL;
    oracle_solver *o = calloc(1, sizeof(*o));
    o->nr = nr; o->nth = nth; o->s = s; o->m = m; o->a = a; o->dt = dt;
    o->parity = (abs(m) % 2 == 0) ? 1 : -1;
    o->rstar_min = rstar_min; o->rstar_max = rstar_max;
    o->h = (rstar_max - rstar_min) / (nr - 1);
    o->dth = ORACLE_PI / nth;
    size_t nn = (size_t)nr * nth, nm = (size_t)(nr - 1) * nth;
    o->r_node = malloc(sizeof(double) * nr); o->Delta_node = malloc(sizeof(double) * nr);
    o->r_mid = malloc(sizeof(double) * (nr - 1)); o->Delta_mid = malloc(sizeof(double) * (nr - 1));
    for (int i = 0; i < nr; ++i) oracle_r_of_rstar(rstar_node(o, i), a, &o->r_node[i], &o->Delta_node[i]);
    for (int i = 0; i < nr - 1; ++i) oracle_r_of_rstar(rstar_mid(o, i), a, &o->r_mid[i], &o->Delta_mid[i]);
    o->b_node = malloc(sizeof(double) * nn); o->kap_node = malloc(sizeof(double) * nn);
    o->b_mid = malloc(sizeof(double) * nm); o->kap_mid = malloc(sizeof(double) * nm);
    o->d_node = malloc(sizeof(cplx) * nn); o->ct_node = malloc(sizeof(cplx) * nn); o->W_node = malloc(sizeof(cplx) * nn);
    o->d_mid = malloc(sizeof(cplx) * nm); o->ct_mid = malloc(sizeof(cplx) * nm); o->W_mid = malloc(sizeof(cplx) * nm);
    fill_coefficients(o->r_node, o->Delta_node, nr, o, o->b_node, o->d_node, o->ct_node, o->W_node, o->kap_node);
    fill_coefficients(o->r_mid, o->Delta_mid, nr - 1, o, o->b_mid, o->d_mid, o->ct_mid, o->W_mid, o->kap_mid);
    o->cot = malloc(sizeof(double) * nth);
    for (int j = 0; j < nth; ++j) o->cot[j] = cos(theta_node(o, j)) / sin(theta_node(o, j));
    o->Phi = calloc(nn, sizeof(cplx)); o->Pi = calloc(nn, sizeof(cplx));
    o->Phi_n = calloc(nn, sizeof(cplx)); o->Pi_n = calloc(nn, sizeof(cplx));
    o->Phi_h = calloc(nm, sizeof(cplx)); o->Pi_h = calloc(nm, sizeof(cplx));
    o->i_ext = -1;
    return o;
}

/* Initial data.  phi (and pi) are interleaved complex [nr][nth].  pi == NULL
 * selects time-symmetric data (d_t Phi = 0): Pi = b d_{r*} Phi by centred
 * differences.  The radial boundary rows are set to zero. */
int oracle_set_initial(oracle_solver *o, const double *phi, const double *pi)
{
    int nr = o->nr, nth = o->nth;
    memcpy(o->Phi, phi, sizeof(cplx) * (size_t)nr * nth);
    for (int j = 0; j < nth; ++j) { o->Phi[j] = 0.0; o->Phi[(nr - 1) * nth + j] = 0.0; }
    if (pi) {
        memcpy(o->Pi, pi, sizeof(cplx) * (size_t)nr * nth);
    } else {
        for (int i = 1; i < nr - 1; ++i)
            for (int j = 0; j < nth; ++j) {
                int k = i * nth + j;
                o->Pi[k] = o->b_node[k] * (o->Phi[k + nth] - o->Phi[k - nth]) / (2.0 * o->h);
            }
    }
    for (int j = 0; j < nth; ++j) { o->Pi[j] = 0.0; o->Pi[(nr - 1) * nth + j] = 0.0; }
    o->nstep = 0;
    o->nsamp = 0;
    return 0;
}

/* Gaussian source profile G(r*, theta) before normalisation; zero where the
 * exponent exceeds 50. */
static double gauss(double rs, double th, double rs0, double sigma, double sigma_th)
{
    double z = (rs - rs0) * (rs - rs0) / (2.0 * sigma * sigma)
             + (th - 0.5 * ORACLE_PI) * (th - 0.5 * ORACLE_PI) / (2.0 * sigma_th * sigma_th);
    return z > 50.0 ? 0.0 : exp(-z);
}

/* Point particle on a circular equatorial orbit at Boyer-Lindquist radius r0,
 * smeared into a Gaussian of width sigma (r*) and sigma/r0 (theta). */
int oracle_set_source(oracle_solver *o, double r0, double sigma, double amplitude, int prograde)
{
    double rp, rm;
    horizons(o->a, &rp, &rm);
    if (!(r0 > rp) || !(sigma > 0)) return -1;
    double rs0 = oracle_rstar_of_r(r0, o->a);
    if (!(rs0 > o->rstar_min && rs0 < o->rstar_max)) return -1;
    double sigma_th = sigma / r0;
    int nr = o->nr, nth = o->nth;
    double norm = 0.0;
    for (int i = 0; i < nr; ++i)
        for (int j = 0; j < nth; ++j)
            norm += gauss(rstar_node(o, i), theta_node(o, j), rs0, sigma, sigma_th) * o->h * o->dth;
    if (!(norm > 0)) return -1;
    free(o->G_node); free(o->G_mid);
    o->G_node = malloc(sizeof(double) * (size_t)nr * nth);
    o->G_mid = malloc(sizeof(double) * (size_t)(nr - 1) * nth);
    for (int i = 0; i < nr; ++i)
        for (int j = 0; j < nth; ++j)
            o->G_node[i * nth + j] = amplitude * gauss(rstar_node(o, i), theta_node(o, j), rs0, sigma, sigma_th) / norm;
    for (int i = 0; i < nr - 1; ++i)
        for (int j = 0; j < nth; ++j)
            o->G_mid[i * nth + j] = amplitude * gauss(rstar_mid(o, i), theta_node(o, j), rs0, sigma, sigma_th) / norm;
    o->Omega = oracle_orbit_omega(r0, o->a, prograde);
    return 0;
}

void oracle_clear_source(oracle_solver *o)
{
    free(o->G_node); free(o->G_mid);
    o->G_node = o->G_mid = NULL;
}

/* Waveform sampling: Phi on the node nearest to rstar_ext, every `every`
 * steps (after steps n with n % every == 0, n >= 1). */
int oracle_set_extraction(oracle_solver *o, double rstar_ext, int every)
{
    int i = (int)floor((rstar_ext - o->rstar_min) / o->h + 0.5);
    if (i < 0 || i >= o->nr || every < 1) return -1;
    o->i_ext = i;
    o->every = every;
    o->nsamp = 0;
    return 0;
}

/* Strength of the angular Kreiss-Oliger dissipation (0 <= eps < 2; 0, the
 * default, is the bare scheme of Eqs. 3-4). */
int oracle_set_dissipation(oracle_solver *o, double eps)
{
    if (!(eps >= 0.0 && eps < 2.0)) return -1;
    o->eps = eps;
    return 0;
}

/* e^{-i m Omega t} */
static cplx source_phase(const oracle_solver *o, double t)
{
    double ph = (double)o->m * o->Omega * t;
    return cos(ph) - I * sin(ph);
}

int oracle_step(oracle_solver *o, long nsteps)
{
    lw_system sys = {o->nr, o->nth, o->parity, o->h, o->dth, o->dt,
                     o->b_node, o->b_mid, o->kap_node, o->kap_mid,
                     o->d_node, o->d_mid, o->ct_node, o->ct_mid, o->W_node, o->W_mid,
                     o->cot, o->G_node, o->G_mid, o->eps};
    for (long k = 0; k < nsteps; ++k) {
        double t_n = (double)o->nstep * o->dt;
        double t_half = ((double)o->nstep + 0.5) * o->dt;
        cplx ph_n = o->G_node ? source_phase(o, t_n) : 0.0;
        cplx ph_h = o->G_node ? source_phase(o, t_half) : 0.0;
        lw_step(&sys, ph_n, ph_h, o->Phi, o->Pi, o->Phi_n, o->Pi_n, o->Phi_h, o->Pi_h);
        cplx *t;
        t = o->Phi; o->Phi = o->Phi_n; o->Phi_n = t;
        t = o->Pi; o->Pi = o->Pi_n; o->Pi_n = t;
        o->nstep += 1;
        if (o->i_ext >= 0 && o->nstep % o->every == 0) {
            if (o->nsamp == o->cap) {
                o->cap = o->cap ? 2 * o->cap : 64;
                o->samp_t = realloc(o->samp_t, sizeof(double) * o->cap);
                o->samp_phi = realloc(o->samp_phi, sizeof(cplx) * o->cap * o->nth);
            }
            o->samp_t[o->nsamp] = (double)o->nstep * o->dt;
            memcpy(o->samp_phi + o->nsamp * o->nth, o->Phi + (size_t)o->i_ext * o->nth,
                   sizeof(cplx) * o->nth);
            o->nsamp += 1;
        }
    }
    return 0;
}

long oracle_num_samples(const oracle_solver *o) { return o->nsamp; }
long oracle_step_count(const oracle_solver *o) { return o->nstep; }

/* Copies min(cap, nsamp) samples: t_out[k], phi_out[k][nth] (interleaved complex). */
long oracle_get_samples(const oracle_solver *o, double *t_out, double *phi_out, long cap)
{
    long n = o->nsamp < cap ? o->nsamp : cap;
    memcpy(t_out, o->samp_t, sizeof(double) * n);
    memcpy(phi_out, o->samp_phi, sizeof(cplx) * n * o->nth);
    return n;
}

int oracle_get_state(const oracle_solver *o, double *phi, double *pi)
{
    size_t nn = (size_t)o->nr * o->nth;
    if (phi) memcpy(phi, o->Phi, sizeof(cplx) * nn);
    if (pi) memcpy(pi, o->Pi, sizeof(cplx) * nn);
    return 0;
}

/* Coefficient fields of a solver, for inspection by tests.  which: 0 = nodes,
 * 1 = mid-points; out holds 8 doubles per point (same order as
 * oracle_coefficients). */
int oracle_get_coefficients(const oracle_solver *o, int which, double *out)
{
    int rows = which ? o->nr - 1 : o->nr;
    for (int k = 0; k < rows * o->nth; ++k) {
        const double *b = which ? o->b_mid : o->b_node;
        const cplx *d = which ? o->d_mid : o->d_node;
        const cplx *ct = which ? o->ct_mid : o->ct_node;
        const cplx *W = which ? o->W_mid : o->W_node;
        const double *kap = which ? o->kap_mid : o->kap_node;
        out[8 * k + 0] = b[k];
        out[8 * k + 1] = creal(d[k]); out[8 * k + 2] = cimag(d[k]);
        out[8 * k + 3] = creal(ct[k]); out[8 * k + 4] = cimag(ct[k]);
        out[8 * k + 5] = creal(W[k]); out[8 * k + 6] = cimag(W[k]);
        out[8 * k + 7] = kap[k];
    }
    return 0;
}

/* Source profile of a solver (nodes or mid-points); zeros when no source. */
int oracle_get_source_profile(const oracle_solver *o, int which, double *out)
{
    int rows = which ? o->nr - 1 : o->nr;
    const double *G = which ? o->G_mid : o->G_node;
    for (int k = 0; k < rows * o->nth; ++k) out[k] = G ? G[k] : 0.0;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Time-step rule (READING)                                                  */
/* ------------------------------------------------------------------------ */

/* dt = min(c_r h / max b, c_theta / omega_max), where omega_max^2 bounds the
 * eigenvalues of the discrete angular-plus-potential operator by Gershgorin:
 * max over nodes and mid-points of |W| + kappa (2/dth^2 + |A_j| + |C_j|),
 * A_j = 1/dth^2 + cot_j/(2 dth), C_j = 1/dth^2 - cot_j/(2 dth).  The S-part of
 * the scheme integrates these oscillations like explicit midpoint RK2, whose
 * amplification |G|^2 = 1 + (omega dt)^4 / 4 exceeds one, so c_theta sets the
 * growth per step of the stiffest mode. */
double oracle_stable_dt(int nr, int nth, double rstar_min, double rstar_max, double a, int s, int m,
                        double c_r, double c_theta)
{
    double h = (rstar_max - rstar_min) / (nr - 1);
    double dth = ORACLE_PI / nth;
    double bmax = 0.0, om2 = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
        int rows = pass ? nr - 1 : nr;
        for (int i = 0; i < rows; ++i) {
            double rs = pass ? rstar_min + (i + 0.5) * h : rstar_min + i * h;
            double r, Delta;
            oracle_r_of_rstar(rs, a, &r, &Delta);
            for (int j = 0; j < nth; ++j) {
                double th = (j + 0.5) * dth;
                double c[8];
                oracle_coefficients(r, Delta, th, a, s, m, c);
                double cot = cos(th) / sin(th);
                double A = 1.0 / (dth * dth) + cot / (2.0 * dth);
                double C = 1.0 / (dth * dth) - cot / (2.0 * dth);
                double g = hypot(c[5], c[6]) + c[7] * (2.0 / (dth * dth) + fabs(A) + fabs(C));
                if (c[0] > bmax) bmax = c[0];
                if (g > om2) om2 = g;
            }
        }
    }
    double dt_r = c_r * h / bmax;
    double dt_th = c_theta / sqrt(om2);
    return dt_r < dt_th ? dt_r : dt_th;
}
