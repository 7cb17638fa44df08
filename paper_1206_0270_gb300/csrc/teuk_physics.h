// teuk_physics.h -- Kerr background and coefficients of the first-order
// Teukolsky system, usable from host and device code of libteuk.
//
// Eq. (1) of arXiv:1206.0270 with Psi = e^{i m phi} r^3 Phi (Eq. 2), divided by
// the coefficient of d_tt, and written for u = (Phi, Pi) with
// Pi = d_t Phi + b d_{r*} Phi, reads  u_t + D u_{r*} = S  with
//   D = [[b, 0], [-d, -b]],  S = (Pi, -c_t Pi - W Phi + kappa L_theta Phi + F),
//   L_theta = d_thth + cot(theta) d_th.
// With w2 = r^2 + a^2, Delta = r^2 - 2r + a^2 (M = 1),
// Sigma^2 = w2^2 - a^2 Delta sin^2(theta), rho = dr/dr* = Delta/w2:
//   b     = w2 / Sigma,       kappa = Delta / Sigma^2,
//   c_t   = [2 s (r Delta - r^2 + a^2) + i (4 a m r + 2 s a Delta cos)] / Sigma^2,
//   c_1   = [2 r Delta + 2 s (r - 1) w2] / Sigma^2,
//   c_0   = [Delta ((m + s cos)^2 / sin^2 - s) - m^2 a^2 - 2 i s m a (r - 1)] / Sigma^2,
//   W     = c_0 - b^2 rho (3 r^2 rho)_r / r^3 - 3 c_1 rho / r,
//   d     = c_t b + 6 b^2 rho / r + c_1 - b rho b_r.
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define TEUK_HD __host__ __device__ __forceinline__
#else
#define TEUK_HD inline
#endif

namespace teuk {

struct PhysCoef {
    double b, kappa;
    double ct_re, ct_im;
    double W_re, W_im;
    double d_re, d_im;
};

TEUK_HD PhysCoef phys_coef(double r, double D, double sn, double cs, double a, int s, int m)
{
    PhysCoef c;
    const double a2 = a * a;
    const double w2 = r * r + a2;
    const double sig2 = w2 * w2 - a2 * D * sn * sn;
    const double sig = sqrt(sig2);
    const double inv_sig2 = 1.0 / sig2;
    const double b = w2 / sig;
    const double rho = D / w2;
    c.b = b;
    c.kappa = D * inv_sig2;

    const double ds = (double)s, dm = (double)m;
    c.ct_re = 2.0 * ds * (r * D - (r * r - a2)) * inv_sig2;
    c.ct_im = (4.0 * a * dm * r + 2.0 * ds * a * D * cs) * inv_sig2;
    const double c1 = (2.0 * r * D + 2.0 * ds * (r - 1.0) * w2) * inv_sig2;
    const double msc = dm + ds * cs;
    const double c0_re = (D * (msc * msc / (sn * sn) - ds) - dm * dm * a2) * inv_sig2;
    const double c0_im = -2.0 * ds * dm * a * (r - 1.0) * inv_sig2;

    // (3 r^2 rho)_r = 3 (2 r rho + r^2 rho_r),  rho_r = (2 (r - 1) w2 - 2 r Delta) / w2^2
    const double rho_r = (2.0 * (r - 1.0) * w2 - 2.0 * r * D) / (w2 * w2);
    const double d3 = 3.0 * (2.0 * r * rho + r * r * rho_r);
    c.W_re = c0_re - b * b * rho * d3 / (r * r * r) - 3.0 * c1 * rho / r;
    c.W_im = c0_im;

    // b_r = (2 r Sigma - w2 Sigma_r) / Sigma^2,  Sigma_r = (Sigma^2)_r / (2 Sigma)
    const double sig2_r = 4.0 * r * w2 - a2 * sn * sn * 2.0 * (r - 1.0);
    const double b_r = (2.0 * r * sig - w2 * sig2_r / (2.0 * sig)) * inv_sig2;
    const double e = 6.0 * b * b * rho / r + c1;
    c.d_re = c.ct_re * b + e - b * rho * b_r;
    c.d_im = c.ct_im * b;

    return c;
}

// Angular stencil of L_theta on the cell-centred grid (weights of
// Phi_{j+1}, Phi_j, Phi_{j-1}), with the pole ghosts Phi_{-1} = p Phi_0 and
// Phi_{nth} = p Phi_{nth-1} folded into the diagonal weight.
TEUK_HD void angular_weights(int j, int nth, int parity, double dth, double cot,
                             double *A, double *B, double *C)
{
    const double i2 = 1.0 / (dth * dth);
    const double c = cot / (2.0 * dth);
    double wa = i2 + c, wb = -2.0 * i2, wc = i2 - c;
    if (j == 0) { wb += parity * wc; wc = 0.0; }
    if (j == nth - 1) { wb += parity * wa; wa = 0.0; }
    *A = wa;
    *B = wb;
    *C = wc;
}

}  // namespace teuk
