// teuk_kernels.cu -- CUDA kernels of libteuk (sm_103a, FP64).
//
// Hot path: one time step of the two-step Lax-Wendroff scheme, Eqs. (3)-(4)
// of arXiv:1206.0270, for u = (Phi, Pi) on an (r*, theta) grid, with the
// point-particle source added to the Pi row and the waveform row copied to a
// ring buffer.  All constants of the scheme are folded into the coefficient
// planes built by setup_kernel (the formulas are in teuk_internal.h).  Per
// point update, the Phi rows and the sums tau, sigma take 20 FP64
// instructions (adds and multiplies issued as FMAs); the Pi rows are sums of
// 38 products evaluated in 64-bit fixed point on the integer pipes
// (teuk_fixed.h), with FP64 FMA chains as the fallback.  All on the FP64
// pipe, the step would be 56 FP64 instructions (100 flops).
//
// Default kernels: lw_predict_split / lw_correct_split, one thread per point
// over theta tiles of at most 128 columns.  The fused kernel assigns one
// thread per theta index j and lets each CTA
// march along r* over a contiguous strip of rows: the predictor value at
// i + 1/2 is computed once, used by the correctors at i and i + 1, and never
// leaves registers; the angular neighbours j +- 1 are exchanged through
// shared memory.  The only redundant work is one predictor row per strip.
#include "teuk_internal.h"
#include "teuk_physics.h"
#include "teuk_fixed.h"

#include <algorithm>

namespace teuk {

// ---------------------------------------------------------------------------
// Complex helpers: acc += c * x with FP64 FMAs
// ---------------------------------------------------------------------------

// FP64 adds and multiplies are issued as fma.rn.f64: a + b = fma(a, 1, b) and
// a * b = fma(a, b, -0) round identically, and on GB300 DFMA issues at
// 1.9/clk/SM against 1.6/clk/SM for DADD and DMUL.  The constants 1 and -0
// come from kernel parameters (Ops) so that the compiler cannot turn the FMA
// back into an add or a multiply.
struct Ops {
    double one, nzero;
};

__device__ __forceinline__ double fma_rn(double a, double b, double c)
{
    double d;
    asm("fma.rn.f64 %0, %1, %2, %3;" : "=d"(d) : "d"(a), "d"(b), "d"(c));
    return d;
}

__device__ __forceinline__ void cfma(double2 &acc, const double2 c, const double2 x)
{
    acc.x = fma(c.x, x.x, acc.x);
    acc.x = fma(-c.y, x.y, acc.x);
    acc.y = fma(c.x, x.y, acc.y);
    acc.y = fma(c.y, x.x, acc.y);
}

__device__ __forceinline__ double2 cmul(const double2 c, const double2 x, const Ops o)
{
    double2 r;
    r.x = fma_rn(c.x, x.x, o.nzero);
    r.x = fma(-c.y, x.y, r.x);
    r.y = fma_rn(c.x, x.y, o.nzero);
    r.y = fma(c.y, x.x, r.y);
    return r;
}

__device__ __forceinline__ void rfma(double2 &acc, const double c, const double2 x)
{
    acc.x = fma(c, x.x, acc.x);
    acc.y = fma(c, x.y, acc.y);
}

__device__ __forceinline__ double2 add2(const double2 a, const double2 b, const Ops o)
{
    return make_double2(fma_rn(a.x, o.one, b.x), fma_rn(a.y, o.one, b.y));
}

template <typename T>
__device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while its predecessor drains.  Everything it reads
// that an earlier kernel writes (state, half step, step counter) is read after
// grid_dependency_wait(); only the constant coefficient planes are loaded
// before.  A predecessor signals with allow_dependents() only after its last
// store, since a dependent is guaranteed to see only the writes made before
// that signal.  Without the launch attribute both instructions are no-ops.
// Loads of data that other kernels write (state, half step, step counter) in
// kernels launched with programmatic dependent launch: cached in L2 only.
// Under PDL the kernel boundary no longer guarantees that the read-only
// (L1/texture) path holds no line from before the predecessor's writes.
template <typename T>
__device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }

__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// e^{-i phase}
__device__ __forceinline__ double2 unit_phase(double ph)
{
    double s, c;
    sincos(ph, &s, &c);
    return make_double2(c, -s);
}

// ---------------------------------------------------------------------------
// Setup: coefficient planes from the radial and angular tables
// ---------------------------------------------------------------------------

// The Pi-row coefficients feed the fixed-point sums, whose coefficient split
// assumes normal numbers or exact zeros: a subnormal value (below 2^-1022,
// far below any coefficient of the scheme) is stored as zero.
__device__ __forceinline__ double normal_or_zero(double v) { return fabs(v) < 0x1p-1022 ? 0.0 : v; }
__device__ __forceinline__ double2 normal_or_zero(double2 v) { return make_double2(normal_or_zero(v.x), normal_or_zero(v.y)); }

__global__ void setup_kernel(SetupParams sp)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int nth = sp.nth;
    const long long total = (long long)(2 * sp.nr - 1) * nth;
    if (idx >= total) return;
    const int row = (int)(idx / nth);
    const int j = (int)(idx - (long long)row * nth);
    const bool mid = row >= sp.nr;
    const int i = mid ? row - sp.nr : row;
    const double r = mid ? sp.r_mid[i] : sp.r_node[i];
    const double D = mid ? sp.D_mid[i] : sp.D_node[i];
    const PhysCoef c = phys_coef(r, D, sp.sin_th[j], sp.cos_th[j], sp.a, sp.s, sp.m);
    double A, B, C;
    angular_weights(j, nth, sp.parity, sp.dth, sp.cot_th[j], &A, &B, &C);
    const double beta = sp.dt * c.b / (2.0 * sp.h);
    const double g_re = sp.dt * c.d_re / (2.0 * sp.h);
    const double g_im = sp.dt * c.d_im / (2.0 * sp.h);
    const double wr = c.W_re - c.kappa * B;  // W - kappa B (diagonal of the angular stencil)
    const double wi = c.W_im;
    const size_t k = (size_t)i * nth + j;
    if (mid) {
        const double q = 0.25 * sp.dt;
        sp.pa[k] = 0.5 + beta;
        sp.pb[k] = 0.5 - beta;
        sp.eb[k] = normal_or_zero(2.0 * beta);
        const double2 P1 = make_double2(0.5 - beta - q * c.ct_re, -q * c.ct_im);
        const double2 Q1 = make_double2(-g_re - q * wr, -g_im - q * wi);
        const double2 Q2 = make_double2(g_re - q * wr, g_im - q * wi);
        if (sp.real_coef) {
            ((double *)sp.P1)[k] = normal_or_zero(P1.x);
            ((double *)sp.Q1)[k] = normal_or_zero(Q1.x);
            ((double *)sp.Q2)[k] = normal_or_zero(Q2.x);
        } else {
            sp.P1[k] = normal_or_zero(P1);
            sp.Q1[k] = normal_or_zero(Q1);
            sp.Q2[k] = normal_or_zero(Q2);
        }
        sp.KAp[k] = normal_or_zero(q * c.kappa * A);
        sp.KCp[k] = normal_or_zero(q * c.kappa * C);
    } else {
        const double hd = 0.5 * sp.dt;
        sp.tb[k] = 2.0 * beta;
        sp.nt2[k] = normal_or_zero(-4.0 * beta);
        const double2 R1 = make_double2(2.0 * beta - hd * c.ct_re, -hd * c.ct_im);
        const double2 R3 = make_double2(2.0 * g_re - hd * wr, 2.0 * g_im - hd * wi);
        const double2 R4 = make_double2(-2.0 * g_re - hd * wr, -2.0 * g_im - hd * wi);
        if (sp.real_coef) {
            ((double *)sp.R1)[k] = normal_or_zero(R1.x);
            ((double *)sp.R3)[k] = normal_or_zero(R3.x);
            ((double *)sp.R4)[k] = normal_or_zero(R4.x);
        } else {
            sp.R1[k] = normal_or_zero(R1);
            sp.R3[k] = normal_or_zero(R3);
            sp.R4[k] = normal_or_zero(R4);
        }
        sp.KAc[k] = normal_or_zero(hd * c.kappa * A);
        sp.KCc[k] = normal_or_zero(hd * c.kappa * C);
        sp.b_node[k] = c.b;
    }
}

cudaError_t launch_setup(const SetupParams &sp, cudaStream_t st)
{
    const long long total = (long long)(2 * sp.nr - 1) * sp.nth;
    const int threads = 256;
    const long long blocks = (total + threads - 1) / threads;
    setup_kernel<<<(unsigned)blocks, threads, 0, st>>>(sp);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Predictor (Eq. 3) and corrector (Eq. 4) at one point
// ---------------------------------------------------------------------------

struct HalfStep {
    double2 phi, pi;
};

// Scheme coefficients of one predictor point (mid-point row) and one corrector
// point (node row), held in registers so that a row's loads can be issued
// one iteration ahead of their use.
struct PredCoef {
    double pa, pb, eb, KA, KC;
    double2 P1, Q1, Q2;
};
struct CorrCoef {
    double tb, nt2, KA, KC;
    double2 R1, R3, R4;
};

// REAL: P1, Q1, Q2 (and R1, R3, R4) are stored as packed real planes (the
// coefficients of a = 0, or of s = m = 0, have no imaginary part).
template <bool REAL>
__device__ __forceinline__ double2 ld_coef(const double2 *plane, size_t k)
{
    if (REAL) return make_double2(ldg((const double *)plane + k), 0.0);
    return ldg(plane + k);
}

template <bool REAL>
__device__ __forceinline__ PredCoef load_pred(const StepParams &p, size_t k)
{
    PredCoef c;
    c.pa = ldg(p.pred.pa + k);
    c.pb = ldg(p.pred.pb + k);
    c.eb = ldg(p.pred.eb + k);
    c.KA = ldg(p.pred.KA + k);
    c.KC = ldg(p.pred.KC + k);
    c.P1 = ld_coef<REAL>(p.pred.P1, k);
    c.Q1 = ld_coef<REAL>(p.pred.Q1, k);
    c.Q2 = ld_coef<REAL>(p.pred.Q2, k);
    return c;
}

template <bool REAL>
__device__ __forceinline__ CorrCoef load_corr(const StepParams &p, size_t k)
{
    CorrCoef c;
    c.tb = ldg(p.corr.tb + k);
    c.nt2 = ldg(p.corr.nt2 + k);
    c.KA = ldg(p.corr.KA + k);
    c.KC = ldg(p.corr.KC + k);
    c.R1 = ld_coef<REAL>(p.corr.R1, k);
    c.R3 = ld_coef<REAL>(p.corr.R3, k);
    c.R4 = ld_coef<REAL>(p.corr.R4, k);
    return c;
}

// acc += c x for a complex coefficient (4 FMAs), or a real one (2 FMAs)
template <bool REAL>
__device__ __forceinline__ void kfma(double2 &acc, const double2 c, const double2 x)
{
    if (REAL) rfma(acc, c.x, x); else cfma(acc, c, x);
}

template <bool REAL>
__device__ __forceinline__ double2 kmul(const double2 c, const double2 x, const Ops o)
{
    if (REAL) return make_double2(fma_rn(c.x, x.x, o.nzero), fma_rn(c.x, x.y, o.nzero));
    return cmul(c, x, o);
}

// Predictor (Eq. 3) at one mid-point.  phi0/pi0: u at row hp, phi1/pi1: u at
// row hp + 1, sup/sdn: sigma = Phi_hp + Phi_{hp+1} at j+1, j-1.
// The Phi row and the sums tau, sigma run on the FP64 pipe; the Pi row
// P1 tau + eb Pi1 + Q1 Phi0 + Q2 Phi1 + KA sup + KC sdn is a fixed-point sum
// on the integer pipe (teuk_fixed.h), with this FP64 evaluation as fallback.
template <bool REAL>
__device__ __forceinline__ double2 pred_pi_fp64(const PredCoef &c, const Ops ops, double2 tau, double2 phi0,
                                                double2 phi1, double2 pi1, double2 sup, double2 sdn)
{
    // P1 Pi_i + P2 Pi_{i+1} = P1 tau + (P2 - P1) Pi_{i+1}, tau = Pi_i + Pi_{i+1}, P2 - P1 = 2 beta (eb)
    double2 o = kmul<REAL>(c.P1, tau, ops);
    rfma(o, c.eb, pi1);
    kfma<REAL>(o, c.Q1, phi0);
    kfma<REAL>(o, c.Q2, phi1);
    rfma(o, c.KA, sup);
    rfma(o, c.KC, sdn);
    return o;
}

// FX: the Pi rows as fixed-point sums (StepParams::fixed_point, the default)
// or as FP64 FMA chains.

template <bool REAL, bool FX>
__device__ __forceinline__ double2 pred_pi(const PredCoef &c, const Ops ops, double2 tau, double2 phi0,
                                           double2 phi1, double2 pi1, double2 sup, double2 sdn)
{
    if (!FX) return pred_pi_fp64<REAL>(c, ops, tau, phi0, phi1, pi1, sup, sdn);
    const Fx tr = fx_unpack(tau.x), ti = fx_unpack(tau.y), pr = fx_unpack(pi1.x), pim = fx_unpack(pi1.y);
    const Fx ar = fx_unpack(phi0.x), ai = fx_unpack(phi0.y), br = fx_unpack(phi1.x), bi = fx_unpack(phi1.y);
    const Fx ur = fx_unpack(sup.x), ui = fx_unpack(sup.y), dr = fx_unpack(sdn.x), di = fx_unpack(sdn.y);
    const Fx P1r = fx_unpack_coef(c.P1.x), eb = fx_unpack_coef(c.eb), Q1r = fx_unpack_coef(c.Q1.x),
             Q2r = fx_unpack_coef(c.Q2.x);
    const Fx KA = fx_unpack_coef(c.KA), KC = fx_unpack_coef(c.KC);
    double2 o;
    bool ok;
    if (REAL) {
        const Fx C[6] = {P1r, eb, Q1r, Q2r, KA, KC};
        const Fx Xr[6] = {tr, pr, ar, br, ur, dr};
        const Fx Xi[6] = {ti, pim, ai, bi, ui, di};
        const uint32_t F[6] = {0, 0, 0, 0, 0, 0};
        ok = fx_dot<6>(C, Xr, F, &o.x);
        ok &= fx_dot<6>(C, Xi, F, &o.y);
    } else {
        const Fx P1i = fx_unpack_coef(c.P1.y), Q1i = fx_unpack_coef(c.Q1.y), Q2i = fx_unpack_coef(c.Q2.y);
        const Fx C[9] = {P1r, P1i, eb, Q1r, Q1i, Q2r, Q2i, KA, KC};
        const Fx Xr[9] = {tr, ti, pr, ar, ai, br, bi, ur, dr};
        const uint32_t Fr[9] = {0, 1, 0, 0, 1, 0, 1, 0, 0};
        const Fx Xi[9] = {ti, tr, pim, ai, ar, bi, br, ui, di};
        const uint32_t Fi[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        ok = fx_dot<9>(C, Xr, Fr, &o.x);
        ok &= fx_dot<9>(C, Xi, Fi, &o.y);
    }
    if (!ok) o = pred_pi_fp64<REAL>(c, ops, tau, phi0, phi1, pi1, sup, sdn);
    return o;
}

template <bool REAL, bool FX>
__device__ __forceinline__ HalfStep predict_c(const PredCoef &c, double q, const Ops ops, double2 phi0,
                                              double2 pi0, double2 phi1, double2 pi1, double2 sup, double2 sdn)
{
    HalfStep o;
    const double2 tau = add2(pi0, pi1, ops);
    o.phi = make_double2(fma_rn(c.pa, phi0.x, ops.nzero), fma_rn(c.pa, phi0.y, ops.nzero));
    rfma(o.phi, c.pb, phi1);
    rfma(o.phi, q, tau);
    o.pi = pred_pi<REAL, FX>(c, ops, tau, phi0, phi1, pi1, sup, sdn);
    return o;
}

__device__ __forceinline__ Ops ops_of(const StepParams &p) { return Ops{p.one, p.nzero}; }

template <bool REAL, bool FX>
__device__ __forceinline__ HalfStep predict(const StepParams &p, size_t k, double2 phi0, double2 pi0,
                                            double2 phi1, double2 pi1, double2 sup, double2 sdn)
{
    return predict_c<REAL, FX>(load_pred<REAL>(p, k), p.q, ops_of(p), phi0, pi0, phi1, pi1, sup, sdn);
}

// Angular Kreiss-Oliger dissipation of the corrector: pair sums
// s_q = u_{j-q} + u_{j+q} (q = 1, 2, 3) of the old state on the node's row and
// the weights k0..k3 of StepParams (formulas in teuk_internal.h).
struct KoSums {
    double2 s1, s2, s3;
};
struct KoCoef {
    double k0, k1, k2, k3, kd;
    int kd_shift;
};
__device__ __forceinline__ KoCoef ko_of(const StepParams &p)
{
    return KoCoef{p.k0, p.k1, p.k2, p.k3, p.kd, p.kd_shift};
}

// What the corrector needs of the dissipation at one node: the FP64
// kernels take the pair sums of the old Phi and Pi, the fixed-point kernels
// the exact sixth differences D6 Phi and D6 Pi (teuk_fixed.h, fx_d6).
struct KoIn {
    KoSums sphi, spi;
    double2 dphi;    // D6 Phi, rounded (it enters Phi's FP64 row)
    FxI ipr, ipi;    // D6 Pi, exact (it enters Pi's fixed-point sum unrounded)
};

// D6 of both components of entries c - 3 .. c + 3 of a row of complex
// values (raw FP64 values, prepared here).
__device__ __forceinline__ double2 ko_d6_raw(const double2 *u, int c)
{
    const double *b = (const double *)(u + c - 3);
    return make_double2(fx_d6_values(b, 2), fx_d6_values(b + 1, 2));
}

// The same from rows of values prepared once each (fx_prep): re[] and im[]
// hold the two components; identical results.
__device__ __forceinline__ double2 ko_d6_prepared(const FxP *re, const FxP *im, int c)
{
    return make_double2(fx_d6(re + c - 3), fx_d6(im + c - 3));
}

// The exact sums (unrounded) of one component of raw values u[0], u[2], ...
__device__ __forceinline__ FxI ko_d6_int_raw(const double *u)
{
    FxP q[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) q[k] = fx_prep(u[2 * k]);
    return fx_d6_int(q);
}

// The dissipation's term kd D6 of a Pi row as an addend of its fixed-point
// sum: P 2^(TP - 2103).  For eps/64 = 2^L the exact sum enters unrounded
// (P = floor(-D / 16), TP = F + L + 1028); otherwise it is D6 rounded to FP64
// times kd, formed as a product of the sum.  *bad: an input was not finite.
__device__ __forceinline__ void ko_pi_term(const FxI &d, const KoCoef &kc, long long *P, int *TP, bool *bad)
{
    *P = 0;
    *TP = -100000;
    if (d.F >= 2047) {
        *bad = true;
        return;
    }
    if (d.D == 0) return;
    if (kc.kd_shift != StepParams::kNotPow2) {
        *P = fx_sar(-d.D, 4u);
        *TP = d.F + kc.kd_shift + 1028;
    } else {
        const Fx g = fx_unpack(fx_ldexp_rn(d.D, d.F - 1079)), w = fx_unpack_coef(kc.kd);
        const long long v = (long long)fx_prod47(w, g);
        *P = (w.neg ^ g.neg) ? -v : v;
        *TP = w.e + g.e;
    }
}

// Theta index j of a row continued past the poles by the ghost rule: the
// reflection across theta = 0 maps j < 0 to -1 - j, the one across theta = pi
// maps j >= nth to 2 nth - 1 - j, each with the factor `parity`; repeated for
// rows shorter than the stencil (nth >= 2 and |offset| <= 3 need at most
// two).  Returns the grid index and sets *sign.
__device__ __forceinline__ int ko_fold(int j, int nth, int parity, double *sign)
{
    double sg = 1.0;
    for (int it = 0; it < 4 && (j < 0 || j >= nth); ++it) {
        j = j < 0 ? -1 - j : 2 * nth - 1 - j;
        sg *= (double)parity;
    }
    *sign = sg;
    return min(max(j, 0), nth - 1);
}

// Value of column j (any integer within 3 of the grid) of a row of a field
// that another kernel writes, with the ghost rule applied.
__device__ __forceinline__ double2 ko_load(const double2 *row, int j, int nth, int parity)
{
    double sg;
    const int jj = ko_fold(j, nth, parity, &sg);
    const double2 v = ldcg(row + jj);
    return make_double2(sg * v.x, sg * v.y);
}

// Pair sums around entry c of a row staged in shared memory.
__device__ __forceinline__ KoSums ko_sums(const double2 *u, int c, const Ops ops)
{
    return KoSums{add2(u[c - 1], u[c + 1], ops), add2(u[c - 2], u[c + 2], ops), add2(u[c - 3], u[c + 3], ops)};
}

// The dissipation inputs of entry c of staged rows of the old Phi and Pi
// (raw FP64 values, columns c - 3 .. c + 3 valid).
template <bool FX>
__device__ __forceinline__ KoIn ko_from_rows(const double2 *uph, const double2 *upi, int c, const Ops ops)
{
    KoIn ko{};
    if (FX) {
        ko.dphi = ko_d6_raw(uph, c);
        const double *b = (const double *)(upi + c - 3);
        ko.ipr = ko_d6_int_raw(b);
        ko.ipi = ko_d6_int_raw(b + 1);
    } else {
        ko.sphi = ko_sums(uph, c, ops);
        ko.spi = ko_sums(upi, c, ops);
    }
    return ko;
}

// Corrector (Eq. 4) at one node.  hp: half step at i + 1/2, hm: at i - 1/2,
// sup/sdn: sigma' = Phi^{i+1/2} + Phi^{i-1/2} at j+1, j-1.  As in the
// predictor, the Pi row is a fixed-point sum with an FP64 fallback.  KO adds
// the dissipation: Pi^n enters with weight k0 and kdpi = k1 s1 + k2 s2 + k3 s3
// (formed in FP64 from the pair sums of Pi^n) with weight one.
// KO with FX: kdpi is D6 Pi and k0 the weight kd = -eps/64 of it; without
// FX: kdpi = k1 s1 + k2 s2 + k3 s3 and k0 the weight of Pi.
template <bool REAL, bool FX, bool KO>
__device__ __forceinline__ double2 corr_pi_fp64(const CorrCoef &c, const Ops ops, double2 pi, double2 tau,
                                                const HalfStep &hp, const HalfStep &hm, double2 sup, double2 sdn,
                                                double k0, double2 kdpi)
{
    // R1 Pi^{+} + R2 Pi^{-} = R1 tau' + (R2 - R1) Pi^{-}, tau' = Pi^{+} + Pi^{-}, R2 - R1 = -2 tb (nt2)
    double2 npi = pi;
    if (KO && FX) npi = make_double2(fma_rn(k0, kdpi.x, pi.x), fma_rn(k0, kdpi.y, pi.y));
    if (KO && !FX) npi = make_double2(fma_rn(k0, pi.x, kdpi.x), fma_rn(k0, pi.y, kdpi.y));
    kfma<REAL>(npi, c.R1, tau);
    rfma(npi, c.nt2, hm.pi);
    kfma<REAL>(npi, c.R3, hp.phi);
    kfma<REAL>(npi, c.R4, hm.phi);
    rfma(npi, c.KA, sup);
    rfma(npi, c.KC, sdn);
    return npi;
}

template <bool REAL, bool FX, bool KO>
__device__ __forceinline__ double2 corr_pi(const CorrCoef &c, const Ops ops, double2 pi, double2 tau,
                                           const HalfStep &hp, const HalfStep &hm, double2 sup, double2 sdn,
                                           double k0, double2 kdpi, const KoIn &ko, const KoCoef &kc)
{
    if (!FX) return corr_pi_fp64<REAL, FX, KO>(c, ops, pi, tau, hp, hm, sup, sdn, k0, kdpi);
    const Fx one = fx_unpack_coef(1.0);
    const Fx c0 = one;
    const Fx pr = fx_unpack(pi.x), pim = fx_unpack(pi.y), tr = fx_unpack(tau.x), ti = fx_unpack(tau.y);
    const Fx mr = fx_unpack(hm.pi.x), mi = fx_unpack(hm.pi.y);
    const Fx ar = fx_unpack(hp.phi.x), ai = fx_unpack(hp.phi.y), br = fx_unpack(hm.phi.x), bi = fx_unpack(hm.phi.y);
    const Fx ur = fx_unpack(sup.x), ui = fx_unpack(sup.y), dr = fx_unpack(sdn.x), di = fx_unpack(sdn.y);
    const Fx R1r = fx_unpack_coef(c.R1.x), nt2 = fx_unpack_coef(c.nt2), R3r = fx_unpack_coef(c.R3.x),
             R4r = fx_unpack_coef(c.R4.x);
    const Fx KA = fx_unpack_coef(c.KA), KC = fx_unpack_coef(c.KC);
    double2 o;
    bool ok;
    if (KO) {
        // the dissipation's term kd D6 Pi, already formed (ko_pi_term)
        long long Pr, Pi_;
        int TPr, TPi;
        bool bad = false;
        ko_pi_term(ko.ipr, kc, &Pr, &TPr, &bad);
        ko_pi_term(ko.ipi, kc, &Pi_, &TPi, &bad);
        if (REAL) {
            const Fx C[7] = {c0, R1r, nt2, R3r, R4r, KA, KC};
            const Fx Xr[7] = {pr, tr, mr, ar, br, ur, dr};
            const Fx Xi[7] = {pim, ti, mi, ai, bi, ui, di};
            const uint32_t F[7] = {0, 0, 0, 0, 0, 0, 0};
            ok = fx_dot<7, true>(C, Xr, F, &o.x, Pr, TPr);
            ok &= fx_dot<7, true>(C, Xi, F, &o.y, Pi_, TPi);
        } else {
            const Fx R1i = fx_unpack_coef(c.R1.y), R3i = fx_unpack_coef(c.R3.y), R4i = fx_unpack_coef(c.R4.y);
            const Fx C[10] = {c0, R1r, R1i, nt2, R3r, R3i, R4r, R4i, KA, KC};
            const Fx Xr[10] = {pr, tr, ti, mr, ar, ai, br, bi, ur, dr};
            const uint32_t Fr[10] = {0, 0, 1, 0, 0, 1, 0, 1, 0, 0};
            const Fx Xi[10] = {pim, ti, tr, mi, ai, ar, bi, br, ui, di};
            const uint32_t Fi[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
            ok = fx_dot<10, true>(C, Xr, Fr, &o.x, Pr, TPr);
            ok &= fx_dot<10, true>(C, Xi, Fi, &o.y, Pi_, TPi);
        }
        ok &= !bad;
        if (!ok) kdpi = make_double2(fx_d6_round(ko.ipr), fx_d6_round(ko.ipi));
    } else if (REAL) {
        const Fx C[7] = {one, R1r, nt2, R3r, R4r, KA, KC};
        const Fx Xr[7] = {pr, tr, mr, ar, br, ur, dr};
        const Fx Xi[7] = {pim, ti, mi, ai, bi, ui, di};
        const uint32_t F[7] = {0, 0, 0, 0, 0, 0, 0};
        ok = fx_dot<7>(C, Xr, F, &o.x);
        ok &= fx_dot<7>(C, Xi, F, &o.y);
    } else {
        const Fx R1i = fx_unpack_coef(c.R1.y), R3i = fx_unpack_coef(c.R3.y), R4i = fx_unpack_coef(c.R4.y);
        const Fx C[10] = {one, R1r, R1i, nt2, R3r, R3i, R4r, R4i, KA, KC};
        const Fx Xr[10] = {pr, tr, ti, mr, ar, ai, br, bi, ur, dr};
        const uint32_t Fr[10] = {0, 0, 1, 0, 0, 1, 0, 1, 0, 0};
        const Fx Xi[10] = {pim, ti, tr, mi, ai, ar, bi, br, ui, di};
        const uint32_t Fi[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        ok = fx_dot<10>(C, Xr, Fr, &o.x);
        ok &= fx_dot<10>(C, Xi, Fi, &o.y);
    }
    if (!ok) o = corr_pi_fp64<REAL, FX, KO>(c, ops, pi, tau, hp, hm, sup, sdn, k0, kdpi);
    return o;
}

// k1 s1 + k2 s2 + k3 s3 of a field's pair sums
__device__ __forceinline__ double2 ko_combine(const KoCoef &kc, const KoSums &ks, const Ops ops)
{
    double2 d = make_double2(fma_rn(kc.k1, ks.s1.x, ops.nzero), fma_rn(kc.k1, ks.s1.y, ops.nzero));
    rfma(d, kc.k2, ks.s2);
    rfma(d, kc.k3, ks.s3);
    return d;
}

template <bool REAL, bool FX, bool KO>
__device__ __forceinline__ void correct_c(const CorrCoef &c, double half_dt, const Ops ops, double2 phi,
                                          double2 pi, const HalfStep &hp, const HalfStep &hm, double2 sup,
                                          double2 sdn, const KoCoef &kc, const KoIn &ko, double2 *phi_out,
                                          double2 *pi_out)
{
    const double2 tau = add2(hp.pi, hm.pi, ops);
    double2 nphi = phi;
    double2 kdpi = make_double2(0.0, 0.0);
    double kw = kc.k0;
    if (KO && FX) {
        nphi = make_double2(fma_rn(kc.kd, ko.dphi.x, phi.x), fma_rn(kc.kd, ko.dphi.y, phi.y));
        kw = kc.kd;  // kdpi (D6 Pi rounded) is formed only if the FP64 fallback needs it
    } else if (KO) {
        const double2 kd = ko_combine(kc, ko.sphi, ops);
        nphi = make_double2(fma_rn(kc.k0, phi.x, kd.x), fma_rn(kc.k0, phi.y, kd.y));
        kdpi = ko_combine(kc, ko.spi, ops);
    }
    rfma(nphi, -c.tb, hp.phi);
    rfma(nphi, c.tb, hm.phi);
    rfma(nphi, half_dt, tau);
    *phi_out = nphi;
    *pi_out = corr_pi<REAL, FX, KO>(c, ops, pi, tau, hp, hm, sup, sdn, kw, kdpi, ko, kc);
}

template <bool REAL, bool FX, bool KO>
__device__ __forceinline__ void correct(const StepParams &p, size_t k, double2 phi, double2 pi,
                                        const HalfStep &hp, const HalfStep &hm, double2 sup,
                                        double2 sdn, const KoIn &ko, double2 *phi_out, double2 *pi_out)
{
    correct_c<REAL, FX, KO>(load_corr<REAL>(p, k), p.half_dt, ops_of(p), phi, pi, hp, hm, sup, sdn, ko_of(p), ko,
                            phi_out, pi_out);
}

// ---------------------------------------------------------------------------
// Fused radial-marching step kernel
// ---------------------------------------------------------------------------

// Shared memory: sigma and sigma' double buffers, each nth + 2 entries with
// a zero ghost at both ends (their stencil weights are zero); with the
// dissipation also the row's old Phi and Pi, double-buffered, nth + 6 entries
// each (three ghost columns past each pole).
size_t fused_smem_bytes(int nth, int ko)
{
    return sizeof(double2) * (4 * (size_t)(nth + 2) + (ko ? 4 * (size_t)(nth + 6) : 0));
}
int fused_block_threads(int nth) { return ((nth + 31) / 32) * 32; }

template <bool REAL, bool FX, bool KO>
__global__ void __launch_bounds__(kFusedMaxNth) lw_step_fused(StepParams p, const double2 *__restrict__ Phi,
                                                      const double2 *__restrict__ Pi,
                                                      double2 *__restrict__ PhiO,
                                                      double2 *__restrict__ PiO, int k, int rpb)
{
    extern __shared__ double2 smem[];
    __shared__ double2 s_phase[2];
    const int nth = p.nth;
    const int W = nth + 2;
    const int KW = nth + 6;
    double2 *s_sig = smem;          // [2][W]
    double2 *s_sgh = smem + 2 * W;  // [2][W]
    double2 *s_u = smem + 4 * W;    // KO: [2][Phi, Pi][KW], entry c = column c - 3
    const int j = threadIdx.x;
    const bool act = j < nth;
    const int jj = act ? j : nth - 1;

    const int i0 = 1 + blockIdx.x * rpb;
    const int i1 = min(i0 + rpb, p.nr - 1);
    if (i0 >= i1) return;  // whole block

    if (threadIdx.x < 2) {
        const double2 z = make_double2(0.0, 0.0);
        s_sig[threadIdx.x * W] = z;
        s_sig[threadIdx.x * W + nth + 1] = z;
        s_sgh[threadIdx.x * W] = z;
        s_sgh[threadIdx.x * W + nth + 1] = z;
    }
    const long long n = *p.step_base + k;
    const SourceWindow &sw = p.src;
    const bool src_mid = sw.active && !(i1 - 1 < sw.mid_lo || i0 - 1 > sw.mid_hi);
    const bool src_node = sw.active && !(i1 - 1 < sw.node_lo || i0 > sw.node_hi);
    if (threadIdx.x == 0 && (src_mid || src_node)) {
        s_phase[0] = unit_phase(sw.m_omega * ((double)n * p.dt));
        s_phase[1] = unit_phase(sw.m_omega * (((double)n + 0.5) * p.dt));
    }
    const bool sample = p.ext.i_ext >= i0 && p.ext.i_ext < i1 && ((n + 1) % p.ext.every) == 0;

    // prologue: predictor at i0 - 1/2 from rows i0 - 1 and i0
    double2 phc = Phi[(size_t)(i0 - 1) * nth + jj], pic = Pi[(size_t)(i0 - 1) * nth + jj];
    double2 phn = Phi[(size_t)i0 * nth + jj], pin = Pi[(size_t)i0 * nth + jj];
    if (act) s_sig[j + 1] = add2(phc, phn, ops_of(p));
    __syncthreads();
    HalfStep hm = predict<REAL, FX>(p, (size_t)(i0 - 1) * nth + jj, phc, pic, phn, pin, s_sig[jj + 2], s_sig[jj]);
    if (src_mid && i0 - 1 >= sw.mid_lo && i0 - 1 <= sw.mid_hi)
        rfma(hm.pi, ldg(sw.gP + (size_t)(i0 - 1 - sw.mid_lo) * nth + jj), s_phase[0]);
    phc = phn;
    pic = pin;

    // Loads for row i are issued one iteration ahead: u_{i+1} and the
    // predictor/corrector coefficients of row i arrive while row i-1 computes.
    double2 phn_nx = Phi[(size_t)(i0 + 1) * nth + jj], pin_nx = Pi[(size_t)(i0 + 1) * nth + jj];
    PredCoef pc_nx = load_pred<REAL>(p, (size_t)i0 * nth + jj);
    CorrCoef cc_nx = load_corr<REAL>(p, (size_t)i0 * nth + jj);
    int buf = 1;
    for (int i = i0; i < i1; ++i) {
        phn = phn_nx;
        pin = pin_nx;
        const PredCoef pc = pc_nx;
        const CorrCoef cc = cc_nx;
        {
            const int inx = min(i + 1, i1 - 1);  // clamped: the last prefetch is unused
            const int unx = min(i + 2, p.nr - 1);
            phn_nx = Phi[(size_t)unx * nth + jj];
            pin_nx = Pi[(size_t)unx * nth + jj];
            pc_nx = load_pred<REAL>(p, (size_t)inx * nth + jj);
            cc_nx = load_corr<REAL>(p, (size_t)inx * nth + jj);
        }
        double2 *sg = s_sig + buf * W;
        if (act) sg[j + 1] = add2(phc, phn, ops_of(p));
        double2 *uph = s_u + buf * 2 * KW, *upi = uph + KW;
        if (KO && act) {
            uph[j + 3] = phc;
            upi[j + 3] = pic;
        }
        __syncthreads();
        if (KO && threadIdx.x < 6) {  // ghost columns -3..-1 and nth..nth+2, from the row itself
            const int e = threadIdx.x < 3 ? threadIdx.x : nth + threadIdx.x;
            double sgn;
            const int jg = ko_fold(e - 3, nth, p.parity, &sgn);
            uph[e] = make_double2(sgn * uph[jg + 3].x, sgn * uph[jg + 3].y);
            upi[e] = make_double2(sgn * upi[jg + 3].x, sgn * upi[jg + 3].y);
        }
        HalfStep hp = predict_c<REAL, FX>(pc, p.q, ops_of(p), phc, pic, phn, pin, sg[jj + 2], sg[jj]);
        if (src_mid && i >= sw.mid_lo && i <= sw.mid_hi)
            rfma(hp.pi, ldg(sw.gP + (size_t)(i - sw.mid_lo) * nth + jj), s_phase[0]);

        double2 *sh = s_sgh + buf * W;
        if (act) sh[j + 1] = add2(hp.phi, hm.phi, ops_of(p));
        __syncthreads();
        const size_t kc = (size_t)i * nth + jj;
        double2 nphi, npi;
        KoIn ko{};
        if (KO) ko = ko_from_rows<FX>(uph, upi, jj + 3, ops_of(p));
        correct_c<REAL, FX, KO>(cc, p.half_dt, ops_of(p), phc, pic, hp, hm, sh[jj + 2], sh[jj], ko_of(p), ko, &nphi,
                                &npi);
        if (src_node && i >= sw.node_lo && i <= sw.node_hi)
            rfma(npi, ldg(sw.gC + (size_t)(i - sw.node_lo) * nth + jj), s_phase[1]);
        if (act) {
            PhiO[kc] = nphi;
            PiO[kc] = npi;
            if (sample && i == p.ext.i_ext) {
                const long long slot = ((n + 1) / p.ext.every - 1) % p.ext.capacity;
                p.ext.ring[(size_t)slot * nth + j] = nphi;
            }
        }
        hm = hp;
        phc = phn;
        pic = pin;
        buf ^= 1;
    }
}

// The four instantiations of a step kernel (real or complex coefficient
// planes, fixed-point or FP64 Pi rows) share one signature; TEUK_PICK3 adds
// the dissipation flag of corrector kernels.
#define TEUK_PICK(K, real, fx) ((real) ? ((fx) ? K<true, true> : K<true, false>) : ((fx) ? K<false, true> : K<false, false>))
#define TEUK_PICK3(K, real, fx, ko)                                                                            \
    ((ko) ? ((real) ? ((fx) ? K<true, true, true> : K<true, false, true>)                                      \
                    : ((fx) ? K<false, true, true> : K<false, false, true>))                                   \
          : ((real) ? ((fx) ? K<true, true, false> : K<true, false, false>)                                    \
                    : ((fx) ? K<false, true, false> : K<false, false, false>)))

const void *fused_kernel_ptr(int real, int fixed_point, int ko)
{
    return (const void *)TEUK_PICK3(lw_step_fused, real, fixed_point, ko);
}

cudaError_t launch_step_fused(const StepParams &p, const double2 *Phi, const double2 *Pi,
                              double2 *PhiO, double2 *PiO, int k, int rows_per_block, int nblocks,
                              cudaStream_t st)
{
    const int threads = fused_block_threads(p.nth);
    TEUK_PICK3(lw_step_fused, p.real_coef, p.fixed_point, p.ko)<<<nblocks, threads, fused_smem_bytes(p.nth, p.ko),
                                                                 st>>>(p, Phi, Pi, PhiO, PiO, k, rows_per_block);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Two-kernel variant: predictor writes the half-step fields to device memory
// ---------------------------------------------------------------------------

template <bool REAL, bool FX>
__global__ void lw_predict_kernel(StepParams p, const double2 *__restrict__ Phi,
                                  const double2 *__restrict__ Pi, double2 *__restrict__ PhiH,
                                  double2 *__restrict__ PiH, int k)
{
    const int nth = p.nth;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)(p.nr - 1) * nth) return;
    const int hp = (int)(idx / nth);
    const int j = (int)(idx - (long long)hp * nth);
    const size_t k0 = (size_t)hp * nth + j, k1 = k0 + nth;
    const double2 phi0 = Phi[k0], pi0 = Pi[k0], phi1 = Phi[k1], pi1 = Pi[k1];
    const int ju = j + 1 < nth ? j + 1 : j, jd = j > 0 ? j - 1 : j;  // edge weights are zero
    const size_t r0 = (size_t)hp * nth, r1 = r0 + nth;
    const double2 sup = add2(Phi[r0 + ju], Phi[r1 + ju], ops_of(p));
    const double2 sdn = add2(Phi[r0 + jd], Phi[r1 + jd], ops_of(p));
    HalfStep o = predict<REAL, FX>(p, k0, phi0, pi0, phi1, pi1, sup, sdn);
    const SourceWindow &sw = p.src;
    if (sw.active && hp >= sw.mid_lo && hp <= sw.mid_hi) {
        const long long n = *p.step_base + k;
        rfma(o.pi, sw.gP[(size_t)(hp - sw.mid_lo) * nth + j], unit_phase(sw.m_omega * ((double)n * p.dt)));
    }
    PhiH[k0] = o.phi;
    PiH[k0] = o.pi;
}

template <bool REAL, bool FX, bool KO>
__global__ void lw_correct_kernel(StepParams p, const double2 *__restrict__ Phi,
                                  const double2 *__restrict__ Pi, const double2 *__restrict__ PhiH,
                                  const double2 *__restrict__ PiH, double2 *__restrict__ PhiO,
                                  double2 *__restrict__ PiO, int k)
{
    const int nth = p.nth;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)(p.nr - 2) * nth) return;
    const int i = 1 + (int)(idx / nth);
    const int j = (int)(idx - (long long)(i - 1) * nth);
    const size_t kc = (size_t)i * nth + j;
    const size_t kp = kc, km = kc - nth;  // half-step rows i (i+1/2) and i-1 (i-1/2)
    HalfStep hp, hm;
    hp.phi = PhiH[kp];
    hp.pi = PiH[kp];
    hm.phi = PhiH[km];
    hm.pi = PiH[km];
    const int ju = j + 1 < nth ? j + 1 : j, jd = j > 0 ? j - 1 : j;
    const double2 sup = add2(PhiH[kp - j + ju], PhiH[km - j + ju], ops_of(p));
    const double2 sdn = add2(PhiH[kp - j + jd], PhiH[km - j + jd], ops_of(p));
    double2 nphi, npi;
    KoIn ko{};
    if (KO) {  // the old state along the row, columns j-3 .. j+3, ghosts by the pole rule
        const double2 *rp = Phi + (size_t)i * nth, *rq = Pi + (size_t)i * nth;
        double2 a[7], b[7];
        for (int q = 0; q < 7; ++q) {
            a[q] = ko_load(rp, j - 3 + q, nth, p.parity);
            b[q] = ko_load(rq, j - 3 + q, nth, p.parity);
        }
        ko = ko_from_rows<FX>(a, b, 3, ops_of(p));
    }
    correct<REAL, FX, KO>(p, kc, Phi[kc], Pi[kc], hp, hm, sup, sdn, ko, &nphi, &npi);
    const long long n = *p.step_base + k;
    const SourceWindow &sw = p.src;
    if (sw.active && i >= sw.node_lo && i <= sw.node_hi)
        rfma(npi, sw.gC[(size_t)(i - sw.node_lo) * nth + j],
             unit_phase(sw.m_omega * (((double)n + 0.5) * p.dt)));
    PhiO[kc] = nphi;
    PiO[kc] = npi;
    if (i == p.ext.i_ext && ((n + 1) % p.ext.every) == 0) {
        const long long slot = ((n + 1) / p.ext.every - 1) % p.ext.capacity;
        p.ext.ring[(size_t)slot * nth + j] = nphi;
    }
}

cudaError_t launch_step_unfused(const StepParams &p, const double2 *Phi, const double2 *Pi,
                                double2 *PhiO, double2 *PiO, double2 *PhiH, double2 *PiH, int k,
                                cudaStream_t st, int part)
{
    const int threads = 256;
    const long long np = (long long)(p.nr - 1) * p.nth, nc = (long long)(p.nr - 2) * p.nth;
    if (part != 1)
        TEUK_PICK(lw_predict_kernel, p.real_coef, p.fixed_point)<<<(unsigned)((np + threads - 1) / threads), threads,
                                                                    0, st>>>(p, Phi, Pi, PhiH, PiH, k);
    if (part != 0)
        TEUK_PICK3(lw_correct_kernel, p.real_coef, p.fixed_point, p.ko)<<<(unsigned)((nc + threads - 1) / threads),
                                                                           threads, 0, st>>>(p, Phi, Pi, PhiH, PiH,
                                                                                             PhiO, PiO, k);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Split variant: predictor and corrector as two kernels over 2D tiles of
// R rows x nth columns (one point per thread); sigma is formed once per point
// and shared with the angular neighbours through shared memory.
// ---------------------------------------------------------------------------

// Split tiles: TW theta columns (16 for rows of at most 16 columns, else a
// multiple of 32, at most 128) by R r* rows,
// one thread per point.  Rows wider than a tile are cut into tiles of TW
// columns, the last one ragged; each tile forms its two halo sums
// sigma(j0 - 1) and sigma(j0 + TW) itself.  Small CTAs keep several tiles
// resident per SM (the fixed-point Pi rows need up to 128 registers per
// thread).
constexpr int kSplitTileMax = 128;  // widest theta tile of the split kernels
// Tile width for rows of nth columns, at most max_width: 16 for nth <= 16,
// otherwise the multiple of 32
// (at least 64 unless nth <= 32) that wastes the fewest lanes in the ragged
// last tile, less a penalty of 0.02 per 32 columns below 128 for the extra
// halo sums and rows of narrower tiles.  Measured on GB300: 32000 x 304 runs
// at 11.5 G updates/s with 64-column tiles (95% of lanes busy) against 9.5
// with 128-column tiles (79%); 8192 x 128 at 11.9 with 128 against 11.5
// with 64 (both 100%).
int tile_width_for(int nth, int max_width)
{
    if (nth <= 16) return 16;  // half-warp rows: 8 rows per 128-thread tile, no idle lanes
    if (nth <= 32 || max_width < 64) return 32;
    int best = 64;
    double best_score = -1.0;
    for (int tw = max_width / 32 * 32; tw >= 64; tw -= 32) {
        const int lanes = (nth + tw - 1) / tw * tw;
        const double score = (double)nth / lanes - (tw < 128 ? 0.02 * (128 - tw) / 32 : 0.0);
        if (score > best_score + 1e-12) {  // ties keep the wider tile
            best = tw;
            best_score = score;
        }
    }
    return best;
}
int split_tile_width(int nth) { return tile_width_for(nth, kSplitTileMax); }
int split_theta_tiles(int nth)
{
    const int tw = split_tile_width(nth);
    return (nth + tw - 1) / tw;
}
// Default tile height: 128-thread CTAs for the fixed-point kernels (the most
// their launch bounds allow), 256-thread CTAs for the FP64 ones.
int split_rows_per_block(int nth, int fixed_point)
{
    const int tw = split_tile_width(nth);
    const int threads = fixed_point ? kFxTileThreads : 2 * kFxTileThreads;
    return tw >= threads ? 1 : threads / tw;
}

// Launch bounds of the split kernels.
//  - Fixed point (FX): CTAs of at most 128 threads, at least five resident
//    per SM.  ptxas then keeps the kernels at 96 registers (about 30 bytes of
//    spills) instead of 122-126, and an SM holds 20 warps instead of 16.
//    Measured on GB300: 12.32 against 12.15 G updates/s on 8192 x 128, 12.54
//    against 12.01 on 32768 x 512, same box and clock.
//  - FP64: the single-argument 1024-thread bound keeps them at 64 registers;
//    the two-argument form (1024, 1) made them 7% slower (10.07 -> 9.36).
#define TEUK_SPLIT_BOUNDS_FX __launch_bounds__(kFxTileThreads, kFxTileMinBlocks)
#define TEUK_SPLIT_BOUNDS_FP64 __launch_bounds__(1024)

// Where a thread sits in a split tile: tile width TW and height R (TW R
// threads), its column tx and row ty, and the tile's r* row block rb and
// theta tile tt.  The split kernels take it from their launch shape; the
// multi-job kernels from the job table.
struct TileIdx {
    int TW, R, tx, ty, rb, tt;
    int sbuf;  // offset (double2 words) of the tile's shared rows in the dynamic shared memory
};
__device__ __forceinline__ TileIdx tile_of_launch()
{
    return TileIdx{(int)blockDim.x, (int)blockDim.y, (int)threadIdx.x, (int)threadIdx.y, (int)blockIdx.x,
                   (int)blockIdx.y, 0};
}

// SIGNAL: end with the programmatic-launch signal (the multi-job kernels
// signal once, after their last tile).
template <bool REAL, bool FX, bool SIGNAL = true>
__device__ __forceinline__ void predict_split_tile(const TileIdx &ti, const StepParams &p, const double2 *__restrict__ Phi,
                                                   const double2 *__restrict__ Pi, double2 *__restrict__ PhiH,
                                                   double2 *__restrict__ PiH, int k)
{
    extern __shared__ double2 smem_all[];
    double2 *smem = smem_all + ti.sbuf;
    const int nth = p.nth, TW = ti.TW, tx = ti.tx;
    const int j0 = ti.tt * TW, j = j0 + tx;
    const bool colok = j < nth;
    const int jj = colok ? j : nth - 1;
    const int hp = ti.rb * ti.R + ti.ty;
    const bool rowok = hp < p.nr - 1;
    const int hq = rowok ? hp : p.nr - 2;
    double2 *row = smem + ti.ty * (TW + 2);
    const size_t k0 = (size_t)hq * nth + jj;
    const PredCoef c = load_pred<REAL>(p, k0);
    grid_dependency_wait();
    const double2 phi0 = ldcg(Phi + k0), pi0 = ldcg(Pi + k0), phi1 = ldcg(Phi + k0 + nth), pi1 = ldcg(Pi + k0 + nth);
    const Ops ops = ops_of(p);
    row[tx + 1] = colok ? add2(phi0, phi1, ops) : make_double2(0.0, 0.0);
    // halo sums from the neighbouring tiles; zero at the poles (the ghost
    // values are folded into the coefficients) and past the last column
    const size_t kr = (size_t)hq * nth;
    if (tx == 0)
        row[0] = j0 > 0 ? add2(ldcg(Phi + kr + j0 - 1), ldcg(Phi + kr + nth + j0 - 1), ops) : make_double2(0.0, 0.0);
    if (tx == TW - 1)
        row[TW + 1] = j0 + TW < nth ? add2(ldcg(Phi + kr + j0 + TW), ldcg(Phi + kr + nth + j0 + TW), ops)
                                    : make_double2(0.0, 0.0);
    __syncthreads();
    HalfStep o = predict_c<REAL, FX>(c, p.q, ops, phi0, pi0, phi1, pi1, row[tx + 2], row[tx]);
    const SourceWindow &sw = p.src;
    if (sw.active && hq >= sw.mid_lo && hq <= sw.mid_hi) {
        const long long n = ldcg(p.step_base) + k;
        rfma(o.pi, ldg(sw.gP + (size_t)(hq - sw.mid_lo) * nth + jj), unit_phase(sw.m_omega * ((double)n * p.dt)));
    }
    if (colok && rowok) {
        PhiH[k0] = o.phi;
        PiH[k0] = o.pi;
    }
    if (SIGNAL) allow_dependents();  // after the last store: the dependent sees only writes made before it
}

template <bool REAL, bool FX, bool KO, bool SIGNAL = true>
__device__ __forceinline__ void correct_split_tile(const TileIdx &ti, const StepParams &p, const double2 *__restrict__ Phi,
                                                   const double2 *__restrict__ Pi, const double2 *__restrict__ PhiH,
                                                   const double2 *__restrict__ PiH, double2 *__restrict__ PhiO,
                                                   double2 *__restrict__ PiO, int k)
{
    extern __shared__ double2 smem_all[];
    double2 *smem = smem_all + ti.sbuf;
    const int nth = p.nth, TW = ti.TW, tx = ti.tx;
    const int j0 = ti.tt * TW, j = j0 + tx;
    const bool colok = j < nth;
    const int jj = colok ? j : nth - 1;
    const int i = 1 + ti.rb * ti.R + ti.ty;
    const bool rowok = i <= p.nr - 2;
    const int iq = rowok ? i : p.nr - 2;
    double2 *row = smem + ti.ty * (TW + 2);
    const size_t kc = (size_t)iq * nth + jj;
    const CorrCoef c = load_corr<REAL>(p, kc);
    grid_dependency_wait();
    HalfStep hp, hm;
    hp.phi = ldcg(PhiH + kc);
    hp.pi = ldcg(PiH + kc);
    hm.phi = ldcg(PhiH + kc - nth);
    hm.pi = ldcg(PiH + kc - nth);
    const double2 phi = ldcg(Phi + kc), pi = ldcg(Pi + kc);
    const Ops ops = ops_of(p);
    row[tx + 1] = colok ? add2(hp.phi, hm.phi, ops) : make_double2(0.0, 0.0);
    const size_t kr = (size_t)iq * nth;
    if (tx == 0)
        row[0] = j0 > 0 ? add2(ldcg(PhiH + kr + j0 - 1), ldcg(PhiH + kr - nth + j0 - 1), ops) : make_double2(0.0, 0.0);
    if (tx == TW - 1)
        row[TW + 1] = j0 + TW < nth ? add2(ldcg(PhiH + kr + j0 + TW), ldcg(PhiH + kr - nth + j0 + TW), ops)
                                    : make_double2(0.0, 0.0);
    // dissipation: the row's old Phi and Pi over columns j0 - 3 .. j0 + TW + 2
    // (entry c = column j0 - 3 + c), past the poles by the ghost rule; lanes
    // past the last column hold ghost values too.  FP64 kernels stage the
    // values; fixed-point kernels stage each component prepared once for the
    // exact sixth difference (fx_prep: Phi re, Phi im, Pi re, Pi im rows).
    const int KW = TW + 6;
    double2 *uph = smem + ti.R * (TW + 2) + ti.ty * 2 * KW, *upi = uph + KW;
    FxP *kp = (FxP *)(smem + ti.R * (TW + 2)) + ti.ty * 4 * KW;
    auto stage = [&](int e, double2 a, double2 b) {
        if (FX) {
            kp[e] = fx_prep(a.x);
            kp[KW + e] = fx_prep(a.y);
            kp[2 * KW + e] = fx_prep(b.x);
            kp[3 * KW + e] = fx_prep(b.y);
        } else {
            uph[e] = a;
            upi[e] = b;
        }
    };
    if (KO) {
        const double2 *rp = Phi + kr, *rq = Pi + kr;
        // Fast staging when every ghost column of the window reflects a column
        // of this tile (rows of at least 6 columns whose last tile has at least
        // 3): the owners write the ghosts (the reflection flips the sign for
        // odd |m|) and only halo columns inside the row are loaded.  Otherwise
        // the edge lanes fold every halo column by the pole rule.
        const bool last = j0 + TW >= nth;
        const bool fast = nth >= 6 && (last ? j0 <= nth - 3 : j0 + TW + 3 <= nth);
        if (fast) {
            if (colok) {
                stage(tx + 3, phi, pi);
                const double2 gph = make_double2(p.parity * phi.x, p.parity * phi.y);
                const double2 gpi = make_double2(p.parity * pi.x, p.parity * pi.y);
                if (j0 == 0 && j <= 2) stage(2 - j, gph, gpi);                      // column -1 - j
                if (last && j >= nth - 3) stage(2 * nth - 1 - j - j0 + 3, gph, gpi);  // column 2 nth - 1 - j
            }
            if (j0 > 0 && tx < 3) stage(tx, ldcg(rp + j0 - 3 + tx), ldcg(rq + j0 - 3 + tx));
            if (!last && tx >= TW - 3) stage(tx + 6, ldcg(rp + j + 3), ldcg(rq + j + 3));
        } else {
            if (colok)
                stage(tx + 3, phi, pi);
            else
                stage(tx + 3, ko_load(rp, j, nth, p.parity), ko_load(rq, j, nth, p.parity));
            if (tx < 3) stage(tx, ko_load(rp, j0 - 3 + tx, nth, p.parity), ko_load(rq, j0 - 3 + tx, nth, p.parity));
            if (tx >= TW - 3) stage(tx + 6, ko_load(rp, j + 3, nth, p.parity), ko_load(rq, j + 3, nth, p.parity));
        }
    }
    __syncthreads();
    double2 nphi, npi;
    KoIn ko{};
    if (KO && FX) {
        ko.dphi = ko_d6_prepared(kp, kp + KW, tx + 3);
        ko.ipr = fx_d6_int(kp + 2 * KW + tx);
        ko.ipi = fx_d6_int(kp + 3 * KW + tx);
    } else if (KO) {
        ko.sphi = ko_sums(uph, tx + 3, ops);
        ko.spi = ko_sums(upi, tx + 3, ops);
    }
    correct_c<REAL, FX, KO>(c, p.half_dt, ops, phi, pi, hp, hm, row[tx + 2], row[tx], ko_of(p), ko, &nphi, &npi);
    const long long n = ldcg(p.step_base) + k;
    const SourceWindow &sw = p.src;
    if (sw.active && iq >= sw.node_lo && iq <= sw.node_hi)
        rfma(npi, ldg(sw.gC + (size_t)(iq - sw.node_lo) * nth + jj),
             unit_phase(sw.m_omega * (((double)n + 0.5) * p.dt)));
    if (colok && rowok) {
        PhiO[kc] = nphi;
        PiO[kc] = npi;
        if (iq == p.ext.i_ext && ((n + 1) % p.ext.every) == 0) {
            const long long slot = ((n + 1) / p.ext.every - 1) % p.ext.capacity;
            p.ext.ring[(size_t)slot * nth + j] = nphi;
        }
    }
    if (SIGNAL) allow_dependents();  // after the last store
}

// The split kernels, one instantiation per (REAL, FX) -- and for the
// corrector per dissipation flag -- with the launch bounds of their
// arithmetic (FX: TEUK_SPLIT_BOUNDS_FX, FP64: TEUK_SPLIT_BOUNDS_FP64).
template <bool REAL, bool FX>
__global__ void lw_predict_split(StepParams p, const double2 *__restrict__ Phi, const double2 *__restrict__ Pi,
                                 double2 *__restrict__ PhiH, double2 *__restrict__ PiH, int k);
template <bool REAL, bool FX, bool KO>
__global__ void lw_correct_split(StepParams p, const double2 *__restrict__ Phi, const double2 *__restrict__ Pi,
                                 const double2 *__restrict__ PhiH, const double2 *__restrict__ PiH,
                                 double2 *__restrict__ PhiO, double2 *__restrict__ PiO, int k);

#define TEUK_SPLIT_PREDICT(REAL, FX, BOUNDS)                                                                  \
    template <>                                                                                             \
    __global__ void BOUNDS lw_predict_split<REAL, FX>(StepParams p, const double2 *__restrict__ Phi,         \
                                                      const double2 *__restrict__ Pi,                        \
                                                      double2 *__restrict__ PhiH, double2 *__restrict__ PiH, \
                                                      int k)                                                 \
    {                                                                                                       \
        predict_split_tile<REAL, FX>(tile_of_launch(), p, Phi, Pi, PhiH, PiH, k);                                             \
    }
#define TEUK_SPLIT_CORRECT(REAL, FX, KO, BOUNDS)                                                              \
    template <>                                                                                             \
    __global__ void BOUNDS lw_correct_split<REAL, FX, KO>(                                                   \
        StepParams p, const double2 *__restrict__ Phi, const double2 *__restrict__ Pi,                        \
        const double2 *__restrict__ PhiH, const double2 *__restrict__ PiH, double2 *__restrict__ PhiO,        \
        double2 *__restrict__ PiO, int k)                                                                    \
    {                                                                                                       \
        correct_split_tile<REAL, FX, KO>(tile_of_launch(), p, Phi, Pi, PhiH, PiH, PhiO, PiO, k);                              \
    }
TEUK_SPLIT_PREDICT(false, true, TEUK_SPLIT_BOUNDS_FX)
TEUK_SPLIT_PREDICT(true, true, TEUK_SPLIT_BOUNDS_FX)
TEUK_SPLIT_PREDICT(false, false, TEUK_SPLIT_BOUNDS_FP64)
TEUK_SPLIT_PREDICT(true, false, TEUK_SPLIT_BOUNDS_FP64)
TEUK_SPLIT_CORRECT(false, true, false, TEUK_SPLIT_BOUNDS_FX)
TEUK_SPLIT_CORRECT(true, true, false, TEUK_SPLIT_BOUNDS_FX)
TEUK_SPLIT_CORRECT(false, false, false, TEUK_SPLIT_BOUNDS_FP64)
TEUK_SPLIT_CORRECT(true, false, false, TEUK_SPLIT_BOUNDS_FP64)
TEUK_SPLIT_CORRECT(false, true, true, TEUK_SPLIT_BOUNDS_FX)
TEUK_SPLIT_CORRECT(true, true, true, TEUK_SPLIT_BOUNDS_FX)
TEUK_SPLIT_CORRECT(false, false, true, TEUK_SPLIT_BOUNDS_FP64)
TEUK_SPLIT_CORRECT(true, false, true, TEUK_SPLIT_BOUNDS_FP64)
#undef TEUK_SPLIT_PREDICT
#undef TEUK_SPLIT_CORRECT

// Shared memory of a split CTA: R rows of TW + 2 sums; the corrector with
// dissipation adds R rows of the old Phi and Pi, TW + 6 entries each (as four
// rows of prepared components, 16 bytes each, in the fixed-point kernels).
size_t split_smem_bytes(int nth, int rows, int ko)
{
    const size_t R = rows > 0 ? rows : split_rows_per_block(nth, 1), TW = split_tile_width(nth);
    static_assert(sizeof(FxP) == sizeof(double2), "prepared components take 16 bytes");
    return sizeof(double2) * (R * (TW + 2) + (ko ? 4 * R * (TW + 6) : 0));
}
const void *split_kernel_ptr(int which, int real, int fixed_point, int ko)
{
    return which ? (const void *)TEUK_PICK3(lw_correct_split, real, fixed_point, ko)
                 : (const void *)TEUK_PICK(lw_predict_split, real, fixed_point);
}

// part: 0 = predictor only, 1 = corrector only, 2 = both.  rows: r* rows per
// CTA tile (0 = 256 / nth rounded to warps, at least 1).
// Let kernel fn take `bytes` of dynamic shared memory: above the 48 KB default
// a kernel launches only after its limit is raised (FP64 tiles of many rows
// with the dissipation's staged rows; the persistent multi-job form's two
// sets of rows).
static cudaError_t allow_smem(const void *fn, size_t bytes)
{
    if (bytes <= 48u * 1024u) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_step_split(const StepParams &p, const double2 *Phi, const double2 *Pi, double2 *PhiO,
                              double2 *PiO, double2 *PhiH, double2 *PiH, int k, cudaStream_t st, bool pdl,
                              int part, int rows)
{
    int R = rows > 0 ? rows : split_rows_per_block(p.nth, p.fixed_point);
    // a height set for FP64 tiles may exceed what the fixed-point kernels launch with
    if (p.fixed_point && R * split_tile_width(p.nth) > kFxTileThreads)
        R = std::max(1, kFxTileThreads / split_tile_width(p.nth));
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    const int TW = split_tile_width(p.nth), tiles = split_theta_tiles(p.nth);
    cfg.blockDim = dim3(TW, R);
    cfg.dynamicSmemBytes = split_smem_bytes(p.nth, R, 0);
    cfg.stream = st;
    cfg.attrs = pdl ? attr : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaError_t e = cudaSuccess;
    if (part != 1) {
        cfg.gridDim = dim3((p.nr - 1 + R - 1) / R, tiles);
        e = allow_smem(split_kernel_ptr(0, p.real_coef, p.fixed_point, p.ko), cfg.dynamicSmemBytes);
        if (e != cudaSuccess) return e;
        e = cudaLaunchKernelEx(&cfg, TEUK_PICK(lw_predict_split, p.real_coef, p.fixed_point), p, Phi, Pi, PhiH, PiH,
                               k);
        if (e != cudaSuccess) return e;
    }
    if (part != 0) {
        cfg.gridDim = dim3((p.nr - 2 + R - 1) / R, tiles);
        cfg.dynamicSmemBytes = split_smem_bytes(p.nth, R, p.ko);
        e = allow_smem(split_kernel_ptr(1, p.real_coef, p.fixed_point, p.ko), cfg.dynamicSmemBytes);
        if (e != cudaSuccess) return e;
        e = cudaLaunchKernelEx(&cfg, TEUK_PICK3(lw_correct_split, p.real_coef, p.fixed_point, p.ko), p, Phi, Pi,
                               (const double2 *)PhiH, (const double2 *)PiH, PhiO, PiO, k);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Multi-job split kernels: one launch covers the tiles of many jobs
// ---------------------------------------------------------------------------

// A template bank is many independent evolutions of uneven size; a single
// job of a small grid cannot fill the GPU, and one launch per job per kernel
// leaves the GPU waiting on launches.  These kernels run the split kernels'
// tile code (predict_split_tile / correct_split_tile, so every job gets the
// bits it gets alone) for the tiles of up to kMultiMaxJobs jobs in one
// launch.  The jobs' parameters sit in the kernel's parameter space
// (MultiArgs, __grid_constant__): a CTA reads them through the constant
// cache, as the split kernels read theirs.
//
// CTA b works on tiles b, b + G, b + 2G, ... (G = gridDim.x): a single tile
// when the grid has one CTA per tile, a persistent loop when the grid is
// capped at the CTAs the GPU holds at once.  A CTA visits tiles in
// increasing order, so its job index only moves forward.

int multi_tile_width(int nth, int block)
{
    int best = 32;
    double best_score = -1.0;
    for (int tw = 128; tw >= 16; tw /= 2) {
        if (tw > block || block % tw) continue;
        const int lanes = (nth + tw - 1) / tw * tw;
        const double score = (double)nth / lanes - (tw < 128 ? 0.02 * (128 - tw) / 32 : 0.0);
        if (score > best_score + 1e-12) {  // ties keep the wider tile
            best = tw;
            best_score = score;
        }
    }
    return best;
}

size_t multi_smem_bytes(int tw, int block, int ko)
{
    const size_t R = (size_t)block / tw;
    return sizeof(double2) * (R * (tw + 2) + (ko ? 4 * R * (tw + 6) : 0));
}

// First job of tile b: the largest q with off[q] <= b.
__device__ __forceinline__ int multi_first_job(const MultiArgs &a, int b)
{
    int lo = 0, hi = a.njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.off[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ TileIdx multi_tile(const JobDesc &J, int t, int sbuf)
{
    const int tw = J.tw, tiles = J.tiles, rb = t / tiles;
    const int ty = (int)threadIdx.x / tw;
    return TileIdx{tw, J.rows, (int)threadIdx.x - ty * tw, ty, rb, t - rb * tiles, sbuf};
}

// PERSIST: loop over tiles b, b + G, ..., alternating two sets of shared
// rows (a.sbuf_words apart): the tile code's own barrier keeps every warp
// within one tile of the others, so a warp that starts the next tile never
// overwrites rows another warp still reads, and no barrier is needed between
// tiles.  Otherwise the grid has one CTA per tile (fewer registers live
// across the tile code).
template <bool REAL, bool FX, bool PERSIST>
__device__ __forceinline__ void predict_multi_body(const MultiArgs &a, int k)
{
    int q = multi_first_job(a, blockIdx.x);
    int it = 0;
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++it) {
        while (PERSIST && q + 1 < a.njobs && a.off[q + 1] <= tile) ++q;
        const JobDesc &J = a.jobs[q];
        const int from = J.cur ^ (k & 1);
        predict_split_tile<REAL, FX, false>(multi_tile(J, tile - a.off[q], (it & 1) * a.sbuf_words), J.p,
                                            J.phi[from], J.pi[from], J.phiH, J.piH, k);
        if (!PERSIST) break;
    }
    allow_dependents();  // after the CTA's last store
}

template <bool REAL, bool FX, bool KO, bool PERSIST>
__device__ __forceinline__ void correct_multi_body(const MultiArgs &a, int k)
{
    int q = multi_first_job(a, blockIdx.x);
    int it = 0;
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++it) {
        while (PERSIST && q + 1 < a.njobs && a.off[q + 1] <= tile) ++q;
        const JobDesc &J = a.jobs[q];
        const int from = J.cur ^ (k & 1);
        correct_split_tile<REAL, FX, KO, false>(multi_tile(J, tile - a.off[q], (it & 1) * a.sbuf_words), J.p,
                                                J.phi[from], J.pi[from], J.phiH, J.piH, J.phi[from ^ 1],
                                                J.pi[from ^ 1], k);
        if (!PERSIST) break;
    }
    allow_dependents();
}

// One instantiation per arithmetic and launch form, with the split kernels'
// launch bounds.
template <bool REAL, bool FX, bool PERSIST>
__global__ void lw_predict_multi(const __grid_constant__ MultiArgs a, int k);
template <bool REAL, bool FX, bool KO, bool PERSIST>
__global__ void lw_correct_multi(const __grid_constant__ MultiArgs a, int k);

#define TEUK_MULTI_PREDICT(REAL, FX, PERSIST, BOUNDS)                                                        \
    template <>                                                                                            \
    __global__ void BOUNDS lw_predict_multi<REAL, FX, PERSIST>(const __grid_constant__ MultiArgs a, int k) \
    {                                                                                                      \
        predict_multi_body<REAL, FX, PERSIST>(a, k);                                                       \
    }
#define TEUK_MULTI_CORRECT(REAL, FX, KO, PERSIST, BOUNDS)                                                        \
    template <>                                                                                                \
    __global__ void BOUNDS lw_correct_multi<REAL, FX, KO, PERSIST>(const __grid_constant__ MultiArgs a, int k) \
    {                                                                                                          \
        correct_multi_body<REAL, FX, KO, PERSIST>(a, k);                                                       \
    }
#define TEUK_MULTI_BOTH(PERSIST)                                                \
    TEUK_MULTI_PREDICT(false, true, PERSIST, TEUK_SPLIT_BOUNDS_FX)              \
    TEUK_MULTI_PREDICT(true, true, PERSIST, TEUK_SPLIT_BOUNDS_FX)               \
    TEUK_MULTI_PREDICT(false, false, PERSIST, TEUK_SPLIT_BOUNDS_FP64)           \
    TEUK_MULTI_PREDICT(true, false, PERSIST, TEUK_SPLIT_BOUNDS_FP64)            \
    TEUK_MULTI_CORRECT(false, true, false, PERSIST, TEUK_SPLIT_BOUNDS_FX)       \
    TEUK_MULTI_CORRECT(true, true, false, PERSIST, TEUK_SPLIT_BOUNDS_FX)        \
    TEUK_MULTI_CORRECT(false, false, false, PERSIST, TEUK_SPLIT_BOUNDS_FP64)    \
    TEUK_MULTI_CORRECT(true, false, false, PERSIST, TEUK_SPLIT_BOUNDS_FP64)     \
    TEUK_MULTI_CORRECT(false, true, true, PERSIST, TEUK_SPLIT_BOUNDS_FX)        \
    TEUK_MULTI_CORRECT(true, true, true, PERSIST, TEUK_SPLIT_BOUNDS_FX)         \
    TEUK_MULTI_CORRECT(false, false, true, PERSIST, TEUK_SPLIT_BOUNDS_FP64)     \
    TEUK_MULTI_CORRECT(true, false, true, PERSIST, TEUK_SPLIT_BOUNDS_FP64)
TEUK_MULTI_BOTH(false)
TEUK_MULTI_BOTH(true)
#undef TEUK_MULTI_BOTH
#undef TEUK_MULTI_PREDICT
#undef TEUK_MULTI_CORRECT

// Kernel of a multi-job launch form (persistent or one CTA per tile).
#define TEUK_PICK_P(K, real, fx, P) \
    ((real) ? ((fx) ? K<true, true, P> : K<true, false, P>) : ((fx) ? K<false, true, P> : K<false, false, P>))
#define TEUK_PICK3_P(K, real, fx, ko, P)                                                                     \
    ((ko) ? ((real) ? ((fx) ? K<true, true, true, P> : K<true, false, true, P>)                              \
                    : ((fx) ? K<false, true, true, P> : K<false, false, true, P>))                            \
          : ((real) ? ((fx) ? K<true, true, false, P> : K<true, false, false, P>)                            \
                    : ((fx) ? K<false, true, false, P> : K<false, false, false, P>)))
static const void *multi_ptr(int which, int real, int fx, int ko, bool persist)
{
    if (which)
        return persist ? (const void *)TEUK_PICK3_P(lw_correct_multi, real, fx, ko, true)
                       : (const void *)TEUK_PICK3_P(lw_correct_multi, real, fx, ko, false);
    return persist ? (const void *)TEUK_PICK_P(lw_predict_multi, real, fx, true)
                   : (const void *)TEUK_PICK_P(lw_predict_multi, real, fx, false);
}

// The persistent form's kernel (for occupancy queries).
const void *multi_kernel_ptr(int which, int real, int fixed_point, int ko)
{
    return multi_ptr(which, real, fixed_point, ko, true);
}

cudaError_t multi_allow_smem(int real, int fixed_point, int ko, size_t smem)
{
    for (int w = 0; w < 2; ++w) {
        cudaError_t e = allow_smem(multi_ptr(w, real, fixed_point, ko, false), smem);
        if (e == cudaSuccess) e = allow_smem(multi_ptr(w, real, fixed_point, ko, true), 2 * smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_step_multi(const MultiArgs &a, int which, int real, int fixed_point, int ko, int block,
                              size_t smem, int ctas, int k, cudaStream_t st, bool pdl)
{
    if (a.ntiles <= 0) return cudaSuccess;
    const bool persist = ctas > 0 && ctas < a.ntiles;  // then smem holds two sets of rows
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(persist ? ctas : a.ntiles);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = persist ? 2 * smem : smem;
    cfg.stream = st;
    cfg.attrs = pdl ? attr : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    void *args[] = {(void *)&a, (void *)&k};
    const cudaError_t e = cudaLaunchKernelExC(&cfg, multi_ptr(which, real, fixed_point, ko, persist), args);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

__global__ void advance_batch_kernel(const JobDesc *jobs, int njobs, long long by)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < njobs) {
        long long *step = (long long *)ldcg((const unsigned long long *)&jobs[j].p.step_base);
        *step += by;
    }
}

cudaError_t launch_advance_batch(const JobDesc *jobs, int njobs, long long by, cudaStream_t st)
{
    advance_batch_kernel<<<(njobs + 127) / 128, 128, 0, st>>>(jobs, njobs, by);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Small kernels
// ---------------------------------------------------------------------------

__global__ void advance_kernel(long long *step_base, long long by) { *step_base += by; }

__global__ void set_counter_kernel(long long *counter, long long value) { *counter = value; }

cudaError_t launch_set_counter(long long *counter, long long value, cudaStream_t st)
{
    set_counter_kernel<<<1, 1, 0, st>>>(counter, value);
    return cudaGetLastError();
}

cudaError_t launch_advance(long long *step_base, long long by, cudaStream_t st)
{
    advance_kernel<<<1, 1, 0, st>>>(step_base, by);
    return cudaGetLastError();
}

// Time-symmetric data (d_t Phi = 0): Pi_i = b_i (Phi_{i+1} - Phi_{i-1}) / (2h); boundary rows 0.
__global__ void time_symmetric_pi_kernel(const double2 *__restrict__ Phi, double2 *__restrict__ Pi,
                                         const double *__restrict__ b_node, int nr, int nth,
                                         double inv_2h)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nr * nth) return;
    const int i = (int)(idx / nth);
    if (i == 0 || i == nr - 1) {
        Pi[idx] = make_double2(0.0, 0.0);
        return;
    }
    const double2 up = Phi[idx + nth], dn = Phi[idx - nth];
    const double b = b_node[idx];
    Pi[idx] = make_double2(b * (up.x - dn.x) * inv_2h, b * (up.y - dn.y) * inv_2h);
}

cudaError_t launch_time_symmetric_pi(const double2 *Phi, double2 *Pi, const double *b_node, int nr,
                                     int nth, double inv_2h, cudaStream_t st)
{
    const long long n = (long long)nr * nth;
    time_symmetric_pi_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Phi, Pi, b_node, nr, nth, inv_2h);
    return cudaGetLastError();
}

__global__ void zero_rows_kernel(double2 *Phi, double2 *Pi, int nr, int nth)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * nth) return;
    const size_t k = t < nth ? (size_t)t : (size_t)(nr - 1) * nth + (t - nth);
    Phi[k] = make_double2(0.0, 0.0);
    Pi[k] = make_double2(0.0, 0.0);
}

cudaError_t launch_zero_boundary_rows(double2 *Phi, double2 *Pi, int nr, int nth, cudaStream_t st)
{
    zero_rows_kernel<<<(2 * nth + 255) / 256, 256, 0, st>>>(Phi, Pi, nr, nth);
    return cudaGetLastError();
}

__global__ void nonfinite_kernel(const double2 *__restrict__ Phi, const double2 *__restrict__ Pi,
                                 long long npts, unsigned long long *count)
{
    unsigned long long c = 0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < npts;
         k += (long long)gridDim.x * blockDim.x) {
        const double2 a = Phi[k], b = Pi[k];
        c += !isfinite(a.x) + !isfinite(a.y) + !isfinite(b.x) + !isfinite(b.y);
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

cudaError_t launch_nonfinite_count(const double2 *Phi, const double2 *Pi, long long npts,
                                   unsigned long long *count, cudaStream_t st)
{
    nonfinite_kernel<<<1216, 256, 0, st>>>(Phi, Pi, npts, count);
    return cudaGetLastError();
}

}  // namespace teuk
