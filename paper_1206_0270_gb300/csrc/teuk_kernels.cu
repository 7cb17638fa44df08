// teuk_kernels.cu -- CUDA kernels of libteuk (sm_103a, FP64).
//
// Hot path: one time step of the two-step Lax-Wendroff scheme, Eqs. (3)-(4)
// of arXiv:1206.0270, for u = (Phi, Pi) on an (r*, theta) grid, with the
// point-particle source added to the Pi row and the waveform row copied to a
// ring buffer.  All constants of the scheme are folded into the coefficient
// planes built by setup_kernel (the formulas are in teuk_internal.h), so the
// step costs 60 FP64 FMA-class instructions per point.
//
// The fused kernel assigns one thread per theta index j and lets each CTA
// march along r* over a contiguous strip of rows: the predictor value at
// i + 1/2 is computed once, used by the correctors at i and i + 1, and never
// leaves registers; the angular neighbours j +- 1 are exchanged through
// shared memory.  The only redundant work is one predictor row per strip.
#include "teuk_internal.h"
#include "teuk_physics.h"

namespace teuk {

// ---------------------------------------------------------------------------
// Complex helpers: acc += c * x with FP64 FMAs
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cfma(double2 &acc, const double2 c, const double2 x)
{
    acc.x = fma(c.x, x.x, acc.x);
    acc.x = fma(-c.y, x.y, acc.x);
    acc.y = fma(c.x, x.y, acc.y);
    acc.y = fma(c.y, x.x, acc.y);
}

__device__ __forceinline__ double2 cmul(const double2 c, const double2 x)
{
    double2 r;
    r.x = c.x * x.x;
    r.x = fma(-c.y, x.y, r.x);
    r.y = c.x * x.y;
    r.y = fma(c.y, x.x, r.y);
    return r;
}

__device__ __forceinline__ void rfma(double2 &acc, const double c, const double2 x)
{
    acc.x = fma(c, x.x, acc.x);
    acc.y = fma(c, x.y, acc.y);
}

__device__ __forceinline__ double2 add2(const double2 a, const double2 b)
{
    return make_double2(a.x + b.x, a.y + b.y);
}

template <typename T>
__device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

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
        sp.P1[k] = make_double2(0.5 - beta - q * c.ct_re, -q * c.ct_im);
        sp.P2[k] = make_double2(0.5 + beta - q * c.ct_re, -q * c.ct_im);
        sp.Q1[k] = make_double2(-g_re - q * wr, -g_im - q * wi);
        sp.Q2[k] = make_double2(g_re - q * wr, g_im - q * wi);
        sp.KAp[k] = q * c.kappa * A;
        sp.KCp[k] = q * c.kappa * C;
    } else {
        const double hd = 0.5 * sp.dt;
        sp.tb[k] = 2.0 * beta;
        sp.R1[k] = make_double2(2.0 * beta - hd * c.ct_re, -hd * c.ct_im);
        sp.R2[k] = make_double2(-2.0 * beta - hd * c.ct_re, -hd * c.ct_im);
        sp.R3[k] = make_double2(2.0 * g_re - hd * wr, 2.0 * g_im - hd * wi);
        sp.R4[k] = make_double2(-2.0 * g_re - hd * wr, -2.0 * g_im - hd * wi);
        sp.KAc[k] = hd * c.kappa * A;
        sp.KCc[k] = hd * c.kappa * C;
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

// Predictor at the mid-point row hp, theta index with plane offset k.
// phi0/pi0: u at row hp, phi1/pi1: u at row hp + 1, sup/sdn: sigma at j+1, j-1.
__device__ __forceinline__ HalfStep predict(const StepParams &p, size_t k, double2 phi0, double2 pi0,
                                            double2 phi1, double2 pi1, double2 sup, double2 sdn)
{
    HalfStep o;
    const double pa = ldg(p.pred.pa + k), pb = ldg(p.pred.pb + k);
    o.phi = make_double2(pa * phi0.x, pa * phi0.y);
    rfma(o.phi, pb, phi1);
    rfma(o.phi, p.q, pi0);
    rfma(o.phi, p.q, pi1);
    o.pi = cmul(ldg(p.pred.P1 + k), pi0);
    cfma(o.pi, ldg(p.pred.P2 + k), pi1);
    cfma(o.pi, ldg(p.pred.Q1 + k), phi0);
    cfma(o.pi, ldg(p.pred.Q2 + k), phi1);
    rfma(o.pi, ldg(p.pred.KA + k), sup);
    rfma(o.pi, ldg(p.pred.KC + k), sdn);
    return o;
}

// Corrector at node row i (plane offset k).  hp: half step at i + 1/2, hm: at i - 1/2,
// sup/sdn: sigma' = Phi^{i+1/2} + Phi^{i-1/2} at j+1, j-1.
__device__ __forceinline__ void correct(const StepParams &p, size_t k, double2 phi, double2 pi,
                                        const HalfStep &hp, const HalfStep &hm, double2 sup,
                                        double2 sdn, double2 *phi_out, double2 *pi_out)
{
    const double tb = ldg(p.corr.tb + k);
    double2 nphi = phi;
    rfma(nphi, -tb, hp.phi);
    rfma(nphi, tb, hm.phi);
    rfma(nphi, p.half_dt, hp.pi);
    rfma(nphi, p.half_dt, hm.pi);
    double2 npi = pi;
    cfma(npi, ldg(p.corr.R1 + k), hp.pi);
    cfma(npi, ldg(p.corr.R2 + k), hm.pi);
    cfma(npi, ldg(p.corr.R3 + k), hp.phi);
    cfma(npi, ldg(p.corr.R4 + k), hm.phi);
    rfma(npi, ldg(p.corr.KA + k), sup);
    rfma(npi, ldg(p.corr.KC + k), sdn);
    *phi_out = nphi;
    *pi_out = npi;
}

// ---------------------------------------------------------------------------
// Fused radial-marching step kernel
// ---------------------------------------------------------------------------

// Shared memory: sigma and sigma' double buffers, each nth + 2 entries with
// a zero ghost at both ends (their stencil weights are zero).
size_t fused_smem_bytes(int nth) { return sizeof(double2) * 4 * (size_t)(nth + 2); }
int fused_block_threads(int nth) { return ((nth + 31) / 32) * 32; }

__global__ void __launch_bounds__(1024) lw_step_fused(StepParams p, const double2 *__restrict__ Phi,
                                                      const double2 *__restrict__ Pi,
                                                      double2 *__restrict__ PhiO,
                                                      double2 *__restrict__ PiO, int k, int rpb)
{
    extern __shared__ double2 smem[];
    __shared__ double2 s_phase[2];
    const int nth = p.nth;
    const int W = nth + 2;
    double2 *s_sig = smem;          // [2][W]
    double2 *s_sgh = smem + 2 * W;  // [2][W]
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
    if (act) s_sig[j + 1] = add2(phc, phn);
    __syncthreads();
    HalfStep hm = predict(p, (size_t)(i0 - 1) * nth + jj, phc, pic, phn, pin, s_sig[jj + 2], s_sig[jj]);
    if (src_mid && i0 - 1 >= sw.mid_lo && i0 - 1 <= sw.mid_hi)
        rfma(hm.pi, ldg(sw.gP + (size_t)(i0 - 1 - sw.mid_lo) * nth + jj), s_phase[0]);
    phc = phn;
    pic = pin;

    int buf = 1;
    for (int i = i0; i < i1; ++i) {
        phn = Phi[(size_t)(i + 1) * nth + jj];
        pin = Pi[(size_t)(i + 1) * nth + jj];
        double2 *sg = s_sig + buf * W;
        if (act) sg[j + 1] = add2(phc, phn);
        __syncthreads();
        HalfStep hp = predict(p, (size_t)i * nth + jj, phc, pic, phn, pin, sg[jj + 2], sg[jj]);
        if (src_mid && i >= sw.mid_lo && i <= sw.mid_hi)
            rfma(hp.pi, ldg(sw.gP + (size_t)(i - sw.mid_lo) * nth + jj), s_phase[0]);

        double2 *sh = s_sgh + buf * W;
        if (act) sh[j + 1] = add2(hp.phi, hm.phi);
        __syncthreads();
        const size_t kc = (size_t)i * nth + jj;
        double2 nphi, npi;
        correct(p, kc, phc, pic, hp, hm, sh[jj + 2], sh[jj], &nphi, &npi);
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

const void *fused_kernel_ptr() { return (const void *)lw_step_fused; }

cudaError_t launch_step_fused(const StepParams &p, const double2 *Phi, const double2 *Pi,
                              double2 *PhiO, double2 *PiO, int k, int rows_per_block, int nblocks,
                              cudaStream_t st)
{
    const int threads = fused_block_threads(p.nth);
    lw_step_fused<<<nblocks, threads, fused_smem_bytes(p.nth), st>>>(p, Phi, Pi, PhiO, PiO, k,
                                                                     rows_per_block);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Two-kernel variant: predictor writes the half-step fields to device memory
// ---------------------------------------------------------------------------

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
    const double2 sup = add2(Phi[r0 + ju], Phi[r1 + ju]);
    const double2 sdn = add2(Phi[r0 + jd], Phi[r1 + jd]);
    HalfStep o = predict(p, k0, phi0, pi0, phi1, pi1, sup, sdn);
    const SourceWindow &sw = p.src;
    if (sw.active && hp >= sw.mid_lo && hp <= sw.mid_hi) {
        const long long n = *p.step_base + k;
        rfma(o.pi, sw.gP[(size_t)(hp - sw.mid_lo) * nth + j], unit_phase(sw.m_omega * ((double)n * p.dt)));
    }
    PhiH[k0] = o.phi;
    PiH[k0] = o.pi;
}

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
    const double2 sup = add2(PhiH[kp - j + ju], PhiH[km - j + ju]);
    const double2 sdn = add2(PhiH[kp - j + jd], PhiH[km - j + jd]);
    double2 nphi, npi;
    correct(p, kc, Phi[kc], Pi[kc], hp, hm, sup, sdn, &nphi, &npi);
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
                                cudaStream_t st)
{
    const int threads = 256;
    const long long np = (long long)(p.nr - 1) * p.nth, nc = (long long)(p.nr - 2) * p.nth;
    lw_predict_kernel<<<(unsigned)((np + threads - 1) / threads), threads, 0, st>>>(p, Phi, Pi, PhiH, PiH, k);
    lw_correct_kernel<<<(unsigned)((nc + threads - 1) / threads), threads, 0, st>>>(p, Phi, Pi, PhiH, PiH,
                                                                                  PhiO, PiO, k);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Small kernels
// ---------------------------------------------------------------------------

__global__ void advance_kernel(long long *step_base, long long by) { *step_base += by; }

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
