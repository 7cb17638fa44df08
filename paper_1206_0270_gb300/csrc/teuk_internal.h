// teuk_internal.h -- device data layout and kernel parameters of libteuk.
//
// One time step of the two-step Lax-Wendroff scheme (Eqs. 3-4 of
// arXiv:1206.0270) is linear in the state with time-independent
// coefficients, apart from the source phase.  The setup kernel folds every
// constant of the scheme (dt, h, dtheta, the 1/2 averages, the diagonal of
// the angular stencil, the pole ghosts) into per-point coefficient planes, so
// that a step is 100 flops per point (56 FP64 instructions; the kernels run 20
// of them on the FP64 pipe and the Pi rows as fixed-point sums on the integer
// pipes: FP64 throughput is the scarce resource on GB300; bytes are not).
//
// With u_i = (Phi_i, Pi_i) the state at node i, sigma_j = Phi_{i,j} +
// Phi_{i+1,j} and tau = Pi_i + Pi_{i+1}, the predictor (Eq. 3) at the
// mid-point h = i + 1/2 reads
//   Phi^h = pa Phi_i + pb Phi_{i+1} + (dt/4) tau
//   Pi^h  = P1 tau + eb Pi_{i+1} + Q1 Phi_i + Q2 Phi_{i+1}
//           + KA sigma_{j+1} + KC sigma_{j-1} + gP e^{-i m Omega t_n}
// (P1 Pi_i + P2 Pi_{i+1} regrouped, eb = P2 - P1) and with
// sigma'_j = Phi^{i+1/2}_j + Phi^{i-1/2}_j, tau' = Pi^{i+1/2} + Pi^{i-1/2} the
// corrector (Eq. 4)
//   Phi^{n+1} = Phi_i - tb Phi^{i+1/2} + tb Phi^{i-1/2} + (dt/2) tau'
//   Pi^{n+1}  = Pi_i + R1 tau' + nt2 Pi^{i-1/2} + R3 Phi^{i+1/2} + R4 Phi^{i-1/2}
//               + KA' sigma'_{j+1} + KC' sigma'_{j-1} + gC e^{-i m Omega (t_n + dt/2)}
// (R1 Pi^{i+1/2} + R2 Pi^{i-1/2} regrouped, nt2 = R2 - R1)
// where (beta = dt b/(2h), gamma = dt d/(2h), A/B/C the angular stencil
// weights of L_theta with the ghosts folded into B at j = 0 and j = nth-1):
//   pa = 1/2 + beta, pb = 1/2 - beta,
//   P1 = 1/2 - beta - (dt/4) c_t,  P2 = 1/2 + beta - (dt/4) c_t,  eb = 2 beta,
//   Q1 = -gamma - (dt/4)(W - kappa B),  Q2 = gamma - (dt/4)(W - kappa B),
//   KA = (dt/4) kappa A, KC = (dt/4) kappa C, gP = (dt/2) G      (mid-point values)
//   tb = 2 beta, R1 = 2 beta - (dt/2) c_t, R2 = -2 beta - (dt/2) c_t, nt2 = -4 beta,
//   R3 = 2 gamma - (dt/2)(W - kappa B), R4 = -2 gamma - (dt/2)(W - kappa B),
//   KA' = (dt/2) kappa A, KC' = (dt/2) kappa C, gC = dt G        (node values)
//
// With the angular Kreiss-Oliger dissipation of strength eps the corrector
// also subtracts (eps/64) D6 u^n, D6 u_j = 20 u_j - 15 s1 + 6 s2 - s3 with the
// pair sums s_q = u_{j-q} + u_{j+q} of the same row (ghosts by reflection
// across the pole with the parity of the pole rule), for Phi and Pi alike:
//   Phi^{n+1} = k0 Phi_i + k1 s1 + k2 s2 + k3 s3 - tb Phi^{i+1/2} + ...
//   Pi^{n+1}  = k0 Pi_i  + k1 s1' + k2 s2' + k3 s3' + R1 tau' + ...
// k0 = 1 - 20 eps/64, k1 = 15 eps/64, k2 = -6 eps/64, k3 = eps/64.  The
// fixed-point kernels instead form D6 of each field exactly in integer
// arithmetic (teuk_fixed.h, fx_d6), round it once, and add kd D6 with
// kd = -eps/64: to Phi with one FP64 FMA, to Pi as one more term of its
// fixed-point sum.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace teuk {

// Thread limits of the step kernels.  Their Pi rows are fixed-point sums
// (teuk_fixed.h) that need up to 128 registers per thread (split and batch
// kernels) or about 230 (the fused kernel, which also holds the next row's
// loads), so their launch bounds admit 512 and 256 threads per CTA.  One
// thread covers one theta point of a tile row.
constexpr int kTileMaxThreads = 512;  // split and batch tiles: nth <= 512
constexpr int kFxTileThreads = 128;   // fixed-point split kernels: threads per CTA at most
constexpr int kFxTileMinBlocks = 5;   // ... and CTAs kept resident per SM (96 registers)
constexpr int kFusedMaxNth = 256;     // fused kernel: nth <= 256

// Predictor planes: rows hp = 0 .. nr-2 (mid-point r*_{hp+1/2}), nth values each.
struct PredPlanes {
    const double *pa, *pb, *eb, *KA, *KC;
    const double2 *P1, *Q1, *Q2;
};

// Corrector planes: rows i = 0 .. nr-1 (rows 0 and nr-1 unused).
struct CorrPlanes {
    const double *tb, *nt2, *KA, *KC;
    const double2 *R1, *R3, *R4;
};

// Source restricted to the rows where the Gaussian is non-zero.
struct SourceWindow {
    int mid_lo, mid_hi;    // predictor rows [mid_lo, mid_hi] (empty if mid_lo > mid_hi)
    int node_lo, node_hi;  // corrector rows [node_lo, node_hi]
    const double *gP;      // [(mid_hi - mid_lo + 1) * nth]  (dt/2) G at mid-points
    const double *gC;      // [(node_hi - node_lo + 1) * nth] dt G at nodes
    double m_omega;        // m * Omega
    int active;
};

struct Extraction {
    int i_ext;             // node row, or -1 when off
    int every;
    long long capacity;    // samples in the ring
    double2 *ring;         // [capacity][nth]
};

struct StepParams {
    int nr, nth;
    double dt, q, half_dt; // dt, dt/4, dt/2
    double one, nzero;     // 1 and -0: operands that turn FP64 adds and multiplies into FMAs
    int real_coef;         // 1: P1, Q1, Q2, R1, R3, R4 are packed real planes (no imaginary parts)
    int fixed_point;       // 1: Pi rows as fixed-point sums (teuk_fixed.h); 0: FP64 FMA chains
    int ko;                // 1: angular Kreiss-Oliger dissipation on (coefficients k0..k3)
    int parity;            // ghost parity of the pole rule (+1 even |m|, -1 odd |m|)
    double k0, k1, k2, k3; // 1 - 20 eps/64, 15 eps/64, -6 eps/64, eps/64 (FP64 arithmetic)
    double kd;             // -eps/64 (fixed-point arithmetic: weight of the exact D6)
    int kd_shift;          // log2(eps/64) when eps/64 is a power of two, else kNotPow2
    static constexpr int kNotPow2 = 0x7FFF;
    PredPlanes pred;
    CorrPlanes corr;
    SourceWindow src;
    Extraction ext;
    const long long *step_base;  // device: steps completed before this chunk
};

// One job of a batch, as the persistent batch kernels see it: its step
// parameters and buffers and its tile geometry.  The kernels work through
// the tiles of all jobs (tile_off[job] is the job's first tile); a tile is
// `rows` r* rows by `tw` theta columns, one thread per point, and a row has
// `tiles` theta tiles.
struct JobDesc {
    StepParams p;
    double2 *phi[2], *pi[2];  // state, ping-pong
    double2 *phiH, *piH;      // half step
    int cur;                  // buffer holding the state at the start of the slice
    int rows;                 // r* rows per tile
    int tw;                   // theta columns per tile (16, 32, 64 or 128)
    int tiles;                // theta tiles per row
};

// The jobs of one multi-job launch (lw_predict_multi / lw_correct_multi), all
// with the same arithmetic (real or complex planes, fixed point or FP64,
// dissipation or not).  It is passed in the kernels' parameter space, so a
// captured graph node keeps its own copy.  Tile t of the launch belongs to
// the job q with off[q] <= t < off[q + 1]; a job's tiles are `rows` r* rows
// by `tw` theta columns, rows * tw = the CTA size.
constexpr int kMultiMaxJobs = 64;  // 64 x 368-byte descriptors: 23.8 KB of the 32 KB parameter space
struct MultiArgs {
    int njobs;
    int ntiles;      // off[njobs]
    int sbuf_words;  // shared rows of one tile (double2 words); the persistent form alternates two sets
    int off[kMultiMaxJobs + 1];
    JobDesc jobs[kMultiMaxJobs];
};

// ---------------------------------------------------------------------------
// Kernels (teuk_kernels.cu)
// ---------------------------------------------------------------------------

struct SetupParams {
    int nr, nth, s, m, parity;
    int real_coef;  // write P1, Q1, Q2, R1, R3, R4 as packed real planes
    double a, h, dth, dt;
    const double *r_node, *D_node, *r_mid, *D_mid;  // radial tables (Delta as D)
    const double *sin_th, *cos_th, *cot_th;         // angular tables
    // outputs
    double *pa, *pb, *eb, *KAp, *KCp;
    double2 *P1, *Q1, *Q2;
    double *tb, *nt2, *KAc, *KCc;
    double2 *R1, *R3, *R4;
    double *b_node;
};

cudaError_t launch_setup(const SetupParams &sp, cudaStream_t st);

cudaError_t launch_step_fused(const StepParams &p, const double2 *Phi, const double2 *Pi,
                              double2 *PhiO, double2 *PiO, int k, int rows_per_block,
                              int nblocks, cudaStream_t st);

// part: 0 = predictor kernel only, 1 = corrector kernel only, 2 = both
cudaError_t launch_step_unfused(const StepParams &p, const double2 *Phi, const double2 *Pi,
                                double2 *PhiO, double2 *PiO, double2 *PhiH, double2 *PiH, int k,
                                cudaStream_t st, int part = 2);

cudaError_t launch_step_split(const StepParams &p, const double2 *Phi, const double2 *Pi, double2 *PhiO,
                              double2 *PiO, double2 *PhiH, double2 *PiH, int k, cudaStream_t st, bool pdl,
                              int part = 2, int rows = 0);

cudaError_t launch_advance(long long *step_base, long long by, cudaStream_t st);

cudaError_t launch_set_counter(long long *counter, long long value, cudaStream_t st);

cudaError_t launch_time_symmetric_pi(const double2 *Phi, double2 *Pi, const double *b_node,
                                     int nr, int nth, double inv_2h, cudaStream_t st);

cudaError_t launch_zero_boundary_rows(double2 *Phi, double2 *Pi, int nr, int nth, cudaStream_t st);

cudaError_t launch_nonfinite_count(const double2 *Phi, const double2 *Pi, long long npts,
                                   unsigned long long *count, cudaStream_t st);

// Multi-job kernels: which = 0 predictor, 1 corrector; `ctas` = 0 gives one
// CTA per tile, otherwise a persistent grid of min(ctas, tiles) CTAs that
// loop over the tiles.  `smem` is one tile's shared rows (a.sbuf_words
// double2 words); the persistent form takes twice that.  real / fixed_point / ko select the instantiation and
// must match every job of `a`.
cudaError_t launch_step_multi(const MultiArgs &a, int which, int real, int fixed_point, int ko, int block,
                              size_t smem, int ctas, int k, cudaStream_t st, bool pdl);
const void *multi_kernel_ptr(int which, int real, int fixed_point, int ko);
// Raise the multi-job kernels' dynamic shared-memory limit to `smem` per tile
// (twice that for the persistent form) where it exceeds the 48 KB default.
cudaError_t multi_allow_smem(int real, int fixed_point, int ko, size_t smem);
// Tile width of a job in a multi-job launch of `block`-thread CTAs: 16, 32,
// 64 or 128 columns, dividing the CTA size.
int multi_tile_width(int nth, int block);
// Dynamic shared memory of a multi-job CTA for a job of tile width tw.
size_t multi_smem_bytes(int tw, int block, int ko);

cudaError_t launch_advance_batch(const JobDesc *jobs, int njobs, long long by, cudaStream_t st);

int tile_width_for(int nth, int max_width);

int fused_block_threads(int nth);
size_t fused_smem_bytes(int nth, int ko);
const void *fused_kernel_ptr(int real, int fixed_point, int ko);
int split_tile_width(int nth);
int split_theta_tiles(int nth);
int split_rows_per_block(int nth, int fixed_point);
size_t split_smem_bytes(int nth, int rows = 0, int ko = 0);
const void *split_kernel_ptr(int which, int real, int fixed_point, int ko = 0);

}  // namespace teuk
