/*
 * teuk.h -- C ABI of the GB300 time-domain Teukolsky solver (libteuk.so).
 *
 * The solver advances one azimuthal mode m of the spin-weight-s Teukolsky
 * equation on a Kerr background (McKennon, Forrester & Khanna,
 * arXiv:1206.0270, section "Teukolsky Code"):
 *   - Eq. (1) is the master equation; Eq. (2) factors Psi = e^{i m phi} r^3 Phi_m.
 *   - The state is u = {Phi_R, Phi_I, Pi_R, Pi_I} (complex Phi and its
 *     momentum Pi = d_t Phi + b d_{r*} Phi) on an (r*, theta) grid.
 *   - One time step is the two-step Lax-Wendroff update of Eqs. (3) and (4)
 *     with second-order centred angular differences, the pole rule (even |m|:
 *     dPhi/dtheta = 0, odd |m|: Phi = 0) and Phi = Pi = 0 on both radial
 *     boundaries.
 *   - The point particle is a narrow Gaussian ("Mathematical Advances",
 *     item 1) moving on a circular equatorial orbit; the waveform is Phi
 *     sampled at an extraction radius.
 * Units: black-hole mass M = 1.  Fields and coefficients are IEEE FP64.  By
 * default the Pi-row sums of each update are formed from exact integer
 * products in 64-bit fixed point and rounded once to FP64, which is at least
 * as accurate as the same sums in FP64 arithmetic (TEUK_OPT_FIXED_POINT,
 * teuk_fixed_dot); everything else is FP64 arithmetic.
 *
 * Grid: r*_i = rstar_min + i h, h = (rstar_max - rstar_min)/(nr - 1),
 * i = 0..nr-1; theta_j = (j + 1/2) pi / nth, j = 0..nth-1 (the poles are not
 * grid points).  Host and device field arrays are row-major [i][j] (theta
 * fastest) of interleaved complex doubles (re, im): 2 * nr * nth doubles.
 *
 * Errors: every call returns TEUK_OK (0) or a negative TEUK_ERR_* code; the
 * handle keeps a message readable with teuk_last_error().  A call that fails
 * leaves the handle usable unless the code is TEUK_ERR_CUDA.
 *
 * Streams: all device work of a handle is issued on the CUDA stream given to
 * teuk_create (NULL: the handle creates and owns a non-blocking stream).
 * teuk_step is asynchronous;
 * calls that return host data synchronise that stream.  A handle must not be
 * used from two threads at once; distinct handles are independent.
 *
 * Ownership: the handle owns its device memory (allocated in teuk_create and
 * teuk_set_extraction, released in teuk_destroy).  Host buffers passed in are
 * owned by the caller and are only read or written during the call.
 */
#ifndef TEUK_H
#define TEUK_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TEUK_OK 0
#define TEUK_ERR_BAD_ARG (-1)   /* an argument is out of range or a pointer is NULL */
#define TEUK_ERR_OOM (-2)       /* device or host allocation failed */
#define TEUK_ERR_CUDA (-3)      /* a CUDA runtime call failed */
#define TEUK_ERR_NONFINITE (-4) /* the state holds a NaN or infinity */
#define TEUK_ERR_STATE (-5)     /* call not valid in the handle's current state */
#define TEUK_ERR_OVERFLOW (-6)  /* waveform samples were overwritten before extraction */

typedef struct teuk_handle teuk_handle;

/* Grid and time step.  nr >= 4, 2 <= nth <= 4096, rstar_min < rstar_max,
 * rstar_min >= -1000, dt > 0 (see teuk_stable_dt). */
typedef struct {
    int nr;
    int nth;
    double rstar_min;
    double rstar_max;
    double dt;
} teuk_grid;

/* Circular equatorial orbit at Boyer-Lindquist radius r0 (> r+), smeared into
 * a Gaussian of width sigma in r* and sigma / r0 in theta around
 * (r*(r0), pi/2), normalised so that sum_ij G_ij h dtheta = 1 and cut to zero
 * where its exponent exceeds 50.  The source added to the Pi equation is
 * amplitude * G * exp(-i m Omega t) with Omega = 1/(r0^{3/2} + a) (prograde)
 * or -1/(r0^{3/2} - a) (retrograde).  This Gaussian stands in for the
 * paper's point-particle source T of Eq. (1). */
typedef struct {
    double r0;
    double sigma;
    double amplitude;
    int prograde;
} teuk_orbit;

/* Time-step rule (the paper gives none): dt = min(c_r h / max b,
 * c_theta / omega_max), where b = (r^2 + a^2)/Sigma_hat is the radial
 * characteristic speed and omega_max^2 is the Gershgorin bound of the
 * discrete angular-plus-potential operator over all nodes and mid-points.
 * The source terms of Eqs. (3)-(4) integrate oscillations of frequency omega
 * like explicit midpoint RK2, whose amplification per step is
 * sqrt(1 + (omega dt)^4 / 4): the stiffest modes, next to the poles, grow
 * unless c_theta is small (0.1) or the angular dissipation of
 * teuk_set_dissipation damps them (eps = 1 allows c_theta = 0.8).  Uses
 * g->nr, nth, rstar_min, rstar_max (g->dt is ignored).  Host-only, no GPU
 * needed. */
int teuk_stable_dt(const teuk_grid *g, double a, int s, int m, double c_r, double c_theta,
                   double *dt_out);

/* Create a solver for spin weight s in {-2, 0, 2}, |a| < 1, any integer m.
 * Allocates the state (two copies of Phi and Pi, 64 B per point) and the
 * precomputed scheme coefficients (168 B per point; the imaginary halves of
 * six planes stay unused when every coefficient is real) on the current device,
 * builds the coefficients with a setup kernel, zeroes the state.
 * cuda_stream: a cudaStream_t (or NULL).  On success *out receives the handle. */
int teuk_create(const teuk_grid *g, double a, int s, int m, void *cuda_stream, teuk_handle **out);

/* Release all device memory of the handle: the state u = {Phi, Pi} of the
 * first-order form of Eq. (2)'s mode equation (section "Teukolsky Code"),
 * the coefficient planes and the waveform ring.  Synchronises its stream.
 * TEUK_ERR_BAD_ARG for NULL, TEUK_ERR_STATE while a batch owns the handle. */
int teuk_destroy(teuk_handle *h);

/* Initial data from HOST arrays phi, pi (interleaved complex [nr][nth]).
 * pi == NULL selects time-symmetric data, d_t Phi = 0, i.e.
 * Pi_i = b_i (Phi_{i+1} - Phi_{i-1}) / (2h).  The radial boundary rows are
 * forced to zero.  Resets the step counter and the waveform buffer. */
int teuk_set_initial(teuk_handle *h, const double *phi, const double *pi);

/* Same as teuk_set_initial with DEVICE arrays (same layout), stream-ordered. */
int teuk_set_initial_device(teuk_handle *h, const double *phi_dev, const double *pi_dev);

/* Set (orbit != NULL) or remove (orbit == NULL) the Gaussian point-particle
 * source.  TEUK_ERR_BAD_ARG if r0 <= r+, sigma <= 0, or r*(r0) lies outside
 * the grid. */
int teuk_set_source(teuk_handle *h, const teuk_orbit *orbit);

/* Waveform sampling (the waveforms of the paper's results section, e.g.
 * Fig. 1, are the field read at a distant observer): after every step n
 * (counted from the last teuk_set_initial) with n % every == 0,
 * Phi(r*_k, theta_j), j < nth, is copied into a device ring buffer of
 * `capacity` samples, k the node nearest to rstar_ext.  Allocates the ring
 * buffer; clears earlier samples.  TEUK_ERR_BAD_ARG if rstar_ext is off the
 * grid, every < 1 or capacity < 1; TEUK_ERR_OOM if the ring does not fit. */
int teuk_set_extraction(teuk_handle *h, double rstar_ext, int every, long capacity);

/* Run the handle's future work on `cuda_stream` (a cudaStream_t owned by the
 * caller; NULL: a stream the handle creates and owns).  Synchronises the
 * handle's current stream first and releases it if the handle created it.
 * Results do not depend on the stream.  Allowed for handles in a batch (the
 * batch's per-job launches use the handle's stream): a scheduler can move a
 * job to a stream of another priority between slices.  The paper has no
 * counterpart. */
int teuk_set_stream(teuk_handle *h, void *cuda_stream);

/* Advance n >= 0 time steps of the two-step Lax-Wendroff scheme, Eqs. (3)
 * and (4) (section "Teukolsky Code"): predictor to the radial mid-points at
 * the half step, corrector to the nodes, angular derivatives and sources in
 * S, Phi = Pi = 0 on the radial boundary rows, plus the angular dissipation
 * if set.  Asynchronous on the handle's stream; full chunks of steps replay a
 * captured CUDA graph.  TEUK_ERR_BAD_ARG for n < 0, TEUK_ERR_STATE while a
 * batch owns the handle, TEUK_ERR_CUDA if a launch fails. */
int teuk_step(teuk_handle *h, long n);

/* Angular Kreiss-Oliger dissipation (Kreiss & Oliger 1973, the sixth-order
 * member of the family; the paper's scheme, Eqs. 3-4, has none, and this is
 * the reading that lets the time step grow): each corrector subtracts
 * (eps/64) D6 u^n from the new state of every interior row, for Phi and Pi,
 *   D6 u_j = -(u_{j-3} + u_{j+3}) + 6 (u_{j-2} + u_{j+2})
 *            - 15 (u_{j-1} + u_{j+1}) + 20 u_j,
 * with the ghost values of the pole rule (reflection across the pole with
 * the parity of |m|).  On cos(k theta) / sin(k theta) it multiplies by
 * 1 - eps sin^6(k dtheta / 2).  eps = 0 (the default) is the bare scheme;
 * otherwise 1e-9 <= eps < 2 (TEUK_ERR_BAD_ARG).  Synchronises the stream;
 * TEUK_ERR_STATE while a batch owns the handle. */
int teuk_set_dissipation(teuk_handle *h, double eps);

/* Copy the waveform samples (see teuk_set_extraction; the observer's signal
 * of the paper's results section) taken since the previous call (oldest
 * first) to the host: t_out[k] and phi_out[k][nth] (interleaved complex), at
 * most cap samples; *n_out receives the number copied.  Synchronises the
 * stream.  TEUK_ERR_STATE if no extraction is set.
 * TEUK_ERR_OVERFLOW if more samples than the ring capacity were taken since
 * the previous call (the newest `capacity` samples are returned). */
int teuk_extract(teuk_handle *h, double *t_out, double *phi_out, long cap, long *n_out);

/* Restore a checkpoint: the state from HOST arrays phi, pi (layout as in
 * teuk_set_initial) taken after `step` time steps.  The step count is set to
 * `step`, so the source phase and the waveform sampling continue where the
 * checkpointed run stood (samples already taken are not replayed); resuming
 * gives bit-identical results to an uninterrupted run.  The radial boundary
 * rows are forced to zero.  Synchronises. */
int teuk_set_state(teuk_handle *h, const double *phi, const double *pi, long step);

/* Copy the current state u = {Phi, Pi} (the solution vector of Eq. (3),
 * section "Teukolsky Code") to HOST arrays, layout as in teuk_set_initial
 * (either pointer may be NULL).  Synchronises.  TEUK_ERR_CUDA if a copy
 * fails. */
int teuk_get_state(teuk_handle *h, double *phi, double *pi);

/* Copy the current state to DEVICE arrays (stream-ordered, asynchronous). */
int teuk_get_state_device(teuk_handle *h, double *phi_dev, double *pi_dev);

/* Steps taken since the last teuk_set_initial. */
long teuk_step_count(const teuk_handle *h);

/* Reduce the state for NaN/Inf on the device; *finite = 1 if all finite.
 * Returns TEUK_ERR_NONFINITE when not.  Synchronises. */
int teuk_check_finite(teuk_handle *h, int *finite);

/* Select the step kernel: 0 = fused radial-marching kernel, 1 = two-kernel
 * predictor/corrector with a half-step buffer in device memory, 2 = the same
 * two kernels over 2D tiles with the angular neighbour sums shared in shared
 * memory (0 needs nth <= 256, 2 needs nth <= 512; the default is 2 where it
 * fits, else 1).  All compute the same Eqs. (3)-(4) and give bit-identical
 * results. */
int teuk_set_kernel(teuk_handle *h, int variant);

/* Launch shape of the fused kernel: radial rows per CTA (one CTA per strip
 * of rows, marching along r*).  0 restores the automatic choice.  Longer
 * strips recompute fewer predictor rows (one per strip) but leave fewer CTAs
 * to hide latency.  Results do not depend on the shape. */
int teuk_set_launch(teuk_handle *h, int rows_per_block);

/* Tuning options (teuk_set_option).  Results do not depend on them.
 *   TEUK_OPT_PDL: 1 (default) launches the split kernels with programmatic
 *     dependent launch, so a kernel loads its constant coefficients while its
 *     predecessor drains; 0 launches them in plain stream order.
 *   TEUK_OPT_GRAPH_CHUNK: time steps per captured CUDA graph, even, 2..4096
 *     (default 64). */
#define TEUK_OPT_PDL 1
#define TEUK_OPT_GRAPH_CHUNK 2
#define TEUK_OPT_BLOCK_THREADS 3  /* batches only (mode 0): CTA threads, a multiple of 32 <= 512, at most 128
                                    for fixed-point jobs; 0 = automatic (128 fixed point, 256 FP64) */
/* TEUK_OPT_REAL_PATH: 1 (default) stores real coefficient planes and uses
 * real-by-complex products when every coefficient is real (a = 0, or
 * s = m = 0: 6 and 7 instead of 9 and 10 products per Pi row); 0 keeps the
 * complex planes.  Both give the same numbers. */
#define TEUK_OPT_REAL_PATH 4
/* TEUK_OPT_SPLIT_ROWS: r* rows per CTA tile of the split kernels; a tile is
 * up to 128 theta columns (16 for rows of at most 16 columns, else a
 * multiple of 32; wider rows are cut into tiles,
 * the last one ragged), one thread per point.  1..128 / (tile width) with
 * the fixed-point Pi rows (their kernels launch at most 128 threads per CTA;
 * a larger height set earlier for FP64 is reduced to that), 1..512 / (tile
 * width) with FP64 Pi rows.  0 (default) picks 128 / tile width (256 / tile
 * width for FP64), at least 1. */
#define TEUK_OPT_SPLIT_ROWS 5
/* TEUK_OPT_BATCH_MODE (batches only): 1 (default) advances every job with its
 * own kernels on its own stream (graph replay per chunk), the jobs running
 * concurrently; 0 advances the jobs with one predictor and one corrector
 * launch per time step for each group of up to 64 jobs that share an
 * arithmetic, each launch covering the tiles of all jobs of its group.
 * Both give the same numbers as stepping each handle alone. */
#define TEUK_OPT_BATCH_MODE 6
/* TEUK_OPT_FIXED_POINT: 1 (default) evaluates the Pi rows of Eqs. (3)-(4) as
 * fixed-point sums on the integer pipes (see teuk_fixed_dot: exact products,
 * one rounding, at least as accurate as the FP64 sum); 0 evaluates every
 * product with FP64 fused multiply-adds.  The two differ only by rounding
 * (both agree with the oracle to about 1e-14 per step). */
#define TEUK_OPT_FIXED_POINT 7
/* TEUK_OPT_BATCH_CTAS (batches only, mode 0): 0 (default) launches one CTA
 * per tile; k = 1..64 launches a persistent grid of k CTAs per SM (at most as
 * many as stay resident), each CTA looping over the tiles. */
#define TEUK_OPT_BATCH_CTAS 8
int teuk_set_option(teuk_handle *h, int option, long value);

/* Current fused-kernel launch shape. */
int teuk_get_launch(const teuk_handle *h, int *rows_per_block, int *nblocks);

/* Time the step kernels: advance n >= 1 steps with plain (non-graph,
 * non-PDL) launches and CUDA events on the handle's stream around each
 * kernel; ms_out[0] and ms_out[1] receive the average duration of the
 * predictor and the corrector kernel (two-kernel variants), or of the fused
 * step kernel and 0.  The steps count as progress.  Synchronises. */
int teuk_time_kernels(teuk_handle *h, long n, double *ms_out);

/* Number of kernel launches one teuk_step(h, n) issues for this handle's
 * configuration (graph replays count their kernel nodes). */
long teuk_launches_for(const teuk_handle *h, long n);

/* One time step that allocates no device memory.  The paper has no
 * counterpart: this entry point serves callers that cannot call cudaMalloc
 * while they step -- real-time loops that must not block in the allocator,
 * and processes whose device memory is owned by another framework's pool
 * (the library must not take memory behind that pool's back).
 *
 * Advances the DEVICE state (phi_in, pi_in) by one time step of the
 * library's scheme (the split kernels, the handle's coefficients, source and
 * dissipation) into the DEVICE buffers (phi_out, pi_out), all interleaved
 * complex [nr][nth] and owned by the caller.  No output may overlap an input
 * or the other output (checked by address range: TEUK_ERR_BAD_ARG).  Rows 0
 * and nr-1 of the inputs must be zero, as in every state this library
 * produces (the radial boundary rows; the kernels read them as they are);
 * the output boundary rows are set to zero, so chained calls keep them so.
 * step_index is passed by value to the kernels of this call: the source
 * phase is that of t = step_index * dt.  Issues its work on the handle's
 * stream and returns without waiting.  No waveform is sampled; the handle's
 * own state, step counter and ring buffer are neither read nor changed.
 *
 * The half step is kept in a static device array of 32 MiB inside libteuk:
 * every GPU that loads the library holds it until the process exits, and it
 * limits the grid to (nr - 1) * nth <= 1,048,576 (larger grids and nth > 512
 * return TEUK_ERR_BAD_ARG).  All calls share that array and it keeps the last
 * call's contents, so calls that overlap on the GPU (different streams or
 * handles running at once) race: issue them one after another on one stream.
 * The first call on each device looks up the array's device address with
 * cudaGetSymbolAddress, a synchronous runtime call.
 * The handle's device must be the current device. */
int teuk_step_noalloc(teuk_handle *h, const double *phi_in, const double *pi_in, double *phi_out,
                      double *pi_out, long step_index);

/* ------------------------------------------------------------------------
 * Batches: many independent evolutions stepped together.
 *
 * A template bank is many independent (a, r0, m) evolutions of uneven grid
 * size and length (the paper's motivation for fast waveform generation; its
 * temporal segments are independent evolutions too).  A batch groups
 * existing handles on one device and advances them together; the arithmetic
 * per point is that of teuk_step, so results are bit-identical to stepping
 * each handle alone.  Two modes (TEUK_OPT_BATCH_MODE):
 *   1 (default): every job advances with its own kernels on its own stream
 *     (graph replay per chunk), all jobs concurrently and independently;
 *   0: per time step, one predictor and one corrector launch for each group
 *     of up to 64 jobs that share an arithmetic cover the theta tiles of all
 *     of them (one CTA per tile, or a persistent grid of resident CTAs that
 *     loop over the tiles: TEUK_OPT_BATCH_CTAS); jobs advance in slices of
 *     min(graph chunk, smallest remaining step count) steps, a job that has
 *     taken its steps leaves at the next slice boundary, and full slices
 *     replay a CUDA graph captured for the current set of jobs.
 * teuk_batch_autotune picks the launch form.
 *
 * Rules: a handle in a batch is driven by the batch only -- teuk_step, the
 * other teuk_set_* calls (teuk_set_stream excepted), teuk_step_noalloc and
 * teuk_destroy on it return TEUK_ERR_STATE until it is removed (or the batch
 * destroyed); call teuk_batch_sync() before reading a job's results through
 * its handle (teuk_extract, teuk_get_state).  Jobs need nth <= 512.  A batch
 * allocates its job table (and a job's half-step buffer if the handle has
 * none).
 * ------------------------------------------------------------------------ */
typedef struct teuk_batch teuk_batch;

/* Create an empty batch on the current device; work is issued on
 * cuda_stream (NULL: the batch creates and owns a non-blocking stream). */
int teuk_batch_create(void *cuda_stream, teuk_batch **out);

/* Add a handle that still has `steps` time steps to take; *job_id receives
 * its index in the batch.  Synchronises the handle's stream. */
int teuk_batch_add(teuk_batch *b, teuk_handle *h, long steps, int *job_id);

/* Remove a job (its handle stays valid).  Synchronises the batch stream. */
int teuk_batch_remove(teuk_batch *b, int job_id);

/* Advance the jobs by up to max_steps time steps of batch time (each job at
 * most its remaining count), asynchronously; *steps_done (may be NULL)
 * receives the batch time advanced. */
int teuk_batch_step(teuk_batch *b, long max_steps, long *steps_done);

/* Steps job_id still has to take (0 once done or removed). */
int teuk_batch_remaining(const teuk_batch *b, int job_id, long *remaining);

/* Wait for the batch's queued work. */
int teuk_batch_sync(teuk_batch *b);

/* TEUK_OPT_PDL, TEUK_OPT_GRAPH_CHUNK, TEUK_OPT_BLOCK_THREADS,
 * TEUK_OPT_BATCH_CTAS (mode 0) or TEUK_OPT_BATCH_MODE. */
int teuk_batch_set_option(teuk_batch *b, int option, long value);

/* Time the launch forms and tile shapes on the batch's own jobs -- per-job
 * launches, the multi-job launches with one CTA per tile at the default CTA
 * size and at 64 threads (tiles of at most 64 theta columns, fewer rows),
 * and the persistent multi-job launches -- and keep the fastest
 * (TEUK_OPT_BATCH_MODE, TEUK_OPT_BATCH_CTAS and TEUK_OPT_BLOCK_THREADS are
 * set accordingly); the timed steps count as progress.  *best (may be NULL)
 * receives 0, 1, 2 or 3 for those four.  Synchronises. */
int teuk_batch_autotune(teuk_batch *b, int *best);

/* Kernel launches that teuk_batch_step(b, n) issues when no job finishes. */
long teuk_batch_launches_for(const teuk_batch *b, long n);

/* Message of the last failed batch call ("" if none). */
const char *teuk_batch_last_error(const teuk_batch *b);

int teuk_batch_destroy(teuk_batch *b);

/* ------------------------------------------------------------------------
 * Arithmetic check.  The Pi rows of Eqs. (3)-(4) are sums of 6 to 10
 * products of FP64 coefficients and fields; the step kernels evaluate them
 * in 64-bit fixed point on the integer pipe: exact 106-bit products, aligned
 * and truncated to 2^-57 of the largest product, summed, and rounded once to
 * FP64 (error <= n 2^-57 max|c_k x_k| + 2^-53 |sum|); where that is not
 * possible (an input not finite, a result below 2^-823 or overflowing) the
 * kernels use FP64 fused multiply-adds instead.  The paper has no
 * counterpart: it is an implementation of its double-precision sums for a
 * GPU whose FP64 pipe is narrow.
 *
 * teuk_fixed_dot evaluates that arithmetic for `count` independent sums of
 * `nterms` (1..16) terms: out[i] = sum_k (-1)^flip[i*nterms+k]
 * c[i*nterms+k] x[i*nterms+k], ok[i] = 1 where the fixed-point sum applies
 * (ok[i] = 0: out[i] unspecified; the kernels would use FP64 there).
 * on_device = 0 runs the host build of the same code, 1 the device build
 * (copies through temporary device buffers; synchronous).  All pointers are
 * host pointers owned by the caller.  Returns TEUK_ERR_BAD_ARG for nterms
 * outside 1..16, count < 0 or a NULL array, TEUK_ERR_OOM / TEUK_ERR_CUDA on
 * device failures. */
int teuk_fixed_dot(int on_device, int nterms, long count, const double *c, const double *x,
                   const unsigned *flip, double *out, int *ok);

/* The angular Kreiss-Oliger dissipation of the corrector subtracts
 * (eps/64) D6 u from each node, D6 u_j = 20 u_j - 15 (u_{j-1} + u_{j+1})
 * + 6 (u_{j-2} + u_{j+2}) - (u_{j-3} + u_{j+3}) along theta (the sixth-order
 * member of Kreiss & Oliger's family; the dissipation is this library's
 * stabiliser of Eqs. (3)-(4), which the paper does not print).  With the
 * fixed-point arithmetic the kernels form D6 of each real component as an
 * exact integer sum: the seven values truncated to units of 2^(F-1079), F
 * the largest biased exponent among them (each loses less than one unit; the
 * largest keeps its 53 bits), rounded once to FP64 (error <= 2^-50 max|u_q|
 * + 2^-53 |D6|); a non-finite value gives NaN.  That rounded D6 enters Phi's
 * FP64 row; in Pi's fixed-point sum the term (-eps/64) D6 enters unrounded
 * when eps/64 is a power of two (the integer sum shifted to the sum's
 * frame), and as the product of -eps/64 with the rounded D6 otherwise.
 *
 * teuk_fixed_d6 evaluates that arithmetic for `count` windows of seven
 * values, u[7 i + q] = u_{j-3+q}: out[i] = D6.  on_device = 0 runs the host
 * build, 1 the device build (temporary device buffers; synchronous).  Host
 * pointers owned by the caller.  TEUK_ERR_BAD_ARG for count < 0 or a NULL
 * array, TEUK_ERR_OOM / TEUK_ERR_CUDA on device failures. */
int teuk_fixed_d6(int on_device, long count, const double *u, double *out);

/* Message of the last failed call on this handle ("" if none). */
const char *teuk_last_error(const teuk_handle *h);

/* Static description of an error code. */
const char *teuk_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* TEUK_H */
