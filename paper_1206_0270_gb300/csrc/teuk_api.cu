// teuk_api.cu -- C ABI of libteuk (declared in include/teuk.h).
//
// Host side: argument checking, the inverse tortoise map and the
// time-step rule, device memory layout, the Gaussian source window, the
// waveform ring buffer, and CUDA-graph replay of chunks of time steps.  Every
// arithmetic step of the time evolution runs in the kernels of
// teuk_kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "teuk.h"
#include "teuk_handle.h"
#include "teuk_internal.h"
#include "teuk_physics.h"

using namespace teuk;

static const double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// Helpers
// ---------------------------------------------------------------------------

static int fail(teuk_handle *h, int code, const std::string &msg)
{
    if (h) h->err = msg;
    return code;
}

#define CU(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(h, TEUK_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static void horizons(double a, double *rp, double *rm)
{
    const double q = std::sqrt(1.0 - a * a);
    *rp = 1.0 + q;
    *rm = 1.0 - q;
}

// r*(r) = r + 2 r+/(r+ - r-) ln((r - r+)/2) - 2 r-/(r+ - r-) ln((r - r-)/2).
static double rstar_of_r(double r, double a)
{
    double rp, rm;
    horizons(a, &rp, &rm);
    return r + 2.0 * rp / (rp - rm) * std::log((r - rp) / 2.0) - 2.0 * rm / (rp - rm) * std::log((r - rm) / 2.0);
}

// Inverse tortoise map: safeguarded Newton iteration on y = ln(r - r+), where
// r*(y) is increasing with d r*/dy = (r^2 + a^2)/(r - r-).  Returns r and
// Delta = x (x + r+ - r-), x = r - r+, accurate near the horizon.
static void r_of_rstar(double rs, double a, double *r_out, double *D_out)
{
    double rp, rm;
    horizons(a, &rp, &rm);
    const double kp = 2.0 * rp / (rp - rm), km = 2.0 * rm / (rp - rm);
    const double dr = rp - rm;
    auto f = [&](double y) {
        const double x = std::exp(y);
        return rp + x + kp * (y - std::log(2.0)) - km * std::log((x + dr) / 2.0) - rs;
    };
    double lo = -1500.0, hi = 30.0;
    // starting guess: near-horizon asymptote, or r ~ r* far out
    double y = rs < 10.0 ? (rs - rp + km * std::log(dr / 2.0)) / kp + std::log(2.0)
                         : std::log(std::max(rs - rp, 1.0));
    y = std::min(std::max(y, lo), hi);
    for (int it = 0; it < 200; ++it) {
        const double fy = f(y);
        if (fy == 0.0) break;
        if (fy < 0) lo = y; else hi = y;
        const double x = std::exp(y);
        const double r = rp + x;
        const double dfy = (r * r + a * a) / (x + dr);
        double yn = y - fy / dfy;
        if (!(yn > lo && yn < hi)) yn = 0.5 * (lo + hi);
        if (std::fabs(yn - y) <= 4e-16 * std::max(1.0, std::fabs(y))) { y = yn; break; }
        y = yn;
    }
    const double x = std::exp(y);
    *r_out = rp + x;
    *D_out = x * (x + dr);
}

static bool valid_grid(const teuk_grid *g)
{
    return g && g->nr >= 4 && g->nth >= 2 && g->nth <= 4096 && g->rstar_min >= -1000.0 &&
           g->rstar_max > g->rstar_min && std::isfinite(g->rstar_max) && g->rstar_max <= 1e6;
}

static bool valid_physics(double a, int s)
{
    return std::isfinite(a) && std::fabs(a) < 1.0 && (s == -2 || s == 0 || s == 2);
}

static void destroy_graphs(teuk_handle *h)
{
    for (auto &row : h->graph)
        for (auto &g : row)
            if (g) { cudaGraphExecDestroy(g); g = nullptr; }
}

// ---------------------------------------------------------------------------
// Time-step rule
// ---------------------------------------------------------------------------

extern "C" int teuk_stable_dt(const teuk_grid *g, double a, int s, int m, double c_r, double c_theta,
                              double *dt_out)
{
    if (!valid_grid(g) || !valid_physics(a, s) || !(c_r > 0) || !(c_theta > 0) || !dt_out)
        return TEUK_ERR_BAD_ARG;
    const int nr = g->nr, nth = g->nth;
    const double hh = (g->rstar_max - g->rstar_min) / (nr - 1);
    const double dth = kPi / nth;
    const int rows = 2 * nr - 1;  // nodes then mid-points
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<double> bmax(nt, 0.0), gmax(nt, 0.0);
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < nt; ++t)
        pool.emplace_back([&, t]() {
            for (int row = (int)t; row < rows; row += (int)nt) {
                const double rs = row < nr ? g->rstar_min + row * hh : g->rstar_min + (row - nr + 0.5) * hh;
                double r, D;
                r_of_rstar(rs, a, &r, &D);
                for (int j = 0; j < nth; ++j) {
                    const double th = (j + 0.5) * dth;
                    const PhysCoef c = phys_coef(r, D, std::sin(th), std::cos(th), a, s, m);
                    const double cot = std::cos(th) / std::sin(th);
                    const double A = 1.0 / (dth * dth) + cot / (2.0 * dth);
                    const double C = 1.0 / (dth * dth) - cot / (2.0 * dth);
                    const double gb = std::hypot(c.W_re, c.W_im) +
                                      c.kappa * (2.0 / (dth * dth) + std::fabs(A) + std::fabs(C));
                    bmax[t] = std::max(bmax[t], c.b);
                    gmax[t] = std::max(gmax[t], gb);
                }
            }
        });
    for (auto &th : pool) th.join();
    const double b = *std::max_element(bmax.begin(), bmax.end());
    const double om = std::sqrt(*std::max_element(gmax.begin(), gmax.end()));
    *dt_out = std::min(c_r * hh / b, c_theta / om);
    return TEUK_OK;
}

// ---------------------------------------------------------------------------
// Create / destroy
// ---------------------------------------------------------------------------

namespace {
struct Arena {
    size_t off = 0;
    template <typename T>
    size_t take(size_t count)
    {
        const size_t o = off;
        off += ((count * sizeof(T) + 255) / 256) * 256;
        return o;
    }
};
}  // namespace

// Automatic launch shape of the fused kernel: about 16 resident warps per SM
// (enough to hide the load latency), in as few, long strips as that allows,
// since every strip recomputes one predictor row.
static void choose_launch(teuk_handle *h, int rows_per_block)
{
    const int rows = h->nr - 2;
    if (rows_per_block <= 0) {
        const int threads = fused_block_threads(h->nth);
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm,
                                                          fused_kernel_ptr(h->sp.real_coef, h->sp.fixed_point, h->sp.ko),
                                                          threads, fused_smem_bytes(h->nth, h->sp.ko)) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        const int want = std::max(1, 16 / std::max(1, threads / 32));
        per_sm = std::min(per_sm, want);
        const int target = std::max(1, h->num_sms * per_sm);
        rows_per_block = (rows + target - 1) / target;
    }
    h->rows_per_block = std::max(1, std::min(rows_per_block, rows));
    h->nblocks = (rows + h->rows_per_block - 1) / h->rows_per_block;
}

extern "C" int teuk_destroy(teuk_handle *h)
{
    if (!h) return TEUK_ERR_BAD_ARG;
    if (h->in_batch) return fail(h, TEUK_ERR_STATE, "teuk_destroy: the handle belongs to a batch (remove it first)");
    if (h->stream || h->own_stream) cudaStreamSynchronize(h->stream);
    destroy_graphs(h);
    if (h->d_src) cudaFree(h->d_src);
    if (h->d_ring) cudaFree(h->d_ring);
    if (h->phiH) cudaFree(h->phiH);
    if (h->arena) cudaFree(h->arena);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return TEUK_OK;
}

extern "C" int teuk_create(const teuk_grid *g, double a, int s, int m, void *cuda_stream, teuk_handle **out)
{
    if (!out) return TEUK_ERR_BAD_ARG;
    *out = nullptr;
    if (!valid_grid(g) || !valid_physics(a, s) || !(g->dt > 0) || !std::isfinite(g->dt) ||
        std::abs(m) > 1000000)
        return TEUK_ERR_BAD_ARG;
    teuk_handle *h = new (std::nothrow) teuk_handle();
    if (!h) return TEUK_ERR_OOM;
    h->nr = g->nr;
    h->nth = g->nth;
    h->s = s;
    h->m = m;
    h->a = a;
    h->parity = (std::abs(m) % 2 == 0) ? 1 : -1;
    h->rstar_min = g->rstar_min;
    h->rstar_max = g->rstar_max;
    h->h = (g->rstar_max - g->rstar_min) / (g->nr - 1);
    h->dth = kPi / g->nth;
    h->dt = g->dt;
    auto bail = [&](int code) { teuk_destroy(h); return code; };

    if (cudaGetDevice(&h->device) != cudaSuccess) return bail(TEUK_ERR_CUDA);
    if (cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
        return bail(TEUK_ERR_CUDA);
    if (cuda_stream) {
        h->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(TEUK_ERR_CUDA);
        h->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return bail(TEUK_ERR_CUDA);

    const int nr = h->nr, nth = h->nth;
    const size_t N = (size_t)nr * nth, Nm = (size_t)(nr - 1) * nth;

    // radial tables (nodes, mid-points) and angular tables
    std::vector<double> tab(2 * (size_t)nr + 2 * (size_t)(nr - 1) + 3 * (size_t)nth);
    double *r_node = tab.data(), *D_node = r_node + nr, *r_mid = D_node + nr, *D_mid = r_mid + (nr - 1);
    double *sin_th = D_mid + (nr - 1), *cos_th = sin_th + nth, *cot_th = cos_th + nth;
    for (int i = 0; i < nr; ++i) r_of_rstar(h->rstar_min + i * h->h, a, &r_node[i], &D_node[i]);
    for (int i = 0; i < nr - 1; ++i) r_of_rstar(h->rstar_min + (i + 0.5) * h->h, a, &r_mid[i], &D_mid[i]);
    for (int j = 0; j < nth; ++j) {
        const double th = (j + 0.5) * h->dth;
        sin_th[j] = std::sin(th);
        cos_th[j] = std::cos(th);
        cot_th[j] = cos_th[j] / sin_th[j];
    }

    Arena ar;
    size_t o_phi[2], o_pi[2];
    for (int b = 0; b < 2; ++b) { o_phi[b] = ar.take<double2>(N); o_pi[b] = ar.take<double2>(N); }
    const size_t o_pa = ar.take<double>(Nm), o_pb = ar.take<double>(Nm), o_eb = ar.take<double>(Nm),
                 o_KAp = ar.take<double>(Nm), o_KCp = ar.take<double>(Nm);
    const size_t o_P1 = ar.take<double2>(Nm), o_Q1 = ar.take<double2>(Nm), o_Q2 = ar.take<double2>(Nm);
    const size_t o_tb = ar.take<double>(N), o_nt2 = ar.take<double>(N), o_KAc = ar.take<double>(N),
                 o_KCc = ar.take<double>(N);
    const size_t o_R1 = ar.take<double2>(N), o_R3 = ar.take<double2>(N), o_R4 = ar.take<double2>(N);
    const size_t o_b = ar.take<double>(N);
    const size_t o_tab = ar.take<double>(tab.size());
    const size_t o_step = ar.take<long long>(1), o_cnt = ar.take<unsigned long long>(1);
    if (cudaMalloc(&h->arena, ar.off) != cudaSuccess) {
        cudaGetLastError();
        return bail(TEUK_ERR_OOM);
    }
    char *A = h->arena;
    for (int b = 0; b < 2; ++b) {
        h->phi[b] = (double2 *)(A + o_phi[b]);
        h->pi[b] = (double2 *)(A + o_pi[b]);
    }
    h->b_node = (double *)(A + o_b);
    h->d_step = (long long *)(A + o_step);
    h->d_count = (unsigned long long *)(A + o_cnt);
    double *d_tab = (double *)(A + o_tab);

    SetupParams su{};
    su.nr = nr; su.nth = nth; su.s = s; su.m = m; su.parity = h->parity;
    // a = 0, or s = m = 0: every coefficient is real
    su.real_coef = (a == 0.0 || (s == 0 && m == 0)) ? 1 : 0;
    su.a = a; su.h = h->h; su.dth = h->dth; su.dt = h->dt;
    su.r_node = d_tab; su.D_node = d_tab + nr; su.r_mid = d_tab + 2 * nr; su.D_mid = su.r_mid + (nr - 1);
    su.sin_th = su.D_mid + (nr - 1); su.cos_th = su.sin_th + nth; su.cot_th = su.cos_th + nth;
    su.pa = (double *)(A + o_pa); su.pb = (double *)(A + o_pb); su.eb = (double *)(A + o_eb);
    su.KAp = (double *)(A + o_KAp); su.KCp = (double *)(A + o_KCp);
    su.P1 = (double2 *)(A + o_P1); su.Q1 = (double2 *)(A + o_Q1); su.Q2 = (double2 *)(A + o_Q2);
    su.tb = (double *)(A + o_tb); su.nt2 = (double *)(A + o_nt2);
    su.KAc = (double *)(A + o_KAc); su.KCc = (double *)(A + o_KCc);
    su.R1 = (double2 *)(A + o_R1); su.R3 = (double2 *)(A + o_R3); su.R4 = (double2 *)(A + o_R4);
    su.b_node = h->b_node;

    if (cudaMemcpyAsync(d_tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream) !=
            cudaSuccess ||
        cudaMemsetAsync(h->arena, 0, o_pa, h->stream) != cudaSuccess ||  // both state copies
        cudaMemsetAsync(h->d_step, 0, 2 * 256, h->stream) != cudaSuccess ||
        launch_setup(su, h->stream) != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess)
        return bail(TEUK_ERR_CUDA);

    StepParams &p = h->sp;
    p.nr = nr; p.nth = nth; p.dt = h->dt; p.q = 0.25 * h->dt; p.half_dt = 0.5 * h->dt;
    p.one = 1.0; p.nzero = -0.0;
    p.real_coef = su.real_coef;
    p.fixed_point = 1;
    p.ko = 0;  // the bare scheme until teuk_set_dissipation
    p.parity = h->parity;
    p.k0 = 1.0; p.k1 = 0.0; p.k2 = 0.0; p.k3 = 0.0;
    p.kd = 0.0;
    p.kd_shift = StepParams::kNotPow2;
    h->su = su;
    p.pred = PredPlanes{su.pa, su.pb, su.eb, su.KAp, su.KCp, su.P1, su.Q1, su.Q2};
    p.corr = CorrPlanes{su.tb, su.nt2, su.KAc, su.KCc, su.R1, su.R3, su.R4};
    p.src = SourceWindow{0, -1, 0, -1, nullptr, nullptr, 0.0, 0};
    p.ext = Extraction{-1, 1, 1, nullptr};
    p.step_base = h->d_step;
    h->variant = nth <= kTileMaxThreads ? 2 : 1;
    // Shared memory stays below the 48 KB default: the fused kernel takes
    // 64 (nth + 2) bytes, plus 64 (nth + 6) with the dissipation, <= 33 KB;
    // a split tile 16 R (TW + 2), plus 32 R (TW + 6), <= 25 KB.
    if (nth <= kFusedMaxNth) choose_launch(h, 0);  // the fused kernel's shape, for when it is selected
    if (h->variant != 0) {  // the two-kernel variants keep the half step in device memory
        if (cudaMalloc(&h->phiH, 2 * Nm * sizeof(double2)) != cudaSuccess) { cudaGetLastError(); return bail(TEUK_ERR_OOM); }
        h->piH = h->phiH + Nm;
    }
    *out = h;
    return TEUK_OK;
}

// ---------------------------------------------------------------------------
// Initial data, source, extraction
// ---------------------------------------------------------------------------

static int reset_counters(teuk_handle *h)
{
    h->cur = 0;
    h->nstep = 0;
    h->drained = 0;
    CU(cudaMemsetAsync(h->d_step, 0, sizeof(long long), h->stream));
    return TEUK_OK;
}

static int finish_initial(teuk_handle *h, bool have_pi)
{
    const int nr = h->nr, nth = h->nth;
    CU(launch_zero_boundary_rows(h->phi[0], h->pi[0], nr, nth, h->stream));
    if (!have_pi) CU(launch_time_symmetric_pi(h->phi[0], h->pi[0], h->b_node, nr, nth, 1.0 / (2.0 * h->h), h->stream));
    // the second copy's boundary rows are never written by the step kernels
    CU(launch_zero_boundary_rows(h->phi[1], h->pi[1], nr, nth, h->stream));
    return reset_counters(h);
}

extern "C" int teuk_set_initial(teuk_handle *h, const double *phi, const double *pi)
{
    if (!h || !phi) return fail(h, TEUK_ERR_BAD_ARG, "teuk_set_initial: NULL argument");
    if (h->in_batch) return fail(h, TEUK_ERR_STATE, "teuk_set_initial: the handle belongs to a batch (remove it first)");
    const size_t bytes = (size_t)h->nr * h->nth * sizeof(double2);
    CU(cudaMemcpyAsync(h->phi[0], phi, bytes, cudaMemcpyHostToDevice, h->stream));
    if (pi) CU(cudaMemcpyAsync(h->pi[0], pi, bytes, cudaMemcpyHostToDevice, h->stream));
    int rc = finish_initial(h, pi != nullptr);
    if (rc) return rc;
    CU(cudaStreamSynchronize(h->stream));
    return TEUK_OK;
}

extern "C" int teuk_set_state(teuk_handle *h, const double *phi, const double *pi, long step)
{
    if (!h || !phi || !pi || step < 0) return fail(h, TEUK_ERR_BAD_ARG, "teuk_set_state: NULL array or step < 0");
    if (h->in_batch) return fail(h, TEUK_ERR_STATE, "teuk_set_state: the handle belongs to a batch (remove it first)");
    const size_t bytes = (size_t)h->nr * h->nth * sizeof(double2);
    CU(cudaMemcpyAsync(h->phi[0], phi, bytes, cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(h->pi[0], pi, bytes, cudaMemcpyHostToDevice, h->stream));
    CU(launch_zero_boundary_rows(h->phi[0], h->pi[0], h->nr, h->nth, h->stream));
    CU(launch_zero_boundary_rows(h->phi[1], h->pi[1], h->nr, h->nth, h->stream));
    CU(launch_set_counter(h->d_step, step, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    h->cur = 0;
    h->nstep = step;
    h->drained = h->sp.ext.i_ext >= 0 ? step / h->sp.ext.every : 0;
    return TEUK_OK;
}

extern "C" int teuk_set_initial_device(teuk_handle *h, const double *phi, const double *pi)
{
    if (!h || !phi) return fail(h, TEUK_ERR_BAD_ARG, "teuk_set_initial_device: NULL argument");
    if (h->in_batch) return fail(h, TEUK_ERR_STATE, "teuk_set_initial_device: the handle belongs to a batch (remove it first)");
    const size_t bytes = (size_t)h->nr * h->nth * sizeof(double2);
    CU(cudaMemcpyAsync(h->phi[0], phi, bytes, cudaMemcpyDeviceToDevice, h->stream));
    if (pi) CU(cudaMemcpyAsync(h->pi[0], pi, bytes, cudaMemcpyDeviceToDevice, h->stream));
    return finish_initial(h, pi != nullptr);
}

extern "C" int teuk_set_source(teuk_handle *h, const teuk_orbit *o)
{
    if (!h) return TEUK_ERR_BAD_ARG;
    if (h->in_batch) return fail(h, TEUK_ERR_STATE, "teuk_set_source: the handle belongs to a batch (remove it first)");
    CU(cudaStreamSynchronize(h->stream));
    destroy_graphs(h);
    if (!o) {
        if (h->d_src) { cudaFree(h->d_src); h->d_src = nullptr; }
        h->sp.src = SourceWindow{0, -1, 0, -1, nullptr, nullptr, 0.0, 0};
        return TEUK_OK;
    }
    double rp, rm;
    horizons(h->a, &rp, &rm);
    if (!(o->r0 > rp) || !std::isfinite(o->r0) || !(o->sigma > 0) || !std::isfinite(o->sigma) ||
        !std::isfinite(o->amplitude))
        return fail(h, TEUK_ERR_BAD_ARG, "teuk_set_source: need r0 > r+, sigma > 0");
    const double rs0 = rstar_of_r(o->r0, h->a);
    if (!(rs0 > h->rstar_min && rs0 < h->rstar_max))
        return fail(h, TEUK_ERR_BAD_ARG, "teuk_set_source: r*(r0) outside the grid");
    const double sig_th = o->sigma / o->r0;
    const int nr = h->nr, nth = h->nth;
    auto gauss = [&](double rs, double th) {
        const double z = (rs - rs0) * (rs - rs0) / (2.0 * o->sigma * o->sigma) +
                         (th - 0.5 * kPi) * (th - 0.5 * kPi) / (2.0 * sig_th * sig_th);
        return z > 50.0 ? 0.0 : std::exp(-z);
    };
    // rows where the Gaussian can be non-zero: |r* - r*0| <= 10 sigma (exponent <= 50)
    const double reach = 10.0 * o->sigma;
    const int lo_n = std::max(0, (int)std::floor((rs0 - reach - h->rstar_min) / h->h) - 1);
    const int hi_n = std::min(nr - 1, (int)std::ceil((rs0 + reach - h->rstar_min) / h->h) + 1);
    double norm = 0.0;
    std::vector<double> gn((size_t)(hi_n - lo_n + 1) * nth), gm((size_t)(hi_n - lo_n + 1) * nth, 0.0);
    for (int i = lo_n; i <= hi_n; ++i)
        for (int j = 0; j < nth; ++j) {
            const double v = gauss(h->rstar_min + i * h->h, (j + 0.5) * h->dth);
            gn[(size_t)(i - lo_n) * nth + j] = v;
            norm += v * h->h * h->dth;
        }
    if (!(norm > 0)) return fail(h, TEUK_ERR_BAD_ARG, "teuk_set_source: Gaussian misses every grid node");
    const int lo_m = lo_n, hi_m = std::min(nr - 2, hi_n);
    for (int i = lo_m; i <= hi_m; ++i)
        for (int j = 0; j < nth; ++j)
            gm[(size_t)(i - lo_m) * nth + j] = gauss(h->rstar_min + (i + 0.5) * h->h, (j + 0.5) * h->dth);
    const double cP = 0.5 * h->dt * o->amplitude / norm, cC = h->dt * o->amplitude / norm;
    for (auto &v : gn) v *= cC;
    for (auto &v : gm) v *= cP;
    const size_t nmid = (size_t)(hi_m - lo_m + 1) * nth, nnode = (size_t)(hi_n - lo_n + 1) * nth;
    std::vector<double> buf(nmid + nnode);
    std::copy(gm.begin(), gm.begin() + nmid, buf.begin());
    std::copy(gn.begin(), gn.end(), buf.begin() + nmid);
    if (h->d_src) { cudaFree(h->d_src); h->d_src = nullptr; }
    if (cudaMalloc(&h->d_src, buf.size() * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, TEUK_ERR_OOM, "teuk_set_source: out of device memory");
    }
    CU(cudaMemcpy(h->d_src, buf.data(), buf.size() * sizeof(double), cudaMemcpyHostToDevice));
    const double Om = o->prograde ? 1.0 / (o->r0 * std::sqrt(o->r0) + h->a)
                                  : -1.0 / (o->r0 * std::sqrt(o->r0) - h->a);
    // interior rows only: the boundary rows 0 and nr-1 are never updated
    h->sp.src = SourceWindow{lo_m, hi_m, std::max(1, lo_n), std::min(nr - 2, hi_n), h->d_src, h->d_src + nmid,
                             (double)h->m * Om, 1};
    // gC is indexed from node_lo: shift the pointer when the window was clipped at row 0
    h->sp.src.gC = h->d_src + nmid + (size_t)(h->sp.src.node_lo - lo_n) * nth;
    return TEUK_OK;
}

extern "C" int teuk_set_extraction(teuk_handle *h, double rstar_ext, int every, long capacity)
{
    if (!h) return TEUK_ERR_BAD_ARG;
    if (h->in_batch) return fail(h, TEUK_ERR_STATE, "teuk_set_extraction: the handle belongs to a batch (remove it first)");
    const int i = (int)std::floor((rstar_ext - h->rstar_min) / h->h + 0.5);
    if (!std::isfinite(rstar_ext) || i < 0 || i >= h->nr || every < 1 || capacity < 1)
        return fail(h, TEUK_ERR_BAD_ARG, "teuk_set_extraction: radius outside the grid, every < 1 or capacity < 1");
    CU(cudaStreamSynchronize(h->stream));
    destroy_graphs(h);
    if (h->d_ring) { cudaFree(h->d_ring); h->d_ring = nullptr; }
    if (cudaMalloc(&h->d_ring, (size_t)capacity * h->nth * sizeof(double2)) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, TEUK_ERR_OOM, "teuk_set_extraction: out of device memory");
    }
    // boundary rows are constant zero: sample row i is still well defined
    h->sp.ext = Extraction{i, every, capacity, h->d_ring};
    h->drained = h->nstep / every;
    return TEUK_OK;
}

// ---------------------------------------------------------------------------
// Stepping
// ---------------------------------------------------------------------------

static cudaError_t launch_one(teuk_handle *h, int from, int k, cudaStream_t st)
{
    // never launch a variant without its buffers
    if (!h->phi[from] || !h->pi[from] || !h->phi[1 - from] || !h->pi[1 - from] ||
        (h->variant != 0 && (!h->phiH || !h->piH)))
        return cudaErrorInvalidValue;
    if (h->variant == 0)
        return launch_step_fused(h->sp, h->phi[from], h->pi[from], h->phi[1 - from], h->pi[1 - from], k,
                                 h->rows_per_block, h->nblocks, st);
    if (h->variant == 2)
        return launch_step_split(h->sp, h->phi[from], h->pi[from], h->phi[1 - from], h->pi[1 - from], h->phiH,
                                 h->piH, k, st, h->pdl != 0, 2, h->split_rows);
    return launch_step_unfused(h->sp, h->phi[from], h->pi[from], h->phi[1 - from], h->pi[1 - from], h->phiH,
                               h->piH, k, st);
}

static int capture_graph(teuk_handle *h, int from)
{
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    int b = from;
    for (int k = 0; k < h->chunk && e == cudaSuccess; ++k) {
        e = launch_one(h, b, k, h->cap_stream);
        b = 1 - b;
    }
    if (e == cudaSuccess) e = launch_advance(h->d_step, h->chunk, h->cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(h, TEUK_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaError_t e3 = cudaGraphInstantiate(&h->graph[h->variant][from], g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) return fail(h, TEUK_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e3));
    return TEUK_OK;
}

// n steps on the handle's stream (graph replay per chunk); also used by
// batches that run their jobs with per-job launches.
int teuk_step_handle(teuk_handle *h, long n)
{
    while (n >= h->chunk) {
        if (!h->graph[h->variant][h->cur]) {
            int rc = capture_graph(h, h->cur);
            if (rc) return rc;
        }
        CU(cudaGraphLaunch(h->graph[h->variant][h->cur], h->stream));
        n -= h->chunk;
        h->nstep += h->chunk;
    }
    if (n > 0) {
        for (int k = 0; k < n; ++k) {
            CU(launch_one(h, h->cur, k, h->stream));
            h->cur = 1 - h->cur;
        }
        CU(launch_advance(h->d_step, n, h->stream));
        h->nstep += n;
    }
    return TEUK_OK;
}

extern "C" int teuk_set_stream(teuk_handle *h, void *cuda_stream)
{
    if (!h) return TEUK_ERR_BAD_ARG;
    CU(cudaStreamSynchronize(h->stream));  // everything queued on the old stream completes first
    if (h->own_stream) {
        cudaStreamDestroy(h->stream);
        h->own_stream = false;
    }
    h->stream = nullptr;
    if (cuda_stream) {
        h->stream = (cudaStream_t)cuda_stream;
    } else {
        CU(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    return TEUK_OK;
}

extern "C" int teuk_step(teuk_handle *h, long n)
{
    if (!h || n < 0) return fail(h, TEUK_ERR_BAD_ARG, "teuk_step: n < 0");
    if (h->in_batch) return fail(h, TEUK_ERR_STATE, "teuk_step: the handle belongs to a batch (remove it first)");
    return teuk_step_handle(h, n);
}

extern "C" int teuk_set_launch(teuk_handle *h, int rows_per_block)
{
    if (!h || rows_per_block < 0) return fail(h, TEUK_ERR_BAD_ARG, "teuk_set_launch: rows_per_block < 0");
    if (h->nth > kFusedMaxNth) return fail(h, TEUK_ERR_STATE, "teuk_set_launch: fused kernel needs nth <= 256");
    CU(cudaStreamSynchronize(h->stream));
    destroy_graphs(h);
    choose_launch(h, rows_per_block);
    return TEUK_OK;
}

extern "C" int teuk_set_option(teuk_handle *h, int option, long value)
{
    if (!h) return TEUK_ERR_BAD_ARG;
    if (h->in_batch) return fail(h, TEUK_ERR_STATE, "teuk_set_option: the handle belongs to a batch (remove it first)");
    switch (option) {
    case TEUK_OPT_PDL:
        if (value != 0 && value != 1) return fail(h, TEUK_ERR_BAD_ARG, "teuk_set_option: PDL is 0 or 1");
        CU(cudaStreamSynchronize(h->stream));
        destroy_graphs(h);
        h->pdl = (int)value;
        return TEUK_OK;
    case TEUK_OPT_GRAPH_CHUNK:
        if (value < 2 || value > 4096 || value % 2)
            return fail(h, TEUK_ERR_BAD_ARG, "teuk_set_option: graph chunk must be even, 2..4096");
        CU(cudaStreamSynchronize(h->stream));
        destroy_graphs(h);
        h->chunk = (int)value;
        return TEUK_OK;
    case TEUK_OPT_SPLIT_ROWS:
        if (value < 0 || value * split_tile_width(h->nth) > (h->sp.fixed_point ? kFxTileThreads : kTileMaxThreads))
            return fail(h, TEUK_ERR_BAD_ARG,
                        "teuk_set_option: split rows must be 0 or 1..(128 fixed point, 512 FP64) / (split tile width)");
        CU(cudaStreamSynchronize(h->stream));
        destroy_graphs(h);
        h->split_rows = (int)value;
        return TEUK_OK;
    case TEUK_OPT_FIXED_POINT:
        if (value != 0 && value != 1) return fail(h, TEUK_ERR_BAD_ARG, "teuk_set_option: fixed point is 0 or 1");
        CU(cudaStreamSynchronize(h->stream));
        destroy_graphs(h);
        h->sp.fixed_point = (int)value;
        if (h->variant == 0) choose_launch(h, h->rows_per_block);  // the fused kernel's occupancy depends on it
        return TEUK_OK;
    case TEUK_OPT_REAL_PATH: {
        if (value != 0 && value != 1) return fail(h, TEUK_ERR_BAD_ARG, "teuk_set_option: real path is 0 or 1");
        const int real = (value == 1 && (h->a == 0.0 || (h->s == 0 && h->m == 0))) ? 1 : 0;
        if (real == h->sp.real_coef) return TEUK_OK;
        CU(cudaStreamSynchronize(h->stream));
        destroy_graphs(h);
        h->su.real_coef = real;
        CU(launch_setup(h->su, h->stream));  // rewrite the planes in the other layout
        CU(cudaStreamSynchronize(h->stream));
        h->sp.real_coef = real;
        return TEUK_OK;
    }
    default:
        return fail(h, TEUK_ERR_BAD_ARG, "teuk_set_option: unknown option");
    }
}

extern "C" int teuk_set_dissipation(teuk_handle *h, double eps)
{
    if (!h) return TEUK_ERR_BAD_ARG;
    if (h->in_batch) return fail(h, TEUK_ERR_STATE, "teuk_set_dissipation: the handle belongs to a batch (remove it first)");
    if (!(eps == 0.0 || (eps >= 1e-9 && eps < 2.0)))
        return fail(h, TEUK_ERR_BAD_ARG, "teuk_set_dissipation: eps must be 0 or in [1e-9, 2)");
    CU(cudaStreamSynchronize(h->stream));
    destroy_graphs(h);  // the graphs hold the step parameters by value
    StepParams &p = h->sp;
    p.ko = eps > 0.0 ? 1 : 0;
    p.k0 = 1.0 - 20.0 * eps / 64.0;
    p.k1 = 15.0 * eps / 64.0;
    p.k2 = -6.0 * eps / 64.0;
    p.k3 = eps / 64.0;
    p.kd = -eps / 64.0;
    {
        int ex = 0;
        const double fr = std::frexp(eps / 64.0, &ex);  // eps/64 = fr 2^ex, fr in [0.5, 1)
        p.kd_shift = (eps > 0.0 && fr == 0.5) ? ex - 1 : StepParams::kNotPow2;
    }
    h->eps = eps;
    if (h->variant == 0 && h->nth <= kFusedMaxNth) choose_launch(h, h->rows_per_block);  // occupancy depends on it
    return TEUK_OK;
}

extern "C" int teuk_get_launch(const teuk_handle *h, int *rows_per_block, int *nblocks)
{
    if (!h || !rows_per_block || !nblocks) return TEUK_ERR_BAD_ARG;
    *rows_per_block = h->rows_per_block;
    *nblocks = h->nblocks;
    return TEUK_OK;
}

extern "C" int teuk_time_kernels(teuk_handle *h, long n, double *ms_out)
{
    if (!h || n < 1 || !ms_out) return fail(h, TEUK_ERR_BAD_ARG, "teuk_time_kernels: n >= 1 and ms_out needed");
    if (h->in_batch) return fail(h, TEUK_ERR_STATE, "teuk_time_kernels: the handle belongs to a batch (remove it first)");
    cudaEvent_t ev[3];
    for (auto &e : ev) CU(cudaEventCreate(&e));
    double acc[2] = {0.0, 0.0};
    int rc = TEUK_OK;
    for (long k = 0; k < n && rc == TEUK_OK; ++k) {
        const int from = h->cur;
        cudaError_t e = cudaEventRecord(ev[0], h->stream);
        if (h->variant == 0) {
            if (e == cudaSuccess)
                e = launch_step_fused(h->sp, h->phi[from], h->pi[from], h->phi[1 - from], h->pi[1 - from], (int)k,
                                      h->rows_per_block, h->nblocks, h->stream);
            if (e == cudaSuccess) e = cudaEventRecord(ev[1], h->stream);
            if (e == cudaSuccess) e = cudaEventRecord(ev[2], h->stream);
        } else {
            for (int part = 0; part < 2 && e == cudaSuccess; ++part) {
                e = h->variant == 2 ? launch_step_split(h->sp, h->phi[from], h->pi[from], h->phi[1 - from],
                                                        h->pi[1 - from], h->phiH, h->piH, (int)k, h->stream, false,
                                                        part, h->split_rows)
                                    : launch_step_unfused(h->sp, h->phi[from], h->pi[from], h->phi[1 - from],
                                                          h->pi[1 - from], h->phiH, h->piH, (int)k, h->stream,
                                                          part);
                if (e == cudaSuccess) e = cudaEventRecord(ev[1 + part], h->stream);
            }
        }
        float t01 = 0, t12 = 0;
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[2]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t01, ev[0], ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t12, ev[1], ev[2]);
        if (e != cudaSuccess) {
            rc = fail(h, TEUK_ERR_CUDA, std::string("teuk_time_kernels: ") + cudaGetErrorString(e));
            break;
        }
        acc[0] += t01;
        acc[1] += h->variant == 0 ? 0.0 : t12;  // the fused variant has one kernel per step
        h->cur = 1 - from;
    }
    if (rc == TEUK_OK) {
        cudaError_t e = launch_advance(h->d_step, n, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = fail(h, TEUK_ERR_CUDA, std::string("teuk_time_kernels: ") + cudaGetErrorString(e));
        h->nstep += n;
        ms_out[0] = acc[0] / n;
        ms_out[1] = acc[1] / n;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    return rc;
}

extern "C" long teuk_launches_for(const teuk_handle *h, long n)
{
    if (!h || n < 0) return -1;
    const long per = h->variant == 0 ? 1 : 2;  // the two-kernel and split variants launch twice per step
    const long full = n / h->chunk, rem = n % h->chunk;
    return full * (h->chunk * per + 1) + (rem ? rem * per + 1 : 0);
}

extern "C" int teuk_set_kernel(teuk_handle *h, int variant)
{
    if (!h || variant < 0 || variant > 2) return fail(h, TEUK_ERR_BAD_ARG, "teuk_set_kernel: variant 0, 1 or 2");
    if (h->in_batch) return fail(h, TEUK_ERR_STATE, "teuk_set_kernel: the handle belongs to a batch (remove it first)");
    if ((variant == 0 && h->nth > kFusedMaxNth) || (variant == 2 && h->nth > kTileMaxThreads))
        return fail(h, TEUK_ERR_BAD_ARG, "teuk_set_kernel: fused kernel needs nth <= 256, split nth <= 512");
    if (variant != 0 && !h->phiH) {
        const size_t Nm = (size_t)(h->nr - 1) * h->nth;
        if (cudaMalloc(&h->phiH, 2 * Nm * sizeof(double2)) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, TEUK_ERR_OOM, "teuk_set_kernel: out of device memory");
        }
        h->piH = h->phiH + Nm;
    }
    h->variant = variant;
    return TEUK_OK;
}


// ---------------------------------------------------------------------------
// One time step without any device allocation
// ---------------------------------------------------------------------------
//
// For callers that cannot call cudaMalloc while they step: real-time loops
// that must not block in the allocator, and processes whose device memory is
// owned by another framework's pool (the library must not take memory behind
// that pool's back).  The half step lives in the static array below instead
// of a per-handle buffer.  The array (32 MiB) is part of the library image:
// every GPU that loads libteuk holds it until the process exits.

static const long long kNoAllocMaxMid = 1LL << 20;  // mid-point values: (nr - 1) * nth <= 1,048,576
// Layout: Phi^{1/2} [kNoAllocMaxMid] double2, Pi^{1/2} [kNoAllocMaxMid] double2, then
// the step counter read by the kernels (one 256-byte slot).
static const size_t kNoAllocScratchBytes = 2 * (size_t)kNoAllocMaxMid * sizeof(double2) + 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Host-side device addresses of g_noalloc_scratch, one per device, looked up
// on the first call made with that device current.
static void *g_noalloc_ptr[128];

extern "C" int teuk_step_noalloc(teuk_handle *h, const double *phi_in, const double *pi_in, double *phi_out,
                                 double *pi_out, long step_index)
{
    if (!h || !phi_in || !pi_in || !phi_out || !pi_out || step_index < 0)
        return fail(h, TEUK_ERR_BAD_ARG, "teuk_step_noalloc: NULL buffer or negative step index");
    if (h->in_batch) return fail(h, TEUK_ERR_STATE, "teuk_step_noalloc: the handle belongs to a batch (remove it first)");
    if (h->nth > kTileMaxThreads)
        return fail(h, TEUK_ERR_BAD_ARG, "teuk_step_noalloc: needs nth <= 512");
    const long long mids = (long long)(h->nr - 1) * h->nth;
    if (mids > kNoAllocMaxMid)
        return fail(h, TEUK_ERR_BAD_ARG,
                    "teuk_step_noalloc: (nr - 1) * nth = " + std::to_string(mids) +
                        " exceeds the static scratch of 1048576 mid-point values (32 MiB)");
    // every buffer spans nr * nth complex values; no output may share a byte with
    // an input or with the other output
    {
        const size_t span = (size_t)h->nr * h->nth * sizeof(double2);
        const char *in[2] = {(const char *)phi_in, (const char *)pi_in};
        const char *out[2] = {(const char *)phi_out, (const char *)pi_out};
        auto overlap = [span](const char *x, const char *y) { return x < y + span && y < x + span; };
        if (overlap(out[0], out[1]) || overlap(out[0], in[0]) || overlap(out[0], in[1]) || overlap(out[1], in[0]) ||
            overlap(out[1], in[1]))
            return fail(h, TEUK_ERR_BAD_ARG, "teuk_step_noalloc: an output buffer overlaps an input or the other output");
    }
    int dev = -1;
    CU(cudaGetDevice(&dev));
    if (dev != h->device || dev < 0 || dev >= 128)
        return fail(h, TEUK_ERR_BAD_ARG, "teuk_step_noalloc: the handle's device must be the current device");
    if (!g_noalloc_ptr[dev]) {
        void *ptr = nullptr;
        CU(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        g_noalloc_ptr[dev] = ptr;
    }
    char *base = (char *)g_noalloc_ptr[dev];
    double2 *phiH = (double2 *)base;
    double2 *piH = phiH + kNoAllocMaxMid;
    long long *step = (long long *)(base + 2 * (size_t)kNoAllocMaxMid * sizeof(double2));

    StepParams p = h->sp;
    p.ext.i_ext = -1;  // no waveform sampling: the caller owns the output state
    p.step_base = step;
    // the step counter is written on the stream before the kernels read it; the
    // half step is fully rewritten by the predictor before the corrector reads it
    CU(launch_set_counter(step, step_index, h->stream));
    CU(launch_step_split(p, (const double2 *)phi_in, (const double2 *)pi_in, (double2 *)phi_out,
                         (double2 *)pi_out, phiH, piH, 0, h->stream, false));
    CU(launch_zero_boundary_rows((double2 *)phi_out, (double2 *)pi_out, h->nr, h->nth, h->stream));
    return TEUK_OK;
}

// ---------------------------------------------------------------------------
// Results
// ---------------------------------------------------------------------------

extern "C" int teuk_extract(teuk_handle *h, double *t_out, double *phi_out, long cap, long *n_out)
{
    if (!h || !n_out || cap < 0 || (cap > 0 && (!t_out || !phi_out)))
        return fail(h, TEUK_ERR_BAD_ARG, "teuk_extract: bad argument");
    *n_out = 0;
    if (h->sp.ext.i_ext < 0) return fail(h, TEUK_ERR_STATE, "teuk_extract: no extraction set");
    CU(cudaStreamSynchronize(h->stream));
    const long long every = h->sp.ext.every, capacity = h->sp.ext.capacity;
    const long long total = h->nstep / every;
    int rc = TEUK_OK;
    if (total - h->drained > capacity) {
        h->drained = total - capacity;
        rc = fail(h, TEUK_ERR_OVERFLOW, "teuk_extract: ring buffer overflowed; oldest samples lost");
    }
    const long long n = std::min<long long>(cap, total - h->drained);
    const size_t row = (size_t)h->nth * sizeof(double2);
    long long done = 0;
    while (done < n) {
        const long long s = h->drained + done + 1;  // 1-based sample number
        const long long slot = (s - 1) % capacity;
        const long long run = std::min<long long>(n - done, capacity - slot);
        CU(cudaMemcpy(phi_out + (size_t)done * 2 * h->nth, h->d_ring + (size_t)slot * h->nth, (size_t)run * row,
                      cudaMemcpyDeviceToHost));
        for (long long q = 0; q < run; ++q) t_out[done + q] = (double)((s + q) * every) * h->dt;
        done += run;
    }
    h->drained += n;
    *n_out = (long)n;
    return rc;
}

extern "C" int teuk_get_state(teuk_handle *h, double *phi, double *pi)
{
    if (!h) return TEUK_ERR_BAD_ARG;
    const size_t bytes = (size_t)h->nr * h->nth * sizeof(double2);
    if (phi) CU(cudaMemcpyAsync(phi, h->phi[h->cur], bytes, cudaMemcpyDeviceToHost, h->stream));
    if (pi) CU(cudaMemcpyAsync(pi, h->pi[h->cur], bytes, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return TEUK_OK;
}

extern "C" int teuk_get_state_device(teuk_handle *h, double *phi, double *pi)
{
    if (!h) return TEUK_ERR_BAD_ARG;
    const size_t bytes = (size_t)h->nr * h->nth * sizeof(double2);
    if (phi) CU(cudaMemcpyAsync(phi, h->phi[h->cur], bytes, cudaMemcpyDeviceToDevice, h->stream));
    if (pi) CU(cudaMemcpyAsync(pi, h->pi[h->cur], bytes, cudaMemcpyDeviceToDevice, h->stream));
    return TEUK_OK;
}

extern "C" long teuk_step_count(const teuk_handle *h) { return h ? (long)h->nstep : -1; }

extern "C" int teuk_check_finite(teuk_handle *h, int *finite)
{
    if (!h || !finite) return fail(h, TEUK_ERR_BAD_ARG, "teuk_check_finite: NULL argument");
    unsigned long long cnt = 0;
    CU(cudaMemsetAsync(h->d_count, 0, sizeof(cnt), h->stream));
    CU(launch_nonfinite_count(h->phi[h->cur], h->pi[h->cur], (long long)h->nr * h->nth, h->d_count, h->stream));
    CU(cudaMemcpyAsync(&cnt, h->d_count, sizeof(cnt), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    *finite = cnt == 0;
    return cnt == 0 ? TEUK_OK : fail(h, TEUK_ERR_NONFINITE, "state holds NaN or Inf");
}

extern "C" const char *teuk_last_error(const teuk_handle *h) { return h ? h->err.c_str() : ""; }

extern "C" const char *teuk_strerror(int code)
{
    switch (code) {
    case TEUK_OK: return "ok";
    case TEUK_ERR_BAD_ARG: return "bad argument";
    case TEUK_ERR_OOM: return "out of memory";
    case TEUK_ERR_CUDA: return "CUDA error";
    case TEUK_ERR_NONFINITE: return "non-finite state";
    case TEUK_ERR_STATE: return "invalid call for the handle's state";
    case TEUK_ERR_OVERFLOW: return "waveform ring buffer overflow";
    default: return "unknown error";
    }
}
