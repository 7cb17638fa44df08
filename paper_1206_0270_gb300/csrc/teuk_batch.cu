// teuk_batch.cu -- batched stepping of many independent solver handles.
//
// A template bank is thousands of independent (a, r0, m) evolutions of
// uneven grid size and length.  Two ways to advance a batch:
//   mode 1: every job with its own split kernels on its own stream (graph
//     replay per chunk), the jobs running concurrently;
//   mode 0: every time step is one predictor and one corrector launch per
//     group of up to kMultiMaxJobs jobs that share an arithmetic
//     (lw_predict_multi / lw_correct_multi over the tiles of all of them),
//     with one CTA per tile or a persistent grid of resident CTAs.  Jobs
//     advance in slices of min(chunk, smallest remaining step count) steps,
//     so a job that reaches its step count leaves at a slice boundary; full
//     slices replay a CUDA graph captured for the current set of jobs.
// Both run the split kernels' tile code, so every job gets the bits it gets
// alone.  teuk_batch_autotune times the launch forms on the jobs themselves
// (the timed steps count as progress).
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "teuk.h"
#include "teuk_handle.h"
#include "teuk_internal.h"

using namespace teuk;

struct teuk_batch {
    int device = 0;
    cudaStream_t stream = nullptr, cap = nullptr;
    bool own_stream = false;
    struct Job {
        teuk_handle *h = nullptr;
        long long remaining = 0;
        bool member = false;     // still in the batch (not removed)
        cudaEvent_t done = nullptr;  // per-job launches: the job's slice has finished
    };
    std::vector<Job> jobs;

    // the active set (rebuilt when it changes): the jobs' descriptors on the
    // device (for the step-counter update) and the multi-job launch groups
    JobDesc *d_jobs = nullptr;
    int cap_jobs = 0;
    std::vector<int> active;  // job ids in table order
    std::vector<JobDesc> host_desc;
    struct Group {
        int real = 0, fx = 0, ko = 0, block = 0;
        size_t smem = 0;
        int ctas = 0;               // CTAs per launch: 0 = one per tile
        std::vector<int> members;   // indices into active
        MultiArgs pred, corr;       // predictor tiles (nr - 1 rows), corrector tiles (nr - 2 rows)
    };
    std::vector<Group> groups;
    int block_request = 0;  // 0 = automatic (128 threads for fixed-point jobs, 256 for FP64 ones)
    int ctas_request = 0;   // 0 = one CTA per tile; k > 0 = persistent, k CTAs per SM (at most what fits)
    bool layout_dirty = true;
    cudaGraphExec_t graph = nullptr;
    int pdl = 1, chunk = 64;
    int mode = 1;                     // 0: multi-job launches per group of jobs; 1: per-job launches
    cudaEvent_t fork = nullptr;       // per-job launches: the slice may start
    std::string err;
};

static int bfail(teuk_batch *b, int code, const std::string &msg)
{
    if (b) b->err = msg;
    return code;
}

#define BCU(call)                                                                                \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return bfail(b, TEUK_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)


static void drop_graph(teuk_batch *b)
{
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
}

extern "C" int teuk_batch_create(void *cuda_stream, teuk_batch **out)
{
    if (!out) return TEUK_ERR_BAD_ARG;
    *out = nullptr;
    teuk_batch *b = new (std::nothrow) teuk_batch();
    if (!b) return TEUK_ERR_OOM;
    if (cudaGetDevice(&b->device) != cudaSuccess) { delete b; return TEUK_ERR_CUDA; }
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) { delete b; return TEUK_ERR_CUDA; }
        b->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
        if (b->own_stream) cudaStreamDestroy(b->stream);
        delete b;
        return TEUK_ERR_CUDA;
    }
    *out = b;
    return TEUK_OK;
}

extern "C" int teuk_batch_destroy(teuk_batch *b)
{
    if (!b) return TEUK_ERR_BAD_ARG;
    cudaStreamSynchronize(b->stream);
    for (auto &j : b->jobs)
        if (j.member) j.h->in_batch = 0;  // the handles are driven by their owner again
    drop_graph(b);
    for (auto &j : b->jobs)
        if (j.done) cudaEventDestroy(j.done);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->d_jobs) cudaFree(b->d_jobs);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return TEUK_OK;
}

extern "C" int teuk_batch_add(teuk_batch *b, teuk_handle *h, long steps, int *job_id)
{
    if (!b || !h || steps < 0 || !job_id) return bfail(b, TEUK_ERR_BAD_ARG, "teuk_batch_add: bad argument");
    *job_id = -1;
    if (h->device != b->device) return bfail(b, TEUK_ERR_BAD_ARG, "teuk_batch_add: handle on another device");
    if (h->nth > kTileMaxThreads) return bfail(b, TEUK_ERR_BAD_ARG, "teuk_batch_add: batched tiles need nth <= 512");
    for (const auto &j : b->jobs)
        if (j.member && j.h == h) return bfail(b, TEUK_ERR_BAD_ARG, "teuk_batch_add: handle already in the batch");
    if (h->in_batch) return bfail(b, TEUK_ERR_STATE, "teuk_batch_add: handle belongs to another batch");
    BCU(cudaStreamSynchronize(h->stream));  // the handle's own queued work comes first
    if (!h->phiH) {
        const size_t Nm = (size_t)(h->nr - 1) * h->nth;
        if (cudaMalloc(&h->phiH, 2 * Nm * sizeof(double2)) != cudaSuccess) {
            cudaGetLastError();
            return bfail(b, TEUK_ERR_OOM, "teuk_batch_add: out of device memory for the half step");
        }
        h->piH = h->phiH + Nm;
    }
    teuk_batch::Job j;
    j.h = h;
    j.remaining = steps;
    j.member = true;
    b->jobs.push_back(j);
    h->in_batch = 1;
    *job_id = (int)b->jobs.size() - 1;
    b->layout_dirty = true;
    return TEUK_OK;
}

extern "C" int teuk_batch_remove(teuk_batch *b, int job_id)
{
    if (!b || job_id < 0 || job_id >= (int)b->jobs.size() || !b->jobs[job_id].member)
        return bfail(b, TEUK_ERR_BAD_ARG, "teuk_batch_remove: unknown job");
    BCU(cudaStreamSynchronize(b->stream));
    b->jobs[job_id].member = false;
    b->jobs[job_id].remaining = 0;
    b->jobs[job_id].h->in_batch = 0;
    b->layout_dirty = true;
    return TEUK_OK;
}

extern "C" int teuk_batch_remaining(const teuk_batch *b, int job_id, long *remaining)
{
    if (!b || !remaining || job_id < 0 || job_id >= (int)b->jobs.size()) return TEUK_ERR_BAD_ARG;
    *remaining = b->jobs[job_id].member ? (long)b->jobs[job_id].remaining : 0;
    return TEUK_OK;
}

extern "C" int teuk_batch_sync(teuk_batch *b)
{
    if (!b) return TEUK_ERR_BAD_ARG;
    BCU(cudaStreamSynchronize(b->stream));
    return TEUK_OK;
}

// CTA threads of a job's multi-job launch: the requested size (fixed-point
// jobs at most kFxTileThreads, the bound their kernels are compiled for) or
// the split kernels' default, 128 for fixed-point and 256 for FP64 jobs.
static int job_block(const teuk_batch *b, const teuk_handle *h)
{
    const int fx = h->sp.fixed_point;
    const int want = b->block_request ? b->block_request : (fx ? kFxTileThreads : 2 * kFxTileThreads);
    return fx ? std::min(want, kFxTileThreads) : want;
}

// Rebuild the job table and the launch groups for the jobs with steps left.
static int rebuild(teuk_batch *b)
{
    b->active.clear();
    b->groups.clear();
    for (int id = 0; id < (int)b->jobs.size(); ++id)
        if (b->jobs[id].member && b->jobs[id].remaining > 0) b->active.push_back(id);
    drop_graph(b);
    const int nj = (int)b->active.size();
    if (nj == 0) {
        b->layout_dirty = false;
        return TEUK_OK;
    }
    if (nj > b->cap_jobs) {
        BCU(cudaStreamSynchronize(b->stream));  // queued slices still read the old table
        if (b->d_jobs) { cudaFree(b->d_jobs); b->d_jobs = nullptr; }
        const int cap = std::max(nj, 2 * b->cap_jobs);
        if (cudaMalloc(&b->d_jobs, (size_t)cap * sizeof(JobDesc)) != cudaSuccess) {
            cudaGetLastError();
            b->cap_jobs = 0;
            return bfail(b, TEUK_ERR_OOM, "batch: out of device memory for the job table");
        }
        b->cap_jobs = cap;
    }
    b->host_desc.assign(nj, JobDesc{});
    int sms = 0;
    BCU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    for (int q = 0; q < nj; ++q) {
        teuk_handle *h = b->jobs[b->active[q]].h;
        JobDesc &d = b->host_desc[q];
        d.p = h->sp;
        d.phi[0] = h->phi[0]; d.phi[1] = h->phi[1];
        d.pi[0] = h->pi[0]; d.pi[1] = h->pi[1];
        d.phiH = h->phiH; d.piH = h->piH;
        d.cur = h->cur;
        const int block = job_block(b, h);
        d.tw = multi_tile_width(h->nth, block);
        d.rows = block / d.tw;
        d.tiles = (h->nth + d.tw - 1) / d.tw;
        // the job's group: same arithmetic and CTA size, room for one more job
        teuk_batch::Group *g = nullptr;
        for (auto &c : b->groups)
            if (c.real == h->sp.real_coef && c.fx == h->sp.fixed_point && c.ko == h->sp.ko && c.block == block &&
                (int)c.members.size() < kMultiMaxJobs)
                g = &c;
        if (!g) {
            b->groups.emplace_back();
            g = &b->groups.back();
            g->real = h->sp.real_coef;
            g->fx = h->sp.fixed_point;
            g->ko = h->sp.ko;
            g->block = block;
            g->pred.njobs = g->corr.njobs = 0;
            g->pred.off[0] = g->corr.off[0] = 0;
        }
        g->smem = std::max(g->smem, multi_smem_bytes(d.tw, block, h->sp.ko));
        const int slot = (int)g->members.size();
        g->members.push_back(q);
        for (int w = 0; w < 2; ++w) {
            MultiArgs &a = w ? g->corr : g->pred;
            const int rows = w ? h->nr - 2 : h->nr - 1;
            a.jobs[slot] = d;
            a.off[slot + 1] = a.off[slot] + (rows + d.rows - 1) / d.rows * d.tiles;
            a.njobs = slot + 1;
            a.ntiles = a.off[slot + 1];
        }
    }
    for (auto &g : b->groups) {
        g.ctas = 0;
        g.pred.sbuf_words = g.corr.sbuf_words = (int)(g.smem / sizeof(double2));
        BCU(multi_allow_smem(g.real, g.fx, g.ko, g.smem));
        if (b->ctas_request > 0) {  // persistent: as many CTAs as stay resident, at most the request per SM
            int per_sm = b->ctas_request;
            for (int w = 0; w < 2; ++w) {
                int n = 0;
                BCU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, multi_kernel_ptr(w, g.real, g.fx, g.ko),
                                                                  g.block, 2 * g.smem));
                per_sm = std::min(per_sm, std::max(1, n));
            }
            g.ctas = sms * per_sm;
        }
    }
    BCU(cudaMemcpyAsync(b->d_jobs, b->host_desc.data(), nj * sizeof(JobDesc), cudaMemcpyHostToDevice, b->stream));
    b->layout_dirty = false;
    return TEUK_OK;
}

// After an odd number of steps the jobs' current buffers flipped: the launch
// groups (baked into a captured graph) are refreshed and the graph dropped.
static int refresh_cur(teuk_batch *b)
{
    for (int q = 0; q < (int)b->active.size(); ++q) b->host_desc[q].cur = b->jobs[b->active[q]].h->cur;
    for (auto &g : b->groups)
        for (int slot = 0; slot < (int)g.members.size(); ++slot)
            g.pred.jobs[slot].cur = g.corr.jobs[slot].cur = b->host_desc[g.members[slot]].cur;
    drop_graph(b);
    return TEUK_OK;
}

// The first predictor of every call follows the table upload or the counter
// update, not a step kernel, so it is launched in plain stream order; the
// other step kernels use programmatic dependent launch when enabled.
static cudaError_t launch_batch_steps(teuk_batch *b, int k0, int n, cudaStream_t st)
{
    for (int k = k0; k < k0 + n; ++k) {
        for (int w = 0; w < 2; ++w)
            for (size_t gi = 0; gi < b->groups.size(); ++gi) {
                const auto &g = b->groups[gi];
                const bool pdl = b->pdl != 0 && !(k == k0 && w == 0 && gi == 0);
                const cudaError_t e = launch_step_multi(w ? g.corr : g.pred, w, g.real, g.fx, g.ko, g.block, g.smem,
                                                        g.ctas, k, st, pdl);
                if (e != cudaSuccess) return e;
            }
    }
    return launch_advance_batch(b->d_jobs, (int)b->active.size(), n, st);
}

static int capture(teuk_batch *b)
{
    cudaGraph_t g = nullptr;
    BCU(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = launch_batch_steps(b, 0, b->chunk, b->cap);
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(b, TEUK_ERR_CUDA, std::string("batch graph capture: ") + cudaGetErrorString(e ? e : e2));
    }
    cudaError_t e3 = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) return bfail(b, TEUK_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e3));
    return TEUK_OK;
}

// Per-job launches: every job advances min(L, its remaining steps) on its
// own stream with its own kernels (graph replay per chunk), the jobs running
// concurrently; the batch stream first releases and then waits for all of
// them.  Returns the largest advance.
static int per_job_slice(teuk_batch *b, long long L, long long *advanced)
{
    if (!b->fork) BCU(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    BCU(cudaEventRecord(b->fork, b->stream));
    long long most = 0;
    for (int id : b->active) {
        auto &j = b->jobs[id];
        const long long n = std::min(L, j.remaining);
        if (!j.done) BCU(cudaEventCreateWithFlags(&j.done, cudaEventDisableTiming));
        BCU(cudaStreamWaitEvent(j.h->stream, b->fork, 0));
        const int rc = teuk_step_handle(j.h, (long)n);
        if (rc) return bfail(b, rc, "batch: " + j.h->err);
        BCU(cudaEventRecord(j.done, j.h->stream));
        BCU(cudaStreamWaitEvent(b->stream, j.done, 0));
        j.remaining -= n;
        if (j.remaining == 0 || (n & 1)) b->layout_dirty = true;  // leaves, or the table's buffer parity is stale
        most = std::max(most, n);
    }
    *advanced = most;
    return TEUK_OK;
}

// One slice of L steps for the active jobs in the current mode (per-job
// launches: each job advances up to L steps).
static int run_slice(teuk_batch *b, long long L)
{
    if (b->mode == 1) {
        long long adv = 0;
        return per_job_slice(b, L, &adv);
    } else {
        if (L == b->chunk) {
            if (!b->graph) {
                int rc = capture(b);
                if (rc) return rc;
            }
            BCU(cudaGraphLaunch(b->graph, b->stream));
        } else {
            BCU(launch_batch_steps(b, 0, (int)L, b->stream));
        }
        for (int id : b->active) {
            b->jobs[id].h->nstep += L;
            b->jobs[id].h->cur ^= (int)(L & 1);
        }
    }
    bool finished = false;
    for (int id : b->active) {
        b->jobs[id].remaining -= L;
        finished |= b->jobs[id].remaining == 0;
    }
    if (finished) {
        b->layout_dirty = true;  // finished jobs leave at this slice boundary
    } else if (b->mode == 0 && (L & 1)) {
        int rc = refresh_cur(b);
        if (rc) return rc;
    }
    return TEUK_OK;
}

extern "C" int teuk_batch_step(teuk_batch *b, long max_steps, long *steps_done)
{
    if (!b || max_steps < 0) return bfail(b, TEUK_ERR_BAD_ARG, "teuk_batch_step: bad argument");
    long done = 0;
    while (done < max_steps) {
        if (b->layout_dirty) {
            int rc = rebuild(b);
            if (rc) return rc;
        }
        if (b->active.empty()) break;
        if (b->mode == 1) {  // jobs advance independently: no common slices
            long long adv = 0;
            int rc = per_job_slice(b, max_steps - done, &adv);
            if (rc) return rc;
            done += (long)adv;
            break;
        }
        long long L = std::min<long long>(b->chunk, max_steps - done);
        for (int id : b->active) L = std::min(L, b->jobs[id].remaining);
        int rc = run_slice(b, L);
        if (rc) return rc;
        done += (long)L;
    }
    if (steps_done) *steps_done = done;
    return TEUK_OK;
}

extern "C" int teuk_batch_set_option(teuk_batch *b, int option, long value)
{
    if (!b) return TEUK_ERR_BAD_ARG;
    BCU(cudaStreamSynchronize(b->stream));
    switch (option) {
    case TEUK_OPT_PDL:
        if (value != 0 && value != 1) return bfail(b, TEUK_ERR_BAD_ARG, "teuk_batch_set_option: PDL is 0 or 1");
        b->pdl = (int)value;
        break;
    case TEUK_OPT_GRAPH_CHUNK:
        if (value < 2 || value > 4096 || value % 2)
            return bfail(b, TEUK_ERR_BAD_ARG, "teuk_batch_set_option: graph chunk must be even, 2..4096");
        b->chunk = (int)value;
        break;
    case TEUK_OPT_BATCH_MODE:
        if (value != 0 && value != 1) return bfail(b, TEUK_ERR_BAD_ARG, "teuk_batch_set_option: batch mode is 0 or 1");
        BCU(cudaStreamSynchronize(b->stream));
        b->mode = (int)value;
        b->layout_dirty = true;
        break;
    case TEUK_OPT_BLOCK_THREADS:
        if (value != 0 && (value < 32 || value > kTileMaxThreads || value % 32))
            return bfail(b, TEUK_ERR_BAD_ARG, "teuk_batch_set_option: block threads 0 or a multiple of 32 <= 512");
        b->block_request = (int)value;
        b->layout_dirty = true;
        break;
    case TEUK_OPT_BATCH_CTAS:
        if (value < 0 || value > 64)
            return bfail(b, TEUK_ERR_BAD_ARG, "teuk_batch_set_option: CTAs per SM is 0 (one per tile) to 64");
        b->ctas_request = (int)value;
        b->layout_dirty = true;
        break;
    default:
        return bfail(b, TEUK_ERR_BAD_ARG, "teuk_batch_set_option: unknown option");
    }
    drop_graph(b);
    return TEUK_OK;
}

extern "C" int teuk_batch_autotune(teuk_batch *b, int *best)
{
    if (!b) return TEUK_ERR_BAD_ARG;
    if (b->layout_dirty) {
        int rc = rebuild(b);
        if (rc) return rc;
    }
    if (b->active.empty()) return bfail(b, TEUK_ERR_STATE, "teuk_batch_autotune: no job has steps left");
    // per-job launches, multi-job launches with one CTA per tile in two tile
    // shapes (the default CTA size, and 64-thread CTAs: tiles of at most 64
    // columns, fewer rows), and the persistent multi-job launch (resident
    // CTAs); each candidate gets an equal share of the steps the shortest job
    // has left
    const int cands[][3] = {{1, 0, 0}, {0, 0, 0}, {0, 0, 64}, {0, 64, 0}};  // {mode, CTAs per SM, CTA threads}
    const int ncand = (int)(sizeof(cands) / sizeof(cands[0]));
    long long share = 1LL << 62;
    for (int id : b->active) share = std::min(share, b->jobs[id].remaining / ncand);
    cudaEvent_t e0, e1;
    BCU(cudaEventCreate(&e0));
    BCU(cudaEventCreate(&e1));
    int best_c = b->mode == 1 ? 0 : (b->ctas_request ? 3 : (b->block_request == 64 ? 2 : 1));
    double best_rate = -1.0;
    for (int ci = 0; ci < ncand; ++ci) {
        const auto &c = cands[ci];
        if (b->layout_dirty) {
            int rc = rebuild(b);
            if (rc) return rc;
        }
        long long pts = 0, minrem = 1LL << 62;
        for (int id : b->active) minrem = std::min(minrem, b->jobs[id].remaining);
        const long long budget = std::min(share, minrem) & ~1LL;
        if (b->active.empty() || budget < 8) break;
        b->mode = c[0];
        if (c[0] == 0) {
            b->ctas_request = c[1];
            b->block_request = c[2];
        }
        b->layout_dirty = true;
        int rc = rebuild(b);
        if (rc) return rc;
        for (int id : b->active) pts += (long long)(b->jobs[id].h->nr - 2) * b->jobs[id].h->nth;
        // warm-up of up to one chunk (captures the graphs it replays), then
        // the timed steps; both count as progress
        const long long warm = std::min<long long>(b->chunk, budget / 2) & ~1LL;
        const long long n = std::min<long long>(2 * b->chunk, budget - warm) & ~1LL;
        rc = run_slice(b, warm);
        if (rc) return rc;
        BCU(cudaEventRecord(e0, b->stream));
        for (long long left = n; left > 0;) {  // whole chunks replay the captured graphs
            const long long L = std::min<long long>(left, b->chunk);
            rc = run_slice(b, L);
            if (rc) return rc;
            left -= L;
        }
        BCU(cudaEventRecord(e1, b->stream));
        BCU(cudaEventSynchronize(e1));
        float ms = 0;
        BCU(cudaEventElapsedTime(&ms, e0, e1));
        const double rate = (double)pts * (double)n / (ms > 0 ? ms : 1e-3);
        if (rate > best_rate) {
            best_rate = rate;
            best_c = ci;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->mode = cands[best_c][0];
    if (b->mode == 0) {
        b->ctas_request = cands[best_c][1];
        b->block_request = cands[best_c][2];
    }
    b->layout_dirty = true;
    if (best) *best = best_c;
    return TEUK_OK;
}

extern "C" long teuk_batch_launches_for(const teuk_batch *b, long n)
{
    if (!b || n < 0) return -1;
    if (b->mode == 1) {  // every job launches its own kernels
        long total = 0;
        for (const auto &j : b->jobs)
            if (j.member && j.remaining > 0) total += teuk_launches_for(j.h, n);
        return total;
    }
    // per step one predictor and one corrector launch per group; each slice
    // adds one counter update.  Groups as the next rebuild forms them.
    long groups = 0;
    if (!b->layout_dirty) {
        groups = (long)b->groups.size();
    } else {
        struct Key { int real, fx, ko, block; long n; };
        std::vector<Key> keys;
        for (const auto &j : b->jobs) {
            if (!j.member || j.remaining <= 0) continue;
            const int block = job_block(b, j.h);
            bool found = false;
            for (auto &k : keys)
                if (k.real == j.h->sp.real_coef && k.fx == j.h->sp.fixed_point && k.ko == j.h->sp.ko &&
                    k.block == block) { ++k.n; found = true; }
            if (!found) keys.push_back(Key{j.h->sp.real_coef, j.h->sp.fixed_point, j.h->sp.ko, block, 1});
        }
        for (const auto &k : keys) groups += (k.n + kMultiMaxJobs - 1) / kMultiMaxJobs;
    }
    const long slices = (n + b->chunk - 1) / b->chunk;
    return 2 * n * groups + slices;
}

extern "C" const char *teuk_batch_last_error(const teuk_batch *b) { return b ? b->err.c_str() : ""; }
