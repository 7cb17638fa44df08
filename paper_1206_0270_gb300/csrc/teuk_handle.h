// teuk_handle.h -- host-side state of one solver handle (libteuk internal).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "teuk_internal.h"

struct teuk_handle {
    int nr = 0, nth = 0, s = 0, m = 0, parity = 1;
    double a = 0, rstar_min = 0, rstar_max = 0, h = 0, dth = 0, dt = 0;
    double eps = 0;  // strength of the angular Kreiss-Oliger dissipation (0: none)
    int device = 0, num_sms = 0;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    bool own_stream = false;

    char *arena = nullptr;         // state, planes, tables, counters
    double2 *phi[2] = {nullptr, nullptr}, *pi[2] = {nullptr, nullptr};
    double2 *phiH = nullptr, *piH = nullptr;  // half-step buffer of the two-kernel variant
    double *b_node = nullptr;
    long long *d_step = nullptr;
    unsigned long long *d_count = nullptr;
    teuk::StepParams sp{};
    teuk::SetupParams su{};  // kept to rebuild the coefficient planes

    double *d_src = nullptr;       // source windows (gP then gC)
    double2 *d_ring = nullptr;
    long long drained = 0;

    int cur = 0;
    long long nstep = 0;
    int variant = 0;
    int rows_per_block = 1, nblocks = 1;
    int pdl = 1;      // programmatic dependent launch of the split kernels
    int in_batch = 0; // batches this handle belongs to (0 or 1): it is driven by the batch
    int split_rows = 0;  // r* rows per CTA tile of the split kernels (0 = automatic)
    int chunk = 64;   // time steps per captured graph (even)
    cudaGraphExec_t graph[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
    std::string err;
};

// n steps on the handle's own stream, without the batch-membership check
// (teuk_step checks, then calls this; batches call it for their jobs).
int teuk_step_handle(teuk_handle *h, long n);

