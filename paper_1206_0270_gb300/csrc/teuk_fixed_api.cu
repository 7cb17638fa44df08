// teuk_fixed_api.cu -- teuk_fixed_dot and teuk_fixed_d6: the fixed-point sums
// of the Pi rows and the exact sixth difference of the angular dissipation
// (teuk_fixed.h) on the host or on the device, for verification.
#include "teuk.h"
#include "teuk_fixed.h"

#include <cuda_runtime.h>
#include <vector>

using namespace teuk;

namespace {

template <int N>
__host__ __device__ void dot_case(const double *c, const double *x, const unsigned *flip, double *out, int *ok)
{
    Fx C[N], X[N];
    uint32_t F[N];
    for (int k = 0; k < N; ++k) {
        // coefficients as the kernels split them (normal or zero; others as fields)
        const uint64_t cb = fx_bits(c[k]) & 0x7FFFFFFFFFFFFFFFull;
        const bool normal_or_zero = cb == 0 || (cb >= 0x0010000000000000ull && cb < 0x7FF0000000000000ull);
        C[k] = normal_or_zero ? fx_unpack_coef(c[k]) : fx_unpack(c[k]);
        X[k] = fx_unpack(x[k]);
        F[k] = flip[k] & 1u;
    }
    *ok = fx_dot<N>(C, X, F, out) ? 1 : 0;
}

__host__ __device__ void dot_any(int n, const double *c, const double *x, const unsigned *flip, double *out, int *ok)
{
    switch (n) {
#define TEUK_FX_CASE(N) \
    case N: dot_case<N>(c, x, flip, out, ok); break;
        TEUK_FX_CASE(1) TEUK_FX_CASE(2) TEUK_FX_CASE(3) TEUK_FX_CASE(4) TEUK_FX_CASE(5) TEUK_FX_CASE(6)
        TEUK_FX_CASE(7) TEUK_FX_CASE(8) TEUK_FX_CASE(9) TEUK_FX_CASE(10) TEUK_FX_CASE(11) TEUK_FX_CASE(12)
        TEUK_FX_CASE(13) TEUK_FX_CASE(14) TEUK_FX_CASE(15) TEUK_FX_CASE(16)
#undef TEUK_FX_CASE
    default: *ok = 0;
    }
}

__global__ void fixed_dot_kernel(int n, long count, const double *c, const double *x, const unsigned *flip,
                                 double *out, int *ok)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    dot_any(n, c + i * n, x + i * n, flip + i * n, out + i, ok + i);
}

__global__ void fixed_d6_kernel(long count, const double *u, double *out)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    out[i] = fx_d6_values(u + i * 7, 1);
}

}  // namespace

extern "C" int teuk_fixed_d6(int on_device, long count, const double *u, double *out)
{
    if (count < 0 || (count > 0 && (!u || !out))) return TEUK_ERR_BAD_ARG;
    if (count == 0) return TEUK_OK;
    if (!on_device) {
        for (long i = 0; i < count; ++i) out[i] = fx_d6_values(u + i * 7, 1);
        return TEUK_OK;
    }
    double *du = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc(&du, (size_t)count * 7 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dout, (size_t)count * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(du, u, (size_t)count * 7 * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const int threads = 128;
        fixed_d6_kernel<<<(unsigned)((count + threads - 1) / threads), threads>>>(count, du, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, (size_t)count * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(du);
    cudaFree(dout);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? TEUK_ERR_OOM : TEUK_ERR_CUDA;
    }
    return TEUK_OK;
}

extern "C" int teuk_fixed_dot(int on_device, int nterms, long count, const double *c, const double *x,
                              const unsigned *flip, double *out, int *ok)
{
    if (nterms < 1 || nterms > 16 || count < 0 || (count > 0 && (!c || !x || !flip || !out || !ok)))
        return TEUK_ERR_BAD_ARG;
    if (count == 0) return TEUK_OK;
    if (!on_device) {
        for (long i = 0; i < count; ++i)
            dot_any(nterms, c + i * nterms, x + i * nterms, flip + i * nterms, out + i, ok + i);
        return TEUK_OK;
    }
    const size_t nin = (size_t)count * nterms;
    double *dc = nullptr, *dx = nullptr, *dout = nullptr;
    unsigned *dflip = nullptr;
    int *dok = nullptr;
    cudaError_t e = cudaMalloc(&dc, nin * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dx, nin * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dflip, nin * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&dout, (size_t)count * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dok, (size_t)count * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(dc, c, nin * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dx, x, nin * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dflip, flip, nin * sizeof(unsigned), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const int threads = 128;
        fixed_dot_kernel<<<(unsigned)((count + threads - 1) / threads), threads>>>(nterms, count, dc, dx, dflip, dout,
                                                                                  dok);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, (size_t)count * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(ok, dok, (size_t)count * sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dx);
    cudaFree(dflip);
    cudaFree(dout);
    cudaFree(dok);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? TEUK_ERR_OOM : TEUK_ERR_CUDA;
    }
    return TEUK_OK;
}
