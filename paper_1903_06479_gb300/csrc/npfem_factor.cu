// One-time FP64 inversion of the constant Hessian approximation H~ = M~/h^2 + L
// (Sec. 2.1.1: H~ is constant and SPD, so it is factored once).  The library keeps
// the dense inverse A^-1 so that every cell sharing a topology applies it as a
// contraction.  Gauss-Jordan elimination without pivoting is stable for SPD
// matrices; each pivot step is two launches (pivot row, rank-1 update).
#include <cuda_bf16.h>

#include "npfem_internal.h"

namespace npfem {
namespace {

// Scales pivot row k and saves column k (before the update) in col[].
__global__ void gj_pivot_row(double* A, double* col, int n, int k, int* not_spd)
{
    double piv = A[(size_t)k * n + k];
    if (!(piv > 0.0)) {
        if (threadIdx.x == 0 && blockIdx.x == 0) *not_spd = 1;
        piv = 1.0;  // keep going; the result is discarded by the host
    }
    double p = 1.0 / piv;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        col[i] = (i == k) ? 0.0 : A[(size_t)i * n + k];
    }
    // every block must have read column k before row k changes: single-block launch
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double a = (j == k) ? 1.0 : A[(size_t)k * n + j];
        A[(size_t)k * n + j] = a * p;
    }
}

// A[i][j] <- (j == k ? 0 : A[i][j]) - col[i] * A[k][j] for every row i != k.
__global__ void gj_update(double* A, const double* col, int n, int k)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (j >= n || i == k) return;
    double f = col[i];
    double a = (j == k) ? 0.0 : A[(size_t)i * n + j];
    A[(size_t)i * n + j] = a - f * A[(size_t)k * n + j];
}

// A <- (A + A^T)/2 in place; each (i < j) pair is owned by one thread.
__global__ void symmetrise_inplace(double* A, int n)
{
    size_t total = (size_t)n * n;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(q / n), j = (int)(q % n);
        if (i < j) {
            double v = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
            A[(size_t)i * n + j] = v;
            A[(size_t)j * n + i] = v;
        }
    }
}

__global__ void symmetrise_publish(const double* A, int n, int n_pad, float* o32, double* o64, __nv_bfloat16* obf,
                                   float* otf)
{
    size_t total = (size_t)n_pad * n_pad;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(q / n_pad), j = (int)(q % n_pad);
        double v = 0.0;
        if (i < n && j < n) v = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
        if (o32) o32[q] = (float)v;
        if (o64) o64[q] = v;
        if (obf) obf[q] = __double2bfloat16(v);
        if (otf) {
            // round to the 10-bit TF32 mantissa (round to nearest, ties away)
            float f = (float)v;
            unsigned u = __float_as_uint(f);
            u = (u + 0x1000u) & 0xffffe000u;
            otf[q] = __uint_as_float(u);
        }
    }
}

__global__ void publish_bf16_blocked(const double* A, int n, int rows_pad, int kpad, __nv_bfloat16* out)
{
    size_t total = (size_t)rows_pad * kpad;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(q / kpad), j = (int)(q % kpad);
        double v = (i < n && j < n) ? A[(size_t)i * n + j] : 0.0;
        out[q] = __double2bfloat16(v);
    }
}

}  // namespace

cudaError_t publish_inverse_bf16_blocked(const double* A, int n, int rows_pad, int kpad, void* out, cudaStream_t s)
{
    publish_bf16_blocked<<<1024, 256, 0, s>>>(A, n, rows_pad, kpad, (__nv_bfloat16*)out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t invert_spd_fp64(double* A, int n, double* col, int* d_flag, cudaStream_t s)
{
    dim3 ub(256), ug((n + 255) / 256, n);
    for (int k = 0; k < n; ++k) {
        gj_pivot_row<<<1, 512, 0, s>>>(A, col, n, k, d_flag);
        gj_update<<<ug, ub, 0, s>>>(A, col, n, k);
        count_launch(2);
    }
    return cudaGetLastError();
}

cudaError_t publish_inverse(const double* A, int n, int n_pad, float* o32, double* o64, void* obf, float* otf,
                            cudaStream_t s)
{
    symmetrise_inplace<<<1024, 256, 0, s>>>(const_cast<double*>(A), n);
    count_launch();
    symmetrise_publish<<<1024, 256, 0, s>>>(A, n, n_pad, o32, o64, (__nv_bfloat16*)obf, otf);
    count_launch();
    return cudaGetLastError();
}

}  // namespace npfem
