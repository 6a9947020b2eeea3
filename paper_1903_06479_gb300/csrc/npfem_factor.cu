// One-time FP64 inversion of the constant Hessian approximation H~ = M~/h^2 + L
// (Sec. 2.1.1: H~ is constant and SPD, so it is factored once).  The library keeps
// the dense inverse A^-1 so that every cell sharing a topology applies it as a
// contraction.  Gauss-Jordan elimination without pivoting is stable for SPD
// matrices; the whole elimination is one cooperative launch.
#include <cuda_bf16.h>

#include "npfem_internal.h"

namespace npfem {
namespace {

// Grid-wide barrier of the cooperative inversion kernel (all blocks co-resident).
// The wait is bounded: after kGjSpinLimit polls the block records flag 2 (reported
// as a timeout by the host) and goes on, and every block stops waiting once the flag
// is set, so the kernel always ends.
constexpr unsigned kGjSpinLimit = 1u << 24;

__device__ __forceinline__ void gj_grid_barrier(unsigned* bar, unsigned& gen, int* flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = bar + 1;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicExch(bar + 1, gen + 1);
        } else {
            volatile int* vflag = flag;
            unsigned it = 0;
            while (*vgen == gen) {
                if (++it > kGjSpinLimit) {
                    atomicExch(flag, 2);
                    break;
                }
                if (*vflag == 2) break;  // another block gave up: the result is discarded anyway
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    ++gen;
    __syncthreads();
}

// In-place Gauss-Jordan inversion of an SPD matrix in one cooperative launch: one
// grid barrier per pivot.  Warps own rows (coalesced over columns).  Pivot step k
// needs row k as it stands after step k-1 while its owner overwrites it, so that row
// is read from a snapshot: the owner of row k+1 writes its updated row into
// prow[(k+1) & 1] during step k, a buffer nobody reads in step k.  Per element the
// arithmetic is the textbook one: the pivot row scaled by 1/a_kk, then
// a_ij <- a_ij - a_ik a'_kj with a'_kk = 1/a_kk and a_ik replaced by 0.
__global__ void __launch_bounds__(256) gj_invert_coop(double* A, double* prow, int n, unsigned* bar, int* flag)
{
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nw = gridDim.x * (blockDim.x >> 5);
    unsigned gen = 0;
    if (gw == 0)
        for (int j = lane; j < n; j += 32) prow[j] = __ldcg(A + j);
    gj_grid_barrier(bar, gen, flag);
    for (int k = 0; k < n; ++k) {
        const double* pk = prow + (size_t)(k & 1) * n;
        double* pn = prow + (size_t)((k + 1) & 1) * n;
        double piv = __ldcg(pk + k);
        if (!(piv > 0.0)) {
            if (gw == 0 && lane == 0) atomicCAS(flag, 0, 1);
            piv = 1.0;  // keep going; the host discards the result
        }
        const double p = 1.0 / piv;
        for (int i = gw; i < n; i += nw) {
            double* Ai = A + (size_t)i * n;
            if (i == k) {
                for (int j = lane; j < n; j += 32) Ai[j] = (j == k ? 1.0 : __ldcg(pk + j)) * p;
                continue;
            }
            const double f = __ldcg(Ai + k);
            __syncwarp();
            for (int j = lane; j < n; j += 32) {
                const double a = j == k ? 0.0 : __ldcg(Ai + j);
                const double v = a - f * ((j == k ? 1.0 : __ldcg(pk + j)) * p);
                Ai[j] = v;
                if (i == k + 1) pn[j] = v;
            }
        }
        gj_grid_barrier(bar, gen, flag);
    }
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

// Element (row i, column k) of A^-1 at its place in the TF32 chunks: chunk (tile, c) of
// 128 rows x 32 K holds 16 x 8 core matrices of 8 rows x 4 elements (128 bytes), K-adjacent
// core matrices 128 bytes apart, row groups 1024 bytes apart.
__global__ void publish_tf32_tiled(const double* A, int n, int tiles, int kpad, float* out)
{
    const int nch = kpad / 32;
    const size_t total = (size_t)tiles * 128 * kpad;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(q / kpad), k = (int)(q % kpad);
        const int t = i >> 7, r = i & 127, c = k >> 5, kk = k & 31;
        double v = (i < n && k < n) ? A[(size_t)i * n + k] : 0.0;
        float f = (float)v;
        unsigned u;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(f));
        const size_t chunk = (size_t)t * nch + c;
        const size_t off = chunk * (128 * 32) + (size_t)(((r >> 3) * 8 + (kk >> 2)) * 32 + (r & 7) * 4 + (kk & 3));
        out[off] = __uint_as_float(u);
    }
}

}  // namespace

cudaError_t publish_inverse_tf32_tiled(const double* A, int n, int tiles, int kpad, float* out, cudaStream_t s)
{
    publish_tf32_tiled<<<1024, 256, 0, s>>>(A, n, tiles, kpad, out);
    count_launch();
    return cudaGetLastError();
}

__global__ void publish_bf16_square(const double* A, int n, int n8, __nv_bfloat16* out)
{
    size_t total = (size_t)n8 * n8;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(q / n8), j = (int)(q % n8);
        out[q] = __double2bfloat16((i < n && j < n) ? A[(size_t)i * n + j] : 0.0);
    }
}

cudaError_t publish_inverse_bf16_square(const double* A, int n, int n8, void* out, cudaStream_t s)
{
    publish_bf16_square<<<1024, 256, 0, s>>>(A, n, n8, static_cast<__nv_bfloat16*>(out));
    count_launch();
    return cudaGetLastError();
}

cudaError_t publish_inverse_bf16_blocked(const double* A, int n, int rows_pad, int kpad, void* out, cudaStream_t s)
{
    publish_bf16_blocked<<<1024, 256, 0, s>>>(A, n, rows_pad, kpad, (__nv_bfloat16*)out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t invert_spd_fp64(double* A, int n, double* prow, int* d_flag, cudaStream_t s)
{
    int dev = 0, coop = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gj_invert_coop, 256, 0);
    if (e != cudaSuccess) return e;
    if (!coop || per_sm < 1) return cudaErrorNotSupported;
    // one block per SM: every block is resident, so the grid barrier cannot wait on an
    // unscheduled block; the barrier words sit behind the flag (d_flag[2], d_flag[3])
    const int grid = sms;
    unsigned* bar = reinterpret_cast<unsigned*>(d_flag + 2);
    void* args[] = {&A, &prow, &n, &bar, &d_flag};
    e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaLaunchCooperativeKernel((const void*)gj_invert_coop, dim3(grid), dim3(256), args, 0, s);
    if (e != cudaSuccess) return e;
    count_launch();
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
