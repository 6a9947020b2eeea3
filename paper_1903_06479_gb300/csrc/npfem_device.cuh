// Device utilities shared by the solver and learning kernels: compensated sums,
// the per-cell shared scalars, block reductions, buffer placement lookup.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "npfem_internal.h"

namespace npfem {

constexpr unsigned kFull = 0xffffffffu;

template <typename T>
struct Unit;
template <>
struct Unit<float> {
    static constexpr double u = 5.9604644775390625e-08;
    static constexpr float sl2_rel = 2.0e-7f;
    static constexpr float tiny = 1.0e-37f;
};
template <>
struct Unit<double> {
    static constexpr double u = 1.1102230246251565e-16;
    static constexpr double sl2_rel = 4.0e-16;
    static constexpr double tiny = 1.0e-300;
};

// Compensated sum (hi + lo) built from error-free two-sums.
template <typename T>
struct Acc {
    T hi, lo;
    __device__ __forceinline__ Acc() : hi(T(0)), lo(T(0)) {}
    __device__ __forceinline__ void add(T x)
    {
        const T s = hi + x;
        const T bb = s - hi;
        lo += (hi - (s - bb)) + (x - bb);
        hi = s;
    }
    __device__ __forceinline__ void merge(T h2, T l2)
    {
        add(h2);
        lo += l2;
    }
};

// Per-cell scalars shared by the block (after the 8 KB of reduction partials).
struct CellShared {
    double out[16];          // results of the last block_reduce
    double V, Vn, E, Ein, Earea, Esk, Ebend, Evol, res, noise;
    double rho[kMaxHistory];
    double alpha[kMaxHistory];
    double post[12];         // centre of mass, its velocity, angular velocity
    float postf[12];         // FP32 copies of post[] and of the warm start's frame (R, y_cm)
    double volc;
    float volcf;
    long long item;          // work item handed to the block
    unsigned long long mbar; // tensor-core path: MMA completion barrier
    unsigned need[16];       // tensor-core path: request flags of the cluster's blocks
    unsigned taddr;          // tensor-core path: tensor-memory base address
    int bad;
    int accept;
    int push;
};
static_assert(sizeof(CellShared) <= kFixedSmem - 8192, "CellShared does not fit");

// A block-wide scalar for the solver's type: the FP64 value for the FP64 path, its
// FP32 copy (written once by thread 0) otherwise, so that the FP32 path's threads
// do no FP64 conversion.
template <typename T>
__device__ __forceinline__ T bcast(double d, float f)
{
    if constexpr (sizeof(T) == 8) return d;
    else return f;
}

__device__ __forceinline__ CellShared* cell_shared(unsigned char* smem)
{
    return reinterpret_cast<CellShared*>(smem + 8192);
}

// Sums K compensated accumulators over the block.  Thread 0 writes the totals to
// sh->out[] and then runs epi(sh) before the closing barrier, so every thread sees
// the totals and whatever the epilogue derived from them.
struct NoEpi {
    __device__ __forceinline__ void operator()(CellShared*) const {}
};

template <typename T, int K, typename Epi = NoEpi>
__device__ __forceinline__ void block_reduce(Acc<T> (&a)[K], unsigned char* smem, Epi epi = Epi())
{
    T* red = reinterpret_cast<T*>(smem);  // [32 warps][K][2]
    CellShared* sh = cell_shared(smem);
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T h2 = __shfl_xor_sync(kFull, a[k].hi, o);
            const T l2 = __shfl_xor_sync(kFull, a[k].lo, o);
            a[k].merge(h2, l2);
        }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            red[(w * K + k) * 2] = a[k].hi;
            red[(w * K + k) * 2 + 1] = a[k].lo;
        }
    }
    __syncthreads();
    if (w == 0) {
        Acc<T> b[K];
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (lane < nw) {
                b[k].hi = red[(lane * K + k) * 2];
                b[k].lo = red[(lane * K + k) * 2 + 1];
            }
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T h2 = __shfl_xor_sync(kFull, b[k].hi, o);
                const T l2 = __shfl_xor_sync(kFull, b[k].lo, o);
                b[k].merge(h2, l2);
            }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) sh->out[k] = (double)b[k].hi + (double)b[k].lo;
            epi(sh);
        }
    }
    __syncthreads();
}

// Like block_reduce, for KC compensated and KP plain sums (out[0..KC) compensated,
// out[KC..KC+KP) plain).
template <typename T, int KC, int KP, typename Epi = NoEpi>
__device__ __forceinline__ void block_reduce_cp(Acc<T> (&a)[KC], T (&p)[KP], unsigned char* smem, Epi epi = Epi())
{
    constexpr int W = 2 * KC + KP;
    T* red = reinterpret_cast<T*>(smem);  // [32 warps][W]
    CellShared* sh = cell_shared(smem);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            const T h2 = __shfl_xor_sync(kFull, a[k].hi, o);
            const T l2 = __shfl_xor_sync(kFull, a[k].lo, o);
            a[k].merge(h2, l2);
        }
#pragma unroll
        for (int k = 0; k < KP; ++k) p[k] += __shfl_xor_sync(kFull, p[k], o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            red[w * W + 2 * k] = a[k].hi;
            red[w * W + 2 * k + 1] = a[k].lo;
        }
#pragma unroll
        for (int k = 0; k < KP; ++k) red[w * W + 2 * KC + k] = p[k];
    }
    __syncthreads();
    if (w == 0) {
        Acc<T> b[KC];
        T q[KP];
#pragma unroll
        for (int k = 0; k < KP; ++k) q[k] = T(0);
        if (lane < nw) {
#pragma unroll
            for (int k = 0; k < KC; ++k) {
                b[k].hi = red[lane * W + 2 * k];
                b[k].lo = red[lane * W + 2 * k + 1];
            }
#pragma unroll
            for (int k = 0; k < KP; ++k) q[k] = red[lane * W + 2 * KC + k];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int k = 0; k < KC; ++k) {
                const T h2 = __shfl_xor_sync(kFull, b[k].hi, o);
                const T l2 = __shfl_xor_sync(kFull, b[k].lo, o);
                b[k].merge(h2, l2);
            }
#pragma unroll
            for (int k = 0; k < KP; ++k) q[k] += __shfl_xor_sync(kFull, q[k], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < KC; ++k) sh->out[k] = (double)b[k].hi + (double)b[k].lo;
#pragma unroll
            for (int k = 0; k < KP; ++k) sh->out[KC + k] = (double)q[k];
            epi(sh);
        }
    }
    __syncthreads();
}

// Plain (uncompensated) block sum of K values, for dot products of the direction.
template <typename T, int K, typename Epi = NoEpi>
__device__ __forceinline__ void block_sum(T (&p)[K], unsigned char* smem, Epi epi = Epi())
{
    T* red = reinterpret_cast<T*>(smem);
    CellShared* sh = cell_shared(smem);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < K; ++k) p[k] += __shfl_xor_sync(kFull, p[k], o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) red[w * K + k] = p[k];
    }
    __syncthreads();
    if (w == 0) {
        T q[K];
#pragma unroll
        for (int k = 0; k < K; ++k) q[k] = lane < nw ? red[lane * K + k] : T(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < K; ++k) q[k] += __shfl_xor_sync(kFull, q[k], o);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) sh->out[k] = (double)q[k];
            epi(sh);
        }
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ T* vec_ptr(const GroupDesc<T>& gd, unsigned char* smem, char* slot, int v)
{
    const int l = gd.loc[v];
    return l >= 0 ? reinterpret_cast<T*>(smem + kFixedSmem + l) : reinterpret_cast<T*>(slot + (-(long long)l - 1));
}

}  // namespace npfem
