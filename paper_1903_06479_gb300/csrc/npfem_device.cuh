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

// A value carried as the unevaluated sum hi + lo of two T (float-float on the FP32
// path): energies and volumes whose differences the solver takes.
template <typename T>
struct Pair {
    T hi, lo;
};

template <typename T>
__device__ __forceinline__ Pair<T> pair_add(Pair<T> a, Pair<T> b)
{
    const T s = a.hi + b.hi;
    const T bb = s - a.hi;
    const T e = (a.hi - (s - bb)) + (b.hi - bb) + a.lo + b.lo;
    const T h = s + e;
    return {h, e - (h - s)};
}

template <typename T>
__device__ __forceinline__ Pair<T> pair_add(Pair<T> a, T b)
{
    return pair_add(a, Pair<T>{b, T(0)});
}

// (hi + lo) / 6 keeping the pair's precision: the remainder of hi / 6 is exact.
template <typename T>
__device__ __forceinline__ Pair<T> pair_div6(T hi, T lo)
{
    const T q = hi / T(6);
    return {q, (fma(-q, T(6), hi) + lo) / T(6)};
}

// a - b, accurate when a and b are close (the high parts subtract exactly).
template <typename T>
__device__ __forceinline__ T pair_diff(Pair<T> a, Pair<T> b)
{
    return (a.hi - b.hi) + (a.lo - b.lo);
}

template <typename T>
__device__ __forceinline__ double pair_f64(Pair<T> a)
{
    return (double)a.hi + (double)a.lo;
}

// Per-cell scalars shared by the block (after the 8 KB of reduction partials), in the
// solver's type: the FP32 path does no FP64 arithmetic (an FP64 operation costs tens
// of FP32 ones on this part, a division or square root hundreds).
template <typename T>
struct CellShared {
    T out[24];               // results of the last block reduction (high parts of compensated sums)
    T outlo[16];             // low parts of the compensated sums
    Pair<T> E, Ein, Earea, Esk, Ebend, V, Vn;
    T Evol, res, noise, volc;
    // L-BFGS history, by slot: rho_i = 1 / s_i^T y_i, the two-loop coefficients, the
    // inner products SY[i][j] = s_i^T y_j of the stored pairs, s_i^T g at the current
    // iterate, y_i^T r (r = H0 q of the last direction) and alpha_i - beta_i
    T rho[kMaxHistory];
    T alpha[kMaxHistory];
    T SY[kMaxHistory][kMaxHistory];
    T sg[kMaxHistory];
    T yr[kMaxHistory];
    T coef[kMaxHistory];
    T post[12];              // centre of mass, its velocity, angular velocity; warm start: R, y_cm
    T* hs[kMaxHistory];      // history vectors s and y by age (newest first), set by first_loop
    T* hy[kMaxHistory];
    T aq[kMaxHistory];       // alpha_i and alpha_i - beta_i by age
    T cq[kMaxHistory];
    long long item;          // work item handed to the block
    unsigned long long mbar; // tensor-core path: MMA completion barrier
    // tensor-core path, asynchronous rounds: results of this block's request delivered
    // (one arrival per block of the cluster), the requests pending at this block (bit d:
    // block d), the batch being served, blocks of the cluster that have finished, and a
    // broadcast word
    unsigned long long dbar;
    unsigned pend, batch, fin, flag;
    unsigned taddr;          // tensor-core path: tensor-memory base address
    // TF32 contraction (SIMT kernel): per stage of the streamed A^-1 ring, "chunk landed"
    // and "MMAs done reading it" barriers, and each stage's uses so far (phase parity)
    unsigned long long tfull[2], tfree[2];
    unsigned tuse[2];
    int tfail;               // a bounded wait gave up: later contractions are skipped
    int bad;
    int accept;
    int push;
};
static_assert(sizeof(CellShared<double>) <= kFixedSmem - 8192, "CellShared does not fit");

template <typename T>
__device__ __forceinline__ CellShared<T>* cell_shared(unsigned char* smem)
{
    return reinterpret_cast<CellShared<T>*>(smem + 8192);
}

// A solver parameter in the solver's type (FP32 copies are set on the host).
template <typename T>
__device__ __forceinline__ T prm(double d, float f)
{
    if constexpr (sizeof(T) == 8) return d;
    else return f;
}

// Sums K compensated accumulators over the block.  Thread 0 writes the totals to
// sh->out[] and then runs epi(sh) before the closing barrier, so every thread sees
// the totals and whatever the epilogue derived from them.
// Reductions of at least this many values run their second stage on all warps (one
// value per warp) instead of on warp 0 alone, at the price of one more barrier.
constexpr int kSpreadReduce = 8;

struct NoEpi {
    template <typename S>
    __device__ __forceinline__ void operator()(S*) const {}
};

template <typename T, int K, typename Epi = NoEpi>
__device__ __forceinline__ void block_reduce(Acc<T> (&a)[K], unsigned char* smem, Epi epi = Epi())
{
    T* red = reinterpret_cast<T*>(smem);  // [32 warps][K][2]
    CellShared<T>* sh = cell_shared<T>(smem);
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
    if constexpr (K >= kSpreadReduce) {
        // value k across the warps' partials on warp k mod nw (the same tree as below)
        for (int k = w; k < K; k += nw) {
            Acc<T> b;
            if (lane < nw) {
                b.hi = red[(lane * K + k) * 2];
                b.lo = red[(lane * K + k) * 2 + 1];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T h2 = __shfl_xor_sync(kFull, b.hi, o);
                const T l2 = __shfl_xor_sync(kFull, b.lo, o);
                b.merge(h2, l2);
            }
            if (lane == 0) {
                sh->out[k] = b.hi;
                sh->outlo[k] = b.lo;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) epi(sh);
    } else if (w == 0) {
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
            for (int k = 0; k < K; ++k) {
                sh->out[k] = b[k].hi;
                sh->outlo[k] = b[k].lo;
            }
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
    CellShared<T>* sh = cell_shared<T>(smem);
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
    if constexpr (KC + KP >= kSpreadReduce) {
        // value v across the warps' partials on warp v mod nw (the same tree as below)
        for (int v = w; v < KC + KP; v += nw) {
            if (v < KC) {
                Acc<T> b;
                if (lane < nw) {
                    b.hi = red[lane * W + 2 * v];
                    b.lo = red[lane * W + 2 * v + 1];
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const T h2 = __shfl_xor_sync(kFull, b.hi, o);
                    const T l2 = __shfl_xor_sync(kFull, b.lo, o);
                    b.merge(h2, l2);
                }
                if (lane == 0) {
                    sh->out[v] = b.hi;
                    sh->outlo[v] = b.lo;
                }
            } else {
                T q = lane < nw ? red[lane * W + 2 * KC + (v - KC)] : T(0);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(kFull, q, o);
                if (lane == 0) sh->out[v] = q;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) epi(sh);
    } else if (w == 0) {
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
            for (int k = 0; k < KC; ++k) {
                sh->out[k] = b[k].hi;
                sh->outlo[k] = b[k].lo;
            }
#pragma unroll
            for (int k = 0; k < KP; ++k) sh->out[KC + k] = q[k];
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
    CellShared<T>* sh = cell_shared<T>(smem);
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
    if constexpr (K >= kSpreadReduce) {
        // value k across the warps' partials on warp k mod nw (the same tree as below)
        for (int k = w; k < K; k += nw) {
            T q = lane < nw ? red[lane * K + k] : T(0);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(kFull, q, o);
            if (lane == 0) sh->out[k] = q;
        }
        __syncthreads();
        if (threadIdx.x == 0) epi(sh);
    } else if (w == 0) {
        T q[K];
#pragma unroll
        for (int k = 0; k < K; ++k) q[k] = lane < nw ? red[lane * K + k] : T(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < K; ++k) q[k] += __shfl_xor_sync(kFull, q[k], o);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) sh->out[k] = q[k];
            epi(sh);
        }
    }
    __syncthreads();
}

// Four consecutive elements of a per-cell vector (3 n_pad values, n_pad a multiple of
// 4, 16-byte aligned): one 16-byte access for FP32, two for FP64.
template <typename T>
__device__ __forceinline__ void ld4(const T* p, T (&r)[4])
{
    if constexpr (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        r[0] = q.x; r[1] = q.y; r[2] = q.z; r[3] = q.w;
    } else {
        const double2 a = *reinterpret_cast<const double2*>(p);
        const double2 b = *reinterpret_cast<const double2*>(p + 2);
        r[0] = a.x; r[1] = a.y; r[2] = b.x; r[3] = b.y;
    }
}

template <typename T>
__device__ __forceinline__ void st4(T* p, const T (&r)[4])
{
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
    } else {
        *reinterpret_cast<double2*>(p) = make_double2(r[0], r[1]);
        *reinterpret_cast<double2*>(p + 2) = make_double2(r[2], r[3]);
    }
}

// Eight consecutive read-only values (32-byte aligned) through the non-coherent path.
template <typename T>
__device__ __forceinline__ void ldg8(const T* p, T (&r)[8])
{
    if constexpr (sizeof(T) == 4) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(p));
        const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
        r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w; r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double2 a = __ldg(reinterpret_cast<const double2*>(p) + q);
            r[2 * q] = a.x;
            r[2 * q + 1] = a.y;
        }
    }
}

// The eight one-ring indices of vertex i from the fixed-width table.
__device__ __forceinline__ void ring8_indices(const unsigned short* t, int i, int (&j)[8])
{
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(t) + i);
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 8; ++q) j[q] = (int)((w[q >> 1] >> (16 * (q & 1))) & 0xffffu);
}

template <typename T>
__device__ __forceinline__ T* vec_ptr(const GroupDesc<T>& gd, unsigned char* smem, char* slot, int v)
{
    const int l = gd.loc[v];
    return l >= 0 ? reinterpret_cast<T*>(smem + kFixedSmem + l) : reinterpret_cast<T*>(slot + (-(long long)l - 1));
}

// A_k (a third of the incident triangle areas) and the unit area-weighted normal of
// vertex i of a cell whose FP32 SoA positions start at xc (immersed-boundary forces,
// collision planes).
__device__ __forceinline__ void vertex_area_normal(const TopoDev<float>& tp, const float* xc, int i, float* A, float n[3])
{
    const int n_ = tp.n;
    float N[3] = {0.f, 0.f, 0.f}, S = 0.f;
    const int b0 = __ldg(&tp.inc_ptr[i]), b1 = __ldg(&tp.inc_ptr[i + 1]);
    for (int q = b0; q < b1; ++q) {
        const unsigned e = __ldg(&tp.inc_idx[q]);
        const ushort4 tv = __ldg(&tp.tri[e >> 2]);
        const int p0 = tv.x, p1 = tv.y, p2 = tv.z;
        float e1[3], e2[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float x0 = xc[c * n_ + p0];
            e1[c] = xc[c * n_ + p1] - x0;
            e2[c] = xc[c * n_ + p2] - x0;
        }
        const float cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
#pragma unroll
        for (int c = 0; c < 3; ++c) N[c] += 0.5f * cr[c];
        S += sqrtf(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    }
    *A = S * (1.f / 6.f);
    const float inv = rsqrtf(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) n[c] = N[c] * inv;
}

}  // namespace npfem
