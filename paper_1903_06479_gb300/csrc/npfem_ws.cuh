// Learned warm start (an addition to the paper's method): device code shared by the
// solver kernels and the training-data kernels.
//
// Per cell, at the first guess y of Algorithm 1:
//   R   = orthogonal polar factor of A = sum_i m_i (y_i - y_cm)(X_i - X_cm)^T, the
//         best-fit rotation of the rest shape (Newton iteration R <- (R + R^-T) / 2);
//   d_i = R^T (y_i - y_cm) - (X_i - X_cm)     displacement from rest (rest frame)
//   l_i = sum_j c_ij (d_j - d_i)              its cotangent Laplacian over the 1-ring
//   f_i = R^T F_ext,i h^2 / m_i               external force as a displacement
// A 3-layer MLP (9 -> 64 -> 64 -> 3, tanh, BF16 weights, FP32 accumulation) maps the
// normalised features to the rest-frame correction, and the warm start is
//   x^(1) = y + R (s_out * MLP((feat - mu) / sigma)).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "npfem_device.cuh"

namespace npfem {

constexpr int kMlpIn = 9, kMlpH = 64, kMlpOut = 3;
constexpr int kPW1 = 0;
constexpr int kPB1 = kPW1 + kMlpH * kMlpIn;
constexpr int kPW2 = kPB1 + kMlpH;
constexpr int kPB2 = kPW2 + kMlpH * kMlpH;
constexpr int kPW3 = kPB2 + kMlpH;
constexpr int kPB3 = kPW3 + kMlpOut * kMlpH;
constexpr int kPMu = kPB3 + kMlpOut;
constexpr int kPSig = kPMu + kMlpIn;
constexpr int kPSout = kPSig + kMlpIn;
constexpr int kMlpParams = kPSout + kMlpOut;   // 5016
constexpr int kMlpTrainable = kPMu;           // weights and biases
// device layout of an installed network: the 5016 parameters (weights rounded to
// BF16), padding to 5024 words, then the BF16 operand fragments of W1 (512 words)
// and W2 (2048 words) for the warp-level m16n8k16 MMAs
constexpr int kFragW1 = 5024;
constexpr int kFragW2 = kFragW1 + 512;
constexpr int kMlpDeviceWords = kFragW2 + 2048;

// Round an FP32 value to the nearest BF16 (ties to even), returned as FP32.
__host__ __device__ inline float bf16_round(float x)
{
    unsigned u;
#ifdef __CUDA_ARCH__
    u = __float_as_uint(x);
#else
    memcpy(&u, &x, 4);
#endif
    if ((u & 0x7f800000u) == 0x7f800000u) return x;
    u += 0x7fffu + ((u >> 16) & 1u);
    u &= 0xffff0000u;
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}

// tanh(x) = 1 - 2 / (1 + exp(2 x)) (absolute error ~1e-7; saturates correctly)
__device__ __forceinline__ float fast_tanh(float x) { return 1.f - __fdividef(2.f, 1.f + __expf(2.f * x)); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The network on 16 rows held by one warp.  Xs: this warp's normalised inputs,
// [16][16] floats (columns 9..15 zero).  Lane (g = lane / 4, t = lane % 4) ends with
// the outputs of rows g and g + 8 (physical units, rest frame) when t == 0.
// Layer 1 and 2 run as BF16 m16n8k16 MMAs with FP32 accumulation; the accumulator
// fragment of layer 1 is the operand fragment of layer 2, so the hidden layer never
// leaves registers.  Layer 3 (64 -> 3) is a dot product reduced over the 4 lanes t.
__device__ __forceinline__ void mlp_warp16(const float* P, const float* Xs, float (&olo)[3], float (&ohi)[3])
{
    const uint32_t* frag = reinterpret_cast<const uint32_t*>(P);
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    uint32_t ax[4];
    ax[0] = pack_bf16x2(Xs[g * 16 + 2 * t], Xs[g * 16 + 2 * t + 1]);
    ax[1] = pack_bf16x2(Xs[(g + 8) * 16 + 2 * t], Xs[(g + 8) * 16 + 2 * t + 1]);
    ax[2] = pack_bf16x2(Xs[g * 16 + 8 + 2 * t], Xs[g * 16 + 8 + 2 * t + 1]);
    ax[3] = pack_bf16x2(Xs[(g + 8) * 16 + 8 + 2 * t], Xs[(g + 8) * 16 + 8 + 2 * t + 1]);
    uint32_t a2[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        mma_bf16_16816(d, ax, frag[kFragW1 + (nt * 32 + lane) * 2], frag[kFragW1 + (nt * 32 + lane) * 2 + 1]);
        const float b0 = P[kPB1 + nt * 8 + 2 * t], b1 = P[kPB1 + nt * 8 + 2 * t + 1];
        const uint32_t lo = pack_bf16x2(fast_tanh(d[0] + b0), fast_tanh(d[1] + b1));
        const uint32_t hi = pack_bf16x2(fast_tanh(d[2] + b0), fast_tanh(d[3] + b1));
        a2[nt >> 1][(nt & 1) ? 2 : 0] = lo;
        a2[nt >> 1][(nt & 1) ? 3 : 1] = hi;
    }
    float plo[3] = {0.f, 0.f, 0.f}, phi[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < 4; ++kt)
            mma_bf16_16816(d, a2[kt], frag[kFragW2 + ((kt * 8 + nt) * 32 + lane) * 2],
                           frag[kFragW2 + ((kt * 8 + nt) * 32 + lane) * 2 + 1]);
        const int c0 = nt * 8 + 2 * t;
        const float b0 = P[kPB2 + c0], b1 = P[kPB2 + c0 + 1];
        const float h0 = fast_tanh(d[0] + b0), h1 = fast_tanh(d[1] + b1);
        const float h2 = fast_tanh(d[2] + b0), h3 = fast_tanh(d[3] + b1);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float w0 = P[kPW3 + c * kMlpH + c0], w1 = P[kPW3 + c * kMlpH + c0 + 1];
            plo[c] += w0 * h0 + w1 * h1;
            phi[c] += w0 * h2 + w1 * h3;
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int o = 1; o <= 2; o <<= 1) {
            plo[c] += __shfl_xor_sync(0xffffffffu, plo[c], o);
            phi[c] += __shfl_xor_sync(0xffffffffu, phi[c], o);
        }
        olo[c] = (plo[c] + P[kPB3 + c]) * P[kPSout + c];
        ohi[c] = (phi[c] + P[kPB3 + c]) * P[kPSout + c];
    }
}

// Word w (0 <= w < 2560) of the BF16 operand fragments of W1 (K padded from 9 to
// 16) and W2 for mlp_warp16, ordered [layer][k tile][n tile][lane][2]; each word
// packs two weights rounded to BF16, the lower k in the low half.
__host__ __device__ inline uint32_t mlp_fragment_word(const float* P, int w)
{
    auto bits = [](float v) -> uint32_t {
        const float r = bf16_round(v);
        uint32_t u;
        memcpy(&u, &r, 4);
        return u >> 16;
    };
    const int half = w & 1, lane = (w >> 1) & 31, g = lane >> 2, t = lane & 3;
    int n, k;
    const float* base;
    int ld, kmax;
    if (w < 512) {
        const int nt = w >> 6;
        n = nt * 8 + g;
        k = 8 * half + 2 * t;
        base = P + kPW1;
        ld = kMlpIn;
        kmax = kMlpIn;
    } else {
        const int q = (w - 512) >> 6, kt = q >> 3, nt = q & 7;
        n = nt * 8 + g;
        k = kt * 16 + 8 * half + 2 * t;
        base = P + kPW2;
        ld = kMlpH;
        kmax = kMlpH;
    }
    const float lo = k < kmax ? base[n * ld + k] : 0.f;
    const float hi = k + 1 < kmax ? base[n * ld + k + 1] : 0.f;
    return bits(lo) | (bits(hi) << 16);
}

// Orthogonal polar factor of a 3x3 matrix (row-major) by the Newton iteration
// R <- (R + R^-T) / 2 started from A scaled to unit Frobenius norm; A must be
// nonsingular with det(A) > 0 (a small deformation of a rotation).  Single thread.
template <typename S>
__device__ inline void polar_rotation(const S (&A)[9], S (&R)[9])
{
    S fn = S(0);
    for (int q = 0; q < 9; ++q) fn += A[q] * A[q];
    fn = sqrt(fn / S(3));
    for (int q = 0; q < 9; ++q) R[q] = A[q] / fn;
    for (int it = 0; it < 24; ++it) {
        // cofactor matrix / det = R^-T
        const S c00 = R[4] * R[8] - R[5] * R[7], c01 = R[5] * R[6] - R[3] * R[8], c02 = R[3] * R[7] - R[4] * R[6];
        const S c10 = R[2] * R[7] - R[1] * R[8], c11 = R[0] * R[8] - R[2] * R[6], c12 = R[1] * R[6] - R[0] * R[7];
        const S c20 = R[1] * R[5] - R[2] * R[4], c21 = R[2] * R[3] - R[0] * R[5], c22 = R[0] * R[4] - R[1] * R[3];
        const S det = R[0] * c00 + R[1] * c01 + R[2] * c02;
        const S id = S(1) / det;
        const S Ri[9] = {c00 * id, c01 * id, c02 * id, c10 * id, c11 * id, c12 * id, c20 * id, c21 * id, c22 * id};
        S delta = S(0);
        for (int q = 0; q < 9; ++q) {
            const S nv = S(0.5) * (R[q] + Ri[q]);
            delta += (nv - R[q]) * (nv - R[q]);
            R[q] = nv;
        }
        // Newton's polar iteration converges quadratically: once a step moves R by
        // ~3e-6 (resp. 1e-13) the remaining error is below the format's rounding
        if (delta < S(sizeof(S) == 4 ? 1e-11 : 1e-26)) break;
    }
}

// Best-fit frame of one cell at local positions Y ([3][n_pad]): R (row-major) and
// y_cm go to sh->post[0..8] and sh->post[9..11]; the rest-frame displacements d go
// to D ([3][n_pad], zero padding).  Block-cooperative.
template <typename T>
__device__ void ws_frame(const TopoDev<T>& tp, const T* Y, T* D, unsigned char* smem)
{
    const int n = tp.n, np = tp.n_pad, tid = threadIdx.x, NT = blockDim.x;
    CellShared<T>* sh = cell_shared<T>(smem);
    // plain sums: the frame only needs the working precision
    T acc[13] = {};  // sum m y Xc^T (9), sum m y (3), sum m
    for (int i = tid; i < n; i += NT) {
        const T m = tp.mass[i];
        T y[3], xc[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            y[c] = Y[c * np + i];
            xc[c] = tp.rest_c[c * n + i];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) acc[3 * a + b] += m * y[a] * xc[b];
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[9 + a] += m * y[a];
        acc[12] += m;
    }
    block_sum<T, 13>(acc, smem, [](CellShared<T>* s) {
        T A[9], R[9];
        for (int q = 0; q < 9; ++q) A[q] = s->out[q];
        polar_rotation<T>(A, R);
        for (int q = 0; q < 9; ++q) s->post[q] = R[q];
        const T im = T(1) / s->out[12];
        for (int a = 0; a < 3; ++a) s->post[9 + a] = s->out[9 + a] * im;
    });
    T R[9], yc[3];
#pragma unroll
    for (int q = 0; q < 9; ++q) R[q] = sh->post[q];
#pragma unroll
    for (int a = 0; a < 3; ++a) yc[a] = sh->post[9 + a];
    for (int i = tid; i < np; i += NT) {
        if (i >= n) {
#pragma unroll
            for (int c = 0; c < 3; ++c) D[c * np + i] = T(0);
            continue;
        }
        const T r[3] = {Y[i] - yc[0], Y[np + i] - yc[1], Y[2 * np + i] - yc[2]};
#pragma unroll
        for (int b = 0; b < 3; ++b)
            D[b * np + i] = (R[b] * r[0] + R[3 + b] * r[1] + R[6 + b] * r[2]) - tp.rest_c[b * n + i];
    }
    __syncthreads();
}

// Feature vector of vertex i: d_i, its cotangent Laplacian over the 1-ring, and
// R^T F_i h^2 / m_i (F: the cell's forces, [3][n]).
template <typename T>
__device__ __forceinline__ void ws_vertex_features(const TopoDev<T>& tp, const T* D, const T* F, int i, const T (&R)[9],
                                                   float (&feat)[kMlpIn])
{
    const int n = tp.n, np = tp.n_pad;
    T lap[3] = {T(0), T(0), T(0)};
    const T di[3] = {D[i], D[np + i], D[2 * np + i]};
    if (tp.k8) {
        int jr[8];
        T cw[8];
        ring8_indices(tp.ring8_idx, i, jr);
        ldg8(tp.ring8_c + 8 * i, cw);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (jr[q] == i) continue;  // padding
#pragma unroll
            for (int c = 0; c < 3; ++c) lap[c] += cw[q] * (D[c * np + jr[q]] - di[c]);
        }
    } else {
        for (int q = tp.ring_ptr[i]; q < tp.ring_ptr[i + 1]; ++q) {
            const int j = tp.ring_idx[q];
            const T cq = tp.ring_c[q];
#pragma unroll
            for (int c = 0; c < 3; ++c) lap[c] += cq * (D[c * np + j] - di[c]);
        }
    }
    const T sc = tp.h * tp.h * tp.inv_mass[i];
    const T f[3] = {F[i], F[n + i], F[2 * n + i]};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        feat[b] = (float)di[b];
        feat[3 + b] = (float)lap[b];
        feat[6 + b] = (float)((R[b] * f[0] + R[3 + b] * f[1] + R[6 + b] * f[2]) * sc);
    }
}

}  // namespace npfem
