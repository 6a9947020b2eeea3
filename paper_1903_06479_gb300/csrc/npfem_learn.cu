// Learned warm start: training-data features, the MLP's loss and gradient, Adam,
// batched inference, and installing a trained network in a handle.  The network
// (9 -> 64 -> 64 -> 3, tanh) and the features are described in npfem_ws.cuh; the
// forward pass always uses the BF16-rounded weights (straight-through: the gradient
// of the rounded network is applied to the FP32 master weights).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "npfem_device.cuh"
#include "npfem_internal.h"
#include "npfem_ws.cuh"

namespace npfem {
namespace {

// One block per cell: features at the first guess y and, if x_next is given, the
// rest-frame target R^T (x_{n+1} - y).
__global__ void __launch_bounds__(256) ws_features_kernel(const TopoDev<float> tp, int n_cells, const float* x,
                                                          const float* v, const float* f, const float* x_next,
                                                          float* feat, float* target)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = tp.n, np = tp.n_pad, tid = threadIdx.x, NT = blockDim.x;
    float* Y = reinterpret_cast<float*>(smem + kFixedSmem);
    float* D = Y + 3 * np;
    float* UY = D + 3 * np;
    CellShared<float>* sh = cell_shared<float>(smem);
    const float h = tp.h, inv_ms = 1.f / tp.inertia_scale;
    for (int cell = blockIdx.x; cell < n_cells; cell += gridDim.x) {
        const long long so = (long long)cell * 3 * n;
        const float o[3] = {x[so], x[so + n], x[so + 2 * n]};
        for (int e = tid; e < 3 * np; e += NT) {
            const int c = e / np, i = e - c * np;
            float yv = 0.f, uy = 0.f;
            if (i < n) {
                uy = (h * v[so + c * n + i] + h * h * f[so + c * n + i] * tp.inv_mass[i]) * inv_ms;
                yv = (x[so + c * n + i] - o[c]) + uy;
            }
            Y[e] = yv;
            UY[e] = uy;
        }
        __syncthreads();
        ws_frame(tp, Y, D, smem);
        float R[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) R[q] = sh->post[q];
        for (int i = tid; i < n; i += NT) {
            float ft[kMlpIn];
            ws_vertex_features(tp, D, f + so, i, R, ft);
            float* out = feat + ((long long)cell * n + i) * kMlpIn;
#pragma unroll
            for (int k = 0; k < kMlpIn; ++k) out[k] = ft[k];
            if (x_next) {
                float dl[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) dl[c] = (x_next[so + c * n + i] - x[so + c * n + i]) - UY[c * np + i];
                float* t = target + ((long long)cell * n + i) * kMlpOut;
#pragma unroll
                for (int b = 0; b < 3; ++b) t[b] = R[b] * dl[0] + R[3 + b] * dl[1] + R[6 + b] * dl[2];
            }
        }
        __syncthreads();
    }
}

// Learned first increments u = (y - x_n) + R MLP(features at y) of the warm start,
// one block per cell (grid-stride), two blocks per SM: the same frame, features and
// network as the solver's in-kernel warm start.  out: u ([3][n] per cell), or the
// positions x_n + u when positions is set.
__global__ void __launch_bounds__(512, 2) ws_increment_kernel(const TopoDev<float> tp, int n_cells, const float* x,
                                                             const float* v, const float* f, float* out, int positions)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = tp.n, np = tp.n_pad, tid = threadIdx.x, NT = blockDim.x, lane = tid & 31;
    const int n16 = (n + 15) & ~15;
    float* Y = reinterpret_cast<float*>(smem + kFixedSmem);
    float* D = Y + 3 * np;
    float* UY = D + 3 * np;
    float* Xs = UY + 3 * np;  // [n16][16] normalised features
    CellShared<float>* sh = cell_shared<float>(smem);
    const float h = tp.h, inv_ms = 1.f / tp.inertia_scale;
    const float* P = tp.mlp;
    for (int cell = blockIdx.x; cell < n_cells; cell += gridDim.x) {
        const long long so = (long long)cell * 3 * n;
        const float o[3] = {x[so], x[so + n], x[so + 2 * n]};
        for (int e = tid; e < 3 * np; e += NT) {
            const int c = e / np, i = e - c * np;
            float yv = 0.f, uy = 0.f;
            if (i < n) {
                uy = (h * v[so + c * n + i] + h * h * f[so + c * n + i] * __ldg(&tp.inv_mass[i])) * inv_ms;
                yv = (x[so + c * n + i] - o[c]) + uy;
            }
            Y[e] = yv;
            UY[e] = uy;
        }
        __syncthreads();
        ws_frame(tp, Y, D, smem);
        float R[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) R[q] = sh->post[q];
        for (int i = tid; i < n16; i += NT) {
            float ft[kMlpIn];
            if (i < n) ws_vertex_features(tp, D, f + so, i, R, ft);
            float4* row = reinterpret_cast<float4*>(Xs + 16 * i);
            float xv[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) xv[k] = (k < kMlpIn && i < n) ? (ft[k] - P[kPMu + k]) / P[kPSig + k] : 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) row[q] = make_float4(xv[4 * q], xv[4 * q + 1], xv[4 * q + 2], xv[4 * q + 3]);
        }
        __syncthreads();
        for (int tile = tid >> 5; tile * 16 < n; tile += NT >> 5) {
            float olo[3], ohi[3];
            mlp_warp16(P, Xs + 256 * tile, olo, ohi);
            if ((lane & 3) == 0) {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int i = tile * 16 + (lane >> 2) + 8 * r;
                    if (i >= n) continue;
                    const float* oo = r ? ohi : olo;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float uc = UY[c * np + i] + (R[3 * c] * oo[0] + R[3 * c + 1] * oo[1] + R[3 * c + 2] * oo[2]);
                        out[so + c * n + i] = positions ? x[so + c * n + i] + uc : uc;
                    }
                }
            }
        }
        __syncthreads();
    }
}

// Temporal network (an addition to the paper's method): along a trajectory, the first
// iterate y_n + c_{n-1} + R MLP(features), c_k = x_{k+1} - y_k the converged correction
// of step k.  Features of vertex i in the rest frame: the trend R^T (c_{n-1} - c_{n-2}),
// the force change as a displacement w_i = R^T h^2 (F_n - F_{n-1})_i / m_i, and its
// cotangent Laplacian over the one-ring.  One block per cell.  Inference (tp.tmlp set
// and out given): out = u_y + c_{n-1} + R o (increments relative to x_n; without a
// network, u_y + c_{n-1}).  Training: the feature rows into feat, and with x_next the
// target R^T (c_n - c_{n-1}) and c_n itself (c_out).
__global__ void __launch_bounds__(512, 2) ws_temporal_kernel(const TopoDev<float> tp, int n_cells, const float* x,
                                                            const float* v, const float* f, const float* f_prev,
                                                            const float* c1, const float* c2, const float* x_next,
                                                            float* feat, float* target, float* c_out, float* out,
                                                            long long stride)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = tp.n, np = tp.n_pad, tid = threadIdx.x, NT = blockDim.x, lane = tid & 31;
    const int n16 = (n + 15) & ~15;
    float* Y = reinterpret_cast<float*>(smem + kFixedSmem);
    float* D = Y + 3 * np;
    float* UY = D + 3 * np;
    float* Wd = UY + 3 * np;  // world-frame h^2 (F_n - F_{n-1}) / m
    float* Xs = Wd + 3 * np;  // [n16][16] normalised features (inference)
    CellShared<float>* sh = cell_shared<float>(smem);
    const float h = tp.h, inv_ms = 1.f / tp.inertia_scale;
    const float* P = tp.tmlp;
    for (int cell = blockIdx.x; cell < n_cells; cell += gridDim.x) {
        const long long so = (long long)cell * stride;
        const float o[3] = {x[so], x[so + n], x[so + 2 * n]};
        for (int e = tid; e < 3 * np; e += NT) {
            const int c = e / np, i = e - c * np;
            float yv = 0.f, uy = 0.f, wd = 0.f;
            if (i < n) {
                const float im = __ldg(&tp.inv_mass[i]);
                uy = (h * v[so + c * n + i] + h * h * f[so + c * n + i] * im) * inv_ms;
                yv = (x[so + c * n + i] - o[c]) + uy;
                wd = h * h * (f[so + c * n + i] - f_prev[so + c * n + i]) * im;
            }
            Y[e] = yv;
            UY[e] = uy;
            Wd[e] = wd;
        }
        __syncthreads();
        ws_frame(tp, Y, D, smem);
        float R[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) R[q] = sh->post[q];
        const bool infer = out && P;
        for (int i = tid; i < (infer ? n16 : n); i += NT) {
            float ft[kMlpIn];
            if (i < n) {
                float lap[3] = {0.f, 0.f, 0.f};
                const float wi[3] = {Wd[i], Wd[np + i], Wd[2 * np + i]};
                if (tp.k8) {
                    int jr[8];
                    float cw[8];
                    ring8_indices(tp.ring8_idx, i, jr);
                    ldg8(tp.ring8_c + 8 * i, cw);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        if (jr[q] == i) continue;
#pragma unroll
                        for (int c = 0; c < 3; ++c) lap[c] += cw[q] * (Wd[c * np + jr[q]] - wi[c]);
                    }
                } else {
                    for (int q = tp.ring_ptr[i]; q < tp.ring_ptr[i + 1]; ++q) {
                        const int j = tp.ring_idx[q];
                        const float cq = tp.ring_c[q];
#pragma unroll
                        for (int c = 0; c < 3; ++c) lap[c] += cq * (Wd[c * np + j] - wi[c]);
                    }
                }
                float tr[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) tr[c] = c1[so + c * n + i] - c2[so + c * n + i];
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    ft[b] = R[b] * tr[0] + R[3 + b] * tr[1] + R[6 + b] * tr[2];
                    ft[3 + b] = R[b] * wi[0] + R[3 + b] * wi[1] + R[6 + b] * wi[2];
                    ft[6 + b] = R[b] * lap[0] + R[3 + b] * lap[1] + R[6 + b] * lap[2];
                }
            }
            if (infer) {
                float4* row = reinterpret_cast<float4*>(Xs + 16 * i);
                float xv[16];
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    xv[k] = (k < kMlpIn && i < n) ? (ft[k] - P[kPMu + k]) / P[kPSig + k] : 0.f;
#pragma unroll
                for (int q = 0; q < 4; ++q) row[q] = make_float4(xv[4 * q], xv[4 * q + 1], xv[4 * q + 2], xv[4 * q + 3]);
                continue;
            }
            if (feat) {
                float* fo = feat + ((long long)cell * n + i) * kMlpIn;
#pragma unroll
                for (int k = 0; k < kMlpIn; ++k) fo[k] = ft[k];
            }
            if (x_next) {
                float cn[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) cn[c] = (x_next[so + c * n + i] - x[so + c * n + i]) - UY[c * np + i];
                if (c_out)
#pragma unroll
                    for (int c = 0; c < 3; ++c) c_out[so + c * n + i] = cn[c];
                if (target) {
                    float dl[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) dl[c] = cn[c] - c1[so + c * n + i];
                    float* t = target + ((long long)cell * n + i) * kMlpOut;
#pragma unroll
                    for (int b = 0; b < 3; ++b) t[b] = R[b] * dl[0] + R[3 + b] * dl[1] + R[6 + b] * dl[2];
                }
            }
            if (out && !P)
#pragma unroll
                for (int c = 0; c < 3; ++c) out[so + c * n + i] = UY[c * np + i] + c1[so + c * n + i];
        }
        __syncthreads();
        if (infer) {
            for (int tile = tid >> 5; tile * 16 < n; tile += NT >> 5) {
                float olo[3], ohi[3];
                mlp_warp16(P, Xs + 256 * tile, olo, ohi);
                if ((lane & 3) == 0) {
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        const int i = tile * 16 + (lane >> 2) + 8 * r;
                        if (i >= n) continue;
                        const float* oo = r ? ohi : olo;
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            out[so + c * n + i] = UY[c * np + i] + c1[so + c * n + i] +
                                                  (R[3 * c] * oo[0] + R[3 * c + 1] * oo[1] + R[3 * c + 2] * oo[2]);
                    }
                }
            }
            __syncthreads();
        }
    }
}

constexpr int kTile = 64;

// Mean squared error of the normalised output, sum_c (o_c - t_c / s_out_c)^2 averaged
// over n samples, and its gradient (added into grad, which the caller zeroes).
__global__ void __launch_bounds__(256) mlp_grad_kernel(const float* __restrict__ P, const float* __restrict__ feat,
                                                      const float* __restrict__ target, const int* __restrict__ idx,
                                                      int n, float inv_n, float* grad, float* loss)
{
    extern __shared__ __align__(16) float sm[];
    float* W = sm;                         // parameters, weights rounded to BF16
    float* G = W + kMlpParams;             // gradient accumulator
    float* X = G + kMlpTrainable + 4;      // [tile][9] normalised inputs (pads to 16 B)
    float* H1 = X + kTile * 12;            // [tile][64]
    float* H2 = H1 + kTile * kMlpH;        // [tile][64]
    float* D2 = H2 + kTile * kMlpH;        // [tile][64]
    float* D1 = D2 + kTile * kMlpH;        // [tile][64]
    float* DO = D1 + kTile * kMlpH;        // [tile][3]
    __shared__ float red[32];
    const int tid = threadIdx.x, NT = blockDim.x;
    for (int q = tid; q < kMlpParams; q += NT) W[q] = q < kMlpTrainable && (q < kPB1 || (q >= kPW2 && q < kPB2) || (q >= kPW3 && q < kPB3)) ? bf16_round(P[q]) : P[q];
    for (int q = tid; q < kMlpTrainable; q += NT) G[q] = 0.f;
    float lsum = 0.f;
    __syncthreads();
    const int ntiles = (n + kTile - 1) / kTile;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int base = tile * kTile, cnt = min(kTile, n - base);
        for (int e = tid; e < kTile * kMlpIn; e += NT) {
            const int s = e / kMlpIn, i = e - s * kMlpIn;
            float xv = 0.f;
            if (s < cnt) {
                const long long smp = idx ? idx[base + s] : base + s;
                xv = bf16_round((feat[smp * kMlpIn + i] - W[kPMu + i]) / W[kPSig + i]);
            }
            X[s * 12 + i] = xv;
        }
        __syncthreads();
        for (int e = tid; e < kTile * kMlpH; e += NT) {
            const int s = e / kMlpH, j = e - s * kMlpH;
            float a = W[kPB1 + j];
#pragma unroll
            for (int i = 0; i < kMlpIn; ++i) a += W[kPW1 + j * kMlpIn + i] * X[s * 12 + i];
            H1[e] = tanhf(a);
        }
        __syncthreads();
        for (int e = tid; e < kTile * kMlpH; e += NT) {
            const int s = e / kMlpH, j = e - s * kMlpH;
            float a = W[kPB2 + j];
            for (int i = 0; i < kMlpH; ++i) a += W[kPW2 + j * kMlpH + i] * bf16_round(H1[s * kMlpH + i]);
            H2[e] = tanhf(a);
        }
        __syncthreads();
        for (int e = tid; e < kTile * kMlpOut; e += NT) {
            const int s = e / kMlpOut, c = e - s * kMlpOut;
            float d = 0.f;
            if (s < cnt) {
                float a = W[kPB3 + c];
                for (int i = 0; i < kMlpH; ++i) a += W[kPW3 + c * kMlpH + i] * H2[s * kMlpH + i];
                const long long smp = idx ? idx[base + s] : base + s;
                const float r = a - target[smp * kMlpOut + c] / W[kPSout + c];
                lsum += r * r;
                d = 2.f * r * inv_n;
            }
            DO[e] = d;
        }
        __syncthreads();
        for (int e = tid; e < kTile * kMlpH; e += NT) {
            const int s = e / kMlpH, i = e - s * kMlpH;
            float a = 0.f;
#pragma unroll
            for (int c = 0; c < kMlpOut; ++c) a += DO[s * kMlpOut + c] * W[kPW3 + c * kMlpH + i];
            const float h2 = H2[e];
            D2[e] = a * (1.f - h2 * h2);
        }
        __syncthreads();
        for (int e = tid; e < kTile * kMlpH; e += NT) {
            const int s = e / kMlpH, i = e - s * kMlpH;
            float a = 0.f;
            for (int j = 0; j < kMlpH; ++j) a += D2[s * kMlpH + j] * W[kPW2 + j * kMlpH + i];
            const float h1 = H1[e];
            D1[e] = a * (1.f - h1 * h1);
        }
        __syncthreads();
        // gradient entries, each owned by one thread
        for (int q = tid; q < kMlpTrainable; q += NT) {
            float a = 0.f;
            if (q < kPB1) {
                const int j = q / kMlpIn, i = q - j * kMlpIn;
                for (int s = 0; s < kTile; ++s) a += D1[s * kMlpH + j] * X[s * 12 + i];
            } else if (q < kPW2) {
                const int j = q - kPB1;
                for (int s = 0; s < kTile; ++s) a += D1[s * kMlpH + j];
            } else if (q < kPB2) {
                const int j = (q - kPW2) / kMlpH, i = (q - kPW2) - j * kMlpH;
                for (int s = 0; s < kTile; ++s) a += D2[s * kMlpH + j] * bf16_round(H1[s * kMlpH + i]);
            } else if (q < kPW3) {
                const int j = q - kPB2;
                for (int s = 0; s < kTile; ++s) a += D2[s * kMlpH + j];
            } else if (q < kPB3) {
                const int c = (q - kPW3) / kMlpH, i = (q - kPW3) - c * kMlpH;
                for (int s = 0; s < kTile; ++s) a += DO[s * kMlpOut + c] * H2[s * kMlpH + i];
            } else {
                const int c = q - kPB3;
                for (int s = 0; s < kTile; ++s) a += DO[s * kMlpOut + c];
            }
            G[q] += a;
        }
        __syncthreads();
    }
    for (int q = tid; q < kMlpTrainable; q += NT) atomicAdd(&grad[q], G[q]);
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(kFull, lsum, o);
    if ((tid & 31) == 0) red[tid >> 5] = lsum;
    __syncthreads();
    if (tid == 0) {
        float t = 0.f;
        for (int w = 0; w < NT / 32; ++w) t += red[w];
        atomicAdd(loss, t * inv_n);
    }
}

// Adam (Kingma & Ba) on the trainable parameters.
__global__ void mlp_adam_kernel(float* P, float* m, float* v, const float* g, int step, float lr, float b1, float b2,
                                float eps)
{
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < kMlpTrainable; q += gridDim.x * blockDim.x) {
        const float gq = g[q];
        const float mq = b1 * m[q] + (1.f - b1) * gq;
        const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
        m[q] = mq;
        v[q] = vq;
        P[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
    }
}

// Device layout of a network (npfem_ws.cuh): the parameters with the weights
// rounded to BF16, followed by the MMA operand fragments of W1 and W2.
__global__ void mlp_round_kernel(const float* P, float* out)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < kMlpDeviceWords; q += gridDim.x * blockDim.x) {
        if (q < kMlpParams) {
            const bool weight = (q < kPB1) || (q >= kPW2 && q < kPB2) || (q >= kPW3 && q < kPB3);
            out[q] = weight ? bf16_round(P[q]) : P[q];
        } else if (q < kFragW1) {
            out[q] = 0.f;
        } else {
            out[q] = __uint_as_float(mlp_fragment_word(P, q - kFragW1));
        }
    }
}

// One warp per 16 feature rows, the same arithmetic as the solver's warm start.
__global__ void __launch_bounds__(128) mlp_predict_kernel(const float* Pr, const float* feat, int n, float* out)
{
    __shared__ float xs[4][256];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float* Xs = xs[wib];
    const int ntiles = (n + 15) / 16;
    for (int tile = blockIdx.x * 4 + wib; tile < ntiles; tile += gridDim.x * 4) {
        if (lane < 16) {
            const int s = tile * 16 + lane;
#pragma unroll
            for (int k = 0; k < 16; ++k)
                Xs[lane * 16 + k] = (k < kMlpIn && s < n) ? (feat[(long long)s * kMlpIn + k] - Pr[kPMu + k]) / Pr[kPSig + k] : 0.f;
        }
        __syncwarp();
        float olo[3], ohi[3];
        mlp_warp16(Pr, Xs, olo, ohi);
        if ((lane & 3) == 0) {
            const int s0 = tile * 16 + (lane >> 2), s1 = s0 + 8;
#pragma unroll
            for (int c = 0; c < kMlpOut; ++c) {
                if (s0 < n) out[(long long)s0 * kMlpOut + c] = olo[c];
                if (s1 < n) out[(long long)s1 * kMlpOut + c] = ohi[c];
            }
        }
        __syncwarp();
    }
}

constexpr size_t kGradSmem = sizeof(float) * (kMlpParams + kMlpTrainable + 4 + kTile * 12 + 4 * kTile * kMlpH + kTile * kMlpOut);

}  // namespace

cudaError_t launch_ws_temporal(const npfem_handle* h, int n_cells, const float* x, const float* v, const float* f,
                               const float* f_prev, const float* c1, const float* c2, const float* x_next, float* feat,
                               float* target, float* c_out, float* out, long long stride, cudaStream_t s)
{
    if (n_cells <= 0) return cudaSuccess;
    const int np = h->n_pad, n16 = (h->n + 15) & ~15;
    const int smem = kFixedSmem + 12 * np * (int)sizeof(float) + 16 * n16 * (int)sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(ws_temporal_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int per_sm = smem <= h->smem_optin / 2 ? 2 : 1;
    const int grid = std::min(n_cells, per_sm * h->sm_count);
    ws_temporal_kernel<<<grid, 512, smem, s>>>(h->tf, n_cells, x, v, f, f_prev, c1, c2, x_next, feat, target, c_out,
                                               out, stride);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_ws_increments(const npfem_handle* h, int n_cells, const float* x, const float* v, const float* f,
                                 float* out, bool positions, cudaStream_t s)
{
    if (n_cells <= 0) return cudaSuccess;
    const int np = h->n_pad, n16 = (h->n + 15) & ~15;
    const int smem = kFixedSmem + 9 * np * (int)sizeof(float) + 16 * n16 * (int)sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(ws_increment_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int per_sm = smem <= h->smem_optin / 2 ? 2 : 1;
    const int grid = std::min(n_cells, per_sm * h->sm_count);
    ws_increment_kernel<<<grid, 512, smem, s>>>(h->tf, n_cells, x, v, f, out, positions ? 1 : 0);
    count_launch();
    return cudaGetLastError();
}

}  // namespace npfem

using namespace npfem;

extern "C" {

int npfem_mlp_nparam(void) { return kMlpParams; }

int npfem_mlp_loss_grad(const float* params, const float* feat, const float* target, const int32_t* idx, int n,
                        float* grad, float* loss, void* stream)
{
    if (!params || !feat || !target || !grad || !loss || n < 1)
        return set_error(NPFEM_ERR_INVALID_ARG, "npfem_mlp_loss_grad: null pointer or n < 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * kMlpParams, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(float), s);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradSmem);
    if (e != cudaSuccess) return set_error(NPFEM_ERR_CUDA, std::string("npfem_mlp_loss_grad: ") + cudaGetErrorString(e));
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = (n + kTile - 1) / kTile;
    const int grid = std::max(1, std::min(tiles, 2 * sms));
    mlp_grad_kernel<<<grid, 256, kGradSmem, s>>>(params, feat, target, idx, n, 1.f / n, grad, loss);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(NPFEM_ERR_CUDA, std::string("npfem_mlp_loss_grad: ") + cudaGetErrorString(e));
    return 0;
}

int npfem_mlp_adam(float* params, float* m, float* v, const float* grad, int step, float lr, float beta1, float beta2,
                   float eps, void* stream)
{
    if (!params || !m || !v || !grad || step < 1) return set_error(NPFEM_ERR_INVALID_ARG, "npfem_mlp_adam: bad argument");
    mlp_adam_kernel<<<20, 256, 0, static_cast<cudaStream_t>(stream)>>>(params, m, v, grad, step, lr, beta1, beta2, eps);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(NPFEM_ERR_CUDA, std::string("npfem_mlp_adam: ") + cudaGetErrorString(e));
    return 0;
}

int npfem_mlp_predict(const float* params, const float* feat, int n, float* out, float* scratch, void* stream)
{
    if (!params || !feat || !out || !scratch || n < 0) return set_error(NPFEM_ERR_INVALID_ARG, "npfem_mlp_predict: bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    mlp_round_kernel<<<20, 256, 0, s>>>(params, scratch);
    if (n > 0) mlp_predict_kernel<<<std::max(1, std::min((n + 63) / 64, 4096)), 128, 0, s>>>(scratch, feat, n, out);
    count_launch(n > 0 ? 2 : 1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(NPFEM_ERR_CUDA, std::string("npfem_mlp_predict: ") + cudaGetErrorString(e));
    return 0;
}

int npfem_ws_features(npfem_handle* h, int n_cells, const float* x, const float* v, const float* f, const float* x_next,
                      float* feat, float* target, void* stream)
{
    if (!h || n_cells < 0 || !x || !v || !f || !feat || (x_next && !target))
        return set_error(NPFEM_ERR_INVALID_ARG, "npfem_ws_features: bad argument");
    if (h->precision == NPFEM_PREC_FP64)
        return set_error(NPFEM_ERR_INVALID_ARG, "npfem_ws_features: FP32 state handles only");
    if (n_cells == 0) return 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int smem = kFixedSmem + 3 * 3 * h->n_pad * (int)sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(ws_features_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return set_error(NPFEM_ERR_CUDA, std::string("npfem_ws_features: ") + cudaGetErrorString(e));
    ws_features_kernel<<<std::min(n_cells, 4 * h->sm_count), 256, smem, s>>>(h->tf, n_cells, x, v, f, x_next, feat, target);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(NPFEM_ERR_CUDA, std::string("npfem_ws_features: ") + cudaGetErrorString(e));
    return 0;
}

int npfem_ws_features_temporal(npfem_handle* h, int n_cells, const float* x, const float* v, const float* f,
                               const float* f_prev, const float* c1, const float* c2, const float* x_next, float* feat,
                               float* target, float* c_out, void* stream)
{
    if (!h || n_cells < 0 || !x || !v || !f || !f_prev || !c1 || !c2 || (target && !x_next) || (c_out && !x_next))
        return set_error(NPFEM_ERR_INVALID_ARG, "npfem_ws_features_temporal: bad argument");
    if (h->precision == NPFEM_PREC_FP64)
        return set_error(NPFEM_ERR_INVALID_ARG, "npfem_ws_features_temporal: FP32 state handles only");
    TopoDev<float> tp = h->tf;
    tp.tmlp = nullptr;  // features only
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n_cells == 0) return 0;
    const int np = h->n_pad, n16 = (h->n + 15) & ~15;
    const int smem = kFixedSmem + 12 * np * (int)sizeof(float) + 16 * n16 * (int)sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(ws_temporal_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) {
        const int grid = std::min(n_cells, 2 * h->sm_count);
        ws_temporal_kernel<<<grid, 512, smem, s>>>(tp, n_cells, x, v, f, f_prev, c1, c2, x_next, feat, target, c_out,
                                                   nullptr, 3LL * h->n);
        count_launch();
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return set_error(NPFEM_ERR_CUDA, std::string("npfem_ws_features_temporal: ") + cudaGetErrorString(e));
    return 0;
}

int npfem_ws_guess_temporal(npfem_handle* h, int n_cells, const float* x, const float* v, const float* f,
                            const float* f_prev, const float* c1, const float* c2, float* u_out, void* stream)
{
    if (!h || n_cells < 0 || !x || !v || !f || !f_prev || !c1 || !c2 || !u_out)
        return set_error(NPFEM_ERR_INVALID_ARG, "npfem_ws_guess_temporal: bad argument");
    if (h->precision == NPFEM_PREC_FP64)
        return set_error(NPFEM_ERR_INVALID_ARG, "npfem_ws_guess_temporal: FP32 state handles only");
    cudaError_t e = launch_ws_temporal(h, n_cells, x, v, f, f_prev, c1, c2, nullptr, nullptr, nullptr, nullptr, u_out,
                                       3LL * h->n, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return set_error(NPFEM_ERR_CUDA, std::string("npfem_ws_guess_temporal: ") + cudaGetErrorString(e));
    return 0;
}

int npfem_set_warmstart_temporal(npfem_handle* h, const float* params_host)
{
    if (!h) return set_error(NPFEM_ERR_INVALID_ARG, "npfem_set_warmstart_temporal: null handle");
    if (h->precision == NPFEM_PREC_FP64)
        return set_error(NPFEM_ERR_INVALID_ARG, "npfem_set_warmstart_temporal: FP32 state handles only");
    if (params_host && h->mat.beta_D != 0.0)
        return set_error(NPFEM_ERR_INVALID_ARG,
                         "npfem_set_warmstart_temporal: the network's features use the lumped first guess; beta_D > 0 "
                         "is not supported");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != h->device) cudaSetDevice(h->device);
    int rc = 0;
    std::lock_guard<std::mutex> lk(h->mu);
    if (!params_host) {
        h->tf.tmlp = nullptr;
    } else {
        if (!h->tmlp) {
            int err = 0;
            h->tmlp = h->alloc<float>(kMlpDeviceWords, &err);
            if (!h->tmlp) rc = err;
        }
        if (!rc) {
            std::vector<float> r(kMlpDeviceWords, 0.f);
            for (int q = 0; q < kMlpParams; ++q) {
                const bool weight = (q < kPB1) || (q >= kPW2 && q < kPB2) || (q >= kPW3 && q < kPB3);
                r[q] = weight ? bf16_round(params_host[q]) : params_host[q];
            }
            for (int w = 0; w < kMlpDeviceWords - kFragW1; ++w) {
                const uint32_t word = mlp_fragment_word(params_host, w);
                memcpy(&r[kFragW1 + w], &word, 4);
            }
            cudaError_t e = cudaMemcpy(h->tmlp, r.data(), sizeof(float) * kMlpDeviceWords, cudaMemcpyHostToDevice);
            if (e != cudaSuccess)
                rc = set_error(NPFEM_ERR_CUDA, std::string("npfem_set_warmstart_temporal: ") + cudaGetErrorString(e));
            else
                h->tf.tmlp = h->tmlp;
        }
    }
    h->hist_sig.clear();  // the trajectory state's layout changes with the network
    if (dev != h->device) cudaSetDevice(dev);
    return rc;
}

int npfem_set_warmstart(npfem_handle* h, const float* params_host, int mode)
{
    if (!h || mode < 0 || mode > 2 || (mode > 0 && !params_host))
        return set_error(NPFEM_ERR_INVALID_ARG, "npfem_set_warmstart: need a handle, mode 0..2 and parameters for mode > 0");
    if (h->precision == NPFEM_PREC_FP64)
        return set_error(NPFEM_ERR_INVALID_ARG, "npfem_set_warmstart: FP32 state handles only");
    if (mode > 0 && h->mat.beta_D != 0.0)
        return set_error(NPFEM_ERR_INVALID_ARG,
                         "npfem_set_warmstart: the network's features use the lumped first guess; beta_D > 0 "
                         "(non-diagonal M~) is not supported");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != h->device) cudaSetDevice(h->device);
    int rc = 0;
    if (mode == 0) {
        h->tf.ws_mode = 0;
        h->tf.mlp = nullptr;
    } else {
        if (!h->mlp) {
            int err = 0;
            h->mlp = h->alloc<float>(kMlpDeviceWords, &err);
            if (!h->mlp) rc = err;
        }
        if (!rc) {
            std::vector<float> r(kMlpDeviceWords, 0.f);
            for (int q = 0; q < kMlpParams; ++q) {
                const bool weight = (q < kPB1) || (q >= kPW2 && q < kPB2) || (q >= kPW3 && q < kPB3);
                r[q] = weight ? bf16_round(params_host[q]) : params_host[q];
            }
            for (int w = 0; w < kMlpDeviceWords - kFragW1; ++w) {
                const uint32_t word = mlp_fragment_word(params_host, w);
                memcpy(&r[kFragW1 + w], &word, 4);
            }
            cudaError_t e = cudaMemcpy(h->mlp, r.data(), sizeof(float) * kMlpDeviceWords, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) rc = set_error(NPFEM_ERR_CUDA, std::string("npfem_set_warmstart: ") + cudaGetErrorString(e));
            h->tf.ws_mode = mode;
            h->tf.mlp = h->mlp;
        }
    }
    if (dev != h->device) cudaSetDevice(dev);
    return rc;
}

}  // extern "C"
