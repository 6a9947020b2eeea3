// npFEM time step on the GPU: one thread block solves one red-blood-cell membrane at
// a time (persistent blocks pull cells from a work counter), with every per-cell
// vector of the quasi-Newton solve resident in shared memory when it fits.
//
// Per cell (Algorithm 1 of arXiv:1903.06479):
//   y = x_n + h M~^{-1} M v_n + h^2 M~^{-1} F_ext             (first guess)
//   repeat: residual test; d = -LBFGS(H~^{-1}) grad g; alpha = 1, 1/2, ...
//           x + alpha d -> projections, energies, g, grad g   (line search)
//   v_{n+1} = (x_{n+1} - x_n)/h; post-convergence dissipation (Sec. 2.1.4)
//
// The solve runs on the increment u = x - x_n in cell-local coordinates (origin at
// the cell's first vertex) so that FP32 keeps the small per-step displacements:
// edges are (X_j - X_i) + (u_j - u_i) and the enclosed volume is V(x_n) + dV(u).
//
// FP64 throughput is a small fraction of FP32 on this part, so the FP32 path does
// no per-thread FP64 arithmetic: block sums are compensated FP32 pairs (error-free
// two-sum), and the few scalar FP64 operations per reduction run on one thread
// and are broadcast through shared memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "npfem_device.cuh"
#include "npfem_internal.h"
#include "npfem_ws.cuh"

namespace npfem {
namespace {

// SL(2) projection of the principal stretches (Sec. 2.1.2, area preservation):
// Sigma* = diag(a, 1/a) closest to diag(s1, s2), s1 >= s2.  With a = 1 + t,
// s1 = 1 + e1, s2 = 1 + e2 the stationarity condition a^4 - s1 a^3 + s2 a - 1 = 0
// reads phi(t) = (t - e1)(1 + t)^3 + t (1 + e2) + e2 = 0.  The minimiser is the
// largest root, the only one in [max(0, (e1 - 1)/2), 1 + e1], where phi is convex
// and changes sign; safeguarded Newton from the small-strain root (e1 - e2)/2.
template <typename T>
__device__ __forceinline__ T sl2_t(T e1, T e2)
{
    T lo = e1 > T(1) ? T(0.5) * (e1 - T(1)) : T(0);
    T hi = T(1) + e1;
    T t = T(0.5) * (e1 - e2);
    t = t < lo ? lo : (t > hi ? hi : t);
    for (int it = 0; it < 60; ++it) {
        const T a1 = T(1) + t;
        const T a2 = a1 * a1;
        const T tm = t - e1;
        const T ph = tm * a2 * a1 + t * (T(1) + e2) + e2;
        if (ph == T(0)) break;
        if (ph < T(0)) lo = t; else hi = t;
        const T dph = a2 * a1 + T(3) * tm * a2 + (T(1) + e2);
        T tn = t - ph / dph;
        if (!(tn > lo && tn < hi)) tn = T(0.5) * (lo + hi);
        const T step = tn - t;
        t = tn;
        if (fabs(step) <= Unit<T>::sl2_rel * (fabs(t) + fabs(e1) + fabs(e2)) + Unit<T>::tiny || hi - lo <= T(0)) break;
    }
    return t;
}

// Triangle t's corner gradients (row: corner j, corner k, normal share / 3, padding)
// into the buffer pass 2 gathers: with fixed-width rings, into the slots of the
// three vertices (corner i gets minus the other two; the volume gradient is formed
// from the ring in pass 2); otherwise the row itself.
template <typename T>
__device__ __forceinline__ void store_corners(const TopoDev<T>& tp, T* TRI, int t, ushort4 tv, const T (&row)[kTriRow])
{
    if (tp.k8) {
        const int np = tp.n_pad;
        const unsigned sl = tv.w;
        const int si = sl & 7u, sj = (sl >> 3) & 7u, sk = (sl >> 6) & 7u;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            TRI[(3 * si + c) * np + tv.x] = -(row[c] + row[3 + c]);
            TRI[(3 * sj + c) * np + tv.y] = row[c];
            TRI[(3 * sk + c) * np + tv.z] = row[3 + c];
        }
    } else {
        T* out = TRI + kTriRow * t;
        st4(out, reinterpret_cast<const T(&)[4]>(row[0]));
        st4(out + 4, reinterpret_cast<const T(&)[4]>(row[4]));
        st4(out + 8, reinterpret_cast<const T(&)[4]>(row[8]));
    }
}

// Objective g and gradient at x_n + U (Eq. GeneralizedObjectiveFunction and its
// derivative): inertia, local area preservation and bending (projective dynamics
// gradients), global volume conservation (PD gradient with the linearised
// projection), modified Skalak (first Piola-Kirchhoff forces).  Results are left in
// cell_shared(smem): E, its parts, V, residual r, rounding estimate of E, bad flag.
// Vn is the volume at x_n (held by the caller).
//
// Gather form, no atomics: pass 1 writes each triangle's corner gradients to TRI
// (with fixed-width rings into per-vertex slots, read back coalesced; otherwise as
// per-triangle rows with the area-weighted normal, gathered through the vertex ->
// triangle incidence); pass 2 sums them per vertex, forms the volume gradient and
// the bending residual w_i r_i into WR; pass 3 gathers the bending gradient from the
// neighbours' WR (transposed cotangent weights) and adds the volume and inertia
// terms.  Every vertex is written by one thread only.
// With kFirst, the same triangle pass also accumulates V(x_n) (left in sh->Vn) and
// Vn is ignored.
template <typename T, bool kFirst = false>
__device__ void evaluate(const TopoDev<T>& tp, const T* XN, const T* U, const T* UY, T* Gout, T* GC, T* TRI, T* WR,
                         Pair<T> Vn, unsigned char* smem, const float4* colp = nullptr, T wcol = T(0))
{
    const int n = tp.n, np = tp.n_pad, tid = threadIdx.x, NT = blockDim.x;
    CellShared<T>* sh = cell_shared<T>(smem);
    const T Cs = tp.C, Bs = tp.B, Ds = tp.Dsk;
    const T sixth = T(1) / T(6);
    Acc<T> ce[5];  // area, Skalak, bending energies; 6 dV; 6 V(x_n) (first evaluation only)
    T pl[3] = {T(0), T(0), T(0)};  // |grad C|^2, rounding estimate, degenerate count

    // ---- pass 1: triangles
    for (int t = tid; t < tp.nt; t += NT) {
        const ushort4 tv = __ldg(&tp.tri[t]);
        const int i = tv.x, j = tv.y, k = tv.z;
        T Di0, Di1, Di2, Di3;
        if constexpr (sizeof(T) == 4) {
            const float4 d4 = __ldg(reinterpret_cast<const float4*>(tp.dminv) + t);
            Di0 = d4.x; Di1 = d4.y; Di2 = d4.z; Di3 = d4.w;
        } else {
            const double2 a2 = __ldg(reinterpret_cast<const double2*>(tp.dminv) + 2 * t);
            const double2 b2 = __ldg(reinterpret_cast<const double2*>(tp.dminv) + 2 * t + 1);
            Di0 = a2.x; Di1 = a2.y; Di2 = b2.x; Di3 = b2.y;
        }
        const T Wt = __ldg(&tp.W[t]);
        T Xi[3], E1[3], E2[3], Ui[3], d1[3], d2[3], e1[3], e2[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Xi[c] = XN[c * np + i];
            E1[c] = XN[c * np + j] - Xi[c];
            E2[c] = XN[c * np + k] - Xi[c];
            Ui[c] = U[c * np + i];
            d1[c] = U[c * np + j] - Ui[c];
            d2[c] = U[c * np + k] - Ui[c];
            e1[c] = E1[c] + d1[c];
            e2[c] = E2[c] + d2[c];
        }
        if (kFirst)
            ce[4].add(Xi[0] * (E1[1] * E2[2] - E1[2] * E2[1]) + Xi[1] * (E1[2] * E2[0] - E1[0] * E2[2]) +
                      Xi[2] * (E1[0] * E2[1] - E1[1] * E2[0]));
        // F = D_s D_m^{-1} (3 x 2), columns F0, F1
        T F0[3], F1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            F0[c] = e1[c] * Di0 + e2[c] * Di2;
            F1[c] = e1[c] * Di1 + e2[c] * Di3;
        }
        const T aa = F0[0] * F0[0] + F0[1] * F0[1] + F0[2] * F0[2];
        const T bb = F0[0] * F1[0] + F0[1] * F1[1] + F0[2] * F1[2];
        const T cc = F1[0] * F1[0] + F1[1] * F1[1] + F1[2] * F1[2];
        // principal stretches from the eigenvalues of C = F^T F, kept as s - 1
        const T meanm1 = T(0.5) * ((aa - T(1)) + (cc - T(1)));
        const T dif = T(0.5) * (aa - cc);
        const T rad = sqrt(dif * dif + bb * bb);
        const T m1 = meanm1 + rad, m2 = meanm1 - rad;
        const T s1 = sqrt(T(1) + m1);
        const T q2 = T(1) + m2;
        const T s2 = q2 > T(0) ? sqrt(q2) : T(0);
        T cr[3];
        cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
        cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
        cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
        if (!(s2 > T(1e-6) * s1) || !(s1 < T(1e30))) {
            pl[2] += T(1);
            T row[kTriRow];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                row[c] = row[3 + c] = T(0);
                row[6 + c] = cr[c] * sixth;
            }
            row[9] = row[10] = row[11] = T(0);
            store_corners(tp, TRI, t, tv, row);
            continue;
        }
        const T e1s = m1 / (s1 + T(1)), e2s = m2 / (s2 + T(1));
        // area preservation: distance to SL(2)
        const T tsl = sl2_t(e1s, e2s);
        const T dd1 = e1s - tsl, dd2 = e2s + tsl / (T(1) + tsl);
        // modified Skalak, f(s) = B/8 (s^2 - 1)^2 + D/4 (s - 1)^4, written in e = s - 1
        const T q1 = e1s * (T(2) + e1s), q2b = e2s * (T(2) + e2s);
        const T f1 = T(0.125) * Bs * q1 * q1 + T(0.25) * Ds * e1s * e1s * e1s * e1s;
        const T f2 = T(0.125) * Bs * q2b * q2b + T(0.25) * Ds * e2s * e2s * e2s * e2s;
        const T fp1 = T(0.5) * Bs * (T(1) + e1s) * q1 + Ds * e1s * e1s * e1s;
        const T fp2 = T(0.5) * Bs * (T(1) + e2s) * q2b + Ds * e2s * e2s * e2s;
        ce[0].add(T(0.5) * Cs * Wt * (dd1 * dd1 + dd2 * dd2));
        ce[1].add(Wt * (f1 + f2));
        // dE/dF = F V diag(k) V^T with k_a = W (C (s_a - s*_a) + f'(s_a)) / s_a
        const T k1 = Wt * (Cs * dd1 + fp1) / s1;
        const T k2 = Wt * (Cs * dd2 + fp2) / s2;
        pl[1] += fabs(k1) * s1 * s1 + fabs(k2) * s2 * s2;
        T vx, vy;
        if (rad == T(0)) {
            vx = T(1); vy = T(0);
        } else if (dif >= T(0)) {
            vx = dif + rad; vy = bb;
        } else {
            vx = bb; vy = rad - dif;
        }
        const T inv = T(1) / sqrt(vx * vx + vy * vy);
        vx *= inv;
        vy *= inv;
        const T K00 = k1 * vx * vx + k2 * vy * vy;
        const T K11 = k1 * vy * vy + k2 * vx * vx;
        const T K01 = (k1 - k2) * vx * vy;
        // cross-product change relative to x_n: E1 x d2 + d1 x E2 + d1 x d2
        T dcr[3];
        dcr[0] = (E1[1] * d2[2] - E1[2] * d2[1]) + (d1[1] * E2[2] - d1[2] * E2[1]) + (d1[1] * d2[2] - d1[2] * d2[1]);
        dcr[1] = (E1[2] * d2[0] - E1[0] * d2[2]) + (d1[2] * E2[0] - d1[0] * E2[2]) + (d1[2] * d2[0] - d1[0] * d2[2]);
        dcr[2] = (E1[0] * d2[1] - E1[1] * d2[0]) + (d1[0] * E2[1] - d1[1] * E2[0]) + (d1[0] * d2[1] - d1[1] * d2[0]);
        ce[3].add((Xi[0] * dcr[0] + Xi[1] * dcr[1] + Xi[2] * dcr[2]) + (Ui[0] * cr[0] + Ui[1] * cr[1] + Ui[2] * cr[2]));
        T row[kTriRow];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T G0 = F0[c] * K00 + F1[c] * K01;
            const T G1 = F0[c] * K01 + F1[c] * K11;
            row[c] = G0 * Di0 + G1 * Di1;      // corner j
            row[3 + c] = G0 * Di2 + G1 * Di3;  // corner k (corner i gets minus both)
            row[6 + c] = cr[c] * sixth;        // share of the area-weighted normal / 3
        }
        row[9] = row[10] = row[11] = T(0);
        store_corners(tp, TRI, t, tv, row);
    }
    __syncthreads();

    // ---- pass 2: gather per vertex; bending projection (Eq. BendingDiscretizedPotential)
    for (int i = tid; i < np; i += NT) {
        if (i >= n) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                Gout[c * np + i] = T(0);
                GC[c * np + i] = T(0);
                WR[c * np + i] = T(0);
            }
            continue;
        }
        T g[3] = {T(0), T(0), T(0)}, gc[3] = {T(0), T(0), T(0)};
        int jr[8];
        int val = 0;
        if (tp.k8) {
            // the corner gradients of the vertex's triangles, one slot per ring entry
            ring8_indices(tp.ring8_idx, i, jr);
#pragma unroll
            for (int q = 0; q < 8; ++q) val += jr[q] != i;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (q < val)
#pragma unroll
                    for (int c = 0; c < 3; ++c) g[c] += TRI[(3 * q + c) * np + i];
        } else {
            const int b0 = __ldg(&tp.inc_ptr[i]), b1 = __ldg(&tp.inc_ptr[i + 1]);
            for (int q = b0; q < b1; ++q) {
                const unsigned e = __ldg(&tp.inc_idx[q]);
                const T* P = TRI + kTriRow * (e >> 2);
                const unsigned corner = e & 3u;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const T gj = P[c], gk = P[3 + c];
                    g[c] += corner == 1u ? gj : (corner == 2u ? gk : -(gj + gk));
                    gc[c] += P[6 + c];
                }
            }
        }
        T dfn[3] = {T(0), T(0), T(0)}, dfu[3] = {T(0), T(0), T(0)};
        T Xi[3], Ui[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Xi[c] = XN[c * np + i];
            Ui[c] = U[c * np + i];
        }
        if (tp.k8) {
            // bending: delta_f = sum_q c_q (x_{r_q} - x_i); volume gradient: one sixth of
            // the sum of e_q x e_{q+1} over the incident triangles (e_q = x_{r_q} - x_i)
            T cw[8];
            ldg8(tp.ring8_c + 8 * i, cw);
            T e0[3] = {T(0), T(0), T(0)}, ep[3] = {T(0), T(0), T(0)};
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (q < val) {
                    T ed[3], eu[3], ee[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        ed[c] = XN[c * np + jr[q]] - Xi[c];
                        eu[c] = U[c * np + jr[q]] - Ui[c];
                        dfn[c] += cw[q] * ed[c];
                        dfu[c] += cw[q] * eu[c];
                        ee[c] = ed[c] + eu[c];
                    }
                    if (q == 0) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) e0[c] = ee[c];
                    } else {
                        gc[0] += ep[1] * ee[2] - ep[2] * ee[1];
                        gc[1] += ep[2] * ee[0] - ep[0] * ee[2];
                        gc[2] += ep[0] * ee[1] - ep[1] * ee[0];
                    }
#pragma unroll
                    for (int c = 0; c < 3; ++c) ep[c] = ee[c];
                }
            }
            gc[0] += ep[1] * e0[2] - ep[2] * e0[1];
            gc[1] += ep[2] * e0[0] - ep[0] * e0[2];
            gc[2] += ep[0] * e0[1] - ep[1] * e0[0];
#pragma unroll
            for (int c = 0; c < 3; ++c) gc[c] *= sixth;
        } else {
            const int r0 = __ldg(&tp.ring_ptr[i]), r1 = __ldg(&tp.ring_ptr[i + 1]);
            for (int q = r0; q < r1; ++q) {
                const int jn = __ldg(&tp.ring_idx[q]);
                const T cq = __ldg(&tp.ring_c[q]);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    dfn[c] += cq * (XN[c * np + jn] - Xi[c]);
                    dfu[c] += cq * (U[c * np + jn] - Ui[c]);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Gout[c * np + i] = g[c];
            GC[c * np + i] = gc[c];
        }
        pl[0] += gc[0] * gc[0] + gc[1] * gc[1] + gc[2] * gc[2];
        const T df[3] = {dfn[0] + dfu[0], dfn[1] + dfu[1], dfn[2] + dfu[2]};
        const T nf = sqrt(df[0] * df[0] + df[1] * df[1] + df[2] * df[2]);
        const T ng = __ldg(&tp.dg_norm[i]);
        T r[3];
        if (ng > T(0) && nf > T(1e-12) * ng) {
            const T sc = (nf - ng) / nf;
#pragma unroll
            for (int c = 0; c < 3; ++c) r[c] = df[c] * sc;
        } else if (ng > T(0)) {
            // delta_f ~ 0: the rotation is free; take the current vertex normal
            const T gn = sqrt(gc[0] * gc[0] + gc[1] * gc[1] + gc[2] * gc[2]);
            const T s = gn > T(0) ? __ldg(&tp.nsign[i]) * ng / gn : T(0);
#pragma unroll
            for (int c = 0; c < 3; ++c) r[c] = df[c] - s * gc[c];
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) r[c] = df[c];
        }
        const T w = __ldg(&tp.bend_w[i]);
        const T rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        ce[2].add(T(0.5) * w * rr);
        pl[1] += w * sqrt(rr) * nf;
#pragma unroll
        for (int c = 0; c < 3; ++c) WR[c * np + i] = w * r[c];
    }
    const T kvol = tp.kvol;
    const Pair<T> V0 = {tp.V0hi, tp.V0lo};
    block_reduce_cp<T, 5, 3>(ce, pl, smem, [=](CellShared<T>* s) {
        s->Earea = {s->out[0], s->outlo[0]};
        s->Esk = {s->out[1], s->outlo[1]};
        s->Ebend = {s->out[2], s->outlo[2]};
        const Pair<T> vn = kFirst ? pair_div6(s->out[4], s->outlo[4]) : Vn;
        s->Vn = vn;
        s->V = pair_add(vn, pair_div6(s->out[3], s->outlo[3]));
        const T Cv = pair_diff(s->V, V0);
        const T inv = T(1) / s->out[5];
        s->Evol = T(0.5) * kvol * Cv * Cv * inv;
        s->volc = kvol * Cv * inv;
        s->noise = s->out[6];
        s->bad = s->out[7] != T(0);
    });
    const T volc = sh->volc;

    // ---- pass 3: bending gather, volume and inertia (M~ = (1 + h alpha_D) M + h beta_D L), residual
    const T ms = tp.inertia_scale * tp.inv_h2, h2 = tp.h * tp.h;
    Acc<T> ci[2];            // inertia energy, collision energy
    T pr[1] = {T(0)};        // sum_i (h^2 |grad_i| / m_i)^2
    for (int i = tid; i < n; i += NT) {
        const T m = __ldg(&tp.mass[i]);
        const T hm = h2 * __ldg(&tp.inv_mass[i]);
        const T cs = __ldg(&tp.csum[i]);
        T gb[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) gb[c] = -cs * WR[c * np + i];
        if (tp.k8) {
            int jr[8];
            T cw[8];
            ring8_indices(tp.ring8_idx, i, jr);
            ldg8(tp.ring8_ct + 8 * i, cw);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (jr[q] == i) continue;  // padding
#pragma unroll
                for (int c = 0; c < 3; ++c) gb[c] += cw[q] * WR[c * np + jr[q]];
            }
        } else {
            const int r0 = __ldg(&tp.ring_ptr[i]), r1 = __ldg(&tp.ring_ptr[i + 1]);
            for (int q = r0; q < r1; ++q) {
                const int jn = __ldg(&tp.ring_idx[q]);
                const T ct = __ldg(&tp.ring_ct[q]);
#pragma unroll
                for (int c = 0; c < 3; ++c) gb[c] += ct * WR[c * np + jn];
            }
        }
        // beta_D > 0: M~/h^2 (x - y) gains (beta_D / h) L (x - y)
        T lb[3] = {T(0), T(0), T(0)};
        if (tp.l_ptr) {
            const int b0 = __ldg(&tp.l_ptr[i]), b1 = __ldg(&tp.l_ptr[i + 1]);
            for (int q = b0; q < b1; ++q) {
                const int j = __ldg(&tp.l_idx[q]);
                const T lv = __ldg(&tp.l_val[q]);
#pragma unroll
                for (int c = 0; c < 3; ++c) lb[c] += lv * (U[c * np + j] - UY[c * np + j]);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) lb[c] *= tp.beta_h;
        }
        // collision (Sec. 3.3): while the vertex lies behind its neighbour's tangent plane
        // (d > 0), (w_col/2) d^2 with gradient -w_col d n; re-tested at every evaluation
        T gcol[3] = {T(0), T(0), T(0)};
        if (colp) {
            const float4 pl = colp[i];
            if (pl.x != 0.f || pl.y != 0.f || pl.z != 0.f) {
                const T d = T(pl.w) - (T(pl.x) * (XN[i] + U[i]) + T(pl.y) * (XN[np + i] + U[np + i]) +
                                       T(pl.z) * (XN[2 * np + i] + U[2 * np + i]));
                if (d > T(0)) {
                    const T wd = wcol * d;
                    gcol[0] = -wd * T(pl.x);
                    gcol[1] = -wd * T(pl.y);
                    gcol[2] = -wd * T(pl.z);
                    ci[1].add(T(0.5) * wd * d);
                }
            }
        }
        T g2 = T(0), ei = T(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T du = U[c * np + i] - UY[c * np + i];
            const T gv = Gout[c * np + i] + gb[c] + volc * GC[c * np + i] + m * ms * du + lb[c] + gcol[c];
            Gout[c * np + i] = gv;
            ei += T(0.5) * (m * ms * du + lb[c]) * du;
            g2 += gv * gv;
        }
        ci[0].add(ei);
        pr[0] += hm * hm * g2;
    }
    const T inv_n = T(1) / T(n), inv_lbar = tp.inv_lbar;
    const T uT = T(Unit<T>::u);
    block_reduce_cp<T, 2, 1>(ci, pr, smem, [=](CellShared<T>* s) {
        s->Ein = {s->out[0], s->outlo[0]};
        s->E = pair_add(pair_add(pair_add(pair_add(pair_add(s->Ein, s->Earea), s->Esk), s->Ebend), s->Evol),
                        Pair<T>{s->out[1], s->outlo[1]});
        const T res = sqrt(s->out[2] * inv_n) * inv_lbar;
        s->res = res;
        s->noise = T(4) * uT * (s->noise + T(2) * s->Ein.hi);
        // non-finite energy or residual marks the evaluation bad
        if (!isfinite(s->E.hi) || !isfinite(res)) s->bad = 1;
    });
}

// R = A Q for the three coordinate rows, A = A^-1 of the topology unless another
// symmetric matrix of the same padded layout is given (M~^-1 for the first guess).
// FP32: a warp owns a tile of 128 rows (4 consecutive rows per lane, float4 loads of
// the symmetric A^-1 by columns, coalesced) and a share of the j range; Q is
// broadcast from shared memory.  The warps' partial sums go to `scratch` (the
// triangle buffer, idle outside the objective evaluation) and are added in a fixed
// order, so the result is deterministic.
template <typename T>
__device__ void contract_simt(const TopoDev<T>& tp, const T* Q, T* R, T* scratch, const T* Amat = nullptr,
                              int scratch_floats = 0)
{
    const int n = tp.n, np = tp.n_pad, N3 = 3 * np;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const T* __restrict__ A = Amat ? Amat : tp.ainv;
    if constexpr (sizeof(T) == 4) {
        if (!Amat && tp.ainv_b16) {
            // BF16 A^-1 (a BF16 handle), FP32 accumulation: 256-row tiles, each lane 8
            // consecutive rows of a column in one 16-byte load; the same balanced split of
            // the columns into parts as below, bounded by the scratch's size
            const unsigned short* __restrict__ Ab = static_cast<const unsigned short*>(tp.ainv_b16);
            const int n8 = tp.n8;
            const int ntile = (n + 255) >> 8;
            const int cap = scratch_floats > 0 ? scratch_floats / 768 : max(32, 4 * ((n + 127) >> 7)) / 2;
            const int pmax = max(1, min(cap / ntile, n / 4));
            int P = 1;
            long long best = -1;
            for (int q = 1; q <= pmax; ++q) {
                const long long cost = (long long)((ntile * q + nw - 1) / nw) * ((((n + q - 1) / q) + 3) & ~3);
                if (best < 0 || cost < best) {
                    best = cost;
                    P = q;
                }
            }
            const int chunk = (((n + P - 1) / P) + 3) & ~3;
            const int nitems = ntile * P;
            for (int item = warp; item < nitems; item += nw) {
                const int tile = item % ntile, part = item / ntile;
                const int j0 = part * chunk, j1 = min(n, j0 + chunk);
                const int row0 = tile * 256 + 8 * lane;
                float acc[3][8];
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int r = 0; r < 8; ++r) acc[c][r] = 0.f;
                if (row0 < n) {
                    int j = j0;
                    for (; j + 4 <= j1; j += 4) {
                        uint4 av[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            av[u] = __ldg(reinterpret_cast<const uint4*>(Ab + (size_t)(j + u) * n8 + row0));
                        const float4 x0 = *reinterpret_cast<const float4*>(Q + j);
                        const float4 x1 = *reinterpret_cast<const float4*>(Q + np + j);
                        const float4 x2 = *reinterpret_cast<const float4*>(Q + 2 * np + j);
                        const float q0[4] = {x0.x, x0.y, x0.z, x0.w}, q1[4] = {x1.x, x1.y, x1.z, x1.w},
                                    q2[4] = {x2.x, x2.y, x2.z, x2.w};
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const unsigned w[4] = {av[u].x, av[u].y, av[u].z, av[u].w};
#pragma unroll
                            for (int r = 0; r < 8; ++r) {
                                // BF16 to FP32: the 16 bits are the float's high half
                                const float a = __uint_as_float((r & 1) ? (w[r >> 1] & 0xffff0000u) : (w[r >> 1] << 16));
                                acc[0][r] += a * q0[u];
                                acc[1][r] += a * q1[u];
                                acc[2][r] += a * q2[u];
                            }
                        }
                    }
                    for (; j < j1; ++j) {
                        const uint4 a4 = __ldg(reinterpret_cast<const uint4*>(Ab + (size_t)j * n8 + row0));
                        const unsigned w[4] = {a4.x, a4.y, a4.z, a4.w};
                        const float qq[3] = {Q[j], Q[np + j], Q[2 * np + j]};
#pragma unroll
                        for (int r = 0; r < 8; ++r) {
                            const float a = __uint_as_float((r & 1) ? (w[r >> 1] & 0xffff0000u) : (w[r >> 1] << 16));
#pragma unroll
                            for (int c = 0; c < 3; ++c) acc[c][r] += a * qq[c];
                        }
                    }
                }
                float* Pp = reinterpret_cast<float*>(scratch) + item * 768;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    *reinterpret_cast<float4*>(Pp + c * 256 + 8 * lane) =
                        make_float4(acc[c][0], acc[c][1], acc[c][2], acc[c][3]);
                    *reinterpret_cast<float4*>(Pp + c * 256 + 8 * lane + 4) =
                        make_float4(acc[c][4], acc[c][5], acc[c][6], acc[c][7]);
                }
            }
            __syncthreads();
            const float* Sb = reinterpret_cast<const float*>(scratch);
            for (int e = threadIdx.x; e < N3; e += blockDim.x) {
                const int c = e / np, row = e - c * np;
                float sum = 0.f;
                if (row < n) {
                    const int tl = row >> 8, rr = row & 255;
                    for (int it = tl; it < nitems; it += ntile) sum += Sb[it * 768 + c * 256 + rr];
                }
                R[e] = sum;
            }
            __syncthreads();
            return;
        }
        const int ntile = (n + 127) >> 7;
        // every tile's j range in P equal parts, items (tile, part) dealt to the warps in
        // turn; P minimises the busiest warp's columns (ceil(ntile P / nw) items of
        // ceil(n / P) columns) within the scratch's max(32, 4 ntile) items of 384 floats.
        // Partials go to scratch[item][c][128].
        const int pmax = max(1, min(max(32, 4 * ntile) / ntile, n / 4));
        int P = 1;
        long long best = -1;
        for (int q = 1; q <= pmax; ++q) {
            const long long cost = (long long)((ntile * q + nw - 1) / nw) * ((((n + q - 1) / q) + 3) & ~3);
            if (best < 0 || cost < best) {
                best = cost;
                P = q;
            }
        }
        const int chunk = (((n + P - 1) / P) + 3) & ~3;
        const int nitems = ntile * P;
        for (int item = warp; item < nitems; item += nw) {
            const int tile = item % ntile, part = item / ntile;
            const int j0 = part * chunk, j1 = min(n, j0 + chunk);
            const int row0 = tile * 128 + 4 * lane;
            float acc[3][4];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int r = 0; r < 4; ++r) acc[c][r] = 0.f;
            if (row0 < n) {
                int j = j0;
                // eight columns at a time: 4 KB of A^-1 in flight per warp
                for (; j + 8 <= j1; j += 8) {
                    float4 av[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        av[u] = __ldg(reinterpret_cast<const float4*>(A + (size_t)(j + u) * np + row0));
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float4 x0 = *reinterpret_cast<const float4*>(Q + j + 4 * h);
                        const float4 x1 = *reinterpret_cast<const float4*>(Q + np + j + 4 * h);
                        const float4 x2 = *reinterpret_cast<const float4*>(Q + 2 * np + j + 4 * h);
                        const float q0[4] = {x0.x, x0.y, x0.z, x0.w}, q1[4] = {x1.x, x1.y, x1.z, x1.w},
                                    q2[4] = {x2.x, x2.y, x2.z, x2.w};
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const float a4[4] = {av[4 * h + u].x, av[4 * h + u].y, av[4 * h + u].z, av[4 * h + u].w};
#pragma unroll
                            for (int r = 0; r < 4; ++r) {
                                acc[0][r] += a4[r] * q0[u];
                                acc[1][r] += a4[r] * q1[u];
                                acc[2][r] += a4[r] * q2[u];
                            }
                        }
                    }
                }
                for (; j + 4 <= j1; j += 4) {
                    float4 av[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        av[u] = __ldg(reinterpret_cast<const float4*>(A + (size_t)(j + u) * np + row0));
                    const float4 x0 = *reinterpret_cast<const float4*>(Q + j);
                    const float4 x1 = *reinterpret_cast<const float4*>(Q + np + j);
                    const float4 x2 = *reinterpret_cast<const float4*>(Q + 2 * np + j);
                    const float q0[4] = {x0.x, x0.y, x0.z, x0.w}, q1[4] = {x1.x, x1.y, x1.z, x1.w},
                                q2[4] = {x2.x, x2.y, x2.z, x2.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float a4[4] = {av[u].x, av[u].y, av[u].z, av[u].w};
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            acc[0][r] += a4[r] * q0[u];
                            acc[1][r] += a4[r] * q1[u];
                            acc[2][r] += a4[r] * q2[u];
                        }
                    }
                }
                for (; j < j1; ++j) {
                    const float4 a = __ldg(reinterpret_cast<const float4*>(A + (size_t)j * np + row0));
                    const float a4[4] = {a.x, a.y, a.z, a.w};
                    const float qq[3] = {Q[j], Q[np + j], Q[2 * np + j]};
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int c = 0; c < 3; ++c) acc[c][r] += a4[r] * qq[c];
                }
            }
            float* P = reinterpret_cast<float*>(scratch) + item * 384;
#pragma unroll
            for (int c = 0; c < 3; ++c)
                *reinterpret_cast<float4*>(P + c * 128 + 4 * lane) =
                    make_float4(acc[c][0], acc[c][1], acc[c][2], acc[c][3]);
        }
        __syncthreads();
        const float* S = reinterpret_cast<const float*>(scratch);
        for (int e = threadIdx.x; e < N3; e += blockDim.x) {
            const int c = e / np, row = e - c * np;
            float s = 0.f;
            if (row < n) {
                const int tl = row >> 7, rr = row & 127;
                for (int it = tl; it < nitems; it += ntile) s += S[it * 384 + c * 128 + rr];
            }
            R[e] = s;
        }
        __syncthreads();
    } else {
        for (int e = threadIdx.x; e < N3; e += blockDim.x) R[e] = T(0);
        __syncthreads();
        const int ntile = (n + 31) >> 5;
        for (int item = warp; item < ntile; item += nw) {
            const int row = item * 32 + lane;
            if (row < n) {
                T a0 = T(0), a1 = T(0), a2 = T(0);
                for (int j = 0; j < n; ++j) {
                    const T av = __ldg(&A[(size_t)j * np + row]);
                    a0 += av * Q[j];
                    a1 += av * Q[np + j];
                    a2 += av * Q[2 * np + j];
                }
                R[row] = a0;
                R[np + row] = a1;
                R[2 * np + row] = a2;
            }
        }
        __syncthreads();
    }
}

namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t cta_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t map_rank(uint32_t local, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}

__device__ __forceinline__ void st_remote_v4(uint32_t addr, uint4 v)
{
    asm volatile("st.shared::cluster.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w)
                 : "memory");
}

__device__ __forceinline__ void st_remote_f32(uint32_t addr, float v)
{
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

__device__ __forceinline__ void st_remote_u32(uint32_t addr, uint32_t v)
{
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const unsigned short l = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const unsigned short h = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return ((uint32_t)h << 16) | l;
}

// byte offset of B element (row nrow, column k) in the no-swizzle K-major layout:
// 8 x 8 core matrices of 128 bytes, K-adjacent core matrices 128 bytes apart
// (leading byte offset), row groups (Kpad / 8) * 128 bytes apart (stride byte offset)
__device__ __forceinline__ uint32_t b_offset(int nrow, int k, int kpad)
{
    return (uint32_t)(((nrow >> 3) * (kpad >> 3) + (k >> 3)) * 128 + (nrow & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of tcgen05; no swizzle, base offset 0
    return d;
}

template <int NCOL>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[NCOL])
{
    uint32_t r[NCOL];
    if constexpr (NCOL == 32) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
            "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
    } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < NCOL; ++j) v[j] = __uint_as_float(r[j]);
}

}  // namespace tc

// ---------------------------------------------------------------------------------
// TF32 tensor-core contraction inside the persistent SIMT kernel (NPFEM_PREC_TF32).
// A TF32 row block of A^-1 (128 rows x K, one 32-bit tensor-memory column per K
// element) does not fit the 512 tensor-memory columns for K = 656, so A^-1 is not kept
// resident as in the BF16 cluster kernel: every block streams it from L2 in chunks of
// 128 rows x 32 K (16 KB, laid out in global memory as the MMA's no-swizzle K-major
// core matrices, one cp.async.bulk each) through a two-stage shared-memory ring, and
// one thread issues tcgen05.mma.kind::tf32 (M 128, N 16, K 8) per 8 K into tensor
// memory (16 FP32 columns per row tile).  B is q in TF32: one 8-row group of core
// matrices (rows 0-2 the three coordinates, rows 3-7 zero) read for both row groups of
// N = 16 (stride byte offset 0), so columns 8-15 repeat 0-7 and are not read.
// Blocks work independently: no cluster, no rounds.
// ---------------------------------------------------------------------------------
namespace tf32 {

constexpr int kChunkK = 32;
constexpr int kChunkBytes = 128 * kChunkK * 4;
constexpr unsigned kWaitLimit = 1u << 22;

__device__ __forceinline__ float round_tf32(float v)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

__device__ __forceinline__ bool wait_parity(unsigned long long* bar, uint32_t parity)
{
    uint32_t done = 0;
    for (unsigned it = 0; it < kWaitLimit && !done; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(tc::smem_addr(bar)), "r"(parity));
    }
    return done != 0;
}

// Copies chunk q of the tiled A^-1 into ring stage q & 1.
__device__ __forceinline__ void load_chunk(const unsigned char* gsrc, unsigned char* stage, unsigned long long* full)
{
    const uint32_t bar = tc::smem_addr(full);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"((uint32_t)kChunkBytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tc::smem_addr(stage)),
                 "l"(gsrc), "r"((uint32_t)kChunkBytes), "r"(bar)
                 : "memory");
}

// Set-up at kernel start (all threads): barriers, zero B operand, tensor memory.
__device__ void setup(int kpad, unsigned char* tcs, CellShared<float>* sh, uint32_t ncols)
{
    const int tid = threadIdx.x;
    unsigned char* bops = tcs + 2 * kChunkBytes;
    for (int q = tid; q < kpad * 8; q += blockDim.x) reinterpret_cast<float*>(bops)[q] = 0.f;
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_addr(&sh->tfull[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_addr(&sh->tfree[s])));
            sh->tuse[s] = 0u;
        }
        sh->tfail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((tid >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_addr(&sh->taddr)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ void teardown(CellShared<float>* sh, uint32_t ncols)
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sh->taddr), "r"(ncols));
}

// R = A^-1 Q (three rows of n_pad) with A^-1 in TF32, FP32 accumulation.
__device__ void contract(const TopoDev<float>& tp, const float* Q, float* R, unsigned char* tcs, CellShared<float>* sh,
                         unsigned int* err)
{
    const int n = tp.n, np = tp.n_pad, kpad = tp.kpad, tid = threadIdx.x, NT = blockDim.x;
    const int nch = kpad / kChunkK, tiles = tp.rb, total = tiles * nch;
    unsigned char* bops = tcs + 2 * kChunkBytes;
    // q in TF32 as B: element (row c, k) of the single row group of core matrices
    for (int e = tid; e < 3 * kpad; e += NT) {
        const int c = e / kpad, k = e - c * kpad;
        const float v = k < n ? Q[c * np + k] : 0.f;
        *reinterpret_cast<float*>(bops + (k >> 2) * 128 + c * 16 + (k & 3) * 4) = round_tf32(v);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    const uint32_t tbase = sh->taddr;
    if (tid == 0 && !sh->tfail) {
        const unsigned char* gA = static_cast<const unsigned char*>(tp.ainv_lp);
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
        const uint32_t sbase = tc::smem_addr(tcs), bbase = tc::smem_addr(bops);
        uint32_t use[2] = {sh->tuse[0], sh->tuse[1]};
        bool ok = true;
        load_chunk(gA, tcs, &sh->tfull[0]);
        if (total > 1) load_chunk(gA + kChunkBytes, tcs + kChunkBytes, &sh->tfull[1]);
        for (int q = 0; q < total && ok; ++q) {
            const int s = q & 1, t = q / nch, c = q - t * nch;
            const uint32_t u = use[s] + (uint32_t)(q >> 1);
            ok = wait_parity(&sh->tfull[s], u & 1u);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int ks = 0; ks < kChunkK / 8; ++ks) {
                const uint64_t ad = tc::smem_desc(sbase + (uint32_t)(s * kChunkBytes + ks * 256), 128u, 1024u);
                const uint64_t bd = tc::smem_desc(bbase + (uint32_t)((c * (kChunkK / 8) + ks) * 256), 128u, 0u);
                const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tbase + (uint32_t)(16 * t)),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                tc::smem_addr(&sh->tfree[s])));
            if (q + 2 < total) {
                // the stage is refilled once its MMAs have read it
                ok = wait_parity(&sh->tfree[s], u & 1u);
                if (ok) load_chunk(gA + (size_t)(q + 2) * kChunkBytes, tcs + s * kChunkBytes, &sh->tfull[s]);
            }
        }
        // the last use of each stage: its MMAs complete in order, after every earlier one
        for (int q = total - 2; q < total && ok; ++q) {
            if (q < 0) continue;
            const int s = q & 1;
            ok = wait_parity(&sh->tfree[s], (use[s] + (uint32_t)(q >> 1)) & 1u);
        }
        sh->tuse[0] = use[0] + (uint32_t)((total + 1) / 2);
        sh->tuse[1] = use[1] + (uint32_t)(total / 2);
        if (!ok) {
            sh->tfail = 1;
            atomicExch(err, 1u);  // reported to the host; results invalid
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // D: warp w reads the lanes of its quadrant (w % 4) of row tiles w / 4, w / 4 + NW / 4, ...
    const int warp = tid >> 5, lane = tid & 31, nwq = (NT >> 5) >> 2;
    if ((warp >> 2) < nwq) {
        const int quad = warp & 3;
        for (int t = warp >> 2; t < tiles; t += nwq) {
            float dv[16];
            tc::tmem_ld<16>(tbase + ((uint32_t)(32 * quad) << 16) + (uint32_t)(16 * t), dv);
            const int row = 128 * t + 32 * quad + lane;
            if (row < np) {
                const bool live = row < n && !sh->tfail;
#pragma unroll
                for (int c = 0; c < 3; ++c) R[c * np + row] = live ? dv[c] : 0.f;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
}

}  // namespace tf32

// Refinement residual e = q - H~ r (H~ = ms M + (1 + beta_D/h) L, L sparse FP32), one row
// (three components) per thread, into tmp (3 x n_pad; zero padding).
template <typename T>
__device__ void refine_residual(const TopoDev<T>& tp, const T* src, const T* R, T* tmp)
{
    const int n = tp.n, np = tp.n_pad, tid = threadIdx.x, NT = blockDim.x;
    const T ms = tp.inertia_scale * tp.inv_h2;
    for (int i = tid; i < np; i += NT) {
        T e0 = T(0), e1 = T(0), e2 = T(0);
        if (i < n) {
            const T mm = ms * __ldg(&tp.mass[i]);
            T h0 = mm * R[i], h1 = mm * R[np + i], h2 = mm * R[2 * np + i];
            const int b0 = __ldg(&tp.h_ptr[i]), b1 = __ldg(&tp.h_ptr[i + 1]);
            for (int p = b0; p < b1; ++p) {
                const T lv = __ldg(&tp.h_val[p]);
                const int j = __ldg(&tp.h_idx[p]);
                h0 += lv * R[j];
                h1 += lv * R[np + j];
                h2 += lv * R[2 * np + j];
            }
            e0 = src[i] - h0;
            e1 = src[np + i] - h1;
            e2 = src[2 * np + i] - h2;
        }
        tmp[i] = e0;
        tmp[np + i] = e1;
        tmp[2 * np + i] = e2;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------------
// One cell's quasi-Newton solve, split into the phases that both kernels drive.
// All threads of the block call every method (control flow is block-uniform).
// ---------------------------------------------------------------------------------
template <typename T>
struct CellSolver {
    const LaunchArgs<T>* a;
    const GroupDesc<T>* gd;
    unsigned char* smem;
    char* slot;
    CellShared<T>* sh;
    T *XN, *u, *ut, *g, *gt, *GCv, *UYv, *Dv, *TRIv, *WRv;
    long long so, item;
    int M, head, count, iters, evals, status;
    Pair<T> E, Vlast, Vn;
    T noiseE, res, gdv;
    bool nonfinite;
    const float4* colp;  // this cell's collision planes, or null
    T wcol;
    // carried L-BFGS pairs: this cell's record (or null); carry_valid: the record holds
    // the pairs of the cell's last solve; carry_in: not yet loaded in this step
    T* crec;
    bool carry_valid, carry_in;
    bool carry_early;  // begin issued the carried pairs' copies (load_pairs only waits)
    unsigned dirty;    // ring slots written by this solve (the others match the record)
    T ccount;  // the record's pair count, read in begin (its latency hidden by the evaluation)
    T clast;   // the record's iteration count of the cell's last step
    // history vectors that do not fit in shared memory live in the record (they may be
    // carried to the next step) rather than in the block's slot, unless the record's
    // pairs are not to be carried (the last solve took more than kCarryMaxIters
    // iterations); evaluated where used, after the header has arrived
    __device__ bool ring_in_record() const
    {
        return crec && M > 0 && (!carry_valid || clast <= T(kCarryMaxIters));
    }

    __device__ const TopoDev<T>& tp() const { return gd->topo; }
    // A solver vector; with carried pairs, a history vector that does not fit in shared
    // memory lives in the cell's record (ring slot order, see load_pairs), not in the
    // block's global slot, so that the pairs persist without a copy.
    __device__ T* hist(int v) const
    {
        if (ring_in_record() && v >= V_SBASE && gd->loc[v] < 0)
            return crec + carry_head_elems(M) + (long long)(v - V_SBASE) * 3 * tp().n_pad;
        return vec_ptr(*gd, smem, slot, v);
    }

    __device__ void bind(const LaunchArgs<T>& la, const GroupDesc<T>& g_, unsigned char* sm)
    {
        a = &la;
        gd = &g_;
        smem = sm;
        sh = cell_shared<T>(sm);
        slot = la.scratch ? la.scratch + (long long)blockIdx.x * la.slot_bytes : nullptr;
        XN = vec_ptr(g_, sm, slot, V_XN);
        u = vec_ptr(g_, sm, slot, V_U);
        ut = vec_ptr(g_, sm, slot, V_UT);
        g = vec_ptr(g_, sm, slot, V_G);
        gt = vec_ptr(g_, sm, slot, V_GT);
        GCv = vec_ptr(g_, sm, slot, V_GC);
        UYv = vec_ptr(g_, sm, slot, V_UY);
        Dv = vec_ptr(g_, sm, slot, V_D);
        TRIv = vec_ptr(g_, sm, slot, V_TRI);
        WRv = vec_ptr(g_, sm, slot, V_WR);
        M = la.p.lbfgs_m;
    }

    // Load the cell (local coordinates around vertex 0), first guess, V(x_n), g and
    // grad g at x^(1).  In evaluation mode writes the gradient and parts and returns
    // false.
    __device__ bool begin(long long cell, long long it)
    {
        const TopoDev<T>& T_ = tp();
        const int n = T_.n, np = T_.n_pad, N3 = 3 * np, tid = threadIdx.x, NT = blockDim.x;
        item = it;
        so = gd->state_off + cell * 3LL * n;
        colp = a->col ? a->col + so / 3 : nullptr;
        wcol = a->col_w;
        const T h = T_.h, inv_ms = T(1) / T_.inertia_scale;
        const bool eval_mode = a->p.mode == 1;
        const bool hist = !eval_mode && a->hist_in;
        crec = (!eval_mode && a->carry) ? a->carry + gd->carry_off + cell * gd->carry_rec : nullptr;
        carry_valid = crec && hist;
        carry_in = carry_valid && M > 0;
        // global words read here come back while the loads below are issued (nothing is
        // stored in between): the record's header, the listed-cell count, vertex 0
        ccount = carry_in ? crec[0] : T(0);
        clast = carry_in ? crec[2] : T(0);
        const unsigned only_prev = a->only ? a->only[2] : 0u;
        const T* x = a->x + so;
        // compensated positions: x_n = x + residue while x holds exactly the value the
        // last step stored (each coordinate checked), else x alone
        const T* XLO = hist && a->pos_stride > 0 ? a->hist_in + a->pos_stride + so : nullptr;
        const T* XHI = XLO ? XLO + a->pos_stride : nullptr;
        const T o0 = x[0], o1 = x[n], o2 = x[2 * n];
        T l0 = T(0), l1 = T(0), l2 = T(0);
        if (XLO) {
            const T h0 = XHI[0], h1 = XHI[n], h2 = XHI[2 * n];
            const T r0 = XLO[0], r1 = XLO[n], r2 = XLO[2 * n];
            l0 = h0 == o0 ? r0 : T(0);
            l1 = h1 == o1 ? r1 : T(0);
            l2 = h2 == o2 ? r2 : T(0);
        }
        carry_early = carry_in && !a->defer;
        if (carry_early) {
            // the cell will most likely ask for a direction: its carried pairs travel while
            // the first evaluation runs (the record into L2; the ring slots held in shared
            // memory and the inner products by asynchronous copies, whatever the record's
            // count; load_pairs waits for them)
            if (threadIdx.x == 0)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(crec),
                             "r"((uint32_t)(gd->carry_rec * (long long)sizeof(T)))
                             : "memory");
            issue_pair_copies();
        }
        // temporal warm start: u = u_y + (x_n - y_{n-1}), the cell's previous correction,
        // folded into this pass (except with a temporal network or beta_D > 0)
        const T* Hc = (hist && !(a->hist_ext && a->u0) && !T_.minv) ? a->hist_in + so : nullptr;
        // U elements per thread at a time, every global load issued before the stores
        // (the stores to shared memory would otherwise hold up the next element's loads)
        constexpr int U = 4;
        for (int e0 = tid; e0 < N3; e0 += U * NT) {
            T xv[U], hv[U], lv[U], vv[U], fv[U], cv[U], mv[U];
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int e = e0 + q * NT, c = e / np, i = e - c * np;
                xv[q] = hv[q] = lv[q] = vv[q] = fv[q] = cv[q] = mv[q] = T(0);
                if (e < N3 && i < n) {
                    const int gi = c * n + i;
                    xv[q] = x[gi];
                    mv[q] = T_.minv ? __ldg(&T_.mass[i]) : __ldg(&T_.inv_mass[i]);
                    if (XLO) {
                        hv[q] = XHI[gi];
                        lv[q] = XLO[gi];
                    }
                    if (eval_mode) {
                        vv[q] = a->y[so + gi];
                    } else {
                        vv[q] = a->v[so + gi];
                        fv[q] = a->f[so + gi];
                    }
                    if (Hc) cv[q] = Hc[gi];
                }
            }
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int e = e0 + q * NT, c = e / np, i = e - c * np;
                if (e >= N3) continue;
                T xn = T(0), uy = T(0);
                if (i < n) {
                    xn = xv[q] - (c == 0 ? o0 : (c == 1 ? o1 : o2));
                    if (XLO) xn += (hv[q] == xv[q] ? lv[q] : T(0)) - (c == 0 ? l0 : (c == 1 ? l1 : l2));
                    if (eval_mode) {
                        uy = vv[q] - xv[q];
                    } else if (T_.minv) {
                        // right-hand side h M v_n + h^2 F_ext of M~ (y - x_n), solved below
                        ut[e] = h * mv[q] * vv[q] + h * h * fv[q];
                    } else {
                        uy = (h * vv[q] + h * h * fv[q] * mv[q]) * inv_ms;
                    }
                } else if (T_.minv && !eval_mode) {
                    ut[e] = T(0);
                }
                XN[e] = xn;
                UYv[e] = uy;
                u[e] = eval_mode ? T(0) : uy + cv[q];
            }
        }
        __syncthreads();
        if (T_.minv && !eval_mode) {
            // beta_D > 0: y - x_n = M~^-1 (h M v_n + h^2 F_ext) (Eq. preOptimizationNewton)
            contract_simt(T_, ut, UYv, TRIv, T_.minv);
            for (int e = tid; e < N3; e += NT) u[e] = UYv[e];
            __syncthreads();
        }
        // learned warm start: u = u_y + R MLP(features at y)
        // temporal warm start: u = u_y + (x_n - y_{n-1}) of this cell's previous step
        const int ws = (!eval_mode && !hist && T_.mlp) ? T_.ws_mode : 0;
        if (hist && a->hist_ext && a->u0) {
            // temporal network: u = u_y + c_{n-1} + R MLP(features), computed before the launch
            const T* U0 = a->u0 + so;
            for (int e = tid; e < N3; e += NT) {
                const int c = e / np, i = e - c * np;
                u[e] = i < n ? U0[c * n + i] : T(0);
            }
            __syncthreads();
        } else if (hist && !Hc) {
            // beta_D > 0: the correction on top of the dense first guess
            const T* Hp = a->hist_in + so;
            for (int e = tid; e < N3; e += NT) {
                const int c = e / np, i = e - c * np;
                u[e] = i < n ? UYv[e] + Hp[c * n + i] : T(0);
            }
            __syncthreads();
        } else if (hist) {
            // applied above
        } else if (ws && a->u0) {
            const T* U0 = a->u0 + so;
            for (int e = tid; e < N3; e += NT) {
                const int c = e / np, i = e - c * np;
                u[e] = i < n ? U0[c * n + i] : T(0);
            }
            __syncthreads();
        } else if (ws) {
            for (int e = tid; e < N3; e += NT) ut[e] = XN[e] + UYv[e];
            __syncthreads();
            ws_frame(T_, ut, WRv, smem);
            T R[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) R[q] = sh->post[q];
            const T* F = a->f + so;
            const float* P = T_.mlp;
            // normalised features of every vertex (one thread each) into the idle
            // triangle buffer, rows of 16 floats (9 used), zero rows up to a multiple of 16
            float* Xs = reinterpret_cast<float*>(TRIv);
            const int n16 = (n + 15) & ~15;
            for (int i = tid; i < n16; i += NT) {
                float ft[kMlpIn];
                if (i < n) ws_vertex_features(T_, WRv, F, i, R, ft);
                float4* row = reinterpret_cast<float4*>(Xs + 16 * i);
                float xv[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) xv[k] = (k < kMlpIn && i < n) ? (ft[k] - P[kPMu + k]) / P[kPSig + k] : 0.f;
#pragma unroll
                for (int q = 0; q < 4; ++q) row[q] = make_float4(xv[4 * q], xv[4 * q + 1], xv[4 * q + 2], xv[4 * q + 3]);
            }
            __syncthreads();
            // the network on 16-vertex tiles, one warp per tile
            const int lane = tid & 31;
            for (int tile = tid >> 5; tile * 16 < n; tile += NT >> 5) {
                float olo[3], ohi[3];
                mlp_warp16(P, Xs + 256 * tile, olo, ohi);
                if ((lane & 3) == 0) {
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        const int i = tile * 16 + (lane >> 2) + 8 * r;
                        if (i >= n) continue;
                        const float* o = r ? ohi : olo;
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            u[c * np + i] = UYv[c * np + i] + (R[3 * c] * (T)o[0] + R[3 * c + 1] * (T)o[1] + R[3 * c + 2] * (T)o[2]);
                    }
                }
            }
            __syncthreads();
        }
        // a listed cell was evaluated once by the first-iterate pass when that pass evaluated
        evals = a->only && 2ll * (long long)only_prev <= a->total_cells ? 2 : 1;
        if (ws == 2) {
            // keep the learned guess only if it lowers g: evaluate at y (trial buffers) first
            for (int e = tid; e < N3; e += NT) ut[e] = UYv[e];
            __syncthreads();
            evaluate<T, true>(T_, XN, ut, UYv, gt, GCv, TRIv, WRv, Pair<T>{T(0), T(0)}, smem, colp, wcol);
            Vn = sh->Vn;
            const Pair<T> Ey = sh->E, Vy = sh->V;
            const T ny = sh->noise, ry = sh->res;
            const bool by = sh->bad;
            evaluate<T, false>(T_, XN, u, UYv, g, GCv, TRIv, WRv, Vn, smem, colp, wcol);
            evals = 2;
            if (!(pair_diff(sh->E, Ey) <= T(0)) && !by) {
                T* t1 = u; u = ut; ut = t1;
                T* t2 = g; g = gt; gt = t2;
                if (tid == 0) {
                    sh->E = Ey;
                    sh->noise = ny;
                    sh->res = ry;
                    sh->V = Vy;
                    sh->bad = 0;
                }
                __syncthreads();
            }
        } else {
            evaluate<T, true>(T_, XN, u, UYv, g, GCv, TRIv, WRv, Pair<T>{T(0), T(0)}, smem, colp, wcol);
            Vn = sh->Vn;
        }
        iters = 0;
        status = NPFEM_CELL_OK;
        head = 0;
        count = 0;
        dirty = 0u;
        if (eval_mode) {
            for (int e = tid; e < 3 * n; e += NT) {
                const int c = e / n, i = e - c * n;
                a->grad_out[so + e] = g[c * np + i];
            }
            if (tid == 0) {
                double* P = a->parts + 8 * item;
                P[0] = pair_f64(sh->Ein); P[1] = pair_f64(sh->Earea); P[2] = pair_f64(sh->Esk);
                P[3] = pair_f64(sh->Ebend); P[4] = (double)sh->Evol;
                P[5] = pair_f64(sh->V); P[6] = pair_f64(sh->E); P[7] = (double)sh->res;
            }
            __syncthreads();
            return false;
        }
        E = sh->E;
        noiseE = sh->noise;
        res = sh->res;
        Vlast = sh->V;
        nonfinite = sh->bad != 0;
        return true;
    }

    // Residual test and iteration cap; false when the cell is finished.
    __device__ bool wants_direction()
    {
        if (nonfinite) return false;
        if (res <= prm<T>(a->p.tol, a->p.tolf)) return false;
        if (iters >= a->p.max_iter) {
            status = NPFEM_CELL_MAXITER;
            return false;
        }
        return true;
    }

    // History slot of the q-th newest pair.
    __device__ int hslot(int q) const { return (head - 1 - q + M) % M; }

    // Pairs carried from the cell's last solve.  The record keeps the history ring as it
    // was: [0] pair count, [1] ring head, [2] the iterations of that solve, from [4]
    // s_i^T y_j by ring slot (m x m), then the s vectors of ring slots 0..m-1 and the y
    // vectors.  The pairs are used while that solve took at most kCarryMaxIters
    // iterations: under a force that changes little from step to step they cut the
    // iterations; where each step needs several iterations anyway (a force redrawn at
    // random every step) they save none and a full window costs more per iteration.  History vectors that live in
    // the record are used in place (hist()); those in shared memory arrive by
    // asynchronous 16-byte copies, all of a thread's in flight at once.  s_i^T g at the
    // current iterate takes one block reduction.  Called at the step's first direction
    // request, so a cell accepted at its first iterate reads nothing.
    // Asynchronous copies of the record's ring slots held in shared memory (all m slots,
    // valid or not) and of its inner products.  The caller waits (cp.async.wait_all)
    // before reading them or reusing the buffers.
    __device__ void issue_pair_copies()
    {
        const int N3 = 3 * tp().n_pad, tid = threadIdx.x, NT = blockDim.x, Mm = M;
        const T* V = crec + carry_head_elems(Mm);
        for (int r = 0; r < 2 * Mm; ++r) {
            if (gd->loc[V_SBASE + r] < 0) continue;  // used in place
            const T* src = V + (long long)r * N3;
            T* dst = vec_ptr(*gd, smem, slot, V_SBASE + r);
            for (int e = 4 * tid; e < N3; e += 4 * NT) {
#pragma unroll
                for (int b = 0; b < (int)sizeof(T) / 4; ++b)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                                     (uint32_t)__cvta_generic_to_shared(dst + e + b * (16 / sizeof(T)))),
                                 "l"(__cvta_generic_to_global(src + e + b * (16 / sizeof(T))))
                                 : "memory");
            }
        }
        for (int k = tid; k < Mm * Mm; k += NT) {
            if constexpr (sizeof(T) == 4)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                                 (uint32_t)__cvta_generic_to_shared(&sh->SY[k / Mm][k % Mm])),
                             "l"(__cvta_generic_to_global(crec + 4 + k))
                             : "memory");
            else
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                                 (uint32_t)__cvta_generic_to_shared(&sh->SY[k / Mm][k % Mm])),
                             "l"(__cvta_generic_to_global(crec + 4 + k))
                             : "memory");
        }
    }

    __device__ void load_pairs()
    {
        carry_in = false;
        const int N3 = 3 * tp().n_pad, tid = threadIdx.x, NT = blockDim.x, Mm = M;
        const bool issued = carry_early;
        if (issued) {
            // the copies begin issued land before any ring slot is written
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncthreads();
            carry_early = false;
        }
        if (!(ccount >= T(1)) || !(clast <= T(kCarryMaxIters))) return;
        const int cnt = ccount < T(Mm) ? (int)ccount : Mm;
        const T hv = crec[1];
        const int hd = hv >= T(0) && hv < T(Mm) ? (int)hv : 0;
        if (!issued) {
            issue_pair_copies();
            asm volatile("cp.async.wait_all;" ::: "memory");
        }
        head = hd;
        count = cnt;
        __syncthreads();
        T acc[kMaxHistory];
#pragma unroll
        for (int q = 0; q < kMaxHistory; ++q) acc[q] = T(0);
        for (int e = 4 * tid; e < N3; e += 4 * NT) {
            T gv[4];
            ld4(g + e, gv);
#pragma unroll
            for (int q = 0; q < kMaxHistory; ++q) {
                if (q < cnt) {
                    T t[4];
                    ld4(hist(V_SBASE + hslot(q)) + e, t);
                    acc[q] += (t[0] * gv[0] + t[1] * gv[1]) + (t[2] * gv[2] + t[3] * gv[3]);
                }
            }
        }
        block_sum<T, kMaxHistory>(acc, smem, [=](CellShared<T>* c) {
            for (int q = 0; q < cnt; ++q) {
                const int i = (hd - 1 - q + Mm) % Mm;
                c->sg[i] = c->out[q];
                c->rho[i] = T(1) / c->SY[i][i];
            }
        });
    }

    // This solve's pairs into the cell's record: the history vectors not already there,
    // the inner products, the ring head, the count and the iterations.  Without an
    // iteration the record already holds the pairs and only the iteration count (0) is
    // written; after a failed line search, a non-finite state or more than
    // kCarryMaxIters iterations (pairs the next step will not use) only the header.
    __device__ void store_pairs()
    {
        const bool fail = nonfinite || status == NPFEM_CELL_LINESEARCH_FAIL;
        const int N3 = 3 * tp().n_pad, tid = threadIdx.x, NT = blockDim.x, Mm = M;
        if (carry_valid && iters == 0 && !fail) {
            // no iteration: the record keeps the pairs this solve would have started from
            // (none when the rule above left them out) and records 0 iterations
            if (tid == 0) {
                if (!(ccount >= T(1) && clast <= T(kCarryMaxIters))) crec[0] = T(0);
                crec[2] = T(0);
            }
            return;
        }
        if (fail || iters > kCarryMaxIters || M == 0) {
            // pairs the next step would not use: the header alone
            if (tid == 0) {
                crec[0] = T(0);
                crec[2] = T(iters);
            }
            return;
        }
        const int cnt = count;
        T* V = crec + carry_head_elems(Mm);
        // a slot loaded from the record and not written since still matches it
        const unsigned todo = carry_valid && ring_in_record() ? dirty : ~0u;
        for (int q = 0; q < 2 * cnt; ++q) {
            const int i = hslot(q >> 1);
            const int r = (q & 1) ? Mm + i : i;
            if (!((todo >> i) & 1u)) continue;
            if (ring_in_record() && gd->loc[V_SBASE + r] < 0) continue;  // already in the record
            const T* src = hist(V_SBASE + r);
            T* dst = V + (long long)r * N3;
            for (int e = 4 * tid; e < N3; e += 4 * NT) {
                T t[4];
                ld4(src + e, t);
                st4(dst + e, t);
            }
        }
        for (int k = tid; k < Mm * Mm; k += NT) crec[4 + k] = sh->SY[k / Mm][k % Mm];
        if (tid == 0) {
            crec[0] = T(cnt);
            crec[1] = T(head);
            crec[2] = T(iters);
        }
    }

    // First loop of the two-loop recursion (Nocedal & Wright Alg. 7.4), newest pair
    // first, on scalars: with s_i^T g and the pairs' inner products s_i^T y_j kept up to
    // date, alpha_i = rho_i (s_i^T g - sum_{j newer} alpha_j s_i^T y_j) on thread 0;
    // one pass then forms q = g - sum_i alpha_i y_i in Dv.  Thread 0 also publishes the
    // history vectors by age for the second loop and the line search.
    __device__ void first_loop()
    {
        if (carry_in) load_pairs();
        const int N3 = 3 * tp().n_pad, tid = threadIdx.x, NT = blockDim.x;
        const int cnt = count;
        if (cnt > 0) {
            if (tid == 0) {
                for (int q = 0; q < cnt; ++q) {
                    const int i = hslot(q);
                    sh->hs[q] = hist(V_SBASE + i);
                    sh->hy[q] = hist(V_SBASE + M + i);
                    T t = sh->sg[i];
                    for (int p = 0; p < q; ++p) {
                        const int j = hslot(p);
                        t -= sh->alpha[j] * sh->SY[i][j];
                    }
                    const T al = sh->rho[i] * t;
                    sh->alpha[i] = al;
                    sh->aq[q] = al;
                }
            }
            __syncthreads();
        }
        // unrolled over the window so that a thread's loads of the pairs (some of them
        // from global memory) are in flight together
        for (int e = 4 * tid; e < N3; e += 4 * NT) {
            T d[4];
            ld4(g + e, d);
#pragma unroll
            for (int q = 0; q < kMaxHistory; ++q) {
                if (q < cnt) {
                    T y[4];
                    ld4(sh->hy[q] + e, y);
                    const T al = sh->aq[q];
#pragma unroll
                    for (int k = 0; k < 4; ++k) d[k] -= al * y[k];
                }
            }
            st4(Dv + e, d);
        }
        __syncthreads();
    }

    // Second loop (oldest pair first) on r = H0 q held in GCv: one block reduction gives
    // y_i^T r for every pair; thread 0 runs beta_i = rho_i (y_i^T r + sum_{j older}
    // (alpha_j - beta_j) s_j^T y_i); one pass forms d = -(r + sum_i (alpha_i - beta_i) s_i)
    // in Dv together with gdv = g^T d.
    __device__ void second_loop()
    {
        const int N3 = 3 * tp().n_pad, tid = threadIdx.x, NT = blockDim.x;
        const int cnt = count, hd = head, Mm = M;
        if (cnt > 0) {
            T yr[kMaxHistory];
#pragma unroll
            for (int q = 0; q < kMaxHistory; ++q) yr[q] = T(0);
            for (int e = 4 * tid; e < N3; e += 4 * NT) {
                T r[4];
                ld4(GCv + e, r);
#pragma unroll
                for (int q = 0; q < kMaxHistory; ++q) {
                    if (q < cnt) {
                        T y[4];
                        ld4(sh->hy[q] + e, y);
                        yr[q] += (y[0] * r[0] + y[1] * r[1]) + (y[2] * r[2] + y[3] * r[3]);
                    }
                }
            }
            block_sum<T, kMaxHistory>(yr, smem, [=](CellShared<T>* c) {
                for (int q = cnt - 1; q >= 0; --q) {
                    const int i = (hd - 1 - q + Mm) % Mm;
                    c->yr[i] = c->out[q];
                    T t = c->out[q];
                    for (int p = cnt - 1; p > q; --p) {
                        const int j = (hd - 1 - p + Mm) % Mm;
                        t += c->coef[j] * c->SY[j][i];
                    }
                    const T cf = c->alpha[i] - c->rho[i] * t;
                    c->coef[i] = cf;
                    c->cq[q] = cf;
                }
            });
        }
        T s1[1] = {T(0)};
        for (int e = 4 * tid; e < N3; e += 4 * NT) {
            T r[4], gv[4];
            ld4(GCv + e, r);
#pragma unroll
            for (int q = 0; q < kMaxHistory; ++q) {
                if (q < cnt) {
                    T sv[4];
                    ld4(sh->hs[q] + e, sv);
                    const T cf = sh->cq[q];
#pragma unroll
                    for (int k = 0; k < 4; ++k) r[k] += cf * sv[k];
                }
            }
            ld4(g + e, gv);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                r[k] = -r[k];
                s1[0] += gv[k] * r[k];
            }
            st4(Dv + e, r);
        }
        block_sum<T, 1>(s1, smem);
        gdv = sh->out[0];
    }

    // d = -GCv into Dv, gdv = g^T d.
    __device__ void negate_direction()
    {
        const int N3 = 3 * tp().n_pad, tid = threadIdx.x, NT = blockDim.x;
        T s[1] = {T(0)};
        for (int e = 4 * tid; e < N3; e += 4 * NT) {
            T r[4], gv[4];
            ld4(GCv + e, r);
            ld4(g + e, gv);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                r[k] = -r[k];
                s[0] += gv[k] * r[k];
            }
            st4(Dv + e, r);
        }
        block_sum<T, 1>(s, smem);
        gdv = sh->out[0];
    }

    __device__ bool descent() const { return gdv < 0.0; }

    // Backtracking line search alpha = 1, 1/2, ... with the Armijo test (the FP32
    // path widens the bound by a multiple of the estimated rounding error of g),
    // history update and acceptance.  Returns false when no step length passed.
    __device__ bool line_search_update()
    {
        const TopoDev<T>& T_ = tp();
        const int N3 = 3 * T_.n_pad, tid = threadIdx.x, NT = blockDim.x;
        const T c1 = prm<T>(a->p.c1, a->p.c1f), c2 = prm<T>(a->p.c2, a->p.c2f);
        const T anoise = prm<T>(a->p.armijo_noise, a->p.armijo_noisef);
        T alpha = T(1);
        bool accepted = false;
        for (int hv = 0; hv <= a->p.max_halvings; ++hv) {
            for (int e = 4 * tid; e < N3; e += 4 * NT) {
                T uv[4], dv[4];
                ld4(u + e, uv);
                ld4(Dv + e, dv);
#pragma unroll
                for (int k = 0; k < 4; ++k) uv[k] += alpha * dv[k];
                st4(ut + e, uv);
            }
            __syncthreads();
            evaluate(T_, XN, ut, UYv, gt, GCv, TRIv, WRv, Vn, smem, colp, wcol);
            ++evals;
            if (tid == 0) {
                const bool ok = !sh->bad && pair_diff(sh->E, E) <= c1 * alpha * gdv + anoise * (sh->noise + noiseE);
                sh->accept = a->p.fixed_alpha || ok;
            }
            __syncthreads();
            if (sh->accept) {
                accepted = true;
                break;
            }
            alpha *= T(0.5);
        }
        if (!accepted) {
            status = NPFEM_CELL_LINESEARCH_FAIL;
            return false;
        }
        // history pair (s, y) = (x_{k+1} - x_k, grad_{k+1} - grad_k), kept when the
        // curvature condition holds and s^T y > 0.  The same pass gives s_j^T g_{k+1}
        // for the stored pairs, which keeps the two-loop's inner products current:
        // s_j^T y_new = s_j^T g_{k+1} - s_j^T g_k, and s_new^T y_j = alpha d^T y_j with
        // d^T y_j = -(y_j^T r + sum_l (alpha_l - beta_l) s_l^T y_j) from the last
        // second loop.
        if (M > 0) {
            const int cnt = count, hd = head, Mm = M;
            T acc[5 + kMaxHistory];  // s^T y, s^T s, y^T y, g_new^T d, s^T g_new, s_j^T g_new
#pragma unroll
            for (int q = 0; q < 5 + kMaxHistory; ++q) acc[q] = T(0);
            for (int e = 4 * tid; e < N3; e += 4 * NT) {
                T gn[4], go[4], un[4], uo[4], dv[4];
                ld4(gt + e, gn);
                ld4(g + e, go);
                ld4(ut + e, un);
                ld4(u + e, uo);
                ld4(Dv + e, dv);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const T se = un[k] - uo[k], ye = gn[k] - go[k];
                    acc[0] += se * ye;
                    acc[1] += se * se;
                    acc[2] += ye * ye;
                    acc[3] += gn[k] * dv[k];
                    acc[4] += se * gn[k];
                }
#pragma unroll
                for (int q = 0; q < kMaxHistory; ++q) {
                    if (q < cnt) {
                        T sv[4];
                        ld4(sh->hs[q] + e, sv);
                        acc[5 + q] += (sv[0] * gn[0] + sv[1] * gn[1]) + (sv[2] * gn[2] + sv[3] * gn[3]);
                    }
                }
            }
            const T gd0 = gdv, al = alpha;
            block_sum<T, 5 + kMaxHistory>(acc, smem, [=](CellShared<T>* c) {
                const T* o = c->out;
                c->push = o[3] >= c2 * gd0 && o[0] > T(1e-12) * sqrt(o[1]) * sqrt(o[2]);
                if (c->push) {
                    T dy[kMaxHistory];
                    for (int q = 0; q < cnt; ++q) {
                        const int j = (hd - 1 - q + Mm) % Mm;
                        T t = c->yr[j];
                        for (int p = 0; p < cnt; ++p) {
                            const int l = (hd - 1 - p + Mm) % Mm;
                            t += c->coef[l] * c->SY[l][j];
                        }
                        dy[q] = -t;
                    }
                    for (int q = 0; q < cnt; ++q) {
                        const int j = (hd - 1 - q + Mm) % Mm;
                        if (j == hd) continue;  // the oldest pair, overwritten
                        c->SY[hd][j] = al * dy[q];
                        c->SY[j][hd] = o[5 + q] - c->sg[j];
                    }
                    c->SY[hd][hd] = o[0];
                    c->rho[hd] = T(1) / o[0];
                }
                for (int q = 0; q < cnt; ++q) c->sg[(hd - 1 - q + Mm) % Mm] = o[5 + q];
                if (c->push) c->sg[hd] = o[4];
            });
            if (sh->push) {
                dirty |= 1u << head;
                T* S = hist(V_SBASE + head);
                T* Y = hist(V_SBASE + M + head);
                for (int e = 4 * tid; e < N3; e += 4 * NT) {
                    T a4[4], b4[4];
                    ld4(ut + e, a4);
                    ld4(u + e, b4);
#pragma unroll
                    for (int k = 0; k < 4; ++k) a4[k] -= b4[k];
                    st4(S + e, a4);
                    ld4(gt + e, a4);
                    ld4(g + e, b4);
#pragma unroll
                    for (int k = 0; k < 4; ++k) a4[k] -= b4[k];
                    st4(Y + e, a4);
                }
                head = (head + 1) % M;
                count = count < M ? count + 1 : M;
            }
        }
        T* t1 = u; u = ut; ut = t1;
        T* t2 = g; g = gt; gt = t2;
        E = sh->E;
        noiseE = sh->noise;
        res = sh->res;
        Vlast = sh->V;
        ++iters;
        nonfinite = sh->bad != 0;
        __syncthreads();
        return true;
    }

    // v_{n+1} = (x_{n+1} - x_n)/h and post-convergence dissipation (Sec. 2.1.4);
    // writes x, v and the cell's statistics.
    __device__ void finish()
    {
        const TopoDev<T>& T_ = tp();
        const int n = T_.n, np = T_.n_pad, tid = threadIdx.x, NT = blockDim.x;
        if (nonfinite) status = NPFEM_CELL_NONFINITE;
        if (carry_early) {
            // copies issued in begin that no direction request waited for
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncthreads();
        }
        if (crec) store_pairs();
        const T inv_h = T(1) / T_.h;
        Acc<T> ps[16];
        if (!nonfinite) {
            for (int i = tid; i < n; i += NT) {
                const T m = __ldg(&T_.mass[i]);
                T xr[3], vr[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    xr[c] = XN[c * np + i] + u[c * np + i];
                    vr[c] = u[c * np + i] * inv_h;
                }
                ps[0].add(m);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    ps[1 + c].add(m * xr[c]);
                    ps[4 + c].add(m * vr[c]);
                }
                ps[7].add(m * (xr[1] * vr[2] - xr[2] * vr[1]));
                ps[8].add(m * (xr[2] * vr[0] - xr[0] * vr[2]));
                ps[9].add(m * (xr[0] * vr[1] - xr[1] * vr[0]));
                ps[10].add(m * xr[0] * xr[0]);
                ps[11].add(m * xr[1] * xr[1]);
                ps[12].add(m * xr[2] * xr[2]);
                ps[13].add(m * xr[0] * xr[1]);
                ps[14].add(m * xr[0] * xr[2]);
                ps[15].add(m * xr[1] * xr[2]);
            }
        }
        const bool nf = nonfinite;
        block_reduce<T, 16>(ps, smem, [=](CellShared<T>* s) {
            const T* o = s->out;
            T* P = s->post;
            for (int q = 0; q < 9; ++q) P[q] = T(0);
            if (nf) return;
            const T Mt = o[0];
            T xc[3], vc[3];
            for (int c = 0; c < 3; ++c) {
                xc[c] = o[1 + c] / Mt;
                vc[c] = o[4 + c] / Mt;
            }
            // angular momentum and inertia tensor about the centre of mass
            const T L0 = o[7] - Mt * (xc[1] * vc[2] - xc[2] * vc[1]);
            const T L1 = o[8] - Mt * (xc[2] * vc[0] - xc[0] * vc[2]);
            const T L2 = o[9] - Mt * (xc[0] * vc[1] - xc[1] * vc[0]);
            const T Sxx = o[10] - Mt * xc[0] * xc[0], Syy = o[11] - Mt * xc[1] * xc[1],
                    Szz = o[12] - Mt * xc[2] * xc[2];
            const T Sxy = o[13] - Mt * xc[0] * xc[1], Sxz = o[14] - Mt * xc[0] * xc[2],
                    Syz = o[15] - Mt * xc[1] * xc[2];
            const T I00 = Syy + Szz, I11 = Sxx + Szz, I22 = Sxx + Syy;
            const T I01 = -Sxy, I02 = -Sxz, I12 = -Syz;
            const T c00 = I11 * I22 - I12 * I12, c01 = I02 * I12 - I01 * I22, c02 = I01 * I12 - I02 * I11;
            const T c11 = I00 * I22 - I02 * I02, c12 = I01 * I02 - I00 * I12, c22 = I00 * I11 - I01 * I01;
            const T det = I00 * c00 + I01 * c01 + I02 * c02;
            const T idet = T(1) / det;
            for (int c = 0; c < 3; ++c) {
                P[c] = xc[c];
                P[3 + c] = vc[c];
            }
            P[6] = (c00 * L0 + c01 * L1 + c02 * L2) * idet;
            P[7] = (c01 * L0 + c11 * L1 + c12 * L2) * idet;
            P[8] = (c02 * L0 + c12 * L1 + c22 * L2) * idet;
        });
        T xc[3], vc[3], w[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xc[c] = sh->post[c];
            vc[c] = sh->post[3 + c];
            w[c] = sh->post[6 + c];
        }
        const T kap = T_.kappa;
        T* x = a->x + so;
        T* v = a->v + so;
        // compensated positions (see begin): x_{n+1} = x + (residue + u) as an FP32 value and
        // its exact rounding error (two-sum, Knuth), which the next step adds back
        T* XLO = a->hist_out && a->pos_stride > 0 ? a->hist_out + a->pos_stride + so : nullptr;
        T* XHI = XLO ? XLO + a->pos_stride : nullptr;
        const bool lo_in = XLO && a->hist_in;
        for (int i = tid; i < n; i += NT) {
            if (nonfinite) {
                for (int c = 0; c < 3; ++c) {
                    v[c * n + i] = T(0);
                    if (XLO) {
                        XLO[c * n + i] = T(0);
                        XHI[c * n + i] = x[c * n + i];
                    }
                }
                continue;
            }
            // the global loads of all three coordinates first (the stores below would
            // otherwise hold them up)
            T xo3[3], hi3[3], lo3[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                xo3[c] = x[c * n + i];
                hi3[c] = lo_in ? XHI[c * n + i] : T(0);
                lo3[c] = lo_in ? XLO[c * n + i] : T(0);
            }
            T r[3];
            for (int c = 0; c < 3; ++c) r[c] = XN[c * np + i] + u[c * np + i] - xc[c];
            const T wr[3] = {w[1] * r[2] - w[2] * r[1], w[2] * r[0] - w[0] * r[2], w[0] * r[1] - w[1] * r[0]};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T uc = u[c * np + i];
                const T vv = uc * inv_h;
                v[c * n + i] = vv + kap * (vc[c] + wr[c] - vv);
                const T xo = xo3[c];
                if (XLO) {
                    const T t = (lo_in && hi3[c] == xo ? lo3[c] : T(0)) + uc;
                    const T sm = xo + t;
                    const T bv = sm - xo;
                    const T err = (xo - (sm - bv)) + (t - bv);
                    x[c * n + i] = sm;
                    XLO[c * n + i] = err;
                    XHI[c * n + i] = sm;
                } else {
                    x[c * n + i] = xo + uc;
                }
            }
        }
        if (a->hist_out) {
            // the converged correction x_{n+1} - y_n for the next step's first iterate; with a
            // temporal network the one it replaces and this step's force are kept too
            T* Hc = a->hist_out + so;
            T* Cp = a->hist_ext ? a->hist_out + 3 * a->pos_stride + so : nullptr;
            T* Fp = a->hist_ext ? a->hist_out + 4 * a->pos_stride + so : nullptr;
            const T* fc = a->f + so;
            for (int e = tid; e < 3 * n; e += NT) {
                const int c = e / n, i = e - c * n;
                if (Cp) {
                    Cp[e] = a->hist_in ? Hc[e] : T(0);
                    Fp[e] = fc[e];
                }
                Hc[e] = nonfinite ? T(0) : u[c * np + i] - UYv[c * np + i];
            }
        }
        if (tid == 0 && a->stats) {
            npfem_cell_stats st;
            st.iterations = iters;
            st.evaluations = evals;
            st.status = status;
            st.residual = (float)res;
            st.objective = pair_f64(E);
            st.volume = pair_f64(Vlast);
            a->stats[item] = st;
        }
        __syncthreads();
    }
};

// Next work item of the launch (block-uniform), or -1.
template <typename T>
__device__ __forceinline__ long long next_item(const LaunchArgs<T>& a, unsigned char* smem)
{
    CellShared<T>* sh = cell_shared<T>(smem);
    if (threadIdx.x == 0) {
        unsigned long long* cw = reinterpret_cast<unsigned long long*>(a.work);
        // a launch over listed cells reads their number, written by an earlier launch
        const long long total = a.only ? (long long)*reinterpret_cast<const volatile unsigned int*>(a.only) : a.total_cells;
        long long item = -1;
        if (a.claim_top) {
            // a slower helper: leaves the last `reserve` cells to the main launch
            const unsigned long long cur = *reinterpret_cast<volatile unsigned long long*>(cw);
            const long long left = total - (long long)(cur & 0xffffffffull) - (long long)(cur >> 32);
            if (left > a.reserve) {
                const unsigned long long old = atomicAdd(cw, 1ull << 32);
                const long long lo = (long long)(old & 0xffffffffull), hi = (long long)(old >> 32);
                if (lo + hi < total) item = total - 1 - hi;
            }
        } else {
            const unsigned long long old = atomicAdd(cw, 1ull);
            const long long lo = (long long)(old & 0xffffffffull), hi = (long long)(old >> 32);
            if (lo + hi < total) item = lo;
        }
        if (item >= 0 && a.only) item = (long long)a.only[3 + item];
        sh->item = item;
    }
    __syncthreads();
    const long long it = sh->item;
    __syncthreads();
    return it;
}

// The last block to finish (of all launches sharing the counters) resets them for the
// next launch.
__device__ __forceinline__ void release_counters(unsigned int* work, int total_blocks)
{
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&work[3], 1u);
        const unsigned total = total_blocks > 0 ? (unsigned)total_blocks : gridDim.x * gridDim.y * gridDim.z;
        if (prev == total - 1) {
            atomicExch(reinterpret_cast<unsigned long long*>(work), 0ull);
            atomicExch(&work[3], 0u);
        }
    }
}

// R = H0 Q for the SIMT kernel: FP32/FP64 on the SIMT pipes, or TF32 tensor cores
// (with the optional refinement sweep r += A^-1 (q - H~ r), its correction in `tmp2`).
template <typename T>
__device__ __forceinline__ void contract_any(const LaunchArgs<T>& a, const TopoDev<T>& tp, const T* Q, T* R,
                                             CellSolver<T>& S, unsigned char* smem)
{
    if constexpr (sizeof(T) == 4) {
        if (a.p.contraction == CONTRACT_TC_TF32) {
            CellShared<float>* sh = cell_shared<float>(smem);
            tf32::contract(tp, Q, R, smem + kFixedSmem, sh, a.work + 2);
            if (a.p.refine) {
                refine_residual(tp, Q, R, S.WRv);
                tf32::contract(tp, S.WRv, S.ut, smem + kFixedSmem, sh, a.work + 2);
                for (int e = threadIdx.x; e < 3 * tp.n_pad; e += blockDim.x) R[e] += S.ut[e];
                __syncthreads();
            }
            return;
        }
    }
    contract_simt(tp, Q, R, S.TRIv, static_cast<const T*>(nullptr), S.gd->scratch_floats);
}

template <typename T, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) cell_kernel(const __grid_constant__ LaunchArgs<T> a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    CellSolver<T> S;
    if constexpr (sizeof(T) == 4) {
        if (a.p.contraction == CONTRACT_TC_TF32)
            tf32::setup(a.p.tf_kpad, smem + kFixedSmem, cell_shared<float>(smem), (uint32_t)a.p.tmem_cols);
    }
    // first-iterate pass: evaluate only while most cells of the last step were accepted
    const bool eval_first = a.defer && 2ll * (long long)a.defer[2] <= a.total_cells;
    for (;;) {
        const long long item = next_item(a, smem);
        if (item < 0) break;
        if (a.defer && !eval_first) {
            if (threadIdx.x == 0) a.defer[3 + atomicAdd(a.defer, 1u)] = (unsigned int)item;
            continue;
        }
        int gi = 0;
        while (gi + 1 < a.n_groups && item >= a.g[gi + 1].cell_begin) ++gi;
        S.bind(a, a.g[gi], smem);
        if (!S.begin(item - a.g[gi].cell_begin, a.g[gi].stats_off + item - a.g[gi].cell_begin)) continue;
        const bool wants = S.wants_direction();
        if (a.need && wants && threadIdx.x == 0) atomicAdd(a.need, 1u);
        if (a.defer && wants) {
            // the cell needs iterations: the launch that follows solves it from the
            // unchanged state
            if (threadIdx.x == 0) a.defer[3 + atomicAdd(a.defer, 1u)] = (unsigned int)item;
            continue;
        }
        const TopoDev<T>& tp = a.g[gi].topo;
        while (S.wants_direction()) {
            S.first_loop();
            contract_any(a, tp, S.Dv, S.GCv, S, smem);  // r = H0 q
            S.second_loop();
            if (!S.descent()) {
                // not a descent direction: drop the history, d = -H~^-1 g
                S.count = 0;
                contract_any(a, tp, S.g, S.GCv, S, smem);
                S.negate_direction();
            }
            if (!S.line_search_update()) break;
        }
        S.finish();
    }
    if constexpr (sizeof(T) == 4) {
        if (a.p.contraction == CONTRACT_TC_TF32) tf32::teardown(cell_shared<float>(smem), (uint32_t)a.p.tmem_cols);
    }
    release_counters(a.work, a.total_blocks);
}

// ---------------------------------------------------------------------------------
// Tensor-core contraction: a cluster of ceil(n / 128) blocks, one block per SM, each
// holding rows [128 r, 128 r + 128) of A^-1 (BF16) in tensor memory for the whole
// launch.  Blocks solve their cells independently; a contraction is a request that
// every block of the cluster serves asynchronously:
//   request -> the requesting block writes its vector (BF16) into rows 3 r + c of the
//              B operand of every block (DSMEM) and sets its bit in every block's
//              pending mask (release);
//   serve   -> at its next poll point a block takes its pending mask (acquire),
//              issues ceil(n/16) tcgen05.mma (M 128, N 16/32, K 16, A from TMEM, B
//              from shared memory, FP32 accumulate in TMEM) for the whole batch,
//              reads its 128 result rows and writes each requester's three columns
//              into that requester's contraction vector (DSMEM), then arrives on the
//              requester's delivery barrier (release);
//   wait    -> the requester serves at its own poll points until all blocks of the
//              cluster have delivered.
// Poll points: while waiting for a result, and between the solver's phases.  A block
// whose cells are done keeps serving until every block of the cluster is done.
// ---------------------------------------------------------------------------------

// Writes BF16(src) (3 rows of the cell, zero beyond n) into rows 3 rank + c of the B
// operand of every block in the cluster.  If with_residual, writes instead the
// refinement residual e = src - H~ r (H~ = ms M + L, sparse FP32) for r = R.
// tmp: 3 x n_pad scratch (the bending buffer, idle outside the evaluation).
template <typename T>
__device__ void tc_post(const TopoDev<T>& tp, const T* src, const T* R, bool with_residual, unsigned char* bbuf,
                        uint32_t rank, uint32_t cs, T* tmp)
{
    const int n = tp.n, np = tp.n_pad, kpad = tp.kpad, tid = threadIdx.x, NT = blockDim.x;
    const int chunks = 3 * (kpad >> 3);
    const uint32_t local = tc::smem_addr(bbuf);
    if (with_residual) {
        refine_residual(tp, src, R, tmp);
        src = tmp;
    }
    for (int q = tid; q < chunks; q += NT) {
        const int c = q / (kpad >> 3), kb = q - c * (kpad >> 3);
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = 8 * kb + u;
            v[u] = k < n ? (float)src[c * np + k] : 0.f;
        }
        const uint4 w = make_uint4(tc::pack_bf16(v[0], v[1]), tc::pack_bf16(v[2], v[3]), tc::pack_bf16(v[4], v[5]),
                                   tc::pack_bf16(v[6], v[7]));
        const uint32_t off = tc::b_offset(3 * (int)rank + c, 8 * kb, kpad);
        for (uint32_t d = 0; d < cs; ++d) tc::st_remote_v4(tc::map_rank(local + off, d), w);
    }
}

// The asynchronous rounds of one block (see above).  Every method is called by all
// threads of the block (control flow block-uniform).
template <typename T, int NCOL>
struct TcRounds {
    CellShared<T>* sh;
    const TopoDev<T>* tp;
    unsigned char* bbuf;
    T* GCv;
    unsigned* err;
    uint32_t tbase, dcol, idesc, sbo, bbase, rank, cs;
    uint32_t nserv, nreq;

    // Serves the requests pending at this block, if any.
    __device__ void serve()
    {
        const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
        if (tid == 0) {
            uint32_t b;
            asm volatile("atom.acquire.cluster.shared::cluster.exch.b32 %0, [%1], 0;"
                         : "=r"(b)
                         : "r"(tc::smem_addr(&sh->pend))
                         : "memory");
            sh->batch = b;
        }
        __syncthreads();
        const uint32_t batch = sh->batch;
        if (batch == 0u) return;
        const int kpad = tp->kpad, n = tp->n, np = tp->n_pad;
        if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int ks = 0; ks < (kpad >> 4); ++ks) {
                const uint64_t bd = tc::smem_desc(bbase + (uint32_t)ks * 256u, 128u, sbo);
                const uint32_t ta = tbase + (uint32_t)(ks * 8);
                const uint32_t acc = ks > 0;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(tbase + dcol),
                    "r"(ta), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                tc::smem_addr(&sh->mbar)));
        }
        uint32_t done = 0;
        for (int it = 0; it < (1 << 22) && !done; ++it) {
            asm volatile(
                "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                : "=r"(done)
                : "r"(tc::smem_addr(&sh->mbar)), "r"(nserv & 1u));
        }
        if (!done && tid == 0) atomicExch(err, 1u);  // reported to the host; results invalid
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (warp < 4) {
            float dv[NCOL];
            tc::tmem_ld<NCOL>(tbase + ((uint32_t)(32 * warp) << 16) + dcol, dv);
            const int row = 128 * (int)rank + 32 * warp + lane;
            if (row < n) {
#pragma unroll
                for (int d = 0; d < NCOL / 3 && d < 8; ++d) {
                    if (!((batch >> d) & 1u)) continue;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const uint32_t loc = tc::smem_addr(GCv + c * np + row);
                        tc::st_remote_f32(tc::map_rank(loc, (uint32_t)d), dv[3 * d + c]);
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid < (int)cs && ((batch >> tid) & 1u)) {
            // the results written above (other threads, ordered by the barrier) are
            // released with the arrival
            const uint32_t rb = tc::map_rank(tc::smem_addr(&sh->dbar), (uint32_t)tid);
            asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(rb) : "memory");
        }
        ++nserv;
    }

    // r = A^-1 src into GCv (BF16 operands, FP32 accumulation); with refine one more
    // sweep r += A^-1 (src - H~ r).  tmp, keep: 3 x n_pad scratch.
    __device__ void contract(const T* src, bool refine, T* tmp, T* keep)
    {
        request(src, false, tmp);
        if (refine) {
            const int N3 = 3 * tp->n_pad;
            for (int e = threadIdx.x; e < N3; e += blockDim.x) keep[e] = GCv[e];
            __syncthreads();
            request(src, true, tmp);
            for (int e = threadIdx.x; e < N3; e += blockDim.x) GCv[e] += keep[e];
            __syncthreads();
        }
    }

    // Posts src (or the refinement residual of src for r = GCv) and waits, serving, for
    // the cs deliveries.
    __device__ void request(const T* src, bool residual, T* tmp)
    {
        const int tid = threadIdx.x;
        tc_post(*tp, src, GCv, residual, bbuf, rank, cs, tmp);
        asm volatile("fence.proxy.async.shared::cluster;" ::: "memory");
        __syncthreads();
        if (tid < (int)cs) {
            const uint32_t pa = tc::map_rank(tc::smem_addr(&sh->pend), (uint32_t)tid);
            asm volatile("red.release.cluster.shared::cluster.or.b32 [%0], %1;" ::"r"(pa), "r"(1u << rank) : "memory");
        }
        const uint32_t par = nreq & 1u;
        bool ok = false;
        for (int it = 0; it < (1 << 22); ++it) {
            serve();
            if (tid == 0) {
                uint32_t d;
                asm volatile(
                    "{\n.reg .pred p;\nmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
                    "selp.u32 %0, 1, 0, p;\n}"
                    : "=r"(d)
                    : "r"(tc::smem_addr(&sh->dbar)), "r"(par)
                    : "memory");
                // the error word (global memory) only now and then: each read costs a round trip
                sh->flag = d | ((it & 255) == 255 && *reinterpret_cast<volatile unsigned*>(err) != 0u ? 2u : 0u);
            }
            __syncthreads();
            const uint32_t f = sh->flag;
            if (f & 1u) {
                ok = true;
                break;
            }
            if (f & 2u) break;  // another block gave up: stop waiting
        }
        if (!ok && tid == 0) atomicExch(err, 1u);
        ++nreq;
    }

    // The block's cells are done: tell every block, then serve until all are done.
    __device__ void finish_and_drain()
    {
        const int tid = threadIdx.x;
        __syncthreads();
        if (tid < (int)cs) {
            const uint32_t fa = tc::map_rank(tc::smem_addr(&sh->fin), (uint32_t)tid);
            asm volatile("red.release.cluster.shared::cluster.add.u32 [%0], 1;" ::"r"(fa) : "memory");
        }
        bool ok = false;
        for (int it = 0; it < (1 << 24); ++it) {
            serve();
            if (tid == 0) {
                uint32_t f;
                asm volatile("ld.acquire.cluster.shared::cluster.u32 %0, [%1];"
                             : "=r"(f)
                             : "r"(tc::smem_addr(&sh->fin))
                             : "memory");
                sh->flag = (f >= cs ? 1u : 0u) |
                           ((it & 255) == 255 && *reinterpret_cast<volatile unsigned*>(err) != 0u ? 2u : 0u);
            }
            __syncthreads();
            const uint32_t f = sh->flag;
            if (f & 1u) {
                ok = true;
                break;
            }
            if (f & 2u) break;
        }
        if (!ok && tid == 0) atomicExch(err, 1u);
        // nothing is left pending: every request was delivered before its block finished
    }
};

template <typename T, int NCOL>
__global__ void __launch_bounds__(512, 1) cell_kernel_tc(const __grid_constant__ LaunchArgs<T> a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const GroupDesc<T>& gd = a.g[0];
    const TopoDev<T>& tp = gd.topo;
    CellShared<T>* sh = cell_shared<T>(smem);
    unsigned char* bbuf = smem + kFixedSmem;  // B operand: NCOL rows x kpad BF16
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t rank = tc::cta_rank(), cs = (uint32_t)a.p.cluster;
    const int kpad = tp.kpad;
    const uint32_t acols = (uint32_t)(kpad >> 1);
    const uint32_t dcol = (acols + 31u) & ~31u;

    // ---- set-up: zero B, flags, barriers, TMEM allocation, A^-1 rows of this block into TMEM
    for (int q = tid; q < NCOL * kpad / 8; q += blockDim.x) reinterpret_cast<uint4*>(bbuf)[q] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        sh->pend = 0u;
        sh->fin = 0u;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_addr(&sh->mbar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc::smem_addr(&sh->dbar)), "r"(cs));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
            tc::smem_addr(&sh->taddr)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = sh->taddr;
    if (warp < 4) {
        const int row = 128 * (int)rank + 32 * warp + lane;
        const uint32_t* src = reinterpret_cast<const uint32_t*>(tp.ainv_lp) + (size_t)row * (kpad >> 1);
        for (int c0 = 0; c0 < (int)acols; c0 += 8) {
            uint32_t r[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) r[j] = __ldg(&src[c0 + j]);
            const uint32_t ta = tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(ta), "r"(r[0]),
                         "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]));
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    tc::cluster_sync();  // every block's barriers and flags are initialised
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    CellSolver<T> S;
    S.bind(a, gd, smem);
    TcRounds<T, NCOL> R;
    R.sh = sh;
    R.tp = &tp;
    R.bbuf = bbuf;
    R.GCv = S.GCv;
    R.err = &a.work[2];
    R.tbase = tbase;
    R.dcol = dcol;
    R.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NCOL >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    R.sbo = (uint32_t)(kpad >> 3) * 128u;
    R.bbase = tc::smem_addr(bbuf);
    R.rank = rank;
    R.cs = cs;
    R.nserv = 0u;
    R.nreq = 0u;
    const bool refine = a.p.refine != 0;

    for (;;) {
        R.serve();
        const long long item = next_item(a, smem);
        if (item < 0) break;
        S.begin(item, item);
        const bool wants = S.wants_direction();
        if (a.need && wants && tid == 0) atomicAdd(a.need, 1u);
        while (S.wants_direction()) {
            R.serve();
            S.first_loop();
            R.contract(S.Dv, refine, S.WRv, S.ut);  // r = H0 q
            S.second_loop();
            if (!S.descent()) {
                // not a descent direction: drop the history, d = -H~^-1 g
                S.count = 0;
                R.contract(S.g, refine, S.WRv, S.ut);
                S.negate_direction();
            }
            if (!S.line_search_update()) break;
        }
        S.finish();
    }
    R.finish_and_drain();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    tc::cluster_sync();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase));
    release_counters(a.work, a.total_blocks);
}

}  // namespace

// SIMT kernel variants by block size: 512 threads (128 registers) and, for FP32, 640
// threads (96 registers; 20 warps, the triangle pass of a 642-vertex cell in two rounds
// instead of three).
template <typename T>
cudaError_t set_cell_kernel_smem(int bytes)
{
    cudaError_t e = cudaFuncSetAttribute(cell_kernel<T, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && sizeof(T) == 4)
        e = cudaFuncSetAttribute(cell_kernel<float, 640>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

template <typename T>
cudaError_t cells_per_sm(int block, int smem, int* n)
{
    if (block <= 512) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, cell_kernel<T, 512>, block, smem);
    if constexpr (sizeof(T) == 4) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, cell_kernel<float, 640>, block, smem);
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_cells(const LaunchArgs<T>& a, int grid, int block, int smem, cudaStream_t s)
{
    if (block <= 512) {
        cell_kernel<T, 512><<<grid, block, smem, s>>>(a);
    } else if constexpr (sizeof(T) == 4) {
        if (block > 640) return cudaErrorInvalidValue;
        cell_kernel<float, 640><<<grid, block, smem, s>>>(a);
    } else {
        return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

static cudaLaunchConfig_t tc_config(int cluster, int block, int smem, int grid, cudaStream_t s, cudaLaunchAttribute* attr)
{
    cudaLaunchConfig_t cfg = {};
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(block);
    cfg.gridDim = dim3(grid);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

cudaError_t query_cells_tc(int cluster, int block, int smem, int* max_clusters)
{
    const bool wide = cluster * 3 > 16;
    auto kern32 = cell_kernel_tc<float, 32>;
    auto kern16 = cell_kernel_tc<float, 16>;
    cudaError_t e = wide ? cudaFuncSetAttribute(kern32, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
                         : cudaFuncSetAttribute(kern16, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = tc_config(cluster, block, smem, cluster, nullptr, attr);
    int n = 0;
    e = wide ? cudaOccupancyMaxActiveClusters(&n, kern32, &cfg) : cudaOccupancyMaxActiveClusters(&n, kern16, &cfg);
    if (e != cudaSuccess) return e;
    if (n < 1) return cudaErrorInvalidConfiguration;
    *max_clusters = n;
    return cudaSuccess;
}

// Cluster launch of the tensor-core kernel for one mesh group.
cudaError_t launch_cells_tc(const LaunchArgs<float>& a, int cluster, int block, int smem, int grid, cudaStream_t s)
{
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = tc_config(cluster, block, smem, grid, s, attr);
    const bool wide = cluster * 3 > 16;
    cudaError_t e = wide ? cudaLaunchKernelEx(&cfg, cell_kernel_tc<float, 32>, a)
                         : cudaLaunchKernelEx(&cfg, cell_kernel_tc<float, 16>, a);
    if (e != cudaSuccess) return e;
    count_launch();
    return cudaGetLastError();
}

template cudaError_t set_cell_kernel_smem<float>(int);
template cudaError_t set_cell_kernel_smem<double>(int);
template cudaError_t launch_cells<float>(const LaunchArgs<float>&, int, int, int, cudaStream_t);
template cudaError_t cells_per_sm<float>(int, int, int*);
template cudaError_t cells_per_sm<double>(int, int, int*);
template cudaError_t launch_cells<double>(const LaunchArgs<double>&, int, int, int, cudaStream_t);

}  // namespace npfem
