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

// Volume of the cell at x_n in local coordinates: V = sum_t X_i . (E1 x E2) / 6.
template <typename T>
__device__ void volume_at_xn(const TopoDev<T>& tp, const T* XN, unsigned char* smem)
{
    const int np = tp.n_pad;
    Acc<T> acc[1];
    for (int t = threadIdx.x; t < tp.nt; t += blockDim.x) {
        const ushort4 tv = __ldg(&tp.tri[t]);
        T Xi[3], E1[3], E2[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Xi[c] = XN[c * np + tv.x];
            E1[c] = XN[c * np + tv.y] - Xi[c];
            E2[c] = XN[c * np + tv.z] - Xi[c];
        }
        const T cx = E1[1] * E2[2] - E1[2] * E2[1], cy = E1[2] * E2[0] - E1[0] * E2[2],
                cz = E1[0] * E2[1] - E1[1] * E2[0];
        acc[0].add(Xi[0] * cx + Xi[1] * cy + Xi[2] * cz);
    }
    block_reduce<T, 1>(acc, smem, [](CellShared* sh) { sh->V = sh->out[0] / 6.0; });
}

// Objective g and gradient at x_n + U (Eq. GeneralizedObjectiveFunction and its
// derivative): inertia, local area preservation and bending (projective dynamics
// gradients), global volume conservation (PD gradient with the linearised
// projection), modified Skalak (first Piola-Kirchhoff forces).  Results are left in
// cell_shared(smem): E, its parts, V, residual r, rounding estimate of E, bad flag.
// Vn is the volume at x_n (held by the caller).
//
// Gather form, no atomics: pass 1 writes each triangle's corner gradients and
// area-weighted normal to TRI; pass 2 gathers them per vertex (vertex -> triangle
// incidence) and computes the bending residual w_i r_i into WR; pass 3 gathers the
// bending gradient from the neighbours' WR (transposed cotangent weights) and adds
// the volume and inertia terms.  Every vertex is written by one thread only.
// With kFirst, the same triangle pass also accumulates V(x_n) (left in sh->Vn) and
// Vn is ignored.
template <typename T, bool kFirst = false>
__device__ void evaluate(const TopoDev<T>& tp, const T* XN, const T* U, const T* UY, T* Gout, T* GC, T* TRI, T* WR,
                         double Vn, unsigned char* smem)
{
    const int n = tp.n, np = tp.n_pad, tid = threadIdx.x, NT = blockDim.x;
    CellShared* sh = cell_shared(smem);
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
        T* out = TRI + 9 * t;
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
#pragma unroll
            for (int c = 0; c < 6; ++c) out[c] = T(0);
#pragma unroll
            for (int c = 0; c < 3; ++c) out[6 + c] = cr[c] * sixth;
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
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T G0 = F0[c] * K00 + F1[c] * K01;
            const T G1 = F0[c] * K01 + F1[c] * K11;
            out[c] = G0 * Di0 + G1 * Di1;      // corner j
            out[3 + c] = G0 * Di2 + G1 * Di3;  // corner k (corner i gets minus both)
            out[6 + c] = cr[c] * sixth;        // share of the area-weighted normal / 3
        }
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
        const int b0 = __ldg(&tp.inc_ptr[i]), b1 = __ldg(&tp.inc_ptr[i + 1]);
        for (int q = b0; q < b1; ++q) {
            const unsigned e = __ldg(&tp.inc_idx[q]);
            const T* P = TRI + 9 * (e >> 2);
            const unsigned corner = e & 3u;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T gj = P[c], gk = P[3 + c];
                g[c] += corner == 1u ? gj : (corner == 2u ? gk : -(gj + gk));
                gc[c] += P[6 + c];
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Gout[c * np + i] = g[c];
            GC[c * np + i] = gc[c];
        }
        pl[0] += gc[0] * gc[0] + gc[1] * gc[1] + gc[2] * gc[2];

        const int r0 = __ldg(&tp.ring_ptr[i]), r1 = __ldg(&tp.ring_ptr[i + 1]);
        T dfn[3] = {T(0), T(0), T(0)}, dfu[3] = {T(0), T(0), T(0)};
        T Xi[3], Ui[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Xi[c] = XN[c * np + i];
            Ui[c] = U[c * np + i];
        }
        for (int q = r0; q < r1; ++q) {
            const int jn = __ldg(&tp.ring_idx[q]);
            const T cq = __ldg(&tp.ring_c[q]);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dfn[c] += cq * (XN[c * np + jn] - Xi[c]);
                dfu[c] += cq * (U[c * np + jn] - Ui[c]);
            }
        }
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
    const double kvol = (double)tp.kvol, V0 = tp.V0;
    block_reduce_cp<T, 5, 3>(ce, pl, smem, [=](CellShared* s) {
        s->Earea = s->out[0];
        s->Esk = s->out[1];
        s->Ebend = s->out[2];
        const double vn = kFirst ? s->out[4] / 6.0 : Vn;
        s->Vn = vn;
        s->V = vn + s->out[3] / 6.0;
        const double Cv = s->V - V0;
        const T inv = T(1) / (T)s->out[5];
        s->Evol = 0.5 * kvol * Cv * Cv * (double)inv;
        s->volc = kvol * Cv * (double)inv;
        s->volcf = (float)s->volc;
        s->noise = s->out[6];
        s->bad = s->out[7] != 0.0;
    });
    const T volc = bcast<T>(sh->volc, sh->volcf);

    // ---- pass 3: bending gather, volume and inertia (M~ = (1 + h alpha_D) M), residual
    const T ms = tp.inertia_scale * tp.inv_h2, h2 = tp.h * tp.h;
    Acc<T> ci[1];            // inertia energy
    T pr[1] = {T(0)};        // sum_i (h^2 |grad_i| / m_i)^2
    for (int i = tid; i < n; i += NT) {
        const T m = __ldg(&tp.mass[i]);
        const T hm = h2 * __ldg(&tp.inv_mass[i]);
        const int r0 = __ldg(&tp.ring_ptr[i]), r1 = __ldg(&tp.ring_ptr[i + 1]);
        const T cs = __ldg(&tp.csum[i]);
        T gb[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) gb[c] = -cs * WR[c * np + i];
        for (int q = r0; q < r1; ++q) {
            const int jn = __ldg(&tp.ring_idx[q]);
            const T ct = __ldg(&tp.ring_ct[q]);
#pragma unroll
            for (int c = 0; c < 3; ++c) gb[c] += ct * WR[c * np + jn];
        }
        T g2 = T(0), ei = T(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T du = U[c * np + i] - UY[c * np + i];
            const T gv = Gout[c * np + i] + gb[c] + volc * GC[c * np + i] + m * ms * du;
            Gout[c * np + i] = gv;
            ei += T(0.5) * m * ms * du * du;
            g2 += gv * gv;
        }
        ci[0].add(ei);
        pr[0] += hm * hm * g2;
    }
    const T inv_n = T(1) / T(n), inv_lbar = tp.inv_lbar;
    const double uT = Unit<T>::u;
    block_reduce_cp<T, 1, 1>(ci, pr, smem, [=](CellShared* s) {
        s->Ein = s->out[0];
        s->E = s->Ein + s->Earea + s->Esk + s->Ebend + s->Evol;
        s->res = (double)(sqrt((T)s->out[1] * inv_n) * inv_lbar);
        s->noise = 4.0 * uT * (s->noise + 2.0 * s->Ein);
    });
}

// R = A^-1 Q for the three coordinate rows.
// FP32: a warp owns a tile of 128 rows (4 consecutive rows per lane, float4 loads of
// the symmetric A^-1 by columns, coalesced) and a share of the j range; Q is
// broadcast from shared memory.  The warps' partial sums go to `scratch` (the
// triangle buffer, idle outside the objective evaluation) and are added in a fixed
// order, so the result is deterministic.
template <typename T>
__device__ void contract_simt(const TopoDev<T>& tp, const T* Q, T* R, T* scratch)
{
    const int n = tp.n, np = tp.n_pad, N3 = 3 * np;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const T* __restrict__ A = tp.ainv;
    if constexpr (sizeof(T) == 4) {
        const int ntile = (n + 127) >> 7;
        // ntile <= nw: warp w takes tile w % ntile and a share of the j range;
        // ntile > nw: warps loop over whole tiles.  Partials go to scratch[item][c][128].
        const bool split = ntile <= nw;
        for (int item = warp; item < (split ? nw : ntile); item += nw) {
            const int tile = split ? item % ntile : item;
            const int part = split ? item / ntile : 0;
            const int nparts = split ? (nw - 1 - tile) / ntile + 1 : 1;
            const int chunk = (((n + nparts - 1) / nparts) + 3) & ~3;
            const int j0 = part * chunk, j1 = min(n, j0 + chunk);
            const int row0 = tile * 128 + 4 * lane;
            float acc[3][4];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int r = 0; r < 4; ++r) acc[c][r] = 0.f;
            if (row0 < n) {
                int j = j0;
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
                if (split) {
                    for (int w = tl; w < nw; w += ntile) s += S[w * 384 + c * 128 + rr];
                } else {
                    s = S[tl * 384 + c * 128 + rr];
                }
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
    CellShared* sh;
    T *XN, *u, *ut, *g, *gt, *GCv, *UYv, *Dv, *TRIv, *WRv;
    long long so, item;
    int M, head, count, iters, evals, status;
    double E, noiseE, res, Vlast, Vn, gdv;
    bool nonfinite;

    __device__ const TopoDev<T>& tp() const { return gd->topo; }
    __device__ T* hist(int v) const { return vec_ptr(*gd, smem, slot, v); }

    __device__ void bind(const LaunchArgs<T>& la, const GroupDesc<T>& g_, unsigned char* sm)
    {
        a = &la;
        gd = &g_;
        smem = sm;
        sh = cell_shared(sm);
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
        const T h = T_.h, inv_ms = T(1) / T_.inertia_scale;
        const bool eval_mode = a->p.mode == 1;
        const T* x = a->x + so;
        const T o0 = x[0], o1 = x[n], o2 = x[2 * n];
        for (int e = tid; e < N3; e += NT) {
            const int c = e / np, i = e - c * np;
            T xn = T(0), uy = T(0);
            if (i < n) {
                const T xv = x[c * n + i];
                xn = xv - (c == 0 ? o0 : (c == 1 ? o1 : o2));
                if (eval_mode) {
                    uy = a->y[so + c * n + i] - xv;
                } else {
                    const T vv = a->v[so + c * n + i], fv = a->f[so + c * n + i];
                    uy = (h * vv + h * h * fv * __ldg(&T_.inv_mass[i])) * inv_ms;
                }
            }
            XN[e] = xn;
            UYv[e] = uy;
            u[e] = eval_mode ? T(0) : uy;
        }
        __syncthreads();
        // learned warm start: u = u_y + R MLP(features at y)
        const int ws = (!eval_mode && T_.mlp) ? T_.ws_mode : 0;
        if (ws && a->u0) {
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
            for (int q = 0; q < 9; ++q) R[q] = sh->postf[q];
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
        evals = 1;
        if (ws == 2) {
            // keep the learned guess only if it lowers g: evaluate at y (trial buffers) first
            for (int e = tid; e < N3; e += NT) ut[e] = UYv[e];
            __syncthreads();
            evaluate<T, true>(T_, XN, ut, UYv, gt, GCv, TRIv, WRv, 0.0, smem);
            Vn = sh->Vn;
            const double Ey = sh->E, ny = sh->noise, ry = sh->res, Vy = sh->V;
            const bool by = sh->bad;
            evaluate<T, false>(T_, XN, u, UYv, g, GCv, TRIv, WRv, Vn, smem);
            evals = 2;
            if (!(sh->E <= Ey) && !by) {
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
            evaluate<T, true>(T_, XN, u, UYv, g, GCv, TRIv, WRv, 0.0, smem);
            Vn = sh->Vn;
        }
        iters = 0;
        status = NPFEM_CELL_OK;
        head = 0;
        count = 0;
        if (eval_mode) {
            for (int e = tid; e < 3 * n; e += NT) {
                const int c = e / n, i = e - c * n;
                a->grad_out[so + e] = g[c * np + i];
            }
            if (tid == 0) {
                double* P = a->parts + 8 * item;
                P[0] = sh->Ein; P[1] = sh->Earea; P[2] = sh->Esk; P[3] = sh->Ebend; P[4] = sh->Evol;
                P[5] = sh->V; P[6] = sh->E; P[7] = sh->res;
            }
            __syncthreads();
            return false;
        }
        E = sh->E;
        noiseE = sh->noise;
        res = sh->res;
        Vlast = sh->V;
        nonfinite = sh->bad || !isfinite(sh->E) || !isfinite(sh->res);
        return true;
    }

    // Residual test and iteration cap; false when the cell is finished.
    __device__ bool wants_direction()
    {
        if (nonfinite) return false;
        if (res <= a->p.tol) return false;
        if (iters >= a->p.max_iter) {
            status = NPFEM_CELL_MAXITER;
            return false;
        }
        return true;
    }

    // First loop of the two-loop recursion: q = g; alpha_i = rho_i s_i^T q;
    // q -= alpha_i y_i (newest first).  q is left in Dv.
    __device__ void first_loop()
    {
        const int N3 = 3 * tp().n_pad, tid = threadIdx.x, NT = blockDim.x;
        for (int e = tid; e < N3; e += NT) Dv[e] = g[e];
        for (int q = 0; q < count; ++q) {
            const int i = (head - 1 - q + M) % M;
            const T* S = hist(V_SBASE + i);
            const T* Y = hist(V_SBASE + M + i);
            T s[1] = {T(0)};
            for (int e = tid; e < N3; e += NT) s[0] += S[e] * Dv[e];
            block_sum<T, 1>(s, smem, [=](CellShared* c) { c->alpha[i] = c->rho[i] * c->out[0]; });
            const T al = (T)sh->alpha[i];
            for (int e = tid; e < N3; e += NT) Dv[e] -= al * Y[e];
        }
        __syncthreads();
    }

    // Second loop (oldest first) on r = H0 q held in GCv: beta = rho_i y_i^T r;
    // r += s_i (alpha_i - beta); then d = -r into Dv and gdv = g^T d.
    __device__ void second_loop()
    {
        const int N3 = 3 * tp().n_pad, tid = threadIdx.x, NT = blockDim.x;
        for (int q = count - 1; q >= 0; --q) {
            const int i = (head - 1 - q + M) % M;
            const T* S = hist(V_SBASE + i);
            const T* Y = hist(V_SBASE + M + i);
            T s[1] = {T(0)};
            for (int e = tid; e < N3; e += NT) s[0] += Y[e] * GCv[e];
            block_sum<T, 1>(s, smem, [=](CellShared* c) { c->out[1] = c->alpha[i] - c->rho[i] * c->out[0]; });
            const T coef = (T)sh->out[1];
            for (int e = tid; e < N3; e += NT) GCv[e] += S[e] * coef;
        }
        negate_direction();
    }

    // d = -GCv into Dv, gdv = g^T d.
    __device__ void negate_direction()
    {
        const int N3 = 3 * tp().n_pad, tid = threadIdx.x, NT = blockDim.x;
        T s[1] = {T(0)};
        for (int e = tid; e < N3; e += NT) {
            const T dv = -GCv[e];
            Dv[e] = dv;
            s[0] += g[e] * dv;
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
        const double c1 = a->p.c1, c2 = a->p.c2, anoise = a->p.armijo_noise;
        double alpha = 1.0;
        T al = T(1);  // alpha in the working type (powers of two: exact)
        bool accepted = false;
        for (int hv = 0; hv <= a->p.max_halvings; ++hv) {
            for (int e = tid; e < N3; e += NT) ut[e] = u[e] + al * Dv[e];
            __syncthreads();
            evaluate(T_, XN, ut, UYv, gt, GCv, TRIv, WRv, Vn, smem);
            ++evals;
            if (tid == 0) {
                const bool ok = !sh->bad && sh->E <= E + c1 * alpha * gdv + anoise * (sh->noise + noiseE);
                sh->accept = a->p.fixed_alpha || ok;
            }
            __syncthreads();
            if (sh->accept) {
                accepted = true;
                break;
            }
            alpha *= 0.5;
            al *= T(0.5);
        }
        if (!accepted) {
            status = NPFEM_CELL_LINESEARCH_FAIL;
            return false;
        }
        // history pair (s, y) = (x_{k+1} - x_k, grad_{k+1} - grad_k), kept when the
        // curvature condition holds and s^T y > 0
        if (M > 0) {
            T acc[4] = {T(0), T(0), T(0), T(0)};  // s^T y, s^T s, y^T y, grad_new^T d
            for (int e = tid; e < N3; e += NT) {
                const T se = ut[e] - u[e], ye = gt[e] - g[e];
                acc[0] += se * ye;
                acc[1] += se * se;
                acc[2] += ye * ye;
                acc[3] += gt[e] * Dv[e];
            }
            const int hd = head;
            const double gd0 = gdv;
            block_sum<T, 4>(acc, smem, [=](CellShared* c) {
                c->push = c->out[3] >= c2 * gd0 && c->out[0] > 1e-12 * sqrt(c->out[1] * c->out[2]);
                if (c->push) c->rho[hd] = 1.0 / c->out[0];
            });
            if (sh->push) {
                T* S = hist(V_SBASE + head);
                T* Y = hist(V_SBASE + M + head);
                for (int e = tid; e < N3; e += NT) {
                    S[e] = ut[e] - u[e];
                    Y[e] = gt[e] - g[e];
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
        nonfinite = sh->bad || !isfinite(sh->E) || !isfinite(sh->res);
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
        block_reduce<T, 16>(ps, smem, [=](CellShared* s) {
            double* o = s->out;
            double* P = s->post;
            for (int q = 0; q < 9; ++q) {
                P[q] = 0.0;
                s->postf[q] = 0.f;
            }
            if (nf) return;
            const double Mt = o[0];
            double xc[3], vc[3];
            for (int c = 0; c < 3; ++c) {
                xc[c] = o[1 + c] / Mt;
                vc[c] = o[4 + c] / Mt;
            }
            // angular momentum and inertia tensor about the centre of mass
            const double L0 = o[7] - Mt * (xc[1] * vc[2] - xc[2] * vc[1]);
            const double L1 = o[8] - Mt * (xc[2] * vc[0] - xc[0] * vc[2]);
            const double L2 = o[9] - Mt * (xc[0] * vc[1] - xc[1] * vc[0]);
            const double Sxx = o[10] - Mt * xc[0] * xc[0], Syy = o[11] - Mt * xc[1] * xc[1],
                         Szz = o[12] - Mt * xc[2] * xc[2];
            const double Sxy = o[13] - Mt * xc[0] * xc[1], Sxz = o[14] - Mt * xc[0] * xc[2],
                         Syz = o[15] - Mt * xc[1] * xc[2];
            const double I00 = Syy + Szz, I11 = Sxx + Szz, I22 = Sxx + Syy;
            const double I01 = -Sxy, I02 = -Sxz, I12 = -Syz;
            const double c00 = I11 * I22 - I12 * I12, c01 = I02 * I12 - I01 * I22, c02 = I01 * I12 - I02 * I11;
            const double c11 = I00 * I22 - I02 * I02, c12 = I01 * I02 - I00 * I12, c22 = I00 * I11 - I01 * I01;
            const double det = I00 * c00 + I01 * c01 + I02 * c02;
            for (int c = 0; c < 3; ++c) {
                P[c] = xc[c];
                P[3 + c] = vc[c];
            }
            P[6] = (c00 * L0 + c01 * L1 + c02 * L2) / det;
            P[7] = (c01 * L0 + c11 * L1 + c12 * L2) / det;
            P[8] = (c02 * L0 + c12 * L1 + c22 * L2) / det;
            for (int q = 0; q < 9; ++q) s->postf[q] = (float)P[q];
        });
        T xc[3], vc[3], w[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xc[c] = bcast<T>(sh->post[c], sh->postf[c]);
            vc[c] = bcast<T>(sh->post[3 + c], sh->postf[3 + c]);
            w[c] = bcast<T>(sh->post[6 + c], sh->postf[6 + c]);
        }
        const T kap = T_.kappa;
        T* x = a->x + so;
        T* v = a->v + so;
        for (int i = tid; i < n; i += NT) {
            if (nonfinite) {
                for (int c = 0; c < 3; ++c) v[c * n + i] = T(0);
                continue;
            }
            T r[3];
            for (int c = 0; c < 3; ++c) r[c] = XN[c * np + i] + u[c * np + i] - xc[c];
            const T wr[3] = {w[1] * r[2] - w[2] * r[1], w[2] * r[0] - w[0] * r[2], w[0] * r[1] - w[1] * r[0]};
            for (int c = 0; c < 3; ++c) {
                const T uc = u[c * np + i];
                const T vv = uc * inv_h;
                v[c * n + i] = vv + kap * (vc[c] + wr[c] - vv);
                x[c * n + i] = x[c * n + i] + uc;
            }
        }
        if (tid == 0 && a->stats) {
            npfem_cell_stats st;
            st.iterations = iters;
            st.evaluations = evals;
            st.status = status;
            st.residual = (float)res;
            st.objective = E;
            st.volume = Vlast;
            a->stats[item] = st;
        }
        __syncthreads();
    }
};

// Next work item of the launch (block-uniform), or -1.
template <typename T>
__device__ __forceinline__ long long next_item(const LaunchArgs<T>& a, unsigned char* smem)
{
    CellShared* sh = cell_shared(smem);
    if (threadIdx.x == 0) sh->item = (long long)atomicAdd(&a.work[0], 1u);
    __syncthreads();
    const long long it = sh->item;
    __syncthreads();
    return it < a.total_cells ? it : -1;
}

// The last block to finish resets the work counters for the next launch.
__device__ __forceinline__ void release_counters(unsigned int* work)
{
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&work[1], 1u);
        if (prev == gridDim.x * gridDim.y * gridDim.z - 1) {
            atomicExch(&work[0], 0u);
            atomicExch(&work[1], 0u);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(512, 1) cell_kernel(const __grid_constant__ LaunchArgs<T> a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    CellSolver<T> S;
    for (;;) {
        const long long item = next_item(a, smem);
        if (item < 0) break;
        int gi = 0;
        while (gi + 1 < a.n_groups && item >= a.g[gi + 1].cell_begin) ++gi;
        S.bind(a, a.g[gi], smem);
        if (!S.begin(item - a.g[gi].cell_begin, item)) continue;
        const TopoDev<T>& tp = a.g[gi].topo;
        while (S.wants_direction()) {
            S.first_loop();
            contract_simt(tp, S.Dv, S.GCv, S.TRIv);  // r = H0 q
            S.second_loop();
            if (!S.descent()) {
                // not a descent direction: drop the history, d = -H~^-1 g
                S.count = 0;
                contract_simt(tp, S.g, S.GCv, S.TRIv);
                S.negate_direction();
            }
            if (!S.line_search_update()) break;
        }
        S.finish();
    }
    release_counters(a.work);
}

// ---------------------------------------------------------------------------------
// Tensor-core contraction: a cluster of ceil(n / 128) blocks, one block per SM, each
// holding rows [128 r, 128 r + 128) of A^-1 (BF16) in tensor memory for the whole
// launch.  A "round" applies A^-1 to the current request of every block of the
// cluster at once:
//   local work  -> each block with a request writes its vector (BF16) into row
//                  3 r + c of the B operand of every block of the cluster (DSMEM);
//   barrier     -> every block issues ceil(n/16) tcgen05.mma (M 128, N 16/32, K 16,
//                  A from TMEM, B from shared memory, FP32 accumulate in TMEM),
//                  reads its 128 result rows and writes them into the requesting
//                  blocks' contraction vectors (DSMEM);
//   barrier     -> results are in place.
// Blocks without work still take part until every block of the cluster is idle, so
// all blocks pass the same sequence of cluster barriers.
// ---------------------------------------------------------------------------------
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
        // e = src - H~ R, one row (three components) per thread
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

enum TcPhase { PH_NONE = 0, PH_DIR1, PH_DIR2, PH_FB1, PH_FB2 };

template <typename T, int NCOL>
__global__ void __launch_bounds__(512, 1) cell_kernel_tc(const __grid_constant__ LaunchArgs<T> a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const GroupDesc<T>& gd = a.g[0];
    const TopoDev<T>& tp = gd.topo;
    CellShared* sh = cell_shared(smem);
    unsigned char* bbuf = smem + kFixedSmem;  // B operand: NCOL rows x kpad BF16
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t rank = tc::cta_rank(), cs = (uint32_t)a.p.cluster;
    const int n = tp.n, np = tp.n_pad, kpad = tp.kpad;
    const uint32_t acols = (uint32_t)(kpad >> 1);
    const uint32_t dcol = (acols + 31u) & ~31u;

    // ---- set-up: zero B, flags, TMEM allocation, A^-1 rows of this block into TMEM
    for (int q = tid; q < NCOL * kpad / 8; q += blockDim.x) reinterpret_cast<uint4*>(bbuf)[q] = make_uint4(0, 0, 0, 0);
    if (tid < 16) sh->need[tid] = 0u;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_addr(&sh->mbar)));
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
    tc::cluster_sync();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NCOL >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const uint32_t lbo = 128u, sbo = (uint32_t)(kpad >> 3) * 128u;
    const uint32_t bbase = tc::smem_addr(bbuf);
    const bool refine = a.p.refine != 0;

    CellSolver<T> S;
    S.bind(a, gd, smem);
    int phase = PH_NONE;
    bool have_result = false, exhausted = false;
    uint32_t round = 0;
    for (;;) {
        // ---- local work up to the next request (or idle)
        bool need = false;
        for (;;) {
            if (phase == PH_NONE) {
                const long long item = exhausted ? -1 : next_item(a, smem);
                if (item < 0) {
                    exhausted = true;
                    break;
                }
                S.begin(item, item);
            } else if (have_result) {
                have_result = false;
                if ((phase == PH_DIR1 || phase == PH_FB1) && refine) {
                    // keep r1, request A^-1 (src - H~ r1)
                    const int N3 = 3 * np;
                    for (int e = tid; e < N3; e += blockDim.x) S.ut[e] = S.GCv[e];
                    __syncthreads();
                    tc_post(tp, phase == PH_DIR1 ? S.Dv : S.g, S.GCv, true, bbuf, rank, cs, S.WRv);
                    phase = phase == PH_DIR1 ? PH_DIR2 : PH_FB2;
                    need = true;
                    break;
                }
                if (phase == PH_DIR2 || phase == PH_FB2) {
                    const int N3 = 3 * np;
                    for (int e = tid; e < N3; e += blockDim.x) S.GCv[e] += S.ut[e];
                    __syncthreads();
                }
                if (phase == PH_DIR1 || phase == PH_DIR2) {
                    S.second_loop();
                    if (!S.descent()) {
                        S.count = 0;
                        tc_post(tp, S.g, S.GCv, false, bbuf, rank, cs, S.WRv);
                        phase = PH_FB1;
                        need = true;
                        break;
                    }
                } else {
                    S.negate_direction();
                }
                if (!S.line_search_update()) {
                    S.finish();
                    phase = PH_NONE;
                    continue;
                }
            }
            if (!S.wants_direction()) {
                S.finish();
                phase = PH_NONE;
                continue;
            }
            S.first_loop();
            tc_post(tp, S.Dv, S.GCv, false, bbuf, rank, cs, S.WRv);
            phase = PH_DIR1;
            need = true;
            break;
        }
        // announce the request flag to every block of the cluster
        if (tid < (int)cs) tc::st_remote_u32(tc::map_rank(tc::smem_addr(&sh->need[rank]), (uint32_t)tid), need ? 1u : 0u);
        asm volatile("fence.proxy.async.shared::cluster;" ::: "memory");
        tc::cluster_sync();
        uint32_t any = 0;
        for (uint32_t d = 0; d < cs; ++d) any |= sh->need[d];
        if (!any) break;

        // ---- the round: MMAs on this block's row block for every request
        if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int ks = 0; ks < (kpad >> 4); ++ks) {
                const uint64_t bd = tc::smem_desc(bbase + (uint32_t)ks * 256u, lbo, sbo);
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
                : "r"(tc::smem_addr(&sh->mbar)), "r"(round & 1u));
        }
        if (!done && tid == 0) atomicExch(&a.work[2], 1u);  // reported to the host; results invalid
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (warp < 4) {
            float dv[NCOL];
            tc::tmem_ld<NCOL>(tbase + ((uint32_t)(32 * warp) << 16) + dcol, dv);
            const int row = 128 * (int)rank + 32 * warp + lane;
            if (row < n) {
#pragma unroll
                for (int d = 0; d < NCOL / 3 && d < 8; ++d) {
                    if (d >= (int)cs || !sh->need[d]) continue;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const uint32_t loc = tc::smem_addr(S.GCv + c * np + row);
                        tc::st_remote_f32(tc::map_rank(loc, (uint32_t)d), dv[3 * d + c]);
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        tc::cluster_sync();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        have_result = need;
        ++round;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    tc::cluster_sync();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase));
    release_counters(a.work);
}

}  // namespace

template <typename T>
cudaError_t set_cell_kernel_smem(int bytes)
{
    return cudaFuncSetAttribute(cell_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <typename T>
cudaError_t launch_cells(const LaunchArgs<T>& a, int grid, int block, int smem, cudaStream_t s)
{
    cell_kernel<T><<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

// Cluster launch of the tensor-core kernel for one mesh group; returns the grid in
// *grid_out (cluster size x co-resident clusters, capped by the cell count).
cudaError_t launch_cells_tc(const LaunchArgs<float>& a, int cluster, int block, int smem, cudaStream_t s,
                            int* grid_out)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const bool wide = cluster * 3 > 16;
    auto kern32 = cell_kernel_tc<float, 32>;
    auto kern16 = cell_kernel_tc<float, 16>;
    cudaError_t e = wide ? cudaFuncSetAttribute(kern32, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
                         : cudaFuncSetAttribute(kern16, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int nclusters = 0;
    cfg.gridDim = dim3(cluster);
    e = wide ? cudaOccupancyMaxActiveClusters(&nclusters, kern32, &cfg)
             : cudaOccupancyMaxActiveClusters(&nclusters, kern16, &cfg);
    if (e != cudaSuccess) return e;
    if (nclusters < 1) return cudaErrorInvalidConfiguration;
    long long want = (a.total_cells + cluster - 1) / cluster;
    if (want > nclusters) want = nclusters;
    cfg.gridDim = dim3((unsigned)(want * cluster));
    *grid_out = (int)(want * cluster);
    e = wide ? cudaLaunchKernelEx(&cfg, kern32, a) : cudaLaunchKernelEx(&cfg, kern16, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template cudaError_t set_cell_kernel_smem<float>(int);
template cudaError_t set_cell_kernel_smem<double>(int);
template cudaError_t launch_cells<float>(const LaunchArgs<float>&, int, int, int, cudaStream_t);
template cudaError_t launch_cells<double>(const LaunchArgs<double>&, int, int, int, cudaStream_t);

}  // namespace npfem
