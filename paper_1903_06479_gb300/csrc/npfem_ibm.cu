// Immersed-boundary force step upstream of the solver (Sec. 2.3 of arXiv:1903.06479):
// the external force of Eq. Fext sampled from a lattice stress field, interpolation
// of a lattice velocity to the membrane vertices, and the multi-direct forcing
// iteration that makes the fluid follow the membrane (Steps 0-5 of Sec. 2.3).
//
// The four-point kernel w(r) of Sec. 2.3 gives each vertex a 4 x 4 x 4 stencil of
// lattice nodes with weights w(r_x - i) w(r_y - j) w(r_z - k).  One thread handles
// one vertex: it forms the vertex's area share A_k (a third of its triangles' areas)
// and unit normal n_k from the current positions, then gathers (or, when spreading,
// scatters with atomics) over its stencil.  Lattice coordinates are formed in FP64
// (a 100 um domain at FP32 would round the fractional lattice offset to ~1e-5); the
// weights and sums are FP32.
//
// Conventions (the paper prints the formulas in lattice units, dx = 1):
//  * interpolation u(X_k) = sum_x u(x) w w w (the dx^3 of W dx^3 cancels);
//  * Eq. Fext: F_k = rho A_k (sum_x sigma(x) w w w) n_k;
//  * spreading f(x) = sum_k f_k (w w w / dx^3) A_k dx: a membrane one spacing thick, so
//    that spreading is the adjoint of interpolation;
//  * stencil nodes outside the lattice contribute nothing.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "npfem_device.cuh"
#include "npfem_internal.h"

namespace npfem {
namespace {

struct LatDev {
    double ox, oy, oz, inv_dx;
    float dx;
    int nx, ny, nz;
};

struct IbmGroup {
    TopoDev<float> topo;
    long long vert_begin;  // first global vertex index of the group
    long long state_off;   // element offset of the group's first cell in the SoA arrays
    int cells;
};

struct IbmArgs {
    IbmGroup g[kMaxGroups];
    int n_groups;
    long long total_verts;
    LatDev lat;
    const float* x;       // SoA positions
    const float* field;   // sigma [nodes][8] (forces) or a velocity [nodes][4]
    const float* field2;  // forcing: the lattice force [nodes][4] (update phase)
    const float* uvert;   // forcing: membrane vertex velocities U_k (SoA)
    float* out;           // SoA vertex output
    float* lat_out;       // forcing: lattice force [nodes][4] (spread phase)
    float rho, dt;
    int mode;             // forces: 0 full stencil, 1 exterior nodes, 2 farthest exterior node
    int phase;            // forcing: 0 f = (U - u*)/dt, 1 spread f, 2 f += (U - u_l)/dt
};

// The paper's one-dimensional four-point kernel (lattice units).
__device__ __forceinline__ float w4(float r)
{
    const float a = fabsf(r);
    if (a <= 1.f) return 0.125f * (3.f - 2.f * a + sqrtf(1.f + 4.f * a - 4.f * a * a));
    if (a <= 2.f) return 0.125f * (5.f - 2.f * a - sqrtf(fmaxf(-7.f + 12.f * a - 4.f * a * a, 0.f)));
    return 0.f;
}

struct Stencil {
    int i0, j0, k0;      // first node in each direction
    float t[3];          // fractional lattice offset of the point in [0, 1)
    float w[3][4];       // weights of nodes i0 + a, a = 0..3
};

__device__ __forceinline__ void make_stencil(const LatDev& L, float X, float Y, float Z, Stencil& s)
{
    const double r[3] = {((double)X - L.ox) * L.inv_dx, ((double)Y - L.oy) * L.inv_dx, ((double)Z - L.oz) * L.inv_dx};
    int b[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        // a point far outside the lattice (or not finite) gets a stencil with no nodes
        const double rd = r[d] == r[d] ? fmin(fmax(r[d], -1.0e6), 1.0e6) : -1.0e6;
        const double f = floor(rd);
        b[d] = (int)f - 1;
        const float t = (float)(rd - f);
        s.t[d] = t;
        s.w[d][0] = w4(t + 1.f);
        s.w[d][1] = w4(t);
        s.w[d][2] = w4(t - 1.f);
        s.w[d][3] = w4(t - 2.f);
    }
    s.i0 = b[0];
    s.j0 = b[1];
    s.k0 = b[2];
}

// Global vertex index -> (group, its topology, cell, vertex).
__device__ __forceinline__ const IbmGroup& locate(const IbmArgs& a, long long gv, long long* cell, int* vert)
{
    int gi = 0;
    while (gi + 1 < a.n_groups && gv >= a.g[gi + 1].vert_begin) ++gi;
    const IbmGroup& G = a.g[gi];
    const long long local = gv - G.vert_begin;
    *cell = local / G.topo.n;
    *vert = (int)(local - *cell * G.topo.n);
    return G;
}

__device__ __forceinline__ bool node_in(const LatDev& L, int i, int j, int k)
{
    return (unsigned)i < (unsigned)L.nx && (unsigned)j < (unsigned)L.ny && (unsigned)k < (unsigned)L.nz;
}

__device__ __forceinline__ long long node_index(const LatDev& L, int i, int j, int k)
{
    return ((long long)k * L.ny + j) * L.nx + i;
}

// Eq. Fext, one vertex per thread.
__global__ void __launch_bounds__(256) ibm_forces_kernel(const __grid_constant__ IbmArgs a)
{
    const LatDev& L = a.lat;
    for (long long gv = blockIdx.x * (long long)blockDim.x + threadIdx.x; gv < a.total_verts;
         gv += (long long)gridDim.x * blockDim.x) {
        long long cell;
        int i;
        const IbmGroup& G = locate(a, gv, &cell, &i);
        const int n = G.topo.n;
        const long long so = G.state_off + cell * 3LL * n;
        const float* xc = a.x + so;
        float A, nv[3];
        vertex_area_normal(G.topo, xc, i, &A, nv);
        Stencil s;
        make_stencil(L, xc[i], xc[n + i], xc[2 * n + i], s);
        float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, wsum = 0.f, dbest = -1.f;
        for (int c = 0; c < 4; ++c)
            for (int b = 0; b < 4; ++b)
                for (int q = 0; q < 4; ++q) {
                    const int ii = s.i0 + q, jj = s.j0 + b, kk = s.k0 + c;
                    if (!node_in(L, ii, jj, kk)) continue;
                    float wgt = s.w[0][q] * s.w[1][b] * s.w[2][c];
                    if (a.mode != 0) {
                        // offset node - X in um; exterior when it points along n
                        const float d[3] = {((float)(q - 1) - s.t[0]) * L.dx, ((float)(b - 1) - s.t[1]) * L.dx,
                                            ((float)(c - 1) - s.t[2]) * L.dx};
                        if (!(d[0] * nv[0] + d[1] * nv[1] + d[2] * nv[2] > 0.f)) continue;
                        if (a.mode == 2) {
                            const float d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                            if (!(d2 > dbest)) continue;  // keep the first among equals
                            dbest = d2;
                            wgt = 1.f;
#pragma unroll
                            for (int e = 0; e < 6; ++e) acc[e] = 0.f;
                            wsum = 0.f;
                        }
                    }
                    const float4* P = reinterpret_cast<const float4*>(a.field + 8 * node_index(L, ii, jj, kk));
                    const float4 s0 = __ldg(P), s1 = __ldg(P + 1);
                    acc[0] += wgt * s0.x; acc[1] += wgt * s0.y; acc[2] += wgt * s0.z;
                    acc[3] += wgt * s0.w; acc[4] += wgt * s1.x; acc[5] += wgt * s1.y;
                    wsum += wgt;
                }
        if (a.mode != 0) {
            const float inv = wsum > 0.f ? 1.f / wsum : 0.f;
#pragma unroll
            for (int e = 0; e < 6; ++e) acc[e] *= inv;
        }
        // (xx, yy, zz, xy, xz, yz) times n, scaled by rho A_k
        const float sc = a.rho * A;
        float* o = a.out + so;
        o[i] = sc * (acc[0] * nv[0] + acc[3] * nv[1] + acc[4] * nv[2]);
        o[n + i] = sc * (acc[3] * nv[0] + acc[1] * nv[1] + acc[5] * nv[2]);
        o[2 * n + i] = sc * (acc[4] * nv[0] + acc[5] * nv[1] + acc[2] * nv[2]);
    }
}

// Stencil sum of a [nodes][4] field (plus dt times a second one, if given).
__device__ __forceinline__ void gather4(const LatDev& L, const Stencil& s, const float* F, const float* F2, float dt,
                                        float out[3])
{
    out[0] = out[1] = out[2] = 0.f;
    for (int c = 0; c < 4; ++c)
        for (int b = 0; b < 4; ++b)
            for (int q = 0; q < 4; ++q) {
                const int ii = s.i0 + q, jj = s.j0 + b, kk = s.k0 + c;
                if (!node_in(L, ii, jj, kk)) continue;
                const float wgt = s.w[0][q] * s.w[1][b] * s.w[2][c];
                const long long nd = node_index(L, ii, jj, kk);
                float4 u = __ldg(reinterpret_cast<const float4*>(F) + nd);
                if (F2) {
                    // the corrected lattice velocity u* + dt f (Step 2) is formed on the fly;
                    // F2 is written by an earlier launch, so a plain (coherent) load
                    const float4 f = reinterpret_cast<const float4*>(F2)[nd];
                    u.x += dt * f.x;
                    u.y += dt * f.y;
                    u.z += dt * f.z;
                }
                out[0] += wgt * u.x;
                out[1] += wgt * u.y;
                out[2] += wgt * u.z;
            }
}

// Velocity interpolation (phase -1) and the phases of the multi-direct forcing.
__global__ void __launch_bounds__(256) ibm_forcing_kernel(const __grid_constant__ IbmArgs a)
{
    const LatDev& L = a.lat;
    for (long long gv = blockIdx.x * (long long)blockDim.x + threadIdx.x; gv < a.total_verts;
         gv += (long long)gridDim.x * blockDim.x) {
        long long cell;
        int i;
        const IbmGroup& G = locate(a, gv, &cell, &i);
        const int n = G.topo.n;
        const long long so = G.state_off + cell * 3LL * n;
        const float* xc = a.x + so;
        Stencil s;
        make_stencil(L, xc[i], xc[n + i], xc[2 * n + i], s);
        float* o = a.out + so;
        if (a.phase == 1) {
            // Step 1: spread f_k with weight A_k dx / dx^3 per unit stencil weight
            float A, nv[3];
            vertex_area_normal(G.topo, xc, i, &A, nv);
            const float sc = A / (L.dx * L.dx);
            const float f[3] = {sc * o[i], sc * o[n + i], sc * o[2 * n + i]};
            for (int c = 0; c < 4; ++c)
                for (int b = 0; b < 4; ++b)
                    for (int q = 0; q < 4; ++q) {
                        const int ii = s.i0 + q, jj = s.j0 + b, kk = s.k0 + c;
                        if (!node_in(L, ii, jj, kk)) continue;
                        const float wgt = s.w[0][q] * s.w[1][b] * s.w[2][c];
                        float* P = a.lat_out + 4 * node_index(L, ii, jj, kk);
                        atomicAdd(P, wgt * f[0]);
                        atomicAdd(P + 1, wgt * f[1]);
                        atomicAdd(P + 2, wgt * f[2]);
                    }
            continue;
        }
        float u[3];
        gather4(L, s, a.field, a.phase == 2 ? a.field2 : nullptr, a.dt, u);
        if (a.phase < 0) {
            o[i] = u[0];
            o[n + i] = u[1];
            o[2 * n + i] = u[2];
            continue;
        }
        const float* U = a.uvert + so;
        const float inv_dt = 1.f / a.dt;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float slip = (U[c * n + i] - u[c]) * inv_dt;
            o[c * n + i] = a.phase == 0 ? slip : o[c * n + i] + slip;  // Step 0, or Step 4
        }
    }
}

int fill_ibm(IbmArgs* a, npfem_handle* const* meshes, int n_groups, const int32_t* cells, const npfem_lattice* lat,
             const char* who)
{
    memset(a, 0, sizeof(*a));
    if (!meshes || n_groups < 1 || n_groups > kMaxGroups || !cells || !lat)
        return set_error(NPFEM_ERR_INVALID_ARG, std::string(who) + ": need 1..8 handles, cell counts and a lattice");
    if (!(lat->dx > 0.0) || lat->nx < 1 || lat->ny < 1 || lat->nz < 1 || !std::isfinite(lat->origin[0]) ||
        !std::isfinite(lat->origin[1]) || !std::isfinite(lat->origin[2]))
        return set_error(NPFEM_ERR_INVALID_ARG, std::string(who) + ": lattice needs dx > 0 and positive sizes");
    long long v = 0, st = 0;
    for (int g = 0; g < n_groups; ++g) {
        npfem_handle* h = meshes[g];
        if (!h || cells[g] < 0) return set_error(NPFEM_ERR_INVALID_ARG, std::string(who) + ": bad handle or cell count");
        if (h->precision == NPFEM_PREC_FP64 || h->device != meshes[0]->device)
            return set_error(NPFEM_ERR_INVALID_ARG, std::string(who) + ": FP32-state handles of one device only");
        a->g[g].topo = h->tf;
        a->g[g].vert_begin = v;
        a->g[g].state_off = st;
        a->g[g].cells = cells[g];
        v += (long long)h->n * cells[g];
        st += 3LL * h->n * cells[g];
    }
    a->n_groups = n_groups;
    a->total_verts = v;
    a->lat.ox = lat->origin[0];
    a->lat.oy = lat->origin[1];
    a->lat.oz = lat->origin[2];
    a->lat.inv_dx = 1.0 / lat->dx;
    a->lat.dx = (float)lat->dx;
    a->lat.nx = lat->nx;
    a->lat.ny = lat->ny;
    a->lat.nz = lat->nz;
    return 0;
}

int ibm_grid(const npfem_handle* h, long long verts)
{
    const long long blocks = (verts + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(blocks, (long long)std::max(h->sm_count, 1) * 8));
}

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int launch_err(const char* who, cudaError_t e)
{
    return set_error(NPFEM_ERR_CUDA, std::string(who) + ": " + cudaGetErrorString(e));
}

}  // namespace
}  // namespace npfem

using namespace npfem;

extern "C" int npfem_ibm_forces(npfem_handle* const* meshes, int n_groups, const int32_t* cells_per_group,
                                const float* x, const npfem_lattice* lattice, const float* sigma, double rho_fluid,
                                int mode, float* f_ext, void* stream)
{
    IbmArgs a;
    if (int rc = fill_ibm(&a, meshes, n_groups, cells_per_group, lattice, "npfem_ibm_forces")) return rc;
    if (!x || !sigma || !f_ext || mode < 0 || mode > 2 || !std::isfinite(rho_fluid))
        return set_error(NPFEM_ERR_INVALID_ARG, "npfem_ibm_forces: null array, mode outside 0..2 or bad rho");
    if (a.total_verts == 0) return 0;
    DevGuard guard(meshes[0]->device);
    a.x = x;
    a.field = sigma;
    a.out = f_ext;
    a.rho = (float)rho_fluid;
    a.mode = mode;
    ibm_forces_kernel<<<ibm_grid(meshes[0], a.total_verts), 256, 0, static_cast<cudaStream_t>(stream)>>>(a);
    count_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 0 : launch_err("npfem_ibm_forces", e);
}

extern "C" int npfem_ibm_interpolate(npfem_handle* const* meshes, int n_groups, const int32_t* cells_per_group,
                                     const float* x, const npfem_lattice* lattice, const float* u_lattice,
                                     float* u_vertex, void* stream)
{
    IbmArgs a;
    if (int rc = fill_ibm(&a, meshes, n_groups, cells_per_group, lattice, "npfem_ibm_interpolate")) return rc;
    if (!x || !u_lattice || !u_vertex) return set_error(NPFEM_ERR_INVALID_ARG, "npfem_ibm_interpolate: null array");
    if (a.total_verts == 0) return 0;
    DevGuard guard(meshes[0]->device);
    a.x = x;
    a.field = u_lattice;
    a.out = u_vertex;
    a.phase = -1;
    ibm_forcing_kernel<<<ibm_grid(meshes[0], a.total_verts), 256, 0, static_cast<cudaStream_t>(stream)>>>(a);
    count_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 0 : launch_err("npfem_ibm_interpolate", e);
}

extern "C" int npfem_ibm_forcing(npfem_handle* const* meshes, int n_groups, const int32_t* cells_per_group,
                                 const float* x, const float* u_vertex, const npfem_lattice* lattice,
                                 const float* u_lattice, double dt_fluid, int cycles, float* f_vertex, float* f_lattice,
                                 void* stream)
{
    IbmArgs a;
    if (int rc = fill_ibm(&a, meshes, n_groups, cells_per_group, lattice, "npfem_ibm_forcing")) return rc;
    if (!x || !u_vertex || !u_lattice || !f_vertex || !f_lattice || !(dt_fluid > 0.0) || cycles < 0 || cycles > 1000)
        return set_error(NPFEM_ERR_INVALID_ARG, "npfem_ibm_forcing: null array, dt <= 0 or cycles outside 0..1000");
    DevGuard guard(meshes[0]->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t lat_bytes = (size_t)lattice->nx * lattice->ny * lattice->nz * 4 * sizeof(float);
    a.x = x;
    a.uvert = u_vertex;
    a.field = u_lattice;
    a.field2 = f_lattice;
    a.out = f_vertex;
    a.lat_out = f_lattice;
    a.dt = (float)dt_fluid;
    const int grid = ibm_grid(meshes[0], a.total_verts);
    cudaError_t e = cudaSuccess;
    auto run = [&](int phase) {
        a.phase = phase;
        if (a.total_verts > 0) {
            ibm_forcing_kernel<<<grid, 256, 0, s>>>(a);
            count_launch();
        }
        return cudaGetLastError();
    };
    e = run(0);  // Step 0: f_0 = (U - u*(X)) / dt
    for (int l = 0; l < cycles && e == cudaSuccess; ++l) {
        e = cudaMemsetAsync(f_lattice, 0, lat_bytes, s);
        if (e == cudaSuccess) e = run(1);  // Step 1: spread f_l
        if (e == cudaSuccess) e = run(2);  // Steps 2-4: f_{l+1} = f_l + (U - u_l(X)) / dt
    }
    // f_imm: the spread of the final Lagrangian force
    if (e == cudaSuccess) e = cudaMemsetAsync(f_lattice, 0, lat_bytes, s);
    if (e == cudaSuccess) e = run(1);
    return e == cudaSuccess ? 0 : launch_err("npfem_ibm_forcing", e);
}
