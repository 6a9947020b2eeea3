// Collision detection of Sec. 3.3 (Proof of capability): for every membrane vertex,
// the nearest vertex of another cell within a cutoff and the tangent plane of that
// cell there.  The solver then adds, for every vertex that lies behind its plane,
// the collision energy (w_col/2)|p_i - x_i|^2 with p_i the vertex moved onto the
// plane; the test is repeated at every evaluation, so the term vanishes as soon as
// the vertex no longer penetrates (evaluate() in npfem_solver.cu).
//
// Detection replaces the paper's two stages (Palabos' fluid-cell lists, then a k-d
// tree per body) by one uniform grid of bins of the cutoff's size, stored as a hash
// table with a fixed number of slots per bucket: one launch inserts every vertex
// (atomic slot counters), one launch scans, for every vertex, the 27 bins around it.
// Hash collisions only add candidates (each is tested by distance); a full bucket
// drops the vertex from the table and is counted, so the caller can tell.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "npfem_device.cuh"
#include "npfem_internal.h"

namespace npfem {
namespace {

constexpr int kSlots = 16;  // vertices per hash bucket

struct ColGroup {
    TopoDev<float> topo;
    long long vert_begin;  // first global vertex of the group
    long long cell_begin;  // first global cell of the group
    long long state_off;   // element offset of the group's first cell in x
};

struct ColArgs {
    ColGroup g[kMaxGroups];
    int n_groups;
    long long total_verts;
    const float* x;
    float inv_cut, cut2;
    unsigned mask;          // buckets - 1 (a power of two)
    unsigned* counts;       // [buckets]
    unsigned* slots;        // [buckets][kSlots] global vertex indices
    unsigned* stats;        // [0] vertices with a neighbour, [1] vertices dropped by a full bucket
    float4* planes;         // [total_verts] (n, offset relative to the cell's vertex 0)
};

__device__ __forceinline__ const ColGroup& col_locate(const ColArgs& a, long long gv, long long* cell, int* vert)
{
    int gi = 0;
    while (gi + 1 < a.n_groups && gv >= a.g[gi + 1].vert_begin) ++gi;
    const ColGroup& G = a.g[gi];
    const long long local = gv - G.vert_begin;
    const long long c = local / G.topo.n;
    *cell = c;
    *vert = (int)(local - c * G.topo.n);
    return G;
}

__device__ __forceinline__ void col_pos(const ColArgs& a, const ColGroup& G, long long cell, int i, float p[3])
{
    const int n = G.topo.n;
    const float* xc = a.x + G.state_off + cell * 3LL * n;
    p[0] = xc[i];
    p[1] = xc[n + i];
    p[2] = xc[2 * n + i];
}

__device__ __forceinline__ int bin_of(float v, float inv_cut)
{
    const float b = floorf(v * inv_cut);
    return (int)fminf(fmaxf(b, -1.0e7f), 1.0e7f);  // far or non-finite positions share an end bin
}

__device__ __forceinline__ unsigned bucket(int bx, int by, int bz, unsigned mask)
{
    return ((unsigned)bx * 73856093u ^ (unsigned)by * 19349663u ^ (unsigned)bz * 83492791u) & mask;
}

__global__ void __launch_bounds__(256) col_insert_kernel(const __grid_constant__ ColArgs a)
{
    for (long long gv = blockIdx.x * (long long)blockDim.x + threadIdx.x; gv < a.total_verts;
         gv += (long long)gridDim.x * blockDim.x) {
        long long cell;
        int i;
        const ColGroup& G = col_locate(a, gv, &cell, &i);
        float p[3];
        col_pos(a, G, cell, i, p);
        const unsigned b = bucket(bin_of(p[0], a.inv_cut), bin_of(p[1], a.inv_cut), bin_of(p[2], a.inv_cut), a.mask);
        const unsigned s = atomicAdd(&a.counts[b], 1u);
        if (s < (unsigned)kSlots)
            a.slots[(size_t)b * kSlots + s] = (unsigned)gv;
        else
            atomicAdd(&a.stats[1], 1u);
    }
}

__global__ void __launch_bounds__(256) col_query_kernel(const __grid_constant__ ColArgs a)
{
    for (long long gv = blockIdx.x * (long long)blockDim.x + threadIdx.x; gv < a.total_verts;
         gv += (long long)gridDim.x * blockDim.x) {
        long long cell;
        int i;
        const ColGroup& G = col_locate(a, gv, &cell, &i);
        const long long my_cell = G.cell_begin + cell;
        float p[3];
        col_pos(a, G, cell, i, p);
        const int bx = bin_of(p[0], a.inv_cut), by = bin_of(p[1], a.inv_cut), bz = bin_of(p[2], a.inv_cut);
        float best = INFINITY;
        long long bj = -1;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const unsigned b = bucket(bx + dx, by + dy, bz + dz, a.mask);
                    const unsigned cnt = min(a.counts[b], (unsigned)kSlots);
                    for (unsigned s = 0; s < cnt; ++s) {
                        const long long j = a.slots[(size_t)b * kSlots + s];
                        long long jc;
                        int jv;
                        const ColGroup& H = col_locate(a, j, &jc, &jv);
                        if (H.cell_begin + jc == my_cell) continue;
                        float q[3];
                        col_pos(a, H, jc, jv, q);
                        const float e0 = q[0] - p[0], e1 = q[1] - p[1], e2 = q[2] - p[2];
                        const float d2 = e0 * e0 + e1 * e1 + e2 * e2;
                        if (d2 <= a.cut2 && (d2 < best || (d2 == best && j < bj))) {
                            best = d2;
                            bj = j;
                        }
                    }
                }
        float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
        if (bj >= 0) {
            long long jc;
            int jv;
            const ColGroup& H = col_locate(a, bj, &jc, &jv);
            const float* xb = a.x + H.state_off + jc * 3LL * H.topo.n;
            float A, nv[3];
            vertex_area_normal(H.topo, xb, jv, &A, nv);
            float q[3], o[3];
            col_pos(a, H, jc, jv, q);
            col_pos(a, G, cell, 0, o);  // the plane offset relative to this cell's vertex 0
            out = make_float4(nv[0], nv[1], nv[2], nv[0] * (q[0] - o[0]) + nv[1] * (q[1] - o[1]) + nv[2] * (q[2] - o[2]));
            atomicAdd(&a.stats[0], 1u);
        }
        a.planes[gv] = out;
    }
}

}  // namespace
}  // namespace npfem

using namespace npfem;

extern "C" int npfem_collision_detect(npfem_handle* const* meshes, int n_groups, const int32_t* cells_per_group,
                                      const float* x, double cutoff, float* planes, unsigned int* stats, void* stream)
{
    if (!meshes || n_groups < 1 || n_groups > kMaxGroups || !cells_per_group || !x || !planes || !stats ||
        !(cutoff > 0.0) || !std::isfinite(cutoff))
        return set_error(NPFEM_ERR_INVALID_ARG, "npfem_collision_detect: null argument, bad group count or cutoff <= 0");
    ColArgs a;
    memset(&a, 0, sizeof(a));
    long long v = 0, c = 0, st = 0;
    for (int g = 0; g < n_groups; ++g) {
        npfem_handle* h = meshes[g];
        if (!h || cells_per_group[g] < 0 || h->precision == NPFEM_PREC_FP64 || h->device != meshes[0]->device)
            return set_error(NPFEM_ERR_INVALID_ARG, "npfem_collision_detect: FP32-state handles of one device only");
        a.g[g].topo = h->tf;
        a.g[g].vert_begin = v;
        a.g[g].cell_begin = c;
        a.g[g].state_off = st;
        v += (long long)h->n * cells_per_group[g];
        c += cells_per_group[g];
        st += 3LL * h->n * cells_per_group[g];
    }
    if (v >= (1LL << 32) - 1) return set_error(NPFEM_ERR_INVALID_ARG, "npfem_collision_detect: too many vertices");
    a.n_groups = n_groups;
    a.total_verts = v;
    a.x = x;
    a.inv_cut = (float)(1.0 / cutoff);
    a.cut2 = (float)(cutoff * cutoff);
    a.planes = reinterpret_cast<float4*>(planes);
    a.stats = stats;
    npfem_handle* h0 = meshes[0];
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != h0->device) cudaSetDevice(h0->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // buckets: a power of two of at least twice the vertices
    size_t buckets = 1024;
    while (buckets < 2 * (size_t)std::max<long long>(v, 1)) buckets <<= 1;
    const size_t need = buckets * (1 + kSlots);
    int rc = 0;
    cudaError_t e = cudaSuccess;
    {
        std::lock_guard<std::mutex> lk(h0->mu);
        if (need > h0->col_table_len) {
            if (h0->col_table) {
                e = cudaStreamSynchronize(s);
                cudaFree(h0->col_table);
                h0->col_table = nullptr;
                h0->col_table_len = 0;
            }
            if (e == cudaSuccess) e = cudaMalloc(&h0->col_table, need * sizeof(unsigned));
            if (e == cudaSuccess) h0->col_table_len = need;
        }
        a.mask = (unsigned)(buckets - 1);
        a.counts = h0->col_table;
        a.slots = h0->col_table + buckets;
        if (e == cudaSuccess) e = cudaMemsetAsync(a.counts, 0, buckets * sizeof(unsigned), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(stats, 0, 2 * sizeof(unsigned), s);
        if (e == cudaSuccess && v > 0) {
            const int grid = (int)std::max<long long>(1, std::min<long long>((v + 255) / 256, (long long)h0->sm_count * 8));
            col_insert_kernel<<<grid, 256, 0, s>>>(a);
            count_launch();
            col_query_kernel<<<grid, 256, 0, s>>>(a);
            count_launch();
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess)
        rc = set_error(e == cudaErrorMemoryAllocation ? NPFEM_ERR_OOM : NPFEM_ERR_CUDA,
                       std::string("npfem_collision_detect: ") + cudaGetErrorString(e));
    if (prev >= 0 && prev != h0->device) cudaSetDevice(prev);
    return rc;
}

extern "C" int npfem_set_collisions(npfem_handle* h, const float* planes, double w_col)
{
    if (!h || !(w_col >= 0.0) || !std::isfinite(w_col))
        return set_error(NPFEM_ERR_INVALID_ARG, "npfem_set_collisions: null handle or w_col < 0");
    std::lock_guard<std::mutex> lk(h->mu);
    h->col_planes = planes && w_col > 0.0 ? planes : nullptr;
    h->col_w = planes ? w_col : 0.0;
    return 0;
}
