// npfem_step_static: the time step of npfem_step without any device allocation.
//
// Who needs it: callers that must not allocate device memory while they step.
// A coupled flow solver, for instance, often hands the whole GPU to its own
// caching pool at start-up, so a raw cudaMalloc from this library can fail even
// though the caller has memory to spare; and cudaMalloc/cudaFree synchronise the
// device, which stalls a time loop that keeps several streams busy.  npfem_step
// may grow a library-owned scratch buffer on the first call that needs it (meshes
// whose solver vectors do not all fit in shared memory); this entry point never
// does.  Its scratch is a fixed array compiled into the library instead.
//
// The array lives in every GPU that loads the library until the process exits.
// All calls on a device share it and it keeps the previous call's contents; the
// two work counters at its start are cleared on the stream before every launch.
// Calls whose kernels overlap on the GPU (different streams, or host threads that
// do not order their streams) race on the array and must be avoided.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "npfem_internal.h"

#define NPFEM_STATIC_SCRATCH_BYTES (32u << 20)  // 32 MiB per device
#define NPFEM_STATIC_COUNTER_BYTES 256u         // work counters, then per-block slots

static __device__ __align__(256) unsigned char g_npfem_static_scratch[NPFEM_STATIC_SCRATCH_BYTES];

namespace {

struct CurrentDevice {
    int prev = -1;
    explicit CurrentDevice(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~CurrentDevice()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Device address of the array on the current device (a host-side reference to it is
// not a device pointer).  Looked up on every call: the lookup allocates nothing, and
// an address kept from an earlier context would be stale after a device reset.
int static_base(char** out)
{
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_npfem_static_scratch);
    if (e != cudaSuccess || !p)
        return npfem::set_error(NPFEM_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch: ") +
                                                    cudaGetErrorString(e));
    *out = static_cast<char*>(p);
    return 0;
}

// One persistent SIMT launch over the groups `sel` (all of one block size), with the
// groups' offsets into the caller's state and stats arrays.
template <typename T>
int run_static(npfem_handle* const* meshes, const std::vector<int>& sel, const int32_t* cells,
               const std::vector<long long>& soff, const std::vector<long long>& coff, int threads, T* x, T* v,
               const T* f, npfem_cell_stats* stats, char* base, cudaStream_t stream)
{
    using namespace npfem;
    npfem_handle* h0 = meshes[sel[0]];
    LaunchArgs<T> a;
    memset(&a, 0, sizeof(a));
    long long total = 0, slot = 0;
    int smem_max = 0;
    const int budget = h0->smem_optin - kFixedSmem - 1024;
    int ng = 0;
    for (int gi : sel) {
        npfem_handle* h = meshes[gi];
        GroupDesc<T>& g = a.g[ng++];
        g.topo = *reinterpret_cast<const TopoDev<T>*>(sizeof(T) == 4 ? (const void*)&h->tf : (const void*)&h->td);
        g.cell_begin = total;
        g.state_off = soff[gi];
        g.stats_off = coff[gi];
        g.cells = cells[gi];
        long long sb = 0;
        place_vectors(&g, h->n_pad, h->nt, h0->opts.lbfgs_m, budget, &sb);
        slot = std::max(slot, sb);
        smem_max = std::max(smem_max, g.smem_bytes);
        total += cells[gi];
    }
    if (total == 0) return 0;
    const long long capacity = (long long)NPFEM_STATIC_SCRATCH_BYTES - NPFEM_STATIC_COUNTER_BYTES;
    if (slot > capacity)
        return set_error(NPFEM_ERR_INVALID_ARG,
                         "npfem_step_static: one block needs " + std::to_string(slot) +
                             " bytes of scratch, more than the static array's " + std::to_string(capacity) +
                             " bytes (mesh too large for the allocation-free path)");
    a.n_groups = ng;
    a.total_cells = total;
    a.x = x;
    a.v = v;
    a.f = f;
    a.stats = stats;
    a.work = reinterpret_cast<unsigned int*>(base);
    a.scratch = slot > 0 ? base + NPFEM_STATIC_COUNTER_BYTES : nullptr;
    a.slot_bytes = slot;
    set_solver_params(&a.p, h0->opts);
    a.p.mode = 0;
    a.p.contraction = CONTRACT_SIMT;
    if (meshes[0]->col_planes) {
        a.col = reinterpret_cast<const float4*>(meshes[0]->col_planes);
        a.col_w = (T)meshes[0]->col_w;
    }

    const int smem = kFixedSmem + smem_max;
    cudaError_t e = set_cell_kernel_smem<T>(smem);
    int per_sm = 1;
    if (e == cudaSuccess) e = cells_per_sm<T>(threads, smem, &per_sm);
    if (e != cudaSuccess) return set_error(NPFEM_ERR_CUDA, std::string("npfem_step_static: ") + cudaGetErrorString(e));
    per_sm = std::max(per_sm, 1);
    long long grid = std::min<long long>(total, (long long)h0->sm_count * per_sm);
    if (slot > 0) grid = std::min<long long>(grid, capacity / slot);  // fewer persistent blocks, same result
    e = cudaMemsetAsync(base, 0, NPFEM_STATIC_COUNTER_BYTES, stream);
    if (e == cudaSuccess) e = launch_cells<T>(a, (int)grid, threads, smem, stream);
    if (e != cudaSuccess) return set_error(NPFEM_ERR_CUDA, std::string("npfem_step_static: ") + cudaGetErrorString(e));
    return 0;
}

// The groups in launches of one block size each (the tuned SIMT block size of every
// handle; 512 threads for FP64), in the order npfem_step launches its SIMT groups.
template <typename T>
int step_static(npfem_handle* const* meshes, int n_groups, const int32_t* cells, T* x, T* v, const T* f,
                npfem_cell_stats* stats, char* base, cudaStream_t stream)
{
    std::vector<long long> soff(n_groups), coff(n_groups);
    long long st = 0, ct = 0;
    for (int g = 0; g < n_groups; ++g) {
        soff[g] = st;
        coff[g] = ct;
        st += 3LL * meshes[g]->n * cells[g];
        ct += cells[g];
    }
    std::vector<char> done(n_groups, 0);
    for (int g0 = 0; g0 < n_groups; ++g0) {
        if (done[g0]) continue;
        const int threads = sizeof(T) == 8 ? 512 : meshes[g0]->threads;
        std::vector<int> sel;
        for (int g = g0; g < n_groups; ++g) {
            if (done[g] || (sizeof(T) == 4 && meshes[g]->threads != threads)) continue;
            sel.push_back(g);
            done[g] = 1;
        }
        if (int rc = run_static<T>(meshes, sel, cells, soff, coff, threads, x, v, f, stats, base, stream)) return rc;
    }
    return 0;
}

}  // namespace

extern "C" int npfem_step_static(npfem_handle* const* meshes, int n_groups, const int32_t* cells_per_group, void* x,
                                 void* v, const void* f_ext, double dt, void* stream, npfem_cell_stats* stats)
{
    if (!meshes || n_groups < 1 || n_groups > npfem::kMaxGroups || !cells_per_group || !x || !v || !f_ext)
        return npfem::set_error(NPFEM_ERR_INVALID_ARG, "npfem_step_static: null argument or bad group count");
    for (int g = 0; g < n_groups; ++g) {
        if (!meshes[g] || cells_per_group[g] < 0)
            return npfem::set_error(NPFEM_ERR_INVALID_ARG, "npfem_step_static: null handle or negative cell count");
        if (meshes[g]->device != meshes[0]->device || meshes[g]->precision != meshes[0]->precision ||
            meshes[g]->dt != meshes[0]->dt)
            return npfem::set_error(NPFEM_ERR_INVALID_ARG, "all handles of one call must share device, precision and dt");
    }
    if (dt != meshes[0]->dt) return npfem::set_error(NPFEM_ERR_INVALID_ARG, "dt differs from the handle's dt");
    CurrentDevice guard(meshes[0]->device);
    char* base = nullptr;
    if (int rc = static_base(&base)) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (meshes[0]->precision == NPFEM_PREC_FP64)
        return step_static<double>(meshes, n_groups, cells_per_group, (double*)x, (double*)v, (const double*)f_ext,
                                   stats, base, s);
    return step_static<float>(meshes, n_groups, cells_per_group, (float*)x, (float*)v, (const float*)f_ext, stats, base,
                              s);
}
