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
#include <mutex>
#include <string>

#include "npfem_internal.h"

#define NPFEM_STATIC_SCRATCH_BYTES (32u << 20)  // 32 MiB per device
#define NPFEM_STATIC_COUNTER_BYTES 256u         // work counters, then per-block slots

static __device__ __align__(256) unsigned char g_npfem_static_scratch[NPFEM_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 256;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices];  // device address of the array, per device

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

// One-time set-up per device, run with that device current: look up the device
// address of the array (a host-side reference to it is not a device pointer).
int static_base(int device, char** out)
{
    if (device < 0 || device >= kMaxDevices) return npfem::set_error(NPFEM_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_npfem_static_scratch);
        if (e != cudaSuccess || !p)
            return npfem::set_error(NPFEM_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch: ") +
                                                        cudaGetErrorString(e));
        g_static_addr[device] = p;
    }
    *out = static_cast<char*>(g_static_addr[device]);
    return 0;
}

template <typename T>
int run_static(npfem_handle* const* meshes, int n_groups, const int32_t* cells, T* x, T* v, const T* f,
               npfem_cell_stats* stats, char* base, cudaStream_t stream)
{
    using namespace npfem;
    npfem_handle* h0 = meshes[0];
    LaunchArgs<T> a;
    memset(&a, 0, sizeof(a));
    long long total = 0, state = 0, slot = 0;
    int smem_max = 0;
    const int budget = h0->smem_optin - kFixedSmem - 1024;
    for (int gi = 0; gi < n_groups; ++gi) {
        npfem_handle* h = meshes[gi];
        GroupDesc<T>& g = a.g[gi];
        g.topo = *reinterpret_cast<const TopoDev<T>*>(sizeof(T) == 4 ? (const void*)&h->tf : (const void*)&h->td);
        g.cell_begin = total;
        g.state_off = state;
        g.cells = cells[gi];
        long long sb = 0;
        place_vectors(&g, h->n_pad, h->nt, h0->opts.lbfgs_m, budget, &sb);
        slot = std::max(slot, sb);
        smem_max = std::max(smem_max, g.smem_bytes);
        total += cells[gi];
        state += 3LL * h->n * cells[gi];
    }
    if (total == 0) return 0;
    const long long capacity = (long long)NPFEM_STATIC_SCRATCH_BYTES - NPFEM_STATIC_COUNTER_BYTES;
    if (slot > capacity)
        return set_error(NPFEM_ERR_INVALID_ARG,
                         "npfem_step_static: one block needs " + std::to_string(slot) +
                             " bytes of scratch, more than the static array's " + std::to_string(capacity) +
                             " bytes (mesh too large for the allocation-free path)");
    a.n_groups = n_groups;
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

    const int smem = kFixedSmem + smem_max;
    const int per_sm = smem > h0->smem_optin / 2 ? 1 : (smem > h0->smem_optin / 3 ? 2 : 3);
    long long grid = std::min<long long>(total, (long long)h0->sm_count * per_sm);
    if (slot > 0) grid = std::min<long long>(grid, capacity / slot);  // fewer persistent blocks, same result
    cudaError_t e = set_cell_kernel_smem<T>(smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(base, 0, NPFEM_STATIC_COUNTER_BYTES, stream);
    if (e == cudaSuccess) e = launch_cells<T>(a, (int)grid, h0->threads, smem, stream);
    if (e != cudaSuccess) return set_error(NPFEM_ERR_CUDA, std::string("npfem_step_static: ") + cudaGetErrorString(e));
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
    if (int rc = static_base(meshes[0]->device, &base)) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (meshes[0]->precision == NPFEM_PREC_FP64)
        return run_static<double>(meshes, n_groups, cells_per_group, (double*)x, (double*)v, (const double*)f_ext, stats,
                                  base, s);
    return run_static<float>(meshes, n_groups, cells_per_group, (float*)x, (float*)v, (const float*)f_ext, stats, base,
                             s);
}
