// CUDA-graph capture of consecutive time steps (npfem_graph_*): the per-step host work
// (argument set-up, launch configuration) runs once at capture; a replay enqueues the
// warm-start, cluster and idle-SM launches of every captured step as one graph.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "npfem_internal.h"

struct npfem_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int device = 0;
    unsigned long long kernels = 0;  // kernel launches one replay performs
};

using namespace npfem;

extern "C" {

int npfem_graph_create(npfem_handle* const* meshes, int n_groups, const int32_t* cells_per_group, void* x, void* v,
                       const void* f_ext, double dt, int steps, npfem_cell_stats* stats, npfem_graph** out)
{
    if (!out || steps < 1 || !meshes || n_groups < 1 || n_groups > kMaxGroups || !cells_per_group || !meshes[0])
        return set_error(NPFEM_ERR_INVALID_ARG, "npfem_graph_create: bad argument");
    *out = nullptr;
    int dev_prev = 0;
    cudaGetDevice(&dev_prev);
    cudaSetDevice(meshes[0]->device);
    size_t elems = 0;
    for (int g = 0; g < n_groups; ++g) {
        if (!meshes[g] || cells_per_group[g] < 0) {
            cudaSetDevice(dev_prev);
            return set_error(NPFEM_ERR_INVALID_ARG, "npfem_graph_create: bad mesh handle or cell count");
        }
        elems += (size_t)3 * meshes[g]->n * cells_per_group[g];
    }
    const size_t bytes = elems * (meshes[0]->precision == NPFEM_PREC_FP64 ? 8 : 4);
    // work already queued on the handles (any stream) uses their work counters: let it
    // finish before the trial step runs on the internal stream
    cudaDeviceSynchronize();
    cudaStream_t s = nullptr;
    void *tx = nullptr, *tv = nullptr;
    npfem_graph* G = new npfem_graph();
    G->device = meshes[0]->device;
    int rc = 0;
    auto cuda_fail = [&](cudaError_t e, const char* what) {
        rc = set_error(e == cudaErrorMemoryAllocation ? NPFEM_ERR_OOM : NPFEM_ERR_CUDA,
                       std::string("npfem_graph_create: ") + what + ": " + cudaGetErrorString(e));
    };
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) cuda_fail(e, "stream");
    // two steps on copies: size every buffer the captured steps use (the second one
    // runs with the temporal warm start, whose launches the first call does not make)
    if (!rc && bytes > 0) {
        e = cudaMalloc(&tx, bytes);
        if (e == cudaSuccess) e = cudaMalloc(&tv, bytes);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tx, x, bytes, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tv, v, bytes, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) cuda_fail(e, "trial buffers");
    }
    // the trial step records no kernel-timing events (those belong to the captured steps)
    const int tev_used = meshes[0]->tev_used;
    meshes[0]->tev_used = (int)meshes[0]->tev.size();
    for (int k = 0; k < 2 && !rc; ++k)
        rc = npfem_step(meshes, n_groups, cells_per_group, bytes ? tx : x, bytes ? tv : v, f_ext, dt, s, stats);
    meshes[0]->tev_used = tev_used;
    if (!rc) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) cuda_fail(e, "trial step");
    }
    if (tx) cudaFree(tx);
    if (tv) cudaFree(tv);
    if (!rc) {
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) cuda_fail(e, "begin capture");
    }
    if (!rc) {
        const unsigned long long k0 = npfem_launch_count();
        for (int k = 0; k < steps && !rc; ++k)
            rc = npfem_step(meshes, n_groups, cells_per_group, x, v, f_ext, dt, s, stats);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(s, &graph);
        if (!rc && e != cudaSuccess) cuda_fail(e, "end capture");
        G->kernels = npfem_launch_count() - k0;
        if (!rc) {
            G->graph = graph;
            e = cudaGraphInstantiate(&G->exec, graph, 0);
            if (e != cudaSuccess) cuda_fail(e, "instantiate");
        } else if (graph) {
            cudaGraphDestroy(graph);
        }
    }
    if (s) cudaStreamDestroy(s);
    cudaSetDevice(dev_prev);
    if (rc) {
        npfem_graph_destroy(G);
        return rc;
    }
    *out = G;
    return 0;
}

int npfem_graph_launch(npfem_graph* g, void* stream)
{
    if (!g || !g->exec) return set_error(NPFEM_ERR_INVALID_ARG, "npfem_graph_launch: null graph");
    int dev_prev = 0;
    cudaGetDevice(&dev_prev);
    cudaSetDevice(g->device);
    cudaError_t e = cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream));
    cudaSetDevice(dev_prev);
    if (e != cudaSuccess) return set_error(NPFEM_ERR_CUDA, std::string("npfem_graph_launch: ") + cudaGetErrorString(e));
    count_launch(g->kernels);
    return 0;
}

int npfem_graph_destroy(npfem_graph* g)
{
    if (!g) return set_error(NPFEM_ERR_INVALID_ARG, "npfem_graph_destroy: null graph");
    int dev_prev = 0;
    cudaGetDevice(&dev_prev);
    cudaSetDevice(g->device);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    cudaSetDevice(dev_prev);
    delete g;
    return 0;
}

}  // extern "C"
