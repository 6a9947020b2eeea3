// C ABI of libnpfem.so (declared in include/npfem.h): handle set-up, placement of the
// per-cell solver vectors in shared or global memory, and the launches.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "npfem_internal.h"

using namespace npfem;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg)
{
    g_last_error = msg;
    return code;
}

}  // namespace

int npfem::set_error(int code, const std::string& msg) { return fail(code, msg); }

namespace npfem {
std::atomic<unsigned long long> g_launches{0};
void count_launch(unsigned long long k) { g_launches.fetch_add(k); }
}  // namespace npfem

namespace {

#define NPFEM_CUDA(call)                                                                               \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return fail(e_ == cudaErrorMemoryAllocation ? NPFEM_ERR_OOM : NPFEM_ERR_CUDA,              \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                           \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace


namespace {

template <typename X, typename S>
int upload(npfem_handle* h, const std::vector<S>& src, const X** out)
{
    int err = 0;
    std::vector<X> tmp(src.size());
    for (size_t i = 0; i < src.size(); ++i) tmp[i] = (X)src[i];
    X* d = h->alloc<X>(std::max<size_t>(tmp.size(), 1), &err);
    if (!d) return err;
    if (!tmp.empty()) NPFEM_CUDA(cudaMemcpy(d, tmp.data(), tmp.size() * sizeof(X), cudaMemcpyHostToDevice));
    *out = d;
    return 0;
}

template <typename T>
int fill_topo(npfem_handle* h, TopoDev<T>* tp, const void* ainv, const void* minv)
{
    const HostTopo& H = h->host;
    int rc;
    std::vector<unsigned short> tri4(4 * (size_t)H.nt, 0);
    for (int t = 0; t < H.nt; ++t)
        for (int a = 0; a < 3; ++a) tri4[4 * t + a] = (unsigned short)H.tri[3 * t + a];
    const unsigned short* dtri = nullptr;
    if ((rc = upload(h, tri4, &dtri))) return rc;
    tp->tri = reinterpret_cast<const ushort4*>(dtri);
    if ((rc = upload(h, H.dminv, &tp->dminv))) return rc;
    if ((rc = upload(h, H.W, &tp->W))) return rc;
    if ((rc = upload(h, H.mass, &tp->mass))) return rc;
    std::vector<double> inv_m(H.n);
    for (int i = 0; i < H.n; ++i) inv_m[i] = 1.0 / H.mass[i];
    if ((rc = upload(h, inv_m, &tp->inv_mass))) return rc;
    if ((rc = upload(h, H.bend_w, &tp->bend_w))) return rc;
    if ((rc = upload(h, H.dg_norm, &tp->dg_norm))) return rc;
    if ((rc = upload(h, H.csum, &tp->csum))) return rc;
    if ((rc = upload(h, H.nsign, &tp->nsign))) return rc;
    if ((rc = upload(h, H.ring_ptr, &tp->ring_ptr))) return rc;
    std::vector<unsigned short> ridx(H.ring_idx.begin(), H.ring_idx.end());
    if ((rc = upload(h, ridx, &tp->ring_idx))) return rc;
    if ((rc = upload(h, H.ring_c, &tp->ring_c))) return rc;
    if ((rc = upload(h, H.ring_ct, &tp->ring_ct))) return rc;
    if ((rc = upload(h, H.rest_c, &tp->rest_c))) return rc;
    tp->mlp = nullptr;
    tp->tmlp = nullptr;
    if ((rc = upload(h, H.inc_ptr, &tp->inc_ptr))) return rc;
    std::vector<unsigned> incu(H.inc_idx.begin(), H.inc_idx.end());
    if ((rc = upload(h, incu, &tp->inc_idx))) return rc;
    // Fixed-width tables: each vertex's one-ring in cyclic order r_0 .. r_{v-1} (v <= 8)
    // so that triangle (i, r_q, r_{q+1 mod v}) is incident triangle q of vertex i, in
    // the mesh's orientation.  Needs every one-ring to be one cycle of at most 8.
    std::vector<std::vector<int>> cyc(H.n);
    bool ok8 = true;
    {
        std::vector<std::vector<std::pair<int, int>>> nxt(H.n);  // (j, k) for triangles (i, j, k)
        for (int t = 0; t < H.nt; ++t)
            for (int a = 0; a < 3; ++a)
                nxt[H.tri[3 * t + a]].push_back({H.tri[3 * t + (a + 1) % 3], H.tri[3 * t + (a + 2) % 3]});
        for (int i = 0; i < H.n && ok8; ++i) {
            const int v = (int)nxt[i].size();
            if (v > 8 || v != H.ring_ptr[i + 1] - H.ring_ptr[i]) {
                ok8 = false;
                break;
            }
            int j = nxt[i][0].first;
            for (int q = 0; q < v; ++q) {
                cyc[i].push_back(j);
                int k = -1;
                for (const auto& e : nxt[i])
                    if (e.first == j) k = e.second;
                if (k < 0) {
                    ok8 = false;
                    break;
                }
                j = k;
            }
            if (ok8 && j != nxt[i][0].first) ok8 = false;
            if (ok8) {
                std::vector<int> sc(cyc[i]);
                std::sort(sc.begin(), sc.end());
                ok8 = std::adjacent_find(sc.begin(), sc.end()) == sc.end();
            }
        }
    }
    tp->k8 = ok8 ? 1 : 0;
    tp->ring8_idx = nullptr;
    tp->ring8_c = tp->ring8_ct = nullptr;
    if (tp->k8) {
        std::vector<unsigned short> r8(8 * (size_t)H.n);
        std::vector<double> c8(8 * (size_t)H.n, 0.0), ct8(8 * (size_t)H.n, 0.0);
        for (int i = 0; i < H.n; ++i) {
            for (int q = 0; q < 8; ++q) r8[8 * i + q] = (unsigned short)i;
            for (int q = 0; q < (int)cyc[i].size(); ++q) {
                const int j = cyc[i][q];
                r8[8 * i + q] = (unsigned short)j;
                for (int p = H.ring_ptr[i]; p < H.ring_ptr[i + 1]; ++p)
                    if (H.ring_idx[p] == j) {
                        c8[8 * i + q] = H.ring_c[p];
                        ct8[8 * i + q] = H.ring_ct[p];
                    }
            }
        }
        // slot of each triangle corner in its vertex's cyclic ring, packed 3 bits per
        // corner into the fourth component of the triangle's index record
        for (int t = 0; t < H.nt; ++t) {
            unsigned packed = 0;
            for (int a = 0; a < 3; ++a) {
                const int i = H.tri[3 * t + a], j = H.tri[3 * t + (a + 1) % 3];
                int slot = 0;
                while (cyc[i][slot] != j) ++slot;
                packed |= (unsigned)slot << (3 * a);
            }
            tri4[4 * t + 3] = (unsigned short)packed;
        }
        NPFEM_CUDA(cudaMemcpy(const_cast<unsigned short*>(dtri), tri4.data(), tri4.size() * sizeof(unsigned short),
                              cudaMemcpyHostToDevice));
        if ((rc = upload(h, r8, &tp->ring8_idx))) return rc;
        if ((rc = upload(h, c8, &tp->ring8_c))) return rc;
        if ((rc = upload(h, ct8, &tp->ring8_ct))) return rc;
    }
    tp->n = H.n;
    tp->nt = H.nt;
    tp->n_pad = h->n_pad;
    tp->nnz = (int)H.ring_idx.size();
    tp->ainv = static_cast<const T*>(ainv);
    tp->minv = static_cast<const T*>(minv);
    tp->l_ptr = nullptr;
    tp->l_idx = nullptr;
    tp->l_val = nullptr;
    tp->beta_h = (T)(h->mat.beta_D / h->dt);
    if (minv) {
        if ((rc = upload(h, H.L_ptr, &tp->l_ptr))) return rc;
        std::vector<unsigned short> lidx(H.L_idx.begin(), H.L_idx.end());
        if ((rc = upload(h, lidx, &tp->l_idx))) return rc;
        if ((rc = upload(h, H.L_val, &tp->l_val))) return rc;
    }
    tp->ainv_lp = nullptr;
    tp->ainv_b16 = nullptr;
    tp->n8 = 0;
    tp->h_ptr = nullptr;
    tp->h_idx = nullptr;
    tp->h_val = nullptr;
    tp->C = (T)h->mat.C;
    tp->B = (T)h->mat.B;
    tp->Dsk = (T)h->mat.D;
    tp->kvol = (T)h->mat.k_vol;
    tp->h = (T)h->dt;
    tp->inv_h2 = (T)(1.0 / (h->dt * h->dt));
    tp->inertia_scale = (T)(1.0 + h->dt * h->mat.alpha_D);
    tp->kappa = (T)h->mat.kappa;
    tp->lbar = (T)H.lbar;
    tp->inv_lbar = (T)(1.0 / H.lbar);
    tp->V0 = H.V0;
    tp->V0hi = (T)H.V0;
    tp->V0lo = (T)(H.V0 - (double)tp->V0hi);
    return 0;
}

int check_opts(const npfem_opts* o)
{
    if (o->precision < NPFEM_PREC_FP64 || o->precision > NPFEM_PREC_BF16)
        return fail(NPFEM_ERR_INVALID_ARG, "opts.precision must be one of NPFEM_PREC_*");
    if (o->lbfgs_m < 0 || o->lbfgs_m > kMaxHistory)
        return fail(NPFEM_ERR_INVALID_ARG, "opts.lbfgs_m must be in 0..8");
    if (o->max_iter < 0 || o->max_halvings < 0 || o->max_halvings > 60)
        return fail(NPFEM_ERR_INVALID_ARG, "opts.max_iter must be >= 0 and max_halvings in 0..60");
    if (!(o->tol >= 0.0) || !(o->c1 > 0.0 && o->c1 < 1.0) || !(o->c2 > o->c1 && o->c2 < 1.0) ||
        !(o->armijo_noise >= 0.0))
        return fail(NPFEM_ERR_INVALID_ARG, "opts: need tol >= 0, 0 < c1 < c2 < 1, armijo_noise >= 0");
    if (o->refine < 0 || o->refine > 1) return fail(NPFEM_ERR_INVALID_ARG, "opts.refine must be 0 or 1");
    if (o->fill_idle_sms < 0 || o->fill_idle_sms > 1)
        return fail(NPFEM_ERR_INVALID_ARG, "opts.fill_idle_sms must be 0 or 1");
    if (o->warm_history < 0 || o->warm_history > 2)
        return fail(NPFEM_ERR_INVALID_ARG, "opts.warm_history must be 0, 1 or 2");
    return 0;
}

template <typename T>
int run_cells(npfem_handle* const* meshes, int n_groups, const int32_t* cells, T* x, T* v, const T* f, const T* y,
              T* grad_out, double* parts, npfem_cell_stats* stats, int mode, cudaStream_t stream,
              const T* u0 = nullptr, const long long* state_offs = nullptr, const long long* stats_offs = nullptr,
              int threads = 0, const T* hist_in = nullptr, T* hist_out = nullptr, long long pos_stride = 0,
              unsigned int* defer = nullptr, int hist_ext = 0, T* carry = nullptr,
              const long long* carry_offs = nullptr)
{
    npfem_handle* h0 = meshes[0];
    LaunchArgs<T> a;
    memset(&a, 0, sizeof(a));
    long long total = 0, state = 0, slot = 0;
    int smem_max = 0;
    // TF32 tensor-core contraction: the A^-1 ring and the B operand sit in front of the
    // per-cell vectors, and every block holds 16 tensor-memory columns per row tile
    const bool tf = sizeof(T) == 4 && mode == 0 && h0->precision == NPFEM_PREC_TF32;
    int tf_kpad = 0, tf_tiles = 0;
    for (int gi = 0; tf && gi < n_groups; ++gi) {
        tf_kpad = std::max(tf_kpad, meshes[gi]->tf.kpad);
        tf_tiles = std::max(tf_tiles, meshes[gi]->tf.rb);
    }
    const int tcb = tf ? tf32_smem_bytes(tf_kpad) : 0;
    const int budget = h0->smem_optin - kFixedSmem - 1024 - tcb;
    for (int gi = 0; gi < n_groups; ++gi) {
        npfem_handle* h = meshes[gi];
        GroupDesc<T>& g = a.g[gi];
        g.topo = *reinterpret_cast<const TopoDev<T>*>(sizeof(T) == 4 ? (const void*)&h->tf : (const void*)&h->td);
        g.cell_begin = total;
        g.state_off = state_offs ? state_offs[gi] : state;
        g.stats_off = stats_offs ? stats_offs[gi] : total;
        g.cells = cells[gi];
        g.carry_rec = carry_rec_elems(h->n_pad, h0->opts.lbfgs_m);
        g.carry_off = carry_offs ? carry_offs[gi] : 0;
        long long sb = 0;
        place_vectors(&g, h->n_pad, h->nt, h0->opts.lbfgs_m, budget, &sb, tcb);
        slot = std::max(slot, sb);
        smem_max = std::max(smem_max, g.smem_bytes);
        total += cells[gi];
        state += 3LL * h->n * cells[gi];
    }
    if (total == 0) return 0;
    a.n_groups = n_groups;
    a.total_cells = total;
    a.x = x;
    a.v = v;
    a.f = f;
    a.y = y;
    a.grad_out = grad_out;
    a.parts = parts;
    a.stats = stats;
    a.work = h0->work;
    set_solver_params(&a.p, h0->opts);
    a.p.mode = mode;
    a.p.contraction = CONTRACT_SIMT;
    int tmem_cols = 0;
    if (tf) {
        a.p.contraction = CONTRACT_TC_TF32;
        a.p.refine = h0->opts.refine;
        a.p.tf_kpad = tf_kpad;
        tmem_cols = 32;
        while (tmem_cols < 16 * tf_tiles) tmem_cols <<= 1;
        if (tmem_cols > 512) return fail(NPFEM_ERR_INVALID_ARG, "TF32 path: mesh too large (more than 32 row tiles)");
        a.p.tmem_cols = tmem_cols;
    }
    a.u0 = u0;
    a.hist_in = hist_in;
    a.hist_out = hist_out;
    a.pos_stride = sizeof(T) == 4 && hist_out ? pos_stride : 0;
    a.hist_ext = sizeof(T) == 4 && hist_out ? hist_ext : 0;
    a.carry = mode == 0 && hist_out ? carry : nullptr;
    a.defer = defer;
    if (mode == 0 && h0->col_planes) {
        a.col = reinterpret_cast<const float4*>(h0->col_planes);
        a.col_w = (T)h0->col_w;
    }

    if (threads <= 0) threads = h0->threads;
    if (sizeof(T) == 8) threads = std::min(threads, 512);
    const int smem = kFixedSmem + smem_max;
    NPFEM_CUDA(set_cell_kernel_smem<T>(smem));
    int per_sm = 1;
    NPFEM_CUDA(cells_per_sm<T>(threads, smem, &per_sm));
    per_sm = std::max(per_sm, 1);
    if (tf) per_sm = std::min(per_sm, 512 / tmem_cols);  // every resident block gets its tensor memory
    long long grid = std::min<long long>(total, (long long)h0->sm_count * per_sm);
    a.slot_bytes = slot;
    if (slot > 0) {
        size_t need = (size_t)slot * (size_t)grid;
        if (need > h0->scratch_bytes) {
            if (h0->scratch) {
                NPFEM_CUDA(cudaStreamSynchronize(stream));
                cudaFree(h0->scratch);
                h0->scratch = nullptr;
                h0->scratch_bytes = 0;
            }
            NPFEM_CUDA(cudaMalloc(&h0->scratch, need));
            h0->scratch_bytes = need;
        }
        a.scratch = h0->scratch;
    }
    NPFEM_CUDA(launch_cells<T>(a, (int)grid, threads, smem, stream));
    return 0;
}

// One tensor-core launch for one mesh group (BF16, n <= kTcMaxVerts).
int run_cells_tc(npfem_handle* h, int cells, float* x, float* v, const float* f, npfem_cell_stats* stats,
                 cudaStream_t stream, const float* u0, const float* hist_in, float* hist_out, long long pos_stride,
                 unsigned int* only, const float* col = nullptr, double col_w = 0.0, int hist_ext = 0,
                 float* carry = nullptr)
{
    if (cells == 0) return 0;
    LaunchArgs<float> a;
    memset(&a, 0, sizeof(a));
    a.hist_ext = hist_out ? hist_ext : 0;
    a.carry = hist_out ? carry : nullptr;
    a.col = reinterpret_cast<const float4*>(col);
    a.col_w = (float)col_w;
    a.u0 = u0;
    a.hist_in = hist_in;
    a.hist_out = hist_out;
    a.pos_stride = hist_out ? pos_stride : 0;
    a.only = only;
    a.need = only ? only + 1 : nullptr;
    GroupDesc<float>& g = a.g[0];
    g.topo = h->tf;
    g.cell_begin = 0;
    g.state_off = 0;
    g.cells = cells;
    g.carry_rec = carry_rec_elems(h->n_pad, h->opts.lbfgs_m);
    g.carry_off = 0;
    const int cluster = h->tf.rb;
    const int ncol = cluster * 3 > 16 ? 32 : 16;
    const int bbytes = (ncol * h->tf.kpad * 2 + 127) & ~127;
    const int budget = h->smem_optin - kFixedSmem - 1024 - bbytes;
    long long slot = 0;
    place_vectors(&g, h->n_pad, h->nt, h->opts.lbfgs_m, budget, &slot, bbytes, true);
    if (g.loc[V_GC] < 0) return fail(NPFEM_ERR_INVALID_ARG, "mesh too large for the tensor-core path's shared memory");
    a.n_groups = 1;
    a.total_cells = cells;
    a.x = x;
    a.v = v;
    a.f = f;
    a.stats = stats;
    a.work = h->work;
    set_solver_params(&a.p, h->opts);
    a.p.mode = 0;
    a.p.contraction = CONTRACT_TC_BF16;
    a.p.cluster = cluster;
    a.p.refine = h->opts.refine;
    // one block per SM: a second block on the SM would wait in the tensor-memory
    // allocation while its cluster waits for it
    int smem = kFixedSmem + g.smem_bytes;
    smem = std::max(smem, h->smem_optin / 2 + 4096);
    if (h->tc_smem != smem) {
        NPFEM_CUDA(query_cells_tc(cluster, kTcThreads, smem, &h->tc_max_clusters));
        h->tc_smem = smem;
    }
    const int max_clusters = h->tc_max_clusters;
    const long long want = std::min<long long>((cells + cluster - 1) / cluster, max_clusters);
    const int grid = (int)(want * cluster);

    // SMs the clusters leave idle (clusters stay within a GPC) run the SIMT kernel on
    // the same work counter: each cell goes to whichever kind of block asks first
    LaunchArgs<float> b;
    long long slot_b = 0;
    int smem_b = 0;
    int helper = h->sm_count - grid;
    if (cells <= grid || h->opts.fill_idle_sms == 0) helper = 0;
    if (helper > 0) {
        b = a;
        place_vectors(&b.g[0], h->n_pad, h->nt, h->opts.lbfgs_m, h->smem_optin - kFixedSmem - 1024, &slot_b);
        b.p.contraction = CONTRACT_SIMT;
        b.p.cluster = 0;
        b.p.refine = 0;
        smem_b = kFixedSmem + b.g[0].smem_bytes;
        if (smem_b <= h->smem_optin / 2) helper = 0;  // would share SMs with the clusters
    }
    a.total_blocks = grid + helper;
    a.slot_bytes = slot;
    const size_t need = (size_t)slot * (size_t)grid + (size_t)slot_b * (size_t)helper;
    if (need > 0) {
        if (need > h->scratch_bytes) {
            if (h->scratch) {
                NPFEM_CUDA(cudaStreamSynchronize(stream));
                cudaFree(h->scratch);
                h->scratch = nullptr;
                h->scratch_bytes = 0;
            }
            NPFEM_CUDA(cudaMalloc(&h->scratch, need));
            h->scratch_bytes = need;
        }
        a.scratch = slot > 0 ? h->scratch : nullptr;
    }
    if (helper > 0) {
        b.total_blocks = a.total_blocks;
        b.claim_top = 1;
        b.reserve = grid;  // about one cell per cluster block: the helper's cells take longer
        b.slot_bytes = slot_b;
        b.scratch = slot_b > 0 ? h->scratch + (size_t)slot * (size_t)grid : nullptr;
        if (!h->side_stream) {
            NPFEM_CUDA(cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking));
            NPFEM_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
            NPFEM_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
        }
        NPFEM_CUDA(cudaEventRecord(h->ev_fork, stream));
    }
    NPFEM_CUDA(launch_cells_tc(a, cluster, kTcThreads, smem, grid, stream));
    if (helper > 0) {
        cudaError_t e = cudaStreamWaitEvent(h->side_stream, h->ev_fork, 0);
        if (e == cudaSuccess) e = set_cell_kernel_smem<float>(smem_b);
        if (e == cudaSuccess) e = launch_cells<float>(b, helper, h->threads, smem_b, h->side_stream);
        if (e != cudaSuccess) {
            // the clusters alone cannot reset the shared counters: clear them behind
            // the launch so that the next step starts clean, and report the failure
            cudaMemsetAsync(h->work, 0, 2 * sizeof(unsigned), stream);
            cudaMemsetAsync(h->work + 3, 0, sizeof(unsigned), stream);
            return fail(NPFEM_ERR_CUDA, std::string("idle-SM launch: ") + cudaGetErrorString(e));
        }
        NPFEM_CUDA(cudaEventRecord(h->ev_join, h->side_stream));
        NPFEM_CUDA(cudaStreamWaitEvent(stream, h->ev_join, 0));
    }
    return 0;
}

// The solver launches of one step: one cluster launch per group that takes the
// tensor-core kernel (BF16, mesh of at most kTcMaxVerts vertices, not tuned away), and
// one persistent SIMT launch per block size over the other groups.
int step_groups(npfem_handle* const* meshes, int n_groups, const int32_t* cells_per_group, void* x, void* v,
                const void* f_ext, cudaStream_t s, npfem_cell_stats* stats, const float* u0, const void* hist_in,
                void* hist_out, long long pos_stride, int hist_ext = 0, void* carry = nullptr)
{
    const int prec = meshes[0]->precision;
    std::vector<long long> soff(n_groups), coff(n_groups), koff(n_groups);
    long long st = 0, ct = 0, kt = 0;
    for (int g = 0; g < n_groups; ++g) {
        soff[g] = st;
        coff[g] = ct;
        koff[g] = kt;
        st += 3LL * meshes[g]->n * cells_per_group[g];
        ct += cells_per_group[g];
        kt += carry_rec_elems(meshes[g]->n_pad, meshes[0]->opts.lbfgs_m) * cells_per_group[g];
    }
    std::vector<char> done(n_groups, 0);
    for (int g = 0; g < n_groups; ++g) {
        if (cells_per_group[g] == 0) {
            done[g] = 1;
            continue;
        }
        if (prec == NPFEM_PREC_BF16 && meshes[g]->n <= kTcMaxVerts && meshes[g]->use_tc) {
            npfem_handle* hg = meshes[g];
            int32_t cg = cells_per_group[g];
            float* xg = (float*)x + soff[g];
            float* vg = (float*)v + soff[g];
            const float* fg = (const float*)f_ext + soff[g];
            npfem_cell_stats* sg = stats ? stats + coff[g] : nullptr;
            const float* hin = hist_in ? (const float*)hist_in + soff[g] : nullptr;
            float* hout = hist_out ? (float*)hist_out + soff[g] : nullptr;
            float* kg = carry ? (float*)carry + koff[g] : nullptr;
            unsigned int* only = nullptr;
            if (hout && (size_t)cg + 3 > hg->defer_len) {
                // allocated with the history (first call of a trajectory), so that the
                // steps that use it allocate nothing (they may be captured in a graph)
                if (hg->defer) {
                    NPFEM_CUDA(cudaStreamSynchronize(s));
                    cudaFree(hg->defer);
                    hg->defer = nullptr;
                    hg->defer_len = 0;
                }
                NPFEM_CUDA(cudaMalloc(&hg->defer, sizeof(unsigned int) * ((size_t)cg + 3)));
                hg->defer_len = (size_t)cg + 3;
                NPFEM_CUDA(cudaMemsetAsync(hg->defer, 0, 3 * sizeof(unsigned int), s));
            }
            if (hin && (size_t)cg + 3 <= hg->defer_len) {
                // along a trajectory many cells are accepted at the first iterate: a SIMT
                // launch on every SM (the clusters' idle SMs included) evaluates each cell
                // there and finishes those, and the cluster kernel takes only the rest
                NPFEM_CUDA(cudaMemcpyAsync(hg->defer + 2, hg->defer + 1, sizeof(unsigned int), cudaMemcpyDeviceToDevice, s));
                NPFEM_CUDA(cudaMemsetAsync(hg->defer, 0, 2 * sizeof(unsigned int), s));
                int rc = run_cells<float>(&hg, 1, &cg, xg, vg, fg, nullptr, nullptr, nullptr, sg, 0, s,
                                          u0 ? u0 + soff[g] : nullptr, nullptr, nullptr, 512, hin, hout, pos_stride,
                                          hg->defer, hist_ext, kg);
                if (rc) return rc;
                only = hg->defer;
            }
            const npfem_handle* hc = meshes[0];
            const float* colg = hc->col_planes ? hc->col_planes + 4 * (soff[g] / 3) : nullptr;
            int rc = run_cells_tc(hg, cg, xg, vg, fg, sg, s, u0 ? u0 + soff[g] : nullptr, hin, hout, pos_stride, only,
                                  colg, hc->col_w, hist_ext, kg);
            if (rc) return rc;
            done[g] = 1;
        }
    }
    for (int g0 = 0; g0 < n_groups; ++g0) {
        if (done[g0]) continue;
        const int threads = prec == NPFEM_PREC_FP64 ? 512 : meshes[g0]->threads;
        std::vector<npfem_handle*> hs;
        std::vector<int32_t> cs;
        std::vector<long long> so, co, ko;
        for (int g = g0; g < n_groups; ++g) {
            if (done[g] || (prec != NPFEM_PREC_FP64 && meshes[g]->threads != threads)) continue;
            hs.push_back(meshes[g]);
            cs.push_back(cells_per_group[g]);
            so.push_back(soff[g]);
            co.push_back(coff[g]);
            ko.push_back(koff[g]);
            done[g] = 1;
        }
        int rc;
        if (prec == NPFEM_PREC_FP64)
            rc = run_cells<double>(hs.data(), (int)hs.size(), cs.data(), (double*)x, (double*)v, (const double*)f_ext,
                                   nullptr, nullptr, nullptr, stats, 0, s, nullptr, so.data(), co.data(), threads,
                                   (const double*)hist_in, (double*)hist_out, 0, nullptr, 0, (double*)carry,
                                   ko.data());
        else
            rc = run_cells<float>(hs.data(), (int)hs.size(), cs.data(), (float*)x, (float*)v, (const float*)f_ext,
                                  nullptr, nullptr, nullptr, stats, 0, s, u0, so.data(), co.data(), threads,
                                  (const float*)hist_in, (float*)hist_out, pos_stride, nullptr, hist_ext,
                                  (float*)carry, ko.data());
        if (rc) return rc;
    }
    return 0;
}

// Learned first increments of every group with a warm start, into meshes[0]'s
// buffer at the groups' state offsets (a separate launch: in the cluster kernel a
// block computing them would hold up its whole cluster).  Null when no group has one.
int precompute_warm_start(npfem_handle* const* meshes, int n_groups, const int32_t* cells, const float* x,
                          const float* v, const float* f, cudaStream_t s, const float** u0)
{
    *u0 = nullptr;
    bool any = false;
    size_t total = 0;
    for (int g = 0; g < n_groups; ++g) {
        any = any || (meshes[g]->tf.ws_mode && meshes[g]->tf.mlp && cells[g] > 0);
        total += (size_t)3 * meshes[g]->n * cells[g];
    }
    if (!any) return 0;
    npfem_handle* h0 = meshes[0];
    if (total > h0->ws_u_len) {
        if (h0->ws_u) {
            NPFEM_CUDA(cudaStreamSynchronize(s));
            cudaFree(h0->ws_u);
            h0->ws_u = nullptr;
            h0->ws_u_len = 0;
        }
        NPFEM_CUDA(cudaMalloc(&h0->ws_u, total * sizeof(float)));
        h0->ws_u_len = total;
    }
    size_t off = 0;
    for (int g = 0; g < n_groups; ++g) {
        if (meshes[g]->tf.ws_mode && meshes[g]->tf.mlp && cells[g] > 0)
            NPFEM_CUDA(launch_ws_increments(meshes[g], cells[g], x + off, v + off, f + off, h0->ws_u + off, false, s));
        off += (size_t)3 * meshes[g]->n * cells[g];
    }
    *u0 = h0->ws_u;
    return 0;
}

// First increments of every group along a trajectory with a temporal network, into
// meshes[0]'s buffer at the groups' state offsets (one launch per group).
int precompute_temporal(npfem_handle* const* meshes, int n_groups, const int32_t* cells, const float* x,
                        const float* v, const float* f, const float* hist, long long pos_stride, cudaStream_t s,
                        const float** u0)
{
    npfem_handle* h0 = meshes[0];
    size_t total = 0;
    for (int g = 0; g < n_groups; ++g) total += (size_t)3 * meshes[g]->n * cells[g];
    if (total > h0->ws_u_len) {
        if (h0->ws_u) {
            NPFEM_CUDA(cudaStreamSynchronize(s));
            cudaFree(h0->ws_u);
            h0->ws_u = nullptr;
            h0->ws_u_len = 0;
        }
        NPFEM_CUDA(cudaMalloc(&h0->ws_u, total * sizeof(float)));
        h0->ws_u_len = total;
    }
    size_t off = 0;
    const float* c1 = hist;                  // c_{n-1}
    const float* c2 = hist + 3 * pos_stride;  // c_{n-2}
    const float* fp = hist + 4 * pos_stride;  // F_{n-1}
    for (int g = 0; g < n_groups; ++g) {
        if (cells[g] > 0)
            NPFEM_CUDA(launch_ws_temporal(meshes[g], cells[g], x + off, v + off, f + off, fp + off, c1 + off, c2 + off,
                                          nullptr, nullptr, nullptr, nullptr, h0->ws_u + off, 3LL * meshes[g]->n, s));
        off += (size_t)3 * meshes[g]->n * cells[g];
    }
    *u0 = h0->ws_u;
    return 0;
}

int validate_group(npfem_handle* const* meshes, int n_groups, const int32_t* cells)
{
    if (!meshes || n_groups < 1 || n_groups > kMaxGroups || !cells)
        return fail(NPFEM_ERR_INVALID_ARG, "need 1..8 mesh handles and a cells_per_group array");
    for (int g = 0; g < n_groups; ++g) {
        if (!meshes[g]) return fail(NPFEM_ERR_INVALID_ARG, "null mesh handle");
        if (cells[g] < 0) return fail(NPFEM_ERR_INVALID_ARG, "negative cell count");
        if (meshes[g]->device != meshes[0]->device || meshes[g]->precision != meshes[0]->precision ||
            meshes[g]->dt != meshes[0]->dt)
            return fail(NPFEM_ERR_INVALID_ARG, "all handles of one call must share device, precision and dt");
    }
    return 0;
}

}  // namespace

extern "C" {

void npfem_default_opts(npfem_opts* o)
{
    if (!o) return;
    o->precision = NPFEM_PREC_FP32;
    o->lbfgs_m = 5;
    o->max_iter = 50;
    o->tol = 1e-6;
    o->c1 = 1e-4;
    o->c2 = 0.9;
    o->max_halvings = 30;
    o->fixed_alpha = 0;
    o->equal_mass = 0;
    o->armijo_noise = 4.0;
    o->refine = 0;
    o->fill_idle_sms = 1;
    o->warm_history = 2;
}

const char* npfem_last_error(void) { return g_last_error.c_str(); }

unsigned long long npfem_launch_count(void) { return npfem::g_launches.load(); }

int npfem_kernel_timing(npfem_handle* h, int capacity)
{
    if (!h || capacity < 0) return fail(NPFEM_ERR_INVALID_ARG, "npfem_kernel_timing: bad argument");
    DeviceGuard guard(h->device);
    std::lock_guard<std::mutex> lk(h->mu);
    NPFEM_CUDA(cudaDeviceSynchronize());
    for (cudaEvent_t e : h->tev) cudaEventDestroy(e);
    h->tev.clear();
    h->tev_used = 0;
    for (int q = 0; q < 2 * capacity; ++q) {
        cudaEvent_t e;
        NPFEM_CUDA(cudaEventCreate(&e));
        h->tev.push_back(e);
    }
    return 0;
}

int npfem_get_tuning(const npfem_handle* h, int* use_tc, int* threads, int* fill_idle_sms)
{
    if (!h || !use_tc || !threads || !fill_idle_sms) return fail(NPFEM_ERR_INVALID_ARG, "npfem_get_tuning: null argument");
    *use_tc = h->use_tc && h->precision == NPFEM_PREC_BF16 && h->n <= kTcMaxVerts;
    *threads = h->threads;
    *fill_idle_sms = h->opts.fill_idle_sms;
    return 0;
}

int npfem_autotune(npfem_handle* const* meshes, int n_groups, const int32_t* cells_per_group, const void* x,
                   const void* v, const void* f_ext, double dt, int trial_steps, float* trial_ms)
{
    if (int rc = validate_group(meshes, n_groups, cells_per_group)) return rc;
    if (!x || !v || !f_ext || trial_steps < 1) return fail(NPFEM_ERR_INVALID_ARG, "npfem_autotune: bad argument");
    DeviceGuard guard(meshes[0]->device);
    NPFEM_CUDA(cudaDeviceSynchronize());
    const int prec = meshes[0]->precision;
    const size_t es = prec == NPFEM_PREC_FP64 ? 8 : 4;
    struct Shape {
        int use_tc, threads, fill, slot;
    };
    if (trial_ms)
        for (int q = 0; q < 5 * n_groups; ++q) trial_ms[q] = -1.f;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    NPFEM_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    NPFEM_CUDA(cudaEventCreate(&e0));
    NPFEM_CUDA(cudaEventCreate(&e1));
    int rc = 0;
    size_t off = 0;
    for (int g = 0; g < n_groups && !rc; ++g) {
        npfem_handle* h = meshes[g];
        const int cells = cells_per_group[g];
        const size_t bytes = (size_t)3 * h->n * cells * es;
        if (cells == 0) continue;
        std::vector<Shape> cand;
        cand.push_back({0, 512, h->opts.fill_idle_sms, 0});
        if (prec != NPFEM_PREC_FP64) cand.push_back({0, 640, h->opts.fill_idle_sms, 1});
        if (prec == NPFEM_PREC_BF16 && h->n <= kTcMaxVerts) {
            cand.push_back({1, 512, 1, 2});
            cand.push_back({1, 512, 0, 3});
            cand.push_back({1, 640, 1, 4});
        }
        void *tx = nullptr, *tv = nullptr;
        cudaError_t ce = cudaMalloc(&tx, bytes);
        if (ce == cudaSuccess) ce = cudaMalloc(&tv, bytes);
        if (ce != cudaSuccess) {
            rc = fail(ce == cudaErrorMemoryAllocation ? NPFEM_ERR_OOM : NPFEM_ERR_CUDA, "npfem_autotune: trial buffers");
        }
        float best = 1e30f;
        Shape pick = {h->use_tc, h->threads, h->opts.fill_idle_sms, -1};
        const int hist_opt = h->opts.warm_history;
        for (const Shape& c : cand) {
            if (rc) break;
            h->use_tc = c.use_tc;
            h->threads = c.threads;
            h->opts.fill_idle_sms = c.fill;
            const char* xs = static_cast<const char*>(x) + off;
            const char* vs = static_cast<const char*>(v) + off;
            const void* fs = static_cast<const char*>(f_ext) + off;
            // one untimed step, then trial_steps back to back (as in a time loop)
            float total = 0.f;
            npfem_handle* one[1] = {h};
            h->hist_sig.clear();  // each candidate's untimed step starts without history
            NPFEM_CUDA(cudaMemcpyAsync(tx, xs, bytes, cudaMemcpyDeviceToDevice, s));
            NPFEM_CUDA(cudaMemcpyAsync(tv, vs, bytes, cudaMemcpyDeviceToDevice, s));
            rc = npfem_step(one, 1, &cells, tx, tv, fs, dt, s, nullptr);
            if (!rc) NPFEM_CUDA(cudaEventRecord(e0, s));
            for (int k = 0; k < trial_steps && !rc; ++k) rc = npfem_step(one, 1, &cells, tx, tv, fs, dt, s, nullptr);
            if (!rc) {
                NPFEM_CUDA(cudaEventRecord(e1, s));
                NPFEM_CUDA(cudaEventSynchronize(e1));
                NPFEM_CUDA(cudaEventElapsedTime(&total, e0, e1));
            }
            if (!rc && trial_ms) trial_ms[5 * g + c.slot] = total / trial_steps;
            if (!rc && total < best) {
                best = total;
                pick = c;
            }
        }
        h->use_tc = pick.use_tc;
        h->threads = pick.threads;
        h->opts.fill_idle_sms = pick.fill;
        h->opts.warm_history = hist_opt;
        h->hist_sig.clear();
        if (tx) cudaFree(tx);
        if (tv) cudaFree(tv);
        off += bytes;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    return rc;
}

int npfem_kernel_time_last(npfem_handle* h, float* ms)
{
    if (!h || !ms) return fail(NPFEM_ERR_INVALID_ARG, "npfem_kernel_time_last: bad argument");
    DeviceGuard guard(h->device);
    std::lock_guard<std::mutex> lk(h->mu);
    if (h->tev_used < 2) return fail(NPFEM_ERR_INVALID_ARG, "npfem_kernel_time_last: nothing recorded");
    NPFEM_CUDA(cudaEventSynchronize(h->tev[1]));
    NPFEM_CUDA(cudaEventElapsedTime(ms, h->tev[0], h->tev[1]));
    return 0;
}

int npfem_kernel_times(npfem_handle* h, float* ms_out, int max, int* count)
{
    if (!h || !count || max < 0 || (max > 0 && !ms_out)) return fail(NPFEM_ERR_INVALID_ARG, "npfem_kernel_times: bad argument");
    DeviceGuard guard(h->device);
    std::lock_guard<std::mutex> lk(h->mu);
    int k = 0;
    for (int q = 0; q + 1 < h->tev_used && k < max; q += 2, ++k) {
        NPFEM_CUDA(cudaEventSynchronize(h->tev[q + 1]));
        NPFEM_CUDA(cudaEventElapsedTime(&ms_out[k], h->tev[q], h->tev[q + 1]));
    }
    *count = k;
    h->tev_used = 0;
    return 0;
}

int npfem_create(const npfem_mesh* mesh, const npfem_material* mat, const npfem_opts* opts, double dt, int device,
                 npfem_handle** out)
{
    g_last_error.clear();
    if (!mesh || !mat || !opts || !out || !mesh->tris || !mesh->rest_xyz)
        return fail(NPFEM_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (!(dt > 0.0) || !isfinite(dt)) return fail(NPFEM_ERR_INVALID_ARG, "dt must be positive");
    if (int rc = check_opts(opts)) return rc;
    if (!(mat->density > 0.0) || mat->kappa < 0.0 || mat->kappa > 1.0 || mat->C < 0 || mat->B < 0 || mat->D < 0 ||
        mat->k_bend < 0 || mat->k_vol < 0 || mat->k_mat_hess < 0 || mat->alpha_D < 0 || !(mat->beta_D >= 0.0))
        return fail(NPFEM_ERR_INVALID_ARG, "material: need density > 0, kappa in [0,1], non-negative moduli");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(NPFEM_ERR_INVALID_ARG, "no such CUDA device");
    DeviceGuard guard(device);

    npfem_handle* h = new npfem_handle();
    h->device = device;
    h->precision = opts->precision;
    h->dt = dt;
    h->opts = *opts;
    h->mat = *mat;
    std::string err;
    int rc = build_host_topo(mesh, mat, opts->equal_mass, &h->host, &err);
    if (rc) {
        delete h;
        return fail(rc, err);
    }
    h->n = h->host.n;
    h->nt = h->host.nt;
    h->n_pad = (h->n + 3) & ~3;
    cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);

    auto bail = [&](int code) {
        h->release();
        delete h;
        return code;
    };
    const int n = h->n, np = h->n_pad;
    int e = 0;
    // dense H~ = M~/h^2 + L in FP64, inverted on the GPU.  Rayleigh damping
    // C = alpha_D M + beta_D L (Sec. 2.1.4) gives M~ = (1 + h alpha_D) M + h beta_D L, so
    // H~ = (1 + h alpha_D)/h^2 M + (1 + beta_D/h) L
    std::vector<double> H((size_t)n * n, 0.0);
    const double ms = (1.0 + dt * mat->alpha_D) / (dt * dt);
    const double lscale = 1.0 + mat->beta_D / dt;
    for (int i = 0; i < n; ++i) {
        H[(size_t)i * n + i] += ms * h->host.mass[i];
        for (int q = h->host.L_ptr[i]; q < h->host.L_ptr[i + 1]; ++q)
            H[(size_t)i * n + h->host.L_idx[q]] += lscale * h->host.L_val[q];
    }
    h->ainv64 = h->alloc<double>((size_t)n * n, &e);
    double* prow = h->alloc<double>(2 * (size_t)n, &e);
    int* flag = h->alloc<int>(4, &e);
    h->work = h->alloc<unsigned int>(4, &e);
    if (e) return bail(e);
    // one inversion on the GPU: the dense FP64 matrix in, its inverse in place
    auto invert = [&](double* dA, const std::vector<double>& A, const char* what) -> int {
        if (cudaMemcpy(dA, A.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(flag, 0, 4 * sizeof(int)) != cudaSuccess)
            return fail(NPFEM_ERR_CUDA, std::string("upload of ") + what + " failed");
        cudaError_t ce = invert_spd_fp64(dA, n, prow, flag, 0);
        if (ce != cudaSuccess) return fail(NPFEM_ERR_CUDA, std::string("inversion of ") + what + ": " + cudaGetErrorString(ce));
        int hflag = 0;
        if (cudaMemcpy(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(NPFEM_ERR_CUDA, std::string("inversion of ") + what + " failed");
        if (hflag == 2) return fail(NPFEM_ERR_TIMEOUT, std::string("inversion of ") + what + ": a grid barrier gave up");
        if (hflag) return fail(NPFEM_ERR_NOT_SPD, std::string(what) + " is not positive definite");
        return 0;
    };
    if (cudaMemset(h->work, 0, 4 * sizeof(unsigned)) != cudaSuccess) return bail(fail(NPFEM_ERR_CUDA, "memset failed"));
    if ((rc = invert(h->ainv64, H, "H~"))) return bail(rc);
    cudaError_t ce = cudaSuccess;
    // beta_D > 0: M~ is not diagonal; the first guess applies M~^-1 (dense, inverted once
    // like H~) and the inertia term needs h beta_D L (sparse, in the solver's type)
    void* minv_t = nullptr;
    if (mat->beta_D > 0.0) {
        std::vector<double> Mt((size_t)n * n, 0.0);
        for (int i = 0; i < n; ++i) {
            Mt[(size_t)i * n + i] += (1.0 + dt * mat->alpha_D) * h->host.mass[i];
            for (int q = h->host.L_ptr[i]; q < h->host.L_ptr[i + 1]; ++q)
                Mt[(size_t)i * n + h->host.L_idx[q]] += dt * mat->beta_D * h->host.L_val[q];
        }
        double* m64 = h->alloc<double>((size_t)n * n, &e);
        if (e) return bail(e);
        if ((rc = invert(m64, Mt, "M~"))) return bail(rc);
        if (h->precision == NPFEM_PREC_FP64) {
            double* o = h->alloc<double>((size_t)np * np, &e);
            if (e) return bail(e);
            ce = publish_inverse(m64, n, np, nullptr, o, nullptr, nullptr, 0);
            minv_t = o;
        } else {
            float* o = h->alloc<float>((size_t)np * np, &e);
            if (e) return bail(e);
            ce = publish_inverse(m64, n, np, o, nullptr, nullptr, nullptr, 0);
            minv_t = o;
        }
        if (ce != cudaSuccess) return bail(fail(NPFEM_ERR_CUDA, "publishing M~^-1 failed"));
    }

    void* ainv_t = nullptr;
    if (h->precision == NPFEM_PREC_FP64) {
        double* a64 = h->alloc<double>((size_t)np * np, &e);
        if (e) return bail(e);
        ce = publish_inverse(h->ainv64, n, np, nullptr, a64, nullptr, nullptr, 0);
        ainv_t = a64;
    } else {
        float* a32 = h->alloc<float>((size_t)np * np, &e);
        if (e) return bail(e);
        ce = publish_inverse(h->ainv64, n, np, a32, nullptr, nullptr, nullptr, 0);
        ainv_t = a32;
    }
    if (ce != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
        return bail(fail(NPFEM_ERR_CUDA, "publishing A^-1 failed"));
    rc = h->precision == NPFEM_PREC_FP64 ? fill_topo<double>(h, &h->td, ainv_t, minv_t)
                                         : fill_topo<float>(h, &h->tf, ainv_t, minv_t);
    if (rc) return bail(rc);
    if (h->precision == NPFEM_PREC_TF32) {
        // TF32 path: A^-1 in chunks of 128 rows x 32 K in the MMA's layout, and L for the
        // refinement residual
        const int kpad = (n + 31) & ~31, tiles = (n + 127) / 128;
        float* atf = h->alloc<float>((size_t)tiles * 128 * kpad, &e);
        if (e) return bail(e);
        if (publish_inverse_tf32_tiled(h->ainv64, n, tiles, kpad, atf, 0) != cudaSuccess ||
            cudaDeviceSynchronize() != cudaSuccess)
            return bail(fail(NPFEM_ERR_CUDA, "publishing the TF32 A^-1 failed"));
        h->tf.ainv_lp = atf;
        h->tf.kpad = kpad;
        h->tf.rb = tiles;
        std::vector<float> lval(h->host.L_val.size());
        for (size_t q = 0; q < lval.size(); ++q) lval[q] = (float)(lscale * h->host.L_val[q]);
        std::vector<unsigned short> lidx(h->host.L_idx.begin(), h->host.L_idx.end());
        if ((rc = upload(h, h->host.L_ptr, &h->tf.h_ptr))) return bail(rc);
        if ((rc = upload(h, lidx, &h->tf.h_idx))) return bail(rc);
        if ((rc = upload(h, lval, &h->tf.h_val))) return bail(rc);
    }
    if (h->precision == NPFEM_PREC_BF16) {
        // tensor-core path: BF16 A^-1 in 128-row blocks with K padded to 16, and L for
        // the refinement residual
        const int kpad = (n + 15) & ~15, rb = (n + 127) / 128;
        void* abf = h->alloc<unsigned short>((size_t)rb * 128 * kpad, &e);
        if (e) return bail(e);
        if (publish_inverse_bf16_blocked(h->ainv64, n, rb * 128, kpad, abf, 0) != cudaSuccess ||
            cudaDeviceSynchronize() != cudaSuccess)
            return bail(fail(NPFEM_ERR_CUDA, "publishing the BF16 A^-1 failed"));
        h->tf.ainv_lp = abf;
        h->tf.kpad = kpad;
        h->tf.rb = rb;
        // the SIMT contraction of a BF16 handle (meshes the clusters do not take, idle-SM
        // blocks) reads A^-1 in BF16 too: half the bytes of FP32
        const int n8 = (n + 7) & ~7;
        void* asq = h->alloc<unsigned short>((size_t)n8 * n8, &e);
        if (e) return bail(e);
        if (publish_inverse_bf16_square(h->ainv64, n, n8, asq, 0) != cudaSuccess ||
            cudaDeviceSynchronize() != cudaSuccess)
            return bail(fail(NPFEM_ERR_CUDA, "publishing the BF16 A^-1 failed"));
        h->tf.ainv_b16 = asq;
        h->tf.n8 = n8;
        // the refinement residual q - H~ r needs H~ = ms M + (1 + beta_D/h) L
        std::vector<float> lval(h->host.L_val.size());
        for (size_t q = 0; q < lval.size(); ++q) lval[q] = (float)(lscale * h->host.L_val[q]);
        std::vector<unsigned short> lidx(h->host.L_idx.begin(), h->host.L_idx.end());
        if ((rc = upload(h, h->host.L_ptr, &h->tf.h_ptr))) return bail(rc);
        if ((rc = upload(h, lidx, &h->tf.h_idx))) return bail(rc);
        if ((rc = upload(h, lval, &h->tf.h_val))) return bail(rc);
    }
    *out = h;
    return 0;
}

int npfem_destroy(npfem_handle* h)
{
    if (!h) return fail(NPFEM_ERR_INVALID_ARG, "null handle");
    {
        DeviceGuard guard(h->device);
        cudaDeviceSynchronize();
        h->release();
    }
    delete h;
    return 0;
}

int npfem_step(npfem_handle* const* meshes, int n_groups, const int32_t* cells_per_group, void* x, void* v,
               const void* f_ext, double dt, void* stream, npfem_cell_stats* stats)
{
    if (int rc = validate_group(meshes, n_groups, cells_per_group)) return rc;
    if (!x || !v || !f_ext) return fail(NPFEM_ERR_INVALID_ARG, "null state pointer");
    if (dt != meshes[0]->dt) return fail(NPFEM_ERR_INVALID_ARG, "dt differs from the handle's dt");
    DeviceGuard guard(meshes[0]->device);
    std::lock_guard<std::mutex> lk(meshes[0]->mu);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    npfem_handle* h0 = meshes[0];
    // temporal warm start: read the last step's corrections when this call steps the
    // same groups and cell counts, and write this step's
    const void* hist_in = nullptr;
    void* hist_out = nullptr;
    long long pos_stride = 0;
    int hist_ext = 0;
    void* carry = nullptr;
    if (h0->opts.warm_history) {
        std::vector<long long> sig;
        size_t elems = 0;
        for (int g = 0; g < n_groups; ++g) {
            sig.push_back(reinterpret_cast<long long>(meshes[g]));
            sig.push_back(cells_per_group[g]);
            elems += (size_t)3 * meshes[g]->n * cells_per_group[g];
            if (meshes[g]->precision != NPFEM_PREC_FP64 && meshes[g]->tf.tmlp) hist_ext = 1;
        }
        sig.push_back(hist_ext);
        // FP64: the corrections; FP32: the corrections, then the positions' rounding
        // residues, then the FP32 positions they belong to (compensated positions); with a
        // temporal network also the previous correction and the last force
        const bool f32 = h0->precision != NPFEM_PREC_FP64;
        pos_stride = f32 ? (long long)elems : 0;
        const size_t bytes = elems * (f32 ? (hist_ext ? 5 : 3) * 4 : 8);
        if (bytes > h0->hist_bytes) {
            if (h0->hist) {
                NPFEM_CUDA(cudaStreamSynchronize(s));
                cudaFree(h0->hist);
                h0->hist = nullptr;
                h0->hist_bytes = 0;
                h0->hist_sig.clear();
            }
            NPFEM_CUDA(cudaMalloc(&h0->hist, bytes));
            h0->hist_bytes = bytes;
        }
        if (h0->opts.warm_history == 2 && bytes > 0) {
            // carried L-BFGS pairs: one record per cell, valid together with the corrections
            size_t kb = 0;
            for (int g = 0; g < n_groups; ++g)
                kb += (size_t)carry_rec_elems(meshes[g]->n_pad, h0->opts.lbfgs_m) * cells_per_group[g];
            kb *= f32 ? 4 : 8;
            if (kb > h0->carry_bytes) {
                if (h0->carry) {
                    NPFEM_CUDA(cudaStreamSynchronize(s));
                    cudaFree(h0->carry);
                    h0->carry = nullptr;
                    h0->carry_bytes = 0;
                }
                h0->hist_sig.clear();
                NPFEM_CUDA(cudaMalloc(&h0->carry, kb));
                h0->carry_bytes = kb;
            }
            carry = h0->carry;
        }
        if (bytes > 0) {
            if (sig == h0->hist_sig) hist_in = h0->hist;
            hist_out = h0->hist;
            h0->hist_sig = sig;
        }
    }
    const float* u0 = nullptr;
    if (meshes[0]->precision != NPFEM_PREC_FP64 && !hist_in) {
        if (int rc = precompute_warm_start(meshes, n_groups, cells_per_group, (const float*)x, (const float*)v,
                                           (const float*)f_ext, s, &u0))
            return rc;
    } else if (hist_in && hist_ext) {
        // along a trajectory with a temporal network: u = u_y + c_{n-1} + R MLP(features)
        // for every group (u_y + c_{n-1} where a group has no network)
        if (int rc = precompute_temporal(meshes, n_groups, cells_per_group, (const float*)x, (const float*)v,
                                         (const float*)f_ext, (const float*)hist_in, pos_stride, s, &u0))
            return rc;
    }
    const bool timed = h0->tev_used + 2 <= (int)h0->tev.size();
    unsigned rec_flags = cudaEventRecordDefault;
    if (timed) {
        // inside a stream capture the pair must become event-record nodes of the graph
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        NPFEM_CUDA(cudaStreamIsCapturing(s, &cap));
        if (cap == cudaStreamCaptureStatusActive) rec_flags = cudaEventRecordExternal;
        NPFEM_CUDA(cudaEventRecordWithFlags(h0->tev[h0->tev_used], s, rec_flags));
    }
    int rc = step_groups(meshes, n_groups, cells_per_group, x, v, f_ext, s, stats, u0, hist_in, hist_out, pos_stride,
                         hist_ext, carry);
    if (rc) h0->hist_sig.clear();
    if (!rc && timed) {
        NPFEM_CUDA(cudaEventRecordWithFlags(h0->tev[h0->tev_used + 1], s, rec_flags));
        h0->tev_used += 2;
    }
    return rc;
}

// The device address of a pinned host buffer mapped into the current device's address
// space (cudaHostAlloc, or cudaHostRegister with mapping), or null for any other pointer.
static void* mapped_host(void* p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();  // not a pointer the runtime knows: clear the error, copy instead
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

int npfem_step_host(npfem_handle* h, int n_cells, void* x_host, void* v_host, const void* f_host, double dt,
                    void* stream, npfem_cell_stats* stats_host)
{
    if (!h || n_cells < 0 || !x_host || !v_host || !f_host) return fail(NPFEM_ERR_INVALID_ARG, "null argument");
    if (dt != h->dt) return fail(NPFEM_ERR_INVALID_ARG, "dt differs from the handle's dt");
    DeviceGuard guard(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t es = h->precision == NPFEM_PREC_FP64 ? 8 : 4;
    const size_t bytes = (size_t)n_cells * 3 * h->n * es;
    {
        std::lock_guard<std::mutex> lk(h->mu);
        if ((size_t)n_cells > h->host_cells) {
            NPFEM_CUDA(cudaStreamSynchronize(s));
            if (h->hx) cudaFree(h->hx);
            if (h->hv) cudaFree(h->hv);
            if (h->hf) cudaFree(h->hf);
            if (h->hstats) cudaFree(h->hstats);
            h->hx = h->hv = h->hf = nullptr;
            h->hstats = nullptr;
            h->host_cells = 0;
            NPFEM_CUDA(cudaMalloc(&h->hx, bytes));
            NPFEM_CUDA(cudaMalloc(&h->hv, bytes));
            NPFEM_CUDA(cudaMalloc(&h->hf, bytes));
            NPFEM_CUDA(cudaMalloc(&h->hstats, sizeof(npfem_cell_stats) * (size_t)std::max(n_cells, 1)));
            h->host_cells = (size_t)n_cells;
        }
    }
    if (n_cells == 0) return 0;
    int32_t cells = n_cells;
    npfem_handle* hs[1] = {h};
    // a synchronous step starts on an idle GPU, where the idle-SM blocks can be placed
    // before the clusters and cost cluster slots (measured: slower), so it runs without
    const int fill = h->opts.fill_idle_sms;
    h->opts.fill_idle_sms = 0;
    // pinned host buffers mapped into the device's address space are stepped in place:
    // the solver's loads at the start of a cell and its stores at the end move x, v and
    // F_ext over the host link while other cells compute, instead of copies before and
    // after the step
    void* xd = mapped_host(x_host);
    void* vd = mapped_host(v_host);
    void* fd = mapped_host(const_cast<void*>(f_host));
    void* sd = stats_host ? mapped_host(stats_host) : nullptr;
    if (xd && vd && fd && (!stats_host || sd)) {
        int rc = npfem_step(hs, 1, &cells, xd, vd, fd, dt, stream, static_cast<npfem_cell_stats*>(sd));
        h->opts.fill_idle_sms = fill;
        if (rc) return rc;
        NPFEM_CUDA(cudaStreamSynchronize(s));
        return 0;
    }
    cudaError_t e = cudaMemcpyAsync(h->hx, x_host, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->hv, v_host, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->hf, f_host, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        h->opts.fill_idle_sms = fill;
        return fail(NPFEM_ERR_CUDA, std::string("npfem_step_host copies in: ") + cudaGetErrorString(e));
    }
    int rc = npfem_step(hs, 1, &cells, h->hx, h->hv, h->hf, dt, stream, stats_host ? h->hstats : nullptr);
    h->opts.fill_idle_sms = fill;
    if (rc) return rc;
    NPFEM_CUDA(cudaMemcpyAsync(x_host, h->hx, bytes, cudaMemcpyDeviceToHost, s));
    NPFEM_CUDA(cudaMemcpyAsync(v_host, h->hv, bytes, cudaMemcpyDeviceToHost, s));
    if (stats_host)
        NPFEM_CUDA(cudaMemcpyAsync(stats_host, h->hstats, sizeof(npfem_cell_stats) * n_cells, cudaMemcpyDeviceToHost, s));
    NPFEM_CUDA(cudaStreamSynchronize(s));
    return 0;
}

int npfem_eval(npfem_handle* h, int n_cells, const void* x, const void* y, void* grad, double* parts, void* stream)
{
    if (!h || n_cells < 0 || !x || !y || !grad || !parts) return fail(NPFEM_ERR_INVALID_ARG, "null argument");
    DeviceGuard guard(h->device);
    std::lock_guard<std::mutex> lk(h->mu);
    npfem_handle* hs[1] = {h};
    int32_t cells = n_cells;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (h->precision == NPFEM_PREC_FP64)
        return run_cells<double>(hs, 1, &cells, (double*)x, nullptr, nullptr, (const double*)y, (double*)grad, parts,
                                 nullptr, 1, s);
    return run_cells<float>(hs, 1, &cells, (float*)x, nullptr, nullptr, (const float*)y, (float*)grad, parts, nullptr,
                            1, s);
}

int npfem_ws_guess(npfem_handle* h, int n_cells, const float* x, const float* v, const float* f, float* x1, void* stream)
{
    if (!h || n_cells < 0 || !x || !v || !f || !x1) return fail(NPFEM_ERR_INVALID_ARG, "npfem_ws_guess: null argument");
    if (h->precision == NPFEM_PREC_FP64) return fail(NPFEM_ERR_INVALID_ARG, "npfem_ws_guess: FP32 state handles only");
    DeviceGuard guard(h->device);
    std::lock_guard<std::mutex> lk(h->mu);
    if (!h->tf.ws_mode || !h->tf.mlp) return fail(NPFEM_ERR_INVALID_ARG, "npfem_ws_guess: no warm start installed");
    if (n_cells == 0) return 0;
    NPFEM_CUDA(launch_ws_increments(h, n_cells, x, v, f, x1, true, static_cast<cudaStream_t>(stream)));
    return 0;
}

int npfem_check_device(npfem_handle* h)
{
    if (!h) return fail(NPFEM_ERR_INVALID_ARG, "null handle");
    DeviceGuard guard(h->device);
    NPFEM_CUDA(cudaDeviceSynchronize());
    unsigned flag = 0;
    NPFEM_CUDA(cudaMemcpy(&flag, h->work + 2, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (flag) {
        NPFEM_CUDA(cudaMemset(h->work + 2, 0, sizeof(unsigned)));
        return fail(NPFEM_ERR_TIMEOUT, "a bounded device wait gave up in a previous step (tensor-core MMA completion)");
    }
    return 0;
}

int npfem_flag_wait_timeout(npfem_handle* h)
{
    if (!h) return fail(NPFEM_ERR_INVALID_ARG, "null handle");
    DeviceGuard guard(h->device);
    NPFEM_CUDA(cudaDeviceSynchronize());
    const unsigned one = 1u;
    NPFEM_CUDA(cudaMemcpy(h->work + 2, &one, sizeof(unsigned), cudaMemcpyHostToDevice));
    return 0;
}

int npfem_get_inverse(npfem_handle* h, double* out_host)
{
    if (!h || !out_host) return fail(NPFEM_ERR_INVALID_ARG, "null argument");
    DeviceGuard guard(h->device);
    NPFEM_CUDA(cudaMemcpy(out_host, h->ainv64, sizeof(double) * (size_t)h->n * h->n, cudaMemcpyDeviceToHost));
    return 0;
}

int npfem_get_rest_info(npfem_handle* h, double* masses_host, double* scalars_host)
{
    if (!h) return fail(NPFEM_ERR_INVALID_ARG, "null handle");
    if (masses_host) memcpy(masses_host, h->host.mass.data(), sizeof(double) * h->n);
    if (scalars_host) {
        scalars_host[0] = h->host.V0;
        scalars_host[1] = h->host.A0;
        scalars_host[2] = h->host.lbar;
        scalars_host[3] = h->host.mtotal;
    }
    return 0;
}

}  // extern "C"
