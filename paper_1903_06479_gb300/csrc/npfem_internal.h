// Internal declarations shared by the translation units of libnpfem.so.
// Not part of the public ABI (see include/npfem.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/npfem.h"

namespace npfem {

constexpr int kMaxGroups = 8;     // meshes per npfem_step launch
constexpr int kMaxHistory = 8;    // L-BFGS window limit
constexpr int kNumBaseVecs = 10;  // XN U UT G GT GC UY D TRI WR, then S[m], Y[m]
constexpr int kMaxVecs = kNumBaseVecs + 2 * kMaxHistory;
constexpr int kFixedSmem = 12288; // reduction scratch (8 KB) + per-cell scalars at the start of dynamic smem

// Per-cell buffers.  All are 3 x n_pad values except TRI (rows of kTriRow values per
// triangle: the gradient contributions of corners j and k and the area-weighted
// normal / 6, padded to 12 for 16-byte accesses).
constexpr int kTriRow = 12;

enum Vec { V_XN = 0, V_U = 1, V_UT = 2, V_G = 3, V_GT = 4, V_GC = 5, V_UY = 6, V_D = 7, V_TRI = 8, V_WR = 9, V_SBASE = 10 };

enum Contraction { CONTRACT_SIMT = 0, CONTRACT_TC_TF32 = 1, CONTRACT_TC_BF16 = 2 };

// Device-side tables of one mesh topology (all pointers are device memory owned by
// the handle).  T is the solver's scalar type (float or double).
template <typename T>
struct TopoDev {
    int n, nt, n_pad, nnz;
    const ushort4* tri;          // [nt] vertex indices (i, j, k, 0)
    const T* dminv;              // [nt][4] row-major D_m^{-1}
    const T* W;                  // [nt] rest triangle areas
    const T* mass;               // [n] lumped masses
    const T* inv_mass;           // [n]
    const T* bend_w;             // [n] k_bend * mixed Voronoi area
    const T* dg_norm;            // [n] |delta_g| of the rest shape
    const T* csum;               // [n] sum_j c_ij
    const T* nsign;              // [n] +-1: orientation of delta_g against the rest normal
    const int* ring_ptr;         // [n + 1]
    const unsigned short* ring_idx;  // [nnz]
    const T* ring_c;             // [nnz] cotangent weights / (2 A_i)
    const T* ring_ct;            // [nnz] weight of vertex i in the ring of its neighbour j
    const int* inc_ptr;          // [n + 1] vertex -> incident triangles
    const unsigned* inc_idx;     // [3 nt] (triangle << 2) | corner
    // Fixed-width one-rings (k8 = 1: every one-ring is a single cycle of at most 8):
    // vertex i's neighbours r_0 .. r_{v-1} in cyclic order, so that incident triangle
    // q of i is (i, r_q, r_{q+1 mod v}); entries past v hold i itself with weight 0.
    // tri[t].w then packs, 3 bits per corner, the slot q of each corner in its
    // vertex's ring, where the triangle pass writes the corner's gradient.
    int k8;
    const unsigned short* ring8_idx;  // [n][8]
    const T* ring8_c;                 // [n][8]
    const T* ring8_ct;                // [n][8]
    const T* ainv;               // [n_pad][n_pad] A^-1 in T (zero padding)
    // Rayleigh damping with beta_D > 0: M~ = (1 + h alpha_D) M + h beta_D L is not
    // diagonal.  minv: [n_pad][n_pad] M~^-1 in T for the first guess; L (CSR, T) for the
    // inertia term's h beta_D L part; beta_h = beta_D / h.  Null pointers when beta_D = 0.
    const T* minv;
    const int* l_ptr;
    const unsigned short* l_idx;
    const T* l_val;
    T beta_h;
    const void* ainv_lp;         // A^-1 for the tensor-core contraction: BF16 row blocks, or TF32 chunks
                                 // of 128 rows x 32 K in the MMA's core-matrix layout
    // BF16 handles: A^-1 in BF16 (round to nearest even), [n8][n8] with n8 = n rounded up
    // to 8 (zero padding), for the SIMT contraction's 256-row tiles (null otherwise)
    const void* ainv_b16;
    int n8;
    const int* h_ptr;            // L (CSR, fp32) for the refinement residual q - H~ r
    const unsigned short* h_idx;
    const float* h_val;
    int kpad, rb;                // tensor-core path: K padded (16 BF16, 32 TF32), row blocks of 128
    const T* rest_c;             // [3][n] rest positions about the rest centre of mass
    const float* mlp;            // learned warm start: packed parameters, weights rounded to BF16 (or null)
    const float* tmlp;           // temporal network along a trajectory (same layout), or null
    int ws_mode;                 // 0 none, 1 learned first iterate, 2 learned iterate kept only if g is lower
    T C, B, Dsk, kvol;           // material
    T h, inv_h2, inertia_scale;  // time step; inertia_scale = 1 + h alpha_D
    T kappa, lbar, inv_lbar;
    double V0;                   // rest volume
    T V0hi, V0lo;                // V0 as an unevaluated sum of two T
};

// One mesh topology inside one launch.
template <typename T>
struct GroupDesc {
    TopoDev<T> topo;
    long long cell_begin;  // first global work item of the group
    long long state_off;   // element offset of the group's first cell in x / v / f
    long long stats_off;   // index of the group's first cell in stats (and eval parts)
    int cells;
    int smem_bytes;        // dynamic smem this group needs (after kFixedSmem)
    int scratch_floats;    // size of the TRI buffer in floats (the SIMT contraction's partials)
    long long carry_off;   // element offset of the group's first carried-pairs record in LaunchArgs::carry
    long long carry_rec;   // elements per record (carry_rec_elems)
    int loc[kMaxVecs];     // >= 0: byte offset in smem; < 0: -(byte offset in the CTA's global slot) - 1
};

struct SolverParams {
    int lbfgs_m, max_iter, max_halvings, fixed_alpha;
    double tol, c1, c2, armijo_noise;
    float tolf, c1f, c2f, armijo_noisef;  // FP32 copies for the FP32 path
    int mode;         // 0 = time step, 1 = objective/gradient evaluation
    int contraction;  // Contraction
    int cluster;      // tensor-core path: blocks per cluster (= row blocks of A^-1)
    int refine;       // tensor-core path: refinement sweeps (0 or 1)
    int tmem_cols;    // TF32 path: tensor-memory columns each block allocates
    int tf_kpad;      // TF32 path: the largest padded K of the launch's groups (B operand size)
};

inline void set_solver_params(SolverParams* p, const npfem_opts& o)
{
    p->lbfgs_m = o.lbfgs_m;
    p->max_iter = o.max_iter;
    p->max_halvings = o.max_halvings;
    p->fixed_alpha = o.fixed_alpha;
    p->tol = o.tol;
    p->c1 = o.c1;
    p->c2 = o.c2;
    p->armijo_noise = o.armijo_noise;
    p->tolf = (float)o.tol;
    p->c1f = (float)o.c1;
    p->c2f = (float)o.c2;
    p->armijo_noisef = (float)o.armijo_noise;
}

template <typename T>
struct LaunchArgs {
    GroupDesc<T> g[kMaxGroups];
    int n_groups;
    long long total_cells;
    T* x;
    T* v;
    const T* f;
    const T* y;        // eval mode: inertia target
    T* grad_out;       // eval mode
    const T* u0;       // precomputed learned first increments x^(1) - x_n ([3][n] per cell) or null
    const T* hist_in;  // previous step's converged corrections x_n - y_{n-1} ([3][n] per cell) or null
    T* hist_out;       // this step's corrections x_{n+1} - y_n are written here (or null)
    // 1: a temporal network is in use: finish() also keeps the previous correction at
    // hist_out + 3 pos_stride and this step's force at hist_out + 4 pos_stride
    int hist_ext;
    // > 0 (FP32 with hist_out): the rounding residue of each stored position, the part of
    // x_n + u below FP32 precision, sits at hist_out + pos_stride and the FP32 value it
    // belongs to at hist_out + 2 pos_stride; hist_in != null marks both as this trajectory's
    long long pos_stride;
    // L-BFGS pairs carried across time steps (opts.warm_history = 2), one record per
    // cell at g.carry_off + cell * g.carry_rec (layout: carry_rec_elems), or null.  With
    // hist_in set the records hold the cell's pairs from its last solve: the first
    // direction request of the step loads them; finish() writes them back when they
    // changed (no write for a cell accepted at its first iterate)
    T* carry;
    // first-iterate pass (SIMT launch): cells not accepted at x^(1) are appended to
    // defer and left untouched.  Layout: [0] cells listed, [1] listed cells that
    // needed iterations (counted by the launch that solves them), [2] that count of the
    // previous step, then the cell indices.  When more than half of the cells needed
    // iterations in the previous step, the pass lists every cell without evaluating.
    // The launch that follows takes only the cells listed in `only` (the same buffer;
    // the count read on the device) and counts into need[0]
    unsigned int* defer;
    const unsigned int* only;
    unsigned int* need;
    double* parts;     // eval mode: 8 doubles per cell
    // collision planes (Sec. 3.3): per vertex of the call (index = element offset / 3) the
    // unit normal of the neighbouring body and the plane's offset relative to the
    // cell's vertex 0; zero normal = none.  Null when the call has no collisions.
    const float4* col;
    T col_w;
    npfem_cell_stats* stats;
    char* scratch;     // per-CTA global slots for vectors that do not fit in smem
    long long slot_bytes;
    // [0..1] 64-bit claim word (low half: cells claimed from the bottom, high half: from
    // the top), [2] error flag, [3] finished blocks; the last block resets [0..1] and [3]
    unsigned int* work;
    int total_blocks;    // blocks of all launches sharing `work` (0: this launch's grid)
    int claim_top;       // 1: claim cells from the top and stop while at most `reserve` remain
    long long reserve;
    SolverParams p;
};

#ifdef __CUDACC__
#define NPFEM_HD __host__ __device__
#else
#define NPFEM_HD
#endif
// Carried L-BFGS pairs of one cell, in elements of the state type: the solver's history
// ring as the last solve left it: [0] the pair count, [1] the ring head, [2] that
// solve's iterations, from [4] the inner products s_i^T y_j by ring slot (m x m, padded
// to a multiple of 4), then the s vectors of ring slots 0..m-1 and the y vectors
// ([3][n_pad] each).  The pairs are used while that solve took at most kCarryMaxIters
// iterations.
constexpr int kCarryMaxIters = 3;
NPFEM_HD inline long long carry_head_elems(int m) { return 4 + (((long long)m * m + 3) & ~3LL); }
NPFEM_HD inline long long carry_rec_elems(int n_pad, int m) { return carry_head_elems(m) + 2LL * m * 3 * n_pad; }

// ---- host-side rest precompute (npfem_setup.cpp) ------------------------------
struct HostTopo {
    int n = 0, nt = 0;
    std::vector<int> tri;                     // [nt][3]
    std::vector<double> dminv, W;             // [nt][4], [nt]
    std::vector<double> mass, avor, bend_w, dg_norm, csum, nsign;  // [n]
    std::vector<int> ring_ptr, ring_idx;      // CSR one-ring
    std::vector<double> ring_c;               // c_ij for entry (i, j)
    std::vector<double> ring_ct;              // c_ji for entry (i, j): weight of i in the ring of j
    std::vector<int> inc_ptr, inc_idx;        // vertex -> incident (triangle << 2 | corner)
    std::vector<double> rest_c;               // [3][n] rest positions about the rest centre of mass
    std::vector<int> L_ptr, L_idx;            // CSR of L (full symmetric)
    std::vector<double> L_val;
    double V0 = 0, A0 = 0, lbar = 0, mtotal = 0;
};

// Returns 0 or a negative NPFEM_ERR code with a message in *err.
int build_host_topo(const npfem_mesh* mesh, const npfem_material* mat, int equal_mass, HostTopo* out,
                    std::string* err);

// ---- kernels (npfem_factor.cu, npfem_solver.cu) ---------------------------------
// In-place FP64 Gauss-Jordan inversion of an SPD n x n matrix on the GPU in one
// cooperative launch.  prow: 2n doubles of scratch; d_flag: 4 ints, zeroed by the
// caller: d_flag[0] becomes 1 when a pivot is not positive, 2 when a grid barrier
// gave up waiting; d_flag[2..3] are the barrier's words.
cudaError_t invert_spd_fp64(double* A, int n, double* prow, int* d_flag, cudaStream_t s);
// Symmetrise A^-1 (FP64, n x n) and write padded copies in fp32 / fp64 / bf16.
cudaError_t publish_inverse(const double* A, int n, int n_pad, float* out32, double* out64, void* out_bf16,
                            float* out_tf32, cudaStream_t s);
// A^-1 in BF16 as [rows_pad][kpad] (zero padding), the layout the tensor-core path
// loads into tensor memory.
cudaError_t publish_inverse_bf16_blocked(const double* A, int n, int rows_pad, int kpad, void* out, cudaStream_t s);
// A^-1 in BF16 as [n8][n8] (rows and columns past n zero) for the SIMT contraction.
cudaError_t publish_inverse_bf16_square(const double* A, int n, int n8, void* out, cudaStream_t s);

template <typename T>
cudaError_t launch_cells(const LaunchArgs<T>& a, int grid, int block, int smem, cudaStream_t s);
template <typename T>
cudaError_t set_cell_kernel_smem(int bytes);
// A^-1 in TF32 (round to nearest) as [row tile][K chunk] blocks of 128 rows x 32 K, each
// in the no-swizzle K-major core-matrix layout the TF32 MMA reads (16 KB per chunk).
cudaError_t publish_inverse_tf32_tiled(const double* A, int n, int tiles, int kpad, float* out, cudaStream_t s);
// Resident SIMT blocks per SM at this block size and dynamic shared memory.
template <typename T>
cudaError_t cells_per_sm(int block, int smem, int* n);
// Tensor-core kernel (BF16, A^-1 row blocks resident in TMEM across a cluster): sets
// its shared-memory size and returns how many clusters can be resident at once.
cudaError_t query_cells_tc(int cluster, int block, int smem, int* max_clusters);
// Launch of one mesh group on `grid` blocks (a multiple of the cluster size).
cudaError_t launch_cells_tc(const LaunchArgs<float>& a, int cluster, int block, int smem, int grid, cudaStream_t s);
// Learned first increments u = x^(1) - x_n ([3][n] per cell, or positions x_n + u
// when positions is set) of n_cells cells of handle h (npfem_learn.cu).
cudaError_t launch_ws_increments(const npfem_handle* h, int n_cells, const float* x, const float* v, const float* f,
                                 float* out, bool positions, cudaStream_t s);
// Temporal network's first increments u = u_y + c_{n-1} (+ R MLP(features) when the
// handle has a network), or, for training, features/targets/corrections; cells are
// `stride` elements apart.
cudaError_t launch_ws_temporal(const npfem_handle* h, int n_cells, const float* x, const float* v, const float* f,
                               const float* f_prev, const float* c1, const float* c2, const float* x_next, float* feat,
                               float* target, float* c_out, float* out, long long stride, cudaStream_t s);
// Largest mesh the tensor-core path takes: A block (kpad / 2 columns) plus a
// 32-column accumulator within 512 TMEM columns, and at most 8 blocks per cluster.
constexpr int kTcMaxVerts = 960;
constexpr int kTcThreads = 512;  // block size of the cluster kernel
// TF32 path: shared memory for the two-stage A^-1 ring and the B operand (8 x kpad TF32).
inline int tf32_smem_bytes(int kpad) { return ((2 * 128 * 32 * 4 + 8 * kpad * 4) + 1023) & ~1023; }

// Records msg as the calling thread's last error and returns code (npfem_api.cu).
int set_error(int code, const std::string& msg);

// Counts a kernel launch of the library (npfem_launch_count).
void count_launch(unsigned long long k = 1);

// Places the per-cell buffers: shared memory in priority order while they fit (the
// randomly gathered ones first; GC first of all with gc_first), the rest in a
// per-block global slot.  smem offsets
// start at base_off.  Returns the smem bytes used in g->smem_bytes.
template <typename T>
inline void place_vectors(GroupDesc<T>* g, int n_pad, int nt, int m, int smem_budget, long long* slot_bytes,
                          int base_off = 0, bool gc_first = false)
{
    const int vb = 3 * n_pad * (int)sizeof(T);
    // TRI (per-triangle rows, or per-vertex corner-gradient slots with fixed-width
    // rings) also serves as the contraction's scratch (max(32, 4 x row tiles) x 384
    // floats) and holds the warm start's normalised features ([n rounded to 16][16] floats)
    const int tri_bytes = kTriRow * nt * (int)sizeof(T);
    const int ctr_bytes = (4 * ((n_pad + 127) / 128) > 32 ? 4 * ((n_pad + 127) / 128) : 32) * 384 * 4;
    const int ws_bytes = ((n_pad + 15) & ~15) * 16 * 4;
    const int slot_bytes8 = 24 * n_pad * (int)sizeof(T);  // [8 slots][3][n_pad] corner gradients
    int tb = tri_bytes > ctr_bytes ? tri_bytes : ctr_bytes;
    tb = tb > slot_bytes8 ? tb : slot_bytes8;
    tb = ((tb > ws_bytes ? tb : ws_bytes) + 15) & ~15;
    int order[kMaxVecs], nv = 0;
    const int base[kNumBaseVecs] = {V_XN, V_U, V_UT, V_TRI, V_WR, V_G, V_GT, V_GC, V_UY, V_D};
    // the tensor-core kernel writes contraction results into GC through distributed
    // shared memory, so it needs GC in shared memory
    if (gc_first) order[nv++] = V_GC;
    for (int q = 0; q < kNumBaseVecs; ++q)
        if (!(gc_first && base[q] == V_GC)) order[nv++] = base[q];
    for (int q = 0; q < m; ++q) {
        order[nv++] = V_SBASE + q;
        order[nv++] = V_SBASE + m + q;
    }
    int used = 0;
    long long gl = 0;
    for (int q = 0; q < kMaxVecs; ++q) g->loc[q] = 0;
    for (int q = 0; q < nv; ++q) {
        const int sz = order[q] == V_TRI ? tb : vb;
        if (used + sz <= smem_budget) {
            g->loc[order[q]] = base_off + used;
            used += sz;
        } else {
            g->loc[order[q]] = -(int)gl - 1;
            gl += sz;
        }
    }
    g->smem_bytes = base_off + used;
    g->scratch_floats = tb / 4;
    *slot_bytes = gl;
}

}  // namespace npfem

// Library-side state of one mesh topology (the opaque npfem_handle of npfem.h).
struct npfem_handle {
    int device = 0;
    int precision = NPFEM_PREC_FP32;
    double dt = 0.0;
    npfem_opts opts{};
    npfem_material mat{};
    npfem::HostTopo host;
    int n = 0, nt = 0, n_pad = 0;
    std::vector<void*> allocs;  // every device allocation owned by the handle
    npfem::TopoDev<float> tf{};
    npfem::TopoDev<double> td{};
    double* ainv64 = nullptr;   // n x n FP64 inverse (unpadded)
    // launch resources (used when this handle is the first of a step call)
    unsigned int* work = nullptr;
    char* scratch = nullptr;
    size_t scratch_bytes = 0;
    float* ws_u = nullptr;  // learned first increments of the cluster kernel's cells
    size_t ws_u_len = 0;
    // temporal warm start: corrections of the last step (element type of the state) and,
    // for FP32, the positions' rounding residues with their FP32 values; valid for the
    // groups and cell counts recorded in hist_sig
    void* hist = nullptr;
    size_t hist_bytes = 0;
    std::vector<long long> hist_sig;
    // carried L-BFGS pairs (opts.warm_history = 2), one record per cell, valid with hist
    void* carry = nullptr;
    size_t carry_bytes = 0;
    // cells the first-iterate pass leaves to the cluster kernel ([0] count, [1] cells
    // that needed iterations, [2] the previous step's [1], then indices)
    unsigned int* defer = nullptr;
    size_t defer_len = 0;
    int sm_count = 0, smem_optin = 0;
    int threads = 512;  // SIMT block size (512 or 640 for FP32 state)
    int use_tc = 1;     // BF16: use the tensor-core cluster kernel when the mesh fits it
    // buffers of npfem_step_host
    float* mlp = nullptr;       // learned warm start parameters on the device (weights BF16-rounded)
    float* tmlp = nullptr;      // temporal network parameters on the device
    void* hx = nullptr;
    void* hv = nullptr;
    void* hf = nullptr;
    npfem_cell_stats* hstats = nullptr;
    size_t host_cells = 0;
    // collisions: planes installed by npfem_set_collisions for the calls through this
    // handle, and the hash table of npfem_collision_detect
    const float* col_planes = nullptr;
    double col_w = 0.0;
    unsigned* col_table = nullptr;
    size_t col_table_len = 0;
    // resident clusters of the tensor-core kernel at tc_smem bytes (queried once)
    int tc_max_clusters = 0, tc_smem = -1;
    // side stream and fork/join events of the idle-SM SIMT launch (tensor-core path)
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // optional timing of the solver kernel launches of npfem_step (event pairs)
    std::vector<cudaEvent_t> tev;
    int tev_used = 0;
    std::mutex mu;

    template <typename X>
    X* alloc(size_t count, int* err)
    {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, count * sizeof(X) + 16);
        if (e != cudaSuccess) {
            *err = npfem::set_error(e == cudaErrorMemoryAllocation ? NPFEM_ERR_OOM : NPFEM_ERR_CUDA,
                        std::string("cudaMalloc: ") + cudaGetErrorString(e));
            return nullptr;
        }
        allocs.push_back(p);
        return static_cast<X*>(p);
    }
    void release()
    {
        for (void* p : allocs) cudaFree(p);
        allocs.clear();
        if (scratch) cudaFree(scratch);
        scratch = nullptr;
        scratch_bytes = 0;
        if (ws_u) cudaFree(ws_u);
        ws_u = nullptr;
        ws_u_len = 0;
        if (hist) cudaFree(hist);
        hist = nullptr;
        hist_bytes = 0;
        hist_sig.clear();
        if (carry) cudaFree(carry);
        carry = nullptr;
        carry_bytes = 0;
        if (defer) cudaFree(defer);
        defer = nullptr;
        defer_len = 0;
        if (col_table) cudaFree(col_table);
        col_table = nullptr;
        col_table_len = 0;
        if (hx) cudaFree(hx);
        if (hv) cudaFree(hv);
        if (hf) cudaFree(hf);
        if (hstats) cudaFree(hstats);
        hx = hv = hf = nullptr;
        hstats = nullptr;
        for (cudaEvent_t e : tev) cudaEventDestroy(e);
        tev.clear();
        tev_used = 0;
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (side_stream) cudaStreamDestroy(side_stream);
        ev_fork = ev_join = nullptr;
        side_stream = nullptr;
    }
};
