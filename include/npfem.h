/*
 * npfem.h -- C ABI of libnpfem.so, the GB300 (sm_103a) npFEM red-blood-cell solver.
 *
 * The library advances many triangulated red-blood-cell membranes by one implicit
 * time step each (Kotsalos, Latt & Chopard, arXiv:1903.06479, Algorithm 1): first
 * guess y_n (Eq. preOptimizationNewton), minimisation of the objective g of
 * Eq. (GeneralizedObjectiveFunction) by L-BFGS with the constant initial matrix
 * H~ = M~/h^2 + L (Sec. 2.1.1) and a backtracking line search, then
 * v_{n+1} = (x_{n+1} - x_n)/h and the post-convergence dissipation of Sec. 2.1.4.
 * Energies: local area preservation and bending (projective, Sec. 2.1.2), global
 * volume conservation (Sec. 2.1.2), modified Skalak strain energy (Sec. 2.1.3).
 *
 * Units: um, us, pN (mass unit pN us^2/um; energy pN um).
 *
 * Conventions shared by every entry point:
 *   - Return value 0 on success, a negative NPFEM_ERR_* code on failure; the
 *     message of the last failure on the calling thread is npfem_last_error().
 *   - Cell state is component-major SoA: for cell c of a mesh with n vertices,
 *     x[c][0..2][0..n-1] (the x, y and z rows), contiguous, cells back to back.
 *     Several meshes (groups) in one call are concatenated in argument order.
 *   - "device" pointers are CUDA global-memory pointers on the handle's device,
 *     owned by the caller; "host" pointers are CPU memory owned by the caller
 *     (pinned memory gives the fastest copies).
 *   - Per-cell non-convergence is not a call error: it is reported in the
 *     optional npfem_cell_stats array.
 */
#ifndef NPFEM_H
#define NPFEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes -------------------------------------------------------- */
#define NPFEM_OK 0
#define NPFEM_ERR_INVALID_ARG (-1) /* a pointer, size or option is out of range        */
#define NPFEM_ERR_BAD_MESH (-2)    /* not a closed, consistently oriented 2-manifold,  */
                                   /* or a degenerate rest triangle                    */
#define NPFEM_ERR_CUDA (-3)        /* a CUDA runtime call failed (message has details) */
#define NPFEM_ERR_OOM (-4)         /* device allocation failed                          */
#define NPFEM_ERR_TIMEOUT (-5)     /* a bounded device wait gave up                      */
#define NPFEM_ERR_NOT_SPD (-6)     /* H~ lost positive definiteness during inversion    */

/* ---- per-cell status (npfem_cell_stats.status) ---------------------------- */
#define NPFEM_CELL_OK 0              /* residual <= tol                                 */
#define NPFEM_CELL_MAXITER 1         /* iteration cap reached; last accepted iterate kept */
#define NPFEM_CELL_LINESEARCH_FAIL 2 /* no step length passed the Armijo test          */
#define NPFEM_CELL_NONFINITE 3       /* NaN/Inf met; x_n kept, v set to zero            */

/* ---- precision of the solve (npfem_opts.precision) ----------------------- */
#define NPFEM_PREC_FP64 0 /* state, energies and the A^-1 contraction in FP64            */
#define NPFEM_PREC_FP32 1 /* state and energies FP32 (sums FP64), A^-1 FP32 on the SIMT  */
                          /* pipes: the plain GPU path                                  */
#define NPFEM_PREC_TF32 2 /* as FP32, but the A^-1 contraction runs on tcgen05 tensor    */
                          /* cores in TF32 with FP32 accumulation: every persistent SIMT */
                          /* block streams A^-1 (TF32, 128 x 32 tiles) from L2 through   */
                          /* shared memory, `refine` refinement sweeps; up to 4096       */
                          /* vertices (npfem_step_static contracts in FP32 instead)      */
#define NPFEM_PREC_BF16 3 /* as FP32, but the A^-1 contraction runs on tcgen05 tensor    */
                          /* cores: BF16 A^-1 resident in tensor memory across a cluster */
                          /* of ceil(n/128) SMs, BF16 q, FP32 accumulation, `refine`     */
                          /* refinement sweeps; meshes above 960 vertices fall back to    */
                          /* the FP32 SIMT contraction                                    */

typedef struct npfem_handle npfem_handle;

/* Closed triangle mesh of one cell topology with its rest shape (host memory).
   tris: [n_tris][3] vertex indices, counter-clockwise seen from outside.
   rest_xyz: [n_verts][3] rest positions in um (AoS). Copied by npfem_create. */
typedef struct {
    int32_t n_verts, n_tris;
    const int32_t* tris;
    const double* rest_xyz;
} npfem_mesh;

/* Material (parameter table of the results section; Sec. 2.1.2-2.1.4).
   B, D: Skalak shear modulus and strain-hardening term (pN/um), Sec. 2.1.3.
   C: area-preservation stiffness (pN/um), weight w_i = C * rest area.
   k_bend: bending stiffness (pN um), weight k_bend * Voronoi area.
   k_vol: volume-conservation weight (pN/um).
   k_mat_hess: stiffness of the optional material term added to L (Sec. 2.1.1,
               "non-PD contribution to the Hessian"); 0 disables it.
   density: mass per rest volume (pN us^2 / um^4); total mass = density * V0.
   alpha_D, beta_D: Rayleigh damping C = alpha_D M + beta_D L (beta_D in us).
   kappa: post-convergence damping coefficient in [0, 1]. */
typedef struct {
    double B, C, D, k_bend, k_vol, k_mat_hess, density, alpha_D, beta_D, kappa;
} npfem_material;

/* Solver options.
   precision: NPFEM_PREC_*.
   lbfgs_m: L-BFGS history window (0..8; 0 = preconditioned descent with H~^-1).
   max_iter: cap on quasi-Newton iterations per step (>= 0).
   tol: stopping residual r = RMS_i(h^2 |grad_i g| / m_i) / mean rest edge length.
   c1: Armijo constant; c2: curvature constant gating the history update.
   max_halvings: line-search trials after alpha = 1 (0..60).
   fixed_alpha: 1 = always take alpha = 1 (the local/global solver of Appendix A).
   equal_mass: 1 = lump the mass equally, 0 = by barycentric rest area.
   armijo_noise: multiple of the estimated rounding error of g added to the
                 Armijo bound (FP32 energies); 0 = exact test.
   refine: NPFEM_PREC_BF16 and NPFEM_PREC_TF32: refinement sweeps of the tensor-core
           A^-1 contraction (0 or 1): r = A^-1 q, then r += A^-1 (q - H~ r).
   fill_idle_sms: NPFEM_PREC_BF16 only: 1 = SMs that the tensor-core clusters leave
           idle run the SIMT solver on the same cells (dynamic split), 0 = clusters only.
   warm_history: 1 = temporal warm start: when a call steps the same groups and cell
           counts as the previous call through meshes[0], each cell starts from
           x^(1) = y + (x_n - y_{n-1}), its previous step's converged correction (kept
           by the library, 12n bytes per cell in the state's type); the iteration still
           runs to the residual tolerance, so stepping other cells in the same layout
           only costs iterations.  With FP32 state the library also keeps, per
           coordinate, the rounding error of storing x_{n+1} = x_n + u in FP32 and the
           FP32 value it belongs to (24n more bytes per cell); the next such call adds
           it back to every coordinate that still holds exactly that value, so that a
           trajectory stepped call after call carries its positions to about twice FP32
           precision (compensated summation).  A coordinate changed by the caller is
           taken as stored.
           2 (the default) = 1, and each solve also starts from the L-BFGS pairs
           (s, y) of the cell's previous solve while that solve took at most 3
           iterations (an addition to Algorithm 1, whose quasi-Newton iteration starts
           every step with an empty history).  Under a force that changes little from
           step to step the carried curvature cuts the iterations (measured: 1.53 ->
           0.84 per cell-step, 1024 x 642 cells, tol 1e-6); where every step needs more
           iterations (a force redrawn at random each step) the pairs are left out and
           the step costs what it costs with 1.  The library keeps one record per cell:
           the history ring, its inner products and the last iteration count
           (2 m 3 n_pad + 4 + m^2 rounded up to a multiple of 4 elements of the state's
           type, n_pad = n rounded up to a multiple of 4); history vectors that
           do not fit in shared memory live in that record while the cell carries.
           0 = off.  Not used by npfem_step_static. */
typedef struct {
    int32_t precision;
    int32_t lbfgs_m;
    int32_t max_iter;
    double tol;
    double c1, c2;
    int32_t max_halvings;
    int32_t fixed_alpha;
    int32_t equal_mass;
    double armijo_noise;
    int32_t refine;
    int32_t fill_idle_sms;
    int32_t warm_history;
} npfem_opts;

/* Per-cell result of one npfem_step call (device memory, 32 bytes). */
typedef struct {
    int32_t iterations;  /* accepted quasi-Newton iterations                 */
    int32_t evaluations; /* objective/gradient evaluations                    */
    int32_t status;      /* NPFEM_CELL_*                                      */
    float residual;      /* final r                                           */
    double objective;    /* final g                                           */
    double volume;       /* enclosed volume at x_{n+1} (um^3)                  */
} npfem_cell_stats;

/* Fills *o with the defaults used throughout the library: FP32, m = 5,
   max_iter = 50, tol = 1e-6, c1 = 1e-4, c2 = 0.9, 30 halvings, area-lumped mass,
   armijo_noise = 4, refine = 1. */
void npfem_default_opts(npfem_opts* o);

/* Creates a handle for one mesh topology on CUDA device `device` and time step dt
   (us): validates the mesh, computes the rest-state tables in FP64 on the host
   (D_m^-1, rest areas, cotangent weights, mixed Voronoi areas, lumped masses, L),
   inverts H~ = M~/h^2 + L in FP64 on the GPU (the one-time prefactorisation of
   Sec. 2.1.1) and keeps A^-1 = H~^-1 resident in the precision of opts->precision.
   The handle owns all its device memory. Blocks until the setup is complete.
   Errors: INVALID_ARG (null pointers, bad sizes/options, dt <= 0), BAD_MESH,
   NOT_SPD, OOM, CUDA. */
int npfem_create(const npfem_mesh* mesh, const npfem_material* mat, const npfem_opts* opts, double dt, int device,
                 npfem_handle** out);

/* Releases the handle and its device memory (synchronises its device). */
int npfem_destroy(npfem_handle* h);

/* Advances every cell of n_groups meshes by one time step (Algorithm 1) on `stream`
   (a cudaStream_t; 0 = legacy default stream): one persistent solver launch over all
   groups (NPFEM_PREC_BF16 with every mesh of at most 960 vertices: one cluster launch
   per group, plus a SIMT launch on SMs the clusters leave idle, forked from and
   joined back to `stream`), preceded by the warm-start launch when a network is
   installed.  With the temporal warm start (opts.warm_history) a cluster group's
   launch is preceded by a SIMT launch over its cells that evaluates each at its first
   iterate and finishes those already within the tolerance; the cluster launch then
   solves only the others.  While more than half of a group's cells needed iterations
   in its previous step, that launch only lists the cells (no evaluation).
   meshes[g] and cells_per_group[g] (host arrays) name each group; all handles must
   share device, precision and dt.
   x, v: device SoA state (float, or double for NPFEM_PREC_FP64), updated in place
   to x_{n+1}, v_{n+1}. f_ext: device SoA external forces (pN), read only.
   dt must equal the handle's dt (a new dt needs a new handle).
   stats: optional device array of sum(cells_per_group) records, or NULL.
   Asynchronous with respect to the host. The library-owned scratch (L-BFGS history
   of large meshes) is per handle set; calls that share handles must be ordered on
   one stream. Errors: INVALID_ARG, CUDA. */
int npfem_step(npfem_handle* const* meshes, int n_groups, const int32_t* cells_per_group, void* x, void* v,
               const void* f_ext, double dt, void* stream, npfem_cell_stats* stats);

/* Allocation-free npfem_step.  The paper has no counterpart: this entry point
   exists for callers that cannot allocate device memory when they step -- a host
   program whose caching allocator has reserved the GPU (so a raw cudaMalloc from
   this library may fail), or a time loop that cannot afford the device-wide
   synchronisation of cudaMalloc/cudaFree.  npfem_step may grow a library-owned
   scratch buffer the first time a mesh needs one; npfem_step_static never
   allocates: its scratch (per-block vector slots for meshes whose solver vectors do
   not fit in shared memory, plus the work counters) is a fixed 32 MiB __device__
   array compiled into the library, held by every GPU that loads the library until
   the process exits.  Arguments, layout, results and errors are those of
   npfem_step, with these differences: every group runs the persistent SIMT solver
   kernel (NPFEM_PREC_BF16 handles included, which then contract a BF16 copy of A^-1
   with FP32 accumulation on the SIMT pipes instead of the tensor-core cluster kernel),
   one launch per distinct
   tuned block size as npfem_step launches its SIMT groups; the temporal warm start
   (opts.warm_history) is not used; with large meshes it may run fewer persistent
   blocks so that their slots fit; and it returns INVALID_ARG when one block's
   scratch exceeds the array.  Every call looks up the array's device address on
   the handles' device (a host reference to it is not a device pointer; the lookup
   allocates nothing).  All calls on a device share the array and it keeps the last
   call's contents (the work counters are cleared on `stream` before each launch):
   calls whose kernels overlap on the GPU race and must be avoided. */
int npfem_step_static(npfem_handle* const* meshes, int n_groups, const int32_t* cells_per_group, void* x, void* v,
                      const void* f_ext, double dt, void* stream, npfem_cell_stats* stats);

/* Same as npfem_step for one handle with HOST buffers x, v, f_ext (SoA, same element
   type; x, v updated in place) and, if stats_host != NULL, host per-cell stats;
   returns after the step's results are in the host buffers.  Pinned host buffers
   that are mapped into the device's address space (cudaHostAlloc, or cudaHostRegister
   with mapping) are stepped in place: the solver kernels read x, v, F_ext and write x,
   v and the stats over the host link while they compute (on a coherent CPU-GPU link
   this overlaps the transfer with the step).  Any other host buffer is copied to
   library-owned device buffers before the step and back after it.  The temporal warm
   start continues a trajectory either way.  Errors as npfem_step, plus OOM. */
int npfem_step_host(npfem_handle* h, int n_cells, void* x_host, void* v_host, const void* f_host, double dt,
                    void* stream, npfem_cell_stats* stats_host);

/* Evaluates the objective g and its gradient (Eq. GeneralizedObjectiveFunction and
   its derivative) for n_cells cells of one handle at positions x with inertia
   target y (device SoA). Writes grad (device SoA) and, per cell, 8 doubles to
   parts (device): inertia, area, Skalak, bending, volume energies, enclosed
   volume, total g, residual r. Used to check the energy kernels one by one.
   Errors: INVALID_ARG, CUDA. */
int npfem_eval(npfem_handle* h, int n_cells, const void* x, const void* y, void* grad, double* parts, void* stream);

/* Copies the handle's FP64 A^-1 (n_verts x n_verts, row-major) to host memory.
   Errors: INVALID_ARG, CUDA. */
int npfem_get_inverse(npfem_handle* h, double* out_host);

/* Copies per-vertex lumped masses (n_verts doubles) and the scalars
   {V0, A0, mean rest edge length, total mass} (4 doubles) to host memory. */
int npfem_get_rest_info(npfem_handle* h, double* masses_host, double* scalars_host);

/* ---- learned warm start (an addition to the paper's method; the paper has no
   counterpart).  A per-vertex MLP (9 -> 64 -> 64 -> 3, tanh, BF16 weights, FP32
   accumulation) proposes the first iterate x^(1) = y + R MLP(features) instead of
   the first guess y of Algorithm 1; the quasi-Newton iteration then runs to the
   same residual tolerance, so the result does not depend on the network.  R is the
   mass-weighted best-fit rotation of the rest shape onto y; the features of vertex
   i are d_i = R^T (y_i - y_cm) - (X_i - X_cm), its cotangent Laplacian over the
   one-ring, and R^T F_ext,i h^2 / m_i.  Parameters are packed FP32:
   W1[64][9] b1[64] W2[64][64] b2[64] W3[3][64] b3[3] mu[9] sigma[9] s_out[3]
   (5016 values; inputs are normalised as (f - mu) / sigma, outputs scaled by
   s_out).  All pointers below are device pointers unless named _host. ---- */

/* Number of packed parameters (5016). */
int npfem_mlp_nparam(void);

/* Training features (FP32, [n_cells * n_verts][9]) of n_cells cells of handle h at
   their first guess y, from x, v, f (device SoA, FP32); if x_next (the converged
   x_{n+1}) is given, also the rest-frame targets R^T (x_{n+1} - y) into target
   ([n_cells * n_verts][3]).  FP32-state handles only.  Errors: INVALID_ARG, CUDA. */
int npfem_ws_features(npfem_handle* h, int n_cells, const float* x, const float* v, const float* f, const float* x_next,
                      float* feat, float* target, void* stream);

/* Mean squared error of the normalised output over n samples (rows idx[0..n) of
   feat/target, or the first n rows if idx is NULL) and its gradient with respect to
   the 4995 weights and biases (grad: 5016 floats, overwritten; the normalisation
   entries stay 0; loss: 1 float, overwritten).  The forward pass is the inference
   network's: BF16-rounded weights, and BF16-rounded operands (normalised inputs,
   first hidden layer) for the two hidden-layer products; the gradient passes the
   operand rounding straight through.  Errors: INVALID_ARG, CUDA. */
int npfem_mlp_loss_grad(const float* params, const float* feat, const float* target, const int32_t* idx, int n,
                        float* grad, float* loss, void* stream);

/* One Adam step (Kingma & Ba, bias-corrected; step >= 1) on the weights and biases of
   params with moment buffers m, v (5016 floats each, caller-owned). */
int npfem_mlp_adam(float* params, float* m, float* v, const float* grad, int step, float lr, float beta1, float beta2,
                   float eps, void* stream);

/* Network outputs (physical units, rest frame, [n][3]) for n feature rows, with the
   arithmetic of the solver's warm start (BF16 operands, FP32 accumulation);
   scratch: 7584 floats (the device layout of the network). */
int npfem_mlp_predict(const float* params, const float* feat, int n, float* out, float* scratch, void* stream);

/* Installs (mode 1: always use the learned first iterate; mode 2: use it only when
   it lowers g, at the cost of one more evaluation) or removes (mode 0,
   params_host = NULL) the warm start of a handle; the weights are rounded to BF16.
   Blocks.  FP32-state handles only.  Errors: INVALID_ARG, OOM, CUDA. */
int npfem_set_warmstart(npfem_handle* h, const float* params_host, int mode);

/* Temporal network (an addition to the paper's method): along a trajectory stepped
   with opts.warm_history, the first iterate of step n is
   y_n + c_{n-1} + R MLP(features) instead of y_n + c_{n-1}, c_k = x_{k+1} - y_k the
   converged correction of step k (kept by the library) and R the mass-weighted best-fit
   rotation of the rest shape onto y_n.  Features of vertex i (9, rest frame): the trend
   R^T (c_{n-1} - c_{n-2}), the force change as a displacement R^T h^2 (F_n - F_{n-1}) / m_i
   and its cotangent Laplacian over the one-ring; the target is R^T (c_n - c_{n-1}).  The
   network has the layout and arithmetic of the warm start above.  With a network
   installed on any group of a call, the trajectory state grows by c_{n-2} and F_{n-1}
   (24n more bytes per cell).  The iteration still runs to the residual tolerance. */

/* Installs (params_host, 5016 FP32, weights rounded to BF16) or removes (NULL) the
   temporal network of h; the next step through h restarts its trajectory.  FP32-state
   handles.  Blocks.  Errors: INVALID_ARG, OOM, CUDA. */
int npfem_set_warmstart_temporal(npfem_handle* h, const float* params_host);

/* Training data of the temporal network for n_cells cells of h (device SoA FP32): the
   features at x, v, f with the previous force f_prev and the corrections c1 = c_{n-1},
   c2 = c_{n-2} into feat ([n_cells * n_verts][9]); with the converged x_next also the
   target into target ([..][3], or NULL) and c_n = x_next - y_n into c_out (SoA, or
   NULL).  Errors: INVALID_ARG, CUDA. */
int npfem_ws_features_temporal(npfem_handle* h, int n_cells, const float* x, const float* v, const float* f,
                               const float* f_prev, const float* c1, const float* c2, const float* x_next, float* feat,
                               float* target, float* c_out, void* stream);

/* The temporal network's first increments u = x^(1) - x_n (device SoA FP32) for n_cells
   cells of h with its installed network (u_y + c1 without one).  Used to check the
   network against a reference.  Errors: INVALID_ARG, CUDA. */
int npfem_ws_guess_temporal(npfem_handle* h, int n_cells, const float* x, const float* v, const float* f,
                            const float* f_prev, const float* c1, const float* c2, float* u_out, void* stream);

/* First iterate of the step (positions, device SoA FP32) for n_cells cells of h
   with the handle's current warm start: y, or y + R MLP(features).  Used to check
   the warm start against a reference.  Errors: INVALID_ARG, CUDA. */
int npfem_ws_guess(npfem_handle* h, int n_cells, const float* x, const float* v, const float* f, float* x1,
                   void* stream);

/* Synchronises the handle's device and reports whether a bounded device-side wait
   of a previous step gave up (the tensor-core path waits for its MMAs with an
   iteration limit): returns NPFEM_ERR_TIMEOUT and clears the flag if so, else 0.
   Errors: INVALID_ARG, CUDA. */
int npfem_check_device(npfem_handle* h);

/* ---- immersed-boundary force step (Sec. 2.3), upstream of npfem_step ------------
   A uniform fluid lattice: node (i, j, k) sits at origin + dx (i, j, k), 0 <= i < nx,
   0 <= j < ny, 0 <= k < nz (um).  Lattice fields are FP32 device arrays, node-major
   with x fastest: index ((k ny + j) nx + i), then the components of the node:
     stress:            8 floats per node, (xx, yy, zz, xy, xz, yz, unused, unused);
     velocity or force: 4 floats per node, (x, y, z, unused).
   Each membrane vertex X_k sees the 4 x 4 x 4 lattice nodes around it, weighted by
   the product of the paper's one-dimensional four-point kernel w(r) (Sec. 2.3) at
   the node's offset in lattice units; nodes outside the lattice contribute nothing
   (a lattice should cover the cells with two nodes to spare).  A_k is a third of the
   areas of the triangles around vertex k and n_k its unit area-weighted normal, both
   at the positions x.  Vertex arrays (x, forces, velocities) use the state's SoA
   layout and group concatenation; FP32-state handles only.  The calls are
   asynchronous on `stream` and allocate nothing.  Errors: INVALID_ARG, CUDA. */
typedef struct {
    double origin[3]; /* position of node (0, 0, 0), um */
    double dx;        /* lattice spacing, um (> 0) */
    int32_t nx, ny, nz;
    int32_t reserved; /* set to 0 */
} npfem_lattice;

/* External force of Eq. Fext from a lattice stress field (pN/um^2, or per unit
   density with rho_fluid the fluid density):
   F_k = rho_fluid A_k (sum over the stencil of sigma(x) w w w) n_k into f_ext (pN).
   mode 0: the whole stencil (Eq. Fext); mode 1: only the stencil nodes on the outside
   of the membrane ((x - X_k) . n_k > 0), their weights renormalised to sum to one
   (the paper disregards the interior fluid); mode 2: the stress of the exterior
   stencil node farthest from X_k (the paper's stabler variant; the first in z, y, x
   order among equals). */
int npfem_ibm_forces(npfem_handle* const* meshes, int n_groups, const int32_t* cells_per_group, const float* x,
                     const npfem_lattice* lattice, const float* sigma, double rho_fluid, int mode, float* f_ext,
                     void* stream);

/* Interpolation of a lattice velocity to the vertices (Sec. 2.3):
   u(X_k) = sum over the stencil of u(x) w w w, into u_vertex (SoA). */
int npfem_ibm_interpolate(npfem_handle* const* meshes, int n_groups, const int32_t* cells_per_group, const float* x,
                          const npfem_lattice* lattice, const float* u_lattice, float* u_vertex, void* stream);

/* Multi-direct forcing (Sec. 2.3, Steps 0-5): with the fluid velocity u* on the
   lattice (u_lattice) and the membrane velocity U_k at the vertices (u_vertex, e.g.
   the v of npfem_step), f_0 = (U_k - u*(X_k))/dt_fluid, then `cycles` times: spread
   f_l(x) = sum_k f_l(X_k) (w w w / dx^3) A_k dx (a membrane one spacing thick),
   u_l = u* + dt_fluid f_l, f_{l+1}(X_k) = f_l(X_k) + (U_k - u_l(X_k))/dt_fluid.
   Writes the final Lagrangian force f_L to f_vertex (SoA, um/us^2) and its spread, the
   body force f_imm of the fluid step, to f_lattice (4 floats per node; also used as
   the working lattice, so it must not alias u_lattice).  Spreading adds with atomics,
   so f_lattice is reproducible to FP32 rounding only.  cycles in 0..1000. */
int npfem_ibm_forcing(npfem_handle* const* meshes, int n_groups, const int32_t* cells_per_group, const float* x,
                      const float* u_vertex, const npfem_lattice* lattice, const float* u_lattice, double dt_fluid,
                      int cycles, float* f_vertex, float* f_lattice, void* stream);

/* ---- collisions between cells (Sec. 3.3) --------------------------------------
   Detection: for every vertex of the call's cells (FP32 SoA positions x, groups as
   in npfem_step), the nearest vertex of ANOTHER cell within `cutoff` (um; ties go to
   the lowest vertex index, counting cells of all groups in order), found through a
   uniform grid of bins of the cutoff's size.  planes (device, 4 floats per vertex,
   vertices in the order of x): the unit outward normal n of the neighbouring cell at
   that vertex (normalised area-weighted normal) and the plane's offset
   n . (x_neighbour - x_0), x_0 the vertex's own cell's first vertex; (0, 0, 0, 0)
   when there is no neighbour.  stats (device, 2 unsigned): vertices with a
   neighbour, and vertices left out of the grid by a full bin (16 vertices per
   hashed bin; nonzero means some neighbours may have been missed).  Grows a
   library-owned table of 68 bytes per bin (bins: a power of two >= 2 vertices) on
   meshes[0].  FP32-state handles.  Errors: INVALID_ARG, OOM, CUDA. */
int npfem_collision_detect(npfem_handle* const* meshes, int n_groups, const int32_t* cells_per_group, const float* x,
                           double cutoff, float* planes, unsigned int* stats, void* stream);

/* Installs collision planes (device, the layout npfem_collision_detect writes, for
   the same groups and cells) and their weight w_col (pN/um) for the npfem_step and
   npfem_step_static calls whose first handle is h, until replaced or removed
   (planes = NULL).  In those steps a vertex whose position x_i lies behind its plane
   (d = offset - n . (x_i - x_0) > 0) adds the collision energy (w_col/2) d^2 and
   force w_col d n to the objective (the non-PD term of Sec. 3.3), tested again at
   every evaluation so that the term vanishes once the vertex no longer penetrates;
   the constant H~ is unchanged.  The planes are read during the steps, so keep the
   array alive; re-detect between steps.  Errors: INVALID_ARG. */
int npfem_set_collisions(npfem_handle* h, const float* planes, double w_col);

/* Test hook for the reporting path of the bounded device waits: sets the handle's
   device-wait flag exactly as a kernel whose wait gave up sets it (a host-side write;
   no device work is made to wait), so that the next npfem_check_device returns
   NPFEM_ERR_TIMEOUT.  Synchronises the handle's device.  Errors: INVALID_ARG, CUDA. */
int npfem_flag_wait_timeout(npfem_handle* h);

/* Message of the last failure on the calling thread ("" if none). */
const char* npfem_last_error(void);

/* Launch-shape autotuner: for every group (cells_per_group[g] > 0) times
   `trial_steps` back-to-back steps of that group alone (after one untimed step) on
   copies of its x, v for each candidate shape, and keeps the fastest in the handle:
   SIMT blocks of 512 or 640 threads (640 for FP32 state only), and for NPFEM_PREC_BF16
   meshes of at most 960 vertices the tensor-core cluster kernel with and without the
   idle-SM SIMT launch (with the handle's temporal warm start, as the steps that
   follow will run).  x, v are not modified.  trial_ms (optional, 5 floats per
   group) receives the mean trial-step time of each candidate in the order SIMT 512,
   SIMT 640, clusters + idle-SM 512, clusters only, clusters + idle-SM 640 (-1 where
   a candidate does not apply).  Blocks.  Errors: INVALID_ARG, CUDA, OOM. */
int npfem_autotune(npfem_handle* const* meshes, int n_groups, const int32_t* cells_per_group, const void* x,
                   const void* v, const void* f_ext, double dt, int trial_steps, float* trial_ms);

/* The launch shape a handle uses: *use_tc (cluster kernel), *threads (SIMT block
   size), *fill_idle_sms.  Errors: INVALID_ARG. */
int npfem_get_tuning(const npfem_handle* h, int* use_tc, int* threads, int* fill_idle_sms);

/* A CUDA graph of `steps` consecutive npfem_step calls on fixed state buffers (the
   batching pattern of a time loop: the whole step, warm start and solver launches
   included, replays as one graph launch).  Creation runs two steps on temporary copies
   of x and v (sizing the handles' buffers; x, v are not modified, stats is written)
   and captures the steps on an internal stream.  The graph holds the pointers it was
   created with; it must be destroyed before the handles.  Errors: INVALID_ARG, CUDA,
   OOM. */
typedef struct npfem_graph npfem_graph;
int npfem_graph_create(npfem_handle* const* meshes, int n_groups, const int32_t* cells_per_group, void* x, void* v,
                       const void* f_ext, double dt, int steps, npfem_cell_stats* stats, npfem_graph** out);
/* Enqueues the graph's steps on `stream` (asynchronous; npfem_launch_count grows by
   the kernels of the captured steps).  Errors: INVALID_ARG, CUDA. */
int npfem_graph_launch(npfem_graph* g, void* stream);
int npfem_graph_destroy(npfem_graph* g);

/* Timing of the solver kernels of npfem_step, for measurement: with capacity > 0,
   the next `capacity` npfem_step calls whose first handle is h record a CUDA event
   before and after their solver launch(es) (after the warm-start launch) on the
   call's stream; capacity 0 stops recording and frees the events.  Blocks.
   Errors: INVALID_ARG, CUDA. */
int npfem_kernel_timing(npfem_handle* h, int capacity);

/* Durations in ms of the recorded solver launches (oldest first) into ms_out (up to
   max entries, *count set to the number written); synchronises on the events and
   restarts the recording.  Errors: INVALID_ARG, CUDA. */
int npfem_kernel_times(npfem_handle* h, float* ms_out, int max, int* count);

/* Duration in ms of the first recorded solver launch pair (synchronises on it, keeps
   the recording): with a CUDA graph captured while timing was on, the pair is
   re-recorded by every replay, so this reads the latest replay.
   Errors: INVALID_ARG (nothing recorded), CUDA. */
int npfem_kernel_time_last(npfem_handle* h, float* ms);

/* Number of kernels the library has launched in this process (all devices, all
   entry points), for counting device work; thread-safe, never fails. */
unsigned long long npfem_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* NPFEM_H */
