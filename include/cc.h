/*
 * cc.h — C ABI of the GB300 (sm_103a) Coordinate Condensation library.
 *
 * The library advances implicit elastodynamics or quasistatics on linear
 * tetrahedral meshes by solving, per time step,
 *
 *     x^{t+1} = argmin_x E(x),                                   (Eq. 1)
 *     E(x)    = 1/2 (x - xt)^T M (x - xt) + h^2 Psi(x)            (Eq. 2)
 *
 * (quasistatic: E = Psi), with the graph-coloured per-vertex Coordinate
 * Condensation sweep of Section 3 (Algorithm 1 is its one-colour Jacobi
 * form).  Psi is stable Neo-Hookean in its rest-stable, log-free form
 *     Psi(F) = mu/2 (|F|^2 - 3) - mu (J - 1) + lam_hat/2 (J - 1)^2,
 *     lam_hat = lam + mu, J = det F,
 * whose rest linearisation is Hooke's law for (E, nu).  M is the lumped
 * mass (rho V_t / 4 per tet corner).
 *
 * Conventions for every entry point
 *   - Device positions are caller-owned float64 buffers in SoA layout
 *     [3][n]: x[a * n + j] is coordinate a of vertex j.  Pinned (Dirichlet)
 *     vertices keep whatever the caller stored there; the library never
 *     writes them.
 *   - Host arrays passed to cc_build_mesh are copied; the caller keeps them.
 *   - All device work is ordered on the stream given to cc_build_mesh
 *     (a cudaStream_t, or NULL for the legacy default stream).  Entry points
 *     that return host scalars synchronise that stream.
 *   - Every call returns a cc_status; CC_OK is 0.  No exception or abort
 *     crosses the ABI.  cc_last_error() returns a thread-local, human
 *     readable message for the last failing call on this thread.
 *   - A cc_mesh is not thread-safe: serialise calls on one mesh.
 */
#ifndef CC_GB300_H
#define CC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CC_OK = 0,
  CC_ERR_INVALID_ARG = 1,   /* bad pointer, size, enum or mesh */
  CC_ERR_CUDA = 2,          /* a CUDA runtime call failed (message has it) */
  CC_ERR_OOM = 3,           /* device allocation failed */
  CC_ERR_NUMERIC = 4,       /* a NaN or Inf appeared in an update or residual */
  CC_ERR_TIMEOUT = 5,       /* a bounded device wait expired */
  CC_ERR_NOT_CONVERGED = 6, /* max_iters reached; stats are valid */
  CC_ERR_STATE = 7          /* call made in the wrong order (e.g. no subspace) */
} cc_status;

typedef struct cc_mesh cc_mesh; /* opaque; owns device and host rest data */

/* Energy density Psi(F) of a mesh (E, nu -> Lame mu, lam):
 *   CC_MODEL_SNH  stable Neo-Hookean, rest-stable form without the log term,
 *                 Psi = mu/2 (|F|^2 - 3) - mu (J - 1) + (lam + mu)/2 (J - 1)^2
 *   CC_MODEL_FCR  Fixed Corotational (the paper's material, Sec. 4.1),
 *                 Psi = mu |F - R|^2 + lam/2 (J - 1)^2, R the polar rotation of F;
 *                 every tet must stay non-inverted (det F > 0): an inverted tet
 *                 makes the update non-finite (CC_ERR_NUMERIC). */
typedef enum { CC_MODEL_SNH = 0, CC_MODEL_FCR = 1 } cc_model;

typedef struct {
  double E;      /* Young's modulus [Pa], > 0 */
  double nu;     /* Poisson ratio, in (-1, 0.5) */
  double rho;    /* density [kg/m^3], >= 0 (used by the mass matrix only) */
  int32_t model; /* cc_model (0: stable Neo-Hookean) */
} cc_material;

/* Arithmetic of a sweep.
 *   CC_PREC_FP64  : everything in float64 ("plain").
 *   CC_PREC_MIXED : per-tet Hessians, the Hessian blocks and the subspace
 *                   coupling products (H U, U^T H U, U^T g) in float32; the
 *                   per-tet gradient in float-float (pairs of float32, about
 *                   48 significant bits); the Schur condensation, the 3x3
 *                   solves, the position update and the residual reduction
 *                   in float64. */
typedef enum { CC_PREC_FP64 = 0, CC_PREC_MIXED = 1 } cc_precision;

/* CC_SCHED_COLORED: for each colour in turn, g and H are re-evaluated at the
 *   current x and every free vertex of that colour is updated (Gauss-Seidel
 *   across colours, Jacobi within one).  CC_SCHED_JACOBI: one evaluation,
 *   every free vertex updated from it (Algorithm 1). */
typedef enum { CC_SCHED_COLORED = 0, CC_SCHED_JACOBI = 1 } cc_schedule;

/* Local update of a free vertex i (g, H at the current x; U = U_i):
 *   CC_UPDATE_CC   dx_i = -(H_ii - S)^{-1} gt,  S = A Ht^{-1} A^T,
 *                  gt = g_i - A Ht^{-1} b,  A = H_iC U, Ht = U^T H_CC U,
 *                  b = U^T g_C                         (Eq. 9-12)
 *   CC_UPDATE_CD   dx_i = -H_ii^{-1} g_i               (Eq. 3, one Newton step)
 *   CC_UPDATE_JGS2 dx_i = -(H_ii + Ht)^{-1} (g_i + b)  (Eq. 7)
 * Guard: a 3x3 system counts as SPD when all Cholesky pivots exceed 1e-12
 * times its largest diagonal entry.  CC falls back to the CD step when U_i is
 * empty, Ht fails the test, or H_ii - S fails it; JGS2 when H_ii + Ht fails.
 * Fallbacks are counted in the stats, they are not errors. */
typedef enum { CC_UPDATE_CC = 0, CC_UPDATE_CD = 1, CC_UPDATE_JGS2 = 2 } cc_update;

typedef struct {
  cc_update update;
  cc_schedule schedule;
  cc_precision precision;
  int32_t color_begin; /* first colour to run (0 for a whole sweep) */
  int32_t color_end;   /* one past the last colour; -1 = all.  Ignored for Jacobi. */
  int32_t corotated;   /* 1: corotated bases (Sec. 3.1): at the start of the sweep every
                          vertex's rotation R_j is estimated from the current x and the
                          bases become U_i^rot[j] = R_j U_i[j].  R_j is the orthogonal
                          polar factor of the neighbourhood's least-squares deformation
                          gradient F_j = A_j C_j^{-1}, A_j = sum over the 1-ring of
                          (x_l - x_j)(X_l - X_j)^T, C_j = sum of (X_l - X_j)(X_l - X_j)^T
                          (I when det F_j <= 0). */
} cc_sweep_opts;

typedef struct {
  int64_t updates;          /* local solves performed */
  int64_t fallback_empty;   /* CC/JGS2 with an empty basis -> CD step */
  int64_t fallback_reduced; /* Ht (CC) / H_ii + Ht (JGS2) not SPD -> CD step */
  int64_t fallback_schur;   /* H_ii - S not SPD -> CD step */
} cc_sweep_stats;

typedef struct {
  cc_update update;
  cc_schedule schedule;
  cc_precision precision;
  double tol;          /* stop when ||g_free(x)|| <= tol * ||g_free(x_start)|| */
  int32_t max_iters;   /* sweeps at most */
  int32_t min_iters;   /* sweeps at least (0 normally) */
  int32_t check_every; /* read the residual on the host every this many sweeps (>= 1) */
  int32_t use_graph;   /* 1: replay the check_every sweeps as one captured CUDA graph */
  double* residual_history; /* host, max_iters + 1 entries (or NULL): ||g_free|| after
                               each checked sweep, entry 0 = start; unchecked entries = -1 */
  int32_t corotated;   /* 1: corotated bases, rotations re-estimated every sweep (see cc_sweep_opts) */
  int32_t restart_every; /* > 0: restarted CC, the bases are rebuilt from the Hessian at the
                            current x (cc_build_subspace_at) before sweeps r, 2r, ... */
  int32_t line_search; /* 1: global backtracking line search (Sec. 4.4): every sweep's displacement
                          d = x_sweep - x becomes a direction, x <- x + a d with the largest
                          a in {1, 1/2, ..., 2^-29} for which E(x + a d) <= E(x) (float64
                          energy), a = 0 if none.  Host-synchronous, no graph replay;
                          cc_solve_batch takes one such step per mesh on its own energy. */
} cc_step_opts;

typedef struct {
  int32_t iterations;  /* sweeps performed */
  int32_t converged;   /* 1 if the tolerance was met */
  double g0;           /* ||g_free|| at the start */
  double g_final;      /* ||g_free|| at the end */
  double energy_final; /* E at the end (float64) */
  cc_sweep_stats sweeps; /* summed over the sweeps */
} cc_step_stats;

typedef struct {
  int64_t n, T, n_free, nnz_blocks;
  int32_t num_colors;  /* 0 until cc_color */
  int32_t k_ring;      /* 0 until cc_build_subspace */
  int64_t support_total; /* sum of |S_i| (0 until cc_build_subspace) */
  int32_t support_max;
  int32_t max_valence; /* tets per vertex, maximum */
  int64_t patch_float64; /* patches of the last basis build that the float32-factor, float64-refined
                            solve handed to the plain float64 solve (non-positive float32 pivot, or
                            refinement not down to 1e-11); 0 when every patch settled */
  int64_t patch_solved;  /* patches the last cc_build_subspace solved */
  int64_t patch_shared;  /* bases it copied from a vertex with an identical patch instead */
} cc_mesh_info;

/* Arrays cc_export can copy to the host (element type in brackets). */
typedef enum {
  CC_ARR_VT_PTR = 0,    /* [n+1] int64: vertex -> tet CSR offsets */
  CC_ARR_VT_TET = 1,    /* [4T] int32: incident tets, ascending per vertex */
  CC_ARR_VT_CORNER = 2, /* [4T] int32: corner of the vertex in that tet */
  CC_ARR_NBR_PTR = 3,   /* [n+1] int64: 1-ring CSR offsets (self excluded) */
  CC_ARR_NBR_IDX = 4,   /* [sum] int32: 1-ring neighbours, ascending */
  CC_ARR_COLOR = 5,     /* [n] int32: greedy colour of every vertex */
  CC_ARR_SUP_PTR = 6,   /* [n+1] int64: support CSR offsets (empty for pinned) */
  CC_ARR_SUP_IDX = 7,   /* [support_total] int32: S_i, ascending */
  CC_ARR_U = 8,         /* [support_total][3][3] float64: U_i blocks, row-major
                           (row = DOF of the support vertex, col = direction) */
  CC_ARR_MASS = 9       /* [n] float64: lumped masses */
} cc_array;

/* Builds the rest data of a mesh (shape matrices, volumes, lumped masses,
 * vertex-tet and 1-ring adjacency, the 3x3-block Hessian pattern).
 *   X       host [n][3] float64 rest positions (row-major, AoS)
 *   tets    host [T][4] int32 vertex ids; every tet must have positive
 *           volume after orientation (corners 1 and 2 are swapped when the
 *           signed volume is negative; a zero-volume tet is an error)
 *   pinned  host [n] uint8, 1 = Dirichlet vertex (may be NULL: none)
 *   h       time step (> 0: dynamic energy of Eq. 2; 0: quasistatic E = Psi)
 *   gravity host [3] acceleration folded into the inertial target by
 *           cc_solve_step (may be NULL: zero); ignored when h == 0
 *   stream  cudaStream_t for all work on this mesh (NULL: default stream)
 * Errors: CC_ERR_INVALID_ARG (n < 4, T < 1, ids out of range, bad material,
 * degenerate tet), CC_ERR_OOM, CC_ERR_CUDA. */
cc_status cc_build_mesh(const double* X, int64_t n, const int32_t* tets, int64_t T,
                        const uint8_t* pinned, const cc_material* mat, double h,
                        const double* gravity, void* stream, cc_mesh** out);

/* Frees all device and host memory of the mesh (NULL is a no-op). */
void cc_destroy_mesh(cc_mesh* mesh);

/* Greedy colouring of the 1-ring graph (vertices share a tet) on the GPU:
 * every vertex, pinned ones included, takes the smallest colour unused by its
 * lower-id neighbours (Jones-Plassmann rounds with index priority, identical
 * to sequential greedy in ascending id).  Same-coloured vertices share no
 * tet.  colors_out: host [n] int32 or NULL; num_colors: host or NULL. */
cc_status cc_color(cc_mesh* mesh, int32_t* colors_out, int32_t* num_colors);

/* A colouring chosen by the caller instead (the coloured schedule of
 * Alg. 1's local updates needs only that no two vertices of a tet share a
 * colour; which valid colouring is used changes the order of the updates,
 * not the method).  colors: host [n] int32 in [0, num_colors).  Checked:
 * CC_ERR_INVALID_ARG if a colour is out of range or two vertices of one tet
 * share a colour.  Example: every Kuhn grid (every edge offset's coordinates
 * sum to 1, 2 or 3) is coloured by (i + j + k) mod 4 of the lattice
 * coordinates, 4 colours where the greedy colouring of cc_color uses 8. */
cc_status cc_set_colors(cc_mesh* mesh, const int32_t* colors, int32_t num_colors);

/* Perturbation bases U_i = -H_PP^{-1} H_Pi at the rest configuration
 * (Eq. 5, Sec. 3.1), one per free vertex i, on the patch P = S_i: the free
 * vertices within k_ring 1-ring hops of i, i excluded, every DOF outside P
 * held fixed.  H is the rest Hessian of E (dynamic meshes: M + h^2 K).
 * Patches of at most 192 unknowns (every 2-ring of a Kuhn grid): float32
 * Cholesky in shared memory with float64 iterative refinement of U to
 * float64 accuracy; larger patches, and those the refinement declines
 * (cc_mesh_info.patch_float64), by dense float64 Cholesky.  Vertices whose
 * patches are translated copies of one another (regular grids: equal support
 * offsets, 1-ring geometry and material) share one solve: the others copy
 * its basis, and every copy is kept only if it satisfies its own patch's
 * Eq. 5 (||H_PP U_i + H_Pi|| / ||H_Pi||) to within 4x the residual of the
 * patch it was computed on (or 1e-10), else it is solved on its own
 * (cc_mesh_info.patch_solved / patch_shared).  A patch
 * whose H_PP is not positive definite keeps its previous basis and fails the
 * call with CC_ERR_NUMERIC.  k_ring in [1, 4].
 * Requires cc_color first (CC_ERR_STATE otherwise). */
cc_status cc_build_subspace(cc_mesh* mesh, int32_t k_ring);

/* Restarted bases (Sec. 4.4, "Subspace quality"): rebuilds every U_i on its
 * current support from the Hessian at x_dev (device [3][n] float64) instead
 * of the rest configuration, in place.  A patch whose H_PP is not positive
 * definite (dense Cholesky) keeps its current basis; kept (host, may be NULL)
 * receives their number.  Requires a subspace (cc_build_subspace). */
cc_status cc_build_subspace_at(cc_mesh* mesh, const double* x_dev, int64_t* kept);

/* Replaces the bases with caller-supplied ones (e.g. noisy or learned):
 * sup_ptr host [n+1] int64, sup_idx host [sup_ptr[n]] int32 (ascending,
 * free vertices other than i), U host [sup_ptr[n]][3][3] float64.
 * Pinned vertices must have empty supports. */
cc_status cc_set_subspace(cc_mesh* mesh, const int64_t* sup_ptr, const int32_t* sup_idx,
                          const double* U);

/* E(x) and the gradient at x.
 *   x_dev       device [3][n] float64
 *   xtilde_dev  device [3][n] inertial target (required iff h > 0)
 *   energy      host out (may be NULL)
 *   grad_dev    device [3][n] float64 out (may be NULL); pinned rows are 0
 *   grad_norm   host out: ||g_free||_2 (may be NULL)
 * precision selects the gradient arithmetic (float64 or float-float). */
cc_status cc_energy_grad(cc_mesh* mesh, const double* x_dev, const double* xtilde_dev,
                         cc_precision precision, double* energy, double* grad_dev,
                         double* grad_norm);

/* One sweep (or the colour range in opts) updating the free rows of x_dev
 * in place.  Requires cc_color; CC and JGS2 also require a subspace.
 * stats: host out or NULL.  CC_ERR_NUMERIC when an update is not finite
 * (x is then left partially updated). */
cc_status cc_sweep(cc_mesh* mesh, double* x_dev, const double* xtilde_dev,
                   const cc_sweep_opts* opts, cc_sweep_stats* stats);

/* One quasistatic solve (v_dev == NULL) or one backward Euler step:
 * xt = x + h v + h^2 gravity; sweeps from x until the tolerance or
 * max_iters; then v = (x_new - x_old) / h.  x_dev, v_dev device [3][n].
 * Returns CC_ERR_NOT_CONVERGED (stats valid, x updated) when max_iters is
 * reached first. */
cc_status cc_solve_step(cc_mesh* mesh, double* x_dev, double* v_dev, const cc_step_opts* opts,
                        cc_step_stats* stats);

cc_status cc_get_info(const cc_mesh* mesh, cc_mesh_info* info);

/* Copies one of the cc_array arrays to host memory dst of capacity elements.
 * count (host, may be NULL) receives the array's length.  CC_ERR_INVALID_ARG
 * if capacity is too small; CC_ERR_STATE if the array does not exist yet. */
cc_status cc_export(const cc_mesh* mesh, cc_array which, void* dst, int64_t capacity,
                    int64_t* count);

/* Per-kernel-class device timing for profiling a caller's timed region.
 * When enabled, every kernel launch of the mesh is bracketed by a pair of
 * CUDA events recorded on the mesh's stream; cc_profile_read synchronises
 * the stream, returns the summed milliseconds and launch counts per class
 * and resets the accumulators.  Classes: 0 per-tet derivatives, 1 gather
 * (gradient + Hessian blocks), 2 local solve (coupling products + Schur
 * solve), 3 reductions, 4 other (mirrors, targets, velocities). */
#define CC_PROFILE_CLASSES 5
typedef struct {
  double ms[CC_PROFILE_CLASSES];
  int64_t launches[CC_PROFILE_CLASSES];
  int64_t total_launches; /* kernel launches since the last read (counted
                             whether or not event timing is enabled) */
} cc_profile;

cc_status cc_profile_enable(cc_mesh* mesh, int32_t on);
cc_status cc_profile_read(cc_mesh* mesh, cc_profile* out);

/* Allocation-free variant of the basis construction (no counterpart in the
 * paper).  It is meant for callers that must not have device memory
 * allocated on their behalf: processes whose GPU memory is entirely reserved
 * by their own pool allocator, where a cudaMalloc would fail or fragment the
 * pool, and time-critical loops that cannot absorb cudaMalloc's implicit
 * synchronisation.  It calls no cudaMalloc, cudaFree or other allocating
 * routine.  Instead of a cudaMalloc'ed workspace it uses one file-scope
 * 16 MiB device array (2^21 doubles) that the CUDA runtime reserves on every
 * GPU that loads this library and keeps until the process exits.
 *
 * It computes, for each vertex i in verts, U_i = -H_PP^{-1} H_Pi on the
 * patch P = S_i (the same dense Cholesky as cc_build_subspace) and writes
 * the blocks of S_i into U_out.  Everything is caller-owned device memory:
 *   H_blocks  [nnzb][3][3] float64 Hessian blocks (row-major within a block)
 *   row_ptr   [n+1] int32, col_idx [nnzb] int32: block rows, columns
 *             ascending, diagonal block included
 *   verts     [count] int32 vertices to process (their supports non-empty
 *             or empty; empty ones are skipped)
 *   sup_ptr   [n+1] int32, sup_idx [sup_ptr[n]] int32 ascending supports
 *   U_out     [sup_ptr[n]][3][3] float64 output (only the rows of verts'
 *             supports are written)
 *   max_support  largest |S_i| over verts (host int); values whose dense
 *             patch does not fit the array (above CC_NOALLOC_MAX_SUPPORT)
 *             are rejected with CC_ERR_INVALID_ARG before any GPU work, and
 *             so is a listed vertex whose support is larger than max_support
 *             (a small device pass reads the supports first; no patch is
 *             solved and U_out is untouched)
 *   stream    cudaStream_t (NULL: default stream); the call synchronises it
 * The first call on a device looks up the array's device address (once per
 * device, with that device current, under a lock, so concurrent first calls
 * from several host threads are safe); make that first call before any
 * stream capture.  All calls on a device share the array and it keeps the last
 * call's contents; the kernel clears what must start at zero.  Calls that
 * overlap on the GPU (e.g. on two streams at once) race on the array: keep
 * them ordered.  CC_ERR_NUMERIC if a patch matrix is not positive definite. */
#define CC_NOALLOC_MAX_SUPPORT 482
cc_status cc_build_bases_noalloc(const double* H_blocks, const int32_t* row_ptr, const int32_t* col_idx,
                                 const int32_t* verts, int64_t count, const int32_t* sup_ptr,
                                 const int32_t* sup_idx, int32_t max_support, double* U_out,
                                 void* stream);

/* A batch: `count` independent meshes solved together (no counterpart in
 * the paper).  The library stores them as one disjoint union: mesh b's
 * vertices follow mesh b-1's in the device arrays (offsets in
 * cc_batch_offsets), tets are renumbered accordingly, and every kernel launch
 * of a sweep covers all meshes.  Colours, supports and bases of each mesh are
 * exactly those it would get on its own (components never interact, and the
 * greedy colouring of the union in ascending id is the per-mesh colouring).
 * Each mesh keeps its own material (E, nu, rho); the energy model, the time
 * step h and gravity are shared (meshes with different models are rejected). */
typedef struct {
  const double* X;       /* host [n][3] */
  int64_t n;
  const int32_t* tets;   /* host [T][4], ids local to this mesh */
  int64_t T;
  const uint8_t* pinned; /* host [n] or NULL */
  cc_material mat;
} cc_mesh_desc;

cc_status cc_build_batch(const cc_mesh_desc* meshes, int32_t count, double h, const double* gravity,
                         void* stream, cc_mesh** out);

/* Vertex offsets of the meshes of a batch: offsets host [count+1]. */
cc_status cc_batch_offsets(const cc_mesh* mesh, int64_t* offsets, int32_t* count);

typedef struct {
  int32_t* iterations;  /* host [count]: sweeps each mesh ran before it stopped */
  int32_t* status;      /* host [count]: 1 converged, 0 max_iters reached, -1 diverged
                           (residual non-finite or above 1e6 times its start) */
  double* g0;           /* host [count]: ||g_free|| at the start */
  double* g_final;      /* host [count]: ||g_free|| when the mesh stopped */
  int32_t sweeps;       /* out: sweeps launched until every mesh had stopped */
  cc_sweep_stats totals;/* out: fallback counts over all meshes */
} cc_batch_stats;

/* Solves every mesh of a batch (cc_solve_step semantics per mesh): the
 * residual of each mesh is reduced separately at every check, and a mesh that
 * converged or diverged stops moving (its vertices are skipped by the
 * condensation kernel) while the others continue.  x_dev, v_dev: device
 * [3][n_total] (v_dev NULL for quasistatics).  opts->line_search: every mesh
 * takes its own backtracking step on its own energy after each sweep (one
 * launch per trial for all meshes; a mesh without a decreasing step stays
 * put).  opts->restart_every: the bases of the whole batch are rebuilt at the
 * current x every that many sweeps.  Returns CC_OK when every mesh
 * converged, CC_ERR_NOT_CONVERGED otherwise (stats valid). */
cc_status cc_solve_batch(cc_mesh* mesh, double* x_dev, double* v_dev, const cc_step_opts* opts,
                         cc_batch_stats* stats);

/* Solves several independent meshes at once (no counterpart in the paper):
 * mesh k runs cc_solve_step(meshes[k], x_dev[k], v_dev[k], &opts[k],
 * &stats[k]) on its own stream (the one given to cc_build_mesh /
 * cc_build_batch), one host thread per mesh (the calling thread takes mesh
 * 0), so that the colours' short kernels of different meshes overlap on the
 * GPU instead of queueing behind one another.  Results are those of the
 * separate cc_solve_step calls, bit for bit.
 *   count    number of meshes (0: nothing to do)
 *   meshes   host [count], distinct meshes with distinct streams that are
 *            neither NULL nor the legacy / per-thread default stream
 *   x_dev    host [count] of device [3][n_k] float64, disjoint
 *   v_dev    host [count] of device [3][n_k] (entries NULL for quasistatic
 *            meshes); the array itself may be NULL when every mesh is
 *            quasistatic
 *   opts     host [count]; residual_history pointers, where given, distinct
 *   stats    host [count] out (may be NULL)
 *   status   host [count] out (may be NULL): each mesh's cc_solve_step status
 * Every mesh runs to its own end even when another fails.  Returns CC_OK when
 * every mesh converged, else the first error other than
 * CC_ERR_NOT_CONVERGED in mesh order, else CC_ERR_NOT_CONVERGED;
 * cc_last_error names the mesh.  CC_ERR_INVALID_ARG (nothing runs) for a
 * NULL argument, a repeated mesh, stream or history, or a default stream.
 * The worker threads use the calling thread's current CUDA device; a mesh
 * whose thread cannot be started runs on the calling thread after mesh 0
 * (same results, less overlap), and every started thread has been joined
 * when the call returns. */
cc_status cc_solve_concurrent(int32_t count, cc_mesh* const* meshes, double* const* x_dev,
                              double* const* v_dev, const cc_step_opts* opts, cc_step_stats* stats,
                              cc_status* status);

/* Launch-configuration autotuner (no counterpart in the paper).  Times
 * `sweeps` coloured CC sweeps from x_dev for each candidate configuration,
 * one parameter at a time in this order: the sweep variant
 * (cc_set_sweep_variant), threads per vertex of the coupling kernel (32 = one
 * warp per vertex, 64, 128, 256), then, unless one warp won, threads per
 * block row of the coupling kernel (1, 2, 4, 8), then block rows per CTA of
 * the row gather (2, 4, 8 warps); it keeps the fastest of each for this
 * mesh.  x_dev is not modified (the sweeps run on a private copy).  Requires
 * cc_color and a subspace.  Results with different configurations agree to
 * the working precision's rounding (the coupling kernel's partial sums are
 * grouped differently). */
typedef struct {
  int32_t couple_threads;
  int32_t couple_row_lanes;
  int32_t gather_warps;
  double couple_ms[4];    /* ms per sweep with 32, 64, 128, 256 threads per vertex */
  double row_lanes_ms[4]; /* ms per sweep with 1, 2, 4, 8 threads per block row (0: not timed) */
  double gather_ms[3];    /* ms per sweep with 2, 4, 8 warps per block */
  int32_t rows_from_positions;  /* chosen sweep variant (cc_set_sweep_variant) */
  int32_t fused_condense;
  double variant_ms[4];   /* ms per sweep with (rows_from_positions, fused_condense) = (0,0), (0,1), (1,0),
                             (1,1), at the default launch shapes; variants a mesh cannot use stay 0 */
} cc_tune_result;

cc_status cc_autotune(cc_mesh* mesh, const double* x_dev, const double* xtilde_dev, cc_precision precision,
                      int32_t sweeps, cc_tune_result* out);

/* Sets the launch shapes cc_autotune chooses among (no counterpart in the
 * paper): couple_threads in {32 (one warp per vertex), 64, 128, 256},
 * gather_warps in {2, 4, 8}, couple_row_lanes (threads sharing one block row
 * of the support in the coupling kernel with 64 or more threads) in
 * {1, 2, 4, 8}; 0 keeps the current value.  CC_ERR_INVALID_ARG for any other
 * value. */
cc_status cc_set_launch_shape(cc_mesh* mesh, int32_t couple_threads, int32_t gather_warps, int32_t couple_row_lanes);

/* Selects between equivalent kernel variants of the sweep (no counterpart in
 * the paper; both settings compute Eq. 9-12 on the same data):
 *   rows_from_positions  1: the mixed path's stable Neo-Hookean float32 block
 *                        rows are formed per row from the positions (no
 *                        per-tet Hessian store); 0: per-tet Hessian store +
 *                        gather.  Fixed Corotational and the float64 path
 *                        always use the store.
 *   fused_condense       1: the coupling kernel condenses its vertices itself
 *                        (the last CTA of every 32 list entries runs the
 *                        float64 3x3 solves of the group, one vertex per
 *                        lane); 0: a separate condensation launch.  The
 *                        one-warp coupling shape always launches it apart.
 * 1 sets, 0 clears, -1 keeps a switch; anything else is CC_ERR_INVALID_ARG.
 * Defaults: both 0 (measured fastest on the 32^3 cube); cc_autotune tries
 * every applicable combination.  The fused and separate
 * condensations give identical results; the two row builds agree within
 * float32 rounding. */
cc_status cc_set_sweep_variant(cc_mesh* mesh, int32_t rows_from_positions, int32_t fused_condense);

/* ======================================================================
 * Learned perturbation bases.  The paper builds every U_i by the patch
 * solve of Eq. 5 (Sec. 3.1) and has no learned component: everything below
 * is an addition.  A multilayer perceptron maps the rest geometry of a
 * vertex's 2-ring and its material to U_i on the 2-ring support (k = 2);
 * bases whose Eq. 5 residual is no better than U_i = 0 fall back to the
 * computed patch solve, vertex by vertex.
 * ====================================================================== */

/* Dense BF16 tensor-core GEMM used by the network, exposed for testing:
 * C = A . B^T with A [M x K], B [N x K] row-major BF16 device arrays
 * (leading dimensions lda, ldb in elements, multiples of 8, base addresses
 * 16-byte aligned) and C [M x N] float32 device (leading dimension ldc).
 * tcgen05 MMA with TMA-loaded, 128-byte-swizzled tiles and a float32
 * accumulator in tensor memory.  n_tile in {0 (automatic), 64, 128, 192,
 * 256}; k_splits >= 1 splits K over CTAs (partial products summed in a fixed
 * order afterwards), 0 = 1; flags: 0 or CC_GEMM_ONE_TILE_PER_CTA.
 * CC_ERR_TIMEOUT if a bounded device wait expired. */
cc_status cc_gemm_bf16_tn(const void* A, int64_t lda, const void* B, int64_t ldb, int32_t M, int32_t N,
                          int32_t K, float* C, int64_t ldc, int32_t n_tile, int32_t k_splits, int32_t flags,
                          void* stream);
/* cc_gemm_bf16_tn flags: the default kernel is persistent and warp-specialised
 * (one CTA per SM looping over tiles: a TMA producer warp, an MMA warp, 16
 * epilogue warps, two tensor-memory accumulators); this flag selects the
 * simpler one-tile-per-CTA kernel instead. */
#define CC_GEMM_ONE_TILE_PER_CTA 1

/* Network inputs: 64 stencil slots x 4 channels + 2 material channels. */
#define CC_LEARNED_D_IN 258
/* Network outputs: 64 slots x one 3x3 block. */
#define CC_LEARNED_D_OUT 576
/* Leading dimension of an input row (CC_LEARNED_D_IN rounded up to 8). */
#define CC_LEARNED_LDX 264

typedef struct cc_mlp cc_mlp;

/* The network's activation arithmetic, exposed for testing: for device
 * float32 x [n], out [n][3] = (erf(x), GELU(x), GELU'(x)) exactly as the GEMM
 * epilogues evaluate them (erf by Abramowitz and Stegun formula 7.1.26,
 * whose own error is at most 1.5e-7, evaluated with the approximate float32
 * reciprocal and 2^x: |error| <= 1e-6 in all; GELU in erf form). */
cc_status cc_mlp_activation(const float* x, int32_t n, float* out, void* stream);

typedef struct {
  int32_t d_in;       /* input width (CC_LEARNED_D_IN for bases) */
  int32_t hidden;     /* width of every hidden layer, multiple of 8 */
  int32_t layers;     /* number of hidden layers, >= 1 */
  int32_t d_out;      /* output width, multiple of 8 (CC_LEARNED_D_OUT) */
  int32_t max_batch;  /* largest training minibatch (rows) */
} cc_mlp_config;

typedef struct {
  float lr, beta1, beta2, eps;  /* Adam (Kingma and Ba 2015, bias-corrected) */
} cc_adam;

/* Network with float32 master parameters, BF16 copies of every weight
 * matrix in both orientations, Adam moments and a training workspace for
 * max_batch rows, all on the current device.  Layers: H = GELU(H W^T + b)
 * (erf form) for the hidden layers, linear output.  Parameters start at
 * zero; load them with cc_mlp_set_params.  stream: cudaStream_t or NULL. */
cc_status cc_mlp_create(const cc_mlp_config* cfg, void* stream, cc_mlp** out);
void cc_mlp_destroy(cc_mlp* net);

/* Number of parameters: sum over layers of d_out_l * d_in_l + d_out_l. */
int64_t cc_mlp_param_count(const cc_mlp* net);

/* Host float32 parameters, layer by layer: W_l row-major [d_out_l][d_in_l],
 * then b_l [d_out_l].  Setting them also resets Adam's moments and step. */
cc_status cc_mlp_set_params(cc_mlp* net, const float* params, int64_t count);
cc_status cc_mlp_get_params(const cc_mlp* net, float* params, int64_t count);

/* Parameters to and from a file (path: host string): the layer widths, then
 * the float32 parameters in the cc_mlp_set_params order.  Loading checks that
 * the widths match this network (CC_ERR_INVALID_ARG otherwise) and, like
 * cc_mlp_set_params, resets Adam's moments; the optimizer state is not saved. */
cc_status cc_mlp_save(const cc_mlp* net, const char* path);
cc_status cc_mlp_load(cc_mlp* net, const char* path);

/* Y [rows x d_out] float32 (device, leading dimension ldy) of the inputs
 * X [rows x d_in] BF16 (device, leading dimension ldx, multiple of 8).
 * Any number of rows; the inference workspace grows as needed. */
cc_status cc_mlp_forward(cc_mlp* net, const void* X, int64_t ldx, int64_t rows, float* Y, int64_t ldy);

/* Inference kernel of cc_mlp_forward and of the learned-basis build.  on = 1
 * (the default): one persistent kernel runs every layer of 128-row tiles with
 * the hidden activations kept in shared memory, SMs in pairs that share each
 * weight tile by TMA multicast (networks of at most 6 layers whose hidden
 * widths are multiples of 64 up to 256 and whose output width is a multiple
 * of 64; other shapes take the per-layer kernels).  on = 2: the same with
 * M = 256 MMAs over each SM pair (tcgen05 cta_group::2), each SM holding half
 * of every weight tile.  on = 0: one GEMM launch per layer, activations
 * through device memory.  All three give the same bits; any other value is
 * CC_ERR_INVALID_ARG. */
cc_status cc_mlp_set_fused(cc_mlp* net, int32_t on);

/* Mean squared error over rows x d_out against T (device float32 [rows x
 * ldt]) and its gradient with respect to every parameter, written to grad
 * (device float32 [param_count], parameter layout) unless NULL.  BF16 is
 * stored at the inputs, the weights, the hidden activations, the output
 * gradient and every pre-activation gradient; products accumulate in
 * float32.  rows <= max_batch. */
cc_status cc_mlp_loss_grad(cc_mlp* net, const void* X, int64_t ldx, const float* T, int64_t ldt,
                           int32_t rows, double* loss, float* grad);

/* One Adam step with a caller-supplied gradient (device float32). */
cc_status cc_mlp_adam_step(cc_mlp* net, const float* grad, const cc_adam* opt);

/* `steps` training steps: step s gathers the rows idx[s*batch .. s*batch +
 * batch) (device int32, each < n_samples) of X (device BF16 [n_samples x
 * ldx]) and T (device float32 [n_samples x ldt]), runs forward, backward
 * and one Adam step.  losses (host [steps], or NULL) receives every step's
 * loss.  batch <= max_batch.  The first step runs directly; the others
 * replay one CUDA graph of a step on the network's stream (recorded on a
 * private stream when that is the legacy default stream), the step number,
 * minibatch offset and Adam's beta^t kept on the device: the results equal
 * those of `steps` calls of one step each, bit for bit. */
cc_status cc_mlp_train(cc_mlp* net, const void* X, int64_t ldx, const float* T, int64_t ldt,
                       int64_t n_samples, const int32_t* idx, int32_t steps, int32_t batch,
                       const cc_adam* opt, double* losses);

/* Network inputs (and optionally targets) of every free vertex of a mesh
 * built on a Kuhn lattice, in ascending vertex id:
 *   l_i = mean over the 1-ring of max_a |X_j[a] - X_i[a]| (the cell size);
 *   for every j within 2 hops: q = (X_j - X_i) / l_i, o = floor(q + 1/2),
 *   slot s = position of o in the 64 offsets of the lattice's 2-ring (the 14
 *   1-ring offsets first, each group in lexicographic order); channels
 *   4s..4s+2 = 8 (q - o), 4s+3 = +1 free / -1 pinned; absent slots zero;
 *   channel 256 = (log10 E - 5.5) / 1.5, channel 257 = 10 (nu - 0.4).
 * X: device BF16 [rows_cap x ldx] (ldx >= CC_LEARNED_LDX, multiple of 8,
 * columns 258.. written as zero).  T: device float32 [rows_cap x ldt] or
 * NULL; when given, the mesh must hold computed k = 2 bases
 * (cc_build_subspace(mesh, 2)) and row r gets U_i[j] at columns
 * 9 s(j) .. 9 s(j) + 8 for j in S_i, zero elsewhere.  rows: host out,
 * number of free vertices.  CC_ERR_INVALID_ARG when a vertex within 2 hops
 * is off the stencil or two share a slot (not a Kuhn lattice). */
cc_status cc_learned_inputs(cc_mesh* mesh, void* X, int64_t ldx, float* T, int64_t ldt, int64_t rows_cap,
                            int64_t* rows);

typedef struct {
  int64_t n_free;      /* vertices with a basis */
  int64_t n_fallback;  /* of them, rebuilt by the patch solve */
  double rho_max;      /* largest Eq. 5 residual of a kept learned basis */
  double rho_mean;     /* mean residual of the learned bases, before fallback */
  double ms_supports;  /* 2-ring supports (host breadth-first search) */
  double ms_inputs;    /* network inputs */
  double ms_infer;     /* network forward */
  double ms_assemble;  /* predictions -> bases */
  double ms_residual;  /* rest Hessian + Eq. 5 residuals */
  double ms_fallback;  /* patch solves of the fallback set */
  double ms_total;     /* wall time of the whole call */
} cc_learned_stats;

/* Replaces the mesh's bases by learned ones on the k = 2 supports: network
 * inputs of every free vertex, one forward pass, bases assembled from the
 * predictions, then the residual of Eq. 5 at rest,
 *   rho_i = ||H_PP U_i + H_Pi||_F / ||H_Pi||_F,
 * for every free vertex; those with rho_i >= tau (tau = 1: no better than
 * U_i = 0, i.e. plain coordinate descent) get the computed basis from the
 * patch solve.  rho (device float64 [n_free], may be NULL) receives every
 * learned basis's residual.  Quasistatic meshes only (h = 0); needs
 * cc_color first.  The network must have d_in = CC_LEARNED_D_IN and
 * d_out = CC_LEARNED_D_OUT. */
cc_status cc_build_learned_subspace(cc_mesh* mesh, cc_mlp* net, double tau, double* rho,
                                    cc_learned_stats* stats);

/* Thread-local message of the last error on this thread ("" if none). */
const char* cc_last_error(void);

/* Library version string. */
const char* cc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CC_GB300_H */
