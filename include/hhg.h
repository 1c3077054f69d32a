/*
 * hhg.h - C ABI of the GB300 full-multigrid (FMG) solver on hierarchical hybrid grids.
 *
 * Method: B. Mann, U. Ruede, "kl-refinement: An adaptive mesh refinement scheme for
 * hierarchical hybrid grids" (arXiv 2508.06049).
 *   - Sec. 2: an unstructured coarse mesh T_0 of macro triangles (2D) or tetrahedra (3D),
 *     each refined uniformly L times (red refinement / Bey's rule).
 *   - Sec. 4.4, Eq. (4.15) and Eq. (5.1): P1 finite elements for -div(k grad u) = f with k
 *     constant on each macro element, Dirichlet data g.
 *   - Sec. 4.4, Alg. 4: FMG with nu V-cycles per level and Gauss-Seidel smoothing, storing the
 *     prolongated coarse solutions w_l; the ErrorEstimate procedure and the local indicators
 *     eta_T (Eq. 4.14, Sec. 4.4), in L2 or, per the Remark in Sec. 4, in the energy norm or a
 *     goal-oriented local seminorm.
 *   - Sec. 5.1 / Sec. 3 / Alg. 3: marking of a top fraction of macro elements and 2D or 3D
 *     red-green refinement of the macro mesh (kl-refinement, Alg. 2).
 *
 * Conventions (all entry points):
 *   - Every function returns an hhg_status; on failure hhg_last_error() gives a message
 *     (thread-local).  No function aborts the process.
 *   - Arrays are owned by the caller.  "host or device" arrays may live in host memory or in
 *     CUDA device memory of the mesh's device; the library copies through unified addressing.
 *   - Level-l vectors use the library's node layout: for each macro cell (in input order) its
 *     closure lattice packed plane by plane (see hhg_level_coords).  Nodes on shared macro
 *     vertices/edges/faces appear once per adjacent cell; inputs must give them equal values,
 *     outputs give them equal values.  N_l = n_cells * closure(2^l) entries, closure(n) =
 *     (n+1)(n+2)/2 in 2D and (n+1)(n+2)(n+3)/6 in 3D.
 *   - All device work of a mesh is ordered on the CUDA stream given at creation.  With NULL the
 *     mesh creates its own non-blocking stream and, at every entry point, orders it after the work
 *     the caller queued on the legacy default stream.  Functions that return host results (and
 *     hhg_fmg_solve, which checks its result for NaN/Inf) synchronise that stream before returning.
 *   - Floating-point is IEEE binary64 unless the solve parameters select the mixed mode, except
 *     the L2 forms of hhg_estimate (binary32 hi/lo pairs, see there).
 */
#ifndef HHG_H
#define HHG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hhg_mesh_s* hhg_mesh;
typedef struct hhg_rg2d_s* hhg_rg2d;
typedef struct hhg_rg3d_s* hhg_rg3d;

typedef enum {
  HHG_OK = 0,
  HHG_ERR_ARG = 1,            /* invalid argument (null pointer, size, range)              */
  HHG_ERR_MESH = 2,           /* invalid or degenerate coarse mesh                          */
  HHG_ERR_CUDA = 3,           /* a CUDA runtime call failed (message names it)              */
  HHG_ERR_OOM = 4,            /* device or host allocation failed                           */
  HHG_ERR_NOT_CONVERGED = 5,  /* an iteration did not reach its target                      */
  HHG_ERR_DIVERGED = 6,       /* NaN/Inf or growth detected in the solution                 */
  HHG_ERR_STATE = 7,          /* call order violated (e.g. estimate before a solve)         */
  HHG_ERR_TIMEOUT = 8         /* reserved: no kernel of this version waits on other blocks  */
} hhg_status;

/* Solve parameters (Alg. 4).  nu: V-cycles per FMG level; pre/post: Gauss-Seidel sweeps
 * before/after the coarse correction; n_extra: extra V-cycles on level L after FMG (they do
 * not update w_l, Sec. 5).
 * precision = 0: every step in binary64.
 * precision = 1 (mixed, no counterpart in the paper): iterative refinement whose level-L right-hand
 *   side b_L = M_L f_L, residual r = b - A u and iterate u (updated u += c) are carried as pairs of
 *   binary32 values with exact products and sums (about 2^-46 relative per operation, which bounds
 *   the attainable algebraic accuracy near 4^L * 2^-46 relative; u_L is returned in binary64,
 *   b_L kept in binary64); the correction c solves A c = r with
 *   FMG (first step) or ir_vcycles V-cycles (later steps) computed in binary32, with the level
 *   vectors of the correction stored as `storage` (0 = binary32, 1 = bfloat16, 2 = binary16) and
 *   accumulated in binary32.  ir_steps refinement steps follow the first one.
 *   binary16 (five exponent bits) stores each coarse level's correction times a power of two set
 *   on the device after the restriction: the largest 2^e with 2^e * B_l * max|r_l| <= 2^10, where
 *   B_l = 2^(l*dim) * |A_0^{-1}|_inf * (largest interface copy count) bounds |A_l^{-1}|_inf for the
 *   partial right-hand side r_l; stores beyond +-65504 saturate.  It needs at least one free macro
 *   vertex (|A_0^{-1}| comes from the direct coarse solve): otherwise HHG_ERR_ARG.
 * One Gauss-Seidel sweep updates, in this order: the macro vertices together with the even
 * edge-local nodes, the odd edge nodes, (3D) the face block - every macro face by Gauss-Seidel
 * over its colours (a + 2b) mod 3 with all nodes outside the face at their values from the start
 * of the block - and the macro-cell interiors by colours (alpha . p) mod m.  Nodes of one stage
 * are updated from the values at the start of the stage.
 * rhs: the coarse levels' right-hand sides (the paper does not fix them): 0 = b_l = M_l f_l with f
 * taken at the level-l nodes; 1 = b_L = M_L f_L and b_l = I^T b_{l+1} (I the interpolation), the
 * load vector of the level-L interpolant of f tested with the level-l hat functions. */
typedef struct {
  int nu, pre, post, n_extra;
  int precision;
  int storage;
  int ir_steps;
  int ir_vcycles;
  int rhs;
} hhg_solve_params;

typedef struct {
  int dim, L, n_cells, n_verts;
  long long n_nodes[16];      /* N_l per level (layout size, with interface copies)        */
  long long n_unknowns;       /* free (non-Dirichlet) distinct nodes on level L            */
  long long n_distinct;       /* distinct nodes on level L                                 */
  long long device_bytes;     /* device memory held by the mesh                            */
  int n_colours;              /* macro-interior colours of the smoother (max over cells)   */
} hhg_mesh_info;

/* Global estimator values; norms are L2 (hhg_estimate) or the norm chosen in hhg_estimate_norm. */
typedef struct {
  double eta_j;    /* theta~_l^j ||e~_l||, l = L - j          (Eq. 4.6)  */
  double theta;    /* ||e~_l|| / ||e~_{l-1}||                 (Eq. 4.5b) */
  double err_l;    /* ||e~_l||     = ||u_L - I w_l||_{L2}     (Eq. 4.5a) */
  double err_lm1;  /* ||e~_{l-1}|| = ||u_L - I w_{l-1}||_{L2}            */
  double err_Lm1;  /* ||e~_{L-1}|| = sqrt(sum_T eta_T^2)                 */
} hhg_estimate_out;

/* Create the HHG hierarchy for a coarse mesh (Sec. 2) and all device data for levels 0..L.
 * dim: 2 (triangles) or 3 (tetrahedra).  coords: host, n_verts*dim.  cells: host,
 * n_cells*(dim+1) vertex ids, 0-based; cell vertex order defines the lattice orientation.
 * vert_is_dirichlet: host, n_verts flags, or NULL = every vertex on the boundary.  A boundary
 * edge/face is Dirichlet when all its vertices are.  L: 1..9 (2D) or 1..8 (3D).
 * cuda_stream: a cudaStream_t or NULL.  Errors: HHG_ERR_ARG, HHG_ERR_MESH (degenerate cell,
 * non-manifold facet, too many coarse unknowns for the direct coarse solve), HHG_ERR_OOM. */
hhg_status hhg_mesh_create(int dim, int n_verts, const double* coords, int n_cells, const int* cells,
                           const unsigned char* vert_is_dirichlet, int L, void* cuda_stream,
                           hhg_mesh* out);
/* Release the hierarchy and every device buffer it owns (no counterpart in the paper: object
 * lifetime).  NULL is accepted. */
hhg_status hhg_mesh_destroy(hhg_mesh mesh);
/* Wait until all work queued on the mesh's stream has completed (no counterpart in the paper:
 * stream ordering).  Errors: HHG_ERR_ARG (NULL), HHG_ERR_CUDA (a failure reported by the stream). */
hhg_status hhg_mesh_synchronize(hhg_mesh mesh);
/* Sizes of the hierarchy (Sec. 2): dimension, L, macro cells and vertices, nodes per level in the
 * layout above, free distinct level-L nodes (the DoF count), device bytes, interior colours. */
hhg_status hhg_mesh_get_info(hhg_mesh mesh, hhg_mesh_info* info);

/* Coordinates of the level-l nodes of the uniformly refined macro cells (Sec. 2) in the layout
 * above (x = x_0 + J p / 2^l per cell).
 * xyz: host or device, N_l*dim doubles, node-major.  Device memory of the mesh's device is written
 * by one kernel on the mesh's stream (the call returns after it completes); any other pointer is
 * filled from host threads in batches of cells.  Both paths round every product and sum
 * separately and give the same bits.  Errors: HHG_ERR_ARG (NULL, level out of range),
 * HHG_ERR_CUDA. */
hhg_status hhg_level_coords(hhg_mesh mesh, int level, double* xyz);

/* Piecewise-constant coefficient k_T > 0 per macro cell (Eq. 5.1 with k); NULL = 1. */
hhg_status hhg_set_coefficient(hhg_mesh mesh, const double* k_per_cell);

/* Source f and Dirichlet data g of Eq. 5.1 at the level-L nodes (host or device, N_L each, one
 * value per interface copy, equal copies).  Copied on the mesh's stream. */
hhg_status hhg_set_data(hhg_mesh mesh, const double* f_L, const double* g_L);

/* FMG solve (Alg. 4): the right-hand sides of every level (params->rhs), FMG with the given
 * parameters, w_l kept for hhg_estimate.  u_L: host or device, N_L doubles (output).  Returns
 * HHG_ERR_DIVERGED if the result holds NaN/Inf. */
hhg_status hhg_fmg_solve(hhg_mesh mesh, const hhg_solve_params* params, double* u_L);

/* ErrorEstimate of Alg. 4 with offset j (1 <= j <= L-1) on the last solve.
 * eta_T: host, n_cells (may be NULL): ||u_L - w_{L-1}||_{L2(T)} over the micro elements of
 * macro T including its boundary (eta'_{1,T}, Eq. 4.14).  eta_jT: host, n_cells (may be NULL):
 * scaled local estimate theta~_{l,T}^j ||e~_l||_T (Eq. 4.10).  out: host, global values.
 * Arithmetic: each difference u_L - I w is formed in binary64; the per-cell quadratic forms are
 * evaluated in binary32 hi/lo pairs with exact products and sums (about 2^-44 relative per node),
 * the per-cell sums in binary64 in a fixed order (deterministic). */
hhg_status hhg_estimate(hhg_mesh mesh, int j, double* eta_T, double* eta_jT, hhg_estimate_out* out);

/* hhg_estimate in another norm (Remark in Sec. 4).  norm 0: L2 (= hhg_estimate).  norm 1: energy,
 * the stiffness matrix A_L (with k_T) in place of the mass matrix, ||v||_T^2 = int_T k |grad v|^2
 * over the micro elements of T, boundary nodes included.  norm 2: goal-oriented local seminorm
 * ||v||_T^2 = w_T ||v||_{L2(T)}^2 of the piecewise constant operator G(v|_T) = sqrt(w_T) v|_T,
 * with cell_weights w_T (host, n_cells, finite, >= 0; e.g. the indicator of a subregion made of
 * macro cells); global values are the sums of the weighted local squares.  cell_weights is read
 * for norm 2 only.  Local squares are clamped at 0 before the square roots (the energy form is
 * semidefinite).  Errors: as hhg_estimate, plus HHG_ERR_ARG for an unknown norm or bad weights. */
hhg_status hhg_estimate_norm(hhg_mesh mesh, int j, int norm, const double* cell_weights, double* eta_T,
                             double* eta_jT, hhg_estimate_out* out);

/* Read an internal level vector of the last solve (Alg. 4) into `out` (host or device, N_l doubles):
 * which = 0: u_l after its FMG V-cycles (l = L: the solution, l < L: overwritten by later
 * corrections, so only l = L is meaningful after the solve), 1: w_l (l = 0..L-1, stored on
 * level l+1, N_{l+1} doubles), 2: b_l summed over interface copies (N_l; after a mixed-precision
 * solve only l = L is kept in binary64, the coarser right-hand sides live in binary32). */
hhg_status hhg_get_vector(hhg_mesh mesh, int which, int level, double* out);

/* Operator application for testing (the operators of Eq. 4.15 and Sec. 4.4, and the smoother of
 * Alg. 4): out = Op_l in on level l with in/out of N_l doubles
 * (host or device), interface rows summed over adjacent cells.
 * op = 0: stiffness A_l (all rows, Dirichlet rows included as plain P1 rows),
 * op = 1: mass M_l, op = 2: interpolation from level l-1 (in has N_{l-1} entries),
 * op = 3: nsweeps Gauss-Seidel sweeps in place on out (the initial guess) with rhs M_l in;
 * op = 4: the same with the mixed mode's binary32 smoother (rhs and initial guess rounded to
 * binary32, the result widened to binary64).  Ops 3 and 4 overwrite the level's solve data: run
 * a solve again before hhg_estimate. */
hhg_status hhg_apply(hhg_mesh mesh, int level, int op, const double* in, double* out, int nsweeps);

/* Top-fraction marking (Sec. 5.1), host only: n = max(1, ceil(fraction*n - 1e-9)) elements
 * with the largest eta, plus every element within a relative 1e-8 of the n-th value (ties).
 * marked: host, n flags (output).  n_marked may be NULL. */
hhg_status hhg_mark(int n, const double* eta, double fraction, unsigned char* marked, int* n_marked);

/* 2D red-green refinement of a macro mesh (Sec. 3), host only.  The object keeps the red
 * history so that green closures are reverted before the next step.  Rules: red = split
 * through the edge midpoints; closure: red-refine triangles with >= 2 split edges or a split
 * edge whose half is split again; green = bisect a triangle with one split edge from the
 * opposite vertex.  New vertices are appended in creation order.  coords: host, n_verts*2;
 * cells: host, n_cells*3, 0-based.  Errors: HHG_ERR_ARG (sizes, vertex ids), HHG_ERR_MESH (a cell
 * with a repeated vertex or zero area), HHG_ERR_OOM. */
hhg_status hhg_rg2d_create(int n_verts, const double* coords, int n_cells, const int* cells, hhg_rg2d* out);
/* One red-green step (Sec. 3) on the current mesh with the given marks. */
hhg_status hhg_rg2d_refine(hhg_rg2d rg, const unsigned char* marked /* host, one flag per current cell */);
/* Current conforming mesh (Sec. 3); pass NULL arrays to query the sizes first. */
hhg_status hhg_rg2d_mesh(hhg_rg2d rg, int* n_verts, double* coords, int* n_cells, int* cells);
hhg_status hhg_rg2d_destroy(hhg_rg2d rg);
/* Marking (Sec. 5.1, as hhg_mark) + one red-green step (Sec. 3): marked (host, n_cells of the
 * current mesh, may be NULL). */
hhg_status hhg_mark_refine(hhg_rg2d rg, const double* eta_T, double fraction, unsigned char* marked);

/* 3D red-green refinement of a tetrahedral macro mesh (Alg. 3, Sec. 3), the k-step of the 3D
 * kl loop (host, sequential).  One step: revert the green families of the previous step (a
 * marked green child marks its parent); red-refine the marked tets (Bey's eight children, all
 * with the parent's orientation); repeat { split the third edge of every face with two split
 * edges; red-refine every tet with more than three split edges, a split edge whose half is split
 * again, or a fully split face with a split midline } until nothing changes; then close each tet
 * with one to three split edges by one of three green types (one edge: 2 children; two opposite
 * edges: 4; the three edges of one face: 4).  New vertices are edge midpoints numbered in
 * creation order; refined tets are replaced in place by their children.  coords: host,
 * n_verts*3; cells: host, n_cells*4, 0-based.  Errors: HHG_ERR_ARG (sizes, vertex ids),
 * HHG_ERR_MESH (a cell with a repeated vertex or zero volume), HHG_ERR_STATE (corrupt state),
 * HHG_ERR_OOM. */
hhg_status hhg_rg3d_create(int n_verts, const double* coords, int n_cells, const int* cells, hhg_rg3d* out);
/* One 3D red-green step (Alg. 3) on the current mesh with the given marks. */
hhg_status hhg_rg3d_refine(hhg_rg3d rg, const unsigned char* marked /* host, one flag per current cell */);
/* Current conforming mesh (Alg. 3); pass NULL arrays to query the sizes first. */
hhg_status hhg_rg3d_mesh(hhg_rg3d rg, int* n_verts, double* coords, int* n_cells, int* cells);
hhg_status hhg_rg3d_destroy(hhg_rg3d rg);
/* Marking (hhg_mark) + one 3D red-green step: marked (host, n_cells of the current mesh, may be NULL). */
hhg_status hhg_rg3d_mark_refine(hhg_rg3d rg, const double* eta_T, double fraction, unsigned char* marked);

/* Adjoint of the discrete solve (no counterpart in the paper): for J(u) = u^T M_S u with
 * M_S the mass matrix of the micro elements inside the macro cells flagged in in_S, on the
 * solution of the last hhg_fmg_solve, solve A lambda = 2 M_S u (lambda = 0 on Dirichlet nodes)
 * and return the results below.  params->precision = 0: FMG + params->n_extra V-cycles in binary64.
 * precision = 1: refinement on binary32 pairs (as in hhg_fmg_solve) from lambda = 0 whose
 * corrections come from binary32
 * V-cycles stored as params->storage (as in hhg_fmg_solve): a first step of ir_vcycles V-cycles
 * (the adjoint right-hand side is given on level L only, so there is no binary32 FMG step), then
 * ir_steps steps of ir_vcycles V-cycles and n_extra steps of one.  The results are
 *   J (host);
 *   grad_f (host or device, N_L, may be NULL): dJ/df_L for every entry of the level-L layout.  The
 *   right-hand side b_L = sum_T M_T f_T takes each cell's own copy of an interface node, so the
 *   entry of copy p in cell T is (M_T lambda)_p; summed over a node's copies it is (M_L lambda)_p,
 *   the derivative with respect to the node's value;
 *   grad_k[T] = -lambda^T A_T^(1) u (dJ/dk_T; host, n_cells, may be NULL). */
hhg_status hhg_adjoint_l2(hhg_mesh mesh, const hhg_solve_params* params, const unsigned char* in_S,
                          double* J, double* grad_f, double* grad_k);

/* Host self-check of the lattice index arithmetic (the structured level-l lattice of a macro cell,
 * Sec. 2) against brute force (no GPU needed): packed indices, neighbour offsets, valid directions
 * and, for even n, the interpolation end points from the side-n/2 lattice (Sec. 4.4's linear
 * interpolation) that the prolongation tables store.
 * Returns 0 if consistent, otherwise the number of mismatches. */
int hhg_lattice_selfcheck(int dim, int n);

/* Profiling support (no counterpart in the paper).  Enqueue `reps` launches of one kernel of the solve on the mesh's stream,
 * exactly as the solve launches it, without synchronising (bracket it with events on that stream).
 * kernel 0: the macro-interior smoothing of level L for the first cell group, the colour-0 stage:
 * precision 0 binary64, precision 1 binary32 as the mixed solve runs it (four cells per thread);
 * kernel 1 (3D, binary64): the level-L macro-face stage (units only; bytes = flops = 0);
 * kernels 2, 3 (binary64): the level-L prolongation-add and residual (every node computed);
 * kernel 4: the estimator's per-cell L2 form of one level-L vector, evaluated in binary32 hi/lo
 * pairs as hhg_estimate does (the vector is split into pairs once, before the launches);
 * units of kernels 2-4 = level-L nodes.
 * precision 1 allocates the mixed path's buffers on first use.  units: nodes updated per launch;
 * bytes / flops: algorithmic bytes and floating-point operations of one launch (the model is stated
 * in the library's design notes).  The launches modify the level-L iterate: run a solve again before
 * hhg_estimate. */
hhg_status hhg_profile_kernel(hhg_mesh mesh, int kernel, int precision, int reps, long long* units,
                              double* bytes, double* flops);

/* Measurement support (no counterpart in the paper).  Number of kernel nodes in the captured graph
 * of a solve (Alg. 4) with these parameters (after a first
 * hhg_fmg_solve with the same parameters), i.e. kernel launches per solve. */
hhg_status hhg_solve_launch_count(hhg_mesh mesh, const hhg_solve_params* params, long long* n_kernels);

/* Per-cell squared L2 norms of a difference on level L without allocating anything: out[T] =
 * (a - b)^T M_{L,T} (a - b) over the micro elements of macro cell T (b may be NULL).  The paper has no
 * counterpart: this is for callers that cannot allocate device memory when they need the local
 * indicators -- a caller recording its own CUDA stream capture (cudaMalloc is not allowed there) or a
 * process running under a fixed, pre-reserved device-memory budget.  With a = u_L and b = w_{L-1}
 * it gives eta_T^2 of hhg_estimate.
 * a, b: device, N_L doubles (mesh layout); out: device, n_cells doubles.  Work is queued on the
 * mesh's stream; the call does not synchronise (read `out` after synchronising that stream).
 * Scratch: a file-scope device array of 2^20 doubles (8 MiB) that every GPU which loads the library
 * holds until the process exits; cells x chunks must fit it (HHG_ERR_ARG beyond 65535 cells).  The
 * first call on a device looks up the array's device address (make that first call before any stream
 * capture).  All calls share the array and every call overwrites the part it uses before reading it
 * (nothing has to start at zero); calls that overlap on the GPU (e.g. on two streams) race on it.
 * No cudaMalloc, cudaFree or allocating library routine is called.  The mesh's device must be
 * current. */
hhg_status hhg_cell_mass_norms_noalloc(hhg_mesh mesh, const double* a, const double* b, double* out);

/* Debug builds (compiled with HHG_CHECK; no counterpart in the paper): first recorded out-of-range
 * index of a kernel
 * (code, block x, block y, thread, index, bound, 0, 1), then cleared; all zeros otherwise. */
hhg_status hhg_debug_check(long long* out8);

/* Message of the last failing call on this thread (no counterpart in the paper). */
const char* hhg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HHG_H */
