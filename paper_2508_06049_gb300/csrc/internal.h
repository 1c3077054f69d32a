// Internal host-side data of an HHG mesh object and the kernel launchers used by the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/hhg.h"
#include "lattice.h"

namespace hhg {

// Macro cells that share one interior stencil zero pattern (and hence one interior colouring).
struct Group {
  int pmask = 0;         // bit q set: lattice direction pair q has a nonzero interior coupling
  int alpha[3] = {0, 0, 0};
  int m = 2;             // number of interior colours
  std::vector<int> cells;
  int* d_cells = nullptr;
};

// Interface primitives of one kind (macro vertices, edges or faces) and their copies in the
// adjacent macro cells.  loc packs the local vertex indices of the primitive's vertices (sorted by
// global id) inside the cell: a0 | a1 << 2 | a2 << 4.
struct Prims {
  int count = 0;
  std::vector<int> ptr, cell, loc;
  std::vector<unsigned char> dir;  // Dirichlet flag per primitive
  int* d_ptr = nullptr;
  int* d_cell = nullptr;
  int* d_loc = nullptr;
  unsigned char* d_dir = nullptr;
  int max_copies = 0;
  // per primitive: 1 / (assembled diagonal of its interior nodes) at unit level scale (0 if Dirichlet)
  double* d_pinv = nullptr;
  float* d_pinvf = nullptr;
  // faces: in-plane couplings per face (8 slots, 6 used), unit level scale
  double* d_fw = nullptr;
  float* d_fwf = nullptr;
};

// threads per block of the node-parallel kernels (and of the per-cell reductions' block sums)
constexpr int kBlock = 256;
// dynamic shared memory a CTA of the face block may use (larger faces sweep in global scratch)
constexpr size_t kMaxTileSmem = 200 * 1024;

struct LevelData {
  int l = 0, n = 1;
  int64_t Nt = 0, N = 0;
  int32_t* d_ijk = nullptr;
  // levels >= 1, per closure node: the level-(l-1) packed indices of its two interpolation end points
  // (equal for a node that is also a coarse node) and its boundary type: x = ia | t << 27, y = ib
  int2* d_itab = nullptr;
  // interior colour lists: for group g and colour c, entries [icol_off[g][c], icol_off[g][c+1]) of
  // (packed local index, j | k << 16)
  std::vector<std::vector<int64_t>> icol_off;
  int2* d_icol = nullptr;
  // boundary-type closure nodes (type != 0), sorted by type: (packed local index, i | j << 10 | k << 20)
  int2* d_bnd = nullptr;
  int64_t nbnd = 0;
  double* d_invl = nullptr;  // per cell: 1 / (level-l interior diagonal)
  float* d_invlf = nullptr;
  // face colour lists (3D): colour c entries [fcol_off[c], fcol_off[c+1]) of a | b << 16
  int64_t fcol_off[4] = {0, 0, 0, 0};
  int32_t* d_fcol = nullptr;
  // binary64 vectors
  double* u = nullptr;    // solution / correction
  double* b = nullptr;    // rhs M_l f_l (partial at interfaces)
  double* rc = nullptr;   // restricted residual (rhs of the coarse correction), l < L
  double* w = nullptr;    // w_l on level l+1 (l < L)
  double* tmp = nullptr;  // residual scratch (l >= 1)
  // mixed-precision vectors (allocated on first mixed solve)
  void* c16 = nullptr;    // correction storage (binary32 / bfloat16 / binary16)
  float* x32 = nullptr;   // binary32 iterate of the FMG top level / level-L correction
  float* b32 = nullptr;   // binary32 copy of b_l
  float* r32 = nullptr;   // rhs of the correction equation (binary32)
  float* t32 = nullptr;   // residual scratch (binary32)
  float* cscale = nullptr;  // device scale of 16-bit correction storage
};

}  // namespace hhg

struct hhg_mesh_s {
  int dim = 2, L = 1, nc = 0, nv = 0, device = 0;
  int sm_count = 152;  // streaming multiprocessors of the device (queried at creation)
  cudaStream_t stream = nullptr;  // caller's stream
  cudaStream_t cap = nullptr;     // internal stream used for graph capture
  cudaStream_t own = nullptr;     // stream owned by the mesh when the caller passes NULL
  cudaEvent_t ev_legacy = nullptr;  // orders the mesh stream after the caller's legacy-stream work
  double* h_red = nullptr;        // pinned host staging of per-cell reductions (4 x n_cells)
  int* h_flag = nullptr;          // pinned host copy of the non-finite flag
  std::vector<double> coords;
  std::vector<int> cells;
  std::vector<double> k;
  std::vector<double> hS1, hM;    // unit-coefficient stiffness and mass stencils [cell][16][15]
  double* dS = nullptr;           // stiffness stencils with k_T (unit level scale)
  double* dM = nullptr;           // mass stencils (unit level scale)
  float* dS32 = nullptr;
  float* dM32 = nullptr;
  float2* dMp = nullptr;          // mass stencils as binary32 hi/lo pairs (estimator, mixed b_L)
  float2* dSp = nullptr;          // stiffness stencils with k_T as hi/lo pairs (mixed refinement)
  double* d_inv0 = nullptr;       // 1 / interior diagonal per cell (unit level scale, with k_T)
  float* d_inv0f = nullptr;
  double* d_tnorm = nullptr;      // per cell: interior stencil divided by its diagonal [cell][16]
  float* d_tnormf = nullptr;
  uint16_t* d_dirmask = nullptr;  // per cell: bit t set if nodes of boundary type t are Dirichlet
  uint16_t* d_nzs = nullptr;      // per cell and boundary type: stiffness slots with a nonzero entry
  std::vector<uint16_t> dirmask;
  std::vector<hhg::Group> groups;
  std::vector<int> group_of_cell;
  hhg::Prims verts, edges, faces;
  // direct coarse solve on level 0
  int n0f = 0;
  std::vector<int> cf_vert;       // compact free-vertex index -> vertex-primitive index
  double* d_Ainv = nullptr;
  double ainv_inf = 0;            // max row sum of |A_ff^{-1}| (range bound of binary16 corrections)
  unsigned* d_rmax = nullptr;     // per level: bit pattern of max |r| (binary16 correction storage)
  double* d_ainv_inf = nullptr;   // device copy of ainv_inf, written on the stream before each binary16 solve
  int* d_cf_vert = nullptr;
  std::vector<hhg::LevelData> lv;
  double* fL = nullptr;
  double* gL = nullptr;
  double* d_part = nullptr;       // per-block partial sums of the reductions
  int64_t part_len = 0;
  double* d_red = nullptr;        // per-cell reduction results (3 x n_cells)
  int* d_flag = nullptr;
  void* d_face_work = nullptr;  // face-block scratch for levels whose faces exceed shared memory
  float* d_scal32 = nullptr;      // scratch scalars for the mixed path
  std::map<std::string, cudaGraphExec_t> graphs;
  std::map<std::string, long long> graph_kernels;  // kernel nodes per captured graph
  bool have_data = false, solved = false, mixed_alloc = false;
  int last_storage = -1;
  long long bytes = 0;
  long long n_unknowns = 0, n_distinct = 0;
  int n_colours = 0;
};

namespace hhg {

// ---- setup (setup.cu) ----
hhg_status build_mesh(hhg_mesh_s* m, const double* coords, const int* cells,
                      const unsigned char* vflag);
hhg_status upload_coefficient(hhg_mesh_s* m);
void free_mesh(hhg_mesh_s* m);
void set_error(const char* fmt, ...);
hhg_status cuda_fail(cudaError_t e, const char* what);

// ---- kernel launchers (kernels.cu); all enqueue on stream s ----
enum class Prec { F64 = 0, F32 = 1, BF16 = 2, F16 = 3 };

void launch_build_rhs(hhg_mesh_s* m, int l, cudaStream_t s);
void launch_init_coarse(hhg_mesh_s* m, cudaStream_t s);
void launch_sweep(hhg_mesh_s* m, int l, const double* rhs, cudaStream_t s);
void launch_residual(hhg_mesh_s* m, int l, const double* rhs, cudaStream_t s);
// the same directly after a Gauss-Seidel sweep (last interior colour has zero residual)
void launch_residual_after(hhg_mesh_s* m, int l, const double* rhs, cudaStream_t s, bool after_sweep);
// coarse = P^T fine on level l-1; zero (may be null): a level-(l-1) vector set to 0 in the same launch
void launch_restrict(hhg_mesh_s* m, int l, const double* fine, double* coarse, cudaStream_t s,
                     double* zero = nullptr);
void launch_prolong_add(hhg_mesh_s* m, int l, cudaStream_t s);
void launch_fmg_prolong(hhg_mesh_s* m, int l, cudaStream_t s);
void launch_coarse_solve(hhg_mesh_s* m, const double* rhs, cudaStream_t s);
void launch_prolong(hhg_mesh_s* m, int l, const double* coarse, double* fine, cudaStream_t s,
                    const double* minuend = nullptr);
void launch_sub(hhg_mesh_s* m, const double* a, const double* b, double* x, int64_t n, cudaStream_t s);
// coordinates of the level-l nodes into device memory xyz (N_l * dim doubles); geom: device, per cell
// x_0 (3 doubles) and J row-major (9 doubles)
void launch_level_coords(hhg_mesh_s* m, int l, const double* geom, double* xyz, cudaStream_t s);
void launch_finite_check(hhg_mesh_s* m, const double* v, int64_t n, cudaStream_t s);
// per-cell reductions on level L: out[T] = (a-b)^T M_T (a-b), b may be null
void launch_mass_norm_sq(hhg_mesh_s* m, const double* a, const double* b, double* out, cudaStream_t s);
// the estimator's pair form: x as binary32 hi/lo pairs (k_sub_pair / k_prolong_diff_pair)
void launch_mass_norm_sq_pair(hhg_mesh_s* m, const float2* x, double* out, cudaStream_t s);
void launch_sub_pair(hhg_mesh_s* m, const double* a, const double* b, float2* x, int64_t n, cudaStream_t s);
void launch_prolong_diff_pair(hhg_mesh_s* m, const double* coarse, const double* minuend, float2* x, cudaStream_t s);
// out[T] = (a-b)^T A_T (a-b) with the cell's stiffness (k_T included), b may be null
void launch_energy_norm_sq(hhg_mesh_s* m, const double* a, const double* b, double* out, cudaStream_t s);
// out[T] = x^T A_T^(1) y (unit-coefficient partial stiffness of cell T), level L
void launch_stiff_bilinear(hhg_mesh_s* m, const double* x, const double* y, double* out, cudaStream_t s);
// operator application on all closure nodes (partial at interfaces), then interface sums
void launch_apply_op(hhg_mesh_s* m, int l, int op, const double* in, double* out, cudaStream_t s);
void launch_sum_interfaces(hhg_mesh_s* m, int l, double* v, cudaStream_t s);
// adjoint rhs: out = 2 M_T u for T in S (partial), 0 elsewhere
void launch_adjoint_rhs(hhg_mesh_s* m, const unsigned char* d_inS, const double* u, double* out, cudaStream_t s);

// profiling: launch the level-L interior smoothing stage (colour 0, group 0) `reps` times
void launch_profile_interior(hhg_mesh_s* m, int precision, int reps, cudaStream_t s, long long* units,
                             double* bytes, double* flops);

// ---- mixed precision (kernels_mixed.cu) ----
void launch_mixed_residual_L(hhg_mesh_s* m, cudaStream_t s);     // r32_L = b_L - A u_L (binary64 -> binary32)
void launch_mixed_update_L(hhg_mesh_s* m, int storage, cudaStream_t s);  // u_L += c_L
void launch_mixed_vcycle_ops(hhg_mesh_s* m, int storage);        // (declared for completeness)
void mixed_enqueue_vcycle(hhg_mesh_s* m, int l, int storage, const hhg_solve_params& p, cudaStream_t s);
void mixed_enqueue_fmg(hhg_mesh_s* m, int storage, const hhg_solve_params& p, cudaStream_t s);
void mixed_enqueue_adjoint(hhg_mesh_s* m, const hhg_solve_params& p, cudaStream_t s);
void mixed_set_scales(hhg_mesh_s* m, int storage, cudaStream_t s);

}  // namespace hhg
