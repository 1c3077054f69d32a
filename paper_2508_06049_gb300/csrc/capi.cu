// C ABI entry points: mesh life cycle, data, the FMG solve (Alg. 4) captured into CUDA graphs,
// the error estimator (Alg. 4 ErrorEstimate), test operators and the adjoint.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace hhg {
const char* last_error();
void launch_init_coarse_g(hhg_mesh_s* m, const double* g, cudaStream_t s);
void launch_fmg_prolong_g(hhg_mesh_s* m, int l, const double* g, double* w, cudaStream_t s);
void launch_restrict_rhs_chain(hhg_mesh_s* m, cudaStream_t s);
hhg_status read_check(long long* out);
hhg_status preload_kernels();
void launch_profile_face(hhg_mesh_s* m, int reps, cudaStream_t s, long long* units);
void launch_profile_level(hhg_mesh_s* m, int kernel, int reps, cudaStream_t s, long long* units, double* bytes,
                          double* flops);
hhg_status mixed_profile_interior(hhg_mesh_s* m, int reps, cudaStream_t s, long long* units, double* bytes,
                                  double* flops);
hhg_status mixed_prepare(hhg_mesh_s* m, int storage);
void mixed_enqueue_solve(hhg_mesh_s* m, const hhg_solve_params& p, cudaStream_t s);
void mixed_enqueue_adjoint(hhg_mesh_s* m, const hhg_solve_params& p, cudaStream_t s);
void mixed_sweeps(hhg_mesh_s* m, int l, int nsweeps, cudaStream_t s);
void launch_to_f32(const double* a, float* b, int64_t n, cudaStream_t s);
void launch_to_f64(const float* a, double* b, int64_t n, cudaStream_t s);
}  // namespace hhg

using namespace hhg;

#define CK(call)                                        \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

#define REQUIRE(cond, code, ...) \
  do {                           \
    if (!(cond)) {               \
      set_error(__VA_ARGS__);    \
      return code;               \
    }                            \
  } while (0)

namespace {

#ifdef HHG_CHECK
// checked build: device pointers are validated before launches, and each launch is synchronised
hhg_status check_dev_ptr(const void* p, const char* name) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess || a.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    set_error("pointer %s = %p is not device memory", name, p);
    return HHG_ERR_STATE;
  }
  return HHG_OK;
}
#define CHECK_PTR(p)                                       \
  do {                                                     \
    hhg_status st_ = check_dev_ptr((const void*)(p), #p);  \
    if (st_ != HHG_OK) return st_;                         \
  } while (0)
#define DBG_SYNC(what)                                     \
  do {                                                     \
    cudaError_t e_ = cudaStreamSynchronize(s);             \
    if (e_ == cudaSuccess) e_ = cudaGetLastError();        \
    if (e_ != cudaSuccess) return cuda_fail(e_, what);     \
  } while (0)
#else
#define CHECK_PTR(p) \
  do {               \
  } while (0)
#define DBG_SYNC(what) \
  do {                 \
  } while (0)
#endif

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

hhg_status check_params(const hhg_mesh_s* m, const hhg_solve_params* p) {
  REQUIRE(p, HHG_ERR_ARG, "params is NULL");
  REQUIRE(p->nu >= 1 && p->nu <= 64, HHG_ERR_ARG, "nu must be in [1,64]");
  REQUIRE(p->pre >= 0 && p->pre <= 64 && p->post >= 0 && p->post <= 64, HHG_ERR_ARG, "pre/post in [0,64]");
  REQUIRE(p->n_extra >= 0 && p->n_extra <= 10000, HHG_ERR_ARG, "n_extra in [0,10000]");
  REQUIRE(p->precision == 0 || p->precision == 1, HHG_ERR_ARG, "precision must be 0 or 1");
  REQUIRE(p->rhs == 0 || p->rhs == 1, HHG_ERR_ARG, "rhs must be 0 (injected f) or 1 (restricted from level L)");
  if (p->precision == 1) {
    REQUIRE(p->storage >= 0 && p->storage <= 2, HHG_ERR_ARG, "storage must be 0, 1 or 2");
    REQUIRE(p->ir_steps >= 0 && p->ir_steps <= 1000, HHG_ERR_ARG, "ir_steps in [0,1000]");
    REQUIRE(p->ir_vcycles >= 1 && p->ir_vcycles <= 64, HHG_ERR_ARG, "ir_vcycles in [1,64]");
  }
  (void)m;
  return HHG_OK;
}

// V(pre, post)-cycle on level l for A u_l = rhs (u_l in place); corrections on coarser levels
void enqueue_vcycle(hhg_mesh_s* m, int l, const double* rhs, const hhg_solve_params& p, cudaStream_t s) {
  if (l == 0) {
    launch_coarse_solve(m, rhs, s);
    return;
  }
  for (int q = 0; q < p.pre; ++q) launch_sweep(m, l, rhs, s);
  launch_residual_after(m, l, rhs, s, p.pre > 0);
  launch_restrict(m, l, m->lv[l].tmp, m->lv[l - 1].rc, s, m->lv[l - 1].u);  // and u_{l-1} = 0
  enqueue_vcycle(m, l - 1, m->lv[l - 1].rc, p, s);
  launch_prolong_add(m, l, s);
  for (int q = 0; q < p.post; ++q) launch_sweep(m, l, rhs, s);
}

// Alg. 4 FMG.  adjoint = true: right-hand side given on level L in lv[L].b (restricted to the
// coarser levels), zero Dirichlet data, w_l not stored.
void enqueue_fmg(hhg_mesh_s* m, const hhg_solve_params& p, bool adjoint, cudaStream_t s) {
  const int L = m->L;
  if (!adjoint && p.rhs == 0) {
    for (int l = 0; l <= L; ++l) launch_build_rhs(m, l, s);
  } else {
    // b_L = M_L f_L (the adjoint's right-hand side is already in b_L), b_{l-1} = I^T b_l
    if (!adjoint) launch_build_rhs(m, L, s);
    launch_restrict_rhs_chain(m, s);
  }
  const double* g = adjoint ? nullptr : m->gL;
  launch_init_coarse_g(m, g, s);
  for (int l = 0; l <= L; ++l) {
    for (int q = 0; q < p.nu; ++q) enqueue_vcycle(m, l, m->lv[l].b, p, s);
    if (l < L) launch_fmg_prolong_g(m, l, g, adjoint ? nullptr : m->lv[l].w, s);
  }
  for (int q = 0; q < p.n_extra; ++q) enqueue_vcycle(m, L, m->lv[L].b, p, s);
  cudaMemsetAsync(m->d_flag, 0, sizeof(int), s);
  launch_finite_check(m, m->lv[L].u, m->lv[L].N, s);
}

std::string graph_key(const char* what, const hhg_solve_params& p) {
  char buf[160];
  snprintf(buf, sizeof(buf), "%s:%d:%d:%d:%d:%d:%d:%d:%d:%d", what, p.nu, p.pre, p.post, p.n_extra, p.precision,
           p.storage, p.ir_steps, p.ir_vcycles, p.rhs);
  return buf;
}

template <typename F>
hhg_status run_graph(hhg_mesh_s* m, const std::string& key, F enqueue) {
  auto it = m->graphs.find(key);
  if (it == m->graphs.end()) {
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal));
    enqueue(m->cap);
    cudaError_t launch_err = cudaGetLastError();
    cudaError_t e = cudaStreamEndCapture(m->cap, &graph);
    if (launch_err != cudaSuccess) return cuda_fail(launch_err, "kernel launch during capture");
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    size_t nn = 0;
    long long nk = 0;
    if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn > 0) {
      std::vector<cudaGraphNode_t> nodes(nn);
      if (cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess)
        for (auto nd : nodes) {
          cudaGraphNodeType ty;
          if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++nk;
        }
    }
    m->graph_kernels[key] = nk;
    cudaGraphExec_t exec;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    it = m->graphs.emplace(key, exec).first;
  }
  CK(cudaGraphLaunch(it->second, m->stream));
  return HHG_OK;
}

// order the mesh's own stream after work the caller queued on the legacy default stream
hhg_status enter(hhg_mesh_s* m) {
  if (!m->own) return HHG_OK;
  CK(cudaEventRecord(m->ev_legacy, (cudaStream_t)0));
  CK(cudaStreamWaitEvent(m->own, m->ev_legacy, 0));
  return HHG_OK;
}

#define ENTER(m)                        \
  do {                                  \
    hhg_status st_e = enter(m);         \
    if (st_e != HHG_OK) return st_e;    \
  } while (0)

hhg_status copy_out(hhg_mesh_s* m, void* dst, const void* src, size_t bytes) {
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, m->stream));
  return HHG_OK;
}

}  // namespace

extern "C" {

const char* hhg_last_error(void) { return hhg::last_error(); }

hhg_status hhg_mesh_create(int dim, int n_verts, const double* coords, int n_cells, const int* cells,
                           const unsigned char* vert_is_dirichlet, int L, void* cuda_stream, hhg_mesh* out) {
  REQUIRE(out, HHG_ERR_ARG, "out is NULL");
  *out = nullptr;
  REQUIRE(dim == 2 || dim == 3, HHG_ERR_ARG, "dim must be 2 or 3");
  REQUIRE(coords && cells, HHG_ERR_ARG, "coords/cells is NULL");
  REQUIRE(n_verts >= dim + 1 && n_cells >= 1, HHG_ERR_ARG, "need at least one cell");
  REQUIRE(L >= 1 && L <= (dim == 2 ? 9 : 8), HHG_ERR_ARG, "L out of range (1..9 in 2D, 1..8 in 3D)");
  int64_t Nt = closure_size(dim, (int64_t)1 << L);
  REQUIRE((double)Nt * n_cells < 2.0e9, HHG_ERR_ARG, "level-L layout exceeds 2e9 nodes");
  int dev = 0;
  CK(cudaGetDevice(&dev));
  hhg_mesh_s* m = new (std::nothrow) hhg_mesh_s();
  REQUIRE(m, HHG_ERR_OOM, "host allocation failed");
  m->dim = dim;
  m->L = L;
  m->nc = n_cells;
  m->nv = n_verts;
  m->device = dev;
  {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0) m->sm_count = sms;
  }
  m->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess && m->stream == nullptr) {
    // NULL: the mesh works on its own stream, ordered after the caller's legacy-stream work at
    // every entry point (and every entry point returning results synchronises it)
    e = cudaStreamCreateWithFlags(&m->own, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->ev_legacy, cudaEventDisableTiming);
    m->stream = m->own;
  }
  if (e != cudaSuccess) {
    if (m->cap) cudaStreamDestroy(m->cap);
    if (m->own) cudaStreamDestroy(m->own);
    delete m;
    return cuda_fail(e, "cudaStreamCreate");
  }
  hhg_status st = preload_kernels();
  if (st == HHG_OK) st = build_mesh(m, coords, cells, vert_is_dirichlet);
  if (st != HHG_OK) {
    free_mesh(m);
    delete m;
    return st;
  }
  *out = m;
  return HHG_OK;
}

hhg_status hhg_mesh_destroy(hhg_mesh m) {
  if (!m) return HHG_OK;
  DeviceGuard g(m->device);
  cudaStreamSynchronize(m->stream);
  free_mesh(m);
  delete m;
  return HHG_OK;
}

hhg_status hhg_mesh_synchronize(hhg_mesh m) {
  REQUIRE(m, HHG_ERR_ARG, "mesh is NULL");
  DeviceGuard g(m->device);
  CK(cudaStreamSynchronize(m->stream));
  return HHG_OK;
}

hhg_status hhg_mesh_get_info(hhg_mesh m, hhg_mesh_info* info) {
  REQUIRE(m && info, HHG_ERR_ARG, "NULL argument");
  memset(info, 0, sizeof(*info));
  info->dim = m->dim;
  info->L = m->L;
  info->n_cells = m->nc;
  info->n_verts = m->nv;
  for (int l = 0; l <= m->L && l < 16; ++l) info->n_nodes[l] = m->lv[l].N;
  info->n_unknowns = m->n_unknowns;
  info->n_distinct = m->n_distinct;
  info->device_bytes = m->bytes;
  info->n_colours = m->n_colours;
  return HHG_OK;
}

hhg_status hhg_level_coords(hhg_mesh m, int level, double* xyz) {
  REQUIRE(m && xyz, HHG_ERR_ARG, "NULL argument");
  REQUIRE(level >= 0 && level <= m->L, HHG_ERR_ARG, "level out of range");
  DeviceGuard g(m->device);
  const int d = m->dim;
  const LevelData& Lv = m->lv[level];
  cudaPointerAttributes pa;
  const bool on_device = cudaPointerGetAttributes(&pa, xyz) == cudaSuccess &&
                         (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged) &&
                         pa.device == m->device;
  cudaGetLastError();  // an unregistered host pointer may leave an error behind
  if (on_device) {
    // device memory of the mesh's device: one kernel from the per-cell x_0 and J
    std::vector<double> geom((size_t)m->nc * 12, 0.0);
    for (int c = 0; c < m->nc; ++c) {
      const int* cv = &m->cells[(size_t)c * (d + 1)];
      const double* x0 = &m->coords[(size_t)cv[0] * d];
      double* G = &geom[(size_t)c * 12];
      for (int r = 0; r < d; ++r) {
        G[r] = x0[r];
        for (int q = 0; q < d; ++q) G[3 + 3 * r + q] = m->coords[(size_t)cv[q + 1] * d + r] - x0[r];
      }
    }
    double* dg = nullptr;
    CK(cudaMalloc(&dg, geom.size() * sizeof(double)));
    cudaError_t e = cudaMemcpy(dg, geom.data(), geom.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      launch_level_coords(m, level, dg, xyz, m->stream);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    cudaFree(dg);
    CK(e);
    return HHG_OK;
  }
  const int planes = d == 3 ? Lv.n + 1 : 1;
  const int64_t per = Lv.Nt * d;  // doubles per cell
  // cells are filled in batches of at most 2^26 doubles (512 MB) by host threads, one (cell,
  // plane) pair per work item, and each batch is copied to xyz (host or device) in one piece
  const int batch = (int)std::max<int64_t>(1, std::min<int64_t>(m->nc, ((int64_t)1 << 26) / per));
  std::vector<double> buf((size_t)batch * per);
  const int nthr = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  for (int c0 = 0; c0 < m->nc; c0 += batch) {
    const int c1 = std::min(m->nc, c0 + batch);
    std::atomic<int64_t> next(0);
    const int64_t items = (int64_t)(c1 - c0) * planes;
    auto work = [&]() {
      for (int64_t it; (it = next.fetch_add(1)) < items;) {
        const int c = c0 + (int)(it / planes), k = (int)(it % planes);
        const int* cv = &m->cells[(size_t)c * (d + 1)];
        const double* x0 = &m->coords[(size_t)cv[0] * d];
        double J[3][3] = {{0}};
        for (int r = 0; r < d; ++r)
          for (int q = 0; q < d; ++q) J[r][q] = m->coords[(size_t)cv[q + 1] * d + r] - x0[r];
        double* out = buf.data() + (size_t)(c - c0) * per;
        for (int j = 0; j <= Lv.n - k; ++j)
          for (int i = 0; i <= Lv.n - k - j; ++i) {
            const int64_t q = packed_index(d, Lv.n, i, j, k);
            const int p[3] = {i, j, k};
            for (int r = 0; r < d; ++r) {
              double v = 0;
              for (int a = 0; a < d; ++a) v += J[r][a] * p[a];
              out[(size_t)q * d + r] = x0[r] + v / Lv.n;
            }
          }
      }
    };
    const int nt = (int)std::min<int64_t>(nthr, items);
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(work);
    work();
    for (auto& th : pool) th.join();
    CK(cudaMemcpy(xyz + (size_t)c0 * per, buf.data(), (size_t)(c1 - c0) * per * sizeof(double),
                  cudaMemcpyDefault));
  }
  return HHG_OK;
}

hhg_status hhg_set_coefficient(hhg_mesh m, const double* k) {
  REQUIRE(m, HHG_ERR_ARG, "mesh is NULL");
  DeviceGuard g(m->device);
  for (int c = 0; c < m->nc; ++c) {
    double v = k ? k[c] : 1.0;
    REQUIRE(std::isfinite(v) && v > 0, HHG_ERR_ARG, "coefficient of cell %d is not positive", c);
  }
  CK(cudaStreamSynchronize(m->stream));
  for (int c = 0; c < m->nc; ++c) m->k[c] = k ? k[c] : 1.0;
  return upload_coefficient(m);
}

hhg_status hhg_set_data(hhg_mesh m, const double* f, const double* gv) {
  REQUIRE(m && f && gv, HHG_ERR_ARG, "NULL argument");
  DeviceGuard g(m->device);
  ENTER(m);
  size_t bytes = sizeof(double) * (size_t)m->lv[m->L].N;
  CK(cudaMemcpyAsync(m->fL, f, bytes, cudaMemcpyDefault, m->stream));
  CK(cudaMemcpyAsync(m->gL, gv, bytes, cudaMemcpyDefault, m->stream));
  m->have_data = true;
  return HHG_OK;
}

hhg_status hhg_fmg_solve(hhg_mesh m, const hhg_solve_params* params, double* u_L) {
  REQUIRE(m, HHG_ERR_ARG, "mesh is NULL");
  hhg_status st = check_params(m, params);
  if (st != HHG_OK) return st;
  REQUIRE(m->have_data, HHG_ERR_STATE, "hhg_set_data must be called before hhg_fmg_solve");
  DeviceGuard g(m->device);
  ENTER(m);
  const hhg_solve_params p = *params;
  if (p.precision == 0) {
    st = run_graph(m, graph_key("fmg", p), [&](cudaStream_t s) { enqueue_fmg(m, p, false, s); });
  } else {
    st = mixed_prepare(m, p.storage);
    if (st != HHG_OK) return st;
    st = run_graph(m, graph_key("mixed", p), [&](cudaStream_t s) { mixed_enqueue_solve(m, p, s); });
  }
  if (st != HHG_OK) return st;
  if (u_L) {
    st = copy_out(m, u_L, m->lv[m->L].u, sizeof(double) * (size_t)m->lv[m->L].N);
    if (st != HHG_OK) return st;
  }
  CK(cudaMemcpyAsync(m->h_flag, m->d_flag, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  m->solved = true;
  REQUIRE(*m->h_flag == 0, HHG_ERR_DIVERGED, "solution contains NaN or Inf");
  return HHG_OK;
}

// ErrorEstimate (Alg. 4) in the norm `norm`: 0 L2 (mass form), 1 energy (stiffness form),
// 2 L2 with per-cell weights applied to the local squares on the host (goal-oriented seminorm)
static hhg_status estimate_impl(hhg_mesh m, int j, int norm, const double* wts, double* eta_T, double* eta_jT,
                                hhg_estimate_out* out) {
  REQUIRE(m, HHG_ERR_ARG, "mesh is NULL");
  REQUIRE(m->solved, HHG_ERR_STATE, "hhg_estimate needs a previous hhg_fmg_solve");
  const int L = m->L;
  REQUIRE(j >= 1 && j <= L - 1, HHG_ERR_ARG, "need 1 <= j <= L-1 (L = %d)", L);
  DeviceGuard g(m->device);
  ENTER(m);
  cudaStream_t s = m->stream;
  const int l = L - j;
  const int nc = m->nc;
  double* red = m->d_red;
  const double* uL = m->lv[L].u;
  CHECK_PTR(red);
  CHECK_PTR(uL);
  CHECK_PTR(m->lv[L - 1].w);
  CHECK_PTR(m->lv[l].w);
  CHECK_PTR(m->lv[l - 1].w);
  CHECK_PTR(m->d_part);
  CHECK_PTR(m->dM);
  CHECK_PTR(m->dMp);
  CHECK_PTR(m->dS);
  CHECK_PTR(m->lv[L].d_ijk);
  CHECK_PTR(m->lv[L].tmp);
  CHECK_PTR(m->lv[L].rc);
  const int jj = j;
  const bool energy = norm == 1;
  auto form = [&](const double* x, double* dst, cudaStream_t cs) {
    if (energy) launch_energy_norm_sq(m, x, nullptr, dst, cs);
    else launch_mass_norm_sq(m, x, nullptr, dst, cs);
  };
  // The differences are formed once into level-L scratch (rc is never a coarse-grid rhs on level L,
  // tmp is free after the solve), so the per-cell form reads one vector.  The L2 forms take the
  // difference in binary64 and evaluate the quadratic form in binary32 hi/lo pairs (the mass
  // stencil's couplings would otherwise keep GB300's binary64 pipe busy); the energy form stays in
  // binary64.
  double* xa = m->lv[L].rc;
  double* xb = m->lv[L].tmp;
  auto diff = [&](const double* v, double* x, cudaStream_t cs) {  // x = u_L - v on level L
    if (energy) launch_sub(m, uL, v, x, m->lv[L].N, cs);
    else launch_sub_pair(m, uL, v, (float2*)x, m->lv[L].N, cs);
  };
  auto form_x = [&](const double* x, double* dst, cudaStream_t cs) {
    if (energy) form(x, dst, cs);
    else launch_mass_norm_sq_pair(m, (const float2*)x, dst, cs);
  };
  // x_L = u_L - I^(L-l0) v for v on level l0 < L (the intermediate levels in binary64)
  auto diff_prolonged = [&](const double* v, int l0, double* x, cudaStream_t cs) {
    for (int q = l0 + 1; q < L; ++q) {
      launch_prolong(m, q, v, m->lv[q].tmp, cs, nullptr);
      v = m->lv[q].tmp;
    }
    if (energy) launch_prolong(m, L, v, x, cs, uL);
    else launch_prolong_diff_pair(m, v, uL, (float2*)x, cs);
  };
  hhg_status st = run_graph(m, "est:" + std::to_string(jj) + (energy ? ":energy" : ""), [&](cudaStream_t cs) {
    // e~_{L-1} = u_L - w_{L-1} (eta_T)
    diff(m->lv[L - 1].w, xa, cs);
    form_x(xa, red, cs);
    // e~_l = u_L - I w_l (w_l lives on level l+1); for j = 1 it is e~_{L-1} again
    if (l == L - 1) {
      cudaMemcpyAsync(red + nc, red, sizeof(double) * nc, cudaMemcpyDeviceToDevice, cs);
    } else {
      diff_prolonged(m->lv[l].w, l + 1, xb, cs);
      form_x(xb, red + nc, cs);
    }
    // e~_{l-1} = u_L - I w_{l-1} (w_{l-1} lives on level l)
    diff_prolonged(m->lv[l - 1].w, l, xb, cs);
    form_x(xb, red + 2 * nc, cs);
  });
  if (st != HHG_OK) return st;
  DBG_SYNC("estimator graph");
  CK(cudaMemcpyAsync(m->h_red, red, sizeof(double) * 3 * (size_t)nc, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  // local squares (weighted for the goal-oriented seminorm); clamped at 0: the energy form is only
  // semidefinite (constants lie in the kernel of A_T), so a near-constant difference can round
  // to a tiny negative square
  std::vector<double> qT(nc), ql(nc), qlm1(nc);
  for (int c = 0; c < nc; ++c) {
    const double w = norm == 2 ? wts[c] : 1.0;
    qT[c] = std::max(0.0, w * m->h_red[c]);
    ql[c] = std::max(0.0, w * m->h_red[nc + c]);
    qlm1[c] = std::max(0.0, w * m->h_red[2 * nc + c]);
  }
  double sT = 0, sl = 0, slm1 = 0;
  for (int c = 0; c < nc; ++c) {
    sT += qT[c];
    sl += ql[c];
    slm1 += qlm1[c];
  }
  double err_l = std::sqrt(sl), err_lm1 = std::sqrt(slm1);
  double theta = err_lm1 > 0 ? err_l / err_lm1 : 0.0;
  if (eta_T)
    for (int c = 0; c < nc; ++c) eta_T[c] = std::sqrt(qT[c]);
  if (eta_jT)
    for (int c = 0; c < nc; ++c) {
      double th = qlm1[c] > 0 ? std::sqrt(ql[c] / qlm1[c]) : 0.0;
      eta_jT[c] = std::pow(th, j) * std::sqrt(ql[c]);
    }
  if (out) {
    out->eta_j = std::pow(theta, j) * err_l;
    out->theta = theta;
    out->err_l = err_l;
    out->err_lm1 = err_lm1;
    out->err_Lm1 = std::sqrt(sT);
  }
  return HHG_OK;
}

hhg_status hhg_estimate(hhg_mesh m, int j, double* eta_T, double* eta_jT, hhg_estimate_out* out) {
  return estimate_impl(m, j, 0, nullptr, eta_T, eta_jT, out);
}

hhg_status hhg_estimate_norm(hhg_mesh m, int j, int norm, const double* cell_weights, double* eta_T,
                             double* eta_jT, hhg_estimate_out* out) {
  REQUIRE(norm >= 0 && norm <= 2, HHG_ERR_ARG, "norm must be 0 (L2), 1 (energy) or 2 (weighted L2)");
  if (norm == 2) {
    REQUIRE(m, HHG_ERR_ARG, "mesh is NULL");
    REQUIRE(cell_weights, HHG_ERR_ARG, "norm 2 needs cell_weights");
    for (int c = 0; c < m->nc; ++c)
      REQUIRE(std::isfinite(cell_weights[c]) && cell_weights[c] >= 0, HHG_ERR_ARG,
              "cell_weights[%d] must be finite and >= 0", c);
  }
  return estimate_impl(m, j, norm, cell_weights, eta_T, eta_jT, out);
}

hhg_status hhg_get_vector(hhg_mesh m, int which, int level, double* out) {
  REQUIRE(m && out, HHG_ERR_ARG, "NULL argument");
  REQUIRE(level >= 0 && level <= m->L, HHG_ERR_ARG, "level out of range");
  DeviceGuard g(m->device);
  ENTER(m);
  const LevelData& Lv = m->lv[level];
  if (which == 0) {
    CK(cudaMemcpyAsync(out, Lv.u, sizeof(double) * Lv.N, cudaMemcpyDefault, m->stream));
  } else if (which == 1) {
    REQUIRE(level < m->L, HHG_ERR_ARG, "w_l exists for l < L");
    CK(cudaMemcpyAsync(out, Lv.w, sizeof(double) * m->lv[level + 1].N, cudaMemcpyDefault, m->stream));
  } else if (which == 2) {
    double* scratch = nullptr;
    CK(cudaMalloc(&scratch, sizeof(double) * Lv.N));
    cudaMemcpyAsync(scratch, Lv.b, sizeof(double) * Lv.N, cudaMemcpyDeviceToDevice, m->stream);
    launch_sum_interfaces(m, level, scratch, m->stream);
    cudaMemcpyAsync(out, scratch, sizeof(double) * Lv.N, cudaMemcpyDefault, m->stream);
    cudaStreamSynchronize(m->stream);
    cudaFree(scratch);
  } else {
    set_error("which must be 0, 1 or 2");
    return HHG_ERR_ARG;
  }
  CK(cudaStreamSynchronize(m->stream));
  CK(cudaGetLastError());
  return HHG_OK;
}

hhg_status hhg_apply(hhg_mesh m, int level, int op, const double* in, double* out, int nsweeps) {
  REQUIRE(m && in && out, HHG_ERR_ARG, "NULL argument");
  REQUIRE(level >= 0 && level <= m->L, HHG_ERR_ARG, "level out of range");
  REQUIRE(op >= 0 && op <= 4, HHG_ERR_ARG, "op must be 0..4");
  REQUIRE(op != 2 || level >= 1, HHG_ERR_ARG, "interpolation needs level >= 1");
  REQUIRE(op < 3 || (level >= 1 && nsweeps >= 0), HHG_ERR_ARG, "sweeps need level >= 1");
  DeviceGuard g(m->device);
  ENTER(m);
  if (op == 4) {  // binary32 buffers of the mixed path before any work is queued
    hhg_status st = mixed_prepare(m, m->mixed_alloc ? m->last_storage : 0);
    if (st != HHG_OK) return st;
  }
  cudaStream_t s = m->stream;
  LevelData& Lv = m->lv[level];
  size_t nin = (size_t)(op == 2 ? m->lv[level - 1].N : Lv.N);
  double *din = nullptr, *dout = nullptr;
  CK(cudaMalloc(&din, sizeof(double) * nin));
  cudaError_t e = cudaMalloc(&dout, sizeof(double) * Lv.N);
  if (e != cudaSuccess) {
    cudaFree(din);
    return cuda_fail(e, "cudaMalloc");
  }
  cudaMemcpyAsync(din, in, sizeof(double) * nin, cudaMemcpyDefault, s);
  if (op == 0 || op == 1) {
    launch_apply_op(m, level, op, din, dout, s);
    launch_sum_interfaces(m, level, dout, s);
  } else if (op == 2) {
    launch_prolong(m, level, din, dout, s);
  } else if (op == 3) {
    // rhs = M in (partial), initial guess from out, sweeps in place on the level's u
    launch_apply_op(m, level, 1, din, Lv.b, s);
    cudaMemcpyAsync(Lv.u, out, sizeof(double) * Lv.N, cudaMemcpyDefault, s);
    for (int q = 0; q < nsweeps; ++q) launch_sweep(m, level, Lv.b, s);
    cudaMemcpyAsync(dout, Lv.u, sizeof(double) * Lv.N, cudaMemcpyDeviceToDevice, s);
    m->solved = false;
  } else {
    // the same in binary32 with the mixed path's smoother: rhs and initial guess rounded to binary32
    launch_apply_op(m, level, 1, din, Lv.b, s);
    launch_to_f32(Lv.b, Lv.b32, Lv.N, s);
    cudaMemcpyAsync(dout, out, sizeof(double) * Lv.N, cudaMemcpyDefault, s);
    launch_to_f32(dout, Lv.x32, Lv.N, s);
    mixed_sweeps(m, level, nsweeps, s);
    launch_to_f64(Lv.x32, dout, Lv.N, s);
    m->solved = false;
  }
  cudaMemcpyAsync(out, dout, sizeof(double) * Lv.N, cudaMemcpyDefault, s);
  e = cudaStreamSynchronize(s);
  cudaFree(din);
  cudaFree(dout);
  if (e != cudaSuccess) return cuda_fail(e, "hhg_apply");
  CK(cudaGetLastError());
  return HHG_OK;
}

hhg_status hhg_adjoint_l2(hhg_mesh m, const hhg_solve_params* params, const unsigned char* in_S, double* J,
                          double* grad_f, double* grad_k) {
  REQUIRE(m && in_S, HHG_ERR_ARG, "NULL argument");
  hhg_status st = check_params(m, params);
  if (st != HHG_OK) return st;
  REQUIRE(m->solved, HHG_ERR_STATE, "hhg_adjoint_l2 needs a previous hhg_fmg_solve");
  DeviceGuard g(m->device);
  ENTER(m);
  if (params->precision == 1) {  // mixed-precision buffers before any work is queued
    st = mixed_prepare(m, params->storage);
    if (st != HHG_OK) return st;
  }
  cudaStream_t s = m->stream;
  const int L = m->L, nc = m->nc;
  LevelData& LL = m->lv[L];
  size_t bytes = sizeof(double) * (size_t)LL.N;
  double* usave = nullptr;
  unsigned char* dS = nullptr;
  CK(cudaMalloc(&usave, bytes));
  cudaError_t e = cudaMalloc(&dS, nc);
  if (e != cudaSuccess) {
    cudaFree(usave);
    return cuda_fail(e, "cudaMalloc");
  }
  cudaMemcpyAsync(usave, LL.u, bytes, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(dS, in_S, nc, cudaMemcpyDefault, s);
  // J = sum_{T in S} u^T M_T u
  launch_mass_norm_sq(m, usave, nullptr, m->d_red, s);
  std::vector<double> h(nc);
  cudaMemcpyAsync(h.data(), m->d_red, sizeof(double) * nc, cudaMemcpyDeviceToHost, s);
  // adjoint rhs 2 M_S u on level L, then FMG with zero Dirichlet data (binary64), or binary64
  // refinement with binary32 V-cycles (mixed)
  launch_adjoint_rhs(m, dS, usave, LL.b, s);
  hhg_solve_params p = *params;
  if (p.precision == 0) {
    st = run_graph(m, graph_key("adjoint", p), [&](cudaStream_t cs) { enqueue_fmg(m, p, true, cs); });
  } else {
    st = run_graph(m, graph_key("mixed-adjoint", p), [&](cudaStream_t cs) { mixed_enqueue_adjoint(m, p, cs); });
  }
  if (st == HHG_OK) {
    if (grad_f) {
      // dJ/df_L per entry of the level-L layout: b_L = sum_T M_T f_T reads each cell's own copy, so
      // the derivative by copy p of cell T is (M_T lambda)_p, the partial (unsummed) mass product
      launch_apply_op(m, L, 1, LL.u, LL.tmp, s);
      cudaMemcpyAsync(grad_f, LL.tmp, bytes, cudaMemcpyDefault, s);
    }
    std::vector<double> hk(nc);
    if (grad_k) {
      launch_stiff_bilinear(m, LL.u, usave, m->d_red + nc, s);
      cudaMemcpyAsync(hk.data(), m->d_red + nc, sizeof(double) * nc, cudaMemcpyDeviceToHost, s);
    }
    int flag = 0;
    cudaMemcpyAsync(&flag, m->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    // restore the forward solution
    cudaMemcpyAsync(LL.u, usave, bytes, cudaMemcpyDeviceToDevice, s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "hhg_adjoint_l2");
    else if (flag) {
      set_error("adjoint solution contains NaN or Inf");
      st = HHG_ERR_DIVERGED;
    }
    if (st == HHG_OK) {
      double Jv = 0;
      for (int c = 0; c < nc; ++c)
        if (in_S[c]) Jv += h[c];
      if (J) *J = Jv;
      if (grad_k)
        for (int c = 0; c < nc; ++c) grad_k[c] = -hk[c] / m->k[c];
    }
  }
  cudaStreamSynchronize(s);
  cudaFree(usave);
  cudaFree(dS);
  // b_L was overwritten by the adjoint rhs: the next forward solve rebuilds it
  return st;
}

hhg_status hhg_profile_kernel(hhg_mesh m, int kernel, int precision, int reps, long long* units, double* bytes,
                              double* flops) {
  REQUIRE(m && units && bytes && flops, HHG_ERR_ARG, "NULL argument");
  REQUIRE(kernel >= 0 && kernel <= 4, HHG_ERR_ARG, "kernel must be 0 .. 4");
  REQUIRE(precision == 0 || precision == 1, HHG_ERR_ARG, "precision must be 0 or 1");
  REQUIRE(reps >= 0 && reps <= 100000, HHG_ERR_ARG, "reps in [0, 100000]");
  DeviceGuard g(m->device);
  ENTER(m);
  if (kernel >= 2) {
    REQUIRE(precision == 0, HHG_ERR_ARG, "the level probes 2 .. 4 are binary64");
    REQUIRE(m->L >= 1, HHG_ERR_ARG, "the level probes need L >= 1");
    launch_profile_level(m, kernel, reps, m->stream, units, bytes, flops);
  } else if (kernel == 1) {
    REQUIRE(precision == 0, HHG_ERR_ARG, "the face-stage probe is binary64");
    launch_profile_face(m, reps, m->stream, units);
    *bytes = 0;
    *flops = 0;
  } else if (precision == 1) {
    hhg_status st = mixed_prepare(m, m->mixed_alloc ? m->last_storage : 1);
    if (st != HHG_OK) return st;
    st = mixed_profile_interior(m, reps, m->stream, units, bytes, flops);
    if (st != HHG_OK) return st;
  } else {
    launch_profile_interior(m, 0, reps, m->stream, units, bytes, flops);
  }
  m->solved = false;
  CK(cudaGetLastError());
  return HHG_OK;
}

hhg_status hhg_solve_launch_count(hhg_mesh m, const hhg_solve_params* params, long long* n) {
  REQUIRE(m && params && n, HHG_ERR_ARG, "NULL argument");
  auto it = m->graph_kernels.find(graph_key(params->precision == 0 ? "fmg" : "mixed", *params));
  *n = it == m->graph_kernels.end() ? 0 : it->second;
  return HHG_OK;
}

hhg_status hhg_debug_check(long long* out8) {
  REQUIRE(out8, HHG_ERR_ARG, "NULL argument");
  return read_check(out8);
}

int hhg_lattice_selfcheck(int dim, int n) {
  if ((dim != 2 && dim != 3) || n < 1 || n > 1000) return -1;
  int bad = 0;
  int64_t Nt = closure_size(dim, n);
  std::vector<int> seen(Nt, 0);
  for (int k = 0; k <= (dim == 3 ? n : 0); ++k)
    for (int j = 0; j <= n - k; ++j)
      for (int i = 0; i <= n - k - j; ++i) {
        int64_t g = packed_index(dim, n, i, j, k);
        if (g < 0 || g >= Nt) {
          ++bad;
          continue;
        }
        seen[g]++;
        int64_t off[15];
        neighbour_offsets(dim, n, j, k, off);
        int t = boundary_type(dim, n, i, j, k);
        uint32_t vm = valid_dirs(dim, t);
        if (vm != valid_dirs_tab(dim, t)) ++bad;
        for (int d = 0; d < (dim == 2 ? 7 : 15); ++d) {
          int di, dj, dk;
          dir_vec(dim, d, di, dj, dk);
          int a = i + di, b = j + dj, c = k + dk;
          bool inside = a >= 0 && b >= 0 && c >= 0 && a + b + c <= n;
          if (inside != (bool)(vm >> d & 1)) ++bad;
          if (inside && packed_index(dim, n, a, b, c) != g + off[d]) ++bad;
          PlaneBasis pb = plane_basis(dim, n, k);
          if (inside && d > 0 && dir_offset(dim, d, pb.m, j, pb.Tm, pb.Tm1) != off[d]) ++bad;
        }
      }
  for (int64_t g = 0; g < Nt; ++g)
    if (seen[g] != 1) ++bad;
  // interpolation end points from the side-n/2 lattice (n even): both are coarse closure nodes, the
  // fine node is their midpoint (fine coordinates = sum of the coarse ones), they are equal exactly
  // for all-even fine coordinates, and otherwise they differ by one lattice direction
  if (n % 2 == 0) {
    const int nc = n / 2;
    const int64_t Ntc = closure_size(dim, nc);
    std::vector<int> cc(3 * Ntc, -1);
    for (int k = 0; k <= (dim == 3 ? nc : 0); ++k)
      for (int j = 0; j <= nc - k; ++j)
        for (int i = 0; i <= nc - k - j; ++i) {
          const int64_t g = packed_index(dim, nc, i, j, k);
          cc[3 * g] = i, cc[3 * g + 1] = j, cc[3 * g + 2] = k;
        }
    for (int k = 0; k <= (dim == 3 ? n : 0); ++k)
      for (int j = 0; j <= n - k; ++j)
        for (int i = 0; i <= n - k - j; ++i) {
          int64_t ia, ib;
          interp_ends(dim, n, i, j, k, ia, ib);
          if (ia < 0 || ia >= Ntc || ib < 0 || ib >= Ntc) {
            ++bad;
            continue;
          }
          const int* a = &cc[3 * ia];
          const int* b = &cc[3 * ib];
          if (a[0] + b[0] != i || a[1] + b[1] != j || a[2] + b[2] != k) ++bad;
          const bool even = !((i | j | k) & 1);
          if (even != (ia == ib)) ++bad;
          if (!even) {
            bool adjacent = false;
            for (int d = 1; d < (dim == 2 ? 7 : 15); ++d) {
              int di, dj, dk;
              dir_vec(dim, d, di, dj, dk);
              if (b[0] - a[0] == di && b[1] - a[1] == dj && b[2] - a[2] == dk) adjacent = true;
            }
            if (!adjacent) ++bad;
          }
        }
  }
  return bad;
}

}  // extern "C"
