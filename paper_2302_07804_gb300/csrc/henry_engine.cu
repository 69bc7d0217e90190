// Host engine and C ABI of libhenry (declared in include/henry.h).
//
// One "group" = the device workspace of a batch of B samples at one MLMC
// level: the fine state, old state and residual (FP64), the Jacobian
// hierarchy (6 block planes per multigrid level), the Krylov and multigrid
// vectors (T = double or float), per-sample coefficients, scalars, flags and
// partial sums.  It is carved out of a single cudaMalloc and kept in the
// handle for reuse by later calls of the same level.
//
// The solve of one group runs the r_l implicit-Euler steps (Sec. 2.3 of
// arXiv 2302.07804); each step runs Newton iterations, each Newton iteration
// assembles the residual and the Jacobian on the fine grid and the coarse
// operators, and solves the Newton system with BiCGStab right-preconditioned
// by one V-cycle.  Per-sample convergence decisions are taken on the device;
// the host only reads "how many samples are still iterating" once per Newton
// and once per BiCGStab iteration to decide when to stop launching.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "henry.h"
#include "henry_kernels.cuh"
#include "henry_misc.cuh"
#include "henry_cta.cuh"
#include "henry_kl.cuh"
#include "henry_adjoint.cuh"
#include "henry_vc.cuh"
#include "henry_vc_solve.cuh"

using namespace hk;

namespace {

thread_local std::string g_err;

int set_err(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return set_err(HENRY_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)
#define CKL()                                                                                        \
  do {                                                                                               \
    cudaError_t e_ = cudaGetLastError();                                                             \
    if (e_ != cudaSuccess) return set_err(HENRY_ECUDA, "kernel launch failed (line %d): %s", __LINE__, \
                                          cudaGetErrorString(e_));                                   \
  } while (0)

inline unsigned nblk(int64_t n, int tpb = TPB) { return (unsigned)((n + tpb - 1) / tpb); }

struct Level {
  int nx, ny, N;
  double h;
  double2 *x, *xo;  // state (fine: Newton iterate; coarse: restricted) and old state
  double2* cc;      // per-cell (phi, K / mu) of the field models (else null)
  double4_32a* fc;      // per-cell east/north face harmonic means of the field models (else null)
  void* J;          // 6 planes of B4
  void *mgx, *mgb;  // multigrid vectors (coarse levels)
  int64_t plane;
};

// Carves sub-arrays out of one allocation (256-byte aligned).
struct Carver {
  char* base;
  size_t off;
  template <typename P>
  P* take(size_t bytes) {
    off = (off + 255) & ~size_t(255);
    P* p = base ? reinterpret_cast<P*>(base + off) : nullptr;
    off += bytes;
    return p;
  }
};

template <typename T>
struct Group {
  typedef typename VT<T>::v2 V2;
  typedef typename VT<T>::b4 B4;
  int level = -1, Bcap = 0, K = 0, nct = 0;
  bool light = false;  // workspace of the fused small-grid solver only
  char* mem = nullptr;
  size_t bytes = 0;
  std::vector<Level> lv;
  double2* F = nullptr;
  double2* xoo = nullptr;  // fine state x^{n-2} (the quadratic predictor)
  V2 *r, *rh, *p, *v, *s, *t, *ph, *sh, *dx;
  Coef* coef;
  double* part;
  int *newton_active, *lin_active, *newton_it, *status, *iters, *counter;
  double* theta;  // per-sample Newton step factor
  double* fin;    // finalised per-sample reduction values [B][NPART] (large grids)
  unsigned long long* totals;  // [0] Newton iterations, [1] BiCGStab iterations
  LinScal* sc;
  T* Ainv;
  void* Jp = nullptr;  // fine-level fallback preconditioner operator (field models only)
  // Instantiated CUDA graphs of one BiCGStab iteration's body, by batch size,
  // preconditioner operator and every setting that changes the body's
  // launches (nu1, nu2, mg_tail_cells, mg_threads); they hold this
  // workspace's pointers and are dropped with it.
  std::map<std::tuple<int, const void*, int, int, int, int>, cudaGraphExec_t> gexec;
  bool graphs = true;  // false: never capture (the allocation-free entry point)
  void drop_graphs() {
    for (auto& kv : gexec) cudaGraphExecDestroy(kv.second);
    gexec.clear();
  }

  // Lay out (or size, with base == nullptr) the workspace for B samples.
  // `light`: only what the fused small-grid solver uses (fine old state,
  // coefficients, status, counters); every other pointer is left null.
  size_t carve(char* base, int B, int nx0, int ny0, double h0, bool light_ws = false, bool fields = false) {
    Carver c{base, 0};
    std::vector<Level> L;
    int nx = nx0, ny = ny0;
    double h = h0;
    for (;;) {
      Level l;
      l.nx = nx; l.ny = ny; l.N = nx * ny; l.h = h;
      l.plane = (int64_t)B * l.N;
      l.x = l.xo = nullptr;
      l.J = l.mgx = l.mgb = nullptr;
      l.cc = nullptr;
      l.fc = nullptr;
      if (fields) {
        l.cc = c.take<double2>(sizeof(double2) * l.plane);
        l.fc = c.take<double4_32a>(sizeof(double4_32a) * l.plane);
      }
      if (light_ws) {
        if (L.empty()) l.xo = c.take<double2>(sizeof(double2) * l.plane);
      } else {
        l.x = c.take<double2>(sizeof(double2) * l.plane);
        l.xo = c.take<double2>(sizeof(double2) * l.plane);
        l.J = c.take<B4>(sizeof(B4) * 6 * l.plane);
        if (!L.empty()) {
          l.mgx = c.take<V2>(sizeof(V2) * l.plane);
          l.mgb = c.take<V2>(sizeof(V2) * l.plane);
        }
      }
      L.push_back(l);
      if (nx <= 2 || ny <= 1) break;
      nx /= 2; ny /= 2; h *= 2.0;
    }
    const int64_t n0 = (int64_t)B * nx0 * ny0;
    V2** vecs[9] = {&r, &rh, &p, &v, &s, &t, &ph, &sh, &dx};
    xoo = c.take<double2>(sizeof(double2) * n0);  // also the fused solver's
    if (light_ws) {
      F = nullptr;
      for (auto vp : vecs) *vp = nullptr;
    } else {
      F = c.take<double2>(sizeof(double2) * n0);
      for (auto vp : vecs) *vp = c.take<V2>(sizeof(V2) * n0);
    }
    coef = c.take<Coef>(sizeof(Coef) * B);
    nct = nx0 * ny0 / TPB;
    part = light_ws ? nullptr : c.take<double>(sizeof(double) * NPART * (size_t)B * nct);
    newton_active = c.take<int>(sizeof(int) * B);
    lin_active = c.take<int>(sizeof(int) * B);
    newton_it = c.take<int>(sizeof(int) * B);
    status = c.take<int>(sizeof(int) * B);
    iters = c.take<int>(sizeof(int) * B);
    theta = c.take<double>(sizeof(double) * B);
    fin = light_ws ? nullptr : c.take<double>(sizeof(double) * NPART * (size_t)B);
    counter = c.take<int>(sizeof(int) * 4);
    totals = c.take<unsigned long long>(sizeof(unsigned long long) * 4);
    sc = light_ws ? nullptr : c.take<LinScal>(sizeof(LinScal) * B);
    Ainv = light_ws ? nullptr : c.take<T>(sizeof(T) * 16 * B);
    Jp = (fields && !light_ws) ? (void*)c.take<B4>(sizeof(B4) * 6 * (size_t)n0) : nullptr;
    if (base) {
      lv = L;
      K = (int)L.size() - 1;
      light = light_ws;
    }
    return c.off + 256;
  }
};

// The workspace of a batch of B samples of the vertex-centred scheme at one
// MLMC level (henry_vc_solve.cuh gives the layout): per multigrid level the
// states (fine: Newton iterate and old state; coarse: injected), 10 block
// planes and the multigrid vectors x, b and a residual; on the fine level
// (stride padded to whole 256-entry blocks) F and the Krylov vectors; the
// per-sample scalars and partial sums.  One cudaMalloc, zeroed once (the
// padding entries of every fine vector stay zero).
template <typename T>
struct VcGroup {
  typedef typename VT<T>::v2 V2;
  typedef typename VT<T>::b4 B4;
  struct Lv {
    int nx, ny, NV, stride;
    int64_t plane;
    double h;
    double2 *x, *xo;
    void* J;
    void *mgx, *mgb, *mgr;
  };
  int level = -1, Bcap = 0, K = 0, nct = 0;
  char* mem = nullptr;
  size_t bytes = 0;
  std::vector<Lv> lv;
  double2* F = nullptr;
  double2* xoo = nullptr;  // fine state x^{n-2} (the quadratic predictor)
  V2 *r, *rh, *p, *v, *s, *t, *ph, *sh, *dx;
  Coef* coef;
  double *part, *theta, *fin;
  int *newton_active, *lin_active, *newton_it, *status, *iters, *counter;
  unsigned long long* totals;
  LinScal* sc;
  T* Ainv;
  std::map<std::tuple<int, int, int>, cudaGraphExec_t> gexec;  // (B, nu1, nu2)
  void drop_graphs() {
    for (auto& kv : gexec) cudaGraphExecDestroy(kv.second);
    gexec.clear();
  }
  size_t carve(char* base, int B, int nx0, int ny0, double h0) {
    Carver c{base, 0};
    std::vector<Lv> L;
    int nx = nx0, ny = ny0;
    double h = h0;
    for (;;) {
      Lv l;
      l.nx = nx; l.ny = ny; l.NV = (nx + 1) * (ny + 1); l.h = h;
      l.stride = L.empty() ? ((l.NV + TPB - 1) / TPB) * TPB : l.NV;
      l.plane = (int64_t)B * l.stride;
      l.x = c.take<double2>(sizeof(double2) * l.plane);
      l.xo = c.take<double2>(sizeof(double2) * l.plane);
      l.J = c.take<B4>(sizeof(B4) * 10 * l.plane);
      l.mgx = L.empty() ? nullptr : c.take<V2>(sizeof(V2) * l.plane);
      l.mgb = L.empty() ? nullptr : c.take<V2>(sizeof(V2) * l.plane);
      l.mgr = c.take<V2>(sizeof(V2) * l.plane);
      L.push_back(l);
      if (nx <= 2 || ny <= 1) break;
      nx /= 2; ny /= 2; h *= 2.0;
    }
    const int64_t n0 = L[0].plane;
    F = c.take<double2>(sizeof(double2) * n0);
    xoo = c.take<double2>(sizeof(double2) * n0);
    V2** vecs[9] = {&r, &rh, &p, &v, &s, &t, &ph, &sh, &dx};
    for (auto vp : vecs) *vp = c.take<V2>(sizeof(V2) * n0);
    coef = c.take<Coef>(sizeof(Coef) * B);
    nct = L[0].stride / TPB;
    part = c.take<double>(sizeof(double) * NPART * (size_t)B * nct);
    newton_active = c.take<int>(sizeof(int) * B);
    lin_active = c.take<int>(sizeof(int) * B);
    newton_it = c.take<int>(sizeof(int) * B);
    status = c.take<int>(sizeof(int) * B);
    iters = c.take<int>(sizeof(int) * B);
    theta = c.take<double>(sizeof(double) * B);
    fin = c.take<double>(sizeof(double) * NPART * (size_t)B);
    counter = c.take<int>(sizeof(int) * 4);
    totals = c.take<unsigned long long>(sizeof(unsigned long long) * 4);
    sc = c.take<LinScal>(sizeof(LinScal) * B);
    Ainv = c.take<T>(sizeof(T) * VC_COARSE_N * VC_COARSE_N * (size_t)B);
    if (base) {
      lv = L;
      K = (int)L.size() - 1;
    }
    return c.off + 256;
  }
};

}  // namespace

// Per-kernel-class timing with CUDA events (off by default): each profiled
// launch is bracketed by two events on its stream; pending pairs are read at
// the next host synchronisation.  Algorithmic bytes per launch are counted
// from the compulsory traffic of the kernel for the samples still iterating.
struct Prof {
  bool on = false;
  struct Pend {
    cudaEvent_t a, b;
    int cls;
    double bytes, flops;
  };
  std::vector<cudaEvent_t> pool;
  std::vector<Pend> pend;
  double ms[HENRY_K_COUNT] = {};
  int64_t launches[HENRY_K_COUNT] = {};
  double bytes[HENRY_K_COUNT] = {};
  double flops[HENRY_K_COUNT] = {};
};

// Device copies of the KL basis evaluated at one grid's cell centres.
struct KLTables {
  int nx = 0, ny = 0;
  int* ti = nullptr;
  int* tj = nullptr;
  double* sl = nullptr;
  double* psx = nullptr;  // [m][nx]
  double* psy = nullptr;  // [m][ny]
};

struct henry_handle {
  henry_config cfg;
  hkl::Basis2D* kl = nullptr;
  std::map<int, KLTables> kl_tables;  // by MLMC level
  std::map<int, Group<double>> g64;
  std::map<int, Group<float>> g32;
  std::map<int, VcGroup<double>> vg64;  // vertex-centred scheme
  std::map<int, VcGroup<float>> vg32;
  int* host_counter = nullptr;  // pinned
  unsigned long long* host_totals = nullptr;
  Prof prof;
  int nact = 0;  // samples iterating in the current Newton / Krylov iteration (for byte counts)
  // henry_batch_solve_mixed: one child handle, stream and host thread per
  // level, plus a buffer for batches whose samples are not sorted by level
  std::map<int, henry_handle*> kids;
  std::map<int, cudaStream_t> kid_streams;
  cudaEvent_t ev_fork = nullptr;
  char* perm_mem = nullptr;
  int perm_cap = 0;
  // henry_adjoint: checkpoints, one segment of states, right-hand side and sensitivity sums
  char* adj_mem = nullptr;
  size_t adj_bytes = 0;
  cudaStream_t cap_stream = nullptr;  // CUDA-graph capture
  std::map<int, henry_tuning> tuned;  // henry_autotune's choices per level
};

namespace {

cudaEvent_t prof_event(Prof& P) {
  if (!P.pool.empty()) {
    cudaEvent_t e = P.pool.back();
    P.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

template <typename F>
void launch(henry_handle* H, cudaStream_t st, int cls, double bytes, double flops, F&& f) {
  if (!H->prof.on) {
    f();
    return;
  }
  Prof& P = H->prof;
  cudaEvent_t a = prof_event(P), b = prof_event(P);
  cudaEventRecord(a, st);
  f();
  cudaEventRecord(b, st);
  P.pend.push_back({a, b, cls, bytes, flops});
}
template <typename F>
void launch(henry_handle* H, cudaStream_t st, int cls, double bytes, F&& f) {
  launch(H, st, cls, bytes, 0.0, f);
}

// Algorithmic flop counts (FMA = 2) of the block-stencil kernels on an
// nx x ny grid: directed neighbour links 4 N - 2 nx - 2 ny, each a 2x2
// block-vector product (8 flops).
inline double links(int nx, int ny) { return 4.0 * nx * ny - 2.0 * nx - 2.0 * ny; }
inline double sweep_flops(int nx, int ny, int mode) {  // one half-sweep
  const double hc = 0.5 * nx * ny;
  return (mode == 0 ? 0.0 : 0.5 * links(nx, ny) * 8.0) + hc * 6.0;
}
inline double spmv_flops(int nx, int ny, int ndot) {
  return links(nx, ny) * 8.0 + nx * ny * (6.0 + 4.0 * ndot);
}
inline double restrict_flops(int nx, int ny) {  // residual of the colour-0 cells + sum
  return 0.5 * links(nx, ny) * 8.0 + 0.5 * nx * ny * (8.0 + 2.0);
}

void prof_drain(henry_handle* H) {
  Prof& P = H->prof;
  for (auto& p : P.pend) {
    float ms = 0.f;
    cudaEventSynchronize(p.b);
    cudaEventElapsedTime(&ms, p.a, p.b);
    P.ms[p.cls] += ms;
    P.launches[p.cls] += 1;
    P.bytes[p.cls] += p.bytes;
    P.flops[p.cls] += p.flops;
    P.pool.push_back(p.a);
    P.pool.push_back(p.b);
  }
  P.pend.clear();
}

// The assembly kernel for an nx x ny grid: the face-once tile form, in
// assembly_tile_w x (TPB / assembly_tile_w) tiles where that tile divides the
// grid, else whole rows per tile where they fit (nx <= TPB), else 128 x 2
// tiles; the per-cell form with tile_assembly = 0.  Same arguments; the tile
// forms evaluate each face with the same source arithmetic wherever it is
// evaluated, the per-cell form evaluates it from both sides (same values up
// to rounding).
// JAC = false: the fine residual alone (same values as with JAC = true).
template <typename T, bool FINE, bool FIELDS = false, bool DROP = false, bool JAC = true>
auto assemble_kernel(const henry_config& c, int nx, int ny) -> decltype(&k_assemble<T, FINE, FIELDS, DROP, JAC>) {
  if (!c.tile_assembly) return &k_assemble<T, FINE, FIELDS, DROP, JAC>;
  const int tw = c.assembly_tile_w;
  if (tw > 0 && nx % tw == 0 && ny % (TPB / tw) == 0) {  // N % TPB == 0 follows
    switch (tw) {
      case 32: return &k_assemble_tile2d<T, FINE, FIELDS, DROP, JAC, 32>;
      case 64: return &k_assemble_tile2d<T, FINE, FIELDS, DROP, JAC, 64>;
      case 128: return &k_assemble_tile2d<T, FINE, FIELDS, DROP, JAC, 128>;
      case 256: return &k_assemble_tile2d<T, FINE, FIELDS, DROP, JAC, 256>;
      default: break;
    }
  }
  if (nx <= TPB) return &k_assemble_tile<T, FINE, FIELDS, DROP, JAC>;
  if (nx % TILE_W_DEFAULT == 0 && ny % (TPB / TILE_W_DEFAULT) == 0)
    return &k_assemble_tile2d<T, FINE, FIELDS, DROP, JAC, TILE_W_DEFAULT>;
  return &k_assemble<T, FINE, FIELDS, DROP, JAC>;
}

// Runs f(std::integral_constant<int, NT>{}) for the multigrid kernels' CTA
// size nt: 64, 128, 256 or 512 threads (anything else: TPB).
template <typename F>
void with_mg_threads(int nt, F&& f) {
  switch (nt) {
    case 64: f(std::integral_constant<int, 64>()); break;
    case 128: f(std::integral_constant<int, 128>()); break;
    case 512: f(std::integral_constant<int, 512>()); break;
    default: f(std::integral_constant<int, TPB>()); break;
  }
}
bool has_fields(const henry_config& c) { return c.coef_model != HENRY_MODEL_UNIFORM3; }
int qoi_count(const henry_config& c) {
  switch (c.qoi_set) {
    case HENRY_QOI_STANDARD: return 2;
    case HENRY_QOI_PAPER: return 15;
    case HENRY_QOI_PAPER_FIELD: return 15 + c.nx0 * c.ny0;
    default: return 15 + c.steps0;  // HENRY_QOI_PAPER_SERIES
  }
}
// QoI set 3: Q_FW after the implicit step `step` (0-based) when it ends a
// level-0 time step (every 2^level fine steps), into column 15 + k.
void record_series(henry_handle* H, int level, int step, int B, int N, double h, const double2* x, double* qoi,
                   const int* status, cudaStream_t st) {
  const henry_config& c = H->cfg;
  if (c.qoi_set != HENRY_QOI_PAPER_SERIES || (step + 1) % (1 << level) != 0) return;
  const int k = (step + 1) / (1 << level) - 1;
  k_qfw<<<B, TPB, 0, st>>>(B, N, h, x, qoi + 15 + k, qoi_count(c), status);
}
QoiSpec qoi_spec(const henry_config& c) { return QoiSpec{c.qoi_set, qoi_count(c), c.nx0, c.ny0, c.Lx, c.Ly}; }
int n_inputs(const henry_config& c) { return c.coef_model == HENRY_MODEL_KL ? 2 * c.kl_terms + 1 : 3; }

Phys phys_of(const henry_config& c) {

  Phys p;
  p.rho0 = c.rho0; p.rho1 = c.rho1; p.drho = c.rho1 - c.rho0; p.g = c.g; p.Ly = c.Ly; p.Dm = c.Dm;
  return p;
}

struct LevelGeom {
  int nx, ny, steps;
  double h, tau;
};
LevelGeom geom(const henry_config& c, int level) {
  LevelGeom g;
  g.nx = c.nx0 << level;
  g.ny = c.ny0 << level;
  g.steps = c.steps0 << level;
  g.h = c.Ly / g.ny;
  g.tau = c.T / g.steps;
  return g;
}

template <typename T>
size_t bytes_per_sample(const henry_config& c, int level, bool light = false) {
  Group<T> g;
  LevelGeom lg = geom(c, level);
  return g.carve(nullptr, 1, lg.nx, lg.ny, lg.h, light, has_fields(c));
}

// The fused one-CTA-per-sample solver is used when enabled, the sample's
// hierarchy fits the shared-memory layout and the device grants that much
// shared memory per CTA.
// (atomic: the levels of henry_batch_solve_mixed reach here from concurrent
// host threads; every thread stores the same attribute value)
std::atomic<int> g_smem_optin[64] = {};
template <typename T>
bool fused_eligible(const henry_config& c, int level, CtaLayout* L) {
  // 1 (default): only with FP32 linear algebra, where it measured faster; on
  // GB300 the FP64 variant (one CTA per SM for lack of shared memory) is
  // FP64-latency bound and slower than the multi-kernel path.  2: always.
  if (c.fused_small_grids <= 0 || has_fields(c) || c.qoi_set != HENRY_QOI_STANDARD ||
      c.scheme != HENRY_SCHEME_CELL)
    return false;
  if (c.fused_small_grids == 1 && sizeof(T) != sizeof(float)) return false;
  const LevelGeom lg = geom(c, level);
  if (!cta_layout(lg.nx, lg.ny, (int)sizeof(T), L)) return false;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  int optin = g_smem_optin[dev].load(std::memory_order_relaxed);
  if (!optin) {
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
    g_smem_optin[dev].store(optin, std::memory_order_relaxed);
  }
  return L->bytes <= optin;
}

int smem_optin();
// Dynamic shared memory the tail kernel may use: the opt-in limit less a
// small margin (the kernel declares no static shared memory; the margin
// keeps room should it ever declare some).
constexpr int TAIL_STATIC_RESERVE = 256;
int tail_dyn_max() { return std::max(0, smem_optin() - TAIL_STATIC_RESERVE); }

// The device's opt-in shared memory per CTA (cached per device; 0 on error).
int smem_optin() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  int optin = g_smem_optin[dev].load(std::memory_order_relaxed);
  if (!optin) {
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    g_smem_optin[dev].store(optin, std::memory_order_relaxed);
  }
  return optin;
}

// Let the fused multigrid tail kernel use up to the opt-in shared memory
// (once per device and precision; outside any stream capture).
template <typename T>
int ensure_tail_attr() {
  static std::atomic<int> done[64] = {};
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_err(HENRY_EINVAL, "device %d outside [0, 64)", dev);
  if (done[dev].load(std::memory_order_relaxed)) return HENRY_OK;
  const int dmax = tail_dyn_max();
  if (dmax > 0) CK(cudaFuncSetAttribute(k_vcycle_tail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, dmax));
  done[dev].store(1, std::memory_order_relaxed);
  return HENRY_OK;
}

template <typename T>
std::map<int, Group<T>>& groups(henry_handle* h);
template <>
std::map<int, Group<double>>& groups<double>(henry_handle* h) { return h->g64; }
template <>
std::map<int, Group<float>>& groups<float>(henry_handle* h) { return h->g32; }

int ensure_pinned(henry_handle* H);

// Workspace for B samples at `level` (reused when large enough).
template <typename T>
int get_group(henry_handle* H, int level, int B, Group<T>** out, bool light = false) {
  int rc0 = ensure_pinned(H);
  if (rc0) return rc0;
  auto& m = groups<T>(H);
  Group<T>& g = m[level];
  if (g.mem && g.Bcap >= B && (light || !g.light)) {
    *out = &g;
    return HENRY_OK;
  }
  if (g.mem) {
    CK(cudaDeviceSynchronize());
    g.drop_graphs();
    CK(cudaFree(g.mem));
    g.mem = nullptr;
  }
  LevelGeom lg = geom(H->cfg, level);
  const size_t bytes = g.carve(nullptr, B, lg.nx, lg.ny, lg.h, light, has_fields(H->cfg));
  char* mem = nullptr;
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    return set_err(HENRY_ENOMEM, "cudaMalloc of %zu bytes for %d samples at level %d failed", bytes, B, level);
  }
  g.mem = mem;
  g.bytes = bytes;
  g.carve(mem, B, lg.nx, lg.ny, lg.h, light, has_fields(H->cfg));
  if (!light) {
    const int rc = ensure_tail_attr<T>();
    if (rc) return rc;
  }
  g.level = level;
  g.Bcap = B;
  *out = &g;
  return HENRY_OK;
}

template <typename T>
int max_batch(const henry_config& c, int level, bool light = false) {
  const double per = (double)bytes_per_sample<T>(c, level, light);
  const double b = std::floor(c.workspace_bytes / per);
  return (int)std::max(1.0, std::min(b, 1.0e6));
}

// Coefficients from xi for B samples (writes coef and status).
// KL basis (once per handle) and its tables at the cell centres of the fine
// grid of `level` (once per level), on the device.
int ensure_kl_tables(henry_handle* H, int level, KLTables** out) {
  const henry_config& c = H->cfg;
  if (!H->kl) {
    H->kl = new hkl::Basis2D();
    H->kl->build(c.Lx, c.Ly, c.kl_terms, c.kl_corr_len);
  }
  KLTables& t = H->kl_tables[level];
  const LevelGeom lg = geom(c, level);
  if (!t.psx) {
    const hkl::Basis2D& b = *H->kl;
    const int m = std::max(b.bx.m, b.by.m);
    std::vector<double> px((size_t)m * lg.nx, 0.0), py((size_t)m * lg.ny, 0.0);
    for (int i = 0; i < b.bx.m; ++i)
      for (int ix = 0; ix < lg.nx; ++ix) px[(size_t)i * lg.nx + ix] = b.bx.eval(i, (ix + 0.5) * lg.h);
    for (int j = 0; j < b.by.m; ++j)
      for (int iy = 0; iy < lg.ny; ++iy) py[(size_t)j * lg.ny + iy] = b.by.eval(j, (iy + 0.5) * lg.h);
    CK(cudaMalloc(&t.ti, sizeof(int) * b.terms));
    CK(cudaMalloc(&t.tj, sizeof(int) * b.terms));
    CK(cudaMalloc(&t.sl, sizeof(double) * b.terms));
    CK(cudaMalloc(&t.psx, sizeof(double) * px.size()));
    CK(cudaMalloc(&t.psy, sizeof(double) * py.size()));
    CK(cudaMemcpy(t.ti, b.ti.data(), sizeof(int) * b.terms, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(t.tj, b.tj.data(), sizeof(int) * b.terms, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(t.sl, b.sqrt_lam.data(), sizeof(double) * b.terms, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(t.psx, px.data(), sizeof(double) * px.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(t.psy, py.data(), sizeof(double) * py.size(), cudaMemcpyHostToDevice));
    t.nx = lg.nx;
    t.ny = lg.ny;
  }
  *out = &t;
  return HENRY_OK;
}

// Coefficients from the random inputs for B samples (writes coef and
// status; for the field models also the per-cell and face coefficients of
// every multigrid level).
template <typename T>
int set_coefficients(henry_handle* H, Group<T>& G, const double* xi, int B, cudaStream_t st) {
  const henry_config& c = H->cfg;
  if (!has_fields(c)) {
    CoefModel m{c.phi_mean, c.K_mean, c.qin_mean, c.phi_amp, c.logK_amp, c.qin_amp, c.mu, c.Dm};
    launch(H, st, HENRY_K_QOI, (double)B * (24 + 32 + 4),
           [&] { k_coefficients<<<nblk(B, 128), 128, 0, st>>>(m, B, xi, G.coef, G.status); });
    CKL();
    return HENRY_OK;
  }
  const int nin = n_inputs(c);
  Level& L0 = G.lv[0];
  const int64_t n0 = (int64_t)B * L0.N;
  k_coefficients_qin<<<nblk(B, 128), 128, 0, st>>>(B, nin, nin - 1, c.qin_mean, c.qin_amp, xi, G.coef, G.status);
  CKL();
  if (c.coef_model == HENRY_MODEL_KL) {
    KLTables* t = nullptr;
    int rc = ensure_kl_tables(H, G.level, &t);
    if (rc) return rc;
    KLParams P{c.kl_terms, nin, 0, c.K_mean, c.kl_sigma_logK, c.phi_mean, c.kl_sigma_phi, c.phi_lo, c.phi_hi, c.mu};
    k_fields_kl<<<nblk(n0), TPB, 0, st>>>(P, B, L0.nx, L0.ny, xi, t->ti, t->tj, t->sl, t->psx, t->psy, L0.cc,
                                          G.status);
  } else {
    const double pm = c.phi_mean;
    TwoLayerParams P{nin, pm, c.K_mean * (1.0 - pm * pm) / (pm * pm * pm), c.mu, c.Ly, -0.75};
    k_fields_two_layer<<<nblk(n0), TPB, 0, st>>>(P, B, L0.nx, L0.ny, L0.h, xi, L0.cc, G.status);
  }
  CKL();
  for (size_t k = 0; k < G.lv.size(); ++k) {
    Level& L = G.lv[k];
    if (k > 0) {
      k_restrict_cc<<<nblk((int64_t)B * L.N), TPB, 0, st>>>(B, L.nx, L.ny, G.lv[k - 1].cc, L.cc);
      CKL();
    }
    k_face_coefs<<<nblk((int64_t)B * L.N), TPB, 0, st>>>(B, L.nx, L.ny, c.Dm, L.cc, L.fc);
    CKL();
  }
  return HENRY_OK;
}


// Coarse-grid operators for every multigrid level below the fine one, plus
// the coarsest inverse.  Expects lv[k].x for k >= 1 up to date when
// rediscretising (call restrict_states first).
template <typename T, bool DROP = false>
int build_coarse_ops(henry_handle* H, Group<T>& G, int B, double inv_tau, double inv_s, cudaStream_t st) {
  typedef typename VT<T>::b4 B4;
  const Phys ph = phys_of(H->cfg);
  const double na = H->nact;
  for (int k = 1; k <= G.K; ++k) {
    Level& L = G.lv[k];
    if (H->cfg.coarse_op == HENRY_COARSE_GALERKIN && !DROP) {
      Level& Lf = G.lv[k - 1];
      launch(H, st, HENRY_K_COARSE_OPS, na * L.N * 26.0 * sizeof(B4), [&] {
        k_galerkin<T><<<nblk((int64_t)B * L.N), TPB, 0, st>>>(B, L.nx, L.ny, (const B4*)Lf.J, Lf.plane, (B4*)L.J,
                                                               L.plane, G.lin_active);
      });
    } else {
      launch(H, st, HENRY_K_COARSE_OPS, na * L.N * (32.0 + 6.0 * sizeof(B4)), [&] {
        if (L.cc)
          assemble_kernel<T, false, true, DROP>(H->cfg, L.nx, L.ny)<<<nblk((int64_t)B * L.N), TPB, 0, st>>>(
              ph, G.coef, B, L.nx, L.ny, L.h, 1.0 / L.h, L.h * L.h * inv_tau * inv_s, inv_s, L.x, L.xo, G.lin_active,
              nullptr, (B4*)L.J, L.plane, nullptr, L.cc, L.fc);
        else
          assemble_kernel<T, false>(H->cfg, L.nx, L.ny)<<<nblk((int64_t)B * L.N), TPB, 0, st>>>(ph, G.coef, B, L.nx, L.ny, L.h, 1.0 / L.h,
                                                                        L.h * L.h * inv_tau * inv_s, inv_s, L.x,
                                                                        L.xo, G.lin_active, nullptr, (B4*)L.J,
                                                                        L.plane, nullptr, nullptr, nullptr);
      });
    }
    CKL();
  }
  Level& Lc = G.lv[G.K];
  launch(H, st, HENRY_K_COARSE_OPS, na * (4.0 * sizeof(B4) + 16.0 * sizeof(T)), [&] {
    k_coarse_inverse<T><<<nblk(B, 64), 64, 0, st>>>(B, (const B4*)Lc.J, Lc.plane, G.Ainv, G.lin_active);
  });
  CKL();
  return HENRY_OK;
}

// x_k -> x_{k+1} (mean of children) for all levels; `old` selects xo.
template <typename T>
int restrict_states(henry_handle* H, Group<T>& G, int B, bool old, const int* active, cudaStream_t st) {
  for (int k = 0; k < G.K; ++k) {
    Level& Lf = G.lv[k];
    Level& Lc = G.lv[k + 1];
    launch(H, st, HENRY_K_STATE_RESTRICT, (double)H->nact * Lc.N * 80.0, [&] {
      k_restrict_state<<<nblk((int64_t)B * Lc.N), TPB, 0, st>>>(B, Lc.nx, Lc.ny, old ? Lf.xo : Lf.x,
                                                                old ? Lc.xo : Lc.x, active);
    });
    CKL();
  }
  return HENRY_OK;
}

// First multigrid level of the fused tail: the first coarse level (k >= 1)
// with at most mg_tail_cells cells per sample (-1: 2048 with FP32 linear
// algebra on fine grids of 128 x 64 cells or more, else 128, as measured),
// if the tail below it has at
// least two levels, its shared-memory layout fits and the batch is small
// enough (B x cells of that level <= mg_tail_batch_cells; larger batches keep
// those levels as separate kernels, which then are large launches and fill
// the FP64 pipe better than the tail's partly idle warps); -1: no tail.
template <typename T>
int tail_level(const henry_config& c, const Group<T>& G, int B, CtaLayout* L) {
  const int cells =
      c.mg_tail_cells >= 0 ? c.mg_tail_cells : (sizeof(T) == sizeof(float) && G.lv[0].N >= 8192 ? 2048 : 128);
  if (cells <= 0) return -1;
  for (int k = 1; k < G.K; ++k) {
    if (G.lv[k].N > cells) continue;
    if (c.mg_tail_batch_cells > 0 && (double)B * G.lv[k].N > (double)c.mg_tail_batch_cells) return -1;
    // the finest tail levels read their operators from global memory (L2)
    // when the layout does not fit otherwise
    for (int ns = 0; ns < G.K - k; ++ns)
      if (tail_layout(G.lv[k].nx, G.lv[k].ny, (int)sizeof(T), L, ns) && L->bytes <= tail_dyn_max()) return k;
    return -1;
  }
  return -1;
}

// One V(nu1, nu2) cycle: x0 = M^{-1} b0 on the fine level (active = lin_active).
template <typename T>
int vcycle(henry_handle* H, Group<T>& G, int B, const typename VT<T>::v2* b0, typename VT<T>::v2* x0,
           cudaStream_t st, const void* J0 = nullptr) {
  typedef typename VT<T>::v2 V2;
  typedef typename VT<T>::b4 B4;
  const int nu1 = H->cfg.nu1, nu2 = H->cfg.nu2;
  const int* act = G.lin_active;
  const double na = H->nact;
  const double b4 = sizeof(B4), v2 = sizeof(V2);
  CtaLayout TL;
  const int kt = tail_level<T>(H->cfg, G, B, &TL);
  const int kend = kt > 0 ? kt : G.K;  // levels 0 .. kend - 1 run as separate kernels
  const int mnt = H->cfg.mg_threads;
  for (int k = 0; k < kend; ++k) {
    Level& L = G.lv[k];
    const V2* b = k == 0 ? b0 : (const V2*)L.mgb;
    V2* x = k == 0 ? x0 : (V2*)L.mgx;
    const B4* J = (const B4*)((k == 0 && J0) ? J0 : L.J);
    const int64_t hn = (int64_t)B * L.N / 2;  // threads per half-sweep
    const double hc = na * L.N / 2;  // swept cells per half-sweep
    const int sm = k == 0 ? HENRY_K_SMOOTH : HENRY_K_SMOOTH_COARSE;
    Level& Lc = G.lv[k + 1];
    auto sweep = [&](int col, auto mode) {
      constexpr int MODE = decltype(mode)::value;
      with_mg_threads(mnt, [&](auto nt) {
        constexpr int NT = decltype(nt)::value;
        k_sweep<T, MODE, NT><<<nblk(hn, NT), NT, 0, st>>>(B, L.nx, L.ny, col, J, L.plane, b, x, nullptr, act);
      });
    };
    if (nu1 > 0) {
      launch(H, st, sm, hc * (b4 + 2 * v2), na * sweep_flops(L.nx, L.ny, 0),
             [&] { sweep(0, std::integral_constant<int, 0>()); });
      launch(H, st, sm, hc * (5 * b4 + 3 * v2), na * sweep_flops(L.nx, L.ny, 1),
             [&] { sweep(1, std::integral_constant<int, 1>()); });
      for (int i = 1; i < nu1; ++i) {
        for (int col = 0; col < 2; ++col)
          launch(H, st, sm, hc * (5 * b4 + 3 * v2), na * sweep_flops(L.nx, L.ny, 1),
                 [&] { sweep(col, std::integral_constant<int, 1>()); });
      }
      launch(H, st, HENRY_K_RESIDUAL_RESTRICT, na * Lc.N * (10 * b4 + 7 * v2), na * restrict_flops(L.nx, L.ny), [&] {
        with_mg_threads(mnt, [&](auto nt) {
          constexpr int NT = decltype(nt)::value;
          k_residual_restrict<T, 0, NT><<<nblk((int64_t)B * Lc.N, NT), NT, 0, st>>>(B, Lc.nx, Lc.ny, J, L.plane, b,
                                                                                   x, (V2*)Lc.mgb, act);
        });
      });
    } else {
      launch(H, st, HENRY_K_RESIDUAL_RESTRICT, na * L.N * v2, [&] {
        with_mg_threads(mnt, [&](auto nt) {
          constexpr int NT = decltype(nt)::value;
          k_zero<T, NT><<<nblk((int64_t)B * L.N, NT), NT, 0, st>>>((int64_t)B * L.N, x);
        });
      });
      launch(H, st, HENRY_K_RESIDUAL_RESTRICT, na * Lc.N * 5 * v2, [&] {
        with_mg_threads(mnt, [&](auto nt) {
          constexpr int NT = decltype(nt)::value;
          k_residual_restrict<T, 1, NT><<<nblk((int64_t)B * Lc.N, NT), NT, 0, st>>>(B, Lc.nx, Lc.ny, J, L.plane, b,
                                                                                   x, (V2*)Lc.mgb, act);
        });
      });
    }
    CKL();
  }
  if (kt > 0) {  // levels kt .. K: one CTA per sample in shared memory
    TailArgs A;
    std::memset(&A, 0, sizeof A);
    double tb = 2.0 * G.lv[kt].N * v2 + 16.0 * sizeof(T), tf = 0.0;
    for (int k = kt; k <= G.K; ++k) {
      const Level& L = G.lv[k];
      A.J[k - kt] = L.J;
      A.plane[k - kt] = L.plane;
      tb += 6.0 * L.N * b4;
      if (k < G.K)
        tf += (nu1 > 0 ? sweep_flops(L.nx, L.ny, 0) + (2 * nu1 - 1) * sweep_flops(L.nx, L.ny, 1) +
                             restrict_flops(L.nx, L.ny)
                       : 0.0) +
              2 * nu2 * sweep_flops(L.nx, L.ny, 1) + (nu2 > 0 ? L.N : 0);
    }
    A.b = G.lv[kt].mgb;
    A.x = G.lv[kt].mgx;
    A.ainv = G.Ainv;
    const int thr = std::min(TAIL_MAX_THREADS, std::max(32, ((G.lv[kt].N / 2 + 31) / 32) * 32));
    launch(H, st, HENRY_K_MG_TAIL, na * tb, na * (tf + 32.0), [&] {
      k_vcycle_tail<T><<<B, thr, TL.bytes, st>>>(TL, A, B, nu1, nu2, act);
    });
    CKL();
  } else {
    Level& Lc = G.lv[G.K];
    launch(H, st, HENRY_K_COARSE_SOLVE, na * (16.0 * sizeof(T) + 4 * v2), [&] {
      k_coarse_solve<T><<<nblk(B, 64), 64, 0, st>>>(B, G.Ainv, (const V2*)Lc.mgb, (V2*)Lc.mgx, act);
    });
    CKL();
  }
  for (int k = kend - 1; k >= 0; --k) {
    Level& L = G.lv[k];
    Level& Lc = G.lv[k + 1];
    const V2* b = k == 0 ? b0 : (const V2*)L.mgb;
    V2* x = k == 0 ? x0 : (V2*)L.mgx;
    const B4* J = (const B4*)((k == 0 && J0) ? J0 : L.J);
    const int64_t hn = (int64_t)B * L.N / 2;
    const double hc = na * L.N / 2;
    const int sm = k == 0 ? HENRY_K_SMOOTH : HENRY_K_SMOOTH_COARSE;
    auto sweep = [&](int col, auto mode) {
      constexpr int MODE = decltype(mode)::value;
      with_mg_threads(mnt, [&](auto nt) {
        constexpr int NT = decltype(nt)::value;
        k_sweep<T, MODE, NT><<<nblk(hn, NT), NT, 0, st>>>(B, L.nx, L.ny, col, J, L.plane, b, x,
                                                          MODE == 2 ? (const V2*)Lc.mgx : nullptr, act);
      });
    };
    if (nu2 > 0) {
      launch(H, st, sm, hc * (5 * b4 + 3.5 * v2), na * (sweep_flops(L.nx, L.ny, 1) + L.N),
             [&] { sweep(0, std::integral_constant<int, 2>()); });
      launch(H, st, sm, hc * (5 * b4 + 3 * v2), na * sweep_flops(L.nx, L.ny, 1),
             [&] { sweep(1, std::integral_constant<int, 1>()); });
      for (int i = 1; i < nu2; ++i) {
        for (int col = 0; col < 2; ++col)
          launch(H, st, sm, hc * (5 * b4 + 3 * v2), na * sweep_flops(L.nx, L.ny, 1),
                 [&] { sweep(col, std::integral_constant<int, 1>()); });
      }
    } else {
      launch(H, st, HENRY_K_RESIDUAL_RESTRICT, na * L.N * 2.25 * v2, [&] {
        with_mg_threads(mnt, [&](auto nt) {
          constexpr int NT = decltype(nt)::value;
          k_prolong_add<T, NT><<<nblk((int64_t)B * L.N, NT), NT, 0, st>>>(B, L.nx, L.ny, x, (const V2*)Lc.mgx, act);
        });
      });
    }
    CKL();
  }
  return HENRY_OK;
}

// Pinned host words for the convergence counters (allocated on first use, so
// that creating a handle touches no GPU).
int ensure_pinned(henry_handle* H) {
  if (!H->host_counter) CK(cudaMallocHost(&H->host_counter, 64));
  if (!H->host_totals) CK(cudaMallocHost(&H->host_totals, 64));
  return HENRY_OK;
}

int read_counter(henry_handle* H, const int* dev, cudaStream_t st, int* out) {
  CK(cudaMemcpyAsync(H->host_counter, dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *out = *H->host_counter;
  if (H->prof.on) prof_drain(H);
  return HENRY_OK;
}

// BiCGStab on the fine level for the samples with lin_active set; right-hand
// side -F; solution in G.dx.  rtol / maxit > 0 override the configuration's
// lin_rtol / lin_maxit.
template <typename T>
int linear_solve(henry_handle* H, Group<T>& G, int B, cudaStream_t st, const void* Jpre0 = nullptr,
                 double rtol = -1.0, int maxit = -1) {
  typedef typename VT<T>::v2 V2;
  typedef typename VT<T>::b4 B4;
  Level& L = G.lv[0];
  const int N = L.N;
  const unsigned g = nblk((int64_t)B * N);
  const double b4 = sizeof(B4), v2 = sizeof(V2);
  launch(H, st, HENRY_K_KRYLOV, (double)H->nact * N * (16 + 5 * v2), [&] {
    k_bicg_init<T><<<g, TPB, 0, st>>>(B, N, G.F, G.r, G.rh, G.p, G.v, G.dx, G.part, G.lin_active);
  });
  CKL();
  // Large grids: reduce each sample's partials once (one warp per sample)
  // instead of in every CTA of the consumer kernel.
  double* fin = (H->cfg.finalize_nct > 0 && G.nct >= H->cfg.finalize_nct) ? G.fin : nullptr;
  auto finalize = [&](int a, int b, cudaStream_t ss) {
    if (!fin) return;
    launch(H, ss, HENRY_K_KRYLOV, (double)B * G.nct * 16.0,
           [&] { k_finalize<<<nblk((int64_t)B * 32, 128), 128, 0, ss>>>(B, G.nct, G.part, a, b, fin); });
  };
  finalize(P_RR, P_RN, st);
  const double rt = rtol > 0.0 ? rtol : H->cfg.lin_rtol;
  const int mi = maxit > 0 ? maxit : H->cfg.lin_maxit;
  const double rtol2 = rt * rt;
  // One iteration after the convergence test: two preconditioned matvecs and
  // the vector updates (every argument fixed for this group and B; the
  // samples' activity is read from lin_active on the device).
  auto body = [&](int n_act, cudaStream_t ss) -> int {
    const double nc = (double)n_act * N;
    int rc = vcycle<T>(H, G, B, G.p, G.ph, ss, Jpre0);
    if (rc) return rc;
    launch(H, ss, HENRY_K_SPMV, nc * (5 * b4 + 3 * v2), n_act * spmv_flops(L.nx, L.ny, 1), [&] {
      k_spmv<T, 1><<<g, TPB, 0, ss>>>(B, L.nx, L.ny, (const B4*)L.J, L.plane, G.ph, G.v, G.rh, G.part, P_RV, 0,
                                       G.lin_active);
    });
    finalize(P_RV, -1, ss);
    launch(H, ss, HENRY_K_KRYLOV, nc * 3 * v2,
           [&] { k_bicg_s<T><<<g, TPB, 0, ss>>>(B, N, G.r, G.v, G.s, G.part, G.sc, G.lin_active, fin); });
    CKL();
    rc = vcycle<T>(H, G, B, G.s, G.sh, ss, Jpre0);
    if (rc) return rc;
    launch(H, ss, HENRY_K_SPMV, nc * (5 * b4 + 3 * v2), n_act * spmv_flops(L.nx, L.ny, 2), [&] {
      k_spmv<T, 2><<<g, TPB, 0, ss>>>(B, L.nx, L.ny, (const B4*)L.J, L.plane, G.sh, G.t, G.s, G.part, P_TS, P_TT,
                                       G.lin_active);
    });
    finalize(P_TS, P_TT, ss);
    launch(H, ss, HENRY_K_KRYLOV, nc * 8 * v2, [&] {
      k_bicg_update<T><<<g, TPB, 0, ss>>>(B, N, G.dx, G.ph, G.sh, G.s, G.t, G.rh, G.r, G.part, G.sc, G.lin_active,
                                           fin);
    });
    finalize(P_RR, P_RN, ss);
    CKL();
    return HENRY_OK;
  };
  // The body is captured once into a CUDA graph and replayed: one launch
  // instead of ~80 at level 0, which matters on launch-bound groups (small
  // grids, coarse levels).  Captured on the handle's own stream (capturing
  // the legacy default stream is not allowed; capture executes nothing) and
  // launched on `st`.  Off while the kernel timer runs.
  const bool use_graph = H->cfg.cuda_graphs && G.graphs && !H->prof.on;
  auto run_graph = [&]() -> int {
    const auto key = std::make_tuple(B, Jpre0, H->cfg.nu1, H->cfg.nu2, H->cfg.mg_tail_cells, H->cfg.mg_threads);
    auto f = G.gexec.find(key);
    if (f == G.gexec.end()) {
      if (!H->cap_stream) CK(cudaStreamCreateWithFlags(&H->cap_stream, cudaStreamNonBlocking));
      cudaGraph_t gr = nullptr;
      CK(cudaStreamBeginCapture(H->cap_stream, cudaStreamCaptureModeThreadLocal));
      const int rc = body(B, H->cap_stream);
      const cudaError_t e = cudaStreamEndCapture(H->cap_stream, &gr);
      if (rc) {
        if (e == cudaSuccess && gr) cudaGraphDestroy(gr);
        return rc;
      }
      if (e != cudaSuccess) return set_err(HENRY_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
      cudaGraphExec_t ex = nullptr;
      const cudaError_t e2 = cudaGraphInstantiate(&ex, gr, 0);
      cudaGraphDestroy(gr);
      if (e2 != cudaSuccess) return set_err(HENRY_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e2));
      f = G.gexec.emplace(key, ex).first;
    }
    CK(cudaGraphLaunch(f->second, st));
    return HENRY_OK;
  };
  for (int it = 0; it <= mi; ++it) {
    CK(cudaMemsetAsync(G.counter + 1, 0, sizeof(int), st));
    launch(H, st, HENRY_K_KRYLOV, (double)H->nact * N * (it == 0 ? 2 : 4) * v2, [&] {
      k_bicg_p<T><<<g, TPB, 0, st>>>(B, N, it, mi, rtol2, G.r, G.p, G.v, G.part, G.sc, G.lin_active,
                                      G.iters, G.status, G.counter + 1, G.totals + 1, fin);
    });
    CKL();
    int n_act = 0;
    int rc = read_counter(H, G.counter + 1, st, &n_act);
    if (rc) return rc;
    if (n_act == 0) break;
    H->nact = n_act;
    rc = use_graph ? run_graph() : body(n_act, st);
    if (rc) return rc;
  }
  return HENRY_OK;
}

// Second linear solve for the samples whose BiCGStab failed: the V-cycle
// runs on the operator without the density derivatives (DROP), fine and
// coarse, while the Krylov matvec keeps the exact Jacobian.  The coarse
// operators of the retried samples are rebuilt by the next Newton iteration.
template <typename T>
int retry_linear_solve(henry_handle* H, Group<T>& G, int B, double inv_tau, double inv_s, cudaStream_t st,
                       int* retried = nullptr) {
  typedef typename VT<T>::b4 B4;
  const henry_config& c = H->cfg;
  const LevelGeom lg = geom(c, G.level);
  Level& L = G.lv[0];
  CK(cudaMemsetAsync(G.counter + 2, 0, sizeof(int), st));
  k_mark_retry<<<nblk(B, 128), 128, 0, st>>>(B, G.newton_active, G.iters, G.lin_active, G.counter + 2);
  CKL();
  int n_retry = 0;
  int rc = read_counter(H, G.counter + 2, st, &n_retry);
  if (rc) return rc;
  if (retried) *retried = n_retry;
  if (n_retry == 0) return HENRY_OK;
  H->nact = n_retry;
  double* pscratch = G.part + P_MAX * (int64_t)B * G.nct;
  assemble_kernel<T, true, true, true>(H->cfg, L.nx, L.ny)<<<nblk((int64_t)B * L.N), TPB, 0, st>>>(
      phys_of(c), G.coef, B, L.nx, L.ny, lg.h, 1.0 / lg.h, lg.h * lg.h * inv_tau * inv_s, inv_s, L.x, L.xo,
      G.lin_active, nullptr, (B4*)G.Jp, L.plane, pscratch, L.cc, L.fc);
  CKL();
  rc = build_coarse_ops<T, true>(H, G, B, inv_tau, inv_s, st);
  if (rc) return rc;
  return linear_solve<T>(H, G, B, st, G.Jp);
}

// One implicit-Euler step (Sec. 2.3) of the B samples of a group: the
// state x^n in lv[0].x (and x^{n-1} in lv[0].xo, for the predictor) becomes
// x^{n+1}, with Newton iterations as described at the top of this file.
// `step` is the step's index (the predictor is used from step 1 on).
template <typename T>
int implicit_step(henry_handle* H, Group<T>& G, int B, int step, cudaStream_t st) {
  typedef typename VT<T>::b4 B4;
  typedef typename VT<T>::v2 V2;
  const henry_config& c = H->cfg;
  const LevelGeom lg = geom(c, G.level);
  const Phys ph = phys_of(c);
  Level& L = G.lv[0];
  const int N = L.N;
  const int64_t n0 = (int64_t)B * N;
  const double inv_tau = 1.0 / lg.tau;
  const double inv_s = 1.0 / (c.rho0 * lg.h * lg.h * inv_tau);
  const double inv_pref = 1.0 / (c.rho0 * c.g * c.Ly);
  double* pmax = G.part + P_MAX * (int64_t)B * G.nct;
  H->nact = B;
  launch(H, st, HENRY_K_NEWTON, (double)n0 * 32, [&] {
    // quadratic predictor from step 2 on (three states), linear at step 1
    const bool quad = c.newton_predictor_order == 2 && G.xoo;
    if (step > 1 && quad && c.newton_predictor > 0.0) {
      k_step_begin_predict2<<<nblk(n0), TPB, 0, st>>>(n0, c.newton_predictor, L.x, L.xo, G.xoo);
    } else {
      if (quad) k_copy_d2<<<nblk(n0), TPB, 0, st>>>(n0, L.xo, G.xoo);
      if (step > 0 && c.newton_predictor > 0.0)
        k_step_begin_predict<<<nblk(n0), TPB, 0, st>>>(n0, c.newton_predictor, L.x, L.xo);
      else
        k_step_begin<<<nblk(n0), TPB, 0, st>>>(n0, L.x, L.xo);
    }
    k_step_flags<<<nblk(B, 128), 128, 0, st>>>(B, G.status, G.newton_active, G.newton_it);
  });
  CKL();
  int rc = restrict_states<T>(H, G, B, true, G.newton_active, st);
  if (rc) return rc;
  const double vt = lg.h * lg.h * inv_tau * inv_s;
  // Fine residual and Jacobian (JAC), or the residual alone, of the samples
  // with newton_active set; F and the per-CTA max |F| into pmax.
  auto assemble_fine = [&](bool jac) {
    if (jac)
      launch(H, st, HENRY_K_ASSEMBLE, (double)H->nact * N * (48.0 + 6.0 * sizeof(B4)), [&] {
        if (L.cc)
          assemble_kernel<T, true, true>(c, L.nx, L.ny)<<<nblk(n0), TPB, 0, st>>>(
              ph, G.coef, B, L.nx, L.ny, lg.h, 1.0 / lg.h, vt, inv_s, L.x, L.xo, G.newton_active, G.F, (B4*)L.J,
              L.plane, pmax, L.cc, L.fc);
        else
          assemble_kernel<T, true>(c, L.nx, L.ny)<<<nblk(n0), TPB, 0, st>>>(ph, G.coef, B, L.nx, L.ny, lg.h, 1.0 / lg.h,
                                                                      vt, inv_s, L.x, L.xo, G.newton_active, G.F,
                                                                      (B4*)L.J, L.plane, pmax, nullptr, nullptr);
      });
    else
      launch(H, st, HENRY_K_RESIDUAL, (double)H->nact * N * 48.0, [&] {
        if (L.cc)
          assemble_kernel<T, true, true, false, false>(c, L.nx, L.ny)<<<nblk(n0), TPB, 0, st>>>(
              ph, G.coef, B, L.nx, L.ny, lg.h, 1.0 / lg.h, vt, inv_s, L.x, L.xo, G.newton_active, G.F, nullptr,
              L.plane, pmax, L.cc, L.fc);
        else
          assemble_kernel<T, true, false, false, false>(c, L.nx, L.ny)<<<nblk(n0), TPB, 0, st>>>(
              ph, G.coef, B, L.nx, L.ny, lg.h, 1.0 / lg.h, vt, inv_s, L.x, L.xo, G.newton_active, G.F, nullptr,
              L.plane, pmax, nullptr, nullptr);
      });
  };
  // Chord Newton (newton_jacobian_every = k > 1): the Jacobian and the
  // coarse operators are assembled at iterations 0, k, 2k, ... of the step
  // (and after a fallback-preconditioner retry, which rebuilt coarse
  // operators for its samples); the other iterations evaluate the residual
  // alone and reuse them.  The FP64 residual test still decides convergence.
  const int jac_every = std::max(1, c.newton_jacobian_every);
  int last_jac = -1;
  bool force_jac = false;
  for (int it = 0; it <= c.newton_maxit; ++it) {
    const bool jac_now = force_jac || last_jac < 0 || it - last_jac >= jac_every;
    // From iteration newton_residual_first on, a sample is most likely
    // converged: its residual is evaluated alone first, and the Jacobian is
    // assembled only for the samples that go on iterating (the residual is
    // recomputed with it, bit-identically).
    const bool res_first = !jac_now || (c.newton_residual_first >= 0 && it >= c.newton_residual_first);
    CK(cudaMemsetAsync(G.counter, 0, sizeof(int), st));
    assemble_fine(!res_first);
    launch(H, st, HENRY_K_NEWTON, (double)B * 8 * G.nct, [&] {
      k_newton_res_check<<<nblk((int64_t)B * 32, 128), 128, 0, st>>>(B, G.nct, c.newton_atol, c.newton_maxit, pmax,
                                                       G.newton_active, G.lin_active, G.newton_it, G.status,
                                                       G.counter, G.totals);
    });
    CKL();
    int n_act = 0;
    rc = read_counter(H, G.counter, st, &n_act);
    if (rc) return rc;
    if (n_act == 0) break;
    H->nact = n_act;
    if (jac_now) {
      if (res_first) {
        assemble_fine(true);
        CKL();
      }
      if (c.coarse_op == HENRY_COARSE_REDISCRETISE) {
        rc = restrict_states<T>(H, G, B, false, G.lin_active, st);
        if (rc) return rc;
      }
      rc = build_coarse_ops<T>(H, G, B, inv_tau, inv_s, st);
      if (rc) return rc;
      last_jac = it;
      force_jac = false;
    }
    rc = linear_solve<T>(H, G, B, st);
    if (rc) return rc;
    if (G.Jp && c.lin_retry) {  // fallback preconditioner for the samples whose solve failed
      int retried = 0;
      rc = retry_linear_solve<T>(H, G, B, inv_tau, inv_s, st, &retried);
      if (rc) return rc;
      if (retried) force_jac = true;
    }
    H->nact = n_act;
    launch(H, st, HENRY_K_NEWTON, (double)n_act * N * (32.0 + sizeof(V2)), [&] {
      double* pdc = G.part + P_DC * (int64_t)B * G.nct;
      k_newton_step_max<T><<<nblk(n0), TPB, 0, st>>>(B, N, inv_pref, G.dx, pmax, pdc, G.newton_active);
      k_newton_theta<<<nblk((int64_t)B * 32, 128), 128, 0, st>>>(B, G.nct, c.newton_dc_limit, pdc, G.newton_active, G.theta);
      k_newton_update<T><<<nblk(n0), TPB, 0, st>>>(B, N, L.x, G.dx, G.theta, G.newton_active);
      k_newton_dx_check<<<nblk((int64_t)B * 32, 128), 128, 0, st>>>(B, G.nct, c.newton_dxtol, pmax, G.newton_active, G.status);
    });
    CKL();
  }
  return HENRY_OK;
}

// Full scenario solves of B samples whose coefficients and status are set.
template <typename T>
int solve_group(henry_handle* H, Group<T>& G, int B, double* qoi, cudaStream_t st) {
  const henry_config& c = H->cfg;
  const LevelGeom lg = geom(c, G.level);
  Level& L = G.lv[0];
  const int64_t n0 = (int64_t)B * L.N;
  CK(cudaMemsetAsync(G.totals, 0, 4 * sizeof(unsigned long long), st));
  H->nact = B;
  launch(H, st, HENRY_K_QOI, (double)n0 * 16,
         [&] { k_init_state<<<nblk(n0), TPB, 0, st>>>(B, L.nx, L.ny, lg.h, c.rho0 * c.g, c.Ly, L.x); });
  CKL();
  for (int step = 0; step < lg.steps; ++step) {
    const int rc = implicit_step<T>(H, G, B, step, st);
    if (rc) return rc;
    record_series(H, G.level, step, B, L.N, lg.h, L.x, qoi, G.status, st);
  }
  launch(H, st, HENRY_K_QOI, (double)n0 * 16, [&] {
    k_qoi<<<B, TPB, 0, st>>>(B, L.nx, L.ny, lg.h, c.rho0, c.rho1 - c.rho0, G.coef, L.x, qoi, L.cc,
                             qoi_spec(c));
  });
  CKL();
  return HENRY_OK;
}

__global__ void k_merge_status(int n, const int* __restrict__ a, int32_t* __restrict__ out, int first) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int v = a[i];
  if (first) out[i] = v;
  else if (out[i] == 0) out[i] = v;
}

// *first = the smallest sample index with a non-zero status (untouched if none).
__global__ void k_first_bad(int n, const int* __restrict__ status, int* __restrict__ first) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && status[i] != 0) atomicMin(first, i);
}

// The whole scenario solve of B samples with the fused one-CTA-per-sample
// kernel (coefficients and status set).
template <typename T>
int solve_group_fused(henry_handle* H, Group<T>& G, int B, const CtaLayout& L, double* qoi, cudaStream_t st) {
  const henry_config& c = H->cfg;
  const LevelGeom lg = geom(c, G.level);
  CtaParams P;
  P.ph = phys_of(c);
  P.nx0 = lg.nx;
  P.ny0 = lg.ny;
  P.steps = lg.steps;
  P.nu1 = c.nu1;
  P.nu2 = c.nu2;
  P.newton_maxit = c.newton_maxit;
  P.lin_maxit = c.lin_maxit;
  P.h0 = lg.h;
  P.tau = lg.tau;
  P.inv_s = 1.0 / (c.rho0 * lg.h * lg.h / lg.tau);
  P.inv_pref = 1.0 / (c.rho0 * c.g * c.Ly);
  P.atol = c.newton_atol;
  P.dxtol = c.newton_dxtol;
  P.rtol2 = c.lin_rtol * c.lin_rtol;
  P.predictor = c.newton_predictor;
  P.predictor_order = c.newton_predictor_order;
  P.dc_limit = c.newton_dc_limit;
  P.rho0g = c.rho0 * c.g;
  P.Ly = c.Ly;
  CK(cudaFuncSetAttribute(k_cta_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, L.bytes));
  CK(cudaMemsetAsync(G.totals, 0, 4 * sizeof(unsigned long long), st));
  H->nact = B;
  launch(H, st, HENRY_K_FUSED, (double)B * (double)lg.nx * lg.ny * lg.steps * 64.0 + (double)B * 48.0, [&] {
    k_cta_solve<T><<<B, CTA_THREADS, L.bytes, st>>>(P, L, B, G.coef, G.lv[0].xo, G.xoo, qoi, G.status, G.totals);
  });
  CKL();
  return HENRY_OK;
}

// ---------------------------------------------------------------------------
// The vertex-centred scheme (henry_vc.cuh, henry_vc_solve.cuh): the same
// Newton / BiCGStab / V-cycle structure as the cell-centred path, on the
// vertex grid, with the BiCGStab and Newton vector kernels shared (they see
// a sample's fine vectors as `stride` entries, padding included).

template <typename T>
std::map<int, VcGroup<T>>& vgroups(henry_handle* h);
template <>
std::map<int, VcGroup<double>>& vgroups<double>(henry_handle* h) { return h->vg64; }
template <>
std::map<int, VcGroup<float>>& vgroups<float>(henry_handle* h) { return h->vg32; }

template <typename T>
size_t vc_bytes_per_sample(const henry_config& c, int level) {
  VcGroup<T> g;
  const LevelGeom lg = geom(c, level);
  return g.carve(nullptr, 1, lg.nx, lg.ny, lg.h);
}

// The face-once vertex assembly: 128-thread CTAs with 73.7 KB of dynamic
// shared memory with the Jacobian (the per-vertex kernel is used where the
// device grants less).
constexpr int VC_TILE_NT = 128;
bool vc_tile_fits() { return smem_optin() >= vc_tile_smem<true, VC_TILE_NT>() + 1024; }
template <typename T>
int ensure_vc_tile_attr() {
  static std::atomic<int> done[64] = {};
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_err(HENRY_EINVAL, "device %d outside [0, 64)", dev);
  if (done[dev].load(std::memory_order_relaxed) || !vc_tile_fits()) return HENRY_OK;
  CK(cudaFuncSetAttribute(k_vc_assemble_tile<T, true, true, VC_TILE_NT>,
                          cudaFuncAttributeMaxDynamicSharedMemorySize, vc_tile_smem<true, VC_TILE_NT>()));
  CK(cudaFuncSetAttribute(k_vc_assemble_tile<T, false, true, VC_TILE_NT>,
                          cudaFuncAttributeMaxDynamicSharedMemorySize, vc_tile_smem<true, VC_TILE_NT>()));
  done[dev].store(1, std::memory_order_relaxed);
  return HENRY_OK;
}

// Residual (and with JAC the Jacobian) of every vertex of a level: the
// face-once tile kernel with tile_assembly (default), else one thread per
// vertex evaluating its eight faces.  Same arguments and outputs, except the
// granularity of FINE's per-CTA maxima (vc_max_parts).
bool vc_use_tile(const henry_config& c) { return c.tile_assembly && vc_tile_fits(); }
template <typename T, bool FINE, bool JAC = true>
void vc_assemble_launch(const henry_config& c, cudaStream_t st, const VcParams& P, const Coef* coef, int B,
                        int stride, int64_t plane, double inv_s, const double2* x, const double2* xo,
                        const int* active, double2* F, typename VT<T>::b4* J, double* rmax_part) {
  if (vc_use_tile(c))
    k_vc_assemble_tile<T, FINE, JAC, VC_TILE_NT>
        <<<nblk((int64_t)B * stride, VC_TILE_NT), VC_TILE_NT, vc_tile_smem<JAC, VC_TILE_NT>(), st>>>(
            P, coef, B, stride, plane, inv_s, x, xo, active, F, J, rmax_part);
  else
    k_vc_assemble_st<T, FINE, JAC><<<nblk((int64_t)B * stride), TPB, 0, st>>>(P, coef, B, stride, plane, inv_s, x,
                                                                              xo, active, F, J, rmax_part);
}

template <typename T>
int vc_get_group(henry_handle* H, int level, int B, VcGroup<T>** out) {
  int rc0 = ensure_pinned(H);
  if (rc0) return rc0;
  rc0 = ensure_vc_tile_attr<T>();
  if (rc0) return rc0;
  VcGroup<T>& g = vgroups<T>(H)[level];
  if (g.mem && g.Bcap >= B) {
    *out = &g;
    return HENRY_OK;
  }
  if (g.mem) {
    CK(cudaDeviceSynchronize());
    g.drop_graphs();
    CK(cudaFree(g.mem));
    g.mem = nullptr;
  }
  const LevelGeom lg = geom(H->cfg, level);
  const size_t bytes = g.carve(nullptr, B, lg.nx, lg.ny, lg.h);
  char* mem = nullptr;
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    return set_err(HENRY_ENOMEM, "cudaMalloc of %zu bytes for %d vertex-centred samples at level %d failed", bytes,
                   B, level);
  }
  CK(cudaMemset(mem, 0, bytes));  // padding entries stay zero from here on
  g.mem = mem;
  g.bytes = bytes;
  g.carve(mem, B, lg.nx, lg.ny, lg.h);
  g.level = level;
  g.Bcap = B;
  *out = &g;
  return HENRY_OK;
}

template <typename T>
VcParams vc_params(const henry_config& c, const typename VcGroup<T>::Lv& L, double tau) {
  return VcParams{L.nx, L.ny, L.h, tau, c.rho0, c.rho1 - c.rho0, c.rho1, c.g, c.Ly};
}
template <typename T>
VcLevelArgs vc_args(const typename VcGroup<T>::Lv& L) {
  return VcLevelArgs{L.nx, L.ny, L.stride, L.plane};
}

// States of the coarse levels by injection, level by level (old: the old state).
template <typename T>
int vc_inject(henry_handle* H, VcGroup<T>& G, int B, bool old, const int* active, cudaStream_t st) {
  for (int k = 1; k <= G.K; ++k) {
    auto& Lf = G.lv[k - 1];
    auto& Lc = G.lv[k];
    launch(H, st, HENRY_K_STATE_RESTRICT, (double)H->nact * Lc.NV * 32.0, [&] {
      k_vc_inject<<<nblk((int64_t)B * Lc.NV), TPB, 0, st>>>(B, Lc.nx, Lc.ny, Lf.stride, Lc.stride,
                                                             old ? Lf.xo : Lf.x, old ? Lc.xo : Lc.x, active);
    });
    CKL();
  }
  return HENRY_OK;
}

// Coarse operators rediscretised at the injected states (call vc_inject for
// the iterate first) and the coarsest inverse, for the samples with lin_active.
template <typename T>
int vc_coarse_ops(henry_handle* H, VcGroup<T>& G, int B, double tau, double inv_s, cudaStream_t st) {
  typedef typename VT<T>::b4 B4;
  for (int k = 1; k <= G.K; ++k) {
    auto& L = G.lv[k];
    launch(H, st, HENRY_K_COARSE_OPS, (double)H->nact * L.NV * (32.0 + 10.0 * sizeof(B4)), [&] {
      vc_assemble_launch<T, false>(H->cfg, st, vc_params<T>(H->cfg, L, tau), G.coef, B, L.stride, L.plane, inv_s, L.x,
                                   L.xo, G.lin_active, nullptr, (B4*)L.J, nullptr);
    });
    CKL();
  }
  auto& Lc = G.lv[G.K];
  launch(H, st, HENRY_K_COARSE_OPS, (double)H->nact * (9.0 * 6 * sizeof(B4) + 144.0 * sizeof(T)), [&] {
    k_vc_coarse_inverse<T><<<nblk(B, 64), 64, 0, st>>>(B, vc_args<T>(Lc), (const B4*)Lc.J, G.Ainv, G.lin_active);
  });
  CKL();
  return HENRY_OK;
}

// One V(nu1, nu2) cycle on the vertex hierarchy: x0 = M^{-1} b0 (fine level,
// active = lin_active).  Colours (ci, cj) in the order 0 (0,0), 1 (1,0),
// 2 (0,1), 3 (1,1) before the coarse correction and 3..0 after it.
template <typename T>
int vc_vcycle(henry_handle* H, VcGroup<T>& G, int B, const typename VT<T>::v2* b0, typename VT<T>::v2* x0,
              cudaStream_t st) {
  typedef typename VT<T>::v2 V2;
  typedef typename VT<T>::b4 B4;
  const int nu1 = H->cfg.nu1, nu2 = H->cfg.nu2;
  const int* act = G.lin_active;
  const double na = H->nact;
  const double b4 = sizeof(B4), v2 = sizeof(V2);
  static const int CI[4] = {0, 1, 0, 1}, CJ[4] = {0, 0, 1, 1};
  auto sweep = [&](int k, int col, const V2* b, V2* x) {
    auto& L = G.lv[k];
    const VcLevelArgs A = vc_args<T>(L);
    const int nv = vc_colour_rows(L.ny + 1, CJ[col]) * vc_colour_cols(L.nx + 1, CI[col]);
    launch(H, st, k == 0 ? HENRY_K_SMOOTH : HENRY_K_SMOOTH_COARSE, na * nv * (9 * b4 + 3 * v2),
           na * nv * (8 * 8.0 + 6.0), [&] {
             k_vc_sweep<T, 1><<<nblk((int64_t)B * nv), TPB, 0, st>>>(B, A, CI[col], CJ[col], (const B4*)L.J, b, x,
                                                                     act);
           });
  };
  for (int k = 0; k < G.K; ++k) {
    auto& L = G.lv[k];
    auto& Lc = G.lv[k + 1];
    const VcLevelArgs A = vc_args<T>(L), Ac = vc_args<T>(Lc);
    const V2* b = k == 0 ? b0 : (const V2*)L.mgb;
    V2* x = k == 0 ? x0 : (V2*)L.mgx;
    const int sm = k == 0 ? HENRY_K_SMOOTH : HENRY_K_SMOOTH_COARSE;
    if (nu1 > 0) {
      launch(H, st, sm, na * L.NV * (0.25 * (b4 + v2) + v2), na * L.NV * 1.5, [&] {
        k_vc_sweep<T, 0><<<nblk((int64_t)B * L.NV), TPB, 0, st>>>(B, A, 0, 0, (const B4*)L.J, b, x, act);
      });
      for (int col = 1; col < 4; ++col) sweep(k, col, b, x);
      for (int i = 1; i < nu1; ++i)
        for (int col = 0; col < 4; ++col) sweep(k, col, b, x);
    } else {
      launch(H, st, HENRY_K_RESIDUAL_RESTRICT, na * L.NV * v2, [&] {
        k_vc_sweep<T, 2><<<nblk((int64_t)B * L.NV), TPB, 0, st>>>(B, A, 0, 0, (const B4*)L.J, b, x, act);
      });
    }
    launch(H, st, HENRY_K_RESIDUAL_RESTRICT, na * L.NV * (9 * b4 + 3 * v2) + na * Lc.NV * v2,
           na * L.NV * 74.0, [&] {
             k_vc_residual<T><<<nblk((int64_t)B * L.NV), TPB, 0, st>>>(B, A, (const B4*)L.J, b, x, (V2*)L.mgr, act);
             k_vc_restrict<T><<<nblk((int64_t)B * Lc.NV), TPB, 0, st>>>(B, A, Ac, (const V2*)L.mgr, (V2*)Lc.mgb,
                                                                        act);
           });
    CKL();
  }
  {
    auto& Lc = G.lv[G.K];
    launch(H, st, HENRY_K_COARSE_SOLVE, na * (144.0 * sizeof(T) + 24 * v2), [&] {
      k_vc_coarse_solve<T><<<nblk(B, 64), 64, 0, st>>>(B, vc_args<T>(Lc), G.Ainv, (const V2*)Lc.mgb, (V2*)Lc.mgx,
                                                       act);
    });
    CKL();
  }
  for (int k = G.K - 1; k >= 0; --k) {
    auto& L = G.lv[k];
    auto& Lc = G.lv[k + 1];
    const V2* b = k == 0 ? b0 : (const V2*)L.mgb;
    V2* x = k == 0 ? x0 : (V2*)L.mgx;
    launch(H, st, HENRY_K_RESIDUAL_RESTRICT, na * (L.NV * 2.0 * v2 + Lc.NV * v2), [&] {
      k_vc_prolong_add<T><<<nblk((int64_t)B * L.NV), TPB, 0, st>>>(B, vc_args<T>(L), vc_args<T>(Lc), x,
                                                                   (const V2*)Lc.mgx, act);
    });
    for (int i = 0; i < nu2; ++i)
      for (int col = 3; col >= 0; --col) sweep(k, col, b, x);
    CKL();
  }
  return HENRY_OK;
}

// BiCGStab on the fine vertex grid for the samples with lin_active set;
// right-hand side -F, solution in G.dx (linear_solve's kernels and order).
template <typename T>
int vc_linear_solve(henry_handle* H, VcGroup<T>& G, int B, cudaStream_t st, double rtol = -1.0, int maxit = -1) {
  typedef typename VT<T>::v2 V2;
  typedef typename VT<T>::b4 B4;
  auto& L = G.lv[0];
  const int N = L.stride;
  const VcLevelArgs A = vc_args<T>(L);
  const unsigned g = nblk((int64_t)B * N);
  const double b4 = sizeof(B4), v2 = sizeof(V2);
  launch(H, st, HENRY_K_KRYLOV, (double)H->nact * N * (16 + 5 * v2), [&] {
    k_bicg_init<T><<<g, TPB, 0, st>>>(B, N, G.F, G.r, G.rh, G.p, G.v, G.dx, G.part, G.lin_active);
  });
  CKL();
  double* fin = (H->cfg.finalize_nct > 0 && G.nct >= H->cfg.finalize_nct) ? G.fin : nullptr;
  auto finalize = [&](int a, int b, cudaStream_t ss) {
    if (!fin) return;
    launch(H, ss, HENRY_K_KRYLOV, (double)B * G.nct * 16.0,
           [&] { k_finalize<<<nblk((int64_t)B * 32, 128), 128, 0, ss>>>(B, G.nct, G.part, a, b, fin); });
  };
  finalize(P_RR, P_RN, st);
  const double rt = rtol > 0.0 ? rtol : H->cfg.lin_rtol;
  const int mi = maxit > 0 ? maxit : H->cfg.lin_maxit;
  const double rtol2 = rt * rt;
  auto body = [&](int n_act, cudaStream_t ss) -> int {
    const double nc = (double)n_act * L.NV;
    int rc = vc_vcycle<T>(H, G, B, G.p, G.ph, ss);
    if (rc) return rc;
    launch(H, ss, HENRY_K_SPMV, nc * (9 * b4 + 3 * v2), nc * (9 * 8.0 + 4.0), [&] {
      k_vc_spmv<T, 1><<<g, TPB, 0, ss>>>(B, A, (const B4*)L.J, G.ph, G.v, G.rh, G.part, P_RV, 0, G.lin_active);
    });
    finalize(P_RV, -1, ss);
    launch(H, ss, HENRY_K_KRYLOV, nc * 3 * v2,
           [&] { k_bicg_s<T><<<g, TPB, 0, ss>>>(B, N, G.r, G.v, G.s, G.part, G.sc, G.lin_active, fin); });
    CKL();
    rc = vc_vcycle<T>(H, G, B, G.s, G.sh, ss);
    if (rc) return rc;
    launch(H, ss, HENRY_K_SPMV, nc * (9 * b4 + 3 * v2), nc * (9 * 8.0 + 8.0), [&] {
      k_vc_spmv<T, 2><<<g, TPB, 0, ss>>>(B, A, (const B4*)L.J, G.sh, G.t, G.s, G.part, P_TS, P_TT, G.lin_active);
    });
    finalize(P_TS, P_TT, ss);
    launch(H, ss, HENRY_K_KRYLOV, nc * 8 * v2, [&] {
      k_bicg_update<T><<<g, TPB, 0, ss>>>(B, N, G.dx, G.ph, G.sh, G.s, G.t, G.rh, G.r, G.part, G.sc, G.lin_active,
                                           fin);
    });
    finalize(P_RR, P_RN, ss);
    CKL();
    return HENRY_OK;
  };
  const bool use_graph = H->cfg.cuda_graphs && !H->prof.on;
  auto run_graph = [&]() -> int {
    const auto key = std::make_tuple(B, H->cfg.nu1, H->cfg.nu2);
    auto f = G.gexec.find(key);
    if (f == G.gexec.end()) {
      if (!H->cap_stream) CK(cudaStreamCreateWithFlags(&H->cap_stream, cudaStreamNonBlocking));
      cudaGraph_t gr = nullptr;
      CK(cudaStreamBeginCapture(H->cap_stream, cudaStreamCaptureModeThreadLocal));
      const int rc = body(B, H->cap_stream);
      const cudaError_t e = cudaStreamEndCapture(H->cap_stream, &gr);
      if (rc) {
        if (e == cudaSuccess && gr) cudaGraphDestroy(gr);
        return rc;
      }
      if (e != cudaSuccess) return set_err(HENRY_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
      cudaGraphExec_t ex = nullptr;
      const cudaError_t e2 = cudaGraphInstantiate(&ex, gr, 0);
      cudaGraphDestroy(gr);
      if (e2 != cudaSuccess) return set_err(HENRY_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e2));
      f = G.gexec.emplace(key, ex).first;
    }
    CK(cudaGraphLaunch(f->second, st));
    return HENRY_OK;
  };
  for (int it = 0; it <= mi; ++it) {
    CK(cudaMemsetAsync(G.counter + 1, 0, sizeof(int), st));
    launch(H, st, HENRY_K_KRYLOV, (double)H->nact * N * (it == 0 ? 2 : 4) * v2, [&] {
      k_bicg_p<T><<<g, TPB, 0, st>>>(B, N, it, mi, rtol2, G.r, G.p, G.v, G.part, G.sc, G.lin_active, G.iters,
                                      G.status, G.counter + 1, G.totals + 1, fin);
    });
    CKL();
    int n_act = 0;
    int rc = read_counter(H, G.counter + 1, st, &n_act);
    if (rc) return rc;
    if (n_act == 0) break;
    H->nact = n_act;
    rc = use_graph ? run_graph() : body(n_act, st);
    if (rc) return rc;
  }
  return HENRY_OK;
}

// Where the fine assembly leaves its per-CTA maxima of |F| and how many a
// sample has: the P_MAX partials (nct per sample) for the per-vertex kernel;
// for the tile kernel's 128-entry CTAs (2 nct per sample) the P_RR and P_RN
// partials, which are free between an assembly and the residual test and
// are rewritten by the next Krylov solve.
template <typename T>
double* vc_max_parts(const henry_handle* H, VcGroup<T>& G, int B, int* nct) {
  if (vc_use_tile(H->cfg)) {
    *nct = G.nct * (TPB / VC_TILE_NT);
    return G.part + P_RR * (int64_t)B * G.nct;
  }
  *nct = G.nct;
  return G.part + P_MAX * (int64_t)B * G.nct;
}

// Fine residual and Jacobian (scaled by inv_s; jac = false: the residual
// alone) of the samples with newton_active set, with the per-CTA max |F|
// into vc_max_parts.
template <typename T>
int vc_assemble_fine(henry_handle* H, VcGroup<T>& G, int B, double tau, double inv_s, cudaStream_t st,
                     bool jac = true) {
  typedef typename VT<T>::b4 B4;
  auto& L = G.lv[0];
  int nct_max = 0;
  double* pm = vc_max_parts<T>(H, G, B, &nct_max);
  if (jac)
    launch(H, st, HENRY_K_ASSEMBLE, (double)H->nact * L.NV * (48.0 + 10.0 * sizeof(B4)), [&] {
      vc_assemble_launch<T, true>(H->cfg, st, vc_params<T>(H->cfg, L, tau), G.coef, B, L.stride, L.plane, inv_s, L.x,
                                  L.xo, G.newton_active, G.F, (B4*)L.J, pm);
    });
  else
    launch(H, st, HENRY_K_RESIDUAL, (double)H->nact * L.NV * 48.0, [&] {
      vc_assemble_launch<T, true, false>(H->cfg, st, vc_params<T>(H->cfg, L, tau), G.coef, B, L.stride, L.plane, inv_s,
                                         L.x, L.xo, G.newton_active, G.F, nullptr, pm);
    });
  CKL();
  return HENRY_OK;
}

// One implicit-Euler step of the vertex-centred scheme (implicit_step's
// Newton iteration and tests).
template <typename T>
int vc_implicit_step(henry_handle* H, VcGroup<T>& G, int B, int step, cudaStream_t st) {
  typedef typename VT<T>::v2 V2;
  const henry_config& c = H->cfg;
  const LevelGeom lg = geom(c, G.level);
  auto& L = G.lv[0];
  const int N = L.stride;
  const int64_t n0 = (int64_t)B * N;
  const double inv_s = 1.0 / (c.rho0 * lg.h * lg.h / lg.tau);
  const double inv_pref = 1.0 / (c.rho0 * c.g * c.Ly);
  double* pmax = G.part + P_MAX * (int64_t)B * G.nct;
  H->nact = B;
  launch(H, st, HENRY_K_NEWTON, (double)n0 * 32, [&] {
    // the predictor as in implicit_step (quadratic from step 2 on)
    const bool quad = c.newton_predictor_order == 2 && G.xoo;
    if (step > 1 && quad && c.newton_predictor > 0.0) {
      k_step_begin_predict2<<<nblk(n0), TPB, 0, st>>>(n0, c.newton_predictor, L.x, L.xo, G.xoo);
    } else {
      if (quad) k_copy_d2<<<nblk(n0), TPB, 0, st>>>(n0, L.xo, G.xoo);
      if (step > 0 && c.newton_predictor > 0.0)
        k_step_begin_predict<<<nblk(n0), TPB, 0, st>>>(n0, c.newton_predictor, L.x, L.xo);
      else
        k_step_begin<<<nblk(n0), TPB, 0, st>>>(n0, L.x, L.xo);
    }
    k_step_flags<<<nblk(B, 128), 128, 0, st>>>(B, G.status, G.newton_active, G.newton_it);
  });
  CKL();
  int rc = vc_inject<T>(H, G, B, true, G.newton_active, st);
  if (rc) return rc;
  // residual-first test and chord Newton as in implicit_step
  const int jac_every = std::max(1, c.newton_jacobian_every);
  int last_jac = -1;
  for (int it = 0; it <= c.newton_maxit; ++it) {
    const bool jac_now = last_jac < 0 || it - last_jac >= jac_every;
    const bool res_first = !jac_now || (c.newton_residual_first >= 0 && it >= c.newton_residual_first);
    CK(cudaMemsetAsync(G.counter, 0, sizeof(int), st));
    rc = vc_assemble_fine<T>(H, G, B, lg.tau, inv_s, st, !res_first);
    if (rc) return rc;
    int nct_f = 0;
    const double* fmax_parts = vc_max_parts<T>(H, G, B, &nct_f);
    launch(H, st, HENRY_K_NEWTON, (double)B * 8 * nct_f, [&] {
      k_newton_res_check<<<nblk((int64_t)B * 32, 128), 128, 0, st>>>(B, nct_f, c.newton_atol, c.newton_maxit, fmax_parts,
                                                       G.newton_active, G.lin_active, G.newton_it, G.status,
                                                       G.counter, G.totals);
    });
    CKL();
    int n_act = 0;
    rc = read_counter(H, G.counter, st, &n_act);
    if (rc) return rc;
    if (n_act == 0) break;
    H->nact = n_act;
    if (jac_now) {
      if (res_first) rc = vc_assemble_fine<T>(H, G, B, lg.tau, inv_s, st);
      if (!rc) rc = vc_inject<T>(H, G, B, false, G.lin_active, st);
      if (!rc) rc = vc_coarse_ops<T>(H, G, B, lg.tau, inv_s, st);
      last_jac = it;
    }
    if (!rc) rc = vc_linear_solve<T>(H, G, B, st);
    if (rc) return rc;
    H->nact = n_act;
    launch(H, st, HENRY_K_NEWTON, (double)n_act * N * (32.0 + sizeof(V2)), [&] {
      double* pdc = G.part + P_DC * (int64_t)B * G.nct;
      k_newton_step_max<T><<<nblk(n0), TPB, 0, st>>>(B, N, inv_pref, G.dx, pmax, pdc, G.newton_active);
      k_newton_theta<<<nblk((int64_t)B * 32, 128), 128, 0, st>>>(B, G.nct, c.newton_dc_limit, pdc, G.newton_active, G.theta);
      k_newton_update<T><<<nblk(n0), TPB, 0, st>>>(B, N, L.x, G.dx, G.theta, G.newton_active);
      k_newton_dx_check<<<nblk((int64_t)B * 32, 128), 128, 0, st>>>(B, G.nct, c.newton_dxtol, pmax, G.newton_active, G.status);
    });
    CKL();
  }
  return HENRY_OK;
}

// Full scenario solves of B samples of the vertex-centred scheme whose
// coefficients and status are set; QoIs [B][2] (salt mass, c at (1.5, 0.25)).
template <typename T>
int vc_solve_group(henry_handle* H, VcGroup<T>& G, int B, double* qoi, cudaStream_t st) {
  const henry_config& c = H->cfg;
  const LevelGeom lg = geom(c, G.level);
  auto& L = G.lv[0];
  CK(cudaMemsetAsync(G.totals, 0, 4 * sizeof(unsigned long long), st));
  H->nact = B;
  launch(H, st, HENRY_K_QOI, (double)B * L.stride * 16, [&] {
    k_vc_init_state<<<nblk((int64_t)B * L.stride), TPB, 0, st>>>(B, L.nx, L.ny, L.stride, lg.h, c.rho0 * c.g,
                                                                c.rho1 * c.g, c.Ly, L.x);
  });
  CKL();
  for (int step = 0; step < lg.steps; ++step) {
    const int rc = vc_implicit_step<T>(H, G, B, step, st);
    if (rc) return rc;
  }
  const int ip = (int)std::lround(1.5 / lg.h), jp = (int)std::lround(0.25 / lg.h);
  launch(H, st, HENRY_K_QOI, (double)B * L.NV * 16, [&] {
    k_vc_qoi<<<B, TPB, 0, st>>>(B, L.nx, L.ny, L.stride, lg.h, c.rho0, c.rho1 - c.rho0, ip, jp, G.coef, L.x,
                                G.status, qoi);
  });
  CKL();
  return HENRY_OK;
}

template <typename T>
int vc_set_coefficients(henry_handle* H, VcGroup<T>& G, const double* xi, int B, cudaStream_t st) {
  const henry_config& c = H->cfg;
  const CoefModel m{c.phi_mean, c.K_mean, c.qin_mean, c.phi_amp, c.logK_amp, c.qin_amp, c.mu, c.Dm};
  launch(H, st, HENRY_K_QOI, (double)B * (24 + 32 + 4),
         [&] { k_coefficients<<<nblk(B, 128), 128, 0, st>>>(m, B, xi, G.coef, G.status); });
  CKL();
  return HENRY_OK;
}

// The level's autotuned settings (henry_autotune) in force for one scope.
struct TuningScope {
  henry_handle* H;
  henry_config saved;
  TuningScope(henry_handle* h, int level) : H(h), saved(h->cfg) {
    auto f = h->tuned.find(level);
    if (f == h->tuned.end()) return;
    h->cfg.lin_rtol = f->second.lin_rtol;
    h->cfg.nu1 = f->second.nu1;
    h->cfg.nu2 = f->second.nu2;
    h->cfg.fused_small_grids = f->second.fused_small_grids;
    h->cfg.mg_tail_cells = f->second.mg_tail_cells;
    h->cfg.newton_residual_first = f->second.newton_residual_first;
    h->cfg.newton_jacobian_every = std::max(1, f->second.newton_jacobian_every);
    h->cfg.assembly_tile_w = f->second.assembly_tile_w;
    h->cfg.mg_threads = f->second.mg_threads;
    if (f->second.newton_predictor_order > 0) h->cfg.newton_predictor_order = f->second.newton_predictor_order;
  }
  ~TuningScope() { H->cfg = saved; }
};

template <typename T>
int vc_batch_solve_level(henry_handle* H, int level, const double* xi, int n, double* qoi, int32_t* status,
                         bool first, henry_stats* stats, cudaStream_t st) {
  TuningScope tuning(H, level);
  const LevelGeom lg = geom(H->cfg, level);
  const double per = (double)vc_bytes_per_sample<T>(H->cfg, level);
  const int Bmax = (int)std::max(1.0, std::min(std::floor(H->cfg.workspace_bytes / per), 1.0e6));
  for (int off = 0; off < n; off += Bmax) {
    const int B = std::min(Bmax, n - off);
    VcGroup<T>* G = nullptr;
    int rc = vc_get_group<T>(H, level, std::min(Bmax, n), &G);
    if (!rc) rc = vc_set_coefficients<T>(H, *G, xi + 3 * (int64_t)off, B, st);
    if (!rc) rc = vc_solve_group<T>(H, *G, B, qoi + 2 * (int64_t)off, st);
    if (rc) return rc;
    k_merge_status<<<nblk(B, 128), 128, 0, st>>>(B, G->status, status + off, first ? 1 : 0);
    CKL();
    if (stats) {
      CK(cudaMemcpyAsync(H->host_totals, G->totals, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      stats->newton_iters += H->host_totals[0];
      stats->linear_iters += H->host_totals[1];
      stats->newton_solves += (int64_t)B * lg.steps;
      stats->cell_steps += (double)B * lg.nx * lg.ny * lg.steps;
    }
  }
  return HENRY_OK;
}

// Per-step entry points of the vertex-centred scheme (states in natural
// vertex order [n][ny + 1][nx + 1][2]); the cell-centred step_entry's cases.
template <typename T>
int vc_step_entry(henry_handle* H, int which, int level, const double* xi, int n, const double* state,
                  const double* state_old, const double* in, double* out, double* out2, int32_t* iters,
                  cudaStream_t st) {
  typedef typename VT<T>::v2 V2;
  typedef typename VT<T>::b4 B4;
  VcGroup<T>* Gp = nullptr;
  int rc = vc_get_group<T>(H, level, n, &Gp);
  if (rc) return rc;
  VcGroup<T>& G = *Gp;
  H->nact = n;
  rc = vc_set_coefficients<T>(H, G, xi, n, st);
  if (rc) return rc;
  auto& L = G.lv[0];
  const int64_t nv = (int64_t)n * L.NV;
  const LevelGeom lg = geom(H->cfg, level);
  const double inv_s = 1.0 / (H->cfg.rho0 * lg.h * lg.h / lg.tau);
  k_vc_to_storage<double2><<<nblk(nv), TPB, 0, st>>>(n, L.nx, L.ny, L.stride, (const double2*)state, L.x);
  k_vc_to_storage<double2><<<nblk(nv), TPB, 0, st>>>(n, L.nx, L.ny, L.stride, (const double2*)state_old, L.xo);
  k_step_flags<<<nblk(n, 128), 128, 0, st>>>(n, G.status, G.newton_active, G.newton_it);
  CK(cudaMemcpyAsync(G.lin_active, G.newton_active, sizeof(int) * n, cudaMemcpyDeviceToDevice, st));
  CKL();
  rc = vc_assemble_fine<T>(H, G, n, lg.tau, inv_s, st);
  if (!rc && which >= 2) {
    rc = vc_inject<T>(H, G, n, true, G.lin_active, st);
    if (!rc) rc = vc_inject<T>(H, G, n, false, G.lin_active, st);
    if (!rc) rc = vc_coarse_ops<T>(H, G, n, lg.tau, inv_s, st);
  }
  if (rc) return rc;
  switch (which) {
    case 0:
      k_vc_from_storage<double2><<<nblk(nv), TPB, 0, st>>>(n, L.nx, L.ny, L.stride, G.F, (double2*)out);
      if (out2) k_vc_blocks_out<B4><<<nblk(nv), TPB, 0, st>>>(n, L.nx, L.ny, L.stride, (const B4*)L.J, L.plane, out2);
      break;
    case 1:
      k_vc_to_storage<V2><<<nblk(nv), TPB, 0, st>>>(n, L.nx, L.ny, L.stride, (const double2*)in, G.p);
      k_vc_spmv<T, 0><<<nblk((int64_t)n * L.stride), TPB, 0, st>>>(n, vc_args<T>(L), (const B4*)L.J, G.p, G.v,
                                                                    nullptr, nullptr, 0, 0, G.lin_active);
      k_vc_from_storage<V2><<<nblk(nv), TPB, 0, st>>>(n, L.nx, L.ny, L.stride, G.v, (double2*)out);
      break;
    case 2:
      k_vc_to_storage<V2><<<nblk(nv), TPB, 0, st>>>(n, L.nx, L.ny, L.stride, (const double2*)in, G.p);
      CKL();
      rc = vc_vcycle<T>(H, G, n, G.p, G.ph, st);
      if (rc) return rc;
      k_vc_from_storage<V2><<<nblk(nv), TPB, 0, st>>>(n, L.nx, L.ny, L.stride, G.ph, (double2*)out);
      break;
    case 3:
      k_vc_to_storage<double2><<<nblk(nv), TPB, 0, st>>>(n, L.nx, L.ny, L.stride, (const double2*)in, G.F);
      k_scale_d2<<<nblk((int64_t)n * L.stride), TPB, 0, st>>>((int64_t)n * L.stride, -1.0, G.F);
      CKL();
      CK(cudaMemsetAsync(G.totals, 0, 4 * sizeof(unsigned long long), st));
      rc = vc_linear_solve<T>(H, G, n, st);
      if (rc) return rc;
      k_vc_from_storage<V2><<<nblk(nv), TPB, 0, st>>>(n, L.nx, L.ny, L.stride, G.dx, (double2*)out);
      if (iters) CK(cudaMemcpyAsync(iters, G.iters, sizeof(int) * n, cudaMemcpyDeviceToDevice, st));
      break;
  }
  CKL();
  return HENRY_OK;
}

template <typename T>
int batch_solve_level(henry_handle* H, int level, const double* xi, int n, double* qoi, int32_t* status, bool first,
                      henry_stats* stats, cudaStream_t st) {
  TuningScope tuning(H, level);
  CtaLayout CL;
  const bool fused = fused_eligible<T>(H->cfg, level, &CL);
  const int Bmax = max_batch<T>(H->cfg, level, fused);
  const LevelGeom lg = geom(H->cfg, level);
  for (int off = 0; off < n; off += Bmax) {
    const int B = std::min(Bmax, n - off);
    Group<T>* G = nullptr;
    int rc = get_group<T>(H, level, std::min(Bmax, n), &G, fused);
    if (rc) return rc;
    rc = set_coefficients<T>(H, *G, xi + (int64_t)n_inputs(H->cfg) * off, B, st);
    if (rc) return rc;
    const int nq = qoi_count(H->cfg);
    rc = fused ? solve_group_fused<T>(H, *G, B, CL, qoi + nq * (int64_t)off, st)
               : solve_group<T>(H, *G, B, qoi + nq * (int64_t)off, st);
    if (rc) return rc;
    k_merge_status<<<nblk(B, 128), 128, 0, st>>>(B, G->status, status + off, first ? 1 : 0);
    CKL();
    if (stats) {
      CK(cudaMemcpyAsync(H->host_totals, G->totals, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      stats->newton_iters += H->host_totals[0];
      stats->linear_iters += H->host_totals[1];
      stats->newton_solves += (int64_t)B * lg.steps;
      stats->cell_steps += (double)B * lg.nx * lg.ny * lg.steps;
    }
  }
  return HENRY_OK;
}

// Per-step entry points: set up one group from given states.
template <typename T>
int setup_from_states(henry_handle* H, int level, const double* xi, int n, const double* state,
                      const double* state_old, Group<T>** out, cudaStream_t st) {
  Group<T>* G = nullptr;
  int rc = get_group<T>(H, level, n, &G);
  if (rc) return rc;
  H->nact = n;
  rc = set_coefficients<T>(H, *G, xi, n, st);
  if (rc) return rc;
  Level& L = G->lv[0];
  const int64_t n0 = (int64_t)n * L.N;
  k_to_storage<double2><<<nblk(n0), TPB, 0, st>>>(n, L.nx, L.ny, (const double2*)state, L.x);
  k_to_storage<double2><<<nblk(n0), TPB, 0, st>>>(n, L.nx, L.ny, (const double2*)state_old, L.xo);
  k_step_flags<<<nblk(n, 128), 128, 0, st>>>(n, G->status, G->newton_active, G->newton_it);
  CK(cudaMemcpyAsync(G->lin_active, G->newton_active, sizeof(int) * n, cudaMemcpyDeviceToDevice, st));
  CKL();
  *out = G;
  return HENRY_OK;
}

// jac = false: the fine residual alone, with the kernel of the Newton
// test's residual-first evaluations.
template <typename T>
int assemble_all(henry_handle* H, Group<T>& G, int n, bool coarse, cudaStream_t st, bool jac = true) {
  typedef typename VT<T>::b4 B4;
  const henry_config& c = H->cfg;
  const LevelGeom lg = geom(c, G.level);
  const double inv_tau = 1.0 / lg.tau;
  const double inv_s = 1.0 / (c.rho0 * lg.h * lg.h * inv_tau);
  Level& L = G.lv[0];
  if (!jac) {
    double* pm = G.part + P_MAX * (int64_t)n * G.nct;
    if (L.cc)
      assemble_kernel<T, true, true, false, false>(c, L.nx, L.ny)<<<nblk((int64_t)n * L.N), TPB, 0, st>>>(
          phys_of(c), G.coef, n, L.nx, L.ny, lg.h, 1.0 / lg.h, lg.h * lg.h * inv_tau * inv_s, inv_s, L.x, L.xo,
          G.newton_active, G.F, nullptr, L.plane, pm, L.cc, L.fc);
    else
      assemble_kernel<T, true, false, false, false>(c, L.nx, L.ny)<<<nblk((int64_t)n * L.N), TPB, 0, st>>>(
          phys_of(c), G.coef, n, L.nx, L.ny, lg.h, 1.0 / lg.h, lg.h * lg.h * inv_tau * inv_s, inv_s, L.x, L.xo,
          G.newton_active, G.F, nullptr, L.plane, pm, nullptr, nullptr);
    CKL();
    return HENRY_OK;
  }
  if (L.cc)
    assemble_kernel<T, true, true>(H->cfg, L.nx, L.ny)<<<nblk((int64_t)n * L.N), TPB, 0, st>>>(
        phys_of(c), G.coef, n, L.nx, L.ny, lg.h, 1.0 / lg.h, lg.h * lg.h * inv_tau * inv_s, inv_s, L.x, L.xo,
        G.newton_active, G.F, (B4*)L.J, L.plane, G.part + P_MAX * (int64_t)n * G.nct, L.cc, L.fc);
  else
    assemble_kernel<T, true>(H->cfg, L.nx, L.ny)<<<nblk((int64_t)n * L.N), TPB, 0, st>>>(phys_of(c), G.coef, n, L.nx, L.ny, lg.h, 1.0 / lg.h,
                                                                 lg.h * lg.h * inv_tau * inv_s, inv_s, L.x, L.xo,
                                                                 G.newton_active, G.F, (B4*)L.J, L.plane,
                                                                 G.part + P_MAX * (int64_t)n * G.nct, nullptr, nullptr);
  CKL();
  if (!coarse) return HENRY_OK;
  int rc = restrict_states<T>(H, G, n, true, G.lin_active, st);
  if (rc) return rc;
  rc = restrict_states<T>(H, G, n, false, G.lin_active, st);
  if (rc) return rc;
  return build_coarse_ops<T>(H, G, n, inv_tau, inv_s, st);
}

bool valid_level(henry_handle* h, int level) { return h && level >= 0 && level <= h->cfg.max_level; }
// ---------------------------------------------------------------------------
// Discrete adjoint (henry_adjoint).  The forward solve keeps the states the
// predictor of the next step reads - (x_n, x_{n-1}), and x_{n-2} with the
// quadratic predictor - every `ckpt` steps, and the states of the last
// segment; the backward sweep visits the segments from the last, recomputes
// each segment's states from its checkpoint (the same kernels and inputs, so
// the same states), and for every step from the last to the first assembles
// the Jacobian at (x_m, x_{m-1}), builds the coarse operators, transposes the
// whole multigrid hierarchy in place, solves J_m^T lam_m = rhs with the same
// BiCGStab and V-cycle, and accumulates the sensitivities (henry_adjoint.cuh).
size_t adjoint_bytes_per_sample(const henry_config& c, int level, int ckpt) {
  const LevelGeom lg = geom(c, level);
  const size_t N = (size_t)lg.nx * lg.ny;
  const size_t nck = (size_t)((lg.steps + ckpt - 1) / ckpt);
  const size_t cw = c.newton_predictor_order == 2 ? 3 : 2;  // states per checkpoint
  return (cw * nck + (size_t)ckpt + 1) * N * sizeof(double2) + (size_t)A_NPLANE * N * sizeof(double);
}

int ensure_adj_mem(henry_handle* H, size_t bytes) {
  if (H->adj_bytes >= bytes) return HENRY_OK;
  if (H->adj_mem) {
    CK(cudaDeviceSynchronize());
    CK(cudaFree(H->adj_mem));
    H->adj_mem = nullptr;
    H->adj_bytes = 0;
  }
  if (cudaMalloc(&H->adj_mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    H->adj_mem = nullptr;
    return set_err(HENRY_ENOMEM, "cudaMalloc of %zu bytes for the adjoint's checkpoints failed", bytes);
  }
  H->adj_bytes = bytes;
  return HENRY_OK;
}

int adjoint_group(henry_handle* H, Group<double>& G, int B, const double* xi, const double* w, double* grad,
                  double* qoi, int C, cudaStream_t st) {
  typedef VT<double>::b4 B4;
  const henry_config& c = H->cfg;
  const LevelGeom lg = geom(c, G.level);
  const Phys ph = phys_of(c);
  Level& L = G.lv[0];
  const int N = L.N;
  const int64_t n0 = (int64_t)B * N;
  const size_t vbytes = sizeof(double2) * (size_t)n0;
  const double inv_tau = 1.0 / lg.tau;
  const double inv_s = 1.0 / (c.rho0 * lg.h * lg.h * inv_tau);
  const double vt = lg.h * lg.h * inv_tau * inv_s;
  const int steps = lg.steps;
  const int nck = (steps + C - 1) / C;
  const int cw = c.newton_predictor_order == 2 ? 3 : 2;  // states per checkpoint
  Carver cv{H->adj_mem, 0};
  double2* ck = cv.take<double2>(vbytes * cw * nck);  // [nck][x_n, x_{n-1} (, x_{n-2})][B N]
  double2* seg = cv.take<double2>(vbytes * C);       // [C][B N]: states of one segment
  double2* rhs = cv.take<double2>(vbytes);
  double* S = cv.take<double>(sizeof(double) * A_NPLANE * (size_t)n0);
  double* pmax = G.part + P_MAX * (int64_t)B * G.nct;
  // forward, with checkpoints
  CK(cudaMemsetAsync(G.totals, 0, 4 * sizeof(unsigned long long), st));
  H->nact = B;
  k_init_state<<<nblk(n0), TPB, 0, st>>>(B, L.nx, L.ny, lg.h, c.rho0 * c.g, c.Ly, L.x);
  CKL();
  CK(cudaMemcpyAsync(L.xo, L.x, vbytes, cudaMemcpyDeviceToDevice, st));
  for (int step = 0; step < steps; ++step) {
    if (step % C == 0) {
      CK(cudaMemcpyAsync(ck + (int64_t)(cw * (step / C)) * n0, L.x, vbytes, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(ck + (int64_t)(cw * (step / C) + 1) * n0, L.xo, vbytes, cudaMemcpyDeviceToDevice, st));
      if (cw == 3)
        CK(cudaMemcpyAsync(ck + (int64_t)(cw * (step / C) + 2) * n0, G.xoo, vbytes, cudaMemcpyDeviceToDevice, st));
    }
    int rc = implicit_step<double>(H, G, B, step, st);
    if (rc) return rc;
    record_series(H, G.level, step, B, N, lg.h, L.x, qoi, G.status, st);
    CK(cudaMemcpyAsync(seg + (int64_t)(step % C) * n0, L.x, vbytes, cudaMemcpyDeviceToDevice, st));
  }
  k_qoi<<<B, TPB, 0, st>>>(B, L.nx, L.ny, lg.h, c.rho0, c.rho1 - c.rho0, G.coef, L.x, qoi, L.cc,
                             qoi_spec(c));
  CKL();
  // backward
  k_step_flags<<<nblk(B, 128), 128, 0, st>>>(B, G.status, G.lin_active, G.newton_it);
  k_adj_start<<<nblk(n0), TPB, 0, st>>>(B, L.nx, L.ny, lg.h, c.rho0, c.rho1 - c.rho0, G.coef, L.cc, w, L.x, rhs, S,
                                         G.lin_active);
  CKL();
  for (int k = nck - 1; k >= 0; --k) {
    const int s0 = k * C, s1 = std::min(s0 + C, steps);
    if (k != nck - 1) {  // recompute the segment's states from its checkpoint
      CK(cudaMemcpyAsync(L.x, ck + (int64_t)(cw * k) * n0, vbytes, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(L.xo, ck + (int64_t)(cw * k + 1) * n0, vbytes, cudaMemcpyDeviceToDevice, st));
      if (cw == 3) CK(cudaMemcpyAsync(G.xoo, ck + (int64_t)(cw * k + 2) * n0, vbytes, cudaMemcpyDeviceToDevice, st));
      for (int step = s0; step < s1; ++step) {
        int rc = implicit_step<double>(H, G, B, step, st);
        if (rc) return rc;
        CK(cudaMemcpyAsync(seg + (int64_t)(step - s0) * n0, L.x, vbytes, cudaMemcpyDeviceToDevice, st));
      }
    }
    for (int step = s1 - 1; step >= s0; --step) {  // state m = step + 1
      const double2* xm = seg + (int64_t)(step - s0) * n0;
      const double2* xm1 = step == s0 ? ck + (int64_t)(cw * k) * n0 : seg + (int64_t)(step - s0 - 1) * n0;
      CK(cudaMemcpyAsync(L.x, xm, vbytes, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(L.xo, xm1, vbytes, cudaMemcpyDeviceToDevice, st));
      k_step_flags<<<nblk(B, 128), 128, 0, st>>>(B, G.status, G.lin_active, G.newton_it);
      CKL();
      H->nact = B;
      launch(H, st, HENRY_K_ASSEMBLE, (double)n0 * (48.0 + 6.0 * sizeof(B4)), [&] {
        if (L.cc)
          assemble_kernel<double, true, true>(H->cfg, L.nx, L.ny)<<<nblk(n0), TPB, 0, st>>>(ph, G.coef, B, L.nx, L.ny, lg.h, 1.0 / lg.h, vt,
                                                                  inv_s, L.x, L.xo, G.lin_active, G.F, (B4*)L.J,
                                                                  L.plane, pmax, L.cc, L.fc);
        else
          assemble_kernel<double, true>(H->cfg, L.nx, L.ny)<<<nblk(n0), TPB, 0, st>>>(ph, G.coef, B, L.nx, L.ny, lg.h, 1.0 / lg.h, vt, inv_s,
                                                            L.x, L.xo, G.lin_active, G.F, (B4*)L.J, L.plane, pmax, nullptr, nullptr);
      });
      CKL();
      int rc;
      if (c.coarse_op == HENRY_COARSE_REDISCRETISE) {
        rc = restrict_states<double>(H, G, B, true, G.lin_active, st);
        if (rc) return rc;
        rc = restrict_states<double>(H, G, B, false, G.lin_active, st);
        if (rc) return rc;
      }
      rc = build_coarse_ops<double>(H, G, B, inv_tau, inv_s, st);
      if (rc) return rc;
      for (int kk = 0; kk <= G.K; ++kk) {
        Level& Lk = G.lv[kk];
        k_transpose_blocks<double><<<nblk((int64_t)B * Lk.N), TPB, 0, st>>>(B, Lk.nx, Lk.ny, (B4*)Lk.J, Lk.plane,
                                                                            G.lin_active);
      }
      Level& Lc = G.lv[G.K];
      k_coarse_inverse<double><<<nblk(B, 64), 64, 0, st>>>(B, (const B4*)Lc.J, Lc.plane, G.Ainv, G.lin_active);
      k_adj_neg<<<nblk(n0), TPB, 0, st>>>(n0, rhs, G.F);
      CKL();
      rc = linear_solve<double>(H, G, B, st, nullptr, c.adj_rtol, c.adj_maxit);
      if (rc) return rc;
      k_adj_lin_status<<<nblk(B, 128), 128, 0, st>>>(B, G.iters, G.status, G.lin_active);
      k_adj_step<<<nblk(n0), TPB, 0, st>>>(ph, G.coef, B, L.nx, L.ny, lg.h, 1.0 / lg.h, vt, inv_s, L.x, L.xo, G.dx,
                                          L.cc, S, rhs, G.lin_active);
      CKL();
    }
  }
  k_adj_cell_grad<<<nblk(n0), TPB, 0, st>>>(B, L.nx, L.ny, c.mu, c.Dm, G.coef, L.cc, S, G.r, G.lin_active);
  CKL();
  AdjModel M;
  std::memset(&M, 0, sizeof M);
  M.model = c.coef_model == HENRY_MODEL_KL ? 1 : (c.coef_model == HENRY_MODEL_TWO_LAYER ? 2 : 0);
  M.n_in = n_inputs(c);
  M.terms = c.kl_terms;
  M.phi_mean = c.phi_mean; M.phi_amp = c.phi_amp; M.K_mean = c.K_mean; M.logK_amp = c.logK_amp;
  M.qin_mean = c.qin_mean; M.qin_amp = c.qin_amp; M.mu = c.mu;
  M.sigma_logK = c.kl_sigma_logK; M.sigma_phi = c.kl_sigma_phi; M.phi_lo = c.phi_lo; M.phi_hi = c.phi_hi;
  M.kappa = c.K_mean * (1.0 - c.phi_mean * c.phi_mean) / (c.phi_mean * c.phi_mean * c.phi_mean);
  M.Ly = c.Ly; M.y_if = -0.75; M.h = lg.h;
  const int *ti = nullptr, *tj = nullptr;
  const double *sl = nullptr, *psx = nullptr, *psy = nullptr;
  if (M.model == 1) {
    KLTables* t = nullptr;
    int rc = ensure_kl_tables(H, G.level, &t);
    if (rc) return rc;
    ti = t->ti; tj = t->tj; sl = t->sl; psx = t->psx; psy = t->psy;
  }
  k_adj_project<<<B, TPB, 0, st>>>(M, B, L.nx, L.ny, G.coef, L.cc, G.r, S, ti, tj, sl, psx, psy, xi, grad,
                                   G.lin_active);
  CKL();
  return HENRY_OK;
}

int adjoint_level(henry_handle* H, int level, const double* xi, int n, const double* w, double* grad, double* qoi,
                  int ckpt, int32_t* status, cudaStream_t st) {
  const henry_config& c = H->cfg;
  const LevelGeom lg = geom(c, level);
  const int C = std::max(1, std::min(ckpt, lg.steps));
  const double per = (double)bytes_per_sample<double>(c, level, false) + (double)adjoint_bytes_per_sample(c, level, C);
  const int Bmax = (int)std::max(1.0, std::min(std::floor(c.workspace_bytes / per), 1.0e6));
  const int Bcap = std::min(Bmax, n);
  const int nin = n_inputs(c);
  int rc = ensure_adj_mem(H, adjoint_bytes_per_sample(c, level, C) * (size_t)Bcap + 8 * 256);
  if (rc) return rc;
  for (int off = 0; off < n; off += Bmax) {
    const int B = std::min(Bmax, n - off);
    Group<double>* G = nullptr;
    rc = get_group<double>(H, level, Bcap, &G);
    if (rc) return rc;
    rc = set_coefficients<double>(H, *G, xi + (int64_t)nin * off, B, st);
    if (rc) return rc;
    rc = adjoint_group(H, *G, B, xi + (int64_t)nin * off, w + 2 * (int64_t)off, grad + (int64_t)nin * off,
                       qoi + qoi_count(c) * (int64_t)off, C, st);
    if (rc) return rc;
    k_merge_status<<<nblk(B, 128), 128, 0, st>>>(B, G->status, status + off, 1);
    CKL();
  }
  return HENRY_OK;
}



template <typename T>
int step_entry(henry_handle* H, int which, int level, const double* xi, int n, const double* state,
               const double* state_old, const double* in, double* out, double* out2, int32_t* iters,
               cudaStream_t st) {
  typedef typename VT<T>::v2 V2;
  typedef typename VT<T>::b4 B4;
  Group<T>* G = nullptr;
  int rc = setup_from_states<T>(H, level, xi, n, state, state_old, &G, st);
  if (rc) return rc;
  Level& L = G->lv[0];
  const int64_t n0 = (int64_t)n * L.N;
  rc = assemble_all<T>(H, *G, n, which >= 2, st, which != 0 || out2 != nullptr);
  if (rc) return rc;
  switch (which) {
    case 0:  // assemble
      k_from_storage<double2><<<nblk(n0), TPB, 0, st>>>(n, L.nx, L.ny, G->F, (double2*)out);
      if (out2) k_blocks_out<B4><<<nblk(n0), TPB, 0, st>>>(n, L.nx, L.ny, (const B4*)L.J, L.plane, out2);
      break;
    case 1:  // apply
      k_to_storage<V2><<<nblk(n0), TPB, 0, st>>>(n, L.nx, L.ny, (const double2*)in, G->p);
      k_spmv<T, 0><<<nblk(n0), TPB, 0, st>>>(n, L.nx, L.ny, (const B4*)L.J, L.plane, G->p, G->v, nullptr, nullptr,
                                             0, 0, G->lin_active);
      k_from_storage<V2><<<nblk(n0), TPB, 0, st>>>(n, L.nx, L.ny, G->v, (double2*)out);
      break;
    case 2:  // precondition
      k_to_storage<V2><<<nblk(n0), TPB, 0, st>>>(n, L.nx, L.ny, (const double2*)in, G->p);
      CKL();
      rc = vcycle<T>(H, *G, n, G->p, G->ph, st);
      if (rc) return rc;
      k_from_storage<V2><<<nblk(n0), TPB, 0, st>>>(n, L.nx, L.ny, G->ph, (double2*)out);
      break;
    case 3:  // linear solve: F := -b, BiCGStab, dx out
      k_to_storage<double2><<<nblk(n0), TPB, 0, st>>>(n, L.nx, L.ny, (const double2*)in, G->F);
      k_scale_d2<<<nblk(n0), TPB, 0, st>>>(n0, -1.0, G->F);
      CKL();
      CK(cudaMemsetAsync(G->totals, 0, 4 * sizeof(unsigned long long), st));
      rc = linear_solve<T>(H, *G, n, st);
      if (rc) return rc;
      k_from_storage<V2><<<nblk(n0), TPB, 0, st>>>(n, L.nx, L.ny, G->dx, (double2*)out);
      if (iters) CK(cudaMemcpyAsync(iters, G->iters, sizeof(int) * n, cudaMemcpyDeviceToDevice, st));
      break;
  }
  CKL();
  return HENRY_OK;
}

// Vertex-centred assembly (henry_vc.cuh): one thread per (sample, vertex);
// states, residuals and Jacobian rows in the natural vertex order.
__global__ void __launch_bounds__(TPB) k_vc_assemble(VcParams P, int B, const Coef* __restrict__ coef,
                                                     const double* __restrict__ x, const double* __restrict__ xo,
                                                     double* __restrict__ R, double* __restrict__ J) {
  const int64_t nv = (int64_t)(P.nx + 1) * (P.ny + 1);
  const int64_t t = (int64_t)blockIdx.x * TPB + threadIdx.x;
  if (t >= (int64_t)B * nv) return;
  const int64_t s = t / nv;
  const int v = (int)(t - s * nv);
  const int j = v / (P.nx + 1), i = v - j * (P.nx + 1);
  const Coef cf = coef[s];
  const VcCoef c{cf.phi, cf.kmu, cf.PD, cf.qin};
  vc_vertex(P, c, x + 2 * s * nv, xo + 2 * s * nv, j, i, R + 2 * t, J ? J + 36 * t : nullptr);
}

int check_step_args(henry_handle* h, int level, const double* xi, int n, const double* state,
                    const double* state_old) {
  if (!h) return set_err(HENRY_EINVAL, "handle is NULL");
  if (!valid_level(h, level)) return set_err(HENRY_EINVAL, "level %d outside [0, %d]", level, h->cfg.max_level);
  if (n <= 0) return set_err(HENRY_EINVAL, "n = %d must be positive", n);
  if (!xi || !state || !state_old) return set_err(HENRY_EINVAL, "NULL input pointer");
  return HENRY_OK;
}

// Configuration checks shared by henry_create and the allocation-free entry
// point (which has no workspace_bytes budget: with_workspace false).
bool valid_tile_w(int w) { return w == 0 || w == 32 || w == 64 || w == 128 || w == 256; }
bool valid_mg_threads(int n) { return n == 0 || n == 64 || n == 128 || n == 256 || n == 512; }

int check_config(const henry_config& c, bool with_workspace) {
  // every floating-point setting finite (a NaN would pass the comparisons below)
  const double reals[] = {c.Lx, c.Ly, c.T, c.rho0, c.rho1, c.mu, c.g, c.Dm, c.phi_mean, c.K_mean, c.qin_mean,
                          c.phi_amp, c.logK_amp, c.qin_amp, c.newton_atol, c.newton_dxtol, c.lin_rtol,
                          c.newton_predictor, c.newton_dc_limit, c.kl_corr_len, c.kl_sigma_logK, c.kl_sigma_phi,
                          c.phi_lo, c.phi_hi, c.adj_rtol};
  for (double v : reals)
    if (!std::isfinite(v)) return set_err(HENRY_EINVAL, "a floating-point setting is NaN or infinite");
  if (with_workspace && !std::isfinite(c.workspace_bytes))
    return set_err(HENRY_EINVAL, "workspace_bytes is NaN or infinite");
  if (!(c.rho0 > 0) || !(c.rho1 > 0) || !(c.mu > 0) || !(c.g > 0) || !(c.Dm > 0) || !(c.K_mean > 0) ||
      !(c.phi_mean > 0 && c.phi_mean < 1) || !(c.newton_atol >= 0) || !(c.newton_dxtol >= 0))
    return set_err(HENRY_EINVAL, "physical constants must be positive (0 < phi_mean < 1), tolerances >= 0");
  if (c.ny0 < 4 || (c.ny0 & (c.ny0 - 1)) != 0 || (int64_t)c.nx0 != 2 * (int64_t)c.ny0)
    return set_err(HENRY_EINVAL, "grid must be nx0 = 2 ny0 with ny0 a power of two >= 4 (got %d x %d)", c.nx0, c.ny0);
  if (std::fabs(c.Lx - 2.0 * c.Ly) > 1e-12 * c.Lx || c.Ly <= 0)
    return set_err(HENRY_EINVAL, "domain must be Lx = 2 Ly (square cells)");
  if (c.max_level < 0 || c.max_level > 8) return set_err(HENRY_EINVAL, "max_level %d outside [0, 8]", c.max_level);
  const int64_t finest_cells = ((int64_t)c.nx0 << c.max_level) * ((int64_t)c.ny0 << c.max_level);
  if (finest_cells > ((int64_t)1 << 30) || c.steps0 > ((1 << 30) >> c.max_level))
    return set_err(HENRY_EINVAL,
                   "finest level too large (%lld cells, %d steps at level 0; limits 2^30 cells and 2^30 steps at "
                   "max_level)",
                   (long long)finest_cells, c.steps0);
  if (finest_cells % TPB != 0 || (int64_t)c.nx0 * c.ny0 < TPB)
    return set_err(HENRY_EINVAL, "cells per sample must be a multiple of %d", TPB);
  if (c.precision != HENRY_FP64 && c.precision != HENRY_MIXED) return set_err(HENRY_EINVAL, "bad precision");
  if (c.coarse_op != HENRY_COARSE_REDISCRETISE && c.coarse_op != HENRY_COARSE_GALERKIN)
    return set_err(HENRY_EINVAL, "bad coarse_op");
  if (c.coef_model < HENRY_MODEL_UNIFORM3 || c.coef_model > HENRY_MODEL_TWO_LAYER)
    return set_err(HENRY_EINVAL, "bad coef_model");
  if (c.qoi_set < HENRY_QOI_STANDARD || c.qoi_set > HENRY_QOI_PAPER_SERIES) return set_err(HENRY_EINVAL, "bad qoi_set");
  if (c.scheme != HENRY_SCHEME_CELL && c.scheme != HENRY_SCHEME_VERTEX) return set_err(HENRY_EINVAL, "bad scheme");
  if (c.scheme == HENRY_SCHEME_VERTEX && (c.coef_model != HENRY_MODEL_UNIFORM3 || c.qoi_set != HENRY_QOI_STANDARD))
    return set_err(HENRY_EINVAL,
                   "the vertex-centred scheme solves the three-parameter model with the two standard QoIs");
  if (c.coef_model == HENRY_MODEL_KL &&
      (c.kl_terms < 1 || c.kl_terms > 256 || !(c.kl_corr_len > 0) || !(c.phi_lo > 0) || !(c.phi_hi < 1) ||
       !(c.phi_lo < c.phi_hi)))
    return set_err(HENRY_EINVAL, "bad random-field settings");
  if (c.steps0 <= 0 || c.T <= 0 || c.newton_maxit <= 0 || c.lin_maxit <= 0 || c.nu1 < 0 || c.nu2 < 0 ||
      c.lin_rtol <= 0 || (with_workspace && c.workspace_bytes <= 0) ||
      !(c.newton_predictor >= 0.0 && c.newton_predictor <= 1.0) || !(c.newton_dc_limit >= 0.0) ||
      c.newton_jacobian_every < 1)
    return set_err(HENRY_EINVAL, "bad solver settings");
  if (!valid_tile_w(c.assembly_tile_w)) return set_err(HENRY_EINVAL, "assembly_tile_w %d not in {0, 32, 64, 128, 256}",
                                                       c.assembly_tile_w);
  if (!valid_mg_threads(c.mg_threads))
    return set_err(HENRY_EINVAL, "mg_threads %d not in {0, 64, 128, 256, 512}", c.mg_threads);
  if (c.newton_predictor_order != 1 && c.newton_predictor_order != 2)
    return set_err(HENRY_EINVAL, "newton_predictor_order %d not in {1, 2}", c.newton_predictor_order);
  return HENRY_OK;
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

void henry_default_config(henry_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof *c);
  c->Lx = 2.0; c->Ly = 1.0; c->T = 7200.0;
  c->rho0 = 1000.0; c->rho1 = 1025.0; c->mu = 1e-3; c->g = 9.81; c->Dm = 1.886e-5;
  c->phi_mean = 0.35; c->K_mean = 1.02e-9; c->qin_mean = 6.6e-5;
  c->phi_amp = 0.2; c->logK_amp = 0.5; c->qin_amp = 0.2;
  c->nx0 = 32; c->ny0 = 16; c->steps0 = 20; c->max_level = 5;
  c->precision = HENRY_FP64;
  c->coarse_op = HENRY_COARSE_REDISCRETISE;
  c->newton_atol = 1e-11;
  c->newton_dxtol = 1e-12;
  c->lin_rtol = 1e-3;  // inexact Newton: the FP64 residual test decides convergence
  c->newton_maxit = 30;
  c->lin_maxit = 40;
  c->nu1 = 2; c->nu2 = 2;
  c->workspace_bytes = 16.0e9;
  c->newton_predictor = 1.0;
  c->newton_dc_limit = 1.0;
  c->lin_retry = 1;
  c->finalize_nct = 512;
  c->adj_rtol = 1e-10;
  c->cuda_graphs = 1;
  c->qoi_set = HENRY_QOI_STANDARD;
  c->tile_assembly = 1;
  c->newton_residual_first = 2;
  c->newton_jacobian_every = 1;
  c->level_priority = 1;
  c->mg_tail_cells = -1;
  c->mg_tail_batch_cells = 1 << 20;
  c->scheme = HENRY_SCHEME_CELL;
  c->assembly_tile_w = 0;
  c->mg_threads = 0;
  c->newton_predictor_order = 2;
  c->adj_maxit = 200;
  c->fused_small_grids = 1;
  c->coef_model = HENRY_MODEL_UNIFORM3;
  c->kl_terms = 32;
  c->kl_corr_len = 0.3;
  c->kl_sigma_logK = 0.5;
  c->kl_sigma_phi = 0.1;
  c->phi_lo = 0.05;
  c->phi_hi = 0.65;
}

void henry_paper_config(henry_config* c) {
  if (!c) return;
  henry_default_config(c);
  c->g = 9.8; c->rho1 = 1024.99; c->Dm = 18.8571e-6; c->K_mean = 1.020408e-9;
  c->qin_amp = 0.5;
  c->T = 6016.0;
  c->steps0 = 188;
  c->coef_model = HENRY_MODEL_TWO_LAYER;
  c->qoi_set = HENRY_QOI_PAPER;
}

int henry_set_tuning(henry_handle* h, int level, const henry_tuning* t) {
  if (!h) return set_err(HENRY_EINVAL, "NULL handle");
  if (!valid_level(h, level)) return set_err(HENRY_EINVAL, "level %d outside [0, %d]", level, h->cfg.max_level);
  if (!t) {
    h->tuned.erase(level);
    return HENRY_OK;
  }
  if (!(t->lin_rtol > 0.0) || t->nu1 < 0 || t->nu2 < 0 || t->nu1 + t->nu2 == 0 || t->mg_tail_cells < -1 ||
      t->newton_jacobian_every < 1 || !valid_tile_w(t->assembly_tile_w) || !valid_mg_threads(t->mg_threads) ||
      t->newton_predictor_order < 0 || t->newton_predictor_order > 2)
    return set_err(HENRY_EINVAL, "bad tuning (lin_rtol %g, nu1 %d, nu2 %d, mg_tail_cells %d)", t->lin_rtol, t->nu1,
                   t->nu2, t->mg_tail_cells);
  h->tuned[level] = *t;
  return HENRY_OK;
}

int henry_get_tuning(henry_handle* h, int level, henry_tuning* out) {
  if (!h || !out) return set_err(HENRY_EINVAL, "NULL argument");
  if (!valid_level(h, level)) return set_err(HENRY_EINVAL, "level %d outside [0, %d]", level, h->cfg.max_level);
  auto f = h->tuned.find(level);
  if (f != h->tuned.end()) {
    *out = f->second;
  } else {
    std::memset(out, 0, sizeof *out);
    out->lin_rtol = h->cfg.lin_rtol;
    out->nu1 = h->cfg.nu1;
    out->nu2 = h->cfg.nu2;
    out->fused_small_grids = h->cfg.fused_small_grids;
    out->mg_tail_cells = h->cfg.mg_tail_cells;
    out->newton_residual_first = h->cfg.newton_residual_first;
    out->newton_jacobian_every = h->cfg.newton_jacobian_every;
    out->assembly_tile_w = h->cfg.assembly_tile_w;
    out->mg_threads = h->cfg.mg_threads;
    out->newton_predictor_order = h->cfg.newton_predictor_order;
  }
  return HENRY_OK;
}

int henry_autotune(henry_handle* h, int level, int with_coarse, const double* xi_dev, int n_trial,
                   henry_tuning* best_out, void* stream) {
  if (!h || !xi_dev) return set_err(HENRY_EINVAL, "NULL argument");
  if (!valid_level(h, level)) return set_err(HENRY_EINVAL, "level %d outside [0, %d]", level, h->cfg.max_level);
  if (n_trial <= 0) return set_err(HENRY_EINVAL, "n_trial = %d must be positive", n_trial);
  if (with_coarse && level == 0) return set_err(HENRY_EINVAL, "level 0 has no coarse partner");
  cudaStream_t st = (cudaStream_t)stream;
  const henry_config& c = h->cfg;
  const int nq = qoi_count(c);
  char* mem = nullptr;
  const size_t qbytes = sizeof(double) * (size_t)n_trial * nq;
  if (cudaMalloc(&mem, 2 * qbytes + sizeof(int32_t) * (size_t)n_trial) != cudaSuccess) {
    cudaGetLastError();
    return set_err(HENRY_ENOMEM, "cudaMalloc for the autotuner's trial outputs failed");
  }
  double* qf = (double*)mem;
  double* qc = (double*)(mem + qbytes);
  int32_t* sd = (int32_t*)(mem + 2 * qbytes);
  std::vector<henry_tuning> cands;
  const double rts[3] = {1e-4, 1e-3, 1e-2};
  const int nus[3][2] = {{2, 2}, {1, 2}, {2, 1}};
  CtaLayout CL;
  const bool can_fuse = (c.precision == HENRY_MIXED ? fused_eligible<float>(c, level, &CL)
                                                    : fused_eligible<double>(c, level, &CL)) ||
                        (c.fused_small_grids == 0);
  for (double rt : rts)
    for (auto& nu : nus)
      for (int fz = 0; fz < 2; ++fz) {
        if (fz == 1 && !can_fuse) continue;
        henry_tuning t;
        std::memset(&t, 0, sizeof t);
        t.lin_rtol = rt;
        t.nu1 = nu[0];
        t.nu2 = nu[1];
        t.fused_small_grids = can_fuse ? (fz == 0 ? 0 : 1) : c.fused_small_grids;
        t.mg_tail_cells = c.mg_tail_cells;
        t.newton_residual_first = c.newton_residual_first;
        t.newton_jacobian_every = c.newton_jacobian_every;
        t.assembly_tile_w = c.assembly_tile_w;
        t.mg_threads = c.mg_threads;
        t.newton_predictor_order = c.newton_predictor_order;
        cands.push_back(t);
      }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = HENRY_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    rc = set_err(HENRY_ECUDA, "cudaEventCreate for the autotuner's timing failed");
  }
  const LevelGeom lg = geom(c, level);
  double cs = (double)n_trial * lg.nx * lg.ny * lg.steps;
  if (with_coarse) {
    const LevelGeom lc = geom(c, level - 1);
    cs += (double)n_trial * lc.nx * lc.ny * lc.steps;
  }
  // a failed run leaves the level's settings as they were
  const auto prior = h->tuned.find(level);
  const bool had_prior = prior != h->tuned.end();
  const henry_tuning prior_t = had_prior ? prior->second : henry_tuning{};
  h->tuned.erase(level);
  int best = -1;
  double best_rate = 0.0;
  // Times candidate i (i = -1: the untimed warm-up that sets up workspaces
  // and graphs); keeps the fastest that solves every sample.
  auto trial = [&](int i) {
    if (i >= 0) h->tuned[level] = cands[i];
    cudaEventRecord(e0, st);
    rc = henry_level_batch_solve(h, level, with_coarse, xi_dev, n_trial, qf, with_coarse ? qc : nullptr, sd, nullptr,
                                 st);
    cudaEventRecord(e1, st);
    if (rc == HENRY_ENOCONV) {  // a candidate that loses samples is not a candidate
      rc = HENRY_OK;
      return;
    }
    if (rc) return;
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (i >= 0 && ms > 0.f) {
      cands[i].cell_steps_per_s = cs / (ms * 1e-3);
      if (cands[i].cell_steps_per_s > best_rate) {
        best_rate = cands[i].cell_steps_per_s;
        best = i;
      }
    }
  };
  // Stage 1: Krylov tolerance x smoothing counts x fused small-grid solver.
  const int n1 = (int)cands.size();
  for (int i = -1; i < n1 && !rc; ++i) trial(i);
  // Stages 2 and 3, one setting at a time from the best so far: the fused
  // multigrid tail (off, from 16 x 8, from 32 x 16 cells) and the
  // residual-first Newton test (never, from iteration 1, from 2).
  // (not when the fused small-grid solver won: it has its own in-kernel V-cycle and Newton loop)
  bool fused_won = false;
  if (best >= 0) {
    henry_config cb = c;
    cb.fused_small_grids = cands[best].fused_small_grids;
    fused_won = c.precision == HENRY_MIXED ? fused_eligible<float>(cb, level, &CL) : fused_eligible<double>(cb, level, &CL);
  }
  const bool cc = c.scheme == HENRY_SCHEME_CELL;  // the tail, tile and CTA-size stages are the cell scheme's
  if (!rc && best >= 0 && !fused_won) {
    const int tails[5] = {0, 32, 128, 512, 2048};
    for (int v : tails) {
      if (!cc) break;
      if (v == cands[best].mg_tail_cells || rc) continue;
      henry_tuning t = cands[best];
      t.mg_tail_cells = v;
      cands.push_back(t);
      trial((int)cands.size() - 1);
    }
    const int rfs[4] = {-1, 2, 3, 4};
    const int b2 = best;
    for (int v : rfs) {
      if (v == cands[b2].newton_residual_first || rc) continue;
      henry_tuning t = cands[b2];
      t.newton_residual_first = v;
      cands.push_back(t);
      trial((int)cands.size() - 1);
    }
    {  // chord Newton: the Jacobian every 1, 2 or 3 iterations
      const int b3 = best;
      for (int v : {1, 2, 3}) {
        if (v == cands[b3].newton_jacobian_every || rc) continue;
        henry_tuning t = cands[b3];
        t.newton_jacobian_every = v;
        cands.push_back(t);
        trial((int)cands.size() - 1);
      }
    }
    if (!rc) {  // the predictor of Newton's first iterate: linear or quadratic in time
      const int b6 = best;
      henry_tuning t = cands[b6];
      t.newton_predictor_order = cands[b6].newton_predictor_order == 2 ? 1 : 2;
      cands.push_back(t);
      trial((int)cands.size() - 1);
    }
  }
  if (!rc && best >= 0 && !fused_won && cc && c.tile_assembly) {
    // Stage 5: the assembly tile (whole rows / 128 x 2 by default, or
    // w x 256 / w tiles), where the level's fine grid takes that tile.
    const int b4 = best;
    for (int v : {0, 32, 64, 128, 256}) {
      if (v == cands[b4].assembly_tile_w || rc) continue;
      if (v > 0 && (lg.nx % v != 0 || lg.ny % (TPB / v) != 0)) continue;
      henry_tuning t = cands[b4];
      t.assembly_tile_w = v;
      cands.push_back(t);
      trial((int)cands.size() - 1);
    }
  }
  if (!rc && best >= 0 && !fused_won && cc) {
    // Stage 6: the CTA size of the smoother, restriction and prolongation
    // kernels (small batches of mid-size grids fill more SMs with smaller CTAs).
    const int b5 = best;
    for (int v : {64, 128, 256, 512}) {
      const int cur = cands[b5].mg_threads == 0 ? TPB : cands[b5].mg_threads;
      if (v == cur || rc) continue;
      henry_tuning t = cands[b5];
      t.mg_threads = v;
      cands.push_back(t);
      trial((int)cands.size() - 1);
    }
  }
  h->tuned.erase(level);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(mem);
  if (rc || best < 0) {
    if (had_prior) h->tuned[level] = prior_t;
    return rc ? rc : set_err(HENRY_ENOCONV, "no candidate solved every trial sample");
  }
  h->tuned[level] = cands[best];
  if (best_out) *best_out = cands[best];
  return HENRY_OK;
}

int henry_kl_basis(const henry_config* cfg, int level, double* sqrt_lam, double* modes) {
  if (!cfg || !sqrt_lam) return set_err(HENRY_EINVAL, "NULL argument");
  const henry_config& c = *cfg;
  if (level < 0 || level > c.max_level) return set_err(HENRY_EINVAL, "level %d outside [0, %d]", level, c.max_level);
  if (c.kl_terms < 1 || c.kl_terms > 256 || !(c.kl_corr_len > 0) || !(c.Lx > 0) || !(c.Ly > 0) || c.nx0 <= 0 ||
      c.ny0 <= 0)
    return set_err(HENRY_EINVAL, "bad random-field settings");
  hkl::Basis2D b;
  b.build(c.Lx, c.Ly, c.kl_terms, c.kl_corr_len);
  for (int t = 0; t < b.terms; ++t) sqrt_lam[t] = b.sqrt_lam[t];
  if (modes) {
    const LevelGeom lg = geom(c, level);
    std::vector<double> px((size_t)b.bx.m * lg.nx), py((size_t)b.by.m * lg.ny);
    for (int i = 0; i < b.bx.m; ++i)
      for (int ix = 0; ix < lg.nx; ++ix) px[(size_t)i * lg.nx + ix] = b.bx.eval(i, (ix + 0.5) * lg.h);
    for (int j = 0; j < b.by.m; ++j)
      for (int iy = 0; iy < lg.ny; ++iy) py[(size_t)j * lg.ny + iy] = b.by.eval(j, (iy + 0.5) * lg.h);
    for (int t = 0; t < b.terms; ++t)
      for (int iy = 0; iy < lg.ny; ++iy)
        for (int ix = 0; ix < lg.nx; ++ix)
          modes[((size_t)t * lg.ny + iy) * lg.nx + ix] =
              py[(size_t)b.tj[t] * lg.ny + iy] * px[(size_t)b.ti[t] * lg.nx + ix];
  }
  return HENRY_OK;
}

int henry_n_qoi(const henry_config* c) {
  if (!c) return -set_err(HENRY_EINVAL, "NULL argument");
  if (c->qoi_set < HENRY_QOI_STANDARD || c->qoi_set > HENRY_QOI_PAPER_SERIES)
    return -set_err(HENRY_EINVAL, "bad qoi_set");
  return qoi_count(*c);
}

int henry_create(const henry_config* cfg, henry_handle** out) {
  if (!cfg || !out) return set_err(HENRY_EINVAL, "NULL argument");
  *out = nullptr;
  const henry_config& c = *cfg;
  const int rc = check_config(c, true);
  if (rc) return rc;
  henry_handle* h = new henry_handle();
  h->cfg = c;
  *out = h;
  return HENRY_OK;
}

void henry_destroy(henry_handle* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  for (auto& kv : h->kids) henry_destroy(kv.second);
  for (auto& kv : h->kid_streams) cudaStreamDestroy(kv.second);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->perm_mem) cudaFree(h->perm_mem);
  if (h->adj_mem) cudaFree(h->adj_mem);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (auto& p : h->prof.pend) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : h->prof.pool) cudaEventDestroy(e);
  for (auto& kv : h->g64) {
    kv.second.drop_graphs();
    if (kv.second.mem) cudaFree(kv.second.mem);
  }
  for (auto& kv : h->g32) {
    kv.second.drop_graphs();
    if (kv.second.mem) cudaFree(kv.second.mem);
  }
  for (auto& kv : h->vg64) {
    kv.second.drop_graphs();
    if (kv.second.mem) cudaFree(kv.second.mem);
  }
  for (auto& kv : h->vg32) {
    kv.second.drop_graphs();
    if (kv.second.mem) cudaFree(kv.second.mem);
  }
  for (auto& kv : h->kl_tables) {
    cudaFree(kv.second.ti);
    cudaFree(kv.second.tj);
    cudaFree(kv.second.sl);
    cudaFree(kv.second.psx);
    cudaFree(kv.second.psy);
  }
  delete h->kl;
  if (h->host_counter) cudaFreeHost(h->host_counter);
  if (h->host_totals) cudaFreeHost(h->host_totals);
  delete h;
}

const char* henry_last_error(void) { return g_err.c_str(); }

int henry_batch_solve_mixed(henry_handle* h, const int32_t* levels_host, int n, int with_coarse,
                            const double* xi_dev, double* qoi_fine_dev, double* qoi_coarse_dev, int32_t* status_dev,
                            henry_stats* stats_host, void* stream) {
  if (!h) return set_err(HENRY_EINVAL, "handle is NULL");
  if (n <= 0) return set_err(HENRY_EINVAL, "n = %d must be positive", n);
  if (!levels_host || !xi_dev || !qoi_fine_dev || !status_dev) return set_err(HENRY_EINVAL, "NULL pointer");
  if (with_coarse && !qoi_coarse_dev) return set_err(HENRY_EINVAL, "qoi_coarse_dev is NULL");
  const int NL = h->cfg.max_level + 1;
  std::vector<int> cnt(NL, 0), first(NL, 0);
  for (int i = 0; i < n; ++i) {
    if (!valid_level(h, levels_host[i]))
      return set_err(HENRY_EINVAL, "levels_host[%d] = %d outside [0, %d]", i, levels_host[i], h->cfg.max_level);
    ++cnt[levels_host[i]];
  }
  for (int l = 1; l < NL; ++l) first[l] = first[l - 1] + cnt[l - 1];
  // perm[j]: original index of the j-th sample in level order (stable)
  std::vector<int> perm(n), pos(first);
  bool sorted = true;
  for (int i = 0; i < n; ++i) {
    const int j = pos[levels_host[i]]++;
    perm[j] = i;
    sorted = sorted && j == i;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int nin = n_inputs(h->cfg);
  const int nq = qoi_count(h->cfg);
  const double* xs = xi_dev;
  double* qf = qoi_fine_dev;
  double* qc = qoi_coarse_dev;
  int32_t* ss = status_dev;
  int* perm_dev = nullptr;
  if (!sorted) {  // gather into level order; results are scattered back below
    auto carve = [&](int cap, char* base, int** pd, double** x, double** f, double** c, int32_t** sd) {
      size_t o = 0;
      auto take = [&](size_t b) {
        char* p = base ? base + o : nullptr;
        o += (b + 255) & ~(size_t)255;
        return p;
      };
      *pd = (int*)take(sizeof(int) * cap);
      *x = (double*)take(sizeof(double) * cap * nin);
      *f = (double*)take(sizeof(double) * cap * nq);
      *c = (double*)take(sizeof(double) * cap * nq);
      *sd = (int32_t*)take(sizeof(int32_t) * cap);
      return o;
    };
    int* pd;
    double *x, *f, *c;
    int32_t* sd;
    if (h->perm_cap < n) {
      if (h->perm_mem) {
        CK(cudaDeviceSynchronize());
        CK(cudaFree(h->perm_mem));
        h->perm_mem = nullptr;
        h->perm_cap = 0;
      }
      const size_t bytes = carve(n, nullptr, &pd, &x, &f, &c, &sd);
      if (cudaMalloc(&h->perm_mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        h->perm_mem = nullptr;
        return set_err(HENRY_ENOMEM, "cudaMalloc of %zu bytes for the level permutation failed", bytes);
      }
      h->perm_cap = n;
    }
    carve(h->perm_cap, h->perm_mem, &pd, &x, &f, &c, &sd);
    perm_dev = pd;
    CK(cudaMemcpyAsync(perm_dev, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    k_permute_rows<double, false><<<nblk((int64_t)n * nin), TPB, 0, st>>>(n, nin, perm_dev, xi_dev, x);
    CKL();
    xs = x;
    qf = f;
    qc = c;
    ss = sd;
  }
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (!h->ev_fork) CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  CK(cudaEventRecord(h->ev_fork, st));
  std::vector<int> act;
  for (int l = NL - 1; l >= 0; --l) {  // finest (longest) level first
    if (!cnt[l]) continue;
    if (!h->kids.count(l)) {
      henry_handle* k = nullptr;
      const int rc = henry_create(&h->cfg, &k);
      if (rc) return rc;
      h->kids[l] = k;
      // level_priority: finer levels (longer solves: the critical path of a
      // pass) get higher stream priorities, so their kernels are scheduled
      // first when the levels compete for SMs
      int least = 0, greatest = 0;
      CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
      const int prio = h->cfg.level_priority
                           ? std::max(greatest, least - (l * (least - greatest)) / std::max(1, h->cfg.max_level))
                           : least;
      cudaStream_t ls = nullptr;
      CK(cudaStreamCreateWithPriority(&ls, cudaStreamNonBlocking, prio));
      h->kid_streams[l] = ls;
    }
    henry_handle* k = h->kids[l];
    k->tuned = h->tuned;
    if (k->prof.on != h->prof.on) {
      const int rc = henry_profile(k, h->prof.on ? 1 : 0);
      if (rc) return rc;
    }
    CK(cudaStreamWaitEvent(h->kid_streams[l], h->ev_fork, 0));
    act.push_back(l);
  }
  std::vector<int> rcs(NL, HENRY_OK);
  std::vector<std::string> msg(NL);
  std::vector<henry_stats> sts(NL);
  std::vector<std::thread> ths;
  for (int l : act) {
    ths.emplace_back([&, l] {
      cudaSetDevice(dev);
      std::memset(&sts[l], 0, sizeof sts[l]);
      const int wc = (with_coarse && l > 0) ? 1 : 0;
      const int64_t o = first[l];
      rcs[l] = henry_level_batch_solve(h->kids[l], l, wc, xs + o * nin, cnt[l], qf + o * nq, wc ? qc + o * nq : nullptr,
                                       ss + o, &sts[l], h->kid_streams[l]);
      if (rcs[l] != HENRY_OK && rcs[l] != HENRY_ENOCONV) msg[l] = henry_last_error();
    });
  }
  for (auto& t : ths) t.join();
  // every level solve synchronised its own stream, so its results are in memory
  for (int l : act)
    if (rcs[l] != HENRY_OK && rcs[l] != HENRY_ENOCONV) return set_err(rcs[l], "level %d: %s", l, msg[l].c_str());
  if (with_coarse && cnt[0]) CK(cudaMemsetAsync(qc + (int64_t)first[0] * nq, 0, sizeof(double) * nq * cnt[0], st));
  if (!sorted) {
    k_permute_rows<double, true><<<nblk((int64_t)n * nq), TPB, 0, st>>>(n, nq, perm_dev, qf, qoi_fine_dev);
    CKL();
    if (with_coarse) {
      k_permute_rows<double, true><<<nblk((int64_t)n * nq), TPB, 0, st>>>(n, nq, perm_dev, qc, qoi_coarse_dev);
      CKL();
    }
    k_permute_rows<int32_t, true><<<nblk(n), TPB, 0, st>>>(n, 1, perm_dev, ss, status_dev);
    CKL();
  }
  CK(cudaStreamSynchronize(st));
  henry_stats tot;
  std::memset(&tot, 0, sizeof tot);
  for (int l : act) {
    tot.newton_iters += sts[l].newton_iters;
    tot.linear_iters += sts[l].linear_iters;
    tot.newton_solves += sts[l].newton_solves;
    tot.failed_samples += sts[l].failed_samples;
    tot.cell_steps += sts[l].cell_steps;
  }
  if (stats_host) *stats_host = tot;
  if (tot.failed_samples)
    return set_err(HENRY_ENOCONV, "%lld of %d samples did not converge", (long long)tot.failed_samples, n);
  return HENRY_OK;
}

int henry_profile(henry_handle* h, int enable) {
  if (!h) return set_err(HENRY_EINVAL, "handle is NULL");
  Prof& P = h->prof;
  if (!P.pend.empty()) {
    CK(cudaDeviceSynchronize());
    prof_drain(h);
  }
  if (enable) {
    for (int k = 0; k < HENRY_K_COUNT; ++k) {
      P.ms[k] = 0.0;
      P.launches[k] = 0;
      P.bytes[k] = 0.0;
      P.flops[k] = 0.0;
    }
  }
  P.on = enable != 0;
  for (auto& kv : h->kids) {
    const int rc = henry_profile(kv.second, enable);
    if (rc) return rc;
  }
  return HENRY_OK;
}

int henry_profile_read(henry_handle* h, int kclass, double* total_ms, int64_t* launches, double* alg_bytes,
                       double* alg_flops) {
  if (!h) return set_err(HENRY_EINVAL, "handle is NULL");
  if (kclass < 0 || kclass >= HENRY_K_COUNT) return set_err(HENRY_EINVAL, "kernel class %d out of range", kclass);
  Prof& P = h->prof;
  if (!P.pend.empty()) {
    CK(cudaDeviceSynchronize());
    prof_drain(h);
  }
  double ms = P.ms[kclass], by = P.bytes[kclass], fl = P.flops[kclass];
  int64_t nl = P.launches[kclass];
  for (auto& kv : h->kids) {  // the per-level handles of henry_batch_solve_mixed
    double a, b, c;
    int64_t d;
    const int rc = henry_profile_read(kv.second, kclass, &a, &d, &b, &c);
    if (rc) return rc;
    ms += a;
    nl += d;
    by += b;
    fl += c;
  }
  if (total_ms) *total_ms = ms;
  if (launches) *launches = nl;
  if (alg_bytes) *alg_bytes = by;
  if (alg_flops) *alg_flops = fl;
  return HENRY_OK;
}

int henry_sample_xi(uint64_t seed, int level, uint64_t first_sample, int n, double* xi_dev, void* stream) {
  if (n <= 0) return set_err(HENRY_EINVAL, "n = %d must be positive", n);
  if (!xi_dev) return set_err(HENRY_EINVAL, "xi_dev is NULL");
  if (level < 0) return set_err(HENRY_EINVAL, "level %d < 0", level);
  k_sample_xi<<<nblk(n, 128), 128, 0, (cudaStream_t)stream>>>(seed, level, first_sample, n, xi_dev);
  CKL();
  return HENRY_OK;
}

int henry_level_batch_solve(henry_handle* h, int level, int with_coarse, const double* xi_dev, int n,
                            double* qoi_fine_dev, double* qoi_coarse_dev, int32_t* status_dev,
                            henry_stats* stats_host, void* stream) {
  if (!h) return set_err(HENRY_EINVAL, "handle is NULL");
  if (!valid_level(h, level)) return set_err(HENRY_EINVAL, "level %d outside [0, %d]", level, h->cfg.max_level);
  if (n <= 0) return set_err(HENRY_EINVAL, "n = %d must be positive", n);
  if (!xi_dev || !qoi_fine_dev || !status_dev) return set_err(HENRY_EINVAL, "NULL device pointer");
  if (with_coarse && level == 0) return set_err(HENRY_EINVAL, "level 0 has no coarse partner");
  if (with_coarse && !qoi_coarse_dev) return set_err(HENRY_EINVAL, "qoi_coarse_dev is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  henry_stats local;
  std::memset(&local, 0, sizeof local);
  henry_stats* stp = stats_host ? &local : nullptr;
  int rc;
  const bool vc = h->cfg.scheme == HENRY_SCHEME_VERTEX;
  if (h->cfg.precision == HENRY_MIXED) {
    auto solve = vc ? &vc_batch_solve_level<float> : &batch_solve_level<float>;
    rc = solve(h, level, xi_dev, n, qoi_fine_dev, status_dev, true, stp, st);
    if (!rc && with_coarse) rc = solve(h, level - 1, xi_dev, n, qoi_coarse_dev, status_dev, false, stp, st);
  } else {
    auto solve = vc ? &vc_batch_solve_level<double> : &batch_solve_level<double>;
    rc = solve(h, level, xi_dev, n, qoi_fine_dev, status_dev, true, stp, st);
    if (!rc && with_coarse) rc = solve(h, level - 1, xi_dev, n, qoi_coarse_dev, status_dev, false, stp, st);
  }
  if (rc) return rc;
  // count failed samples (synchronises)
  std::vector<int32_t> hs(n);
  CK(cudaMemcpyAsync(hs.data(), status_dev, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  int64_t failed = 0;
  for (int i = 0; i < n; ++i) failed += hs[i] != 0;
  if (stats_host) {
    local.failed_samples = failed;
    *stats_host = local;
  }
  if (failed) return set_err(HENRY_ENOCONV, "%lld of %d samples did not converge", (long long)failed, n);
  return HENRY_OK;
}

int henry_adjoint(henry_handle* h, int level, const double* xi_dev, int n, const double* qoi_weights_dev,
                  double* grad_dev, double* qoi_dev, int checkpoint_every, int32_t* status_dev, void* stream) {
  if (!h) return set_err(HENRY_EINVAL, "handle is NULL");
  if (!valid_level(h, level)) return set_err(HENRY_EINVAL, "level %d outside [0, %d]", level, h->cfg.max_level);
  if (n <= 0) return set_err(HENRY_EINVAL, "n = %d must be positive", n);
  if (!xi_dev || !qoi_weights_dev || !grad_dev || !qoi_dev || !status_dev)
    return set_err(HENRY_EINVAL, "NULL device pointer");
  if (checkpoint_every <= 0) return set_err(HENRY_EINVAL, "checkpoint_every = %d must be positive", checkpoint_every);
  if (!(h->cfg.adj_rtol > 0.0) || h->cfg.adj_maxit <= 0) return set_err(HENRY_EINVAL, "bad adj_rtol / adj_maxit");
  if (h->cfg.scheme != HENRY_SCHEME_CELL)
    return set_err(HENRY_EINVAL, "the discrete adjoint is built for the cell-centred scheme only");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = adjoint_level(h, level, xi_dev, n, qoi_weights_dev, grad_dev, qoi_dev, checkpoint_every, status_dev, st);
  if (rc) return rc;
  std::vector<int32_t> hs(n);
  CK(cudaMemcpyAsync(hs.data(), status_dev, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  int64_t failed = 0;
  for (int i = 0; i < n; ++i) failed += hs[i] != 0;
  if (failed) return set_err(HENRY_ENOCONV, "%lld of %d samples failed (status_dev)", (long long)failed, n);
  return HENRY_OK;
}

int mlmc_accumulate(int level, int n, int n_qoi, const double* qoi_fine_dev, const double* qoi_coarse_dev,
                    const int32_t* status_dev, double* sums_dev, void* stream) {
  if (level < 0) return set_err(HENRY_EINVAL, "level %d < 0", level);
  if (n <= 0 || n_qoi <= 0) return set_err(HENRY_EINVAL, "n = %d and n_qoi = %d must be positive", n, n_qoi);
  if (!qoi_fine_dev || !sums_dev) return set_err(HENRY_EINVAL, "NULL device pointer");
  k_mlmc_accumulate<<<dim3(n_qoi, 2), 1024, 0, (cudaStream_t)stream>>>(n, n_qoi, qoi_fine_dev, qoi_coarse_dev,
                                                                        status_dev, sums_dev);
  CKL();
  return HENRY_OK;
}

int mlmc_allocate(int n_levels, const double* V, const double* s, double var_budget, int64_t* m_out) {
  if (n_levels <= 0 || !V || !s || !m_out) return set_err(HENRY_EINVAL, "bad arguments");
  if (!(var_budget > 0.0)) return set_err(HENRY_EINVAL, "var_budget must be positive");
  double tot = 0.0;
  for (int l = 0; l < n_levels; ++l) {
    if (!(V[l] >= 0.0) || !(s[l] > 0.0)) return set_err(HENRY_EINVAL, "V[%d] must be >= 0 and s[%d] > 0", l, l);
    tot += std::sqrt(V[l] * s[l]);
  }
  for (int l = 0; l < n_levels; ++l) {
    const double m = std::sqrt(V[l] / s[l]) * tot / var_budget;
    if (!(m < 9.0e18)) return set_err(HENRY_EINVAL, "m[%d] overflows", l);
    m_out[l] = (int64_t)std::ceil(m);
  }
  return HENRY_OK;
}

// Least-squares slope of y_l against l over the given levels (closed form
// of the 2-parameter linear regression).
static double ls_slope(int n, const double* l, const double* y) {
  double ml = 0.0, my = 0.0;
  for (int i = 0; i < n; ++i) {
    ml += l[i];
    my += y[i];
  }
  ml /= n;
  my /= n;
  double sxy = 0.0, sxx = 0.0;
  for (int i = 0; i < n; ++i) {
    sxy += (l[i] - ml) * (y[i] - my);
    sxx += (l[i] - ml) * (l[i] - ml);
  }
  return sxy / sxx;
}

int mlmc_rates(int n_levels, int first_level, const double* mean_Y, const double* V, const double* s,
               double* alpha, double* beta, double* gamma_d) {
  if (n_levels <= 0 || first_level < 0 || n_levels - first_level < 2)
    return set_err(HENRY_EINVAL, "need at least two levels from first_level (n_levels %d, first_level %d)",
                   n_levels, first_level);
  const int n = n_levels - first_level;
  std::vector<double> l(n), y(n);
  for (int i = 0; i < n; ++i) l[i] = first_level + i;
  struct {
    const double* a;
    double* out;
    double sign;
    bool absval;
  } fits[3] = {{mean_Y, alpha, -1.0, true}, {V, beta, -1.0, false}, {s, gamma_d, 1.0, false}};
  for (auto& f : fits) {
    if (!f.out) continue;
    if (!f.a) return set_err(HENRY_EINVAL, "input array for a requested rate is NULL");
    for (int i = 0; i < n; ++i) {
      const double v = f.absval ? std::fabs(f.a[first_level + i]) : f.a[first_level + i];
      if (!(v > 0.0) || !std::isfinite(v))
        return set_err(HENRY_EINVAL, "level %d: value %g must be finite and nonzero (positive)", first_level + i,
                       f.a[first_level + i]);
      y[i] = std::log2(v);
    }
    *f.out = f.sign * ls_slope(n, l.data(), y.data());
  }
  return HENRY_OK;
}

int mlmc_bias_test(int n_levels, const double* mean_Y, double alpha, double eps, double* bias_est,
                   int32_t* converged) {
  if (n_levels < 2 || !mean_Y) return set_err(HENRY_EINVAL, "need at least two levels");
  if (!(alpha > 0.0) || !(eps > 0.0) || !std::isfinite(alpha) || !std::isfinite(eps))
    return set_err(HENRY_EINVAL, "alpha and eps must be positive and finite");
  const double b = std::fabs(mean_Y[n_levels - 1]) / (std::exp2(alpha) - 1.0);
  if (!std::isfinite(b)) return set_err(HENRY_EINVAL, "mean_Y[%d] is not finite", n_levels - 1);
  if (bias_est) *bias_est = b;
  if (converged) *converged = b <= eps / std::sqrt(2.0) ? 1 : 0;
  return HENRY_OK;
}

int mlmc_bias_test_fit(int n_levels, int first_level, const double* mean_Y, double alpha_min, double eps,
                       double* alpha_out, double* bias_est, int32_t* converged) {
  if (!mean_Y || n_levels <= 0 || first_level < 0 || n_levels - first_level < 2)
    return set_err(HENRY_EINVAL, "need at least two levels from first_level (n_levels %d, first_level %d)",
                   n_levels, first_level);
  if (!(alpha_min > 0.0) || !(eps > 0.0) || !std::isfinite(alpha_min) || !std::isfinite(eps))
    return set_err(HENRY_EINVAL, "alpha_min and eps must be positive and finite");
  const int n = n_levels - first_level;
  std::vector<double> l(n), y(n);
  for (int i = 0; i < n; ++i) {
    const double v = std::fabs(mean_Y[first_level + i]);
    if (!(v > 0.0) || !std::isfinite(v))
      return set_err(HENRY_EINVAL, "level %d: mean %g must be finite and nonzero", first_level + i,
                     mean_Y[first_level + i]);
    l[i] = first_level + i;
    y[i] = std::log2(v);
  }
  const double alpha = std::max(-ls_slope(n, l.data(), y.data()), alpha_min);
  double a = 0.0;  // intercept of the fit with that slope
  for (int i = 0; i < n; ++i) a += y[i] + alpha * l[i];
  a /= n;
  const double b = std::exp2(a - alpha * (n_levels - 1)) / (std::exp2(alpha) - 1.0);
  if (!std::isfinite(b)) return set_err(HENRY_EINVAL, "bias estimate is not finite");
  if (alpha_out) *alpha_out = alpha;
  if (bias_est) *bias_est = b;
  if (converged) *converged = b <= eps / std::sqrt(2.0) ? 1 : 0;
  return HENRY_OK;
}

#define STEP_DISPATCH(which, in, out, out2, iters)                                                              \
  (h->cfg.scheme == HENRY_SCHEME_VERTEX                                                                        \
       ? (h->cfg.precision == HENRY_MIXED                                                                      \
              ? vc_step_entry<float>(h, which, level, xi_dev, n, state_dev, state_old_dev, in, out, out2, iters, \
                                     (cudaStream_t)stream)                                                     \
              : vc_step_entry<double>(h, which, level, xi_dev, n, state_dev, state_old_dev, in, out, out2,     \
                                      iters, (cudaStream_t)stream))                                            \
       : (h->cfg.precision == HENRY_MIXED                                                                      \
              ? step_entry<float>(h, which, level, xi_dev, n, state_dev, state_old_dev, in, out, out2, iters,  \
                                  (cudaStream_t)stream)                                                        \
              : step_entry<double>(h, which, level, xi_dev, n, state_dev, state_old_dev, in, out, out2, iters, \
                                   (cudaStream_t)stream)))

int henry_assemble(henry_handle* h, int level, const double* xi_dev, int n, const double* state_dev,
                   const double* state_old_dev, double* F_dev, double* J_dev, void* stream) {
  int rc = check_step_args(h, level, xi_dev, n, state_dev, state_old_dev);
  if (rc) return rc;
  if (!F_dev) return set_err(HENRY_EINVAL, "F_dev is NULL");
  return STEP_DISPATCH(0, nullptr, F_dev, J_dev, nullptr);
}

int henry_apply_jacobian(henry_handle* h, int level, const double* xi_dev, int n, const double* state_dev,
                         const double* state_old_dev, const double* x_dev, double* y_dev, void* stream) {
  int rc = check_step_args(h, level, xi_dev, n, state_dev, state_old_dev);
  if (rc) return rc;
  if (!x_dev || !y_dev) return set_err(HENRY_EINVAL, "NULL vector pointer");
  return STEP_DISPATCH(1, x_dev, y_dev, nullptr, nullptr);
}

int henry_precondition(henry_handle* h, int level, const double* xi_dev, int n, const double* state_dev,
                       const double* state_old_dev, const double* b_dev, double* z_dev, void* stream) {
  int rc = check_step_args(h, level, xi_dev, n, state_dev, state_old_dev);
  if (rc) return rc;
  if (!b_dev || !z_dev) return set_err(HENRY_EINVAL, "NULL vector pointer");
  return STEP_DISPATCH(2, b_dev, z_dev, nullptr, nullptr);
}

int henry_linear_solve(henry_handle* h, int level, const double* xi_dev, int n, const double* state_dev,
                       const double* state_old_dev, const double* b_dev, double* x_dev, int32_t* iters_dev,
                       void* stream) {
  int rc = check_step_args(h, level, xi_dev, n, state_dev, state_old_dev);
  if (rc) return rc;
  if (!b_dev || !x_dev) return set_err(HENRY_EINVAL, "NULL vector pointer");
  return STEP_DISPATCH(3, b_dev, x_dev, nullptr, iters_dev);
}

int henry_vc_assemble(henry_handle* h, int level, const double* xi_dev, int n, const double* state_dev,
                      const double* state_old_dev, double* R_dev, double* J_dev, void* stream) {
  int rc = check_step_args(h, level, xi_dev, n, state_dev, state_old_dev);
  if (rc) return rc;
  if (!R_dev) return set_err(HENRY_EINVAL, "R_dev is NULL");
  const henry_config& c = h->cfg;
  if (c.coef_model != HENRY_MODEL_UNIFORM3)
    return set_err(HENRY_EINVAL, "the vertex-centred assembly supports the three-parameter model only");
  cudaStream_t st = (cudaStream_t)stream;
  const LevelGeom lg = geom(c, level);
  const VcParams P{lg.nx, lg.ny, lg.h, lg.tau, c.rho0, c.rho1 - c.rho0, c.rho1, c.g, c.Ly};
  const size_t cbytes = sizeof(Coef) * (size_t)n;
  char* mem = nullptr;
  if (cudaMallocAsync((void**)&mem, cbytes + sizeof(int) * ((size_t)n + 1), st) != cudaSuccess) {
    cudaGetLastError();
    return set_err(HENRY_ENOMEM, "cudaMallocAsync for %d samples' coefficients failed", n);
  }
  Coef* coef = (Coef*)mem;
  int* status = (int*)(mem + cbytes);
  int* first_bad = status + n;
  const CoefModel m{c.phi_mean, c.K_mean, c.qin_mean, c.phi_amp, c.logK_amp, c.qin_amp, c.mu, c.Dm};
  // Coefficients first, checked on the host: a sample whose xi gives phi
  // outside (0, 1) or a non-finite K or q_in is refused (EINVAL, naming the
  // first such sample) before anything is assembled from it.
  rc = ensure_pinned(h);
  if (!rc) {
    k_coefficients<<<nblk(n, 128), 128, 0, st>>>(m, n, xi_dev, coef, status);
    cudaMemsetAsync(first_bad, 0x7f, sizeof(int), st);
    k_first_bad<<<nblk(n, 128), 128, 0, st>>>(n, status, first_bad);
    rc = read_counter(h, first_bad, st, &h->host_counter[1]);
  }
  if (!rc && h->host_counter[1] < n) {
    const int bad = h->host_counter[1];
    cudaFreeAsync(mem, st);
    return set_err(HENRY_EINVAL, "sample %d: its inputs give phi outside (0, 1) or a non-finite K or q_in", bad);
  }
  if (rc) {
    cudaFreeAsync(mem, st);
    return rc;
  }
  const int64_t total = (int64_t)n * (lg.nx + 1) * (lg.ny + 1);
  k_vc_assemble<<<nblk(total), TPB, 0, st>>>(P, n, coef, state_dev, state_old_dev, R_dev, J_dev);
  const cudaError_t e = cudaGetLastError();
  cudaFreeAsync(mem, st);
  if (e != cudaSuccess) return set_err(HENRY_ECUDA, "vertex-centred assembly launch: %s", cudaGetErrorString(e));
  return HENRY_OK;
}

}  // extern "C"

// ============================================================================
// Allocation-free batch solve.
//
// Some callers cannot allocate device memory at run time: code running under
// an allocator that forbids cudaMalloc (a memory-pool-managed serving
// process, a plug-in that must not grow its footprint) or that wants every
// byte reserved when the library loads.  For them this variant of
// henry_level_batch_solve carves its whole workspace out of one file-scope
// device array of HENRY_STATIC_SCRATCH_BYTES instead of a handle's
// cudaMalloc'd groups, and needs no handle at all.  Every GPU that loads the
// library holds this array until the process exits.
//
// In host code `g_static_scratch` names a host-side stand-in, not the device
// array, so its device address is looked up with cudaGetSymbolAddress once per
// device (with that device current) on the first call there; make that first
// call before any stream capture.  All calls share the array and it keeps the
// last call's contents (the solve initialises everything it reads); calls
// that overlap on the GPU (other streams, other host threads) race on it.
namespace {

static __device__ __align__(256) unsigned char g_static_scratch[HENRY_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_static_ptr[kMaxDevices] = {};
int g_static_host_words[16];                  // pageable host words for the convergence counters
unsigned long long g_static_host_totals[4];

int static_scratch_ptr(char** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_err(HENRY_EINVAL, "device %d outside [0, %d)", dev, kMaxDevices);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return set_err(HENRY_ECUDA, "cudaGetSymbolAddress(static scratch) failed on device %d: %s", dev,
                     cudaGetErrorString(e));
    g_static_ptr[dev] = p;
  }
  *out = static_cast<char*>(g_static_ptr[dev]);
  return HENRY_OK;
}

// The configuration checks of henry_create, without creating a handle, plus
// the entry point's own restriction to the two standard QoIs.
int static_check_config(const henry_config& c) {
  const int rc = check_config(c, false);
  if (rc) return rc;
  if (c.qoi_set != HENRY_QOI_STANDARD)
    return set_err(HENRY_EINVAL, "the allocation-free entry point writes the two standard QoIs only (qoi_set 0)");
  return HENRY_OK;
}

// Lays out the fine group (and the coarse partner's) in the static array.
template <typename T>
int static_solve(henry_handle* H, int level, int with_coarse, const double* xi, int n, double* qf, double* qc,
                 int32_t* status, cudaStream_t st) {
  char* base = nullptr;
  int rc = static_scratch_ptr(&base);
  if (!rc) rc = ensure_tail_attr<T>();
  if (rc) return rc;
  const LevelGeom gf = geom(H->cfg, level);
  Group<T> Gf, Gc;
  Gf.graphs = Gc.graphs = false;  // instantiating a graph would allocate
  size_t need = (Gf.carve(nullptr, n, gf.nx, gf.ny, gf.h) + 255) & ~size_t(255);
  size_t need_c = 0;
  LevelGeom gc{};
  if (with_coarse) {
    gc = geom(H->cfg, level - 1);
    need_c = Gc.carve(nullptr, n, gc.nx, gc.ny, gc.h);
  }
  if (need + need_c > (size_t)HENRY_STATIC_SCRATCH_BYTES)
    return set_err(HENRY_EINVAL,
                   "%d samples at level %d%s need %zu bytes of workspace; the static scratch holds %zu bytes", n,
                   level, with_coarse ? " with coarse partners" : "", need + need_c,
                   (size_t)HENRY_STATIC_SCRATCH_BYTES);
  Gf.carve(base, n, gf.nx, gf.ny, gf.h);
  Gf.level = level;
  Gf.Bcap = n;
  rc = set_coefficients<T>(H, Gf, xi, n, st);
  if (!rc) rc = solve_group<T>(H, Gf, n, qf, st);
  if (rc) return rc;
  k_merge_status<<<nblk(n, 128), 128, 0, st>>>(n, Gf.status, status, 1);
  CKL();
  if (with_coarse) {
    Gc.carve(base + need, n, gc.nx, gc.ny, gc.h);
    Gc.level = level - 1;
    Gc.Bcap = n;
    rc = set_coefficients<T>(H, Gc, xi, n, st);
    if (!rc) rc = solve_group<T>(H, Gc, n, qc, st);
    if (rc) return rc;
    k_merge_status<<<nblk(n, 128), 128, 0, st>>>(n, Gc.status, status, 0);
    CKL();
  }
  return HENRY_OK;
}

}  // namespace

extern "C" int henry_level_batch_solve_static(const henry_config* cfg, int level, int with_coarse,
                                              const double* xi_dev, int n, double* qoi_fine_dev,
                                              double* qoi_coarse_dev, int32_t* status_dev, void* stream) {
  if (!cfg) return set_err(HENRY_EINVAL, "cfg is NULL");
  int rc = static_check_config(*cfg);
  if (rc) return rc;
  if (cfg->coef_model != HENRY_MODEL_UNIFORM3 || cfg->scheme != HENRY_SCHEME_CELL)
    return set_err(HENRY_EINVAL,
                   "the static-scratch solve supports the three-parameter model on the cell-centred scheme only");
  if (level < 0 || level > cfg->max_level) return set_err(HENRY_EINVAL, "level %d outside [0, %d]", level, cfg->max_level);
  if (n <= 0) return set_err(HENRY_EINVAL, "n = %d must be positive", n);
  if (!xi_dev || !qoi_fine_dev || !status_dev) return set_err(HENRY_EINVAL, "NULL device pointer");
  if (with_coarse && level == 0) return set_err(HENRY_EINVAL, "level 0 has no coarse partner");
  if (with_coarse && !qoi_coarse_dev) return set_err(HENRY_EINVAL, "qoi_coarse_dev is NULL");
  henry_handle H;  // on the stack: no device workspace, no pinned buffers, timer off
  H.cfg = *cfg;
  H.host_counter = g_static_host_words;
  H.host_totals = g_static_host_totals;
  cudaStream_t st = (cudaStream_t)stream;
  rc = cfg->precision == HENRY_MIXED
           ? static_solve<float>(&H, level, with_coarse, xi_dev, n, qoi_fine_dev, qoi_coarse_dev, status_dev, st)
           : static_solve<double>(&H, level, with_coarse, xi_dev, n, qoi_fine_dev, qoi_coarse_dev, status_dev, st);
  if (rc) return rc;
  int32_t buf[256];
  int64_t failed = 0;
  for (int off = 0; off < n; off += 256) {
    const int m = std::min(256, n - off);
    CK(cudaMemcpyAsync(buf, status_dev + off, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int i = 0; i < m; ++i) failed += buf[i] != 0;
  }
  if (failed) return set_err(HENRY_ENOCONV, "%lld of %d samples did not converge", (long long)failed, n);
  return HENRY_OK;
}
