// Host side of the library: C ABI, device MPO store, router/planner, wave scheduler,
// unswap driver and the output-MPS queries.  See include/peaked_mpo.h for the contract.
//
// The contraction follows Algorithm 1 of Kremer & Dupuis: route each gate to a line
// (Sec. II.A), absorb the innermost layer of C_L then of C_R (Sec. II.B.1), unswap when
// size(M) >= tau (Sec. II.B.2, App. A.1), rewire by continuing with the updated layouts
// (Sec. II.B.3), finally project onto |0...0> (Sec. II.C).
//
// The MPO is held as a local-dimension-4 MPS (p = 2*out + in) in Vidal form with Hastings'
// update: right-canonical site tensors B_j and bond spectra lambda_j.  Updates on disjoint
// site pairs read and write disjoint data, so the updates of a layer are grouped into
// waves (as-soon-as-possible over shared sites) and each wave runs as one batch of
// kernels; the result is identical to applying them one by one.
#include "../../include/peaked_mpo.h"
#include "pc_internal.h"

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <complex>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <queue>
#include <string>
#include <thread>
#include <vector>

using cplx = std::complex<double>;

namespace {

const char* kVersion = "peaked-mpo-gb300 0.1 (sm_103a, FP64 one-sided Jacobi)";

struct Layout {
  std::vector<int> pos;    // logical qubit -> site
  std::vector<int> site;   // site -> logical qubit
  void reset(int n) {
    pos.resize(n);
    site.resize(n);
    for (int i = 0; i < n; ++i) pos[i] = site[i] = i;
  }
  void swap_sites(int j) {
    const int a = site[j], b = site[j + 1];
    site[j] = b;
    site[j + 1] = a;
    pos[a] = j + 1;
    pos[b] = j;
  }
};

struct PlanOp {       // one two-site update emitted by the router
  int side;           // PC_SIDE_LEFT / PC_SIDE_RIGHT
  int bond;
  int kind;           // 0 routing swap, 1 gate
  int gate;           // gate index or -1
};

// 16x16 operator on (p1, p2) with p = 2*o + i for M <- g M h; g acts on (o1, o2) with basis
// index 2*o1 + o2, h on (i1, i2) as M[o, i] <- sum_i' M[o, i'] h[i', i].  Null means identity.
void two_site_op(const cplx* g, const cplx* h, cplx* U) {
  auto G = [&](int r, int c) -> cplx { return g ? g[4 * r + c] : (r == c ? cplx(1, 0) : cplx(0, 0)); };
  auto H = [&](int r, int c) -> cplx { return h ? h[4 * r + c] : (r == c ? cplx(1, 0) : cplx(0, 0)); };
  for (int row = 0; row < 16; ++row) {
    const int p1 = row >> 2, p2 = row & 3;
    const int o1 = p1 >> 1, i1 = p1 & 1, o2 = p2 >> 1, i2 = p2 & 1;
    for (int col = 0; col < 16; ++col) {
      const int q1 = col >> 2, q2 = col & 3;
      const int a1 = q1 >> 1, b1 = q1 & 1, a2 = q2 >> 1, b2 = q2 & 1;
      U[16 * row + col] = G(2 * o1 + o2, 2 * a1 + a2) * H(2 * b1 + b2, 2 * i1 + i2);
    }
  }
}

const cplx kSwap4[16] = {1, 0, 0, 0, 0, 0, 1, 0, 0, 1, 0, 0, 0, 0, 0, 1};

void swap_op(int side, cplx* U) {
  if (side == PC_SIDE_LEFT) two_site_op(kSwap4, nullptr, U);
  else if (side == PC_SIDE_RIGHT) two_site_op(nullptr, kSwap4, U);
  else two_site_op(kSwap4, kSwap4, U);
}

// Greedy as-soon-as-possible layering in absorption order: a gate goes one layer past the
// last layer that used either of its qubits.
std::vector<std::vector<int>> make_layers(const std::vector<int>& order, const int32_t* pairs, int n) {
  std::vector<int> last(n, -1);
  std::vector<std::vector<int>> layers;
  for (int g : order) {
    const int a = pairs[2 * g], b = pairs[2 * g + 1];
    const int lay = std::max(last[a], last[b]) + 1;
    if (lay == (int)layers.size()) layers.emplace_back();
    layers[lay].push_back(g);
    last[a] = last[b] = lay;
  }
  return layers;
}

// Routes one gate of one side: the first-listed qubit moves one site at a time toward the
// second (a SWAP update per step), then the gate is applied on the bond they share.
void route_gate(int side, int g, const int32_t* pairs, Layout& lay, std::vector<PlanOp>& out) {
  const int a = pairs[2 * g], b = pairs[2 * g + 1];
  int p = lay.pos[a];
  const int q = lay.pos[b];
  while (std::abs(p - q) > 1) {
    const int j = p < q ? p : p - 1;
    out.push_back({side, j, 0, -1});
    lay.swap_sites(j);
    p = lay.pos[a];
  }
  out.push_back({side, std::min(p, q), 1, g});
}

inline double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

uint64_t splitmix64(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

struct pc_ctx {
  pc_config cfg;
  int sm_count = 0;
  std::string last_error;
};

namespace {

// ---------------------------------------------------------------------------------------
// Workspaces.  Every factorisation of a wave (Sec. II.B.1) needs scratch of the size of its
// own bond matrix; it is bump-allocated from a device arena per launch, so one workspace
// serves updates of any mix of bond dimensions, from one circuit or from many.
struct TaskScratch {
  double2* X = nullptr;      // the Jacobi matrix: the rows of the bond matrix, or its columns
  double2* T0 = nullptr;     // merged and gated, without lambda
  double2* Q = nullptr;      // accumulated rotations (column path, FP32 preconditioning)
  double2* Qb = nullptr;     // Newton-Schulz second buffer
  double2* Y = nullptr;      // Q X after preconditioning
  float2* X32 = nullptr;
  float2* Q32 = nullptr;
  int32_t* stamp = nullptr;      // FP64 sweeps
  int32_t* stamp32 = nullptr;    // FP32 sweeps
  double* nrm2 = nullptr;
  double* lam = nullptr;
  double* sraw = nullptr;
  int32_t* idx = nullptr;
};

inline size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// Arena bytes of one update whose bond matrix is m x n.
size_t task_bytes(int m, int n, bool precond) {
  const size_t v = (size_t)std::min(m, n), mn = (size_t)m * n;
  size_t b = 2 * al256(mn * sizeof(double2)) + al256(v * v * sizeof(double2)) + 3 * al256(v * sizeof(double)) +
             2 * al256(v * sizeof(int32_t));
  if (precond)
    b += al256(mn * sizeof(float2)) + al256(v * v * sizeof(float2)) + al256(v * v * sizeof(double2)) +
         al256(mn * sizeof(double2)) + al256(v * sizeof(int32_t));
  return b;
}

struct Workspace {
  int cap = 0;                     // tasks per launch
  int sm_count = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  char* d_arena = nullptr;
  size_t arena_alloc = 0;          // bytes allocated
  size_t arena_limit = 0;          // bytes a launch may use (the arena grows up to this)
  void* d_tcws = nullptr;          // split operands of the tensor-core merge
  size_t tcws_bytes = 0;
  cplx* h_ops = nullptr;
  double2* d_ops = nullptr;
  pc::UpdateTask *h_tasks = nullptr, *d_tasks = nullptr;
  pc::GemmDesc *h_merge = nullptr, *d_merge = nullptr;
  pc::JacobiTask *h_jt = nullptr, *d_jt = nullptr;       // merged matrices
  pc::JacobiTask *h_jsub = nullptr, *d_jsub = nullptr;   // preconditioned subset
  pc::JacobiTask *h_jy = nullptr, *d_jy = nullptr;       // FP64 sweeps
  pc::JacobiTask *h_jfb = nullptr, *d_jfb = nullptr;     // FP64-only redo subset
  pc::JacobiTask32 *h_j32 = nullptr, *d_j32 = nullptr;
  double2 **h_q64 = nullptr, **d_q64 = nullptr;
  pc::GemmDesc *h_ns = nullptr, *d_ns = nullptr;         // [5][cap]
  pc::TruncTask *h_tt = nullptr, *d_tt = nullptr;        // [2][cap]: main, redo
  pc::TruncOut *h_tout = nullptr, *d_tout = nullptr;
  pc::JacobiStatus *h_jst = nullptr, *d_jst = nullptr;   // [2][cap]
  double *h_fro2 = nullptr, *d_fro2 = nullptr;
  pc::SplitRowsDesc *h_split = nullptr, *d_split = nullptr;
  pc::GemmDesc *h_gemm2 = nullptr, *d_gemm2 = nullptr;
  unsigned int* d_bar = nullptr;
  int *d_err = nullptr, *h_err = nullptr;                // [0] Jacobi barrier, [1] tensor-core merge
  // unswap-trial certificate: C = P X^H, its FP64 Jacobi and sorted row norms
  pc::GemmDesc *h_cg = nullptr, *d_cg = nullptr;
  pc::JacobiTask *h_jc = nullptr, *d_jc = nullptr;
  pc::TruncTask *h_tc = nullptr, *d_tc = nullptr;
  pc::TruncOut *h_ctout = nullptr, *d_ctout = nullptr;
  pc::JacobiStatus *h_jst3 = nullptr, *d_jst3 = nullptr;
  double *h_cfro2 = nullptr, *d_cfro2 = nullptr;
  std::map<std::pair<int, int>, double2*> srft;          // (row length, rows) -> P on the device
  // deflation floors of the FP64 sweeps
  pc::DeflateTask *h_df = nullptr, *d_df = nullptr;
  double *h_dead2 = nullptr, *d_dead2 = nullptr;         // [2][cap]: floor, s_c
  // kernel accounting: 0 merge+gate, 1 factorisation, 2 truncation, 3 split, 4 other,
  // 5 unswap-trial certificates
  bool timing = false;
  cudaEvent_t ev[6] = {};
  int64_t t_launch[6] = {};
  double t_ms[6] = {};
  double t_flops[6] = {};
  int64_t n_launches = 0;          // combined launches (batch accounting)
  int64_t n_tasks = 0;
  int max_tasks_seen = 0;
};

void ws_destroy(Workspace* w) {
  if (!w) return;
  cudaFree(w->d_arena); cudaFree(w->d_tcws); cudaFree(w->d_ops); cudaFree(w->d_tasks); cudaFree(w->d_merge);
  cudaFree(w->d_jt); cudaFree(w->d_jsub); cudaFree(w->d_jy); cudaFree(w->d_jfb); cudaFree(w->d_j32);
  cudaFree(w->d_q64); cudaFree(w->d_ns); cudaFree(w->d_tt); cudaFree(w->d_tout); cudaFree(w->d_jst);
  cudaFree(w->d_fro2); cudaFree(w->d_split); cudaFree(w->d_gemm2); cudaFree(w->d_bar); cudaFree(w->d_err);
  cudaFree(w->d_cg); cudaFree(w->d_jc); cudaFree(w->d_tc); cudaFree(w->d_ctout); cudaFree(w->d_jst3);
  cudaFree(w->d_cfro2); cudaFree(w->d_df); cudaFree(w->d_dead2);
  cudaFreeHost(w->h_cg); cudaFreeHost(w->h_jc); cudaFreeHost(w->h_tc); cudaFreeHost(w->h_ctout);
  cudaFreeHost(w->h_jst3); cudaFreeHost(w->h_cfro2); cudaFreeHost(w->h_df); cudaFreeHost(w->h_dead2);
  for (auto& kv : w->srft) cudaFree(kv.second);
  cudaFreeHost(w->h_ops); cudaFreeHost(w->h_tasks); cudaFreeHost(w->h_merge); cudaFreeHost(w->h_jt);
  cudaFreeHost(w->h_jsub); cudaFreeHost(w->h_jy); cudaFreeHost(w->h_jfb); cudaFreeHost(w->h_j32);
  cudaFreeHost(w->h_q64); cudaFreeHost(w->h_ns); cudaFreeHost(w->h_tt); cudaFreeHost(w->h_tout);
  cudaFreeHost(w->h_jst); cudaFreeHost(w->h_fro2); cudaFreeHost(w->h_split); cudaFreeHost(w->h_gemm2);
  cudaFreeHost(w->h_err);
  for (auto& e : w->ev) if (e) cudaEventDestroy(e);
  if (w->own_stream && w->stream) cudaStreamDestroy(w->stream);
  delete w;
}

// A workspace for `cap` tasks per launch whose arena may grow to `arena_limit` bytes.
// stream: the stream to launch on (nullptr: the workspace creates its own).
cudaError_t ws_create(int cap, size_t arena_limit, int sm_count, cudaStream_t stream, Workspace** out) {
  *out = nullptr;
  auto* w = new Workspace();
  w->cap = cap;
  w->arena_limit = arena_limit;
  w->sm_count = sm_count;
  cudaError_t e = cudaSuccess;
  auto dev = [&](auto** p, size_t n) { if (e == cudaSuccess) e = cudaMalloc((void**)p, n * sizeof(**p)); };
  auto pin = [&](auto** p, size_t n) { if (e == cudaSuccess) e = cudaMallocHost((void**)p, n * sizeof(**p)); };
  if (stream) {
    w->stream = stream;
  } else {
    e = cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking);
    w->own_stream = e == cudaSuccess;
  }
  const size_t C = (size_t)cap;
  dev(&w->d_ops, C * 256); pin(&w->h_ops, C * 256);
  dev(&w->d_tasks, C); pin(&w->h_tasks, C);
  dev(&w->d_merge, C); pin(&w->h_merge, C);
  dev(&w->d_jt, C); pin(&w->h_jt, C);
  dev(&w->d_jsub, C); pin(&w->h_jsub, C);
  dev(&w->d_jy, C); pin(&w->h_jy, C);
  dev(&w->d_jfb, C); pin(&w->h_jfb, C);
  dev(&w->d_j32, C); pin(&w->h_j32, C);
  dev(&w->d_q64, C); pin(&w->h_q64, C);
  dev(&w->d_ns, 5 * C); pin(&w->h_ns, 5 * C);
  dev(&w->d_tt, 2 * C); pin(&w->h_tt, 2 * C);
  dev(&w->d_tout, C); pin(&w->h_tout, C);
  dev(&w->d_jst, 2 * C); pin(&w->h_jst, 2 * C);
  dev(&w->d_fro2, C); pin(&w->h_fro2, C);
  dev(&w->d_split, C); pin(&w->h_split, C);
  dev(&w->d_gemm2, C); pin(&w->h_gemm2, C);
  dev(&w->d_bar, 2);
  dev(&w->d_err, 2); pin(&w->h_err, 2);
  dev(&w->d_cg, C); pin(&w->h_cg, C);
  dev(&w->d_jc, C); pin(&w->h_jc, C);
  dev(&w->d_tc, C); pin(&w->h_tc, C);
  dev(&w->d_ctout, C); pin(&w->h_ctout, C);
  dev(&w->d_jst3, C); pin(&w->h_jst3, C);
  dev(&w->d_cfro2, C); pin(&w->h_cfro2, C);
  dev(&w->d_df, C); pin(&w->h_df, C);
  dev(&w->d_dead2, 2 * C); pin(&w->h_dead2, 2 * C);
  for (auto& ev : w->ev)
    if (e == cudaSuccess) e = cudaEventCreate(&ev);
  if (e != cudaSuccess) { ws_destroy(w); return e; }
  *out = w;
  return cudaSuccess;
}

// Grows the arena to at least `bytes` (never beyond what a launch may use).
cudaError_t ws_reserve(Workspace* w, size_t bytes) {
  if (bytes <= w->arena_alloc) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(w->stream);
  if (e != cudaSuccess) return e;
  cudaFree(w->d_arena);
  w->d_arena = nullptr;
  w->arena_alloc = 0;
  e = cudaMalloc(&w->d_arena, bytes);
  if (e == cudaSuccess) w->arena_alloc = bytes;
  return e;
}

}  // namespace

struct pc_batch;

struct pc_circuit {
  pc_ctx* ctx = nullptr;
  int n = 0;
  int chi_max = 0;
  int max_tasks = 0;
  std::vector<int32_t> pairs;
  std::vector<cplx> mats;
  int64_t split = 0;
  std::vector<int32_t> oneq_q;
  std::vector<cplx> oneq_m;
  std::vector<std::vector<int>> left_layers, right_layers;
  size_t lcur = 0, rcur = 0;
  bool oneq_done = true;
  Layout lay[2];
  std::vector<int> chi;           // chi[k], k = 0..n: left bond of site k; chi[0] = chi[n] = 1
  std::vector<int> cap;           // capacity of chi[k] in the site store
  std::vector<size_t> site_off;   // element offset of each site slot
  cudaStream_t stream = nullptr;
  double2* d_sites = nullptr;
  double* d_lam = nullptr;        // bond b spectrum at d_lam + b * chi_max
  double2* d_g2 = nullptr;
  pc::GemmDesc* h_gemm = nullptr; // [2] the circuit's own GEMMs (projection, sampling)
  // recanonicalisation scratch (allocated on first use, sized by chi_max)
  char* d_rc = nullptr;
  struct {
    double2 *Z, *Q, *T, *C;
    double *nrm2, *lam, *sraw, *fro2;
    int32_t *stamp, *idx;
    pc::JacobiTask* jt;
    pc::TruncTask* tt;
    pc::TruncOut* tout;
    pc::JacobiStatus* jst;
    unsigned int* bar;
    int* err;
  } rc{};
  pc::GemmDesc* d_gemm = nullptr;
  Workspace* ws = nullptr;        // private workspace, created by the first standalone wave
  pc_batch* batch = nullptr;      // set while the circuit's waves go through a batch launcher
  // output MPS (environments)
  bool projected = false;
  double2* d_env = nullptr;
  std::vector<size_t> env_off;
  double norm2 = 0.0;
  // logs and stats
  std::vector<std::array<int32_t, 5>> plan_log;
  std::vector<std::array<int32_t, 4>> unswap_log;
  pc_stats stats{};
  int stage = 0;
  std::vector<pc_trace_record> trace;
  double t_loaded = 0.0;
  bool timing = false;
  int64_t other_launches = 0;     // class 4 launches on the circuit's own stream
  // device-side checkpoint
  double2* d_snap_sites = nullptr;
  double* d_snap_lam = nullptr;
  bool has_snapshot = false;
  std::vector<int> snap_chi;
  Layout snap_lay[2];
  size_t snap_lcur = 0, snap_rcur = 0;
  bool snap_oneq_done = true;
  // App. A.3 adaptive side selection: the state before a step and after its left trial
  struct Saved {
    double2* sites = nullptr;
    double* lam = nullptr;
    std::vector<int> chi;
    Layout lay[2];
    size_t lcur = 0, rcur = 0;
    bool oneq_done = true;
    std::vector<std::array<int32_t, 5>> plan;
    int64_t nupd = 0;
  } saved[2];
};

namespace {

pc_status fail(pc_ctx* ctx, pc_status st, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return st;
}

#define CUDA_TRY(ctx, expr)                                                                      \
  do {                                                                                           \
    cudaError_t e_ = (expr);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return fail((ctx), e_ == cudaErrorMemoryAllocation ? PC_ERR_OOM : PC_ERR_CUDA,             \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));                           \
  } while (0)

double2* site_ptr(pc_circuit* c, int j) { return c->d_sites + c->site_off[j]; }
double* lam_ptr(pc_circuit* c, int b) { return c->d_lam + (size_t)b * c->chi_max; }

int64_t mpo_size(const pc_circuit* c) {
  int64_t s = 0;
  for (int j = 0; j < c->n; ++j) s += (int64_t)c->chi[j] * 4 * c->chi[j + 1];
  return s;
}

int max_bond(const pc_circuit* c) {
  int m = 1;
  for (int k = 1; k < c->n; ++k) m = std::max(m, c->chi[k]);
  return m;
}

// Capacity of bond k (left of site k) in the site store: 1 at the two ends, chi_max inside.
int bond_cap(int n, int k, int chi_max) { return (k <= 0 || k >= n) ? 1 : chi_max; }

// Device bytes of a circuit's store: sites at their caps, spectra, right environments
// (allocated at projection), the peak-search pool and the buffers of n_samples samples.
size_t store_bytes(int n, int chi_max, int64_t n_samples) {
  size_t b = 0, env = 0;
  for (int j = 0; j < n; ++j) {
    const size_t cl = bond_cap(n, j, chi_max), cr = bond_cap(n, j + 1, chi_max);
    b += cl * 4 * cr * sizeof(double2);
    env += cl * cl * sizeof(double2);
  }
  b += (size_t)std::max(1, n - 1) * chi_max * sizeof(double) + env + (size_t)chi_max * chi_max * sizeof(double2);
  b += (size_t)4096 * chi_max * sizeof(double2);
  b += (size_t)std::min<int64_t>(n_samples, 4096) * chi_max * 5 * sizeof(double2);
  return b;
}

void free_circuit(pc_circuit* c) {
  if (!c) return;
  ws_destroy(c->ws);
  cudaFree(c->d_sites); cudaFree(c->d_lam); cudaFree(c->d_g2); cudaFree(c->d_gemm); cudaFreeHost(c->h_gemm);
  cudaFree(c->d_env);
  cudaFree(c->d_rc);
  cudaFree(c->d_snap_sites);
  cudaFree(c->d_snap_lam);
  for (auto& sv : c->saved) { cudaFree(sv.sites); cudaFree(sv.lam); }
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

pc_status alloc_circuit(pc_circuit* c) {
  pc_ctx* ctx = c->ctx;
  const int n = c->n, X = c->chi_max;
  c->chi.assign(n + 1, 1);
  c->cap.resize(n + 1);
  for (int k = 0; k <= n; ++k) c->cap[k] = bond_cap(n, k, X);
  c->site_off.resize(n + 1);
  size_t off = 0;
  for (int j = 0; j < n; ++j) {
    c->site_off[j] = off;
    off += (size_t)c->cap[j] * 4 * c->cap[j + 1];
  }
  c->site_off[n] = off;
  c->max_tasks = std::max(1, std::min(n / 2, 32));
  CUDA_TRY(ctx, cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
  CUDA_TRY(ctx, cudaMalloc(&c->d_sites, off * sizeof(double2)));
  CUDA_TRY(ctx, cudaMalloc(&c->d_lam, (size_t)std::max(1, n - 1) * X * sizeof(double)));
  CUDA_TRY(ctx, cudaMalloc(&c->d_g2, 4 * sizeof(double2)));
  CUDA_TRY(ctx, cudaMalloc(&c->d_gemm, 2 * sizeof(pc::GemmDesc)));
  CUDA_TRY(ctx, cudaMallocHost(&c->h_gemm, 2 * sizeof(pc::GemmDesc)));
  return PC_OK;
}

// The private workspace of a circuit that runs its waves itself: max_tasks tasks per launch,
// arena for max_tasks of its largest bond matrices.
pc_status private_workspace(pc_circuit* c) {
  if (c->ws) return PC_OK;
  int big = 1;
  for (int k = 1; k < c->n; ++k) big = std::max(big, c->cap[k]);
  const bool precond = c->ctx->cfg.fp32_precondition && 4 * big >= 64;
  const size_t limit = (size_t)c->max_tasks * task_bytes(4 * big, 4 * big, precond);
  CUDA_TRY(c->ctx, ws_create(c->max_tasks, limit, c->ctx->sm_count, c->stream, &c->ws));
  c->ws->timing = c->timing;
  return PC_OK;
}

// Identity MPO (Algorithm 1: M <- I, bond dimension 1): B_j[0, p, 0] = delta_{o,i} / sqrt 2.
pc_status reset_identity(pc_circuit* c) {
  std::vector<double2> h(4 * c->n);
  const double r = 1.0 / std::sqrt(2.0);
  for (int j = 0; j < c->n; ++j) {
    h[4 * j + 0] = make_double2(r, 0.0);
    h[4 * j + 1] = make_double2(0.0, 0.0);
    h[4 * j + 2] = make_double2(0.0, 0.0);
    h[4 * j + 3] = make_double2(r, 0.0);
  }
  std::fill(c->chi.begin(), c->chi.end(), 1);
  for (int j = 0; j < c->n; ++j)
    CUDA_TRY(c->ctx, cudaMemcpyAsync(site_ptr(c, j), &h[4 * j], 4 * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
  std::vector<double> ones(std::max(1, c->n - 1), 1.0);
  for (int b = 0; b + 1 < c->n; ++b)
    CUDA_TRY(c->ctx, cudaMemcpyAsync(lam_ptr(c, b), &ones[b], sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c->ctx, cudaStreamSynchronize(c->stream));
  c->lay[0].reset(c->n);
  c->lay[1].reset(c->n);
  c->projected = false;
  return PC_OK;
}

inline void count_launch(pc_circuit* c, int k = 1) { c->other_launches += k; }

// One update of a wave: bond j and its 16x16 operator.
struct WaveItem {
  int bond;
  cplx op[256];
};

// One circuit's share of a wave: factorise every item, then split the committed ones.
// commit_mask (may be null: commit all) or, with decide_by_accept, the unswap rule decides
// per item from its count (strict: count < chi, equal: count <= chi).
struct WaveReq {
  pc_circuit* c = nullptr;
  const std::vector<WaveItem>* items = nullptr;
  const std::vector<int>* commit_mask = nullptr;
  bool decide_by_accept = false;
  bool accept_equal = false;
  // unswap trials whose count only matters against the bond's current dimension (strict:
  // count < chi_old accepts; equal: count <= chi_old): a certified lower bound that reaches
  // the rejection threshold decides them without the full factorisation
  bool trial_only = false;
  std::vector<int> counts, accepted;
  pc_status status = PC_OK;
  bool done = false;
};

struct FlatTask {
  WaveReq* r;
  int k;
};

void timer_mark(Workspace* w, int i) {
  if (w->timing) cudaEventRecord(w->ev[i], w->stream);
}

// Records an error on every circuit of a chunk.
pc_status chunk_fail(std::vector<FlatTask>& flat, size_t b0, size_t b1, pc_status st, const std::string& msg) {
  for (size_t i = b0; i < b1; ++i) {
    flat[i].r->status = st;
    fail(flat[i].r->c->ctx, st, msg);
  }
  return st;
}

#define WS_TRY(expr)                                                                             \
  do {                                                                                           \
    cudaError_t e_ = (expr);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return chunk_fail(flat, b0, b1, e_ == cudaErrorMemoryAllocation ? PC_ERR_OOM : PC_ERR_CUDA, \
                        std::string(#expr) + ": " + cudaGetErrorString(e_));                     \
  } while (0)

// Merge and gate of one launch: for each input, X = lambda-scaled gated merge (or its transpose
// for a tall bond matrix) and T0 = the same without lambda (Sec. II.B.1: contract the gate with
// the two site tensors).  FP64 merges run on gemm_kernel, mixed-precision ones on the tensor
// cores.  Fills the workspace's operator, task and merge tables and launches on w->stream.
struct MergeIn {
  pc_circuit* c;
  const WaveItem* it;
  double2* X;
  double2* T0;
};

cudaError_t stage_merge_gate(Workspace* w, const std::vector<MergeIn>& in) {
  const int T = (int)in.size();
  cudaStream_t s = w->stream;
  std::vector<pc::GemmDesc> g64, gtc;
  int max_cl = 0, max_cr = 0, tc_m = 0, tc_n = 0, tc_k = 0;
  for (int t = 0; t < T; ++t) {
    pc_circuit* c = in[t].c;
    const int j = in[t].it->bond;
    const int cl = c->chi[j], cm = c->chi[j + 1], cr = c->chi[j + 2];
    const int m = 4 * cl, n = 4 * cr;
    std::memcpy(w->h_ops + (size_t)t * 256, in[t].it->op, 256 * sizeof(cplx));
    pc::UpdateTask& u = w->h_tasks[t];
    u.Bl = site_ptr(c, j);
    u.Br = site_ptr(c, j + 1);
    u.lam_l = j > 0 ? lam_ptr(c, j - 1) : nullptr;
    u.op = w->d_ops + (size_t)t * 256;
    u.X = in[t].X;
    u.T0 = in[t].T0;
    u.chi_l = cl; u.chi_m = cm; u.chi_r = cr;
    u.m = m; u.n = n;
    u.transposed = m > n ? 1 : 0;
    pc::GemmDesc g{};
    g.A = u.Bl; g.B = u.Br; g.C = u.T0;   // the gate reads the merge from T0 and writes X
    g.M = m; g.N = n; g.K = cm;
    g.lda = cm; g.ldb = n; g.ldc = n;
    g.opB = 0; g.alpha = 1.0; g.beta = 0.0;
    if (c->ctx->cfg.precision == PC_PRECISION_TF32X3) {
      gtc.push_back(g);
      tc_m = std::max(tc_m, m); tc_n = std::max(tc_n, n); tc_k = std::max(tc_k, cm);
    } else {
      g64.push_back(g);
    }
    max_cl = std::max(max_cl, cl); max_cr = std::max(max_cr, cr);
    const double mg = 8.0 * m * (double)cm * n + 8.0 * 256.0 * cl * (double)cr;
    w->t_flops[0] += mg;
    c->stats.alg_flops += mg;
  }
  const int n64 = (int)g64.size(), ntc = (int)gtc.size();
  for (int i = 0; i < n64; ++i) w->h_merge[i] = g64[i];
  for (int i = 0; i < ntc; ++i) w->h_merge[n64 + i] = gtc[i];
  cudaError_t e = cudaSuccess;
  if (ntc > 0) {
    const size_t tb = pc::tc_merge_workspace_bytes(ntc, tc_m, tc_n, tc_k);
    if (tb > w->tcws_bytes) {
      e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return e;
      cudaFree(w->d_tcws);
      w->d_tcws = nullptr;
      w->tcws_bytes = 0;
      e = cudaMalloc(&w->d_tcws, tb);
      if (e != cudaSuccess) return e;
      w->tcws_bytes = tb;
    }
  }
  if ((e = cudaMemcpyAsync(w->d_ops, w->h_ops, (size_t)T * 256 * sizeof(cplx), cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(w->d_tasks, w->h_tasks, T * sizeof(pc::UpdateTask), cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(w->d_merge, w->h_merge, T * sizeof(pc::GemmDesc), cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(w->d_err, 0, 2 * sizeof(int), s)) != cudaSuccess) return e;
  timer_mark(w, 0);
  if (n64 > 0) {
    int mm = 0, nn = 0;
    for (auto& g : g64) { mm = std::max(mm, g.M); nn = std::max(nn, g.N); }
    if ((e = pc::launch_gemm(w->d_merge, n64, mm, nn, s)) != cudaSuccess) return e;
    w->t_launch[0] += 1;
  }
  if (ntc > 0) {
    // merge as complex 3xTF32 on the tensor cores (two launches: operand split, MMA)
    e = pc::launch_tc_merge(w->d_merge + n64, ntc, tc_m, tc_n, tc_k, w->d_tcws, w->tcws_bytes, w->d_err + 1, s);
    if (e != cudaSuccess) return e;
    w->t_launch[0] += 2;
  }
  if ((e = pc::launch_gate_apply(w->d_tasks, T, max_cl, max_cr, s)) != cudaSuccess) return e;
  w->t_launch[0] += 1;
  return cudaSuccess;
}

// A fixed random projection with orthonormal rows (a subsampled randomised Fourier transform:
// Woolfe, Liberty, Rokhlin and Tygert 2008): P[s][k] = e^{i (phi_k - 2 pi f_s k / L)} / sqrt(L)
// with distinct frequencies f_s and phases phi_k drawn from SplitMix64.  Built once per
// (L, r) on the host and kept on the device.
cudaError_t srft_matrix(Workspace* w, int L, int r, double2** out) {
  auto key = std::make_pair(L, r);
  auto it = w->srft.find(key);
  if (it != w->srft.end()) { *out = it->second; return cudaSuccess; }
  std::vector<int> freq(L);
  for (int k = 0; k < L; ++k) freq[k] = k;
  for (int k = L - 1; k > 0; --k) {          // Fisher-Yates with a counter-based stream
    const int j = (int)(splitmix64(0x5EED0000u + (uint64_t)L, (uint64_t)k) % (uint64_t)(k + 1));
    std::swap(freq[k], freq[j]);
  }
  std::vector<double2> h((size_t)r * L);
  const double two_pi = 6.283185307179586476925286766559;
  const double inv = 1.0 / std::sqrt((double)L);
  std::vector<double> phi(L);
  for (int k = 0; k < L; ++k)
    phi[k] = two_pi * (double)(splitmix64(0xFA5E0000u + (uint64_t)L, (uint64_t)k) >> 11) * (1.0 / 9007199254740992.0);
  for (int q = 0; q < r; ++q)
    for (int k = 0; k < L; ++k) {
      const double a = phi[k] - two_pi * (double)(((int64_t)freq[q] * k) % L) / (double)L;
      h[(size_t)q * L + k] = make_double2(std::cos(a) * inv, std::sin(a) * inv);
    }
  double2* d = nullptr;
  cudaError_t e = cudaMalloc(&d, h.size() * sizeof(double2));
  if (e != cudaSuccess) return e;
  // stream-ordered and complete before the host buffer goes: a pageable cudaMemcpy may return
  // before its DMA lands, and the kernels that read P run on a non-blocking stream
  e = cudaMemcpyAsync(d, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice, w->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
  if (e != cudaSuccess) { cudaFree(d); return e; }
  w->srft[key] = d;
  *out = d;
  return cudaSuccess;
}

// Rejection threshold of an unswap trial (App. A.1/A.2 and Algorithm 1): strict acceptance
// rejects count >= chi_old, equal acceptance rejects count >= chi_old + 1.  0 when no count
// the truncation can return reaches it (the trial must run in full).
int trial_threshold(const FlatTask& f) {
  if (!f.r->trial_only) return 0;
  pc_circuit* c = f.r->c;
  const int j = (*f.r->items)[f.k].bond;
  const int v = std::min(4 * c->chi[j], 4 * c->chi[j + 2]);
  const int k = c->chi[j + 1] + (f.r->accept_equal ? 1 : 0);
  return k <= std::min(v, c->chi_max) ? k : 0;
}

constexpr int kCertOversample = 32;
constexpr int kCertMinVectors = 128;

// Scratch of one certificate: X and T0 of the trial (m x n each), C = P X^H (r x v) with its
// FP32 copy, and the Jacobi and truncation vectors.
size_t cert_bytes(int m, int n, int r) {
  const size_t v = (size_t)std::min(m, n);
  return 2 * al256((size_t)m * n * sizeof(double2)) + al256((size_t)r * v * sizeof(double2)) +
         al256((size_t)r * v * sizeof(float2)) + 3 * al256((size_t)r * sizeof(double)) +
         3 * al256((size_t)r * sizeof(int32_t)) + al256((size_t)r * sizeof(float));
}

int cert_rows(const FlatTask& f) {
  const int k = trial_threshold(f);
  if (k == 0) return 0;
  pc_circuit* c = f.r->c;
  const int j = (*f.r->items)[f.k].bond;
  const int v = std::min(4 * c->chi[j], 4 * c->chi[j + 2]);
  const int r = k + kCertOversample;
  return (v >= kCertMinVectors && r <= v) ? r : 0;
}

// The certificate of a batch of unswap trials (Sec. II.B.2 needs only each trial's count).
// For a trial with stored matrix Xs (v vectors of length L; its singular values are those of
// the bond matrix) and threshold k: C = P Xs^H in FP64 with the fixed projection P (r = k + 32
// orthonormal rows), then the one-sided Jacobi on the r rows of C, in FP32 (fp32: C rounded to
// FP32 first) or in FP64.  Interlacing gives sigma_k(X) >= sigma_k(C) / |P|_2, and
// |P|_2 <= |P|_F.  The converged rows are J (C + dC) with J unitary, where dC holds the FP64
// product's rounding (|.|_F <= 4 gamma_L |P|_F |X|_F), the rounding to FP32 (<= u32 |C|_F, FP32
// only) and the backward error of the sweeps (<= 16 S r u |C|_F, S sweeps, u the unit roundoff
// of the sweeps; r counts the rotations of a row per sweep, ~2 r in the blocked FP32 kernel);
// their mutual cosines are below cos = tol + 3 gamma_v (the convergence test's
// tolerance plus the rounding of its inner products and norms), so by Gershgorin on the top k
// rows sigma_k >= c_k sqrt(1 - (k - 1) cos), with c_k the k-th largest converged row norm.  The
// trial is certified to keep at least k values when
//     c_k sqrt(1 - (k - 1) cos) - 4 gamma_L |P|_F |X|_F - |dC from the sweeps| > eps |X|_F |P|_F,
// since s_0 <= |X|_F.  Certified trials are rejected without factorising the bond matrix;
// the others stay resolved[] = 0.  The FP32 pass is cheap (the FP32 pipe of this part is ~60
// times its FP64 pipe) but its error term, ~6e-3 |C|_F at r = 288 and 12 sweeps, certifies only trials whose
// k-th value is well above that; the FP64 pass certifies down to ~1e-11 |C|_F.
pc_status certify_chunk(Workspace* w, std::vector<FlatTask>& flat, size_t b0, size_t b1,
                        std::vector<char>& resolved, bool fp32) {
  const int T = (int)(b1 - b0);
  cudaStream_t s = w->stream;
  size_t need = 0;
  // position i of every launch array holds task ord[i]: rows of at most 1024 elements first
  // (the blocked FP32 kernel), the longer ones after (the row-pair FP32 kernel)
  std::vector<int> ord;
  auto vec_len = [&](int t) {
    const FlatTask& f = flat[b0 + t];
    pc_circuit* c = f.r->c;
    const int j = (*f.r->items)[f.k].bond;
    return std::min(4 * c->chi[j], 4 * c->chi[j + 2]);
  };
  for (int t = 0; t < T; ++t)
    if (vec_len(t) <= 1024) ord.push_back(t);
  const int Tb = (int)ord.size();
  for (int t = 0; t < T; ++t)
    if (vec_len(t) > 1024) ord.push_back(t);
  for (int t = 0; t < T; ++t) {
    const FlatTask& f = flat[b0 + t];
    pc_circuit* c = f.r->c;
    const int j = (*f.r->items)[f.k].bond;
    need += cert_bytes(4 * c->chi[j], 4 * c->chi[j + 2], cert_rows(f));
  }
  WS_TRY(ws_reserve(w, need));
  size_t off = 0;
  auto take = [&](size_t bytes) -> void* {
    void* p = w->d_arena + off;
    off += al256(bytes);
    return p;
  };
  std::vector<MergeIn> in(T);
  std::vector<int> kk(T), rr(T), vv(T), ll(T);
  int max_r = 0, max_v = 0, max_vb = 1, max_ve = 1, pairs_e = 0, pairs_b = 0;
  for (int i = 0; i < T; ++i) {
    const FlatTask& f = flat[b0 + ord[i]];
    pc_circuit* c = f.r->c;
    const WaveItem& it = (*f.r->items)[f.k];
    const int j = it.bond;
    const int m = 4 * c->chi[j], n = 4 * c->chi[j + 2];
    const int v = std::min(m, n), L = std::max(m, n);
    const int r = cert_rows(f);
    kk[i] = trial_threshold(f); rr[i] = r; vv[i] = v; ll[i] = L;
    in[i] = {c, &it, (double2*)take((size_t)m * n * sizeof(double2)), (double2*)take((size_t)m * n * sizeof(double2))};
    double2* Cm = (double2*)take((size_t)r * v * sizeof(double2));
    double2* P = nullptr;
    WS_TRY(srft_matrix(w, L, r, &P));
    pc::GemmDesc& g = w->h_cg[i];
    g = pc::GemmDesc{};
    g.A = P; g.lda = L;
    g.B = in[i].X; g.ldb = L; g.opB = 1;     // the stored matrix: v rows of length L
    g.C = Cm; g.ldc = v;
    g.M = r; g.N = v; g.K = L; g.alpha = 1.0;
    pc::JacobiTask& jc = w->h_jc[i];
    jc = pc::JacobiTask{};
    jc.X = Cm;
    jc.Q = nullptr;
    jc.nrm2 = (double*)take((size_t)r * sizeof(double));
    jc.fro2 = w->d_cfro2 + i;
    jc.stamp = (int32_t*)take((size_t)r * sizeof(int32_t));
    jc.dead2_ovr = nullptr;
    const double dr = c->ctx->cfg.eps / (10.0 * r);
    jc.dead_rel = dr * dr;
    jc.m = r; jc.n = v; jc.mp = r + (r & 1);
    pc::JacobiTask32& j32 = w->h_j32[i];
    j32 = pc::JacobiTask32{};
    j32.X = (float2*)take((size_t)r * v * sizeof(float2));
    j32.Q = nullptr;
    j32.nrm2 = (float*)take((size_t)r * sizeof(float));
    j32.fro2 = jc.fro2;
    j32.stamp = (int32_t*)take((size_t)r * sizeof(int32_t));
    j32.dead2_ovr = nullptr;
    j32.dead_rel = jc.dead_rel;
    j32.m = jc.m; j32.n = jc.n; j32.mp = jc.mp;
    pc::TruncTask& tt = w->h_tc[i];
    tt = pc::TruncTask{};
    tt.X = Cm;
    tt.idx = (int32_t*)take((size_t)r * sizeof(int32_t));
    tt.lam = (double*)take((size_t)r * sizeof(double));
    tt.sraw = (double*)take((size_t)r * sizeof(double));
    tt.out = w->d_ctout + i;
    tt.eps = 0.0;
    tt.m = r; tt.n = v;
    tt.chi_max = kk[i];
    // the bond matrix's own Jacobi task (for |X|_F^2)
    pc::JacobiTask& jt = w->h_jt[i];
    jt = pc::JacobiTask{};
    jt.X = in[i].X; jt.m = v; jt.n = L; jt.mp = v + (v & 1);
    max_r = std::max(max_r, r); max_v = std::max(max_v, v);
    if (i < Tb) { max_vb = std::max(max_vb, v); pairs_b += jc.mp / 2; }
    else { max_ve = std::max(max_ve, v); pairs_e += jc.mp / 2; }
  }
  WS_TRY(stage_merge_gate(w, in));
  timer_mark(w, 1);
  WS_TRY(cudaMemcpyAsync(w->d_jt, w->h_jt, T * sizeof(pc::JacobiTask), cudaMemcpyHostToDevice, s));
  WS_TRY(cudaMemcpyAsync(w->d_cg, w->h_cg, T * sizeof(pc::GemmDesc), cudaMemcpyHostToDevice, s));
  WS_TRY(cudaMemcpyAsync(w->d_jc, w->h_jc, T * sizeof(pc::JacobiTask), cudaMemcpyHostToDevice, s));
  WS_TRY(cudaMemcpyAsync(w->d_j32, w->h_j32, T * sizeof(pc::JacobiTask32), cudaMemcpyHostToDevice, s));
  WS_TRY(cudaMemcpyAsync(w->d_tc, w->h_tc, T * sizeof(pc::TruncTask), cudaMemcpyHostToDevice, s));
  WS_TRY(pc::launch_fro2(w->d_jt, T, w->d_fro2, s));
  WS_TRY(pc::launch_gemm(w->d_cg, T, max_r, max_v, s));
  WS_TRY(pc::launch_fro2(w->d_jc, T, w->d_cfro2, s));
  WS_TRY(cudaMemsetAsync(w->d_jst3, 0, T * sizeof(pc::JacobiStatus), s));
  int max_sweeps = 1;
  for (int t = 0; t < T; ++t) max_sweeps = std::max(max_sweeps, flat[b0 + t].r->c->ctx->cfg.jacobi_max_sweeps);
  if (fp32) {
    WS_TRY(pc::launch_narrow_rows(w->d_jc, w->d_j32, T, max_r, max_v, s));
    WS_TRY(pc::launch_init_stamps32(w->d_j32, T, max_r, s));
    if (Tb > 0) {
      WS_TRY(cudaMemsetAsync(w->d_bar, 0, 2 * sizeof(unsigned int), s));
      WS_TRY(pc::launch_jacobi32_blocked(w->d_j32, Tb, w->d_jst3, max_sweeps, w->d_bar, w->d_err, w->sm_count,
                                         max_vb, s));
    }
    if (T > Tb) {
      WS_TRY(cudaMemsetAsync(w->d_bar, 0, 2 * sizeof(unsigned int), s));
      WS_TRY(pc::launch_jacobi32(w->d_j32 + Tb, T - Tb, w->d_jst3 + Tb, max_sweeps, w->d_bar, w->d_err, w->sm_count,
                                 max_ve, pairs_e, s));
    }
    WS_TRY(pc::launch_widen_rows(w->d_j32, w->d_jc, T, max_r, max_v, s));
  } else {
    WS_TRY(pc::launch_init_stamps(w->d_jc, T, max_r, s));
    WS_TRY(cudaMemsetAsync(w->d_bar, 0, 2 * sizeof(unsigned int), s));
    WS_TRY(pc::launch_jacobi(w->d_jc, T, w->d_jst3, max_sweeps, w->d_bar, w->d_err, w->sm_count, max_v,
                             pairs_e + pairs_b, s));
  }
  WS_TRY(pc::launch_truncate_tasks(w->d_tc, T, s));
  timer_mark(w, 2);
  w->t_launch[5] += fp32 ? 3 + (Tb > 0) + (T > Tb) : 3;
  w->t_launch[4] += fp32 ? 4 : 3;
  WS_TRY(cudaMemcpyAsync(w->h_ctout, w->d_ctout, T * sizeof(pc::TruncOut), cudaMemcpyDeviceToHost, s));
  WS_TRY(cudaMemcpyAsync(w->h_jst3, w->d_jst3, T * sizeof(pc::JacobiStatus), cudaMemcpyDeviceToHost, s));
  WS_TRY(cudaMemcpyAsync(w->h_fro2, w->d_fro2, T * sizeof(double), cudaMemcpyDeviceToHost, s));
  WS_TRY(cudaMemcpyAsync(w->h_cfro2, w->d_cfro2, T * sizeof(double), cudaMemcpyDeviceToHost, s));
  WS_TRY(cudaMemcpyAsync(w->h_err, w->d_err, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  WS_TRY(cudaStreamSynchronize(s));
  if (w->timing) {
    float a = 0, b = 0;
    cudaEventElapsedTime(&a, w->ev[0], w->ev[1]);
    cudaEventElapsedTime(&b, w->ev[1], w->ev[2]);
    w->t_ms[0] += a;
    w->t_ms[5] += b;
  }
  for (int i = 0; i < T; ++i)   // the FP64 projection GEMM and the rotations of the sweeps
    w->t_flops[5] += 8.0 * rr[i] * (double)vv[i] * ll[i] + 12.0 * w->h_jst3[i].sweeps * (double)rr[i] * rr[i] * vv[i];
  if (w->h_err[0]) return chunk_fail(flat, b0, b1, PC_ERR_TIMEOUT, "Jacobi grid barrier wait exceeded its limit");
  if (w->h_err[1]) return chunk_fail(flat, b0, b1, PC_ERR_TIMEOUT, "a tensor-core merge wait exceeded its limit");
  const double u = 1.1102230246251565e-16;      // FP64 unit roundoff, 2^-53
  const double us = fp32 ? 5.9604644775390625e-08 : u;   // unit roundoff of the sweeps (FP32: 2^-24)
  for (int i = 0; i < T; ++i) {
    const FlatTask& f = flat[b0 + ord[i]];
    const pc::TruncOut& o = w->h_ctout[i];
    const pc::JacobiStatus& js = w->h_jst3[i];
    const int k = kk[i], r = rr[i], L = ll[i], v = vv[i];
    const double xf = std::sqrt(std::max(0.0, w->h_fro2[i])), cf = std::sqrt(std::max(0.0, w->h_cfro2[i]));
    const double pf = std::sqrt((double)r) * (1.0 + 1e-12);
    const double gam = L * u / (1.0 - L * u);
    const double gam_v = v * us / (1.0 - v * us);
    const double cosb = 2.0 * (2.0 * us) * std::sqrt((double)v) + 3.0 * gam_v;   // tol = 2 eps sqrt(v), eps = 2 u
    const double dead = std::sqrt(w->h_jc[i].dead_rel) * cf, marg = std::sqrt(6.0 * r) * dead;
    const double ck = o.s_last_kept;
    // rotations a row takes part in per sweep: r - 1 in the row-pair kernel; in the blocked FP32
    // kernel 15 per block round (the inner sweep over its 16-row block pair), ceil(r / 8) rounds
    const double rot = (fp32 && i < Tb) ? 15.0 * ((r + 7) / 8 + 1) : (double)r;
    const double lower = ck * std::sqrt(std::max(0.0, 1.0 - (k - 1) * cosb)) - 4.0 * gam * pf * xf -
                         ((fp32 ? 1.0 : 0.0) + 16.0 * js.sweeps * rot) * us * cf;
    const double eps = f.r->c->ctx->cfg.eps;
    const bool ok = js.converged && o.count == k && ck > marg && lower > eps * xf * pf;
    if (ok) {
      resolved[b0 + ord[i]] = 1;
      f.r->counts[f.k] = k;
      f.r->accepted[f.k] = 0;
      f.r->c->stats.n_trials_certified += 1;
      f.r->c->stats.alg_flops += 4.0 * (4.0 * (double)L * v * v - 4.0 * (double)v * v * v / 3.0);
    }
  }
  w->n_launches += 1;
  w->n_tasks += T;
  return PC_OK;
}

// Factorises and commits the tasks flat[b0, b1) in one set of launches on w->stream.
pc_status run_chunk(Workspace* w, std::vector<FlatTask>& flat, size_t b0, size_t b1) {
  const int T = (int)(b1 - b0);
  cudaStream_t s = w->stream;
  std::vector<TaskScratch> sc(T);
  std::vector<char> precond(T, 0);
  std::vector<int> m_of(T), n_of(T), v_of(T), bond_of(T);
  size_t need = 0;
  for (int t = 0; t < T; ++t) {
    const FlatTask& f = flat[b0 + t];
    pc_circuit* c = f.r->c;
    const int j = (*f.r->items)[f.k].bond;
    const int m = 4 * c->chi[j], n = 4 * c->chi[j + 2];
    precond[t] = c->ctx->cfg.fp32_precondition && std::min(m, n) >= 64;
    need += task_bytes(m, n, precond[t]);
  }
  WS_TRY(ws_reserve(w, need));
  size_t off = 0;
  auto take = [&](size_t bytes) -> void* {
    void* p = w->d_arena + off;
    off += al256(bytes);
    return p;
  };
  int max_v = 0, max_len = 0, total_pairs = 0;
  std::vector<MergeIn> min_(T);
  for (int t = 0; t < T; ++t) {
    const FlatTask& f = flat[b0 + t];
    pc_circuit* c = f.r->c;
    const WaveItem& it = (*f.r->items)[f.k];
    const int j = it.bond;
    const int cl = c->chi[j], cr = c->chi[j + 2];
    const int m = 4 * cl, n = 4 * cr, v = std::min(m, n), L = std::max(m, n);
    const bool transposed = m > n;
    m_of[t] = m; n_of[t] = n; v_of[t] = v; bond_of[t] = j;
    TaskScratch& x = sc[t];
    x.X = (double2*)take((size_t)m * n * sizeof(double2));
    x.T0 = (double2*)take((size_t)m * n * sizeof(double2));
    x.Q = (double2*)take((size_t)v * v * sizeof(double2));
    x.nrm2 = (double*)take((size_t)v * sizeof(double));
    x.lam = (double*)take((size_t)v * sizeof(double));
    x.sraw = (double*)take((size_t)v * sizeof(double));
    x.idx = (int32_t*)take((size_t)v * sizeof(int32_t));
    x.stamp = (int32_t*)take((size_t)v * sizeof(int32_t));
    if (precond[t]) {
      x.stamp32 = (int32_t*)take((size_t)v * sizeof(int32_t));
      x.X32 = (float2*)take((size_t)m * n * sizeof(float2));
      x.Q32 = (float2*)take((size_t)v * v * sizeof(float2));
      x.Qb = (double2*)take((size_t)v * v * sizeof(double2));
      x.Y = (double2*)take((size_t)m * n * sizeof(double2));
    }
    min_[t] = {c, &it, x.X, x.T0};
    // The Jacobi orthogonalises min(m, n) vectors: the rows of X, or for a tall bond matrix
    // its columns, with the rotations accumulated into Q (the right singular vectors).
    pc::JacobiTask& jt = w->h_jt[t];
    jt.X = x.X;
    jt.Q = transposed ? x.Q : nullptr;
    jt.nrm2 = x.nrm2;
    jt.fro2 = w->d_fro2 + t;
    jt.stamp = x.stamp;
    jt.dead2_ovr = nullptr;
    jt.m = v;
    jt.n = L;
    jt.mp = v + (v & 1);
    jt.pad_ = 0;
    const double r = c->ctx->cfg.eps / (10.0 * v);
    jt.dead_rel = r * r;
    pc::TruncTask& tt = w->h_tt[t];
    tt.X = precond[t] ? x.Y : x.X;
    tt.idx = x.idx; tt.lam = x.lam; tt.sraw = x.sraw;
    tt.out = w->d_tout + t;
    tt.eps = c->ctx->cfg.eps;
    tt.m = v; tt.n = L;
    tt.chi_max = c->chi_max;
    tt.pad_ = 0;
    max_v = std::max(max_v, v);
    max_len = std::max(max_len, L);
    total_pairs += jt.mp / 2;
    w->t_flops[1] += 4.0 * (4.0 * (double)L * L * v + 22.0 * (double)v * v * v);
    c->stats.n_full += 1;
    c->stats.alg_flops += f.r->trial_only ? 4.0 * (4.0 * (double)L * v * v - 4.0 * (double)v * v * v / 3.0)
                                          : 4.0 * (4.0 * (double)L * L * v + 22.0 * (double)v * v * v);
  }
  WS_TRY(stage_merge_gate(w, min_));
  WS_TRY(cudaMemcpyAsync(w->d_jt, w->h_jt, T * sizeof(pc::JacobiTask), cudaMemcpyHostToDevice, s));
  WS_TRY(cudaMemcpyAsync(w->d_tt, w->h_tt, T * sizeof(pc::TruncTask), cudaMemcpyHostToDevice, s));
  timer_mark(w, 1);
  WS_TRY(pc::launch_fro2(w->d_jt, T, w->d_fro2, s));
  WS_TRY(pc::launch_init_accumulators(w->d_jt, T, max_v, s));
  w->t_launch[1] += 1;
  w->t_launch[4] += 1;
  // FP32 preconditioning of the tasks with enough vectors: FP32 sweeps with the rotations
  // accumulated in Q32; Q = polar(Q32) in FP64 by two Newton-Schulz steps
  // Q <- 1.5 Q - 0.5 (Q Q^H) Q; Y = Q X; then the FP64 sweeps run on Y.
  // Each task's FP32 kernel is chosen by its own row length (blocked: rows in shared memory up
  // to length 1024), so a task is factorised the same way alone and in any batch.
  auto blocked32 = [&](int t) { return w->h_jt[t].n <= 1024; };
  std::vector<int> psub;
  for (int t = 0; t < T; ++t)
    if (precond[t] && blocked32(t)) psub.push_back(t);
  const int P32b = (int)psub.size();
  for (int t = 0; t < T; ++t)
    if (precond[t] && !blocked32(t)) psub.push_back(t);
  const int P = (int)psub.size();
  int pv = 0, pl = 0, ppairs = 0;
  for (int i = 0; i < P; ++i) {
    const int t = psub[i];
    const pc::JacobiTask& jt = w->h_jt[t];
    const TaskScratch& x = sc[t];
    w->h_jsub[i] = jt;
    pc::JacobiTask32& j32 = w->h_j32[i];
    j32.X = x.X32;
    j32.Q = x.Q32;
    j32.nrm2 = reinterpret_cast<float*>(x.nrm2);
    j32.fro2 = jt.fro2;
    j32.stamp = x.stamp32;
    j32.dead2_ovr = nullptr;
    {
      // FP32 noise: a preconditioner may skip any pair below its floor
      const double fr = flat[b0 + t].r->c->ctx->cfg.fp32_dead_rel;
      j32.dead_rel = fr > 0.0 ? fr : 1e-12 / jt.m;
    }
    j32.m = jt.m; j32.n = jt.n; j32.mp = jt.mp; j32.pad_ = 0;
    w->h_q64[i] = x.Q;
    const int v = jt.m, L = jt.n;
    double2 *QA = x.Q, *QB = x.Qb, *Y = x.Y;
    auto gd = [&](int stage) -> pc::GemmDesc& { return w->h_ns[stage * P + i]; };
    for (int k = 0; k < 5; ++k) gd(k) = pc::GemmDesc{};
    gd(0).A = QA; gd(0).lda = v; gd(0).B = QA; gd(0).ldb = v; gd(0).opB = 1; gd(0).C = Y; gd(0).ldc = v;
    gd(0).M = v; gd(0).N = v; gd(0).K = v; gd(0).alpha = 1.0;
    gd(1).A = Y; gd(1).lda = v; gd(1).B = QA; gd(1).ldb = v; gd(1).C = QB; gd(1).ldc = v; gd(1).D = QA;
    gd(1).M = v; gd(1).N = v; gd(1).K = v; gd(1).alpha = -0.5; gd(1).beta = 1.5;
    gd(2).A = QB; gd(2).lda = v; gd(2).B = QB; gd(2).ldb = v; gd(2).opB = 1; gd(2).C = Y; gd(2).ldc = v;
    gd(2).M = v; gd(2).N = v; gd(2).K = v; gd(2).alpha = 1.0;
    gd(3).A = Y; gd(3).lda = v; gd(3).B = QB; gd(3).ldb = v; gd(3).C = QA; gd(3).ldc = v; gd(3).D = QB;
    gd(3).M = v; gd(3).N = v; gd(3).K = v; gd(3).alpha = -0.5; gd(3).beta = 1.5;
    gd(4).A = QA; gd(4).lda = v; gd(4).B = jt.X; gd(4).ldb = L; gd(4).C = Y; gd(4).ldc = L;
    gd(4).M = v; gd(4).N = L; gd(4).K = v; gd(4).alpha = 1.0;
    pv = std::max(pv, v); pl = std::max(pl, L);
    ppairs += jt.mp / 2;
  }
  if (P > 0) {
    WS_TRY(cudaMemcpyAsync(w->d_jsub, w->h_jsub, P * sizeof(pc::JacobiTask), cudaMemcpyHostToDevice, s));
    WS_TRY(cudaMemcpyAsync(w->d_j32, w->h_j32, P * sizeof(pc::JacobiTask32), cudaMemcpyHostToDevice, s));
    WS_TRY(cudaMemcpyAsync(w->d_q64, w->h_q64, P * sizeof(double2*), cudaMemcpyHostToDevice, s));
    WS_TRY(cudaMemcpyAsync(w->d_ns, w->h_ns, 5 * (size_t)P * sizeof(pc::GemmDesc), cudaMemcpyHostToDevice, s));
    WS_TRY(cudaMemsetAsync(w->d_jst + w->cap, 0, P * sizeof(pc::JacobiStatus), s));
    WS_TRY(cudaMemsetAsync(w->d_bar, 0, 2 * sizeof(unsigned int), s));
    WS_TRY(pc::launch_precond_init(w->d_jsub, w->d_j32, P, pv, pl, s));
    WS_TRY(pc::launch_init_stamps32(w->d_j32, P, pv, s));
    int pre_sweeps = 1;
    for (int i = 0; i < P; ++i)
      pre_sweeps = std::max(pre_sweeps, flat[b0 + psub[i]].r->c->ctx->cfg.precondition_sweeps);
    int pl_b = 1, pl_e = 1, pairs_e = 0;
    for (int i = 0; i < P; ++i) {
      const pc::JacobiTask& jt = w->h_jt[psub[i]];
      if (i < P32b) pl_b = std::max(pl_b, jt.n);
      else { pl_e = std::max(pl_e, jt.n); pairs_e += jt.mp / 2; }
    }
    if (P32b > 0)
      WS_TRY(pc::launch_jacobi32_blocked(w->d_j32, P32b, w->d_jst + w->cap, pre_sweeps, w->d_bar, w->d_err,
                                         w->sm_count, pl_b, s));
    if (P > P32b) {
      WS_TRY(cudaMemsetAsync(w->d_bar, 0, 2 * sizeof(unsigned int), s));
      WS_TRY(pc::launch_jacobi32(w->d_j32 + P32b, P - P32b, w->d_jst + w->cap + P32b, pre_sweeps, w->d_bar, w->d_err,
                                 w->sm_count, pl_e, pairs_e, s));
    }
    WS_TRY(pc::launch_widen_q(w->d_j32, w->d_q64, P, pv, s));
    for (int k = 0; k < 4; ++k) WS_TRY(pc::launch_gemm(w->d_ns + k * P, P, pv, pv, s));
    WS_TRY(pc::launch_gemm(w->d_ns + 4 * P, P, pv, pl, s));
    w->t_launch[1] += 8;
  }
  // Deflation floors of the FP64 sweeps (tasks with more vectors than chi_max, FP32 rows
  // available): set on the device from the FP32 row norms, verified after the sweeps.
  std::vector<char> defl(T, 0);
  WS_TRY(cudaMemsetAsync(w->d_dead2, 0, 2 * (size_t)w->cap * sizeof(double), s));
  {
    int nd = 0;
    for (int i = 0; i < P; ++i) {
      const int t = psub[i];
      pc_circuit* c = flat[b0 + t].r->c;
      if (!c->ctx->cfg.deflate || v_of[t] <= c->chi_max) continue;
      pc::DeflateTask& d = w->h_df[nd++];
      d.X32 = sc[t].X32;
      d.fro2 = w->d_fro2 + t;
      d.dead2_out = w->d_dead2 + t;
      d.sc_out = w->d_dead2 + w->cap + t;
      d.m = v_of[t];
      d.n = w->h_jt[t].n;
      d.chi_max = c->chi_max;
      d.pad_ = 0;
      defl[t] = 1;
    }
    if (nd > 0) {
      WS_TRY(cudaMemcpyAsync(w->d_df, w->h_df, nd * sizeof(pc::DeflateTask), cudaMemcpyHostToDevice, s));
      WS_TRY(pc::launch_deflate_floor(w->d_df, nd, s));
      w->t_launch[1] += 1;
    }
  }
  // FP64 sweeps: on Y = Q X for the preconditioned tasks (accumulating into Q on the column
  // path), on X itself for the others
  for (int t = 0; t < T; ++t) {
    w->h_jy[t] = w->h_jt[t];
    if (precond[t]) w->h_jy[t].X = sc[t].Y;
    if (defl[t]) w->h_jy[t].dead2_ovr = w->d_dead2 + t;
  }
  WS_TRY(cudaMemcpyAsync(w->d_jy, w->h_jy, T * sizeof(pc::JacobiTask), cudaMemcpyHostToDevice, s));
  WS_TRY(cudaMemsetAsync(w->d_jst, 0, T * sizeof(pc::JacobiStatus), s));
  WS_TRY(cudaMemsetAsync(w->d_bar, 0, 2 * sizeof(unsigned int), s));
  int max_sweeps = 1;
  for (int t = 0; t < T; ++t) max_sweeps = std::max(max_sweeps, flat[b0 + t].r->c->ctx->cfg.jacobi_max_sweeps);
  WS_TRY(pc::launch_init_stamps(w->d_jy, T, max_v, s));
  // FP64 sweeps: the row-pair kernel (FP64-pipe bound; a blocked variant with rows in shared
  // memory measured slower: its exact per-pair norms double the FP64 work of a check)
  WS_TRY(pc::launch_jacobi(w->d_jy, T, w->d_jst, max_sweeps, w->d_bar, w->d_err, w->sm_count, max_len, total_pairs, s));
  w->t_launch[1] += 1;
  timer_mark(w, 2);
  WS_TRY(pc::launch_truncate_tasks(w->d_tt, T, s));
  w->t_launch[2] += 1;
  timer_mark(w, 3);
  WS_TRY(cudaMemcpyAsync(w->h_tout, w->d_tout, T * sizeof(pc::TruncOut), cudaMemcpyDeviceToHost, s));
  WS_TRY(cudaMemcpyAsync(w->h_jst, w->d_jst, T * sizeof(pc::JacobiStatus), cudaMemcpyDeviceToHost, s));
  WS_TRY(cudaMemcpyAsync(w->h_err, w->d_err, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  WS_TRY(cudaMemcpyAsync(w->h_fro2, w->d_fro2, T * sizeof(double), cudaMemcpyDeviceToHost, s));
  WS_TRY(cudaMemcpyAsync(w->h_dead2, w->d_dead2, T * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (P > 0)
    WS_TRY(cudaMemcpyAsync(w->h_jst + w->cap, w->d_jst + w->cap, P * sizeof(pc::JacobiStatus), cudaMemcpyDeviceToHost, s));
  WS_TRY(cudaStreamSynchronize(s));
  for (int i = 0; i < P; ++i) {
    pc_circuit* c = flat[b0 + psub[i]].r->c;
    c->stats.max_sweeps_fp32 = std::max(c->stats.max_sweeps_fp32, w->h_jst[w->cap + i].sweeps);
  }

  if (w->timing) {
    float a = 0, b = 0, d = 0;
    cudaEventElapsedTime(&a, w->ev[0], w->ev[1]);
    cudaEventElapsedTime(&b, w->ev[1], w->ev[2]);
    cudaEventElapsedTime(&d, w->ev[2], w->ev[3]);
    w->t_ms[0] += a; w->t_ms[1] += b; w->t_ms[2] += d;
  }
  if (w->h_err[0]) return chunk_fail(flat, b0, b1, PC_ERR_TIMEOUT, "Jacobi grid barrier wait exceeded its limit");
  if (w->h_err[1]) return chunk_fail(flat, b0, b1, PC_ERR_TIMEOUT, "a tensor-core merge wait exceeded its limit");
  // Safety net of the preconditioning: Q X must keep the Frobenius norm of X (Q unitary).
  // A task that fails the check is factorised again in FP64 only, from its merged matrix.
  std::vector<int> redo;
  for (int t = 0; t < T; ++t) {
    if (!precond[t]) continue;
    const double x2 = w->h_fro2[t], y2 = w->h_tout[t].total2;
    bool ok = std::fabs(y2 - x2) <= 1e-9 * x2;
    // A deflated task is exact when it kept chi_max values and the smallest kept value lies
    // above the Frobenius bound sqrt(6) m sqrt(dead2) of the block below the second floor.
    const double d2 = w->h_dead2[t];
    if (ok && d2 > 0.0) {
      pc_circuit* c = flat[b0 + t].r->c;
      const pc::TruncOut& o = w->h_tout[t];
      ok = o.count == c->chi_max && o.s_last_kept > 1.01 * std::sqrt(6.0) * v_of[t] * std::sqrt(d2);
      if (ok) c->stats.n_deflated += 1;
    }
    if (!ok) redo.push_back(t);
  }
  std::vector<double2*> final_x(T);
  for (int t = 0; t < T; ++t) final_x[t] = precond[t] ? sc[t].Y : sc[t].X;
  if (!redo.empty()) {
    const int R = (int)redo.size();
    int rv = 0, rl = 0, rpairs = 0;
    for (int i = 0; i < R; ++i) {
      const int t = redo[i];
      w->h_jfb[i] = w->h_jt[t];
      w->h_tt[w->cap + i] = w->h_tt[t];
      w->h_tt[w->cap + i].X = sc[t].X;
      final_x[t] = sc[t].X;
      rv = std::max(rv, w->h_jt[t].m); rl = std::max(rl, w->h_jt[t].n);
      rpairs += w->h_jt[t].mp / 2;
      flat[b0 + t].r->c->stats.fallbacks += 1;
    }
    WS_TRY(cudaMemcpyAsync(w->d_jfb, w->h_jfb, R * sizeof(pc::JacobiTask), cudaMemcpyHostToDevice, s));
    WS_TRY(cudaMemcpyAsync(w->d_tt + w->cap, w->h_tt + w->cap, R * sizeof(pc::TruncTask), cudaMemcpyHostToDevice, s));
    WS_TRY(cudaMemsetAsync(w->d_jst + w->cap, 0, R * sizeof(pc::JacobiStatus), s));
    WS_TRY(cudaMemsetAsync(w->d_bar, 0, 2 * sizeof(unsigned int), s));
    WS_TRY(pc::launch_init_accumulators(w->d_jfb, R, rv, s));
    WS_TRY(pc::launch_init_stamps(w->d_jfb, R, rv, s));
    WS_TRY(pc::launch_jacobi(w->d_jfb, R, w->d_jst + w->cap, max_sweeps, w->d_bar, w->d_err, w->sm_count, rl, rpairs, s));
    WS_TRY(pc::launch_truncate_tasks(w->d_tt + w->cap, R, s));
    w->t_launch[1] += 1; w->t_launch[2] += 1; w->t_launch[4] += 1;
    WS_TRY(cudaMemcpyAsync(w->h_tout, w->d_tout, T * sizeof(pc::TruncOut), cudaMemcpyDeviceToHost, s));
    WS_TRY(cudaMemcpyAsync(w->h_jst + w->cap, w->d_jst + w->cap, R * sizeof(pc::JacobiStatus), cudaMemcpyDeviceToHost, s));
    WS_TRY(cudaMemcpyAsync(w->h_err, w->d_err, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    WS_TRY(cudaStreamSynchronize(s));
    if (w->h_err[0]) return chunk_fail(flat, b0, b1, PC_ERR_TIMEOUT, "Jacobi grid barrier wait exceeded its limit");
    for (int i = 0; i < R; ++i) w->h_jst[redo[i]] = w->h_jst[w->cap + i];
  }
  // counts, convergence and commit decisions
  std::vector<char> commit(T, 0);
  for (int t = 0; t < T; ++t) {
    const FlatTask& f = flat[b0 + t];
    pc_circuit* c = f.r->c;
    const int cnt = w->h_tout[t].count;
    f.r->counts[f.k] = cnt;
    c->stats.max_sweeps = std::max(c->stats.max_sweeps, w->h_jst[t].sweeps);
    if (!w->h_jst[t].converged) {
      const pc::JacobiStatus& js = w->h_jst[t];
      f.r->status = fail(c->ctx, PC_ERR_NOCONVERGE,
                         "one-sided Jacobi reached the sweep cap on bond " + std::to_string(bond_of[t]) + " (" +
                             std::to_string(m_of[t]) + " x " + std::to_string(n_of[t]) + ", " +
                             std::to_string(js.sweeps) + " sweeps, rotations in the last three: " +
                             std::to_string(js.rot[0]) + " " + std::to_string(js.rot[1]) + " " +
                             std::to_string(js.rot[2]) + ")");
      continue;
    }
    bool ok = f.r->commit_mask ? (*f.r->commit_mask)[f.k] != 0 : true;
    if (f.r->decide_by_accept) {
      const int old = c->chi[bond_of[t] + 1];
      ok = f.r->accept_equal ? (cnt <= old) : (cnt < old);
    }
    f.r->accepted[f.k] = ok ? 1 : 0;
    commit[t] = ok && f.r->status == PC_OK;
  }
  int nc = 0, max_cnt = 0, max_nn = 0, max_mm = 0;
  for (int t = 0; t < T; ++t) {
    if (!commit[t]) continue;
    pc_circuit* c = flat[b0 + t].r->c;
    const int j = bond_of[t];
    const int cnt = w->h_tout[t].count;
    const int m = m_of[t], n = n_of[t];
    pc::SplitRowsDesc& sd = w->h_split[nc];
    sd.X = final_x[t];
    sd.Q = m > n ? sc[t].Q : nullptr;
    sd.dst = site_ptr(c, j + 1);
    sd.idx = sc[t].idx;
    sd.sraw = sc[t].sraw;
    sd.count = cnt;
    sd.n = n;
    pc::GemmDesc& g = w->h_gemm2[nc];
    g = pc::GemmDesc{};
    g.A = sc[t].T0; g.B = sd.dst; g.C = site_ptr(c, j); g.row_scale = nullptr;
    g.M = m; g.N = cnt; g.K = n;
    g.lda = n; g.ldb = n; g.ldc = cnt;
    g.opB = 1; g.alpha = 1.0 / w->h_tout[t].nrm; g.beta = 0.0; g.D = nullptr;
    max_cnt = std::max(max_cnt, cnt); max_nn = std::max(max_nn, n); max_mm = std::max(max_mm, m);
    w->t_flops[3] += 8.0 * m * (double)n * cnt;
    ++nc;
  }
  if (nc > 0) {
    timer_mark(w, 4);
    WS_TRY(cudaMemcpyAsync(w->d_split, w->h_split, nc * sizeof(pc::SplitRowsDesc), cudaMemcpyHostToDevice, s));
    WS_TRY(cudaMemcpyAsync(w->d_gemm2, w->h_gemm2, nc * sizeof(pc::GemmDesc), cudaMemcpyHostToDevice, s));
    WS_TRY(pc::launch_split_rows(w->d_split, nc, max_cnt, max_nn, s));
    WS_TRY(pc::launch_gemm(w->d_gemm2, nc, max_mm, max_cnt, s));
    w->t_launch[3] += 2;
    for (int t = 0; t < T; ++t) {
      if (!commit[t]) continue;
      pc_circuit* c = flat[b0 + t].r->c;
      const int j = bond_of[t];
      WS_TRY(cudaMemcpyAsync(lam_ptr(c, j), sc[t].lam, w->h_tout[t].count * sizeof(double), cudaMemcpyDeviceToDevice, s));
      c->chi[j + 1] = w->h_tout[t].count;
    }
    timer_mark(w, 5);
    if (w->timing) {
      WS_TRY(cudaStreamSynchronize(s));
      float e = 0;
      cudaEventElapsedTime(&e, w->ev[4], w->ev[5]);
      w->t_ms[3] += e;
    }
  }
  // circuits with their own stream read these sites next: finish before returning to them
  bool foreign = false;
  for (int t = 0; t < T; ++t) foreign |= flat[b0 + t].r->c->stream != s;
  if (foreign) WS_TRY(cudaStreamSynchronize(s));
  w->n_launches += 1;
  w->n_tasks += T;
  w->max_tasks_seen = std::max(w->max_tasks_seen, T);
  return PC_OK;
}

// Runs the waves of several circuits together (their items are pairwise disjoint within
// each circuit; circuits share nothing), in chunks that fit the workspace.
pc_status execute_waves(Workspace* w, std::vector<WaveReq*>& reqs) {
  std::vector<FlatTask> all;
  for (WaveReq* r : reqs) {
    r->status = PC_OK;
    r->counts.assign(r->items->size(), 0);
    r->accepted.assign(r->items->size(), 0);
    for (int k = 0; k < (int)r->items->size(); ++k) all.push_back({r, k});
  }
  pc_status worst = PC_OK;
  // unswap trials with a rejection threshold first go through the certificate
  std::vector<FlatTask> cand;
  for (const FlatTask& f : all)
    if (f.r->c->ctx->cfg.certify_trials && cert_rows(f) > 0) cand.push_back(f);
  std::vector<char> resolved(cand.size(), 0);
  // two passes: FP32 sweeps on every candidate, then FP64 sweeps on the ones the FP32 bound left
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<FlatTask> sub;
    std::vector<size_t> at;
    for (size_t i = 0; i < cand.size(); ++i)
      if (!resolved[i]) { sub.push_back(cand[i]); at.push_back(i); }
    std::vector<char> res(sub.size(), 0);
    for (size_t pos = 0; pos < sub.size();) {
      size_t end = pos, need = 0;
      while (end < sub.size() && (int)(end - pos) < w->cap) {
        const FlatTask& f = sub[end];
        pc_circuit* c = f.r->c;
        const int j = (*f.r->items)[f.k].bond;
        const size_t b = cert_bytes(4 * c->chi[j], 4 * c->chi[j + 2], cert_rows(f));
        if (need + b > w->arena_limit && end > pos) break;
        need += b;
        ++end;
      }
      pc_status st = certify_chunk(w, sub, pos, end, res, pass == 0);
      if (st != PC_OK) worst = st;
      pos = end;
    }
    for (size_t i = 0; i < sub.size(); ++i)
      if (res[i]) resolved[at[i]] = 1;
  }
  std::vector<FlatTask> flat;
  {
    size_t ci = 0;
    for (const FlatTask& f : all) {
      if (ci < cand.size() && cand[ci].r == f.r && cand[ci].k == f.k) {
        if (!resolved[ci++]) flat.push_back(f);
      } else {
        flat.push_back(f);
      }
    }
  }
  size_t pos = 0;
  while (pos < flat.size()) {
    size_t end = pos, need = 0;
    while (end < flat.size() && (int)(end - pos) < w->cap) {
      const FlatTask& f = flat[end];
      pc_circuit* c = f.r->c;
      const int j = (*f.r->items)[f.k].bond;
      const int m = 4 * c->chi[j], n = 4 * c->chi[j + 2];
      const size_t b = task_bytes(m, n, c->ctx->cfg.fp32_precondition && std::min(m, n) >= 64);
      if (need + b > w->arena_limit && end > pos) break;
      need += b;
      ++end;
    }
    pc_status st = run_chunk(w, flat, pos, end);
    if (st != PC_OK) worst = st;
    pos = end;
  }
  for (WaveReq* r : reqs) {
    r->c->stats.n_waves += 1;
    r->c->stats.max_chi = std::max(r->c->stats.max_chi, max_bond(r->c));
    r->c->projected = false;
  }
  return worst;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Batch launcher: circuits attached to a batch post their waves here; one host thread
// combines the waves posted by every participating circuit into one set of launches.
struct pc_batch {
  pc_ctx* ctx = nullptr;
  Workspace* ws = nullptr;
  std::mutex mu;
  std::condition_variable cv_post, cv_done;
  std::vector<WaveReq*> pending;
  int participants = 0;           // circuits inside a contraction that will post waves
  bool stop = false;
  double window_s = 0.002;        // longest wait for the remaining participants' waves
  std::thread launcher;
};

namespace {

void batch_loop(pc_batch* b) {
  cudaSetDevice(b->ctx->cfg.device);
  std::unique_lock<std::mutex> lk(b->mu);
  for (;;) {
    b->cv_post.wait(lk, [&] { return b->stop || !b->pending.empty(); });
    if (b->pending.empty()) break;   // stop requested and nothing left
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(b->window_s);
    b->cv_post.wait_until(lk, deadline, [&] { return b->stop || (int)b->pending.size() >= b->participants; });
    std::vector<WaveReq*> reqs;
    reqs.swap(b->pending);
    lk.unlock();
    execute_waves(b->ws, reqs);
    lk.lock();
    for (WaveReq* r : reqs) r->done = true;
    b->cv_done.notify_all();
  }
}

void batch_enter(pc_batch* b) {
  std::lock_guard<std::mutex> lk(b->mu);
  b->participants += 1;
}

void batch_leave(pc_batch* b) {
  {
    std::lock_guard<std::mutex> lk(b->mu);
    b->participants -= 1;
  }
  b->cv_post.notify_all();
}

// One circuit's wave: through its batch launcher if attached, else on its own workspace.
pc_status run_wave(pc_circuit* c, const std::vector<WaveItem>& items, std::vector<int>& counts,
                   const std::vector<int>* commit_mask, bool decide_by_accept, bool accept_equal,
                   std::vector<int>* accepted_out, bool trial_only = false) {
  counts.assign(items.size(), 0);
  if (items.empty()) return PC_OK;
  if ((int)items.size() > c->max_tasks) return fail(c->ctx, PC_ERR_INVALID_ARG, "wave wider than the task limit");
  WaveReq req;
  req.c = c;
  req.items = &items;
  req.commit_mask = commit_mask;
  req.decide_by_accept = decide_by_accept;
  req.accept_equal = accept_equal;
  req.trial_only = trial_only;
  pc_status st;
  if (c->batch) {
    pc_batch* b = c->batch;
    // the circuit's own stream may still hold copies into its sites (restore, set-up)
    CUDA_TRY(c->ctx, cudaStreamSynchronize(c->stream));
    std::unique_lock<std::mutex> lk(b->mu);
    b->pending.push_back(&req);
    b->cv_post.notify_all();
    b->cv_done.wait(lk, [&] { return req.done; });
    st = req.status;
  } else {
    st = private_workspace(c);
    if (st != PC_OK) return st;
    std::vector<WaveReq*> one{&req};
    execute_waves(c->ws, one);
    st = req.status;
  }
  counts = req.counts;
  if (accepted_out) *accepted_out = req.accepted;
  return st;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// The planner proper.  Orientation is resolved at planning time (the layout right after a
// gate's own routing), so a planned op carries its final 16x16 operator.
namespace {

struct ResolvedOp {
  int side, bond, kind, gate;
  bool reversed;
};

std::vector<ResolvedOp> plan_layer(int side, const std::vector<int>& layer, const int32_t* pairs, Layout& lay) {
  std::vector<ResolvedOp> out;
  for (int g : layer) {
    std::vector<PlanOp> one;
    route_gate(side, g, pairs, lay, one);
    for (const PlanOp& op : one) {
      bool rev = false;
      if (op.kind == 1) rev = lay.pos[pairs[2 * g]] > lay.pos[pairs[2 * g + 1]];
      out.push_back({op.side, op.bond, op.kind, op.gate, rev});
    }
  }
  return out;
}

void build_op(pc_circuit* c, const ResolvedOp& op, cplx* U) {
  if (op.kind == 0) { swap_op(op.side, U); return; }
  cplx g[16];
  const cplx* m = &c->mats[(size_t)op.gate * 16];
  for (int r = 0; r < 4; ++r)
    for (int col = 0; col < 4; ++col) {
      const int rr = op.reversed ? ((r & 1) << 1 | (r >> 1)) : r;
      const int cc = op.reversed ? ((col & 1) << 1 | (col >> 1)) : col;
      g[4 * r + col] = m[4 * rr + cc];
    }
  if (op.side == PC_SIDE_LEFT) two_site_op(g, nullptr, U);
  else two_site_op(nullptr, g, U);
}

pc_status apply_resolved(pc_circuit* c, const std::vector<ResolvedOp>& ops) {
  const int n = c->n;
  std::vector<int> wave_of(ops.size());
  std::vector<int> last(n, -1);
  int nw = 0;
  for (size_t u = 0; u < ops.size(); ++u) {
    const int j = ops[u].bond;
    const int w = std::max(last[j], last[j + 1]) + 1;
    wave_of[u] = w;
    last[j] = last[j + 1] = w;
    nw = std::max(nw, w + 1);
  }
  std::vector<std::vector<size_t>> waves(nw);
  for (size_t u = 0; u < ops.size(); ++u) waves[wave_of[u]].push_back(u);
  std::vector<WaveItem> items;
  std::vector<int> counts;
  std::vector<int> chi_after(ops.size(), 0);
  for (int w = 0; w < nw; ++w) {
    const auto& idx = waves[w];
    for (size_t base = 0; base < idx.size(); base += c->max_tasks) {
      const size_t cnt = std::min(idx.size() - base, (size_t)c->max_tasks);
      items.resize(cnt);
      for (size_t k = 0; k < cnt; ++k) {
        items[k].bond = ops[idx[base + k]].bond;
        build_op(c, ops[idx[base + k]], items[k].op);
      }
      pc_status st = run_wave(c, items, counts, nullptr, false, false, nullptr);
      if (st != PC_OK) return st;
      for (size_t k = 0; k < cnt; ++k) chi_after[idx[base + k]] = counts[k];
    }
  }
  for (size_t u = 0; u < ops.size(); ++u)
    c->plan_log.push_back({ops[u].side, ops[u].bond, ops[u].kind, ops[u].gate, chi_after[u]});
  c->stats.n_updates += (int64_t)ops.size();
  return PC_OK;
}

pc_status apply_oneq_layer(pc_circuit* c) {
  for (size_t k = 0; k < c->oneq_q.size(); ++k) {
    const int j = c->lay[PC_SIDE_LEFT].pos[c->oneq_q[k]];
    CUDA_TRY(c->ctx, cudaMemcpyAsync(c->d_g2, &c->oneq_m[4 * k], 4 * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c->ctx, pc::launch_one_site(site_ptr(c, j), c->chi[j], c->chi[j + 1], c->d_g2, PC_SIDE_LEFT, c->stream));
    count_launch(c);
    CUDA_TRY(c->ctx, cudaStreamSynchronize(c->stream));
  }
  c->projected = false;
  return PC_OK;
}

int64_t gates_absorbed(const pc_circuit* c) {
  int64_t g = 0;
  for (size_t k = 0; k < c->lcur; ++k) g += (int64_t)c->left_layers[k].size();
  for (size_t k = 0; k < c->rcur; ++k) g += (int64_t)c->right_layers[k].size();
  return g;
}

void trace_point(pc_circuit* c, int phase, int accepted) {
  c->trace.push_back({c->stage, phase, gates_absorbed(c), mpo_size(c), max_bond(c), accepted, now_s() - c->t_loaded});
}

bool layers_remain(const pc_circuit* c) {
  return c->lcur < c->left_layers.size() || !c->oneq_done || c->rcur < c->right_layers.size();
}

pc_status absorb_left_layer(pc_circuit* c) {
  if (c->lcur < c->left_layers.size()) {
    auto ops = plan_layer(PC_SIDE_LEFT, c->left_layers[c->lcur], c->pairs.data(), c->lay[PC_SIDE_LEFT]);
    c->lcur++;
    return apply_resolved(c, ops);
  }
  if (!c->oneq_done) {
    pc_status st = apply_oneq_layer(c);
    if (st != PC_OK) return st;
    c->oneq_done = true;
  }
  return PC_OK;
}

pc_status absorb_right_layer(pc_circuit* c) {
  if (c->rcur < c->right_layers.size()) {
    auto ops = plan_layer(PC_SIDE_RIGHT, c->right_layers[c->rcur], c->pairs.data(), c->lay[PC_SIDE_RIGHT]);
    c->rcur++;
    return apply_resolved(c, ops);
  }
  return PC_OK;
}

// Device copy of the contraction state into / out of saved slot k (the circuit's stream).
pc_status save_state(pc_circuit* c, int k) {
  pc_circuit::Saved& sv = c->saved[k];
  const size_t nsite = c->site_off[c->n], nlam = (size_t)std::max(1, c->n - 1) * c->chi_max;
  if (!sv.sites) {
    CUDA_TRY(c->ctx, cudaMalloc(&sv.sites, nsite * sizeof(double2)));
    CUDA_TRY(c->ctx, cudaMalloc(&sv.lam, nlam * sizeof(double)));
  }
  CUDA_TRY(c->ctx, cudaMemcpyAsync(sv.sites, c->d_sites, nsite * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(c->ctx, cudaMemcpyAsync(sv.lam, c->d_lam, nlam * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  sv.chi = c->chi;
  sv.lay[0] = c->lay[0];
  sv.lay[1] = c->lay[1];
  sv.lcur = c->lcur;
  sv.rcur = c->rcur;
  sv.oneq_done = c->oneq_done;
  sv.plan = c->plan_log;
  sv.nupd = c->stats.n_updates;
  return PC_OK;
}

pc_status load_state(pc_circuit* c, int k) {
  pc_circuit::Saved& sv = c->saved[k];
  const size_t nsite = c->site_off[c->n], nlam = (size_t)std::max(1, c->n - 1) * c->chi_max;
  CUDA_TRY(c->ctx, cudaMemcpyAsync(c->d_sites, sv.sites, nsite * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(c->ctx, cudaMemcpyAsync(c->d_lam, sv.lam, nlam * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  c->chi = sv.chi;
  c->lay[0] = sv.lay[0];
  c->lay[1] = sv.lay[1];
  c->lcur = sv.lcur;
  c->rcur = sv.rcur;
  c->oneq_done = sv.oneq_done;
  c->plan_log = sv.plan;
  c->stats.n_updates = sv.nupd;
  c->projected = false;
  return PC_OK;
}

// App. A.3: absorb the next layer of C_L and, from the same state, the next layer of C_R;
// keep the one with the smaller size(M) (ties: left, as Algorithm 1 absorbs the left side
// first).  When one side has no layer left the other is absorbed.  The one-qubit layer X^s
// counts as the last layer of C_L.  Only the kept absorption stays in the plan and in
// n_updates.
pc_status absorb_step_adaptive(pc_circuit* c) {
  const bool can_l = c->lcur < c->left_layers.size() || !c->oneq_done;
  const bool can_r = c->rcur < c->right_layers.size();
  if (!can_r) return absorb_left_layer(c);
  if (!can_l) return absorb_right_layer(c);
  pc_status st = save_state(c, 0);
  if (st == PC_OK) st = absorb_left_layer(c);
  if (st != PC_OK) return st;
  const int64_t size_l = mpo_size(c);
  st = save_state(c, 1);
  if (st == PC_OK) st = load_state(c, 0);
  if (st == PC_OK) st = absorb_right_layer(c);
  if (st != PC_OK) return st;
  if (size_l <= mpo_size(c)) st = load_state(c, 1);
  if (st == PC_OK) CUDA_TRY(c->ctx, cudaStreamSynchronize(c->stream));
  return st;
}

// One factorisation of a recanonicalisation step (Algorithm 1, "compress M to canonical form
// via SVD"): Z = X (rows x cols) or its transpose, so that Z has no more rows than columns;
// the FP64 one-sided Jacobi orthogonalises the rows of Z with the rotations W accumulated;
// the row norms (singular values) are sorted and cut (s_k > eps s_0, at most chi_max).
// Returns the kept count in *count (host).
pc_status recanon_factor(pc_circuit* c, const double2* X, int rows, int cols, bool transpose, double eps,
                         int chi_max, int* count) {
  pc_ctx* ctx = c->ctx;
  auto& r = c->rc;
  const int mz = transpose ? cols : rows, nz = transpose ? rows : cols;
  CUDA_TRY(ctx, pc::launch_recanon_load(X, rows, cols, transpose ? 1 : 0, r.Z, c->stream));
  pc::JacobiTask jt{};
  jt.X = r.Z; jt.Q = r.Q; jt.nrm2 = r.nrm2; jt.fro2 = r.fro2; jt.stamp = r.stamp; jt.dead2_ovr = nullptr;
  const double dr = (eps > 0.0 ? eps : 1e-14) / (10.0 * mz);
  jt.dead_rel = dr * dr;
  jt.m = mz; jt.n = nz; jt.mp = mz + (mz & 1);
  pc::TruncTask tt{};
  tt.X = r.Z; tt.idx = r.idx; tt.lam = r.lam; tt.sraw = r.sraw; tt.out = r.tout;
  tt.eps = eps; tt.m = mz; tt.n = nz; tt.chi_max = chi_max;
  CUDA_TRY(ctx, cudaMemcpyAsync(r.jt, &jt, sizeof(jt), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(r.tt, &tt, sizeof(tt), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(ctx, cudaMemsetAsync(r.jst, 0, sizeof(pc::JacobiStatus), c->stream));
  CUDA_TRY(ctx, cudaMemsetAsync(r.bar, 0, 2 * sizeof(unsigned int), c->stream));
  CUDA_TRY(ctx, cudaMemsetAsync(r.err, 0, sizeof(int), c->stream));
  CUDA_TRY(ctx, pc::launch_fro2(r.jt, 1, r.fro2, c->stream));
  CUDA_TRY(ctx, pc::launch_init_accumulators(r.jt, 1, mz, c->stream));
  CUDA_TRY(ctx, pc::launch_init_stamps(r.jt, 1, mz, c->stream));
  CUDA_TRY(ctx, pc::launch_jacobi(r.jt, 1, r.jst, ctx->cfg.jacobi_max_sweeps, r.bar, r.err, ctx->sm_count, nz,
                                  jt.mp / 2, c->stream));
  CUDA_TRY(ctx, pc::launch_truncate_tasks(r.tt, 1, c->stream));
  count_launch(c, 6);
  pc::TruncOut o;
  pc::JacobiStatus js;
  int err = 0;
  CUDA_TRY(ctx, cudaMemcpyAsync(&o, r.tout, sizeof(o), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(&js, r.jst, sizeof(js), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(&err, r.err, sizeof(err), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(c->stream));
  if (err) return fail(ctx, PC_ERR_TIMEOUT, "Jacobi grid barrier wait exceeded its limit (recanonicalisation)");
  if (!js.converged) return fail(ctx, PC_ERR_NOCONVERGE, "one-sided Jacobi reached the sweep cap (recanonicalisation)");
  if (!(o.s0 > 0.0)) return fail(ctx, PC_ERR_STATE, "a site tensor of the MPO vanished (recanonicalisation)");
  *count = o.count;
  return PC_OK;
}

// Algorithm 1, "compress M to canonical form via SVD with eps".  A left-to-right sweep makes
// every site left-orthonormal (a QR step written as X = U (S V^dagger): U stays, S V^dagger
// moves into the next site); a right-to-left sweep then factorises each site with everything
// to its left orthonormal: B_j <- V^dagger (right-canonical), lambda_{j-1} <- the singular
// values (the bond's Schmidt values, cut at eps s_0 and chi_max, renormalised), U S moves into
// the previous site.  The result is the Vidal/Hastings form of the operator the sites hold;
// |M>> is renormalised.  Only numerically zero values (below 1e-14 s_0) are dropped by the
// first sweep.
pc_status recanonicalise(pc_circuit* c) {
  pc_ctx* ctx = c->ctx;
  const int n = c->n, X = c->chi_max;
  auto& r = c->rc;
  if (!c->d_rc) {
    const size_t cap2 = (size_t)X * X, big = 4 * cap2;
    size_t off = 0;
    auto sz = [&](size_t b) { const size_t o = off; off += al256(b); return o; };
    const size_t oZ = sz(big * sizeof(double2)), oQ = sz(cap2 * sizeof(double2)), oT = sz(big * sizeof(double2)),
                 oC = sz(cap2 * sizeof(double2)), oN = sz(X * sizeof(double)), oL = sz(X * sizeof(double)),
                 oS = sz(X * sizeof(double)), oF = sz(sizeof(double)), oSt = sz(X * sizeof(int32_t)),
                 oI = sz(X * sizeof(int32_t)), oJ = sz(sizeof(pc::JacobiTask)), oTt = sz(sizeof(pc::TruncTask)),
                 oO = sz(sizeof(pc::TruncOut)), oJs = sz(sizeof(pc::JacobiStatus)), oB = sz(2 * sizeof(unsigned int)),
                 oE = sz(sizeof(int));
    CUDA_TRY(ctx, cudaMalloc(&c->d_rc, off));
    char* b = c->d_rc;
    r.Z = (double2*)(b + oZ); r.Q = (double2*)(b + oQ); r.T = (double2*)(b + oT); r.C = (double2*)(b + oC);
    r.nrm2 = (double*)(b + oN); r.lam = (double*)(b + oL); r.sraw = (double*)(b + oS); r.fro2 = (double*)(b + oF);
    r.stamp = (int32_t*)(b + oSt); r.idx = (int32_t*)(b + oI); r.jt = (pc::JacobiTask*)(b + oJ);
    r.tt = (pc::TruncTask*)(b + oTt); r.tout = (pc::TruncOut*)(b + oO); r.jst = (pc::JacobiStatus*)(b + oJs);
    r.bar = (unsigned int*)(b + oB); r.err = (int*)(b + oE);
  }
  auto gemm = [&](const double2* A, int lda, const double2* Bm, int ldb, double2* C, int ldc, int M, int N,
                  int K) -> pc_status {
    pc::GemmDesc g{};
    g.A = A; g.lda = lda; g.B = Bm; g.ldb = ldb; g.C = C; g.ldc = ldc; g.M = M; g.N = N; g.K = K;
    g.opB = 0; g.alpha = 1.0; g.beta = 0.0;
    c->h_gemm[0] = g;
    CUDA_TRY(ctx, cudaMemcpyAsync(c->d_gemm, c->h_gemm, sizeof(pc::GemmDesc), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(ctx, pc::launch_gemm(c->d_gemm, 1, M, N, c->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(c->stream));
    count_launch(c);
    return PC_OK;
  };
  // left-to-right: site j = U, R = S V^dagger into site j+1
  for (int j = 0; j + 1 < n; ++j) {
    const int cl = c->chi[j], cr = c->chi[j + 1], cn = c->chi[j + 2];
    const bool tall = 4 * cl >= cr;
    int k = 0;
    pc_status st = recanon_factor(c, site_ptr(c, j), 4 * cl, cr, tall, 1e-14, 1 << 30, &k);
    if (st != PC_OK) return st;
    if (tall) {
      CUDA_TRY(ctx, pc::launch_recanon_emit(r.Z, nullptr, 4 * cl, r.idx, r.sraw, k, 4 * cl, 0, 1, 1, site_ptr(c, j), c->stream));
      CUDA_TRY(ctx, pc::launch_recanon_emit(r.Z, r.Q, cr, r.idx, r.sraw, k, cr, 1, 2, 0, r.C, c->stream));
    } else {
      CUDA_TRY(ctx, pc::launch_recanon_emit(r.Z, r.Q, 4 * cl, r.idx, r.sraw, k, 4 * cl, 1, 0, 1, site_ptr(c, j), c->stream));
      CUDA_TRY(ctx, pc::launch_recanon_emit(r.Z, nullptr, cr, r.idx, r.sraw, k, cr, 0, 0, 0, r.C, c->stream));
    }
    count_launch(c, 2);
    st = gemm(r.C, cr, site_ptr(c, j + 1), 4 * cn, r.T, 4 * cn, k, 4 * cn, cr);
    if (st != PC_OK) return st;
    CUDA_TRY(ctx, cudaMemcpyAsync(site_ptr(c, j + 1), r.T, (size_t)k * 4 * cn * sizeof(double2), cudaMemcpyDeviceToDevice,
                                  c->stream));
    c->chi[j + 1] = k;
  }
  // right-to-left: site j = V^dagger, lambda_{j-1} = S, U S into site j-1
  for (int j = n - 1; j >= 1; --j) {
    const int cl = c->chi[j], cr = c->chi[j + 1], cp = c->chi[j - 1];
    const bool wide = cl <= 4 * cr;
    int k = 0;
    pc_status st = recanon_factor(c, site_ptr(c, j), cl, 4 * cr, !wide, ctx->cfg.eps, c->chi_max, &k);
    if (st != PC_OK) return st;
    if (wide) {
      CUDA_TRY(ctx, pc::launch_recanon_emit(r.Z, nullptr, 4 * cr, r.idx, r.sraw, k, 4 * cr, 0, 1, 0, site_ptr(c, j), c->stream));
      CUDA_TRY(ctx, pc::launch_recanon_emit(r.Z, r.Q, cl, r.idx, r.sraw, k, cl, 1, 2, 1, r.C, c->stream));
    } else {
      CUDA_TRY(ctx, pc::launch_recanon_emit(r.Z, r.Q, 4 * cr, r.idx, r.sraw, k, 4 * cr, 1, 0, 0, site_ptr(c, j), c->stream));
      CUDA_TRY(ctx, pc::launch_recanon_emit(r.Z, nullptr, cl, r.idx, r.sraw, k, cl, 0, 0, 1, r.C, c->stream));
    }
    count_launch(c, 2);
    CUDA_TRY(ctx, cudaMemcpyAsync(lam_ptr(c, j - 1), r.lam, k * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    st = gemm(site_ptr(c, j - 1), cl, r.C, k, r.T, k, 4 * cp, k, cl);
    if (st != PC_OK) return st;
    CUDA_TRY(ctx, cudaMemcpyAsync(site_ptr(c, j - 1), r.T, (size_t)4 * cp * k * sizeof(double2), cudaMemcpyDeviceToDevice,
                                  c->stream));
    c->chi[j] = k;
  }
  // renormalise |M>> (site 0 carries the norm)
  const size_t n0 = (size_t)4 * c->chi[1];
  std::vector<double2> h(n0);
  CUDA_TRY(ctx, cudaMemcpyAsync(h.data(), site_ptr(c, 0), n0 * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(c->stream));
  double nn = 0.0;
  for (const double2& v : h) nn += v.x * v.x + v.y * v.y;
  const double inv = 1.0 / std::sqrt(nn);
  for (double2& v : h) { v.x *= inv; v.y *= inv; }
  CUDA_TRY(ctx, cudaMemcpyAsync(site_ptr(c, 0), h.data(), n0 * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(c->stream));
  c->projected = false;
  c->stats.n_recanon += 1;
  return PC_OK;
}

pc_status absorb_layer_pair(pc_circuit* c) {
  std::vector<ResolvedOp> ops;
  bool do_oneq = false;
  if (c->lcur < c->left_layers.size()) {
    auto l = plan_layer(PC_SIDE_LEFT, c->left_layers[c->lcur], c->pairs.data(), c->lay[PC_SIDE_LEFT]);
    ops.insert(ops.end(), l.begin(), l.end());
    c->lcur++;
  } else if (!c->oneq_done) {
    do_oneq = true;
  }
  if (c->rcur < c->right_layers.size()) {
    auto r = plan_layer(PC_SIDE_RIGHT, c->right_layers[c->rcur], c->pairs.data(), c->lay[PC_SIDE_RIGHT]);
    ops.insert(ops.end(), r.begin(), r.end());
    c->rcur++;
  }
  // The one-qubit layer sits outermost on the left: apply it after the left's (empty) layer
  // and before the right's layer, exactly as absorbed in order; it commutes with the right
  // layer's updates only if they avoid its sites, so keep the order: left, one-qubit, right.
  if (do_oneq) {
    pc_status st = apply_oneq_layer(c);
    if (st != PC_OK) return st;
    c->oneq_done = true;
  }
  return apply_resolved(c, ops);
}

// App. A.1 parallel swap selection.
pc_status unswap_parallel(pc_circuit* c, int* n_acc) {
  pc_ctx* ctx = c->ctx;
  const int order[6][2] = {{PC_SIDE_BOTH, 0}, {PC_SIDE_BOTH, 1}, {PC_SIDE_LEFT, 0},
                           {PC_SIDE_LEFT, 1}, {PC_SIDE_RIGHT, 0}, {PC_SIDE_RIGHT, 1}};
  int total = 0;
  std::vector<WaveItem> items;
  std::vector<int> counts, acc;
  for (int it = 0; it < ctx->cfg.max_unswap_iter; ++it) {
    bool any = false;
    for (const auto& sp : order) {
      const int side = sp[0], parity = sp[1];
      std::vector<int> bonds;
      for (int b = parity; b + 1 < c->n; b += 2) bonds.push_back(b);
      for (size_t base = 0; base < bonds.size(); base += c->max_tasks) {
        const size_t cnt = std::min(bonds.size() - base, (size_t)c->max_tasks);
        items.resize(cnt);
        for (size_t k = 0; k < cnt; ++k) {
          items[k].bond = bonds[base + k];
          swap_op(side, items[k].op);
        }
        pc_status st = run_wave(c, items, counts, nullptr, true, ctx->cfg.accept_equal != 0, &acc, true);
        if (st != PC_OK) return st;
        c->stats.n_trials += (int64_t)cnt;
        for (size_t k = 0; k < cnt; ++k) {
          if (!acc[k]) continue;
          const int b = bonds[base + k];
          if (side == PC_SIDE_LEFT || side == PC_SIDE_BOTH) c->lay[PC_SIDE_LEFT].swap_sites(b);
          if (side == PC_SIDE_RIGHT || side == PC_SIDE_BOTH) c->lay[PC_SIDE_RIGHT].swap_sites(b);
          c->unswap_log.push_back({c->stage, it, side, b});
          c->plan_log.push_back({side, b, 2, -1, counts[k]});
          any = true;
          ++total;
        }
      }
    }
    if (!any) break;
  }
  c->stats.n_accepted += total;
  if (n_acc) *n_acc = total;
  return PC_OK;
}

// Algorithm 1 sequential unswapping: largest available bond (smallest index on ties), the
// three sides tried as one wave (the trials share sites, so they run as three separate
// one-task waves that do not commit), best = smallest count, ties in side order.
pc_status unswap_sequential(pc_circuit* c, int* n_acc) {
  pc_ctx* ctx = c->ctx;
  const int nb = c->n - 1;
  std::vector<char> avail(nb, 1);
  int navail = nb, total = 0;
  const long long cap = (long long)ctx->cfg.max_unswap_iter * std::max(c->n, 1) * 4;
  long long steps = 0;
  std::vector<WaveItem> items(1);
  std::vector<int> counts, none(1, 0);
  while (navail > 0 && steps < cap) {
    ++steps;
    int i = -1;
    for (int b = 0; b < nb; ++b)
      if (avail[b] && (i < 0 || c->chi[b + 1] > c->chi[i + 1])) i = b;
    int best_cnt = 1 << 30, best_side = -1;
    for (int side = 0; side < 3; ++side) {
      items[0].bond = i;
      swap_op(side, items[0].op);
      pc_status st = run_wave(c, items, counts, &none, false, ctx->cfg.accept_equal != 0, nullptr, true);
      if (st != PC_OK) return st;
      c->stats.n_trials += 1;
      if (counts[0] < best_cnt) { best_cnt = counts[0]; best_side = side; }
    }
    const int old = c->chi[i + 1];
    const bool ok = ctx->cfg.accept_equal ? best_cnt <= old : best_cnt < old;
    if (ok) {
      // recompute the winning trial and commit it
      items[0].bond = i;
      swap_op(best_side, items[0].op);
      std::vector<int> one(1, 1);
      pc_status st = run_wave(c, items, counts, &one, false, false, nullptr);
      if (st != PC_OK) return st;
      if (best_side == PC_SIDE_LEFT || best_side == PC_SIDE_BOTH) c->lay[PC_SIDE_LEFT].swap_sites(i);
      if (best_side == PC_SIDE_RIGHT || best_side == PC_SIDE_BOTH) c->lay[PC_SIDE_RIGHT].swap_sites(i);
      c->unswap_log.push_back({c->stage, (int)(steps - 1), best_side, i});
      c->plan_log.push_back({best_side, i, 2, -1, counts[0]});
      ++total;
      avail[i] = 0; --navail;
      for (int nbnd : {i - 1, i + 1})
        if (nbnd >= 0 && nbnd < nb && !avail[nbnd]) { avail[nbnd] = 1; ++navail; }
    } else {
      avail[i] = 0; --navail;
    }
  }
  c->stats.n_accepted += total;
  if (n_acc) *n_acc = total;
  return PC_OK;
}

pc_status unswap_stage(pc_circuit* c, int* n_acc) {
  if (n_acc) *n_acc = 0;
  if (c->n < 2) return PC_OK;
  switch (c->ctx->cfg.unswap_mode) {
    case PC_UNSWAP_PARALLEL: return unswap_parallel(c, n_acc);
    case PC_UNSWAP_SEQUENTIAL: return unswap_sequential(c, n_acc);
    default: return PC_OK;
  }
}

// Right environments of M|0>: env_n = 1, env_j = sum_s A_j^s env_{j+1} A_j^s^dagger with
// A_j^s = B_j[:, 2 s, :] (in-leg set to 0).
pc_status project(pc_circuit* c) {
  if (c->projected) return PC_OK;
  pc_ctx* ctx = c->ctx;
  const int n = c->n;
  c->env_off.assign(n + 1, 0);
  size_t off = 0;
  for (int j = 0; j <= n; ++j) { c->env_off[j] = off; off += (size_t)c->chi[j] * c->chi[j]; }
  cudaFree(c->d_env);
  c->d_env = nullptr;
  CUDA_TRY(ctx, cudaMalloc(&c->d_env, (off + (size_t)c->chi_max * c->chi_max) * sizeof(double2)));
  double2* tmp = c->d_env + off;   // chi_l x chi_r scratch
  const double2 one = make_double2(1.0, 0.0);
  CUDA_TRY(ctx, cudaMemcpyAsync(c->d_env + c->env_off[n], &one, sizeof(double2), cudaMemcpyHostToDevice, c->stream));
  for (int j = n - 1; j >= 0; --j) {
    const int cl = c->chi[j], cr = c->chi[j + 1];
    for (int sgm = 0; sgm < 2; ++sgm) {
      pc::GemmDesc g1{}, g2{};
      g1.A = site_ptr(c, j) + 2 * sgm * cr; g1.lda = 4 * cr;
      g1.B = c->d_env + c->env_off[j + 1]; g1.ldb = cr;
      g1.C = tmp; g1.ldc = cr;
      g1.M = cl; g1.N = cr; g1.K = cr; g1.opB = 0; g1.alpha = 1.0; g1.beta = 0.0;
      g2.A = tmp; g2.lda = cr;
      g2.B = site_ptr(c, j) + 2 * sgm * cr; g2.ldb = 4 * cr;
      g2.C = c->d_env + c->env_off[j]; g2.ldc = cl;
      g2.M = cl; g2.N = cl; g2.K = cr; g2.opB = 1; g2.alpha = 1.0; g2.beta = sgm;
      c->h_gemm[0] = g1;
      CUDA_TRY(ctx, cudaMemcpyAsync(c->d_gemm, c->h_gemm, sizeof(pc::GemmDesc), cudaMemcpyHostToDevice, c->stream));
      CUDA_TRY(ctx, pc::launch_gemm(c->d_gemm, 1, cl, cr, c->stream));
      CUDA_TRY(ctx, cudaStreamSynchronize(c->stream));
      count_launch(c, 2);
      c->h_gemm[0] = g2;
      CUDA_TRY(ctx, cudaMemcpyAsync(c->d_gemm, c->h_gemm, sizeof(pc::GemmDesc), cudaMemcpyHostToDevice, c->stream));
      CUDA_TRY(ctx, pc::launch_gemm(c->d_gemm, 1, cl, cl, c->stream));
      CUDA_TRY(ctx, cudaStreamSynchronize(c->stream));
    }
  }
  double2 z;
  CUDA_TRY(ctx, cudaMemcpy(&z, c->d_env + c->env_off[0], sizeof(double2), cudaMemcpyDeviceToHost));
  c->norm2 = z.x;
  c->projected = true;
  return PC_OK;
}

pc_status check_circuit(pc_circuit* c) {
  if (!c || !c->ctx) return PC_ERR_INVALID_ARG;
  return PC_OK;
}

}  // namespace

// =======================================================================================
extern "C" {

const char* pc_version(void) { return kVersion; }

void pc_default_config(pc_config* cfg) {
  if (!cfg) return;
  cfg->eps = 1e-10;
  cfg->chi_max = 256;
  cfg->tau = 1e6;
  cfg->max_unswap_iter = 20;
  cfg->accept_equal = 0;
  cfg->unswap_mode = PC_UNSWAP_PARALLEL;
  cfg->jacobi_max_sweeps = 60;
  cfg->device = 0;
  cfg->fp32_precondition = 1;
  cfg->precision = PC_PRECISION_FP64;
  cfg->precondition_sweeps = 20;
  cfg->side_mode = PC_SIDE_ALTERNATE;
  cfg->certify_trials = 1;
  cfg->deflate = 1;
  cfg->fp32_dead_rel = 0.0;
  cfg->recanonicalise = 1;
}

pc_status pc_create(const pc_config* cfg, pc_ctx** out) {
  if (!cfg || !out) return PC_ERR_INVALID_ARG;
  *out = nullptr;
  if (!(cfg->eps >= 0.0) || cfg->chi_max < 1 || cfg->chi_max > 1024 || !(cfg->tau > 0.0) ||
      cfg->max_unswap_iter < 0 || cfg->jacobi_max_sweeps < 1 || cfg->unswap_mode < 0 || cfg->unswap_mode > 2 ||
      cfg->precision < PC_PRECISION_FP64 || cfg->precision > PC_PRECISION_TF32X3 || cfg->precondition_sweeps < 1 ||
      cfg->side_mode < PC_SIDE_ALTERNATE || cfg->side_mode > PC_SIDE_ADAPTIVE || !(cfg->fp32_dead_rel >= 0.0) ||
      cfg->fp32_dead_rel >= 1.0)
    return PC_ERR_INVALID_ARG;
  auto* ctx = new pc_ctx();
  ctx->cfg = *cfg;
  cudaError_t e = cudaSetDevice(cfg->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, cfg->device);
  if (e != cudaSuccess) {
    delete ctx;
    return PC_ERR_CUDA;
  }
  *out = ctx;
  return PC_OK;
}

pc_status pc_destroy(pc_ctx* ctx) {
  delete ctx;
  return PC_OK;
}

const char* pc_last_error(pc_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

pc_status pc_load_gates(pc_ctx* ctx, int32_t n_qubits, int64_t n_gates, const int32_t* pairs, const double* mats,
                        int64_t split_index, int64_t n_oneq, const int32_t* oneq_qubits, const double* oneq_mats,
                        pc_circuit** out) {
  if (!ctx || !out) return PC_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_qubits < 2 || n_qubits > 4096 || n_gates < 0 || n_oneq < 0 || (n_gates > 0 && (!pairs || !mats)) ||
      (n_oneq > 0 && (!oneq_qubits || !oneq_mats)))
    return fail(ctx, PC_ERR_INVALID_ARG, "bad sizes or null pointers");
  if (split_index < 0) split_index = n_gates / 2;
  if (split_index > n_gates) return fail(ctx, PC_ERR_INVALID_ARG, "split_index beyond the gate list");
  if (cudaSetDevice(ctx->cfg.device) != cudaSuccess) return fail(ctx, PC_ERR_CUDA, "cudaSetDevice");
  auto* c = new pc_circuit();
  c->ctx = ctx;
  c->n = n_qubits;
  c->chi_max = ctx->cfg.chi_max;
  c->pairs.assign(pairs, pairs + 2 * n_gates);
  c->mats.resize(16 * n_gates);
  for (int64_t g = 0; g < n_gates; ++g) {
    const int a = pairs[2 * g], b = pairs[2 * g + 1];
    if (a < 0 || b < 0 || a >= n_qubits || b >= n_qubits || a == b) {
      delete c;
      return fail(ctx, PC_ERR_INVALID_ARG, "gate " + std::to_string(g) + " has a bad qubit pair");
    }
    for (int k = 0; k < 16; ++k) c->mats[16 * g + k] = cplx(mats[32 * g + 2 * k], mats[32 * g + 2 * k + 1]);
    double dev = 0.0;
    for (int r = 0; r < 4; ++r)
      for (int col = 0; col < 4; ++col) {
        cplx acc = 0;
        for (int k = 0; k < 4; ++k) acc += std::conj(c->mats[16 * g + 4 * k + r]) * c->mats[16 * g + 4 * k + col];
        dev = std::max(dev, std::abs(acc - (r == col ? 1.0 : 0.0)));
      }
    if (!(dev <= 1e-6)) {
      delete c;
      return fail(ctx, PC_ERR_NONUNITARY, "gate " + std::to_string(g) + " is not unitary");
    }
  }
  c->oneq_q.assign(oneq_qubits, oneq_qubits + n_oneq);
  c->oneq_m.resize(4 * n_oneq);
  for (int64_t k = 0; k < n_oneq; ++k) {
    if (oneq_qubits[k] < 0 || oneq_qubits[k] >= n_qubits) {
      delete c;
      return fail(ctx, PC_ERR_INVALID_ARG, "one-qubit gate on a bad qubit");
    }
    for (int e = 0; e < 4; ++e) c->oneq_m[4 * k + e] = cplx(oneq_mats[8 * k + 2 * e], oneq_mats[8 * k + 2 * e + 1]);
  }
  c->split = split_index;
  std::vector<int> lorder, rorder;
  for (int64_t g = split_index; g < n_gates; ++g) lorder.push_back((int)g);
  for (int64_t g = split_index - 1; g >= 0; --g) rorder.push_back((int)g);
  c->left_layers = make_layers(lorder, c->pairs.data(), n_qubits);
  c->right_layers = make_layers(rorder, c->pairs.data(), n_qubits);
  c->oneq_done = n_oneq == 0;
  c->t_loaded = now_s();
  pc_status st = alloc_circuit(c);
  if (st != PC_OK) { free_circuit(c); return st; }
  st = reset_identity(c);
  if (st != PC_OK) { free_circuit(c); return st; }
  *out = c;
  return PC_OK;
}

pc_status pc_destroy_circuit(pc_circuit* c) {
  free_circuit(c);
  return PC_OK;
}

pc_status pc_contract_iterations(pc_circuit* c, int32_t max_iterations, pc_stats* stats, int32_t* done) {
  if (check_circuit(c) != PC_OK || max_iterations < 0) return PC_ERR_INVALID_ARG;
  pc_ctx* ctx = c->ctx;
  if (cudaSetDevice(ctx->cfg.device) != cudaSuccess) return fail(ctx, PC_ERR_CUDA, "cudaSetDevice");
  const double t0 = now_s();
  c->stats = pc_stats{};
  // while it contracts, an attached circuit is one of the batch's participants: the launcher
  // waits (briefly) for its waves to combine them with the others'
  struct Participation {
    pc_batch* b;
    explicit Participation(pc_batch* bb) : b(bb) { if (b) batch_enter(b); }
    ~Participation() { if (b) batch_leave(b); }
  } participation(c->batch);
  const double tau = ctx->cfg.tau;
  pc_status st = PC_OK;
  for (int32_t it = 0; it < max_iterations && layers_remain(c); ++it) {
    // Algorithm 1: absorb layer pairs while size(M) < tau (progress rule: at least one)
    bool first = true;
    while ((first || (double)mpo_size(c) < tau) && layers_remain(c)) {
      st = ctx->cfg.side_mode == PC_SIDE_ADAPTIVE ? absorb_step_adaptive(c) : absorb_layer_pair(c);
      if (st == PC_OK && ctx->cfg.recanonicalise) st = recanonicalise(c);
      if (st != PC_OK) return st;
      first = false;
    }
    trace_point(c, 0, 0);
    int acc = 0;
    st = unswap_stage(c, &acc);
    if (st != PC_OK) return st;
    trace_point(c, 1, acc);
    if ((double)mpo_size(c) >= tau && layers_remain(c)) c->stats.stalled = 1;
    c->stats.n_stages += 1;
    c->stage += 1;
  }
  c->stats.final_size = mpo_size(c);
  c->stats.max_chi = std::max(c->stats.max_chi, max_bond(c));
  c->stats.seconds = now_s() - t0;
  if (stats) *stats = c->stats;
  if (done) *done = layers_remain(c) ? 0 : 1;
  return PC_OK;
}

pc_status pc_contract(pc_circuit* c, pc_stats* stats) {
  pc_stats local{};
  int32_t done = 0;
  pc_status st = pc_contract_iterations(c, INT32_MAX, &local, &done);
  if (st != PC_OK) return st;
  if (stats) *stats = local;
  return local.stalled ? PC_WARN_STALLED : PC_OK;
}

pc_status pc_get_trace(pc_circuit* c, int64_t cap, pc_trace_record* rec, int64_t* n_rec) {
  if (check_circuit(c) != PC_OK || !n_rec || cap < 0) return PC_ERR_INVALID_ARG;
  *n_rec = (int64_t)c->trace.size();
  for (int64_t k = 0; rec && k < cap && k < *n_rec; ++k) rec[k] = c->trace[k];
  return PC_OK;
}

pc_status pc_get_stats(pc_circuit* c, pc_stats* stats) {
  if (check_circuit(c) != PC_OK || !stats) return PC_ERR_INVALID_ARG;
  *stats = c->stats;
  return PC_OK;
}

pc_status pc_get_cursors(pc_circuit* c, int64_t* left, int64_t* right) {
  if (check_circuit(c) != PC_OK) return PC_ERR_INVALID_ARG;
  if (left) *left = (int64_t)c->lcur;
  if (right) *right = (int64_t)c->rcur;
  return PC_OK;
}

pc_status pc_set_cursors(pc_circuit* c, int64_t left, int64_t right) {
  if (check_circuit(c) != PC_OK || left < 0 || right < 0 || left > (int64_t)c->left_layers.size() ||
      right > (int64_t)c->right_layers.size())
    return PC_ERR_INVALID_ARG;
  c->lcur = (size_t)left;
  c->rcur = (size_t)right;
  c->oneq_done = c->oneq_q.empty();
  return PC_OK;
}

pc_status pc_snapshot(pc_circuit* c) {
  if (check_circuit(c) != PC_OK) return PC_ERR_INVALID_ARG;
  pc_ctx* ctx = c->ctx;
  const size_t nsite = c->site_off[c->n], nlam = (size_t)std::max(1, c->n - 1) * c->chi_max;
  if (!c->d_snap_sites) {
    CUDA_TRY(ctx, cudaMalloc(&c->d_snap_sites, nsite * sizeof(double2)));
    CUDA_TRY(ctx, cudaMalloc(&c->d_snap_lam, nlam * sizeof(double)));
  }
  CUDA_TRY(ctx, cudaMemcpyAsync(c->d_snap_sites, c->d_sites, nsite * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(c->d_snap_lam, c->d_lam, nlam * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  c->snap_chi = c->chi;
  c->snap_lay[0] = c->lay[0];
  c->snap_lay[1] = c->lay[1];
  c->snap_lcur = c->lcur;
  c->snap_rcur = c->rcur;
  c->snap_oneq_done = c->oneq_done;
  c->has_snapshot = true;
  return PC_OK;
}

pc_status pc_restore(pc_circuit* c) {
  if (check_circuit(c) != PC_OK) return PC_ERR_INVALID_ARG;
  if (!c->has_snapshot) return fail(c->ctx, PC_ERR_STATE, "no snapshot to restore");
  pc_ctx* ctx = c->ctx;
  const size_t nsite = c->site_off[c->n], nlam = (size_t)std::max(1, c->n - 1) * c->chi_max;
  CUDA_TRY(ctx, cudaMemcpyAsync(c->d_sites, c->d_snap_sites, nsite * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(c->d_lam, c->d_snap_lam, nlam * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  c->chi = c->snap_chi;
  c->lay[0] = c->snap_lay[0];
  c->lay[1] = c->snap_lay[1];
  c->lcur = c->snap_lcur;
  c->rcur = c->snap_rcur;
  c->oneq_done = c->snap_oneq_done;
  c->projected = false;
  return PC_OK;
}

namespace {
constexpr uint64_t kCkptMagic = 0x31544b4350434d50ull;   // "PMCPCKT1"

bool write_all(FILE* f, const void* p, size_t bytes) { return bytes == 0 || fwrite(p, 1, bytes, f) == bytes; }
bool read_all(FILE* f, void* p, size_t bytes) { return bytes == 0 || fread(p, 1, bytes, f) == bytes; }
}  // namespace

pc_status pc_checkpoint_write(pc_circuit* c, const char* path) {
  if (check_circuit(c) != PC_OK || !path) return PC_ERR_INVALID_ARG;
  pc_ctx* ctx = c->ctx;
  if (cudaSetDevice(ctx->cfg.device) != cudaSuccess) return fail(ctx, PC_ERR_CUDA, "cudaSetDevice");
  CUDA_TRY(ctx, cudaStreamSynchronize(c->stream));
  const int n = c->n;
  std::vector<double2> sites;
  for (int j = 0; j < n; ++j) {
    const size_t cnt = (size_t)c->chi[j] * 4 * c->chi[j + 1];
    const size_t o = sites.size();
    sites.resize(o + cnt);
    CUDA_TRY(ctx, cudaMemcpy(sites.data() + o, site_ptr(c, j), cnt * sizeof(double2), cudaMemcpyDeviceToHost));
  }
  std::vector<double> lam;
  for (int b = 0; b + 1 < n; ++b) {
    const size_t o = lam.size();
    lam.resize(o + c->chi[b + 1]);
    CUDA_TRY(ctx, cudaMemcpy(lam.data() + o, lam_ptr(c, b), c->chi[b + 1] * sizeof(double), cudaMemcpyDeviceToHost));
  }
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(ctx, PC_ERR_STATE, std::string("cannot write ") + path);
  const int64_t hdr[8] = {(int64_t)kCkptMagic, n, (int64_t)c->left_layers.size(), (int64_t)c->right_layers.size(),
                          (int64_t)c->lcur, (int64_t)c->rcur, c->oneq_done ? 1 : 0, c->stage};
  bool ok = write_all(f, hdr, sizeof(hdr)) && write_all(f, c->chi.data(), (n + 1) * sizeof(int)) &&
            write_all(f, c->lay[0].pos.data(), n * sizeof(int)) && write_all(f, c->lay[1].pos.data(), n * sizeof(int));
  const int64_t ns = (int64_t)sites.size(), nl = (int64_t)lam.size();
  ok = ok && write_all(f, &ns, sizeof(ns)) && write_all(f, sites.data(), sites.size() * sizeof(double2)) &&
       write_all(f, &nl, sizeof(nl)) && write_all(f, lam.data(), lam.size() * sizeof(double));
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return fail(ctx, PC_ERR_STATE, std::string("short write to ") + path);
  return PC_OK;
}

pc_status pc_checkpoint_read(pc_circuit* c, const char* path) {
  if (check_circuit(c) != PC_OK || !path) return PC_ERR_INVALID_ARG;
  pc_ctx* ctx = c->ctx;
  if (cudaSetDevice(ctx->cfg.device) != cudaSuccess) return fail(ctx, PC_ERR_CUDA, "cudaSetDevice");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(ctx, PC_ERR_STATE, std::string("cannot read ") + path);
  const int n = c->n;
  int64_t hdr[8];
  std::vector<int> chi(n + 1), pos0(n), pos1(n);
  int64_t ns = -1, nl = -1;
  bool ok = read_all(f, hdr, sizeof(hdr)) && hdr[0] == (int64_t)kCkptMagic && hdr[1] == n &&
            hdr[2] == (int64_t)c->left_layers.size() && hdr[3] == (int64_t)c->right_layers.size() &&
            hdr[4] >= 0 && hdr[4] <= hdr[2] && hdr[5] >= 0 && hdr[5] <= hdr[3];
  ok = ok && read_all(f, chi.data(), (n + 1) * sizeof(int)) && read_all(f, pos0.data(), n * sizeof(int)) &&
       read_all(f, pos1.data(), n * sizeof(int));
  // bond dimensions within the store, layouts permutations
  if (ok) {
    ok = chi[0] == 1 && chi[n] == 1;
    for (int k = 1; ok && k < n; ++k) ok = chi[k] >= 1 && chi[k] <= c->cap[k];
    std::vector<char> seen0(n, 0), seen1(n, 0);
    for (int q = 0; ok && q < n; ++q) {
      ok = pos0[q] >= 0 && pos0[q] < n && !seen0[pos0[q]] && pos1[q] >= 0 && pos1[q] < n && !seen1[pos1[q]];
      if (ok) seen0[pos0[q]] = seen1[pos1[q]] = 1;
    }
  }
  size_t want_s = 0, want_l = 0;
  for (int j = 0; ok && j < n; ++j) want_s += (size_t)chi[j] * 4 * chi[j + 1];
  for (int b = 0; ok && b + 1 < n; ++b) want_l += chi[b + 1];
  std::vector<double2> sites;
  std::vector<double> lam;
  ok = ok && read_all(f, &ns, sizeof(ns)) && ns == (int64_t)want_s;
  if (ok) { sites.resize(want_s); ok = read_all(f, sites.data(), want_s * sizeof(double2)); }
  ok = ok && read_all(f, &nl, sizeof(nl)) && nl == (int64_t)want_l;
  if (ok) { lam.resize(want_l); ok = read_all(f, lam.data(), want_l * sizeof(double)); }
  std::fclose(f);
  if (!ok) return fail(ctx, PC_ERR_INVALID_ARG, std::string("checkpoint does not match this circuit: ") + path);
  CUDA_TRY(ctx, cudaStreamSynchronize(c->stream));
  size_t so = 0, lo = 0;
  for (int j = 0; j < n; ++j) {
    const size_t cnt = (size_t)chi[j] * 4 * chi[j + 1];
    CUDA_TRY(ctx, cudaMemcpyAsync(site_ptr(c, j), sites.data() + so, cnt * sizeof(double2), cudaMemcpyHostToDevice,
                                  c->stream));
    so += cnt;
  }
  for (int b = 0; b + 1 < n; ++b) {
    CUDA_TRY(ctx, cudaMemcpyAsync(lam_ptr(c, b), lam.data() + lo, chi[b + 1] * sizeof(double), cudaMemcpyHostToDevice,
                                  c->stream));
    lo += chi[b + 1];
  }
  CUDA_TRY(ctx, cudaStreamSynchronize(c->stream));
  c->chi = chi;
  for (int side = 0; side < 2; ++side) {
    const std::vector<int>& pos = side == 0 ? pos0 : pos1;
    c->lay[side].pos = pos;
    for (int q = 0; q < n; ++q) c->lay[side].site[pos[q]] = q;
  }
  c->lcur = (size_t)hdr[4];
  c->rcur = (size_t)hdr[5];
  c->oneq_done = hdr[6] != 0;
  c->stage = (int)hdr[7];
  c->projected = false;
  return PC_OK;
}

pc_status pc_unswap(pc_circuit* c, int32_t* n_accepted) {
  if (check_circuit(c) != PC_OK) return PC_ERR_INVALID_ARG;
  int acc = 0;
  pc_status st = unswap_stage(c, &acc);
  c->stage += 1;
  if (n_accepted) *n_accepted = acc;
  return st;
}

pc_status pc_get_bond_dims(pc_circuit* c, int32_t* chi) {
  if (check_circuit(c) != PC_OK || !chi) return PC_ERR_INVALID_ARG;
  for (int b = 0; b + 1 < c->n; ++b) chi[b] = c->chi[b + 1];
  return PC_OK;
}

pc_status pc_get_layouts(pc_circuit* c, int32_t* layout_l, int32_t* layout_r) {
  if (check_circuit(c) != PC_OK) return PC_ERR_INVALID_ARG;
  for (int q = 0; q < c->n; ++q) {
    if (layout_l) layout_l[q] = c->lay[PC_SIDE_LEFT].pos[q];
    if (layout_r) layout_r[q] = c->lay[PC_SIDE_RIGHT].pos[q];
  }
  return PC_OK;
}

pc_status pc_get_spectrum(pc_circuit* c, int32_t bond, int32_t cap, double* s, int32_t* len) {
  if (check_circuit(c) != PC_OK || bond < 0 || bond + 1 >= c->n || !len) return PC_ERR_INVALID_ARG;
  const int k = c->chi[bond + 1];
  *len = k;
  if (s && cap > 0) {
    CUDA_TRY(c->ctx, cudaStreamSynchronize(c->stream));
    CUDA_TRY(c->ctx, cudaMemcpy(s, lam_ptr(c, bond), std::min(k, cap) * sizeof(double), cudaMemcpyDeviceToHost));
  }
  return PC_OK;
}

pc_status pc_get_site(pc_circuit* c, int32_t j, int64_t cap, double* out, int32_t* dims) {
  if (check_circuit(c) != PC_OK || j < 0 || j >= c->n) return PC_ERR_INVALID_ARG;
  const int64_t cnt = (int64_t)c->chi[j] * 4 * c->chi[j + 1];
  if (dims) { dims[0] = c->chi[j]; dims[1] = c->chi[j + 1]; }
  if (out) {
    if (cap < cnt) return fail(c->ctx, PC_ERR_INVALID_ARG, "site buffer too small");
    CUDA_TRY(c->ctx, cudaStreamSynchronize(c->stream));
    CUDA_TRY(c->ctx, cudaMemcpy(out, site_ptr(c, j), cnt * sizeof(double2), cudaMemcpyDeviceToHost));
  }
  return PC_OK;
}

pc_status pc_set_state(pc_circuit* c, const int32_t* chi, const double* sites, const double* lam) {
  if (check_circuit(c) != PC_OK || !chi || !sites || !lam) return PC_ERR_INVALID_ARG;
  if (chi[0] != 1 || chi[c->n] != 1) return fail(c->ctx, PC_ERR_INVALID_ARG, "boundary bond dimensions must be 1");
  for (int k = 1; k < c->n; ++k)
    if (chi[k] < 1 || chi[k] > c->chi_max) return fail(c->ctx, PC_ERR_INVALID_ARG, "bond dimension out of range");
  size_t so = 0, lo = 0;
  for (int j = 0; j < c->n; ++j) {
    const size_t cnt = (size_t)chi[j] * 4 * chi[j + 1];
    CUDA_TRY(c->ctx, cudaMemcpyAsync(site_ptr(c, j), sites + 2 * so, cnt * sizeof(double2), cudaMemcpyHostToDevice,
                                     c->stream));
    so += cnt;
  }
  for (int b = 0; b + 1 < c->n; ++b) {
    CUDA_TRY(c->ctx, cudaMemcpyAsync(lam_ptr(c, b), lam + lo, chi[b + 1] * sizeof(double), cudaMemcpyHostToDevice,
                                     c->stream));
    lo += chi[b + 1];
  }
  // the uploads are complete before any launch on another stream reads the sites
  CUDA_TRY(c->ctx, cudaStreamSynchronize(c->stream));
  for (int k = 0; k <= c->n; ++k) c->chi[k] = chi[k];
  c->lay[0].reset(c->n);
  c->lay[1].reset(c->n);
  c->projected = false;
  return PC_OK;
}

pc_status pc_apply_updates(pc_circuit* c, int32_t n_ops, const int32_t* bonds, const double* ops, int32_t* chi_out) {
  if (check_circuit(c) != PC_OK || n_ops < 0 || (n_ops > 0 && (!bonds || !ops))) return PC_ERR_INVALID_ARG;
  if (n_ops > c->max_tasks) return fail(c->ctx, PC_ERR_INVALID_ARG, "more updates than the batch limit (n/2, at most 32)");
  std::vector<int> sorted(bonds, bonds + n_ops);
  std::sort(sorted.begin(), sorted.end());
  for (int k = 0; k < n_ops; ++k) {
    if (sorted[k] < 0 || sorted[k] + 1 >= c->n) return fail(c->ctx, PC_ERR_INVALID_ARG, "bond out of range");
    if (k > 0 && sorted[k] - sorted[k - 1] < 2) return fail(c->ctx, PC_ERR_INVALID_ARG, "bonds must be non-adjacent");
  }
  std::vector<WaveItem> items(n_ops);
  for (int k = 0; k < n_ops; ++k) {
    items[k].bond = bonds[k];
    for (int e = 0; e < 256; ++e) items[k].op[e] = cplx(ops[512 * k + 2 * e], ops[512 * k + 2 * e + 1]);
  }
  std::vector<int> counts;
  pc_status st = run_wave(c, items, counts, nullptr, false, false, nullptr);
  if (st != PC_OK) return st;
  if (chi_out) for (int k = 0; k < n_ops; ++k) chi_out[k] = counts[k];
  return PC_OK;
}

pc_status pc_plan_routing(int32_t n_qubits, int64_t n_gates, const int32_t* pairs, int64_t split_index, int64_t cap,
                          int32_t* rec, int64_t* n_rec) {
  if (n_qubits < 2 || n_gates < 0 || (n_gates > 0 && !pairs) || !n_rec) return PC_ERR_INVALID_ARG;
  if (split_index < 0) split_index = n_gates / 2;
  if (split_index > n_gates) return PC_ERR_INVALID_ARG;
  for (int64_t g = 0; g < n_gates; ++g) {
    const int a = pairs[2 * g], b = pairs[2 * g + 1];
    if (a < 0 || b < 0 || a >= n_qubits || b >= n_qubits || a == b) return PC_ERR_INVALID_ARG;
  }
  std::vector<int> lorder, rorder;
  for (int64_t g = split_index; g < n_gates; ++g) lorder.push_back((int)g);
  for (int64_t g = split_index - 1; g >= 0; --g) rorder.push_back((int)g);
  auto L = make_layers(lorder, pairs, n_qubits);
  auto R = make_layers(rorder, pairs, n_qubits);
  Layout lay[2];
  lay[0].reset(n_qubits);
  lay[1].reset(n_qubits);
  int64_t k = 0;
  auto emit = [&](const std::vector<ResolvedOp>& ops) {
    for (const auto& op : ops) {
      if (rec && k < cap) {
        rec[4 * k + 0] = op.side; rec[4 * k + 1] = op.bond; rec[4 * k + 2] = op.kind; rec[4 * k + 3] = op.gate;
      }
      ++k;
    }
  };
  const size_t nl = std::max(L.size(), R.size());
  for (size_t i = 0; i < nl; ++i) {
    if (i < L.size()) emit(plan_layer(PC_SIDE_LEFT, L[i], pairs, lay[0]));
    if (i < R.size()) emit(plan_layer(PC_SIDE_RIGHT, R[i], pairs, lay[1]));
  }
  *n_rec = k;
  return PC_OK;
}

pc_status pc_get_plan(pc_circuit* c, int64_t cap, int32_t* rec, int64_t* n_rec) {
  if (check_circuit(c) != PC_OK || !n_rec) return PC_ERR_INVALID_ARG;
  *n_rec = (int64_t)c->plan_log.size();
  for (int64_t k = 0; rec && k < cap && k < *n_rec; ++k)
    for (int e = 0; e < 5; ++e) rec[5 * k + e] = c->plan_log[k][e];
  return PC_OK;
}

pc_status pc_get_unswap_log(pc_circuit* c, int64_t cap, int32_t* rec, int64_t* n_rec) {
  if (check_circuit(c) != PC_OK || !n_rec) return PC_ERR_INVALID_ARG;
  *n_rec = (int64_t)c->unswap_log.size();
  for (int64_t k = 0; rec && k < cap && k < *n_rec; ++k)
    for (int e = 0; e < 4; ++e) rec[4 * k + e] = c->unswap_log[k][e];
  return PC_OK;
}

pc_status pc_extract_peak(pc_circuit* c, int64_t max_expansions, uint8_t* bits, double* p_peak, double* norm2) {
  if (check_circuit(c) != PC_OK || !bits || !p_peak) return PC_ERR_INVALID_ARG;
  pc_ctx* ctx = c->ctx;
  pc_status st = project(c);
  if (st != PC_OK) return st;
  const int n = c->n;
  const double Z = c->norm2;
  if (!(Z > 0.0)) return fail(ctx, PC_ERR_STATE, "M|0> has zero norm");
  if (max_expansions <= 0) max_expansions = 100000;
  // Best-first search: pop the open prefix with the largest marginal (ties: lexicographic
  // prefix, shorter first); the first complete string popped is the exact argmax.
  struct Node {
    double marg;
    std::vector<uint8_t> prefix;
    int64_t slot;
  };
  auto worse = [](const Node& a, const Node& b) {
    if (a.marg != b.marg) return a.marg < b.marg;
    return b.prefix < a.prefix;
  };
  std::priority_queue<Node, std::vector<Node>, decltype(worse)> heap(worse);
  const int CH = c->chi_max;
  int64_t cap_slots = 4096;
  double2* pool = nullptr;
  double* d_marg = nullptr;
  CUDA_TRY(ctx, cudaMalloc(&pool, (size_t)cap_slots * CH * sizeof(double2)));
  CUDA_TRY(ctx, cudaMalloc(&d_marg, 2 * sizeof(double)));
  CUDA_TRY(ctx, pc::launch_fill_ones(pool, 1, c->stream));
  count_launch(c);
  int64_t used = 1;
  heap.push(Node{1.0, {}, 0});
  int64_t expansions = 0;
  pc_status result = PC_ERR_NOT_PEAKED;
  double hm[2];
  while (!heap.empty()) {
    Node top = heap.top();
    heap.pop();
    if ((int)top.prefix.size() == n) {
      for (int q = 0; q < n; ++q) bits[q] = top.prefix[c->lay[PC_SIDE_LEFT].pos[q]];
      *p_peak = top.marg;
      if (norm2) *norm2 = Z * std::ldexp(1.0, n);
      result = PC_OK;
      break;
    }
    if (++expansions > max_expansions) break;
    if (used + 2 > cap_slots) {
      double2* bigger = nullptr;
      cudaError_t e = cudaMalloc(&bigger, (size_t)cap_slots * 2 * CH * sizeof(double2));
      if (e != cudaSuccess) { cudaFree(pool); cudaFree(d_marg); return fail(ctx, PC_ERR_OOM, "peak search pool"); }
      cudaMemcpyAsync(bigger, pool, (size_t)used * CH * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream);
      cudaStreamSynchronize(c->stream);
      cudaFree(pool);
      pool = bigger;
      cap_slots *= 2;
    }
    const int j = (int)top.prefix.size();
    const int cl = c->chi[j], cr = c->chi[j + 1];
    double2* w0 = pool + (size_t)used * CH;
    double2* w1 = pool + (size_t)(used + 1) * CH;
    cudaError_t e = pc::launch_expand(pool + (size_t)top.slot * CH, site_ptr(c, j), cl, cr, c->d_env + c->env_off[j + 1],
                                      w0, w1, d_marg, c->stream);
    count_launch(c);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hm, d_marg, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { cudaFree(pool); cudaFree(d_marg); return fail(ctx, PC_ERR_CUDA, cudaGetErrorString(e)); }
    for (int sg = 0; sg < 2; ++sg) {
      Node ch{hm[sg] / Z, top.prefix, used + sg};
      ch.prefix.push_back((uint8_t)sg);
      heap.push(std::move(ch));
    }
    used += 2;
  }
  cudaFree(pool);
  cudaFree(d_marg);
  if (result != PC_OK) return fail(ctx, PC_ERR_NOT_PEAKED, "peak search exceeded the expansion cap");
  return PC_OK;
}

namespace {

// Shared driver of sampling and amplitudes: V (rows x chi_j) is pushed through each site.
pc_status sweep_rows(pc_circuit* c, int rows, const double* d_u, uint8_t* d_site_bits, bool sampling,
                     double2* d_amp_out) {
  pc_ctx* ctx = c->ctx;
  const int n = c->n, CH = c->chi_max;
  double2 *V = nullptr, *V2 = nullptr, *W0 = nullptr, *W1 = nullptr, *Y = nullptr;
  double *m0 = nullptr, *m1 = nullptr;
  const size_t sz = (size_t)rows * CH * sizeof(double2);
  auto cleanup = [&]() { cudaFree(V); cudaFree(V2); cudaFree(W0); cudaFree(W1); cudaFree(Y); cudaFree(m0); cudaFree(m1); };
  if (cudaMalloc(&V, sz) != cudaSuccess || cudaMalloc(&V2, sz) != cudaSuccess || cudaMalloc(&W0, sz) != cudaSuccess ||
      cudaMalloc(&W1, sz) != cudaSuccess || cudaMalloc(&Y, sz) != cudaSuccess ||
      cudaMalloc(&m0, rows * sizeof(double)) != cudaSuccess || cudaMalloc(&m1, rows * sizeof(double)) != cudaSuccess) {
    cleanup();
    return fail(ctx, PC_ERR_OOM, "sampling buffers");
  }
  cudaError_t e = pc::launch_fill_ones(V, rows, c->stream);
  count_launch(c);
  for (int j = 0; j < n && e == cudaSuccess; ++j) {
    const int cl = c->chi[j], cr = c->chi[j + 1];
    pc::GemmDesc g[2];
    for (int sg = 0; sg < 2; ++sg) {
      g[sg] = pc::GemmDesc{};
      g[sg].A = V; g[sg].lda = cl;
      g[sg].B = site_ptr(c, j) + 2 * sg * cr; g[sg].ldb = 4 * cr;
      g[sg].C = sg ? W1 : W0; g[sg].ldc = cr;
      g[sg].M = rows; g[sg].N = cr; g[sg].K = cl; g[sg].opB = 0; g[sg].alpha = 1.0;
    }
    c->h_gemm[0] = g[0];
    c->h_gemm[1] = g[1];
    e = cudaMemcpyAsync(c->d_gemm, c->h_gemm, 2 * sizeof(pc::GemmDesc), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = pc::launch_gemm(c->d_gemm, 2, rows, cr, c->stream);
    count_launch(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) break;
    if (sampling) {
      for (int sg = 0; sg < 2 && e == cudaSuccess; ++sg) {
        pc::GemmDesc q{};
        q.A = sg ? W1 : W0; q.lda = cr;
        q.B = c->d_env + c->env_off[j + 1]; q.ldb = cr;
        q.C = Y; q.ldc = cr;
        q.M = rows; q.N = cr; q.K = cr; q.opB = 0; q.alpha = 1.0;
        c->h_gemm[0] = q;
        e = cudaMemcpyAsync(c->d_gemm, c->h_gemm, sizeof(pc::GemmDesc), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = pc::launch_gemm(c->d_gemm, 1, rows, cr, c->stream);
        if (e == cudaSuccess) e = pc::launch_quadform_rows(q.A, Y, rows, cr, cr, sg ? m1 : m0, c->stream);
        count_launch(c, 2);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      }
      if (e == cudaSuccess) e = pc::launch_sample_pick(W0, W1, m0, m1, d_u, rows, cr, j, n, V2, d_site_bits, c->stream);
    } else {
      e = pc::launch_amp_pick(W0, W1, d_site_bits, rows, cr, j, n, V2, c->stream);
    }
    count_launch(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    std::swap(V, V2);
  }
  pc_status st = PC_OK;
  if (e != cudaSuccess) st = fail(ctx, PC_ERR_CUDA, cudaGetErrorString(e));
  // amplitudes: the final V is rows x 1 (chi_n = 1)
  if (st == PC_OK && !sampling) e = cudaMemcpy(d_amp_out, V, rows * sizeof(double2), cudaMemcpyDeviceToDevice);
  cleanup();
  if (e != cudaSuccess && st == PC_OK) st = fail(ctx, PC_ERR_CUDA, cudaGetErrorString(e));
  return st;
}

}  // namespace

pc_status pc_sample(pc_circuit* c, int64_t n_samples, uint64_t seed, uint8_t* bits) {
  if (check_circuit(c) != PC_OK || n_samples < 0 || (n_samples > 0 && !bits)) return PC_ERR_INVALID_ARG;
  pc_ctx* ctx = c->ctx;
  pc_status st = project(c);
  if (st != PC_OK) return st;
  const int n = c->n;
  const int64_t chunk = 4096;
  std::vector<double> u;
  std::vector<uint8_t> sb;
  for (int64_t base = 0; base < n_samples; base += chunk) {
    const int rows = (int)std::min(chunk, n_samples - base);
    u.resize((size_t)rows * n);
    for (int s = 0; s < rows; ++s)
      for (int j = 0; j < n; ++j)
        u[(size_t)s * n + j] = (double)(splitmix64(seed, (uint64_t)(base + s) * n + j) >> 11) * (1.0 / 9007199254740992.0);
    double* d_u = nullptr;
    uint8_t* d_sb = nullptr;
    CUDA_TRY(ctx, cudaMalloc(&d_u, u.size() * sizeof(double)));
    if (cudaMalloc(&d_sb, (size_t)rows * n) != cudaSuccess) { cudaFree(d_u); return fail(ctx, PC_ERR_OOM, "sample bits"); }
    if (cudaMemcpyAsync(d_u, u.data(), u.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
      cudaFree(d_u);
      cudaFree(d_sb);
      return fail(ctx, PC_ERR_CUDA, "uniforms upload");
    }
    st = sweep_rows(c, rows, d_u, d_sb, true, nullptr);
    sb.resize((size_t)rows * n);
    if (st == PC_OK) cudaMemcpy(sb.data(), d_sb, sb.size(), cudaMemcpyDeviceToHost);
    cudaFree(d_u);
    cudaFree(d_sb);
    if (st != PC_OK) return st;
    for (int s = 0; s < rows; ++s)
      for (int q = 0; q < n; ++q) bits[(size_t)(base + s) * n + q] = sb[(size_t)s * n + c->lay[PC_SIDE_LEFT].pos[q]];
  }
  return PC_OK;
}

pc_status pc_amplitudes(pc_circuit* c, int64_t k, const uint8_t* bits, double* amp) {
  if (check_circuit(c) != PC_OK || k < 0 || (k > 0 && (!bits || !amp))) return PC_ERR_INVALID_ARG;
  pc_ctx* ctx = c->ctx;
  pc_status st = project(c);
  if (st != PC_OK) return st;
  const int n = c->n;
  const int64_t chunk = 4096;
  const double scale = std::pow(2.0, n / 2.0);
  std::vector<uint8_t> sb;
  std::vector<double2> res;
  for (int64_t base = 0; base < k; base += chunk) {
    const int rows = (int)std::min(chunk, k - base);
    sb.resize((size_t)rows * n);
    for (int s = 0; s < rows; ++s)
      for (int q = 0; q < n; ++q) sb[(size_t)s * n + c->lay[PC_SIDE_LEFT].pos[q]] = bits[(size_t)(base + s) * n + q];
    uint8_t* d_sb = nullptr;
    double2* d_amp = nullptr;
    CUDA_TRY(ctx, cudaMalloc(&d_sb, sb.size()));
    if (cudaMalloc(&d_amp, rows * sizeof(double2)) != cudaSuccess) { cudaFree(d_sb); return fail(ctx, PC_ERR_OOM, "amplitudes"); }
    if (cudaMemcpyAsync(d_sb, sb.data(), sb.size(), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
      cudaFree(d_sb);
      cudaFree(d_amp);
      return fail(ctx, PC_ERR_CUDA, "bit strings upload");
    }
    st = sweep_rows(c, rows, nullptr, d_sb, false, d_amp);
    res.resize(rows);
    if (st == PC_OK && cudaMemcpy(res.data(), d_amp, rows * sizeof(double2), cudaMemcpyDeviceToHost) != cudaSuccess)
      st = fail(ctx, PC_ERR_CUDA, "amplitude copy");
    cudaFree(d_sb);
    cudaFree(d_amp);
    if (st != PC_OK) return st;
    for (int s = 0; s < rows; ++s) {
      amp[2 * (base + s)] = res[s].x * scale;
      amp[2 * (base + s) + 1] = res[s].y * scale;
    }
  }
  return PC_OK;
}

pc_status pc_batch_create(pc_ctx* ctx, int32_t max_tasks, int64_t arena_bytes, pc_batch** out) {
  if (!ctx || !out || max_tasks < 1 || max_tasks > 256 || arena_bytes < 0) return PC_ERR_INVALID_ARG;
  *out = nullptr;
  if (cudaSetDevice(ctx->cfg.device) != cudaSuccess) return fail(ctx, PC_ERR_CUDA, "cudaSetDevice");
  auto* b = new pc_batch();
  b->ctx = ctx;
  const size_t limit = arena_bytes > 0 ? (size_t)arena_bytes : (size_t)8 << 30;
  cudaError_t e = ws_create(max_tasks, limit, ctx->sm_count, nullptr, &b->ws);
  if (e != cudaSuccess) {
    delete b;
    return fail(ctx, e == cudaErrorMemoryAllocation ? PC_ERR_OOM : PC_ERR_CUDA, cudaGetErrorString(e));
  }
  b->launcher = std::thread(batch_loop, b);
  *out = b;
  return PC_OK;
}

pc_status pc_batch_destroy(pc_batch* b) {
  if (!b) return PC_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(b->mu);
    b->stop = true;
  }
  b->cv_post.notify_all();
  if (b->launcher.joinable()) b->launcher.join();
  ws_destroy(b->ws);
  delete b;
  return PC_OK;
}

pc_status pc_batch_attach(pc_batch* b, pc_circuit* c) {
  if (!b || check_circuit(c) != PC_OK) return PC_ERR_INVALID_ARG;
  if (c->batch && c->batch != b) return fail(c->ctx, PC_ERR_STATE, "circuit is attached to another batch");
  if (c->ctx->cfg.device != b->ctx->cfg.device) return fail(c->ctx, PC_ERR_INVALID_ARG, "batch on another device");
  c->batch = b;
  return PC_OK;
}

pc_status pc_batch_detach(pc_batch* b, pc_circuit* c) {
  if (!b || check_circuit(c) != PC_OK || c->batch != b) return PC_ERR_INVALID_ARG;
  c->batch = nullptr;
  return PC_OK;
}

pc_status pc_batch_contract(pc_batch* b, int32_t n, pc_circuit* const* circuits, pc_status* statuses,
                            pc_stats* stats) {
  if (!b || n < 0 || (n > 0 && (!circuits || !statuses))) return PC_ERR_INVALID_ARG;
  for (int32_t k = 0; k < n; ++k) {
    if (check_circuit(circuits[k]) != PC_OK) return PC_ERR_INVALID_ARG;
    for (int32_t i = 0; i < k; ++i)
      if (circuits[i] == circuits[k]) return PC_ERR_INVALID_ARG;
  }
  for (int32_t k = 0; k < n; ++k) {
    pc_status st = pc_batch_attach(b, circuits[k]);
    if (st != PC_OK) {
      for (int32_t i = 0; i < k; ++i) pc_batch_detach(b, circuits[i]);
      return st;
    }
  }
  std::vector<std::thread> th;
  th.reserve(n);
  for (int32_t k = 0; k < n; ++k)
    th.emplace_back([=] {
      pc_stats local{};
      statuses[k] = pc_contract(circuits[k], &local);
      if (stats) stats[k] = local;
    });
  for (auto& t : th) t.join();
  for (int32_t k = 0; k < n; ++k) pc_batch_detach(b, circuits[k]);
  pc_status worst = PC_OK;
  for (int32_t k = 0; k < n; ++k)
    if (statuses[k] < 0) worst = statuses[k];
  return worst;
}

pc_status pc_batch_counters(pc_batch* b, int64_t* launches, int64_t* tasks, int32_t* max_tasks, double* ms,
                            double* flops) {
  if (!b) return PC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(b->mu);
  if (launches) *launches = b->ws->n_launches;
  if (tasks) *tasks = b->ws->n_tasks;
  if (max_tasks) *max_tasks = b->ws->max_tasks_seen;
  for (int k = 0; k < 6; ++k) {
    if (ms) ms[k] = b->ws->t_ms[k];
    if (flops) flops[k] = b->ws->t_flops[k];
  }
  return PC_OK;
}

pc_status pc_batch_set_timing(pc_batch* b, int32_t enable) {
  if (!b) return PC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(b->mu);
  b->ws->timing = enable != 0;
  return PC_OK;
}

int64_t pc_projected_bytes(int32_t n_qubits, int32_t chi_max, int64_t n_samples) {
  if (n_qubits < 2 || chi_max < 1 || n_samples < 0) return -1;
  return (int64_t)store_bytes(n_qubits, chi_max, n_samples);
}

pc_status pc_kernel_timers(pc_circuit* c, int64_t* launches, double* ms, double* flops) {
  if (check_circuit(c) != PC_OK) return PC_ERR_INVALID_ARG;
  for (int k = 0; k < 6; ++k) {
    const Workspace* w = c->ws;
    if (launches) launches[k] = (w ? w->t_launch[k] : 0) + (k == 4 ? c->other_launches : 0);
    if (ms) ms[k] = w ? w->t_ms[k] : 0.0;
    if (flops) flops[k] = w ? w->t_flops[k] : 0.0;
  }
  return PC_OK;
}

pc_status pc_autotune(int32_t device, int32_t n_shapes, const int32_t* lens, const int32_t* batches,
                      const char* path, double* ms_out) {
  if (n_shapes < 1 || !lens || !batches) return PC_ERR_INVALID_ARG;
  for (int i = 0; i < n_shapes; ++i)
    if (lens[i] < 4 || lens[i] > 4096 || batches[i] < 1 || batches[i] > 64) return PC_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return PC_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return PC_ERR_CUDA;
  std::FILE* f = path ? std::fopen(path, "w") : nullptr;
  if (path && !f) return PC_ERR_INVALID_ARG;
  if (f) std::fprintf(f, "# FP64 Jacobi group width: len_bucket pairs_bucket width ms(w=1) ms(w=2) ms(w=4)\n");
  pc_status res = PC_OK;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    res = PC_ERR_CUDA;
  for (int i = 0; i < n_shapes && res == PC_OK; ++i) {
    const int L = lens[i], T = batches[i];
    const size_t cells = (size_t)L * L;
    // T random square matrices (SplitMix64 uniforms), a pristine copy and a working copy
    std::vector<double2> h(cells * T);
    for (size_t e = 0; e < h.size(); ++e) {
      const double a = (double)(splitmix64(0xA070u + (uint64_t)L, 2 * e) >> 11) * (1.0 / 9007199254740992.0);
      const double b = (double)(splitmix64(0xA070u + (uint64_t)L, 2 * e + 1) >> 11) * (1.0 / 9007199254740992.0);
      h[e] = make_double2(a - 0.5, b - 0.5);
    }
    double2 *d0 = nullptr, *d1 = nullptr;
    double* nrm = nullptr;
    int32_t* stamp = nullptr;
    pc::JacobiTask* dt = nullptr;
    pc::JacobiStatus* ds = nullptr;
    unsigned int* bar = nullptr;
    int* err = nullptr;
    std::vector<pc::JacobiTask> ht(T);
    if (cudaMalloc(&d0, h.size() * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&d1, h.size() * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&nrm, (size_t)T * L * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&stamp, (size_t)T * L * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&dt, T * sizeof(pc::JacobiTask)) != cudaSuccess ||
        cudaMalloc(&ds, T * sizeof(pc::JacobiStatus)) != cudaSuccess ||
        cudaMalloc(&bar, 2 * sizeof(unsigned int)) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
      res = PC_ERR_OOM;
    }
    if (res == PC_OK &&
        (cudaMemcpyAsync(d0, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice, st) != cudaSuccess ||
         cudaStreamSynchronize(st) != cudaSuccess))
      res = PC_ERR_CUDA;
    for (int t = 0; t < T && res == PC_OK; ++t) {
      pc::JacobiTask& j = ht[t];
      j = pc::JacobiTask{};
      j.X = d1 + (size_t)t * cells; j.nrm2 = nrm + (size_t)t * L; j.stamp = stamp + (size_t)t * L;
      j.m = L; j.n = L; j.mp = L + (L & 1);
    }
    if (res == PC_OK && cudaMemcpyAsync(dt, ht.data(), T * sizeof(pc::JacobiTask), cudaMemcpyHostToDevice, st) != cudaSuccess)
      res = PC_ERR_CUDA;
    const int pairs = T * ((L + (L & 1)) / 2);
    double best_ms = 1e300, ms_g[3] = {0, 0, 0};
    int best_g = 0;
    for (int gi = 0; gi < 3 && res == PC_OK; ++gi) {
      const int g = 1 << gi;
      double best_rep = 1e300;
      for (int rep = 0; rep < 3 && res == PC_OK; ++rep) {    // the first run warms up
        float ms = 0.0f;
        if (cudaMemcpyAsync(d1, d0, h.size() * sizeof(double2), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            pc::launch_init_stamps(dt, T, L, st) != cudaSuccess ||
            cudaMemsetAsync(ds, 0, T * sizeof(pc::JacobiStatus), st) != cudaSuccess ||
            cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned int), st) != cudaSuccess ||
            cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess || cudaEventRecord(e0, st) != cudaSuccess ||
            pc::launch_jacobi(dt, T, ds, 2, bar, err, sms, L, pairs, st, g) != cudaSuccess ||
            cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          res = PC_ERR_CUDA;
          break;
        }
        if (rep > 0) best_rep = std::min(best_rep, (double)ms);
      }
      ms_g[gi] = best_rep;
      if (best_rep < best_ms) { best_ms = best_rep; best_g = g; }
    }
    int herr = 0;
    if (res == PC_OK && (cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || herr))
      res = herr ? PC_ERR_TIMEOUT : PC_ERR_CUDA;
    if (res == PC_OK) {
      int bl = 0, bp = 0;
      while ((1 << bl) < L && bl < pc::JAC_TUNE_LEN - 1) ++bl;
      while ((2 << bp) <= pairs && bp < pc::JAC_TUNE_PAIRS - 1) ++bp;
      pc::set_jacobi_tuning(bl, bp, best_g);
      if (f) std::fprintf(f, "%d %d %d %.4f %.4f %.4f\n", bl, bp, best_g, ms_g[0], ms_g[1], ms_g[2]);
      if (ms_out) for (int k = 0; k < 3; ++k) ms_out[3 * i + k] = ms_g[k];
    }
    cudaFree(d0); cudaFree(d1); cudaFree(nrm); cudaFree(stamp); cudaFree(dt); cudaFree(ds); cudaFree(bar); cudaFree(err);
  }
  if (f) std::fclose(f);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  return res;
}

pc_status pc_load_tuning(const char* path) {
  if (!path) return PC_ERR_INVALID_ARG;
  std::FILE* f = std::fopen(path, "r");
  if (!f) return PC_ERR_INVALID_ARG;
  char line[512];
  int n = 0;
  while (std::fgets(line, sizeof line, f)) {
    if (line[0] == '#') continue;
    int bl = -1, bp = -1, g = 0;
    if (std::sscanf(line, "%d %d %d", &bl, &bp, &g) == 3 && (g == 0 || g == 1 || g == 2 || g == 4)) {
      pc::set_jacobi_tuning(bl, bp, g);
      ++n;
    }
  }
  std::fclose(f);
  return n > 0 ? PC_OK : PC_ERR_INVALID_ARG;
}

pc_status pc_measure_alu_peaks(int32_t device, double* fp64_tflops, double* fp32_tflops) {
  if (!fp64_tflops || !fp32_tflops) return PC_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return PC_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return PC_ERR_CUDA;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  void* out = nullptr;
  pc_status res = PC_OK;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess || cudaMalloc(&out, 16) != cudaSuccess)
    res = PC_ERR_CUDA;
  const int blocks = sms * 8;
  for (int fp64 = 1; fp64 >= 0 && res == PC_OK; --fp64) {
    const int iters = fp64 ? 4096 : 65536;
    double best = 0.0;
    for (int rep = 0; rep < 4 && res == PC_OK; ++rep) {   // first launch is a warm-up
      float ms = 0.0f;
      if (cudaEventRecord(e0, st) != cudaSuccess || pc::launch_fma_probe(fp64, blocks, iters, out, st) != cudaSuccess ||
          cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        res = PC_ERR_CUDA;
        break;
      }
      const double flops = 2.0 * 8.0 * (double)iters * 256.0 * blocks;
      if (rep > 0 && ms > 0.0f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
    (fp64 ? *fp64_tflops : *fp32_tflops) = best;
  }
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  return res;
}

pc_status pc_get_stream(pc_circuit* c, void** stream) {
  if (check_circuit(c) != PC_OK || !stream) return PC_ERR_INVALID_ARG;
  *stream = (void*)c->stream;
  return PC_OK;
}

pc_status pc_reset_kernel_timers(pc_circuit* c, int32_t enable) {
  if (check_circuit(c) != PC_OK) return PC_ERR_INVALID_ARG;
  c->other_launches = 0;
  c->timing = enable != 0;
  if (c->ws) {
    for (int k = 0; k < 6; ++k) { c->ws->t_launch[k] = 0; c->ws->t_ms[k] = 0.0; c->ws->t_flops[k] = 0.0; }
    c->ws->timing = c->timing;
  }
  return PC_OK;
}

}  // extern "C"
