// pc_factorise_noalloc: one bond factorisation that allocates no device memory.
//
// Callers such as a host application that must keep its device-memory footprint fixed
// after start-up, a plugin living inside a framework that owns every device allocation, or
// code that runs where cudaMalloc is not allowed (e.g. a critical section of a stream-ordered
// memory pool) cannot let the library allocate scratch per call.  This entry point runs the
// same one-sided Jacobi, truncation and V^dagger extraction as a two-site update, but every
// byte of scratch lives in one file-scope __device__ array of fixed size, so it needs no
// allocation at all: the caller passes the input and output device buffers.
//
// Limits and sharing rules (also in include/peaked_mpo.h):
//   - bond matrices up to NA_MAX_DIM x NA_MAX_DIM (256 x 256, i.e. bond dimensions <= 64);
//   - every GPU that loads the library holds the array (about 2.1 MB) until the process exits;
//   - every call on a device shares the array; calls that overlap on the GPU race;
//   - the first call on a device resolves the array's device address (cudaGetSymbolAddress
//     with that device current); make that first call before any stream capture;
//   - the call is synchronous: it reads the kept count back and synchronises the stream
//     before it returns;
//   - the resolved address is cached per device for the life of the process; after a
//     cudaDeviceReset of that device it is stale, so do not call this entry point again
//     in a process that reset the device.
#include "../../include/peaked_mpo.h"
#include "pc_internal.h"

#include <mutex>

namespace {

constexpr int NA_MAX_DIM = 256;
constexpr size_t NA_MAT = (size_t)NA_MAX_DIM * NA_MAX_DIM;
constexpr int NA_MAX_DEVICES = 64;
constexpr int NA_MAX_SWEEPS = 60;

struct NoAllocScratch {
  double2 X[NA_MAT];            // working matrix: the rows, or the columns when m > n
  double2 Q[NA_MAT];            // accumulated rotations (column path)
  double nrm2[NA_MAX_DIM];
  int32_t idx[NA_MAX_DIM];
  double lam[NA_MAX_DIM];
  double sraw[NA_MAX_DIM];
  int32_t stamp[NA_MAX_DIM];
  pc::JacobiTask jtask;
  pc::JacobiStatus jst;
  pc::TruncOut tout;
  unsigned int bar[2];
  int err;
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

NoAllocScratch* g_scratch_dev[NA_MAX_DEVICES] = {};
int g_sm_count[NA_MAX_DEVICES] = {};
std::mutex g_setup_mutex;

// Writes the task descriptor and resets everything that must start cleared (status,
// barrier, error flag, row stamps at -1).
__global__ void noalloc_setup_kernel(NoAllocScratch* s, int m, int n, int transposed) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  pc::JacobiTask t;
  t.X = s->X;
  t.Q = transposed ? s->Q : nullptr;
  t.nrm2 = s->nrm2;
  t.fro2 = nullptr;
  t.stamp = s->stamp;
  t.dead2_ovr = nullptr;
  for (int k = 0; k < NA_MAX_DIM; ++k) s->stamp[k] = -1;
  t.dead_rel = 0.0;
  t.m = transposed ? n : m;
  t.n = transposed ? m : n;
  t.mp = t.m + (t.m & 1);
  t.pad_ = 0;
  s->jtask = t;
  s->jst = pc::JacobiStatus{};
  s->tout = pc::TruncOut{};
  s->bar[0] = s->bar[1] = 0u;
  s->err = 0;
}

// Copies the caller's m x n bond matrix into the scratch, transposed when m > n.
__global__ void noalloc_load_kernel(NoAllocScratch* s, const double2* x, int m, int n, int transposed) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)m * n) return;
  const int r = (int)(e / n), c = (int)(e % n);
  s->X[transposed ? (size_t)c * m + r : (size_t)e] = x[e];
}

// Kept values (normalised) and kept right singular vectors as rows of V^dagger.
__global__ void noalloc_emit_kernel(const NoAllocScratch* s, int n, int transposed, double* s_out,
                                    double2* vh_out) {
  const int count = s->tout.count;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) s_out[e] = s->lam[e];
  if (e >= (long long)count * n) return;
  const int k = (int)(e / n), c = (int)(e % n);
  const int row = s->idx[k];
  if (transposed) {
    const double2 q = s->Q[(size_t)row * n + c];
    vh_out[e] = make_double2(q.x, -q.y);
  } else {
    const double2 v = s->X[(size_t)row * n + c];
    const double inv = 1.0 / s->sraw[k];
    vh_out[e] = make_double2(v.x * inv, v.y * inv);
  }
}

}  // namespace

extern "C" pc_status pc_factorise_noalloc(const double* x_dev, int32_t m, int32_t n, double eps, int32_t chi_max,
                                          double* s_dev, double* vh_dev, int32_t* count, void* stream) {
  if (!x_dev || !s_dev || !vh_dev || !count || m < 1 || n < 1 || m > NA_MAX_DIM || n > NA_MAX_DIM ||
      !(eps >= 0.0) || chi_max < 1)
    return PC_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return PC_ERR_CUDA;
  NoAllocScratch* scr = nullptr;
  int sms = 0;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_dev[dev]) {
      // once per device, with that device current: the device address of the array
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PC_ERR_CUDA;
      int count_sm = 0;
      if (cudaDeviceGetAttribute(&count_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PC_ERR_CUDA;
      g_scratch_dev[dev] = static_cast<NoAllocScratch*>(p);
      g_sm_count[dev] = count_sm;
    }
    scr = g_scratch_dev[dev];
    sms = g_sm_count[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int transposed = m > n ? 1 : 0;
  const int nvec = transposed ? n : m, len = transposed ? m : n;
  const int keep_max = chi_max < nvec ? chi_max : nvec;
  noalloc_setup_kernel<<<1, 1, 0, st>>>(scr, m, n, transposed);
  noalloc_load_kernel<<<(unsigned)(((long long)m * n + 255) / 256), 256, 0, st>>>(
      scr, reinterpret_cast<const double2*>(x_dev), m, n, transposed);
  if (cudaGetLastError() != cudaSuccess) return PC_ERR_CUDA;
  if (pc::launch_init_accumulators(&scr->jtask, 1, nvec, st) != cudaSuccess) return PC_ERR_CUDA;
  if (pc::launch_jacobi(&scr->jtask, 1, &scr->jst, NA_MAX_SWEEPS, scr->bar, &scr->err, sms, len, (nvec + 1) / 2,
                       st) != cudaSuccess)
    return PC_ERR_CUDA;
  if (pc::launch_truncate(&scr->jtask, 1, eps, keep_max, scr->idx, 0, scr->lam, scr->sraw, 0, &scr->tout, st) !=
      cudaSuccess)
    return PC_ERR_CUDA;
  noalloc_emit_kernel<<<(unsigned)(((long long)keep_max * n + 255) / 256), 256, 0, st>>>(
      scr, n, transposed, s_dev, reinterpret_cast<double2*>(vh_dev));
  if (cudaGetLastError() != cudaSuccess) return PC_ERR_CUDA;
  int32_t k = 0, converged = 0, err = 0;
  if (cudaMemcpyAsync(&k, &scr->tout.count, sizeof(k), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&converged, &scr->jst.converged, sizeof(converged), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&err, &scr->err, sizeof(err), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PC_ERR_CUDA;
  if (err) return PC_ERR_TIMEOUT;
  if (!converged) return PC_ERR_NOCONVERGE;
  *count = k;
  return PC_OK;
}
