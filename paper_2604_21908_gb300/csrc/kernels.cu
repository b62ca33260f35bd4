// CUDA kernels of the middle-out MPO contraction (sm_103a).
//
// The hot path of every two-site update (Sec. II.B.1 of the paper: contract the gate with
// the two MPO site tensors, then an SVD with cutoff eps) is split into
//   merge      : T0 = B_j . B_j+1                        (batched complex FP64 GEMM)
//   gate       : T0 <- U16 T0 on the 16-dim (p_j, p_j+1) index; X = T0 scaled by
//                lambda_{j-1} row-wise, transposed for a tall matrix (gate_apply_kernel)
//   factorise  : one-sided Jacobi on the rows of X      (jacobi_kernel, cooperative)
//   truncate   : sort row norms, relative cutoff, chi_max, renormalise (truncate_kernel)
//   split      : B_j+1 = normalised kept rows (V^dagger), B_j = T0 V / |s| (GEMM)
// All arithmetic is FP64 (double / double2 complex).
#include "pc_internal.h"

#include <cstdio>

namespace pc {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {   // a*b + c
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ double2 conjd(double2 a) { return make_double2(a.x, -a.y); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------------------
// Batched complex FP64 GEMM: 64x64 output tile per CTA, K-step 16, 4x4 outputs per thread.
constexpr int GBM = 64, GBN = 64, GBK = 16;

__global__ void __launch_bounds__(256) gemm_kernel(const GemmDesc* __restrict__ descs) {
  const GemmDesc d = descs[blockIdx.z];
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  if (m0 >= d.M || n0 >= d.N) return;
  __shared__ double2 As[GBK][GBM];
  __shared__ double2 Bs[GBK][GBN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);

  for (int k0 = 0; k0 < d.K; k0 += GBK) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int idx = tid + 256 * i;
      const int r = idx >> 4, c = idx & 15;
      const int gr = m0 + r, gc = k0 + c;
      double2 v = make_double2(0.0, 0.0);
      if (gr < d.M && gc < d.K) {
        v = d.A[(size_t)gr * d.lda + gc];
        if (d.row_scale) { const double s = d.row_scale[gr]; v.x *= s; v.y *= s; }
      }
      As[c][r] = v;
    }
    if (d.opB == 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int idx = tid + 256 * i;
        const int kk = idx >> 6, c = idx & 63;
        const int gk = k0 + kk, gc = n0 + c;
        double2 v = make_double2(0.0, 0.0);
        if (gk < d.K && gc < d.N) v = d.B[(size_t)gk * d.ldb + gc];
        Bs[kk][c] = v;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int idx = tid + 256 * i;
        const int nn = idx >> 4, kk = idx & 15;
        const int gn = n0 + nn, gk = k0 + kk;
        double2 v = make_double2(0.0, 0.0);
        if (gk < d.K && gn < d.N) v = conjd(d.B[(size_t)gn * d.ldb + gk]);
        Bs[kk][nn] = v;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GBK; ++kk) {
      double2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cfma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gr = m0 + ty + 16 * i;
    if (gr >= d.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gc = n0 + tx + 16 * j;
      if (gc >= d.N) continue;
      double2 v = make_double2(d.alpha * acc[i][j].x, d.alpha * acc[i][j].y);
      double2* cp = d.C + (size_t)gr * d.ldc + gc;
      if (d.beta != 0.0) {
        const double2 o = d.D ? d.D[(size_t)gr * d.ldc + gc] : *cp;
        v.x = fma(d.beta, o.x, v.x);
        v.y = fma(d.beta, o.y, v.y);
      }
      *cp = v;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Gate application on the merged two-site tensor.  The merge leaves Theta[l, p1, p2, r] in T0 as
// the (4 chi_l) x (4 chi_r) matrix T0[(l,p1), (p2,r)]; for each (l, r) the 16-vector over
// P = 4 p1 + p2 is multiplied by U.  Each thread reads and rewrites its own 16 entries of T0
// (the gated tensor without lambda) and writes the lambda-scaled entries to X, transposed for a
// tall bond matrix: X is a different buffer, so the transposition never overwrites an entry
// another thread has still to read.
__global__ void __launch_bounds__(256) gate_apply_kernel(const UpdateTask* __restrict__ tasks) {
  const UpdateTask t = tasks[blockIdx.y];
  __shared__ double2 U[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) U[i] = t.op[i];
  __syncthreads();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)t.chi_l * t.chi_r) return;
  const int l = (int)(idx / t.chi_r), r = (int)(idx % t.chi_r);
  const int n = t.n;
  double2 v[16];
#pragma unroll
  for (int p1 = 0; p1 < 4; ++p1)
#pragma unroll
    for (int p2 = 0; p2 < 4; ++p2) v[4 * p1 + p2] = t.T0[(size_t)(4 * l + p1) * n + p2 * t.chi_r + r];
  const double lam = t.lam_l ? t.lam_l[l] : 1.0;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int p = 0; p < 16; ++p) acc = cfma(U[16 * q + p], v[p], acc);
    const int row = 4 * l + (q >> 2), col = (q & 3) * t.chi_r + r;
    t.T0[(size_t)row * n + col] = acc;
    const size_t xo = t.transposed ? (size_t)col * t.m + row : (size_t)row * n + col;
    t.X[xo] = make_double2(acc.x * lam, acc.y * lam);
  }
}

// ---------------------------------------------------------------------------------------
// Grid barrier for the cooperative Jacobi kernel.  The wait is bounded: after about
// 2^26 polls (seconds) the CTA records an error and the kernel returns.
__device__ bool grid_barrier(unsigned int* bar, int* err, unsigned int nblocks) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = bar + 1;
    const unsigned int gen = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(bar, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long polls = 0;
      while (*vgen == gen) {
        if (++polls > (1LL << 26) || *(volatile int*)err) { atomicExch(err, 1); break; }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)err == 0;
}

constexpr int JAC_MAX_TASKS = 256;
constexpr int JAC_THREADS = 512;
constexpr int JAC_E = 8;            // row elements per thread held in registers

// Element and task types of the Jacobi kernel in FP64 (the factorisation) and FP32 (the
// preconditioning sweeps).
template <typename R> struct JacTraits;
template <> struct JacTraits<double> {
  using C = double2;
  using Task = JacobiTask;
  static constexpr double eps = 2.220446049250313e-16;   // 2^-52
  static constexpr double tiny = 1e-280;                   // floor for squared row norms
  static constexpr double g2min = 1e-290;                  // |g|^2 below this is not rotated
  static constexpr double huge = 1e100;
  // Carried squared norms are recomputed exactly (a) when the two of a pair differ by more
  // than `recompute` (each rotation moves a carried value by roundoff of the larger norm),
  // (b) when they agree to `degenerate` (the rotation angle depends on their difference,
  // which carried roundoff would swamp), (c) when an update cancelled below `cancel` of the
  // old value (marked by a negative carried value).
  static constexpr double recompute = 1e-8;
  static constexpr double degenerate = 1e-8;
  static constexpr double cancel = 1e-3;
};
template <> struct JacTraits<float> {
  using C = float2;
  using Task = JacobiTask32;
  static constexpr float eps = 1.1920929e-7f;              // 2^-23
  // Rows of a normalised bond matrix below 1e-15 in norm, and inner products whose square
  // would be subnormal in FP32 (where |g| / sqrt(g^2) is no longer 1 to FP32 precision and
  // the rotation would stop being unitary), are left to the FP64 sweeps.
  static constexpr float tiny = 1e-30f;
  static constexpr float g2min = 1e-36f;
  static constexpr float huge = 1e18f;
  static constexpr float recompute = 1e-3f;
  static constexpr float degenerate = 1e-3f;
  static constexpr float cancel = 0.1f;
};

__device__ __forceinline__ double2 mk2(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ float2 mk2(float x, float y) { return make_float2(x, y); }

template <typename R>
struct Rot {
  R c, sn, wx, wy, zx, zy;
};

// Products that the compiler must not fuse into a neighbouring addition (an explicit rounding).
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

// [u, v] <- [c u - s e v, s u + c e v] with e = e^{-i phi} (exactly unitary for c^2+s^2=1, |e|=1).
// Written with explicit fused multiply-adds and unfused products, so no multiply-add is left for
// the compiler to contract: the rounding is the same in every code path that applies a rotation.
template <typename R, typename C>
__device__ __forceinline__ void rot_apply(const Rot<R>& q, C& u, C& v) {
  C na, nb;
  na.x = fma(q.c, u.x, -fma(q.wx, v.x, -mul_rn(q.wy, v.y)));
  na.y = fma(q.c, u.y, -fma(q.wx, v.y, mul_rn(q.wy, v.x)));
  nb.x = fma(q.sn, u.x, fma(q.zx, v.x, -mul_rn(q.zy, v.y)));
  nb.y = fma(q.sn, u.y, fma(q.zx, v.y, mul_rn(q.zy, v.x)));
  u = na;
  v = nb;
}

template <typename R>
__device__ __forceinline__ R warp_sum_t(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Inner products of a row pair in a fixed order that does not depend on the group width G, so a
// task's rotations (and so its singular values and vectors) are bit-identical in every launch it
// can be part of (alone, batched, any tuned width).  The row, padded to n_pad = 128 ceil(n / 128),
// is cut into four quarters of qseg = n_pad / 128 segments of 32 elements; lane l sums, per quarter,
// its elements 32 s + l in increasing s as one FMA chain (jac_accum); the quarter sums are added as
// (Q0 + Q1) + (Q2 + Q3) and then reduced over the 32 lanes by an xor butterfly (jac_reduce).  In a
// group of G warps, warp w owns quarters w (4 / G) ... (w + 1)(4 / G) - 1.
// a[0] += |u|^2, a[1] += |v|^2 (only when exact), a[2] + i a[3] += conj(u) v
template <typename R, typename C>
__device__ __forceinline__ void jac_accum(R (&a)[4], const C u, const C v, bool exact) {
  a[2] = fma(u.x, v.x, fma(u.y, v.y, a[2]));
  a[3] = fma(u.x, v.y, fma(-u.y, v.x, a[3]));
  if (exact) {
    a[0] = fma(u.x, u.x, fma(u.y, u.y, a[0]));
    a[1] = fma(v.x, v.x, fma(v.y, v.y, a[1]));
  }
}

// The quarter sums of the group's threads -> the four totals, identical on every thread of the
// group.  xs: this group's exchange slab in shared memory, [4][32 G] values (unused for G = 1).
template <typename R, int G>
__device__ __forceinline__ void jac_reduce(R (&acc)[4 / G][4], R* xs, int grp, int gl, R& a, R& b, R& c,
                                           R& d) {
  constexpr int GT = 32 * G;
  R t[4];
  if constexpr (G == 1) {
#pragma unroll
    for (int v = 0; v < 4; ++v) t[v] = (acc[0][v] + acc[1][v]) + (acc[2][v] + acc[3][v]);
  } else {
    const int lane = gl & 31;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      if constexpr (G == 2) xs[v * GT + gl] = acc[0][v] + acc[1][v];
      else xs[v * GT + gl] = acc[0][v];
    }
    __syncwarp();   // bar.sync wants each warp converged
    asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(GT) : "memory");
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const R* x = xs + v * GT + lane;
      if constexpr (G == 2) t[v] = x[0] + x[32];
      else t[v] = (x[0] + x[32]) + (x[64] + x[96]);
    }
  }
  a = warp_sum_t(t[0]);
  b = warp_sum_t(t[1]);
  c = warp_sum_t(t[2]);
  d = warp_sum_t(t[3]);
}

// Bytes of dynamic shared memory of jacobi_kernel<R, G>: the double-buffered exchange slabs.
template <typename R, int G>
constexpr int jac_dyn_smem() { return G == 1 ? 0 : 2 * JAC_THREADS * 4 * (int)sizeof(R); }

// One-sided (Hestenes) Jacobi on the rows of each task's matrix: rotate pairs of rows until
// every pair is orthogonal to |<x_a, x_b>| <= tol |x_a| |x_b|, tol = 2 eps sqrt(n) (eps the
// unit roundoff of R).  Pairs follow the round-robin (circle) ordering: in round r of a sweep
// over mp rows, pair 0 = (mp-1, r), pair i = ((r+i) mod (mp-1), (r-i) mod (mp-1)).  Each
// global iteration runs one round of every unfinished task (tasks of different sizes advance
// their own sweeps), then all CTAs meet at a grid barrier.  A group of G warps rotates one pair;
// its inner products follow the width-independent order of jac_accum / jac_reduce.
// Squared row norms are computed exactly in round 0 of every sweep and carried through the
// sweep with the exact-arithmetic update a' = a - t|g|, b' = b + t|g|; a sweep with no
// rotation leaves them untouched, so the convergence decision always uses exact norms.
template <typename R, int G>
__global__ void __launch_bounds__(JAC_THREADS, 1) jacobi_kernel(const typename JacTraits<R>::Task* __restrict__ tasks,
                                                               int ntasks, JacobiStatus* st,
                                                               int max_sweeps, unsigned int* bar,
                                                               int* err) {
  using C = typename JacTraits<R>::C;
  using Task = typename JacTraits<R>::Task;
  constexpr int GT = 32 * G;
  constexpr int NG = JAC_THREADS / GT;
  __shared__ int s_off[JAC_MAX_TASKS + 1];
  __shared__ unsigned char s_done[JAC_MAX_TASKS];
  __shared__ Task s_task[JAC_MAX_TASKS];
  extern __shared__ __align__(16) unsigned char jac_dyn[];
  R* const s_xch = reinterpret_cast<R*>(jac_dyn);     // [2][JAC_THREADS][4] when G > 1
  __shared__ R s_rot[NG][8];
  __shared__ R s_dead2[JAC_MAX_TASKS];
  __shared__ R s_marg2[JAC_MAX_TASKS];
  for (int t = threadIdx.x; t < ntasks; t += blockDim.x) {
    s_done[t] = 0;
    s_task[t] = tasks[t];
    R d2 = s_task[t].fro2 ? (R)(s_task[t].dead_rel * *s_task[t].fro2) : R(0);
    if (s_task[t].dead2_ovr) d2 = fmax(d2, (R)*s_task[t].dead2_ovr);
    s_dead2[t] = d2;
    s_marg2[t] = R(6 * s_task[t].m) * s_dead2[t];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int off = 0;
    for (int t = 0; t < ntasks; ++t) { s_off[t] = off; off += s_task[t].mp >> 1; }
    s_off[ntasks] = off;
  }
  __syncthreads();
  const int grp = threadIdx.x / GT, gl = threadIdx.x % GT;
  // consecutive pairs go to consecutive CTAs, so a round with fewer pairs than groups still
  // spreads over every SM
  const int ggrp = grp * gridDim.x + blockIdx.x, ngrp = gridDim.x * NG;
  const int total = s_off[ntasks];
  const R eps = JacTraits<R>::eps;
  int parity = 0;

  for (long long g = 0;; ++g) {
    for (int t = threadIdx.x; t < ntasks; t += blockDim.x) {
      if (s_done[t]) continue;
      const long long Rr = s_task[t].mp - 1;
      const long long s = g / Rr;
      const long long r = g - s * Rr;
      if (r == 0 && s > 0) {
        const unsigned int rc = *(volatile unsigned int*)&st[t].rot[(s - 1) % 3];
        if (rc == 0 || s >= max_sweeps) {
          s_done[t] = 1;
          if (blockIdx.x == 0) { st[t].sweeps = (int)s; st[t].converged = rc == 0 ? 1 : 0; }
          continue;
        }
      }
      if (r == 0 && blockIdx.x == 0) st[t].rot[(s + 1) % 3] = 0u;
    }
    __syncthreads();
    int mine = 1;
    for (int t = threadIdx.x; t < ntasks; t += blockDim.x) mine &= s_done[t];
    if (__syncthreads_and(mine)) break;

    for (int item = ggrp; item < total; item += ngrp) {
      int lo = 0, hi = ntasks - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_off[mid] <= item) lo = mid; else hi = mid - 1;
      }
      const int t = lo;
      if (s_done[t]) continue;
      const Task& tk = s_task[t];
      const int Rr = tk.mp - 1;
      const long long s = g / Rr;
      const int r = (int)(g - s * Rr);
      const int i = item - s_off[t];
      int a, b;
      if (i == 0) { a = tk.mp - 1; b = r; }
      else { a = (r + i) % Rr; b = (r - i + Rr) % Rr; }
      const bool full = (r == 0);
      // unchanged since this pair's check one sweep ago (then below tolerance): skip
      if (s > 0 && a < tk.m && b < tk.m) {
        const int prev = (int)(g - Rr);
        if (tk.stamp[a] < prev && tk.stamp[b] < prev) continue;
      }
      R* const xs = s_xch + (size_t)parity * JAC_THREADS * 4 + (size_t)grp * GT * 4;
      const int n = tk.n;
      const int qseg = (n + 127) >> 7;                    // 32-element segments per quarter
      const int lane = gl & 31, wq = (gl >> 5) * (4 / G);  // this warp's first quarter
      R acc[4 / G][4];
#pragma unroll
      for (int ql = 0; ql < 4 / G; ++ql) acc[ql][0] = acc[ql][1] = acc[ql][2] = acc[ql][3] = R(0);
      if (a >= tk.m || b >= tk.m) {
        // the padding row: in round 0 the real row still gets its exact norm
        if (full) {
          const int v = a < tk.m ? a : b;
          const C* xv = tk.X + (size_t)v * n;
#pragma unroll
          for (int ql = 0; ql < 4 / G; ++ql) {
            const int k0 = 32 * (wq + ql) * qseg + lane;
            for (int j = 0; j < qseg; ++j) {
              const int k = k0 + 32 * j;
              if (k < n) jac_accum(acc[ql], xv[k], xv[k], true);
            }
          }
          R nv, z1, z2, z3;
          jac_reduce<R, G>(acc, xs, grp, gl, nv, z1, z2, z3);
          if (gl == 0) tk.nrm2[v] = nv;
          parity ^= 1;
        }
        continue;
      }
      C* xa = tk.X + (size_t)a * n;
      C* xb = tk.X + (size_t)b * n;
      // the carried norms, fetched early so their latency overlaps the row loads
      R na_pre = R(0), nb_pre = R(0);
      bool exact = full;
      if (!full) {
        na_pre = tk.nrm2[a];
        nb_pre = tk.nrm2[b];
        exact = !(fmin(na_pre, nb_pre) > JacTraits<R>::recompute * fmax(na_pre, nb_pre)) ||
                fabs(na_pre - nb_pre) < JacTraits<R>::degenerate * (na_pre + nb_pre);
      }
      // register slot e holds segment (wq + e / (2G)) qseg + e % (2G) of the pair when the row fits
      const bool in_regs = qseg <= 2 * G;
      C ra[JAC_E], rb[JAC_E];
      if (in_regs) {
#pragma unroll
        for (int e = 0; e < JAC_E; ++e) {
          const int j = e % (2 * G);
          const int k = 32 * ((wq + e / (2 * G)) * qseg + j) + lane;
          const bool ok = j < qseg && k < n;
          ra[e] = ok ? xa[k] : mk2(R(0), R(0));
          rb[e] = ok ? xb[k] : mk2(R(0), R(0));
        }
#pragma unroll
        for (int e = 0; e < JAC_E; ++e) jac_accum(acc[e / (2 * G)], ra[e], rb[e], exact);
      } else {
#pragma unroll
        for (int ql = 0; ql < 4 / G; ++ql) {
          const int k0 = 32 * (wq + ql) * qseg + lane;
          for (int j = 0; j < qseg; ++j) {
            const int k = k0 + 32 * j;
            if (k < n) jac_accum(acc[ql], xa[k], xb[k], exact);
          }
        }
      }
      R aa, bb, gr, gi;
      jac_reduce<R, G>(acc, xs, grp, gl, aa, bb, gr, gi);
      parity ^= 1;
      // The rotation's scalars cost the same pipe time on every warp that computes them
      // (whatever its active lanes), so only the group's first warp does; it shares them
      // through shared memory.  Scalars: |g|^2 against tol^2 a b (no square roots),
      // zeta = (b - a) / (2|g|), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
      // c = 1/sqrt(1 + t^2), s = c t, e = conj(g)/|g|.
      Rot<R> q;
      R tg = R(0);                            // t |g|, for the norm update
      int rotate;
      if (G == 1 || gl < 32) {
        if (!exact) { aa = na_pre; bb = nb_pre; }
        const R g2 = fma(gr, gr, mul_rn(gi, gi));
        const R tol = R(2) * eps * sqrt(R(n));
        // rows at the underflow floor are zero for every purpose here
        // Floors: no pair of two rows below dead2, and no pair of a row below dead2 with a row
        // below marg2 = 6 m dead2, is rotated.  The rows below marg2 stay below the cutoff and
        // are orthogonalised among themselves and against every row above marg2; the rows
        // above marg2 against everything.  Without the second floor a row just above dead2
        // keeps re-mixing the (mutually non-orthogonal) rows below it and converges linearly.
        const R dead2 = s_dead2[t], marg2 = s_marg2[t];
        const R lo2 = fmin(aa, bb), hi2 = fmax(aa, bb);
        rotate = !(aa < JacTraits<R>::tiny || bb < JacTraits<R>::tiny) && !(hi2 < dead2) &&
                 !(lo2 < dead2 && hi2 < marg2) &&
                 g2 >= JacTraits<R>::g2min && (g2 > (tol * tol) * aa * bb);
        if (rotate) {
          const R gabs = sqrt(g2);
          const R inv_g = R(1) / gabs;
          const R zeta = R(0.5) * (bb - aa) * inv_g;
          R tt;
          if (fabs(zeta) > JacTraits<R>::huge) tt = R(0.5) / zeta;
          else tt = copysign(R(1), zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, R(1))));
          // correctly rounded 1/sqrt: an approximate reciprocal square root has a one-signed
          // error that compounds over the tens of thousands of rotations a row takes part in
          q.c = R(1) / sqrt(fma(tt, tt, R(1)));
          q.sn = q.c * tt;
          const R ex = gr * inv_g, ey = -gi * inv_g;        // e^{-i phi}
          q.wx = q.sn * ex; q.wy = q.sn * ey;               // s e^{-i phi}
          q.zx = q.c * ex; q.zy = q.c * ey;                 // c e^{-i phi}
          tg = mul_rn(tt, gabs);
        }
        if constexpr (G > 1) {
          if (gl == 0) {
            R* sh = s_rot[grp];
            sh[0] = rotate ? R(1) : R(0);
            sh[1] = q.c; sh[2] = q.sn; sh[3] = q.wx; sh[4] = q.wy; sh[5] = q.zx; sh[6] = q.zy;
          }
        }
      }
      if constexpr (G > 1) {
        __syncwarp();
        asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(32 * G) : "memory");
        if (gl >= 32) {
          const R* sh = s_rot[grp];
          rotate = sh[0] != R(0);
          q.c = sh[1]; q.sn = sh[2]; q.wx = sh[3]; q.wy = sh[4]; q.zx = sh[5]; q.zy = sh[6];
        }
        // the next write of s_rot comes after the next reduction's barrier, which every warp
        // of the group reaches only after reading these values
      }
      if (!rotate) {
        if (exact && gl == 0) { tk.nrm2[a] = aa; tk.nrm2[b] = bb; }
        continue;
      }
      if (in_regs) {
#pragma unroll
        for (int e = 0; e < JAC_E; ++e) {
          const int j = e % (2 * G);
          const int k = 32 * ((wq + e / (2 * G)) * qseg + j) + lane;
          if (j < qseg && k < n) {
            rot_apply(q, ra[e], rb[e]);
            xa[k] = ra[e];
            xb[k] = rb[e];
          }
        }
      } else {
#pragma unroll
        for (int ql = 0; ql < 4 / G; ++ql) {
          const int k0 = 32 * (wq + ql) * qseg + lane;
          for (int j = 0; j < qseg; ++j) {
            const int k = k0 + 32 * j;
            if (k < n) {
              C u = xa[k], v = xb[k];
              rot_apply(q, u, v);
              xa[k] = u;
              xb[k] = v;
            }
          }
        }
      }
      if (tk.Q) {
        C* qa = tk.Q + (size_t)a * tk.m;
        C* qb = tk.Q + (size_t)b * tk.m;
        for (int k = gl; k < tk.m; k += GT) {
          C u = qa[k], v = qb[k];
          rot_apply(q, u, v);
          qa[k] = u;
          qb[k] = v;
        }
      }
      if (gl == 0) {
        R na = aa - tg, nb = bb + tg;
        if (na < JacTraits<R>::cancel * aa) na = -na;
        if (nb < JacTraits<R>::cancel * bb) nb = -nb;
        tk.nrm2[a] = na;
        tk.nrm2[b] = nb;
        tk.stamp[a] = (int)g;
        tk.stamp[b] = (int)g;
        atomicAdd(&st[t].rot[s % 3], 1u);
      }
    }
    if (!grid_barrier(bar, err, gridDim.x)) return;
  }
}

// ---------------------------------------------------------------------------------------
// Blocked one-sided Jacobi (used for the FP32 preconditioning sweeps).  The v rows of a task
// are cut into blocks of BLK = 8 rows; the blocks are paired round-robin (NB - 1 block rounds per sweep, one
// grid barrier each).  A CTA takes one block pair: its 2 BLK rows go to shared memory (128 KB
// at row length 1024), one inner sweep rotates every pair of them there
// (2 BLK - 1 inner rounds of BLK pairs, two warps per pair), the rotations are accumulated
// into a 2BLK x 2BLK matrix W, and the rows of X and of the accumulator Q (if any) are
// written back once (Q <- W Q).  Per pair of rows this moves a fraction ~1/BLK of the data of
// the row-pair kernel through L2 and needs one grid barrier per block round.  Rotation rule,
// floors and tolerance are the row-pair kernel's; norms are exact (from shared memory).
constexpr int BJ_THREADS = 512;
constexpr int BJ_MAX_LEN = 1024;

template <typename R> struct BjBlock;
template <> struct BjBlock<float> { static constexpr int value = 8; };

template <typename R>
__global__ void __launch_bounds__(BJ_THREADS, 1) bjac_kernel(const typename JacTraits<R>::Task* __restrict__ tasks,
                                                             int ntasks, JacobiStatus* st, int max_sweeps,
                                                             unsigned int* bar, int* err) {
  using C = typename JacTraits<R>::C;
  using Task = typename JacTraits<R>::Task;
  using Tr = JacTraits<R>;
  constexpr int BJ_BLOCK = BjBlock<R>::value;
  constexpr int BJ_ROWS = 2 * BJ_BLOCK;
  extern __shared__ __align__(16) unsigned char bj_raw[];
  C* bj_rows = reinterpret_cast<C*>(bj_raw);               // [BJ_ROWS][Lmax]
  __shared__ C W[BJ_ROWS][BJ_ROWS];
  __shared__ R red[BJ_ROWS / 2][2][4];
  __shared__ int s_grow[BJ_ROWS];
  __shared__ int s_nrot, s_skip;
  __shared__ int s_off[JAC_MAX_TASKS + 1];
  __shared__ int s_nbp[JAC_MAX_TASKS];
  __shared__ unsigned char s_done[JAC_MAX_TASKS];
  __shared__ R s_dead2[JAC_MAX_TASKS], s_marg2[JAC_MAX_TASKS];
  for (int t = threadIdx.x; t < ntasks; t += blockDim.x) {
    const Task tk = tasks[t];
    const int nb = (tk.m + BJ_BLOCK - 1) / BJ_BLOCK;
    s_nbp[t] = nb + (nb & 1);
    s_done[t] = 0;
    s_dead2[t] = tk.fro2 ? (R)(tk.dead_rel * *tk.fro2) : R(0);
    if (tk.dead2_ovr) s_dead2[t] = fmax(s_dead2[t], (R)*tk.dead2_ovr);
    s_marg2[t] = (R)(6 * tk.m) * s_dead2[t];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int off = 0;
    for (int t = 0; t < ntasks; ++t) { s_off[t] = off; off += s_nbp[t] >> 1; }
    s_off[ntasks] = off;
  }
  __syncthreads();
  const int total = s_off[ntasks];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pr = warp >> 1;                                 // the pair this warp serves
  const int t64 = threadIdx.x & 63;

  for (long long g = 0;; ++g) {
    for (int t = threadIdx.x; t < ntasks; t += blockDim.x) {
      if (s_done[t]) continue;
      const long long Rb = s_nbp[t] - 1;
      const long long s = g / Rb, r = g - s * Rb;
      if (r == 0 && s > 0) {
        const unsigned int rc = *(volatile unsigned int*)&st[t].rot[(s - 1) % 3];
        if (rc == 0 || s >= max_sweeps) {
          s_done[t] = 1;
          if (blockIdx.x == 0) { st[t].sweeps = (int)s; st[t].converged = rc == 0 ? 1 : 0; }
          continue;
        }
      }
      if (r == 0 && blockIdx.x == 0) st[t].rot[(s + 1) % 3] = 0u;
    }
    __syncthreads();
    int mine = 1;
    for (int t = threadIdx.x; t < ntasks; t += blockDim.x) mine &= s_done[t];
    if (__syncthreads_and(mine)) break;

    for (int item = blockIdx.x; item < total; item += gridDim.x) {
      int lo = 0, hi = ntasks - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_off[mid] <= item) lo = mid; else hi = mid - 1;
      }
      const int t = lo;
      if (s_done[t]) continue;                             // uniform over the CTA
      const Task tk = tasks[t];
      const int Rb = s_nbp[t] - 1;
      const long long s = g / Rb;
      const int r = (int)(g - s * Rb);
      const int i = item - s_off[t];
      int A, B;
      if (i == 0) { A = s_nbp[t] - 1; B = r; }
      else { A = (r + i) % Rb; B = (r - i + Rb) % Rb; }
      const int L = tk.n, v = tk.m;
      if (threadIdx.x == 0) {
        // blocks unchanged since this block pair's check one sweep ago: skip
        const int prev = (int)(g - Rb);
        const int nb = (v + BJ_BLOCK - 1) / BJ_BLOCK;
        const int sa = A < nb ? __ldcg(tk.stamp + A) : -1, sb = B < nb ? __ldcg(tk.stamp + B) : -1;
        s_skip = (s > 0 && sa < prev && sb < prev) ? 1 : 0;
        s_nrot = 0;
      }
      if (threadIdx.x < BJ_ROWS) {
        const int blk = threadIdx.x < BJ_BLOCK ? A : B;
        const int row = blk * BJ_BLOCK + (threadIdx.x % BJ_BLOCK);
        s_grow[threadIdx.x] = row < v ? row : -1;
      }
      for (int e = threadIdx.x; e < BJ_ROWS * BJ_ROWS; e += blockDim.x)
        W[e / BJ_ROWS][e % BJ_ROWS] = mk2((e / BJ_ROWS) == (e % BJ_ROWS) ? R(1) : R(0), R(0));
      __syncthreads();
      if (s_skip) { __syncthreads(); continue; }
      for (int e = threadIdx.x; e < BJ_ROWS * L; e += blockDim.x) {
        const int rr = e / L, k = e - rr * L;
        const int gr = s_grow[rr];
        bj_rows[rr * L + k] = gr >= 0 ? __ldcg(tk.X + (size_t)gr * L + k) : mk2(R(0), R(0));
      }
      __syncthreads();
      const R tol = R(2) * Tr::eps * sqrt((R)L);
      const R dead2 = s_dead2[t], marg2 = s_marg2[t];
      for (int q = 0; q < BJ_ROWS - 1; ++q) {
        int ia, ib;
        if (pr == 0) { ia = BJ_ROWS - 1; ib = q; }
        else { ia = (q + pr) % (BJ_ROWS - 1); ib = (q - pr + BJ_ROWS - 1) % (BJ_ROWS - 1); }
        if (pr < BJ_BLOCK && s_grow[ia] >= 0 && s_grow[ib] >= 0) {   // uniform over the pair's 64 threads
          C* ra = bj_rows + ia * L;
          C* rb = bj_rows + ib * L;
          R aa = R(0), bb = R(0), gr = R(0), gi = R(0);
          for (int k = t64; k < L; k += 64) {
            const C u = ra[k], w = rb[k];
            aa = fma(u.x, u.x, fma(u.y, u.y, aa));
            bb = fma(w.x, w.x, fma(w.y, w.y, bb));
            gr = fma(u.x, w.x, fma(u.y, w.y, gr));
            gi = fma(u.x, w.y, fma(-u.y, w.x, gi));
          }
          aa = warp_sum_t(aa); bb = warp_sum_t(bb); gr = warp_sum_t(gr); gi = warp_sum_t(gi);
          if (lane == 0) { red[pr][warp & 1][0] = aa; red[pr][warp & 1][1] = bb; red[pr][warp & 1][2] = gr; red[pr][warp & 1][3] = gi; }
          __syncwarp();
          asm volatile("bar.sync %0, %1;" ::"r"(pr + 1), "r"(64) : "memory");
          aa = red[pr][0][0] + red[pr][1][0];
          bb = red[pr][0][1] + red[pr][1][1];
          gr = red[pr][0][2] + red[pr][1][2];
          gi = red[pr][0][3] + red[pr][1][3];
          const R g2 = fma(gr, gr, mul_rn(gi, gi));
          const R lo2 = fmin(aa, bb), hi2 = fmax(aa, bb);
          const bool rotate = !(aa < Tr::tiny || bb < Tr::tiny) && !(hi2 < dead2) && !(lo2 < dead2 && hi2 < marg2) &&
                              g2 >= Tr::g2min && (g2 > (tol * tol) * aa * bb);
          if (rotate) {
            const R gabs = sqrt(g2), inv_g = R(1) / gabs;
            const R zeta = R(0.5) * (bb - aa) * inv_g;
            R tt;
            if (fabs(zeta) > Tr::huge) tt = R(0.5) / zeta;
            else tt = copysign(R(1), zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, R(1))));
            Rot<R> rot;
            // correctly rounded 1/sqrt (as in the row-pair kernel)
            rot.c = R(1) / sqrt(fma(tt, tt, R(1)));
            rot.sn = rot.c * tt;
            const R ex = gr * inv_g, ey = -gi * inv_g;
            rot.wx = rot.sn * ex; rot.wy = rot.sn * ey;
            rot.zx = rot.c * ex; rot.zy = rot.c * ey;
            for (int k = t64; k < L; k += 64) {
              C u = ra[k], w = rb[k];
              rot_apply(rot, u, w);
              ra[k] = u;
              rb[k] = w;
            }
            if (t64 < BJ_ROWS) {
              C u = W[ia][t64], w = W[ib][t64];
              rot_apply(rot, u, w);
              W[ia][t64] = u;
              W[ib][t64] = w;
            }
            if (t64 == 0) atomicAdd(&s_nrot, 1);
          }
        }
        __syncthreads();
      }
      if (s_nrot > 0) {
        for (int e = threadIdx.x; e < BJ_ROWS * L; e += blockDim.x) {
          const int rr = e / L, k = e - rr * L;
          const int gr = s_grow[rr];
          if (gr >= 0) tk.X[(size_t)gr * L + k] = bj_rows[rr * L + k];
        }
        // Q rows of the block pair <- W Q (columns split over the threads)
        for (int cidx = threadIdx.x; tk.Q && cidx < v; cidx += blockDim.x) {
          C qv[BJ_ROWS];
#pragma unroll
          for (int rr = 0; rr < BJ_ROWS; ++rr)
            qv[rr] = s_grow[rr] >= 0 ? __ldcg(tk.Q + (size_t)s_grow[rr] * v + cidx) : mk2(R(0), R(0));
#pragma unroll
          for (int ii = 0; ii < BJ_ROWS; ++ii) {
            if (s_grow[ii] < 0) continue;
            C acc = mk2(R(0), R(0));
#pragma unroll
            for (int rr = 0; rr < BJ_ROWS; ++rr) {
              const C w = W[ii][rr];
              acc.x = fma(w.x, qv[rr].x, fma(-w.y, qv[rr].y, acc.x));
              acc.y = fma(w.x, qv[rr].y, fma(w.y, qv[rr].x, acc.y));
            }
            tk.Q[(size_t)s_grow[ii] * v + cidx] = acc;
          }
        }
        if (threadIdx.x == 0) {
          const int nb = (v + BJ_BLOCK - 1) / BJ_BLOCK;
          if (A < nb) tk.stamp[A] = (int)g;
          if (B < nb) tk.stamp[B] = (int)g;
          atomicAdd(&st[t].rot[s % 3], (unsigned int)s_nrot);
        }
      }
      __syncthreads();
    }
    if (!grid_barrier(bar, err, gridDim.x)) return;
  }
}

// FP32 preconditioning set-up: X32 = float(X) row by row (the FP64 task's layout), Q32 = I.
__global__ void precond_init_kernel(const JacobiTask* __restrict__ t64, const JacobiTask32* __restrict__ t32) {
  const JacobiTask a = t64[blockIdx.y];
  const JacobiTask32 b = t32[blockIdx.y];
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < (long long)a.m * a.n) {
    const double2 v = a.X[e];
    b.X[e] = make_float2((float)v.x, (float)v.y);
  }
  if (e < (long long)a.m * a.m) {
    const int i = (int)(e / a.m), j = (int)(e % a.m);
    b.Q[e] = make_float2(i == j ? 1.0f : 0.0f, 0.0f);
  }
}

// FP64 <-> FP32 copies of the rows of a task's matrix (m x n, same layout in both tasks).
__global__ void narrow_rows_kernel(const JacobiTask* __restrict__ t64, const JacobiTask32* __restrict__ t32) {
  const JacobiTask a = t64[blockIdx.y];
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)a.m * a.n) return;
  const double2 v = a.X[e];
  t32[blockIdx.y].X[e] = make_float2((float)v.x, (float)v.y);
}

__global__ void widen_rows_kernel(const JacobiTask32* __restrict__ t32, const JacobiTask* __restrict__ t64) {
  const JacobiTask32 b = t32[blockIdx.y];
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)b.m * b.n) return;
  const float2 v = b.X[e];
  t64[blockIdx.y].X[e] = make_double2((double)v.x, (double)v.y);
}

// Squared Frobenius norm of each task's FP64 matrix (fixed-order block reduction).
__global__ void __launch_bounds__(1024) fro2_kernel(const JacobiTask* __restrict__ t64, double* out) {
  __shared__ double red[32];
  const JacobiTask a = t64[blockIdx.x];
  const long long cells = (long long)a.m * a.n;
  double acc = 0.0;
  for (long long e = threadIdx.x; e < cells; e += blockDim.x) acc = fma(a.X[e].x, a.X[e].x, fma(a.X[e].y, a.X[e].y, acc));
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) out[blockIdx.x] = v;
  }
}

__global__ void widen_q_kernel(const JacobiTask32* __restrict__ t32, double2* const* __restrict__ q64) {
  const JacobiTask32 b = t32[blockIdx.y];
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)b.m * b.m) return;
  const float2 v = b.Q[e];
  q64[blockIdx.y][e] = make_double2((double)v.x, (double)v.y);
}

// ---------------------------------------------------------------------------------------
// Truncation: row norms of the orthogonalised matrix are the singular values.  Sort them
// descending (bitonic, ties by row index), keep s_k > eps * s_0 (at least 1, at most
// chi_max) and renormalise the kept values to unit 2-norm.
constexpr int TR_MAX = 4096;

// One CTA truncates the m rows of X (length n) of one task; outputs at idx_out, lam_out,
// sraw_out (count entries each) and *out.
__device__ void truncate_body(const double2* X, int m, int n, double eps, int chi_max, int32_t* idx_out,
                              double* lam_out, double* sraw_out, TruncOut* out) {
  extern __shared__ unsigned char smem_raw[];
  double* sv = reinterpret_cast<double*>(smem_raw);
  int* id = reinterpret_cast<int*>(sv + TR_MAX);
  __shared__ double red[32];
  __shared__ int s_count;
  struct { const double2* X; int m, n; } t{X, m, n};
  int P = 1;
  while (P < t.m) P <<= 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < P; i += nw) {
    double acc = 0.0;
    if (i < t.m) {
      const double2* row = t.X + (size_t)i * t.n;
      for (int k = lane; k < t.n; k += 32) acc = fma(row[k].x, row[k].x, fma(row[k].y, row[k].y, acc));
      acc = warp_sum(acc);
    }
    if (lane == 0) { sv[i] = i < t.m ? sqrt(acc) : -1.0; id[i] = i; }
  }
  __syncthreads();
  // bitonic sort, descending by value, ascending by index on ties
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const double a = sv[i], b = sv[ixj];
          const int ia = id[i], ib = id[ixj];
          const bool a_first = (a > b) || (a == b && ia < ib);
          const bool up = (i & k) == 0;
          if (up ? !a_first : a_first) { sv[i] = b; sv[ixj] = a; id[i] = ib; id[ixj] = ia; }
        }
      }
      __syncthreads();
    }
  }
  const double s0 = sv[0];
  const double thr = eps * s0;
  if (threadIdx.x == 0) s_count = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < t.m; i += blockDim.x) {
    const bool keep = sv[i] > thr;
    const bool next_keep = (i + 1 < t.m) && (sv[i + 1] > thr);
    if (keep && !next_keep) s_count = i + 1;
  }
  __syncthreads();
  int count = s_count;
  if (count < 1) count = 1;
  if (count > chi_max) count = chi_max;
  // renormalisation: fixed-order tree reduction of the kept squares
  double part = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) part = fma(sv[i], sv[i], part);
  part = warp_sum(part);
  if (lane == 0) red[warp] = part;
  __syncthreads();
  if (warp == 0) {
    double v = lane < nw ? red[lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  const double nrm = sqrt(red[0]);
  __syncthreads();
  double all = 0.0;
  for (int i = threadIdx.x; i < t.m; i += blockDim.x) all = fma(sv[i], sv[i], all);
  all = warp_sum(all);
  if (lane == 0) red[warp] = all;
  __syncthreads();
  if (warp == 0) {
    double v = lane < nw ? red[lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0) red[1] = v;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < count; k += blockDim.x) {
    idx_out[k] = id[k];
    lam_out[k] = sv[k] / nrm;
    sraw_out[k] = sv[k];
  }
  if (threadIdx.x == 0) {
    TruncOut o;
    o.count = count;
    o.m = t.m;
    o.s0 = s0;
    o.nrm = nrm;
    o.s_first_dropped = count < t.m ? sv[count] : 0.0;
    o.total2 = red[1];
    o.s_last_kept = sv[count - 1];
    *out = o;
  }
}

__global__ void __launch_bounds__(1024) truncate_kernel(const JacobiTask* __restrict__ tasks, double eps,
                                                        int chi_max, int32_t* idx_out, int idx_stride,
                                                        double* lam_out, double* sraw_out, int lam_stride,
                                                        TruncOut* out) {
  const JacobiTask t = tasks[blockIdx.x];
  truncate_body(t.X, t.m, t.n, eps, chi_max, idx_out + (size_t)blockIdx.x * idx_stride,
                lam_out + (size_t)blockIdx.x * lam_stride, sraw_out + (size_t)blockIdx.x * lam_stride,
                out + blockIdx.x);
}

__global__ void __launch_bounds__(1024) truncate_tasks_kernel(const TruncTask* __restrict__ tasks) {
  const TruncTask t = tasks[blockIdx.x];
  truncate_body(t.X, t.m, t.n, t.eps, t.chi_max, t.idx, t.lam, t.sraw, t.out);
}

__global__ void __launch_bounds__(256) split_rows_kernel(const SplitRowsDesc* __restrict__ descs) {
  const SplitRowsDesc d = descs[blockIdx.y];
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)d.count * d.n) return;
  const int k = (int)(e / d.n), c = (int)(e % d.n);
  if (d.Q) {
    const double2 q = d.Q[(size_t)d.idx[k] * d.n + c];
    d.dst[e] = make_double2(q.x, -q.y);
  } else {
    const double inv = 1.0 / d.sraw[k];
    const double2 v = d.X[(size_t)d.idx[k] * d.n + c];
    d.dst[e] = make_double2(v.x * inv, v.y * inv);
  }
}

__global__ void init_accumulators_kernel(const JacobiTask* __restrict__ tasks) {
  const JacobiTask t = tasks[blockIdx.y];
  if (!t.Q) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)t.m * t.m) return;
  const int i = (int)(e / t.m), j = (int)(e % t.m);
  t.Q[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
}

// stamp[k] = -1 for every row of every task (before a Jacobi launch).
template <typename Task>
__global__ void init_stamps_kernel(const Task* __restrict__ tasks) {
  const Task t = tasks[blockIdx.y];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < t.m; e += gridDim.x * blockDim.x) t.stamp[e] = -1;
}

__global__ void one_site_kernel(double2* B, int chi_l, int chi_r, const double2* g, int side) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)chi_l * 2 * chi_r) return;
  const int r = (int)(e % chi_r);
  const int x = (int)((e / chi_r) % 2);      // the leg that is not acted on
  const int l = (int)(e / (2LL * chi_r));
  double2 g00 = g[0], g01 = g[1], g10 = g[2], g11 = g[3];
  if (side == 0) {   // out-legs: new[o] = sum_o' g[o][o'] B[(o', i)]
    double2* p0 = B + ((size_t)(4 * l + 0 + x)) * chi_r + r;      // o = 0, i = x
    double2* p1 = B + ((size_t)(4 * l + 2 + x)) * chi_r + r;      // o = 1, i = x
    const double2 b0 = *p0, b1 = *p1;
    *p0 = cfma(g01, b1, cmul(g00, b0));
    *p1 = cfma(g11, b1, cmul(g10, b0));
  } else {           // in-legs: new[i] = sum_i' B[(o, i')] h[i'][i]
    double2* p0 = B + ((size_t)(4 * l + 2 * x + 0)) * chi_r + r;
    double2* p1 = B + ((size_t)(4 * l + 2 * x + 1)) * chi_r + r;
    const double2 b0 = *p0, b1 = *p1;
    *p0 = cfma(b1, g10, cmul(b0, g00));
    *p1 = cfma(b1, g11, cmul(b0, g01));
  }
}

// Peak search expansion: both children of one prefix vector, and their marginals.
__global__ void __launch_bounds__(256) expand_kernel(const double2* v, const double2* Bj, int chi_l,
                                                    int chi_r, const double2* E, double2* w0,
                                                    double2* w1, double* marg) {
  __shared__ double red[2][8];
  for (int r = threadIdx.x; r < chi_r; r += blockDim.x) {
    double2 a0 = make_double2(0.0, 0.0), a1 = make_double2(0.0, 0.0);
    for (int l = 0; l < chi_l; ++l) {
      const double2 vl = v[l];
      a0 = cfma(vl, Bj[(size_t)(4 * l + 0) * chi_r + r], a0);
      a1 = cfma(vl, Bj[(size_t)(4 * l + 2) * chi_r + r], a1);
    }
    w0[r] = a0;
    w1[r] = a1;
  }
  __syncthreads();
  double m0 = 0.0, m1 = 0.0;
  for (int c = threadIdx.x; c < chi_r; c += blockDim.x) {
    double2 y0 = make_double2(0.0, 0.0), y1 = make_double2(0.0, 0.0);
    for (int r = 0; r < chi_r; ++r) {
      const double2 e = E[(size_t)r * chi_r + c];
      y0 = cfma(w0[r], e, y0);
      y1 = cfma(w1[r], e, y1);
    }
    const double2 c0 = w0[c], c1 = w1[c];
    m0 += y0.x * c0.x + y0.y * c0.y;
    m1 += y1.x * c1.x + y1.y * c1.y;
  }
  m0 = warp_sum(m0);
  m1 = warp_sum(m1);
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = m0; red[1][threadIdx.x >> 5] = m1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { s0 += red[0][w]; s1 += red[1][w]; }
    marg[0] = s0;
    marg[1] = s1;
  }
}

__global__ void quadform_rows_kernel(const double2* W, const double2* Y, int rows, int cols, int ld,
                                     double* out) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  double acc = 0.0;
  for (int c = lane; c < cols; c += 32) {
    const double2 y = Y[(size_t)row * ld + c], w = W[(size_t)row * ld + c];
    acc += y.x * w.x + y.y * w.y;
  }
  acc = warp_sum(acc);
  if (lane == 0) out[row] = acc;
}

__global__ void sample_pick_kernel(const double2* W0, const double2* W1, const double* m0,
                                   const double* m1, const double* u, int S, int chi, int site,
                                   int n_sites, double2* Vnext, uint8_t* site_bits) {
  const int s = blockIdx.x;
  if (s >= S) return;
  const double p0 = m0[s], p1 = m1[s];
  const double P0 = p0 / (p0 + p1);
  const int bit = u[(size_t)s * n_sites + site] >= P0 ? 1 : 0;
  const double inv = 1.0 / sqrt(bit ? p1 : p0);
  const double2* W = bit ? W1 : W0;
  for (int c = threadIdx.x; c < chi; c += blockDim.x) {
    const double2 w = W[(size_t)s * chi + c];
    Vnext[(size_t)s * chi + c] = make_double2(w.x * inv, w.y * inv);
  }
  if (threadIdx.x == 0) site_bits[(size_t)s * n_sites + site] = (uint8_t)bit;
}

__global__ void amp_pick_kernel(const double2* W0, const double2* W1, const uint8_t* site_bits, int K,
                                int chi, int site, int n_sites, double2* Vnext) {
  const int k = blockIdx.x;
  if (k >= K) return;
  const double2* W = site_bits[(size_t)k * n_sites + site] ? W1 : W0;
  for (int c = threadIdx.x; c < chi; c += blockDim.x) Vnext[(size_t)k * chi + c] = W[(size_t)k * chi + c];
}

// Recanonicalisation (Algorithm 1, "compress M to canonical form"): Z = X or X^T, X row-major
// rows x cols.
__global__ void recanon_load_kernel(const double2* __restrict__ X, int rows, int cols, int transpose,
                                    double2* __restrict__ Z) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  const int r = (int)(e / cols), c = (int)(e % cols);
  Z[transpose ? (size_t)c * rows + r : (size_t)e] = X[e];
}

// One factor of a factorised Z (see recanon_emit in pc_internal.h).
__global__ void recanon_emit_kernel(const double2* __restrict__ Z, const double2* __restrict__ Q, int ld,
                                    const int32_t* __restrict__ idx, const double* __restrict__ sraw, int count,
                                    int n_out, int use_q, int scale, int transpose_out, double2* __restrict__ out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)count * n_out) return;
  const int k = (int)(e / n_out), a = (int)(e % n_out);
  const int row = idx[k];
  double2 v;
  if (use_q) {
    const double2 q = Q[(size_t)row * ld + a];
    v = make_double2(q.x, -q.y);
  } else {
    v = Z[(size_t)row * ld + a];
  }
  if (scale == 1) { const double inv = 1.0 / sraw[k]; v.x *= inv; v.y *= inv; }
  else if (scale == 2) { const double s = sraw[k]; v.x *= s; v.y *= s; }
  out[transpose_out ? (size_t)a * count + k : (size_t)k * n_out + a] = v;
}

// Deflation floor (see DeflateTask): one CTA per task.
__global__ void __launch_bounds__(1024) deflate_floor_kernel(const DeflateTask* __restrict__ tasks) {
  extern __shared__ unsigned char smem_raw[];
  double* sv = reinterpret_cast<double*>(smem_raw);
  const DeflateTask t = tasks[blockIdx.x];
  int P = 1;
  while (P < t.m) P <<= 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < P; i += nw) {
    double acc = 0.0;
    if (i < t.m) {
      const float2* row = t.X32 + (size_t)i * t.n;
      for (int k = lane; k < t.n; k += 32) {
        const double x = row[k].x, y = row[k].y;
        acc = fma(x, x, fma(y, y, acc));
      }
      acc = warp_sum(acc);
    }
    if (lane == 0) sv[i] = i < t.m ? sqrt(acc) : -1.0;
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const double a = sv[i], b = sv[ixj];
          const bool up = (i & k) == 0;
          if (up ? (a < b) : (a > b)) { sv[i] = b; sv[ixj] = a; }
        }
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    double d2 = 0.0, sc = 0.0;
    const double fro = sqrt(*t.fro2);
    if (t.m > t.chi_max && t.chi_max >= 1) {
      const double c = sv[t.chi_max - 1];
      if (c >= 1e-4 * fro) {
        sc = c;
        const double d = c / (8.0 * t.m);
        d2 = d * d;
      }
    }
    *t.dead2_out = d2;
    *t.sc_out = sc;
  }
}

// FMA-chain throughput probe: every thread runs 8 independent chains of `iters` fused
// multiply-adds (2 flops each); the result is written so the work cannot be removed.
template <typename R>
__global__ void __launch_bounds__(256) fma_probe_kernel(R a, R b, int iters, R* out) {
  R x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (R)(threadIdx.x + k) * (R)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  R acc = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) acc += x[k];
  if (acc == (R)12345.678) out[0] = acc;
}

__global__ void fill_ones_kernel(double2* v, int rows) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < rows) v[i] = make_double2(1.0, 0.0);
}

}  // namespace

// ---------------------------------------------------------------------------------------
cudaError_t launch_gemm(const GemmDesc* d_desc, int batch, int max_m, int max_n, cudaStream_t stream) {
  if (batch <= 0 || max_m <= 0 || max_n <= 0) return cudaSuccess;
  dim3 grid((max_n + GBN - 1) / GBN, (max_m + GBM - 1) / GBM, batch);
  gemm_kernel<<<grid, 256, 0, stream>>>(d_desc);
  return cudaGetLastError();
}

cudaError_t launch_gate_apply(const UpdateTask* d_tasks, int ntasks, int max_chi_l, int max_chi_r,
                              cudaStream_t stream) {
  if (ntasks <= 0) return cudaSuccess;
  const long long cells = (long long)max_chi_l * max_chi_r;
  dim3 grid((unsigned)((cells + 255) / 256), ntasks);
  gate_apply_kernel<<<grid, 256, 0, stream>>>(d_tasks);
  return cudaGetLastError();
}

cudaError_t launch_init_stamps(const JacobiTask* d_tasks, int ntasks, int max_m, cudaStream_t stream) {
  if (ntasks <= 0) return cudaSuccess;
  init_stamps_kernel<JacobiTask><<<dim3((max_m + 255) / 256, ntasks), 256, 0, stream>>>(d_tasks);
  return cudaGetLastError();
}

cudaError_t launch_init_stamps32(const JacobiTask32* d_tasks, int ntasks, int max_m, cudaStream_t stream) {
  if (ntasks <= 0) return cudaSuccess;
  init_stamps_kernel<JacobiTask32><<<dim3((max_m + 255) / 256, ntasks), 256, 0, stream>>>(d_tasks);
  return cudaGetLastError();
}

cudaError_t launch_init_accumulators(const JacobiTask* d_tasks, int ntasks, int max_m, cudaStream_t stream) {
  if (ntasks <= 0) return cudaSuccess;
  const long long cells = (long long)max_m * max_m;
  dim3 grid((unsigned)((cells + 255) / 256), ntasks);
  init_accumulators_kernel<<<grid, 256, 0, stream>>>(d_tasks);
  return cudaGetLastError();
}

template <typename R, int G>
cudaError_t launch_jacobi_g(const typename JacTraits<R>::Task* d_tasks, int ntasks, JacobiStatus* d_status,
                            int max_sweeps, unsigned int* d_bar, int* d_err, int sm_count, cudaStream_t stream) {
  constexpr int dyn = jac_dyn_smem<R, G>();
  static int blocks_per_sm = -1;
  if (blocks_per_sm < 0) {
    if (dyn > 0) {
      cudaError_t e = cudaFuncSetAttribute(jacobi_kernel<R, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, jacobi_kernel<R, G>, JAC_THREADS, dyn);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm > 1) blocks_per_sm = 1;
    if (blocks_per_sm < 1) return cudaErrorLaunchOutOfResources;
  }
  const int grid = sm_count * blocks_per_sm;
  void* args[] = {(void*)&d_tasks, (void*)&ntasks, (void*)&d_status, (void*)&max_sweeps, (void*)&d_bar,
                  (void*)&d_err};
  return cudaLaunchCooperativeKernel((const void*)jacobi_kernel<R, G>, dim3(grid), dim3(JAC_THREADS), args, dyn,
                                     stream);
}

// Group width table of the FP64 row-pair sweeps, filled by the autotuner (pc_autotune /
// pc_load_tuning): entry [len bucket][pairs bucket] = warps per pair (1, 2, 4), 0 = use the
// heuristic below.  len bucket = ceil(log2(longest row)), pairs bucket = floor(log2(pairs per
// round)), both clamped to the table.
int g_jac_tuning[JAC_TUNE_LEN][JAC_TUNE_PAIRS] = {};

int tuned_group_width(int max_len, int total_pairs) {
  int bl = 0, bp = 0;
  while ((1 << bl) < max_len && bl < JAC_TUNE_LEN - 1) ++bl;
  while ((2 << bp) <= total_pairs && bp < JAC_TUNE_PAIRS - 1) ++bp;
  return g_jac_tuning[bl][bp];
}

// Group width: at least enough threads to hold the longest row in registers; wider (up to
// four warps per pair) when a round has fewer pairs than the grid has warps; a tuned width,
// when the table has one for the launch's shape, overrides the FP64 choice.
template <typename R>
cudaError_t launch_jacobi_t(const typename JacTraits<R>::Task* d_tasks, int ntasks, JacobiStatus* d_status,
                            int max_sweeps, unsigned int* d_bar, int* d_err, int sm_count, int max_len,
                            int total_pairs, cudaStream_t stream, int force_g = 0) {
  if (ntasks <= 0) return cudaSuccess;
  if (ntasks > JAC_MAX_TASKS) return cudaErrorInvalidValue;
  const int warps = sm_count * (JAC_THREADS / 32);
  int g = max_len <= 32 * JAC_E ? 1 : (max_len <= 64 * JAC_E ? 2 : 4);
  while (g < 4 && total_pairs > 0 && (long long)total_pairs * 2 * g <= warps) g *= 2;
  if (force_g == 1 || force_g == 2 || force_g == 4) g = force_g;
  if (g == 1) return launch_jacobi_g<R, 1>(d_tasks, ntasks, d_status, max_sweeps, d_bar, d_err, sm_count, stream);
  if (g == 2) return launch_jacobi_g<R, 2>(d_tasks, ntasks, d_status, max_sweeps, d_bar, d_err, sm_count, stream);
  return launch_jacobi_g<R, 4>(d_tasks, ntasks, d_status, max_sweeps, d_bar, d_err, sm_count, stream);
}

cudaError_t launch_jacobi(const JacobiTask* d_tasks, int ntasks, JacobiStatus* d_status, int max_sweeps,
                          unsigned int* d_bar, int* d_err, int sm_count, int max_len, int total_pairs,
                          cudaStream_t stream, int force_g) {
  if (force_g == 0) force_g = tuned_group_width(max_len, total_pairs);
  return launch_jacobi_t<double>(d_tasks, ntasks, d_status, max_sweeps, d_bar, d_err, sm_count, max_len,
                                 total_pairs, stream, force_g);
}

void set_jacobi_tuning(int bl, int bp, int g) {
  if (bl >= 0 && bl < JAC_TUNE_LEN && bp >= 0 && bp < JAC_TUNE_PAIRS) g_jac_tuning[bl][bp] = g;
}

int jacobi_tuning(int bl, int bp) {
  return (bl >= 0 && bl < JAC_TUNE_LEN && bp >= 0 && bp < JAC_TUNE_PAIRS) ? g_jac_tuning[bl][bp] : 0;
}

cudaError_t launch_jacobi32(const JacobiTask32* d_tasks, int ntasks, JacobiStatus* d_status, int max_sweeps,
                            unsigned int* d_bar, int* d_err, int sm_count, int max_len, int total_pairs,
                            cudaStream_t stream) {
  return launch_jacobi_t<float>(d_tasks, ntasks, d_status, max_sweeps, d_bar, d_err, sm_count, max_len,
                                total_pairs, stream);
}

template <typename R>
cudaError_t launch_bjac(const typename JacTraits<R>::Task* d_tasks, int ntasks, JacobiStatus* d_status,
                        int max_sweeps, unsigned int* d_bar, int* d_err, int sm_count, int max_len,
                        cudaStream_t stream) {
  using C = typename JacTraits<R>::C;
  constexpr int rows = 2 * BjBlock<R>::value;
  if (ntasks <= 0) return cudaSuccess;
  if (ntasks > JAC_MAX_TASKS || max_len > BJ_MAX_LEN) return cudaErrorInvalidValue;
  const int smem = rows * max_len * (int)sizeof(C);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(bjac_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         rows * BJ_MAX_LEN * (int)sizeof(C));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bjac_kernel<R>, BJ_THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  void* args[] = {(void*)&d_tasks, (void*)&ntasks, (void*)&d_status, (void*)&max_sweeps, (void*)&d_bar, (void*)&d_err};
  return cudaLaunchCooperativeKernel((const void*)bjac_kernel<R>, dim3(sm_count), dim3(BJ_THREADS), args, smem, stream);
}

cudaError_t launch_jacobi32_blocked(const JacobiTask32* d_tasks, int ntasks, JacobiStatus* d_status, int max_sweeps,
                                    unsigned int* d_bar, int* d_err, int sm_count, int max_len, cudaStream_t stream) {
  return launch_bjac<float>(d_tasks, ntasks, d_status, max_sweeps, d_bar, d_err, sm_count, max_len, stream);
}

cudaError_t launch_precond_init(const JacobiTask* d_t64, const JacobiTask32* d_t32, int ntasks, int max_m, int max_n,
                                cudaStream_t stream) {
  if (ntasks <= 0) return cudaSuccess;
  const long long cells = (long long)max_m * (max_n > max_m ? max_n : max_m);
  dim3 grid((unsigned)((cells + 255) / 256), ntasks);
  precond_init_kernel<<<grid, 256, 0, stream>>>(d_t64, d_t32);
  return cudaGetLastError();
}

cudaError_t launch_narrow_rows(const JacobiTask* d_t64, const JacobiTask32* d_t32, int ntasks, int max_m, int max_n,
                               cudaStream_t stream) {
  if (ntasks <= 0) return cudaSuccess;
  const long long cells = (long long)max_m * max_n;
  dim3 grid((unsigned)((cells + 255) / 256), ntasks);
  narrow_rows_kernel<<<grid, 256, 0, stream>>>(d_t64, d_t32);
  return cudaGetLastError();
}

cudaError_t launch_widen_rows(const JacobiTask32* d_t32, const JacobiTask* d_t64, int ntasks, int max_m, int max_n,
                              cudaStream_t stream) {
  if (ntasks <= 0) return cudaSuccess;
  const long long cells = (long long)max_m * max_n;
  dim3 grid((unsigned)((cells + 255) / 256), ntasks);
  widen_rows_kernel<<<grid, 256, 0, stream>>>(d_t32, d_t64);
  return cudaGetLastError();
}

cudaError_t launch_fro2(const JacobiTask* d_t64, int ntasks, double* d_out, cudaStream_t stream) {
  if (ntasks <= 0) return cudaSuccess;
  fro2_kernel<<<ntasks, 1024, 0, stream>>>(d_t64, d_out);
  return cudaGetLastError();
}

cudaError_t launch_widen_q(const JacobiTask32* d_t32, double2* const* d_q64, int ntasks, int max_m,
                           cudaStream_t stream) {
  if (ntasks <= 0) return cudaSuccess;
  const long long cells = (long long)max_m * max_m;
  dim3 grid((unsigned)((cells + 255) / 256), ntasks);
  widen_q_kernel<<<grid, 256, 0, stream>>>(d_t32, d_q64);
  return cudaGetLastError();
}

cudaError_t launch_truncate(const JacobiTask* d_tasks, int ntasks, double eps, int chi_max, int32_t* d_idx,
                            int idx_stride, double* d_lam, double* d_sraw, int lam_stride, TruncOut* d_out,
                            cudaStream_t stream) {
  if (ntasks <= 0) return cudaSuccess;
  const size_t smem = TR_MAX * (sizeof(double) + sizeof(int));
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(truncate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  truncate_kernel<<<ntasks, 1024, smem, stream>>>(d_tasks, eps, chi_max, d_idx, idx_stride, d_lam, d_sraw,
                                                  lam_stride, d_out);
  return cudaGetLastError();
}

cudaError_t launch_truncate_tasks(const TruncTask* d_tasks, int ntasks, cudaStream_t stream) {
  if (ntasks <= 0) return cudaSuccess;
  const size_t smem = TR_MAX * (sizeof(double) + sizeof(int));
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(truncate_tasks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  truncate_tasks_kernel<<<ntasks, 1024, smem, stream>>>(d_tasks);
  return cudaGetLastError();
}

cudaError_t launch_split_rows(const SplitRowsDesc* d_desc, int ntasks, int max_count, int max_n,
                              cudaStream_t stream) {
  if (ntasks <= 0) return cudaSuccess;
  const long long cells = (long long)max_count * max_n;
  dim3 grid((unsigned)((cells + 255) / 256), ntasks);
  split_rows_kernel<<<grid, 256, 0, stream>>>(d_desc);
  return cudaGetLastError();
}

cudaError_t launch_deflate_floor(const DeflateTask* d_tasks, int ntasks, cudaStream_t stream) {
  if (ntasks <= 0) return cudaSuccess;
  const size_t smem = TR_MAX * sizeof(double);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(deflate_floor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  deflate_floor_kernel<<<ntasks, 1024, smem, stream>>>(d_tasks);
  return cudaGetLastError();
}

cudaError_t launch_recanon_load(const double2* X, int rows, int cols, int transpose, double2* Z, cudaStream_t stream) {
  const long long cells = (long long)rows * cols;
  if (cells <= 0) return cudaSuccess;
  recanon_load_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, stream>>>(X, rows, cols, transpose, Z);
  return cudaGetLastError();
}

cudaError_t launch_recanon_emit(const double2* Z, const double2* Q, int ld, const int32_t* idx, const double* sraw,
                                int count, int n_out, int use_q, int scale, int transpose_out, double2* out,
                                cudaStream_t stream) {
  const long long cells = (long long)count * n_out;
  if (cells <= 0) return cudaSuccess;
  recanon_emit_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, stream>>>(Z, Q, ld, idx, sraw, count, n_out, use_q,
                                                                           scale, transpose_out, out);
  return cudaGetLastError();
}

cudaError_t launch_one_site(double2* B, int chi_l, int chi_r, const double2* g2_dev, int side,
                            cudaStream_t stream) {
  const long long cells = (long long)chi_l * 2 * chi_r;
  one_site_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, stream>>>(B, chi_l, chi_r, g2_dev, side);
  return cudaGetLastError();
}

cudaError_t launch_expand(const double2* v, const double2* Bj, int chi_l, int chi_r, const double2* E,
                          double2* w0, double2* w1, double* marg, cudaStream_t stream) {
  expand_kernel<<<1, 256, 0, stream>>>(v, Bj, chi_l, chi_r, E, w0, w1, marg);
  return cudaGetLastError();
}

cudaError_t launch_quadform_rows(const double2* W, const double2* Y, int rows, int cols, int ld, double* out,
                                 cudaStream_t stream) {
  quadform_rows_kernel<<<(rows + 7) / 8, 256, 0, stream>>>(W, Y, rows, cols, ld, out);
  return cudaGetLastError();
}

cudaError_t launch_sample_pick(const double2* W0, const double2* W1, const double* m0, const double* m1,
                               const double* u, int S, int chi, int site, int n_sites, double2* Vnext,
                               uint8_t* site_bits, cudaStream_t stream) {
  sample_pick_kernel<<<S, 128, 0, stream>>>(W0, W1, m0, m1, u, S, chi, site, n_sites, Vnext, site_bits);
  return cudaGetLastError();
}

cudaError_t launch_amp_pick(const double2* W0, const double2* W1, const uint8_t* site_bits, int K, int chi,
                            int site, int n_sites, double2* Vnext, cudaStream_t stream) {
  amp_pick_kernel<<<K, 128, 0, stream>>>(W0, W1, site_bits, K, chi, site, n_sites, Vnext);
  return cudaGetLastError();
}

cudaError_t launch_fma_probe(int fp64, int blocks, int iters, void* out, cudaStream_t stream) {
  if (fp64)
    fma_probe_kernel<double><<<blocks, 256, 0, stream>>>(0.999999, 1e-9, iters, (double*)out);
  else
    fma_probe_kernel<float><<<blocks, 256, 0, stream>>>(0.999999f, 1e-9f, iters, (float*)out);
  return cudaGetLastError();
}

cudaError_t launch_fill_ones(double2* v, int rows, cudaStream_t stream) {
  fill_ones_kernel<<<(rows + 255) / 256, 256, 0, stream>>>(v, rows);
  return cudaGetLastError();
}

}  // namespace pc
