// Mixed-precision merge on the 5th-generation tensor cores (sm_103a, tcgen05 + TMA).
//
// The two-site merge of Sec. II.B.1, X = B_j . B_j+1 (a complex GEMM of (4 chi_l) x chi_m by
// chi_m x (4 chi_r)), runs in complex FP32 arithmetic as 3xTF32 on the tensor cores with FP32
// accumulation in tensor memory; inputs and output stay FP64 in global memory.
//
// Complex -> real.  With A' the complex A read as a real M x 2K matrix (re, im interleaved,
// i.e. A's own memory) and B'' the 2N x 2K real matrix
//     B''[2n + 0][2k + 0] =  re B[k][n]     B''[2n + 0][2k + 1] = -im B[k][n]
//     B''[2n + 1][2k + 0] =  im B[k][n]     B''[2n + 1][2k + 1] =  re B[k][n]
// the real product A' B''^T is C with (re, im) interleaved.  Both operands are then K-major,
// the native operand order of tcgen05.mma.
//
// 3xTF32.  Every operand value x is split x = hi + lo with hi = tf32(x), lo = tf32(x - hi);
// C = A_hi B_hi + A_hi B_lo + A_lo B_hi, three MMAs per K step into one accumulator.  The
// dropped lo*lo term and the TF32 rounding of lo leave a relative error of about 2^-21 per
// product, summed in FP32.
//
// Kernel structure (one 128 x 256 output tile per CTA, 192 threads):
//   warp 4  (one thread)  TMA producer: 128B-swizzled tiles of A_hi, A_lo, B_hi, B_lo into a
//                         two-stage shared-memory ring, completion on "full" mbarriers
//   warp 5  (one thread)  MMA issuer: tcgen05.mma.kind::tf32 M=128 N=256 K=8, 12 per stage;
//                         tcgen05.commit frees the stage ("empty") and finally signals "accum"
//   warps 0-3             epilogue: tcgen05.ld of the 128 lanes x 256 columns accumulator,
//                         FP32 -> FP64, stored to C
// Warp 5 also allocates and frees the 256 tensor-memory columns.  Every mbarrier wait is
// bounded; on a timeout the CTA records an error, waits (bounded) for its own copies and
// MMAs, frees its tensor memory and returns without storing.
#include "pc_internal.h"

#include <cuda.h>
#include <cstdint>
#include <mutex>

namespace pc {

namespace {

constexpr int TC_BM = 128;                                  // UMMA M (rows of A / C)
constexpr int TC_BN = 256;                                  // UMMA N (real columns of C)
constexpr int TC_BK = 32;                                   // FP32 elements per 128-byte row
constexpr int TC_STAGES = 2;
constexpr int TC_A_BYTES = TC_BM * TC_BK * 4;               // 16 KB
constexpr int TC_B_BYTES = TC_BN * TC_BK * 4;               // 32 KB
constexpr int TC_STAGE_BYTES = 2 * (TC_A_BYTES + TC_B_BYTES);
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024 + 128;
constexpr int TC_THREADS = 192;
constexpr uint32_t TC_TMEM_COLS = 256;

// Instruction descriptor of tcgen05.mma.kind::tf32: FP32 accumulator (bits 4-5 = 1), A and
// B TF32 (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                              ((uint32_t)(TC_BM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase of the given parity to complete.  Gives up (returns false) after a
// bounded number of polls, or at once when another role of the CTA has given up.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* s_abort) {
  for (int i = 0; i < (1 << 22); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*s_abort) return false;
    if (i > 32) __nanosleep(128);
  }
  return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y,
                                            int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile stored with the 128-byte
// swizzle (rows of 128 bytes, 8-row groups 1024 bytes apart): start address >> 4 at bits
// 0-13, leading byte offset (unused for this layout) 16 B, stride byte offset 1024 B at bits
// 32-45, descriptor version 1 at bits 46-47, swizzle mode 2 (128 B) at bits 61-63.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)2u << 61;
  return d;
}

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(TC_IDESC), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// The load and its wait are one asm statement: tcgen05.ld writes its registers asynchronously,
// so no instruction may read them before tcgen05.wait::ld, and the compiler only orders
// register uses after the statement that defines them.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Operand preparation: the padded hi/lo planes of A' ([T][Mp][K2p]) and B'' ([T][N2p][K2p]),
// zero outside each task's own extent.
__global__ void __launch_bounds__(256) tc_split_kernel(const GemmDesc* __restrict__ descs, float* __restrict__ a_hi,
                                                        float* __restrict__ a_lo, float* __restrict__ b_hi,
                                                        float* __restrict__ b_lo, int Mp, int N2p, int K2p) {
  const GemmDesc d = descs[blockIdx.y];
  const long long a_cells = (long long)Mp * K2p, b_cells = (long long)N2p * K2p;
  const size_t a_base = (size_t)blockIdx.y * a_cells, b_base = (size_t)blockIdx.y * b_cells;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < a_cells + b_cells;
       e += (long long)gridDim.x * blockDim.x) {
    double x = 0.0;
    if (e < a_cells) {
      const int r = (int)(e / K2p), kk = (int)(e % K2p);
      if (r < d.M && kk < 2 * d.K) {
        const double2 v = d.A[(size_t)r * d.lda + (kk >> 1)];
        x = (kk & 1) ? v.y : v.x;
      }
      const float hi = tf32_round((float)x);
      a_hi[a_base + e] = hi;
      a_lo[a_base + e] = tf32_round((float)(x - (double)hi));
    } else {
      const long long f = e - a_cells;
      const int c = (int)(f / K2p), kk = (int)(f % K2p);
      if (c < 2 * d.N && kk < 2 * d.K) {
        const double2 b = d.B[(size_t)(kk >> 1) * d.ldb + (c >> 1)];
        const int part = c & 1, kp = kk & 1;
        x = part == 0 ? (kp == 0 ? b.x : -b.y) : (kp == 0 ? b.y : b.x);
      }
      const float hi = tf32_round((float)x);
      b_hi[b_base + f] = hi;
      b_lo[b_base + f] = tf32_round((float)(x - (double)hi));
    }
  }
}

struct TcMaps {
  CUtensorMap a_hi, a_lo, b_hi, b_lo;
};

__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_merge_kernel(const __grid_constant__ TcMaps maps, const GemmDesc* __restrict__ descs, int* err) {
  extern __shared__ uint8_t tc_smem_raw[];
  __shared__ uint64_t s_full[TC_STAGES], s_empty[TC_STAGES], s_accum;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;

  const GemmDesc d = descs[blockIdx.z];
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * TC_BN;   // n0: real column
  if (m0 >= d.M || n0 >= 2 * d.N) return;                      // uniform over the CTA
  const int nk = (2 * d.K + TC_BK - 1) / TC_BK;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // 1024-byte aligned stage ring: per stage A_hi | A_lo | B_hi | B_lo
  const uint32_t base = (smem_u32(tc_smem_raw) + 1023u) & ~1023u;
  auto a_tile = [&](int s, int lo) { return base + s * TC_STAGE_BYTES + lo * TC_A_BYTES; };
  auto b_tile = [&](int s, int lo) { return base + s * TC_STAGE_BYTES + 2 * TC_A_BYTES + lo * TC_B_BYTES; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(smem_u32(&s_full[s]), 1);
      mbar_init(smem_u32(&s_empty[s]), 1);
    }
    mbar_init(smem_u32(&s_accum), 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  volatile int* abort_flag = &s_abort;
  const int tz = blockIdx.z;

  if (warp == 4 && lane == 0) {
    // TMA producer
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % TC_STAGES;
      if (kb >= TC_STAGES && !mbar_wait(smem_u32(&s_empty[s]), ((kb / TC_STAGES) - 1) & 1, abort_flag)) {
        *abort_flag = 1;
        break;
      }
      const uint32_t fb = smem_u32(&s_full[s]);
      mbar_expect_tx(fb, TC_STAGE_BYTES);
      const int kx = kb * TC_BK;
      tma_load_3d(a_tile(s, 0), &maps.a_hi, fb, kx, m0, tz);
      tma_load_3d(a_tile(s, 1), &maps.a_lo, fb, kx, m0, tz);
      tma_load_3d(b_tile(s, 0), &maps.b_hi, fb, kx, n0, tz);
      tma_load_3d(b_tile(s, 1), &maps.b_lo, fb, kx, n0, tz);
      ++issued;
    }
    // every copy this thread issued has landed before the CTA may leave
    for (int kb = issued - TC_STAGES < 0 ? 0 : issued - TC_STAGES; kb < issued; ++kb) {
      const int s = kb % TC_STAGES;
      for (int i = 0; i < (1 << 22) && !mbar_try_wait(smem_u32(&s_full[s]), (kb / TC_STAGES) & 1); ++i)
        __nanosleep(128);
    }
  } else if (warp == 5 && lane == 0) {
    // MMA issuer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % TC_STAGES;
      if (!mbar_wait(smem_u32(&s_full[s]), (kb / TC_STAGES) & 1, abort_flag)) {
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int k = 0; k < TC_BK / 8; ++k) {
        const uint64_t ah = sdesc_sw128(a_tile(s, 0) + 32 * k), al = sdesc_sw128(a_tile(s, 1) + 32 * k);
        const uint64_t bh = sdesc_sw128(b_tile(s, 0) + 32 * k), bl = sdesc_sw128(b_tile(s, 1) + 32 * k);
        umma_tf32(tmem, ah, bh, (kb | k) != 0 ? 1u : 0u);
        umma_tf32(tmem, ah, bl, 1u);
        umma_tf32(tmem, al, bh, 1u);
      }
      umma_commit(smem_u32(&s_empty[s]));
    }
    // tracks completion of every MMA issued above
    umma_commit(smem_u32(&s_accum));
  } else if (warp < 4) {
    // epilogue: lane quarter `warp` of the accumulator = rows m0 + 32 warp + lane
    // one decision per warp: tcgen05.ld is warp-collective
    int go = 0;
    if (lane == 0) {
      go = mbar_wait(smem_u32(&s_accum), 0, abort_flag) ? 1 : 0;
      if (!go) *abort_flag = 1;
      else if (*abort_flag) go = 0;
    }
    go = __shfl_sync(0xffffffffu, go, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (go) {
      const int row = m0 + 32 * warp + lane;
      const uint32_t lane_addr = tmem + ((uint32_t)(32 * warp) << 16);
      for (int c = 0; c < TC_BN / 32; ++c) {
        float v[32];
        tmem_ld32(lane_addr + 32 * c, v);
        const int ncol = (n0 + 32 * c) >> 1;                 // complex column of v[0]
        if (row < d.M) {
          double2* out = d.C + (size_t)row * d.ldc + ncol;
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (ncol + j < d.N) out[j] = make_double2((double)v[2 * j], (double)v[2 * j + 1]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 5) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
  if (threadIdx.x == 0 && s_abort) atomicExch(err, 1);
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

bool encode_3d(CUtensorMap* map, float* base, int inner, int rows, int T, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)rows, (cuuint64_t)T};
  const cuuint64_t strides[2] = {(cuuint64_t)inner * 4, (cuuint64_t)inner * 4 * rows};
  const cuuint32_t box[3] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace

size_t tc_merge_workspace_bytes(int T, int max_m, int max_n, int max_k) {
  const size_t Mp = round_up(max_m, TC_BM), N2p = round_up(2 * max_n, TC_BN), K2p = round_up(2 * max_k, TC_BK);
  return (size_t)T * (Mp + N2p) * K2p * 2 * sizeof(float);
}

cudaError_t launch_tc_merge(const GemmDesc* d_desc, int T, int max_m, int max_n, int max_k, void* workspace,
                            size_t workspace_bytes, int* d_err, cudaStream_t stream) {
  if (T <= 0 || max_m <= 0 || max_n <= 0) return cudaSuccess;
  if (max_k <= 0) return cudaErrorInvalidValue;
  const int Mp = round_up(max_m, TC_BM), N2p = round_up(2 * max_n, TC_BN), K2p = round_up(2 * max_k, TC_BK);
  if (tc_merge_workspace_bytes(T, max_m, max_n, max_k) > workspace_bytes || T > 65535)
    return cudaErrorInvalidValue;
  float* a_hi = static_cast<float*>(workspace);
  float* a_lo = a_hi + (size_t)T * Mp * K2p;
  float* b_hi = a_lo + (size_t)T * Mp * K2p;
  float* b_lo = b_hi + (size_t)T * N2p * K2p;
  TcMaps maps;
  if (!encode_3d(&maps.a_hi, a_hi, K2p, Mp, T, TC_BM) || !encode_3d(&maps.a_lo, a_lo, K2p, Mp, T, TC_BM) ||
      !encode_3d(&maps.b_hi, b_hi, K2p, N2p, T, TC_BN) || !encode_3d(&maps.b_lo, b_lo, K2p, N2p, T, TC_BN))
    return cudaErrorInvalidValue;
  const long long cells = (long long)(Mp + N2p) * K2p;
  int split_blocks = (int)((cells + 255) / 256);
  if (split_blocks > 1024) split_blocks = 1024;
  tc_split_kernel<<<dim3(split_blocks, T), 256, 0, stream>>>(d_desc, a_hi, a_lo, b_hi, b_lo, Mp, N2p, K2p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  static bool attr = false;
  if (!attr) {
    e = cudaFuncSetAttribute(tc_merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid(N2p / TC_BN, Mp / TC_BM, T);
  tc_merge_kernel<<<grid, TC_THREADS, TC_SMEM, stream>>>(maps, d_desc, d_err);
  return cudaGetLastError();
}

}  // namespace pc
