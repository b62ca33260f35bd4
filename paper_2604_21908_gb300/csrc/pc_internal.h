// Internal declarations shared by the library's host code (pc_api.cpp) and its kernels
// (kernels.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace pc {

// One complex FP64 GEMM of a batch: C = alpha * A * op(B) + beta * D, where D is the
// matrix D (same leading dimension as C) or, when D is null, C itself.
//   A  : M x K row-major, leading dimension lda (complex elements)
//   B  : op == 0: K x N row-major (ldb);  op == 1: N x K row-major (ldb), used as its
//        conjugate transpose
//   C  : M x N row-major (ldc)
// Optional row scaling of A by a real vector (row_scale[i] multiplies row i of A).
struct GemmDesc {
  const double2* A;
  const double2* B;
  double2* C;
  const double* row_scale;
  int32_t M, N, K;
  int32_t lda, ldb, ldc;
  int32_t opB;          // 0: B, 1: B^H
  int32_t pad_;
  double alpha;
  double beta;          // 0: C is only written
  const double2* D;     // addend (nullptr: C)
};

// One two-site update of a wave (Sec. II.B.1): sites (j, j+1) with bond dims
// chi_l = chi_{j-1}, chi_m = chi_j, chi_r = chi_{j+1}.
struct UpdateTask {
  const double2* Bl;      // B_j  [chi_l][4][chi_m]
  const double2* Br;      // B_j+1 [chi_m][4][chi_r]
  const double* lam_l;    // lambda_{j-1} [chi_l], nullptr for the left boundary (1)
  const double2* op;      // 16x16 operator on (p_j, p_j+1), row-major
  double2* X;             // Jacobi input: the merged, gated, lambda-scaled bond matrix,
                          // m x n row-major, or its transpose (n x m) when transposed
  double2* T0;            // m x n: the merge (written by the merge GEMM), then gated in
                          // place by the gate kernel (without lambda)
  int32_t chi_l, chi_m, chi_r;
  int32_t m, n;           // 4*chi_l, 4*chi_r
  int32_t transposed;     // 1 when m > n: the Jacobi orthogonalises the n columns
};

// Per-factorisation state of the batched one-sided Jacobi kernel.  The kernel makes the
// m rows of X (each of length n) mutually orthogonal; m <= n always (the host transposes a
// tall bond matrix), because more vectors than dimensions cannot all be made orthogonal.
// When Q is given (m x m, set to the identity), every rotation is also applied to the rows
// of Q, which then holds the accumulated unitary.
// Noise floors (nullptr fro2: none): with dead2 = dead_rel * |X|_F^2 and marg2 = 6 m dead2,
// a pair is not rotated when both rows are below dead2, or one is below dead2 and the other
// below marg2.  With dead_rel <= (eps_cut / (10 m))^2 and eps_cut * s_0 >= eps_cut |X|_F /
// sqrt(m): every row above marg2 ends orthogonal to every other row (its norm is a singular
// value), the rows between the floors are mutually orthogonal, and the block of all rows
// below marg2 has no singular value above 0.35 eps_cut s_0, so the kept set is exact.
// stamp (m entries, set to -1 by the caller before the launch) records the round in which
// each row was last rotated: a pair neither of whose rows changed since the pair's own
// check one sweep earlier has the same inner product and is skipped.
// dead2_ovr (nullable): a device value that raises dead2 above dead_rel * |X|_F^2 (the
// deflation floor set after the FP32 sweeps when the chi_max cap decides the count).
struct JacobiTask {
  double2* X;             // m x n row-major; rows are orthogonalised in place
  double2* Q;             // optional m x m accumulator (nullptr: none)
  double* nrm2;           // m squared row norms (scratch owned by the kernel)
  const double* fro2;     // squared Frobenius norm of X (or nullptr)
  int32_t* stamp;         // m rounds of last rotation (scratch, -1 at launch)
  const double* dead2_ovr;
  double dead_rel;
  int32_t m, n;
  int32_t mp;             // m rounded up to even
  int32_t pad_;
};
// The same for the FP32 preconditioning sweeps (single-precision complex).
struct JacobiTask32 {
  float2* X;
  float2* Q;
  float* nrm2;
  const double* fro2;
  int32_t* stamp;
  const double* dead2_ovr;
  double dead_rel;
  int32_t m, n;
  int32_t mp;
  int32_t pad_;
};
struct JacobiStatus {
  unsigned int rot[3];    // rotations per sweep (ring of three)
  int32_t sweeps;         // sweeps completed when the task stopped
  int32_t converged;      // 1 converged, 0 hit the sweep cap
  int32_t pad_[3];
};

// Result of truncation (Sec. II.B.1 cutoff, App. A.4 chi_max): count kept rows, their row
// indices into X in descending order of norm, the kept normalised values and the norm.
struct TruncOut {
  int32_t count;
  int32_t m;              // rows examined
  double s0;              // largest singular value
  double nrm;             // sqrt(sum of kept s^2)
  double s_first_dropped; // first singular value not kept (0 if none)
  double total2;          // sum of the squares of all row norms (= squared Frobenius norm)
  double s_last_kept;     // smallest kept singular value (unnormalised)
};

// Launch wrappers (all asynchronous on `stream`; return cudaError_t of the launch).
cudaError_t launch_gemm(const GemmDesc* d_desc, int batch, int max_m, int max_n, cudaStream_t stream);
cudaError_t launch_gate_apply(const UpdateTask* d_tasks, int ntasks, int max_chi_l, int max_chi_r,
                              cudaStream_t stream);
// FP32 preconditioning: X32 = float(X) and Q32 = I for every task (dims from the FP64 task).
cudaError_t launch_precond_init(const JacobiTask* d_t64, const JacobiTask32* d_t32, int ntasks, int max_m,
                                int max_n, cudaStream_t stream);
// Squared Frobenius norm of each task's FP64 matrix into d_out[t].
// X32 = float(X) and X = double(X32) for each task pair (same m x n layout).
cudaError_t launch_narrow_rows(const JacobiTask* d_t64, const JacobiTask32* d_t32, int ntasks, int max_m, int max_n,
                               cudaStream_t stream);
cudaError_t launch_widen_rows(const JacobiTask32* d_t32, const JacobiTask* d_t64, int ntasks, int max_m, int max_n,
                              cudaStream_t stream);
cudaError_t launch_fro2(const JacobiTask* d_t64, int ntasks, double* d_out, cudaStream_t stream);
// Q64 = double(Q32) for every task (m x m).
cudaError_t launch_widen_q(const JacobiTask32* d_t32, double2* const* d_q64, int ntasks, int max_m,
                           cudaStream_t stream);
cudaError_t launch_jacobi32(const JacobiTask32* d_tasks, int ntasks, JacobiStatus* d_status, int max_sweeps,
                            unsigned int* d_bar, int* d_err, int sm_count, int max_len, int total_pairs,
                            cudaStream_t stream);
// stamp[k] = -1 for every row of every task (required before each Jacobi launch).
cudaError_t launch_init_stamps(const JacobiTask* d_tasks, int ntasks, int max_m, cudaStream_t stream);
cudaError_t launch_init_stamps32(const JacobiTask32* d_tasks, int ntasks, int max_m, cudaStream_t stream);
// The FP32 preconditioning sweeps in blocks of 8 rows (one block pair per CTA, rows in shared
// memory, accumulator Q updated once per block pair).  Needs every task's row length
// <= 1024 (returns cudaErrorInvalidValue otherwise: use launch_jacobi32) and stamp entries
// for (m + 7) / 8 + 1 blocks set to -1; bar = 2 zeroed unsigned ints, err as launch_jacobi.
cudaError_t launch_jacobi32_blocked(const JacobiTask32* d_tasks, int ntasks, JacobiStatus* d_status, int max_sweeps,
                                    unsigned int* d_bar, int* d_err, int sm_count, int max_len, cudaStream_t stream);
// Sets every task's accumulator Q (if any) to the identity.
cudaError_t launch_init_accumulators(const JacobiTask* d_tasks, int ntasks, int max_m, cudaStream_t stream);
// Cooperative persistent Jacobi over all tasks.  bar = 2 unsigned ints (zeroed by the
// caller), err = 1 int (zeroed): set to 1 if a grid barrier wait exceeded its limit.
// total_pairs = sum over tasks of mp/2 (pairs per round); it sets the group width.
// force_g: warps per row pair (1, 2, 4) for this launch; 0 = the tuning table, else the
// heuristic.
cudaError_t launch_jacobi(const JacobiTask* d_tasks, int ntasks, JacobiStatus* d_status,
                          int max_sweeps, unsigned int* d_bar, int* d_err, int sm_count,
                          int max_len, int total_pairs, cudaStream_t stream, int force_g = 0);
// The FP64 sweeps' group-width table (see launch_jacobi): buckets ceil(log2(longest row)) and
// floor(log2(pairs per round)).
constexpr int JAC_TUNE_LEN = 14;
constexpr int JAC_TUNE_PAIRS = 16;
void set_jacobi_tuning(int len_bucket, int pairs_bucket, int g);
int jacobi_tuning(int len_bucket, int pairs_bucket);
cudaError_t launch_truncate(const JacobiTask* d_tasks, int ntasks, double eps, int chi_max,
                            int32_t* d_idx, int idx_stride, double* d_lam, double* d_sraw,
                            int lam_stride, TruncOut* d_out, cudaStream_t stream);
// Truncation of a batch whose tasks carry their own cutoff, cap and output buffers (tasks
// of several circuits in one launch).
struct TruncTask {
  const double2* X;       // orthogonalised rows, m x n row-major
  int32_t* idx;           // kept row indices in descending order of norm [count]
  double* lam;            // kept values normalised to unit 2-norm [count]
  double* sraw;           // kept values, unnormalised [count]
  TruncOut* out;
  double eps;
  int32_t m, n;
  int32_t chi_max;
  int32_t pad_;
};
cudaError_t launch_truncate_tasks(const TruncTask* d_tasks, int ntasks, cudaStream_t stream);
// B_{j+1}'[k][c] = X[idx[k]][c] / s_idx[k] (rows path) or conj(Q[idx[k]][c]) (transposed
// path: the accumulated right singular vectors) for each task; dst pointers per task.
struct SplitRowsDesc {
  const double2* X;
  const double2* Q;       // non-null selects the transposed path
  double2* dst;
  const int32_t* idx;
  const double* sraw;     // kept singular values (row norms), unnormalised
  int32_t count, n;
};
cudaError_t launch_split_rows(const SplitRowsDesc* d_desc, int ntasks, int max_count, int max_n,
                              cudaStream_t stream);
// Deflation floor of the FP64 sweeps from the FP32 preconditioned rows.  For each task: the
// row norms of X32 (accumulated in FP64), sorted; s_c = the chi_max-th largest.  When the
// matrix has more than chi_max rows and s_c >= 1e-4 |X|_F (far above the FP32 rounding
// level), dead2_out = (s_c / (8 m))^2, else 0 (no deflation).  With that floor every row
// above the second floor 6 m dead2 ends orthogonal to every row, and the rows below it form
// a block of Frobenius norm <= sqrt(6) s_c / 8 < s_c: the chi_max largest singular values
// and their vectors are exact (checked after the FP64 sweeps, see pc_api.cpp).
struct DeflateTask {
  const float2* X32;      // m x n, the FP32 rows after the preconditioning sweeps
  const double* fro2;     // |X|_F^2 of the FP64 matrix
  double* dead2_out;
  double* sc_out;         // s_c (0 when not deflated)
  int32_t m, n;
  int32_t chi_max;
  int32_t pad_;
};
cudaError_t launch_deflate_floor(const DeflateTask* d_tasks, int ntasks, cudaStream_t stream);
// Recanonicalisation steps: Z = X (rows x cols, row-major) or its transpose.
cudaError_t launch_recanon_load(const double2* X, int rows, int cols, int transpose, double2* Z, cudaStream_t stream);
// After the one-sided Jacobi of Z (rows of length ld; rotations W in Q, ld x ld, when given) and
// the sort of its row norms (idx, sraw: kept rows, descending), one factor: element (k, a) for
// kept row k and a < n_out is conj(W[idx_k][a]) (use_q) or Z[idx_k][a], divided (scale 1) or
// multiplied (scale 2) by sraw_k, written to out[k][a] or, transposed, out[a][k].
cudaError_t launch_recanon_emit(const double2* Z, const double2* Q, int ld, const int32_t* idx, const double* sraw,
                                int count, int n_out, int use_q, int scale, int transpose_out, double2* out,
                                cudaStream_t stream);
cudaError_t launch_one_site(double2* B, int chi_l, int chi_r, const double2* g2_dev, int side,
                            cudaStream_t stream);
// Peak search: children of a prefix vector v (length chi_l) through site tensor B_j:
// w_sigma = v A^sigma (A^sigma = B_j[:, 2 sigma, :]), m_sigma = w E w^H.
cudaError_t launch_expand(const double2* v, const double2* Bj, int chi_l, int chi_r,
                          const double2* E, double2* w0, double2* w1, double* marg,
                          cudaStream_t stream);
// Sampling/amplitude helpers.
cudaError_t launch_quadform_rows(const double2* W, const double2* Y, int rows, int cols, int ld,
                                 double* out, cudaStream_t stream);
cudaError_t launch_sample_pick(const double2* W0, const double2* W1, const double* m0,
                               const double* m1, const double* u, int S, int chi, int site,
                               int n_sites, double2* Vnext, uint8_t* site_bits,
                               cudaStream_t stream);
cudaError_t launch_amp_pick(const double2* W0, const double2* W1, const uint8_t* site_bits, int K,
                            int chi, int site, int n_sites, double2* Vnext, cudaStream_t stream);
cudaError_t launch_fill_ones(double2* v, int rows, cudaStream_t stream);
// FMA-chain probe: blocks x 256 threads x 8 chains x iters FMAs in FP64 (fp64 = 1) or FP32.
cudaError_t launch_fma_probe(int fp64, int blocks, int iters, void* out, cudaStream_t stream);

// Mixed-precision merge on tcgen05 tensor cores (merge_tc.cu): for each descriptor of the
// batch, C = A * B (opB = 0, alpha = 1, beta = 0, no row scaling) as complex 3xTF32 with FP32
// accumulation; A, B and C are FP64 in global memory.  The workspace holds the split
// operands, tc_merge_workspace_bytes() of them for the batch's largest M, N, K.
// err (device int) is set to 1 if a bounded wait inside the kernel gave up.
size_t tc_merge_workspace_bytes(int T, int max_m, int max_n, int max_k);
cudaError_t launch_tc_merge(const GemmDesc* d_desc, int T, int max_m, int max_n, int max_k, void* workspace,
                            size_t workspace_bytes, int* d_err, cudaStream_t stream);

}  // namespace pc
