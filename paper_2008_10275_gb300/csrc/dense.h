// Dense linear algebra building blocks (FP64 unless templated).
#pragma once

#include "common.h"

namespace lrfsi {

// C(i,j) = alpha * sum_l A(i,l) B(l,j) + beta * C(i,j), element (i,j) of X at
// X.p[i * X.rs + j * X.cs].  beta == 0 never reads C.
// Optional: gate (run condition, see Gate); sel != nullptr && *sel != 0 reads
// A_alt instead of A (same strides).
template <class T>
struct GemmDesc {
  int m, n, k;
  const T* A; long a_rs, a_cs;
  const T* B; long b_rs, b_cs;
  T* C; long c_rs, c_cs;
  T alpha, beta;
  Gate gate;
  const T* A_alt = nullptr;
  const int* sel = nullptr;
  // 1: a tall product (m >= 2048, k <= 400) that may run on the tensor cores
  // (ozaki.h); set where the error bound |A| |B| is the one that matters
  int tc = 0;
};
constexpr int kMaxGemmDescs = 32;
template <class T>
int gemm_grouped(const GemmDesc<T>* descs, int n, cudaStream_t s);
// Split-K workspace of the grouped GEMM on the calling thread: by default a
// process-wide buffer grown on demand; between gemm_ws_bind(p, bytes) and
// gemm_ws_bind(nullptr, 0) the calls use p instead and fail (LRFSI_EINVAL)
// rather than grow it (a launch sequence captured into a CUDA graph must not
// see its workspace move).  gemm_ws_peak() is the largest need since the last
// gemm_ws_peak_reset().
void gemm_ws_bind(void* p, size_t bytes);
size_t gemm_ws_peak();
void gemm_ws_peak_reset();

// Batched tall Gram G_b = A_b^T B_b (p_b x q_b, row-major ldg) with
// A_b: M x p_b (row-major, lda), B_b: M x q_b (ldb); split over rows and
// reduced in fixed order.  work must hold nbatch * nsplit * pmax * qmax doubles.
struct GramDesc {
  const double* A; int lda, p;
  const double* B; int ldb, q;
  double* G; int ldg;
  Gate gate;
};
int gram_batched(const GramDesc* d, int nbatch, long M, double* work, size_t work_len, cudaStream_t s);
size_t gram_work_len(int nbatch, long M, int pmax, int qmax);

// Truncation helpers, one CTA per problem (see dense.cu for the algorithm).
struct TruncDesc {
  // inputs
  int p;             // concatenated rank
  int m;             // parameter-side rows
  const double* Vc;  // m x p row-major (ldv)
  int ldv;
  double* G;         // p x p Gram of the tall factor (in: X^T X), workspace afterwards
  double* G2;        // p x p Gram of Q1 (filled between the two passes)
  double* T1;        // p x p: Q1 = X T1 after pass 1; final tall coefficients after the SVD (ld p)
  double* T2;        // p x p: inverse Cholesky factor of the latest QR pass (ld p)
  double* Vout;      // m x rank output (row-major, ldvo)
  int ldvo;
  double* work;      // scratch for the small SVD (>= trunc_small_work(p, m) doubles)
  const double* core;  // k x m core for the SVD (ld m): one of the two core buffers of work
  int* iwork;        // >= 2 p ints
  int* info;         // [0] k (kept after pass 1), [1] rank, [2] status, [3] sweeps, [4] needs another QR pass
  double* sv;        // >= p singular values (descending)
  double* frob2;     // output: squared Frobenius norm of the input product (sum of s^2)
  double tol;        // relative Frobenius truncation tolerance
  int rank_cap;
  double drop;       // pass-1 pivot threshold on the unit-diagonal Gram
  // optional (device-driven launch sequences):
  Gate gate;                        // run condition of every kernel of this problem
  const double* core_alt = nullptr;  // SVD core when sel != nullptr && *sel != 0
  const int* sel = nullptr;
  int* rank_out = nullptr;          // SVD: the chosen rank is also written here
  int* count = nullptr;             // SVD: incremented once per truncation
  int* broke = nullptr;             // Cholesky-QR: set to 1 on a breakdown (sticky)
};
size_t trunc_small_work(int p, int m);
// Cluster size of the SVD kernel: 0 = chosen from the number of problems,
// else 2, 4, 8 or 16; c < 0 only queries.  Returns the previous setting.
int svd_cluster(int c);
// upload = false: d_dev already holds the n descriptors (d is still read on
// the host for launch shapes)
int trunc_pass1(const TruncDesc* d, int n, cudaStream_t s, TruncDesc* d_dev, bool upload = true);
// write_third = 0: a later pass that must not overwrite the "another pass"
// flag (info[4]) of the first QR pass
// pmax: the largest p of the n problems (sizes the shared-memory working copy)
int trunc_qr(int n, cudaStream_t s, TruncDesc* d_dev, int write_third = 1, int pmax = 0);
int trunc_svd(const TruncDesc* d, int n, cudaStream_t s, TruncDesc* d_dev, bool upload = true);

// Offsets of the per-problem scratch (doubles): Dsc (p) | Rk (p*p) | Rki (p*p) |
// Y (p*m) | C (p*m) | A (n'*n') | Vm (n'*n'), n' = max(p, m).  Rk holds the
// scaled pass-1 factor, later W_r; Rki the zero-padded factor of the latest QR
// pass; Y and C the two core buffers.
struct TruncWork {
  double *Dsc, *Rk, *Rki, *Y, *C, *A, *Vm, *Jg;
  __host__ __device__ TruncWork(double* w, int p, int m) {
    const size_t n = (size_t)(p > m ? p : m);
    Dsc = w;
    Rk = Dsc + p;
    Rki = Rk + (size_t)p * p;
    Y = Rki + (size_t)p * p;
    C = Y + (size_t)p * m;
    A = C + (size_t)p * m;
    Vm = A + n * n;
    Jg = Vm + n * n;  // column blocks of the cluster SVD when they exceed shared memory
  }
};
// Doubles of Jg per problem for a cluster of C CTAs: C x 4 b (L + n + 2),
// b = ceil(n / 2C) (a column: its n + n entries and its norm, padded).
__host__ __device__ inline size_t trunc_svd_global_len(int p, int m, int C) {
  const int n = p < m ? p : m, L = p < m ? m : p;
  const int b = (n + 2 * C - 1) / (2 * C);
  return (size_t)C * 4 * b * (size_t)(L + n + 2);
}
// The QR preconditioning of the SVD (after Jg, sized for p x m): Householder
// vectors Aw (L x n, column-major), X = R^T (n x n, column c = row c of R),
// tau (n), the column permutation (n ints), the trailing norms (n) and one
// length-L scratch vector per warp of a 16-CTA cluster.
struct QrWork {
  double *Aw, *Rt, *tau, *nrm, *scr;
  int* perm;
  __host__ __device__ QrWork(const TruncWork& W, int p, int m) {
    const size_t n = (size_t)(p < m ? p : m), L = (size_t)(p < m ? m : p);
    Aw = W.Jg + trunc_svd_global_len(p, m, 16);
    Rt = Aw + L * n;
    tau = Rt + n * n;
    nrm = tau + n;
    perm = (int*)(nrm + n);
    scr = nrm + 2 * n;  // perm takes n ints (<= n doubles)
  }
};
__host__ __device__ inline size_t trunc_qr_len(int p, int m) {
  const size_t n = (size_t)(p < m ? p : m), L = (size_t)(p < m ? m : p);
  return L * n + n * n + 3 * n + 16 * 8 * L;
}

}  // namespace lrfsi
