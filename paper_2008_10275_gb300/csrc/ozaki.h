// FP64 Gram products G = A^T B of tall factors on the BF16 tensor cores by
// an error-free splitting (Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012).
//
// Every column of A and B is scaled by a power of two fixed by its largest
// entry and written as a 56-bit fixed-point integer, cut into 8 balanced
// base-128 digits (the slices: the first in [-128, 128], the others in
// [-64, 63]); a digit is exact in BF16.  The product of two slices summed over
// at most 256 rows stays below 2^24, so the FP32 accumulation of the tensor
// core is exact there; the slice products are grouped by level t + u (8
// levels, pairs with t + u >= 8 dropped: below 2^-54 of the column scales),
// read out of tensor memory every 256 rows and summed as integers.  The only
// rounding is the 56-bit fixed point of each input and the final FP64
// combination of the 8 levels: the result is as accurate as an FP64 Gram.
#pragma once

#include <vector>

#include "dense.h"

namespace lrfsi {

// Workspace (bytes) of ozaki_gram for nbatch products of M rows with at most
// pmax columns of A and qmax of B (B == A needs no slices of its own).
size_t ozaki_work_bytes(int nbatch, long M, int pmax, int qmax);
// G_b = A_b^T B_b for the descriptors (GramDesc, gates honoured); work: at
// least ozaki_work_bytes(...) bytes, 256-byte aligned.
int ozaki_gram(const GramDesc* d, int nbatch, long M, void* work, size_t work_bytes, cudaStream_t s);

// flag = 1 if a pipeline wait of the tensor-core Gram ran out since the last
// call (the products of that launch are wrong); synchronises the stream.
int ozaki_error(cudaStream_t s, int* flag);

// Tall GEMMs on the tensor cores (GemmDesc::tc, m >= 2048, 1 <= k <= 400).
bool ozaki_gemm_eligible(const GemmDesc<double>& g);
size_t ozaki_gemm_work_bytes(const GemmDesc<double>* d, int n);
int ozaki_gemm(const GemmDesc<double>* d, int n, void* work, size_t work_bytes, cudaStream_t s);

// Gram product path: 1 = tensor cores (this file), 0 = FP64 SIMT kernels.
int gram_path();
void set_gram_path(int p);

// ---------------------------------------------------------------------------
// GEMMs with fixed left operands on the tensor cores: C_i = alpha_i A_i B_i +
// beta_i C_i (row-major FP64), where the A_i (m_i x k_i, k_i <= 400) change
// rarely and the B_i (k_i x ncols) at every call -- the solves of a factored
// matrix.  slice() cuts the A_i into their slices once after they change (the
// contraction index is equilibrated by the column scales of A_i, as in
// ozaki_gemm); gemm() slices only the B_i and runs the slice products.  The
// result has the accuracy of ozaki_gemm.
// ---------------------------------------------------------------------------
struct OzFixedGemm {
  const double* A;  // m x k, row-major (lda); read by slice()
  int lda, m, k;
  const double* B;  // k x ncols, row-major (ldb); read by gemm()
  long ldb;
  double* C;        // m x ncols, row-major (ldc)
  long ldc;
  int q;            // problem index: gemm() skips the GEMM when gates.g[q] is closed
  double alpha, beta;
};
struct OzGates {
  Gate g[kMaxGemmDescs];
};
// whether a left operand of this shape goes to the tensor cores
bool ozaki_fixed_eligible(int m, int k);

class OzFixedPlan {
 public:
  // A group of GEMMs run by one gemm() call, ordered by problem index q
  // (ascending, q < nprob of build()); returns the group index.
  int add_group(const std::vector<OzFixedGemm>& g);
  // Lays out and uploads the descriptors into one device buffer with the A
  // slices and the B workspace for up to max_cols columns.
  int build(int max_cols, int nprob);
  // The A slices of the problems q < nprob (after their A_i changed).
  int slice(int nprob, cudaStream_t s) const;
  // Group g for the problems q < nprob with ncols (<= max_cols) columns of B.
  int gemm(int g, int ncols, int nprob, const OzGates& gates, cudaStream_t s) const;
  bool empty(int g) const { return g < 0 || g >= (int)groups_.size() || groups_[g].gemms.empty(); }
  size_t device_bytes() const { return buf_.bytes(); }
  // device bytes that build() would allocate
  size_t bytes_needed(int max_cols) const;

 private:
  struct Group {
    std::vector<OzFixedGemm> gemms;
    std::vector<int> prefix;   // GEMMs of the problems < q (q = 0 .. nprob)
    size_t d_off = 0;          // device descriptors (OzNdG)
    int mmax = 0, kmax = 0, ntmax = 0;
  };
  std::vector<Group> groups_;
  int nprob_ = 0, max_cols_ = 0;
  size_t e_off_ = 0, a_off_ = 0;  // slicing descriptors (OzOp, problem-major)
  std::vector<int> sl_prefix_;     // slicing descriptors of the problems < q
  std::vector<size_t> aex_prefix_; // bytes of the A exponents of the problems < q
  size_t aex_off_ = 0, bex_off_ = 0, bsl_off_ = 0;
  int sl_rows_max_ = 0, sl_n_max_ = 0, sl_nch_max_ = 0, sl_nt_max_ = 0;
  DevBuf<unsigned char> buf_;
};

}  // namespace lrfsi
