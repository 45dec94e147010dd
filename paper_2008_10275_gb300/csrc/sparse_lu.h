// Sparse operator application and the block-tridiagonal preconditioner LU.
#pragma once

#include "dense.h"
#include "mesh.h"

namespace lrfsi {

// Y-blocks of the affine operator applied to a tall factor U (M x r, ldu):
//   split mode: Y[:, o_t + j] = s_t * (J_t U)[:, j] for t = 0, 1, 2 (J0, Jmu', Jnu')
//   combined  : Y[:, o_0 + j] = s_0 * ((J0 + a1 Jmu' + a2 Jnu') U)[:, j]   (o_1 < 0)
template <class T>
struct SpmmDesc {
  const T* J3;        // nnz x 3 interleaved values
  const T* U; int ldu, r;
  T* Y; int ldy;
  int o[3];           // output column offsets (o[1] < 0: combined mode)
  T sc[3];            // output scales
  T a1, a2;           // combined-mode coefficients
  Gate gate;          // run condition (see Gate)
};
template <class T>
int spmm_batched(const lrfsi_mesh_s* m, const SpmmDesc<T>* d, int n, cudaStream_t s);
// The autotuner's table: chosen shape (-1: not tuned) and timed ms of the shapes.
int spmm_autotune_table(int precision, int bucket, int* variant, float* ms);

// Block-tridiagonal LU of A_b = J0_b + alpha_b Jmu'_b + beta_b Jnu'_b over
// the slab ordering: per slab s, S_s = D_s - Lo_{s-1} W_{s-1} (dense, FP64)
// is factored with partial pivoting, W_s = S_s^{-1} Up_s and the explicit
// inverse Sinv_s = S_s^{-1} are kept, so that a solve is a chain of GEMMs.
struct BlockLU {
  int nslab = 0, nmax = 0, nprob = 0;
  std::vector<long> off;           // slab offsets (host)
  DevBuf<double> ws;               // per problem: D | Up(->W) | Lo | Sinv | RHS scratch
  DevBuf<int> piv;                 // per problem: nslab x nmax
  DevBuf<int> status;              // per problem
  size_t per_prob = 0;             // doubles per problem in ws
  size_t off_up = 0, off_lo = 0, off_inv = 0, off_rhs = 0;
  size_t bytes() const { return ws.bytes() + piv.bytes() + status.bytes(); }
};
int blocklu_alloc(const lrfsi_mesh_s* m, int nprob, BlockLU& lu);
// J3[b] (device, nnz x 3) and the coefficients per problem.
// Single-solve mode (b != nullptr): instead of keeping S_s^{-1}, the forward
// sweep of one right-hand side per problem (b[q], stride ldb) is carried
// through the factorisation and the backward sweep follows it, so that y[q]
// (stride ldb) receives A_q^{-1} b[q]; the factors cannot be reused for
// blocklu_solve afterwards.
int blocklu_factor(const lrfsi_mesh_s* m, BlockLU& lu, const double* const* J3, const double* alpha,
                   const double* beta, int nprob, cudaStream_t s, const double* const* b = nullptr,
                   double* const* y = nullptr, int ldb = 0);
// Y_b = A_b^{-1} X_b for r columns; X_b is overwritten (scratch).  X, Y: M x r, ld.
// gates (optional, nprob entries): the run condition of each problem's GEMMs.
int blocklu_solve(BlockLU& lu, double* const* X, double* const* Y, const int* r, int ld, int nprob,
                  cudaStream_t s, const Gate* gates = nullptr);
// Host copy of per-problem status (0 ok, LRFSI_ESINGULAR).
int blocklu_status(BlockLU& lu, int nprob, std::vector<int>& out, cudaStream_t s);

}  // namespace lrfsi
