// Sparse LU of the affine operators by nested dissection and dense fronts
// (multifrontal), for the mean-based preconditioner P_T^k = J(x~; mu_bar,
// nu_bar) (Sec. 4.2; the paper factors it with a permuted sparse LU) and the
// Newton steps of the median problems (Sec. 3.2).
//
// Fill-reducing ordering: the structured node grid of the channel is bisected
// recursively along vertex lines (even node indices: a Q2 cell spans three
// node columns, so only a vertex line separates the cells on its two sides).
// Each separator is a front: its DOFs are eliminated together, after the two
// halves it separates.  Fronts of equal height in the separator tree are
// independent and are factored in the same launches ("level scheduling"),
// and so are the two sweeps of a solve.
#pragma once

#include <memory>

#include "dense.h"
#include "mesh.h"

namespace lrfsi {

// Symbolic structure (host, per mesh).
struct NdFront {
  int f = 0, b = 0, n = 0;      // fully summed DOFs, boundary DOFs, n = f + b
  int parent = -1, slot = 0;     // parent front, index among the parent's children (0 or 1)
  int height = 0;                // 0 for leaves
  long start = 0;                // first row of the front's F DOFs in the elimination order
  long boff = 0;                 // first row of its boundary block in the solve buffer (after the M rows)
  size_t off_front = 0;          // n x n front matrix (row-major) in the factor workspace
  size_t off_inv = 0;            // f x f inverse of the pivot block
  size_t off_piv = 0;            // f pivots
  size_t off_map = 0;            // b entries of the parent map / the boundary rows (int arrays)
};

struct NdSymbolic {
  std::vector<NdFront> fr;
  std::vector<std::vector<int>> by_height;  // fronts of each height
  std::vector<int> perm;          // elimination position -> DOF (M)
  std::vector<int> pos;           // DOF -> elimination position (M)
  std::vector<long long> entry_off;  // CSR entry -> offset in the front workspace
  std::vector<int> pmap;          // per front, b entries: solve-buffer row of each boundary DOF in the parent
                                  // (parent F: its elimination position; parent B: M + parent.boff + index)
  std::vector<int> fmap;          // per front, b entries: front-local row of each boundary DOF in the parent
  std::vector<int> brow;          // per front, b entries: elimination position of each boundary DOF
  size_t ws_doubles = 0, inv_doubles = 0, piv_ints = 0, map_ints = 0;
  long bsum = 0;                  // sum of b over the fronts (solve buffer rows after M)
  int maxf = 0, maxb = 0, maxn = 0, heights = 0;
  double factor_flops = 0;        // algorithmic FP64 work of one factorisation
};
int nd_symbolic(const MeshHost& h, NdSymbolic& sym);

// Device copies of the symbolic arrays (per mesh).
struct NdDevice {
  DevBuf<int> perm, pos, pmap, fmap, brow;
  DevBuf<long long> entry_off;
};

// Numeric factors of up to nprob problems (per handle).
struct NdPlan;  // the launch descriptors of a handle (nd_lu.cu)
struct NdLU {
  const NdSymbolic* sym = nullptr;
  const NdDevice* dsym = nullptr;
  int nprob = 0;
  DevBuf<double> ws;     // per problem: fronts, then the pivot-block inverses
  DevBuf<int> piv;       // per problem: pivots
  DevBuf<int> status;    // per problem
  DevBuf<int> zero;      // a device flag that stays 0 (closes the gate of a problem without columns)
  size_t per_prob = 0;   // doubles per problem in ws
  // solve buffers (per problem, (M + bsum) x ld and M x ld), sized on demand
  DevBuf<double> zu, yp;
  int ld = 0;
  std::shared_ptr<NdPlan> plan;
  size_t bytes() const { return ws.bytes() + piv.bytes() + status.bytes() + zu.bytes() + yp.bytes(); }
};
// ld: the largest number of right-hand sides of a solve (solve buffers).
int ndlu_alloc(lrfsi_mesh_s* m, int nprob, int ld, NdLU& lu);
// Factor A_q = J0_q + alpha_q Jmu'_q + beta_q Jnu'_q (values nnz x 3) for q < nprob.
int ndlu_factor(const lrfsi_mesh_s* m, NdLU& lu, const double* const* J3, const double* alpha, const double* beta,
                int nprob, cudaStream_t s);
// Y_q = A_q^{-1} X_q for r_q columns (X, Y: M x r, row-major, ld); X is not modified.
// gates (optional): the run condition of each problem's launches.
int ndlu_solve(NdLU& lu, double* const* X, double* const* Y, const int* r, int ld, int nprob, cudaStream_t s,
               const Gate* gates = nullptr);
int ndlu_status(NdLU& lu, int nprob, std::vector<int>& out, cudaStream_t s);

}  // namespace lrfsi
