// Nested-dissection multifrontal LU of the affine operators (see nd_lu.h).
//
// Symbolic phase (host, once per mesh): recursive bisection of the node grid
// along vertex lines gives the separator tree; the fronts are numbered in
// post order (children before parents), which is also the elimination order.
// Front t holds its fully summed DOFs F_t (the separator, or all DOFs of a
// leaf region) followed by its boundary DOFs B_t (the DOFs of ancestor
// separators coupled to its subtree, in elimination order).
//
// Numeric phase, per height of the tree (all fronts of one height at once):
//   P_t A_FF = L U                      panel LU, pivots among the F rows
//   [W | A_FF^{-1}] = A_FF^{-1} [A_FB | I]   triangular solves, explicit inverse
//   S_BB = A_BB - A_BF W                Schur complement (GEMM)
//   parent front += S_BB                extend-add (siblings in separate launches)
// The explicit inverses make every step of a solve a GEMM:
//   forward (heights up):   y_F = A_FF^{-1} z_F,  z_B -= A_BF y_F, z_B added to the parent
//   backward (heights down): x_F = y_F - W x_B
#include <algorithm>
#include <cmath>
#include <functional>
#include <mutex>
#include <numeric>

#include "nd_lu.h"
#include "ozaki.h"

namespace lrfsi {

// ---------------------------------------------------------------------------
// symbolic phase
// ---------------------------------------------------------------------------
constexpr int kNdLeafNodes = 25;  // regions of at most 5 x 5 nodes are not bisected further

int nd_symbolic(const MeshHost& h, NdSymbolic& sym) {
  const int NX = 2 * h.nx + 1, NY = 2 * h.ny + 1;
  const long M = h.M;
  std::vector<std::vector<int>> node_dofs((size_t)NX * NY);
  for (long d = 0; d < M; ++d) node_dofs[(size_t)h.dof_ix[d] + (size_t)NX * h.dof_iy[d]].push_back((int)d);
  sym.fr.clear();
  std::vector<std::vector<int>> F;      // F DOFs per front
  std::vector<std::vector<int>> kids;   // children per front
  std::vector<int> owner(M, -1);
  // recursive bisection of the node rectangle [x0, x1] x [y0, y1]; returns the front id
  std::function<int(int, int, int, int)> build = [&](int x0, int x1, int y0, int y1) -> int {
    auto even_cut = [](int a0, int a1) -> int {  // even index strictly inside (a0, a1), nearest the middle
      const int mid = (a0 + a1) / 2;
      for (int dlt = 0; dlt <= (a1 - a0); ++dlt) {
        for (int c : {mid - dlt, mid + dlt})
          if (c > a0 && c < a1 && (c & 1) == 0) return c;
      }
      return -1;
    };
    const int nxr = x1 - x0 + 1, nyr = y1 - y0 + 1;
    int cx = -1, cy = -1;
    if ((long)nxr * nyr > kNdLeafNodes) {
      cx = even_cut(x0, x1);
      cy = even_cut(y0, y1);
    }
    std::vector<int> children, fd;
    if (cx >= 0 && (nxr >= nyr || cy < 0)) {
      children.push_back(build(x0, cx - 1, y0, y1));
      children.push_back(build(cx + 1, x1, y0, y1));
      for (int y = y0; y <= y1; ++y)
        for (int d : node_dofs[(size_t)cx + (size_t)NX * y]) fd.push_back(d);
    } else if (cy >= 0) {
      children.push_back(build(x0, x1, y0, cy - 1));
      children.push_back(build(x0, x1, cy + 1, y1));
      for (int x = x0; x <= x1; ++x)
        for (int d : node_dofs[(size_t)x + (size_t)NX * cy]) fd.push_back(d);
    } else {  // leaf: every DOF of the region
      for (int y = y0; y <= y1; ++y)
        for (int x = x0; x <= x1; ++x)
          for (int d : node_dofs[(size_t)x + (size_t)NX * y]) fd.push_back(d);
    }
    const int id = (int)F.size();
    for (int d : fd) owner[d] = id;
    F.push_back(std::move(fd));
    kids.push_back(std::move(children));
    return id;
  };
  build(0, NX - 1, 0, NY - 1);
  const int nf = (int)F.size();
  for (long d = 0; d < M; ++d)
    if (owner[d] < 0) return fail(LRFSI_EINVAL, "nested dissection: a DOF belongs to no front");
  sym.fr.assign(nf, NdFront{});
  std::vector<int> first(nf);
  for (int t = 0; t < nf; ++t) {
    first[t] = t;
    int hgt = 0;
    for (int slot = 0; slot < (int)kids[t].size(); ++slot) {
      const int c = kids[t][slot];
      sym.fr[c].parent = t;
      sym.fr[c].slot = slot;
      first[t] = std::min(first[t], first[c]);
      hgt = std::max(hgt, sym.fr[c].height + 1);
    }
    sym.fr[t].height = hgt;
    sym.fr[t].f = (int)F[t].size();
  }
  // elimination order: fronts in post order, each front's F DOFs in order
  sym.perm.assign(M, 0);
  sym.pos.assign(M, 0);
  {
    long p = 0;
    for (int t = 0; t < nf; ++t) {
      sym.fr[t].start = p;
      for (int d : F[t]) {
        sym.perm[p] = d;
        sym.pos[d] = (int)p;
        ++p;
      }
    }
  }
  // symmetric adjacency of the union pattern
  std::vector<int> tptr(M + 1, 0), tidx(h.colidx.size());
  for (size_t e = 0; e < h.colidx.size(); ++e) tptr[h.colidx[e] + 1]++;
  for (long i = 0; i < M; ++i) tptr[i + 1] += tptr[i];
  {
    std::vector<int> fill(tptr.begin(), tptr.end() - 1);
    for (long i = 0; i < M; ++i)
      for (int e = h.rowptr[i]; e < h.rowptr[i + 1]; ++e) tidx[fill[h.colidx[e]]++] = (int)i;
  }
  // boundary sets, bottom up
  std::vector<std::vector<int>> B(nf);
  std::vector<int> mark(M, -1);
  for (int t = 0; t < nf; ++t) {
    std::vector<int> cand;
    auto take = [&](int j) {
      if (owner[j] > t && mark[j] != t) {
        mark[j] = t;
        cand.push_back(j);
      } else if (owner[j] < first[t]) {
        cand.push_back(-1);  // coupling across separated regions: not a valid dissection
      }
    };
    for (int c : kids[t])
      for (int j : B[c]) take(j);
    for (int i : F[t]) {
      for (int e = h.rowptr[i]; e < h.rowptr[i + 1]; ++e) take(h.colidx[e]);
      for (int e = tptr[i]; e < tptr[i + 1]; ++e) take(tidx[e]);
    }
    if (std::find(cand.begin(), cand.end(), -1) != cand.end())
      return fail(LRFSI_EINVAL, "nested dissection: separator does not separate");
    std::sort(cand.begin(), cand.end(), [&](int a, int b) { return sym.pos[a] < sym.pos[b]; });
    B[t] = std::move(cand);
    sym.fr[t].b = (int)B[t].size();
    sym.fr[t].n = sym.fr[t].f + sym.fr[t].b;
  }
  // offsets, heights, maps
  size_t of = 0, oi = 0, op = 0;
  long ob = 0;
  sym.maxf = sym.maxb = sym.maxn = 0;
  sym.heights = 0;
  sym.factor_flops = 0;
  for (int t = 0; t < nf; ++t) {
    NdFront& fr = sym.fr[t];
    fr.off_front = of;
    fr.off_inv = oi;
    fr.off_piv = op;
    fr.boff = ob;
    fr.off_map = (size_t)ob;
    of += (size_t)fr.n * fr.n;
    oi += (size_t)fr.f * fr.f;
    op += (size_t)fr.f;
    ob += fr.b;
    sym.maxf = std::max(sym.maxf, fr.f);
    sym.maxb = std::max(sym.maxb, fr.b);
    sym.maxn = std::max(sym.maxn, fr.n);
    sym.heights = std::max(sym.heights, fr.height + 1);
    const double f = fr.f, b = fr.b;
    sym.factor_flops += (2.0 / 3.0) * f * f * f + 2.0 * f * f * (b + f) + 2.0 * b * b * f;
  }
  sym.ws_doubles = of;
  sym.inv_doubles = oi;
  sym.piv_ints = op;
  sym.bsum = ob;
  sym.map_ints = (size_t)ob;
  sym.by_height.assign(sym.heights, {});
  for (int t = 0; t < nf; ++t) sym.by_height[sym.fr[t].height].push_back(t);
  sym.pmap.assign(ob, 0);
  sym.fmap.assign(ob, 0);
  sym.brow.assign(ob, 0);
  std::vector<int> loc(M, -1);
  for (int p = 0; p < nf; ++p) {
    const NdFront& P = sym.fr[p];
    for (int i = 0; i < P.f; ++i) loc[F[p][i]] = i;
    for (int i = 0; i < P.b; ++i) loc[B[p][i]] = P.f + i;
    for (int c : kids[p]) {
      const NdFront& Cf = sym.fr[c];
      for (int i = 0; i < Cf.b; ++i) {
        const int j = B[c][i];
        const int lj = loc[j];
        if (lj < 0) return fail(LRFSI_EINVAL, "nested dissection: boundary DOF missing in the parent front");
        sym.fmap[Cf.off_map + i] = lj;
        sym.pmap[Cf.off_map + i] = lj < P.f ? (int)(P.start + lj) : (int)(M + P.boff + (lj - P.f));
      }
    }
    for (int i = 0; i < P.b; ++i) sym.brow[P.off_map + i] = sym.pos[B[p][i]];
    for (int i = 0; i < P.f; ++i) loc[F[p][i]] = -1;
    for (int i = 0; i < P.b; ++i) loc[B[p][i]] = -1;
  }
  // CSR entry -> front slot: the front of whichever of (i, j) is eliminated first
  const size_t nnz = h.colidx.size();
  sym.entry_off.assign(nnz, -1);
  std::vector<std::vector<std::pair<int, int>>> bucket(nf);  // (entry, row)
  for (long i = 0; i < M; ++i)
    for (int e = h.rowptr[i]; e < h.rowptr[i + 1]; ++e)
      bucket[std::min(owner[i], owner[h.colidx[e]])].push_back({e, (int)i});
  for (int t = 0; t < nf; ++t) {
    const NdFront& T = sym.fr[t];
    for (int i = 0; i < T.f; ++i) loc[F[t][i]] = i;
    for (int i = 0; i < T.b; ++i) loc[B[t][i]] = T.f + i;
    for (auto& er : bucket[t]) {
      const int li = loc[er.second], lj = loc[h.colidx[er.first]];
      if (li < 0 || lj < 0) return fail(LRFSI_EINVAL, "nested dissection: matrix entry outside its front");
      sym.entry_off[er.first] = (long long)T.off_front + (long long)li * T.n + lj;
    }
    for (int i = 0; i < T.f; ++i) loc[F[t][i]] = -1;
    for (int i = 0; i < T.b; ++i) loc[B[t][i]] = -1;
  }
  return LRFSI_OK;
}

// ---------------------------------------------------------------------------
// numeric phase: kernels
// ---------------------------------------------------------------------------
constexpr int kNdNb = 32;             // panel width
constexpr int kNdPanelThreads = 256;
constexpr int kNdCols = 8;            // columns per CTA of the column-parallel kernels
constexpr int kNdColThreads = 512;
constexpr size_t kNdSmem = 220 * 1024;

// One front of one problem in the factorisation.
struct NdFD {
  double* A;    // n x n front (row-major, ld n)
  double* inv;  // f x f inverse of the pivot block
  int* piv;     // f pivots (absolute rows of the F block)
  int* status;  // the problem's status word
  int n, f;
};
// C (m x n, ldc) = alpha A (m x k, lda) B (k x n, ldb) + beta C, row-major; q = problem (gate index).
struct NdGemm {
  const double* A; const double* B; double* C;
  int m, n, k, lda, ldb, ldc, q;
  double alpha, beta;
};
// Extend-add of a b x b block (ldS) into rows/columns map[] of the parent (ldP).
struct NdExt {
  const double* S; double* P; const int* map;
  int b, ldS, ldP, q;
};
struct NdProbs {
  double* ws[kMaxGemmDescs];
  const double* J3[kMaxGemmDescs];
  double alpha[kMaxGemmDescs], beta[kMaxGemmDescs];
};
using NdGates = OzGates;

__global__ void k_nd_extract(NdProbs pp, const long long* __restrict__ entry_off, long nnz) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  const int q = blockIdx.y;
  const double* J = pp.J3[q];
  pp.ws[q][entry_off[e]] = J[3 * e] + pp.alpha[q] * J[3 * e + 1] + pp.beta[q] * J[3 * e + 2];
}

__device__ __forceinline__ unsigned long long nd_abs_key(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
}
__device__ __forceinline__ void nd_argmax(unsigned long long& v, int& i, unsigned long long v2, int i2) {
  if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
}

// Panel LU with partial pivoting of columns [j0, j0 + nb) of the F block
// (pivot rows among the F rows j0 .. f-1), staged in shared memory; one CTA
// per front.  Keys of |x| compared as integers; a NaN or zero pivot sets the
// status (reported, the factorisation continues without NaNs from it).
__global__ void __launch_bounds__(kNdPanelThreads) k_nd_panel(const NdFD* __restrict__ fds, int j0, int nbw) {
  constexpr int kWarps = kNdPanelThreads / 32;
  const NdFD d = fds[blockIdx.x];
  if (j0 >= d.f) return;
  const int nb = min(nbw, d.f - j0);
  const int rows = d.f - j0, sl = nb + 1, ld = d.n;
  double* A = d.A;
  extern __shared__ double sp[];
  __shared__ unsigned long long s_val[kWarps];
  __shared__ int s_idx[kWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (long e = tid; e < (long)rows * nb; e += kNdPanelThreads) {
    const int i = (int)(e / nb), c = (int)(e % nb);
    sp[(size_t)i * sl + c] = A[(size_t)(j0 + i) * ld + j0 + c];
  }
  __syncthreads();
  auto warp_argmax = [&](unsigned long long best, int bi) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v2 = __shfl_xor_sync(0xffffffffu, best, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      nd_argmax(best, bi, v2, i2);
    }
    if (lane == 0) { s_val[warp] = best; s_idx[warp] = bi; }
  };
  {
    unsigned long long best = 0;
    int bi = 0x7fffffff;
    for (int i = tid; i < rows; i += kNdPanelThreads) nd_argmax(best, bi, nd_abs_key(sp[(size_t)i * sl]), i);
    warp_argmax(best, bi);
  }
  __syncthreads();
  for (int jj = 0; jj < nb; ++jj) {
    unsigned long long pk = 0;
    int pr = 0x7fffffff;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) nd_argmax(pk, pr, s_val[w], s_idx[w]);
    double pv = __longlong_as_double((long long)pk);
    if (pr >= rows) { pr = jj; pv = 0.0; }
    if (tid == 0) {
      d.piv[j0 + jj] = j0 + pr;
      if (!(pv > 0.0)) *d.status = LRFSI_ESINGULAR;
    }
    if (pr != jj)
      for (int c = tid; c < nb; c += kNdPanelThreads) {
        const double t = sp[(size_t)jj * sl + c];
        sp[(size_t)jj * sl + c] = sp[(size_t)pr * sl + c];
        sp[(size_t)pr * sl + c] = t;
      }
    __syncthreads();
    const double* rj = sp + (size_t)jj * sl;
    double dgn = rj[jj];
    if (dgn == 0.0) dgn = 1e-300;
    const double inv = 1.0 / dgn;
    const int w = nb - jj - 1;
    unsigned long long best = 0;
    int bi = 0x7fffffff;
    for (int i = jj + 1 + tid; i < rows; i += kNdPanelThreads) {
      double* ri = sp + (size_t)i * sl;
      const double l = ri[jj] * inv;
      ri[jj] = l;
      for (int c = 0; c < w; ++c) ri[jj + 1 + c] = fma(-l, rj[jj + 1 + c], ri[jj + 1 + c]);
      if (w > 0) nd_argmax(best, bi, nd_abs_key(ri[jj + 1]), i);
    }
    warp_argmax(best, bi);
    __syncthreads();
  }
  for (long e = tid; e < (long)rows * nb; e += kNdPanelThreads) {
    const int i = (int)(e / nb), c = (int)(e % nb);
    A[(size_t)(j0 + i) * ld + j0 + c] = sp[(size_t)i * sl + c];
  }
}

// After the panel [j0, j0 + nb) of the F block: its row interchanges applied to
// the other columns of the F block, then for the columns right of the panel
// U12 = L11^{-1} A12 and A22 -= L21 U12 (F rows only).  CTA (t, front): 8
// columns; the first ceil(j0 / 8) CTAs take the columns left of the panel
// (interchanges only).
__global__ void __launch_bounds__(kNdColThreads) k_nd_update(const NdFD* __restrict__ fds, int j0, int nbw) {
  extern __shared__ double usm[];
  const NdFD d = fds[blockIdx.y];
  const int n = d.f, ld = d.n;
  if (j0 >= n) return;
  const int nb = min(nbw, n - j0);
  double* A = d.A;
  const int* piv = d.piv;
  const int nleft = (j0 + kNdCols - 1) / kNdCols;
  const bool left = (int)blockIdx.x < nleft;
  const int cb = left ? blockIdx.x * kNdCols : j0 + nb + (blockIdx.x - nleft) * kNdCols;
  const int ce = left ? min(cb + kNdCols, j0) : min(cb + kNdCols, n);
  if (cb >= ce) return;
  const int tid = threadIdx.x;
  if (left) {
    if (tid < ce - cb) {
      const int c = cb + tid;
      for (int j = j0; j < j0 + nb; ++j) {
        const int p = piv[j];
        if (p != j && p >= 0 && p < n) {
          const double t = A[(size_t)j * ld + c];
          A[(size_t)j * ld + c] = A[(size_t)p * ld + c];
          A[(size_t)p * ld + c] = t;
        }
      }
    }
    return;
  }
  const int rows = n - j0;
  double* Bt = usm;                                  // rows x 8 tile (rows j0 .. n-1)
  double* Ls = usm + (size_t)rows * kNdCols;         // 32 x 33: L11
  int* idx = reinterpret_cast<int*>(Ls + 32 * 33);   // row permutation of rows j0 .. n-1
  if (tid == 0) {
    for (int i = 0; i < rows; ++i) idx[i] = i;
    for (int j = j0; j < j0 + nb; ++j) {
      const int p = piv[j];
      if (p != j && p >= j0 && p < n) { const int t = idx[j - j0]; idx[j - j0] = idx[p - j0]; idx[p - j0] = t; }
    }
  }
  for (int e = tid; e < 32 * 32; e += kNdColThreads) {
    const int i = e >> 5, l = e & 31;
    Ls[i * 33 + l] = (i < nb && l < nb) ? A[(size_t)(j0 + i) * ld + j0 + l] : 0.0;
  }
  __syncthreads();
  for (int e = tid; e < rows * kNdCols; e += kNdColThreads) {
    const int r = e / kNdCols, c = e % kNdCols;
    Bt[e] = cb + c < ce ? A[(size_t)(j0 + idx[r]) * ld + cb + c] : 0.0;
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  if (warp == 0) {  // U12 = L11^{-1} A12 (unit lower), four lanes per column
    const int lq = lane & 3, lbase = lane & ~3, lc = lane >> 2;
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int i = lq + 4 * k;
      x[k] = i < nb ? Bt[(size_t)i * kNdCols + lc] : 0.0;
    }
#pragma unroll
    for (int l = 0; l < 32; ++l) {
      const double xl = __shfl_sync(0xffffffffu, x[l >> 2], lbase + (l & 3));
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int i = lq + 4 * k;
        if (i > l) x[k] = fma(-Ls[i * 33 + l], xl, x[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int i = lq + 4 * k;
      if (i < nb) Bt[(size_t)i * kNdCols + lc] = x[k];
    }
  }
  __syncthreads();
  {  // A22 -= L21 U12 (L21: the panel's rows below, already interchanged by the panel kernel)
    const int c = tid % kNdCols;
    for (int r = nb + tid / kNdCols; r < rows; r += kNdColThreads / kNdCols) {
      const double* ar = A + (size_t)(j0 + r) * ld + j0;
      double acc = Bt[(size_t)r * kNdCols + c];
#pragma unroll 8
      for (int l = 0; l < nb; ++l) acc = fma(-ar[l], Bt[(size_t)l * kNdCols + c], acc);
      Bt[(size_t)r * kNdCols + c] = acc;
    }
  }
  __syncthreads();
  for (int e = tid; e < rows * kNdCols; e += kNdColThreads) {
    const int r = e / kNdCols, c = e % kNdCols;
    if (cb + c < ce) A[(size_t)(j0 + r) * ld + cb + c] = Bt[e];
  }
}

// [W | A_FF^{-1}] = A_FF^{-1} [A_FB | I] with the factored F block (P A_FF = L U):
// CTA (t, front) takes columns [8 t, 8 t + 8) of the right-hand side (b + f
// columns), applies the interchanges, solves L then U, and writes W over A_FB
// and the inverse to its slot.  Each CTA reads and writes only its own
// right-hand-side columns; the factors are read-only.
__global__ void __launch_bounds__(kNdColThreads) k_nd_rhs(const NdFD* __restrict__ fds) {
  extern __shared__ double rsm[];
  const NdFD d = fds[blockIdx.y];
  const int n = d.f, b = d.n - d.f, w = d.n, ld = d.n;
  const int c0 = blockIdx.x * kNdCols;
  if (c0 >= w || n <= 0) return;
  double* Bt = rsm;                                  // n x 8 tile
  double* Ls = rsm + (size_t)n * kNdCols;            // 32 x 33 diagonal block
  int* idx = reinterpret_cast<int*>(Ls + 32 * 33);   // row permutation (n)
  const double* A = d.A;
  const int* piv = d.piv;
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int i = 0; i < n; ++i) idx[i] = i;
    for (int j = 0; j < n; ++j) {
      const int p = piv[j];
      if (p != j && p >= 0 && p < n) { const int t = idx[j]; idx[j] = idx[p]; idx[p] = t; }
    }
  }
  __syncthreads();
  for (int e = tid; e < n * kNdCols; e += kNdColThreads) {
    const int r = e / kNdCols, c = e % kNdCols, j = c0 + c;
    double v = 0.0;
    if (j < b) v = A[(size_t)idx[r] * ld + n + j];
    else if (j < w) v = (idx[r] == j - b) ? 1.0 : 0.0;
    Bt[e] = v;
  }
  const int lane = tid & 31, warp = tid >> 5;
  const int lq = lane & 3, lbase = lane & ~3, lc = lane >> 2;
  for (int pass = 0; pass < 2; ++pass) {
    const bool upper = pass == 1;
    const int nblk = (n + 31) / 32;
    for (int bb = 0; bb < nblk; ++bb) {
      const int blk = upper ? nblk - 1 - bb : bb;
      const int i0 = blk * 32, nbk = n - i0 < 32 ? n - i0 : 32;
      __syncthreads();
      for (int e = tid; e < 32 * 32; e += kNdColThreads) {
        const int i = e >> 5, l = e & 31;
        Ls[i * 33 + l] = (i < nbk && l < nbk) ? A[(size_t)(i0 + i) * ld + i0 + l] : 0.0;
      }
      __syncthreads();
      if (warp == 0) {
        double x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int i = lq + 4 * k;
          x[k] = i < nbk ? Bt[(size_t)(i0 + i) * kNdCols + lc] : 0.0;
        }
        if (!upper) {
#pragma unroll
          for (int l = 0; l < 32; ++l) {
            const double xl = __shfl_sync(0xffffffffu, x[l >> 2], lbase + (l & 3));
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const int i = lq + 4 * k;
              if (i > l) x[k] = fma(-Ls[i * 33 + l], xl, x[k]);
            }
          }
        } else {
#pragma unroll
          for (int l = 31; l >= 0; --l) {
            if (lq == (l & 3)) {
              const double dg = Ls[l * 33 + l];
              x[l >> 2] = (l < nbk) ? x[l >> 2] / (dg == 0.0 ? 1e-300 : dg) : 0.0;
            }
            const double xl = __shfl_sync(0xffffffffu, x[l >> 2], lbase + (l & 3));
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const int i = lq + 4 * k;
              if (i < l) x[k] = fma(-Ls[i * 33 + l], xl, x[k]);
            }
          }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int i = lq + 4 * k;
          if (i < nbk) Bt[(size_t)(i0 + i) * kNdCols + lc] = x[k];
        }
      }
      __syncthreads();
      const int rlo = upper ? 0 : i0 + nbk, rhi = upper ? i0 : n;
      const int c = tid % kNdCols;
      for (int r = rlo + tid / kNdCols; r < rhi; r += kNdColThreads / kNdCols) {
        const double* ar = A + (size_t)r * ld + i0;
        double acc = Bt[(size_t)r * kNdCols + c];
#pragma unroll 8
        for (int l = 0; l < nbk; ++l) acc = fma(-ar[l], Bt[(size_t)(i0 + l) * kNdCols + c], acc);
        Bt[(size_t)r * kNdCols + c] = acc;
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < n * kNdCols; e += kNdColThreads) {
    const int r = e / kNdCols, c = e % kNdCols, j = c0 + c;
    if (j >= w) continue;
    if (j < b) d.A[(size_t)r * ld + n + j] = Bt[e];
    else d.inv[(size_t)r * n + (j - b)] = Bt[e];
  }
}

// Batched FP64 GEMM over a device array of descriptors (blockIdx.z), 64 x 64
// tiles, 256 threads with 4 x 4 outputs each; ncols > 0 overrides every
// descriptor's n (the number of right-hand sides of a solve).  Descriptors
// whose problem's gate is closed are skipped.
// Tiles of 16 RM rows (RM = 2, 4) x 16 NC columns (NC = 1..4): a thread
// accumulates RM rows x NC columns, so a solve with few right-hand sides
// computes no padded columns beyond the next multiple of 16, and lists of
// GEMMs with at most 32 rows no padded rows beyond 32.
template <int NC, int RM>
__global__ void __launch_bounds__(256) k_nd_gemm(const NdGemm* __restrict__ ds, int ncols, NdGates gates) {
  constexpr int TN = 16 * NC, TM = 16 * RM;
  const NdGemm g = ds[blockIdx.z];
  const int n = ncols > 0 ? ncols : g.n;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  if (m0 >= g.m || n0 >= n || !gate_open(gates.g[g.q])) return;
  __shared__ double As[16][TM + 1];
  __shared__ double Bs[16][TN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[RM][NC];
#pragma unroll
  for (int r = 0; r < RM; ++r)
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[r][c] = 0.0;
  for (int k0 = 0; k0 < g.k; k0 += 16) {
    for (int idx = threadIdx.x; idx < TM * 16; idx += 256) {
      const int l = idx % 16, i = idx / 16;
      const int gi = m0 + i, gl = k0 + l;
      As[l][i] = (gi < g.m && gl < g.k) ? g.A[(size_t)gi * g.lda + gl] : 0.0;
    }
    for (int idx = threadIdx.x; idx < TN * 16; idx += 256) {
      const int j = idx % TN, l = idx / TN;
      const int gj = n0 + j, gl = k0 + l;
      Bs[l][j] = (gj < n && gl < g.k) ? g.B[(size_t)gl * g.ldb + gj] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < 16; ++l) {
      double a[RM], bb[NC];
#pragma unroll
      for (int r = 0; r < RM; ++r) a[r] = As[l][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < NC; ++c) bb[c] = Bs[l][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[r][c] = fma(a[r], bb[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < RM; ++r) {
    const int gi = m0 + ty + 16 * r;
    if (gi >= g.m) continue;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int gj = n0 + tx + 16 * c;
      if (gj >= n) continue;
      double* cp = g.C + (size_t)gi * g.ldc + gj;
      double v = g.alpha * acc[r][c];
      if (g.beta != 0.0) v += g.beta * *cp;
      *cp = v;
    }
  }
}

// Extend-add of the Schur complements into the parents' fronts (matrices).
__global__ void k_nd_extend(const NdExt* __restrict__ ds) {
  const NdExt d = ds[blockIdx.y];
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)d.b * d.b) return;
  const int i = (int)(e / d.b), j = (int)(e % d.b);
  d.P[(size_t)d.map[i] * d.ldP + d.map[j]] += d.S[(size_t)i * d.ldS + j];
}

// Solve buffers: zu[q] ((M + bsum) x ld), yp[q] (M x ld), elimination order.
struct NdSolvePtrs {
  const double* X[kMaxGemmDescs];
  double* Y[kMaxGemmDescs];
  int r[kMaxGemmDescs];  // right-hand sides of each problem (<= the launch's r)
  double* zu[kMaxGemmDescs];
  double* yp[kMaxGemmDescs];
};

// zu rows 0..M-1 = X rows in elimination order; rows M.. (boundary blocks) = 0
__global__ void k_nd_gather(NdSolvePtrs sp, const int* __restrict__ perm, long M, long rows, int r, int ldx, int ld,
                            NdGates gates) {
  const int q = blockIdx.y;
  if (!gate_open(gates.g[q])) return;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * r) return;
  const long i = e / r;
  const int c = (int)(e % r);
  sp.zu[q][(size_t)i * ld + c] = (i < M && c < sp.r[q]) ? sp.X[q][(size_t)perm[i] * ldx + c] : 0.0;
}

// Y rows = yp rows back in DOF order
__global__ void k_nd_scatter(NdSolvePtrs sp, const int* __restrict__ perm, long M, int r, int ldy, int ld,
                             NdGates gates) {
  const int q = blockIdx.y;
  if (!gate_open(gates.g[q])) return;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * r) return;
  const long i = e / r;
  const int c = (int)(e % r);
  if (c < sp.r[q]) sp.Y[q][(size_t)perm[i] * ldy + c] = sp.yp[q][(size_t)i * ld + c];
}

// A front's boundary block of the solve (b rows of r columns, rows `from` in
// zu) added into the rows pmap[] of zu (the parent's F rows or boundary block).
struct NdVec {
  double* zu; const int* map; long from; int b, q;
};
__global__ void k_nd_vextend(const NdVec* __restrict__ ds, int r, int ld, NdGates gates) {
  const NdVec d = ds[blockIdx.y];
  if (!gate_open(gates.g[d.q])) return;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)d.b * r) return;
  const int i = (int)(e / r), c = (int)(e % r);
  d.zu[(size_t)d.map[i] * ld + c] += d.zu[(size_t)(d.from + i) * ld + c];
}

// Backward sweep: the boundary values x_B of a front (rows brow[] of yp)
// copied into its boundary block of zu.
struct NdBg {
  const double* yp; double* zu; const int* rows; long to; int b, q;
};
__global__ void k_nd_bgather(const NdBg* __restrict__ ds, int r, int ld, NdGates gates) {
  const NdBg d = ds[blockIdx.y];
  if (!gate_open(gates.g[d.q])) return;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)d.b * r) return;
  const int i = (int)(e / r), c = (int)(e % r);
  d.zu[(size_t)(d.to + i) * ld + c] = d.yp[(size_t)d.rows[i] * ld + c];
}

// ---------------------------------------------------------------------------
// numeric phase: drivers
// ---------------------------------------------------------------------------
// Descriptor lists of one factorisation / solve, grouped per height (and per
// child slot for the extend-adds); all live in one device buffer of the
// handle, built once when it is allocated.
struct NdList {
  size_t off = 0;  // byte offset in the descriptor buffer
  int count = 0, m = 0, n = 0, f = 0;  // count; largest m / n (GEMMs), largest f / n (fronts), b (extends)
  double mk = 0;   // GEMM lists: sum of m k over the GEMMs of one problem
};

struct NdPlan {
  std::vector<NdList> fd, schur, ext[2], fwd1, fwd2, vext[2], bg, bwd;  // per height
  DevBuf<unsigned char> buf;
  // the solve GEMMs on the tensor cores (fixed left operands: the inverses,
  // A_BF and W of the fronts, sliced after every factorisation): per height
  // the group of each sweep list, and the FP64 lists of the GEMMs left out
  OzFixedPlan tc;
  bool tc_built = false;
  int tc_sliced = 0;  // problems whose slices match their factors
  std::vector<int> g_fwd1, g_fwd2, g_bwd;
  std::vector<NdList> fwd1s, fwd2s, bwds;
};

int ndlu_status(NdLU& lu, int nprob, std::vector<int>& out, cudaStream_t s) {
  out.assign(nprob, 0);
  LRFSI_CUDA(cudaMemcpyAsync(out.data(), lu.status.p, sizeof(int) * nprob, cudaMemcpyDeviceToHost, s));
  LRFSI_CUDA(cudaStreamSynchronize(s));
  return LRFSI_OK;
}

static int nd_attrs() {
  static bool done = false;
  if (done) return LRFSI_OK;
  LRFSI_CUDA(cudaFuncSetAttribute(k_nd_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kNdSmem));
  LRFSI_CUDA(cudaFuncSetAttribute(k_nd_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kNdSmem));
  LRFSI_CUDA(cudaFuncSetAttribute(k_nd_rhs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kNdSmem));
  done = true;
  return LRFSI_OK;
}

// The mesh's symbolic structure and its device copies (built on first use;
// handles of one mesh may be created from several host threads).
static std::mutex g_nd_mesh_mu;
static int nd_mesh(lrfsi_mesh_s* m) {
  std::lock_guard<std::mutex> lk(g_nd_mesh_mu);
  if (m->nd && m->ndd) return LRFSI_OK;
  auto sym = std::make_shared<NdSymbolic>();
  LRFSI_TRY(nd_symbolic(m->h, *sym));
  auto dv = std::make_shared<NdDevice>();
  LRFSI_TRY(dv->perm.upload(sym->perm));
  LRFSI_TRY(dv->pos.upload(sym->pos));
  LRFSI_TRY(dv->pmap.upload(sym->pmap));
  LRFSI_TRY(dv->fmap.upload(sym->fmap));
  LRFSI_TRY(dv->brow.upload(sym->brow));
  LRFSI_TRY(dv->entry_off.upload(sym->entry_off));
  LRFSI_CUDA(cudaDeviceSynchronize());
  m->nd = sym;
  m->ndd = dv;
  return LRFSI_OK;
}

int ndlu_alloc(lrfsi_mesh_s* m, int nprob, int ld, NdLU& lu) {
  if (nprob < 1 || nprob > kMaxGemmDescs || ld < 1) return fail(LRFSI_EINVAL, "sparse LU: 1..32 problems, ld >= 1");
  LRFSI_TRY(nd_mesh(m));
  LRFSI_TRY(nd_attrs());
  const NdSymbolic& sym = *m->nd;
  const NdDevice& dv = *m->ndd;
  if (sym.maxf > 800) return fail(LRFSI_EINVAL, "sparse LU: separator larger than the panel kernel supports");
  const long M = m->h.M;
  lu.sym = &sym;
  lu.dsym = &dv;
  lu.nprob = nprob;
  lu.ld = ld;
  lu.per_prob = sym.ws_doubles + sym.inv_doubles;
  LRFSI_TRY(lu.ws.alloc(lu.per_prob * nprob));
  LRFSI_TRY(lu.piv.alloc(std::max<size_t>(sym.piv_ints, 1) * nprob));
  LRFSI_TRY(lu.status.alloc(nprob));
  LRFSI_TRY(lu.zero.alloc(1));
  LRFSI_CUDA(cudaMemset(lu.zero.p, 0, sizeof(int)));
  LRFSI_TRY(lu.zu.alloc((size_t)(M + sym.bsum) * ld * nprob));
  LRFSI_TRY(lu.yp.alloc((size_t)M * ld * nprob));
  // the descriptor plan
  auto plan = std::make_shared<NdPlan>();
  const int H = sym.heights;
  std::vector<unsigned char> bytes;
  auto put = [&](const void* p, size_t sz) {
    while (bytes.size() % 16) bytes.push_back(0);
    const size_t o = bytes.size();
    bytes.insert(bytes.end(), (const unsigned char*)p, (const unsigned char*)p + sz);
    return o;
  };
  for (auto* v : {&plan->fd, &plan->schur, &plan->ext[0], &plan->ext[1], &plan->fwd1, &plan->fwd2, &plan->vext[0],
                  &plan->vext[1], &plan->bg, &plan->bwd, &plan->fwd1s, &plan->fwd2s, &plan->bwds})
    v->assign(H, NdList{});
  plan->g_fwd1.assign(H, -1);
  plan->g_fwd2.assign(H, -1);
  plan->g_bwd.assign(H, -1);
  // a sweep GEMM goes to the tensor cores when its left operand is large
  // enough (ozaki_fixed_eligible); the rest stay on the FP64 kernel
  auto split_tc = [&](const std::vector<NdGemm>& all, std::vector<NdGemm>& small, NdList& Ls,
                      std::vector<OzFixedGemm>& tcg) {
    for (const NdGemm& g : all) {
      if (ozaki_fixed_eligible(g.m, g.k)) {
        tcg.push_back(OzFixedGemm{g.A, g.lda, g.m, g.k, g.B, g.ldb, g.C, g.ldc, g.q, g.alpha, g.beta});
      } else {
        small.push_back(g);
        Ls.m = std::max(Ls.m, g.m);
        if (g.q == 0) Ls.mk += (double)g.m * g.k;
      }
    }
  };
  for (int h = 0; h < H; ++h) {
    std::vector<NdFD> fd;
    std::vector<NdGemm> schur, fwd1, fwd2, bwd;
    std::vector<NdExt> ext[2];
    std::vector<NdVec> vext[2];
    std::vector<NdBg> bg;
    NdList L[10];
    for (int q = 0; q < nprob; ++q) {
      double* base = lu.ws.p + lu.per_prob * q;
      double* zu = lu.zu.p + (size_t)(M + sym.bsum) * ld * q;
      double* yp = lu.yp.p + (size_t)M * ld * q;
      for (int t : sym.by_height[h]) {
        const NdFront& fr = sym.fr[t];
        double* A = base + fr.off_front;
        double* inv = base + sym.ws_doubles + fr.off_inv;
        fd.push_back(NdFD{A, inv, lu.piv.p + std::max<size_t>(sym.piv_ints, 1) * q + fr.off_piv, lu.status.p + q,
                          fr.n, fr.f});
        L[0].m = std::max(L[0].m, fr.n);
        L[0].f = std::max(L[0].f, fr.f);
        fwd1.push_back(NdGemm{inv, zu + (size_t)fr.start * ld, yp + (size_t)fr.start * ld, fr.f, 0, fr.f, fr.f, ld,
                              ld, q, 1.0, 0.0});
        L[4].m = std::max(L[4].m, fr.f);
        if (fr.b > 0) {
          schur.push_back(NdGemm{A + (size_t)fr.f * fr.n, A + fr.f, A + (size_t)fr.f * fr.n + fr.f, fr.b, fr.b, fr.f,
                                 fr.n, fr.n, fr.n, q, -1.0, 1.0});
          L[1].m = std::max(L[1].m, fr.b);
          L[1].n = std::max(L[1].n, fr.b);
          double* zb = zu + (size_t)(M + fr.boff) * ld;
          fwd2.push_back(NdGemm{A + (size_t)fr.f * fr.n, yp + (size_t)fr.start * ld, zb, fr.b, 0, fr.f, fr.n, ld, ld,
                                q, -1.0, 1.0});
          L[5].m = std::max(L[5].m, fr.b);
          bg.push_back(NdBg{yp, zu, dv.brow.p + fr.off_map, M + fr.boff, fr.b, q});
          L[8].m = std::max(L[8].m, fr.b);
          bwd.push_back(NdGemm{A + fr.f, zb, yp + (size_t)fr.start * ld, fr.f, 0, fr.b, fr.n, ld, ld, q, -1.0, 1.0});
          L[9].m = std::max(L[9].m, fr.f);
          if (fr.parent >= 0) {
            const NdFront& pf = sym.fr[fr.parent];
            ext[fr.slot].push_back(NdExt{A + (size_t)fr.f * fr.n + fr.f, base + pf.off_front, dv.fmap.p + fr.off_map,
                                         fr.b, fr.n, pf.n, q});
            L[2 + fr.slot].m = std::max(L[2 + fr.slot].m, fr.b);
            vext[fr.slot].push_back(NdVec{zu, dv.pmap.p + fr.off_map, M + fr.boff, fr.b, q});
            L[6 + fr.slot].m = std::max(L[6 + fr.slot].m, fr.b);
          }
        }
      }
    }
    auto stash = [&](NdList& dst, NdList src, const void* p, size_t n, size_t sz) {
      dst = src;
      dst.count = (int)n;
      dst.off = n ? put(p, n * sz) : 0;
    };
    stash(plan->fd[h], L[0], fd.data(), fd.size(), sizeof(NdFD));
    stash(plan->schur[h], L[1], schur.data(), schur.size(), sizeof(NdGemm));
    stash(plan->ext[0][h], L[2], ext[0].data(), ext[0].size(), sizeof(NdExt));
    stash(plan->ext[1][h], L[3], ext[1].data(), ext[1].size(), sizeof(NdExt));
    stash(plan->fwd1[h], L[4], fwd1.data(), fwd1.size(), sizeof(NdGemm));
    stash(plan->fwd2[h], L[5], fwd2.data(), fwd2.size(), sizeof(NdGemm));
    stash(plan->vext[0][h], L[6], vext[0].data(), vext[0].size(), sizeof(NdVec));
    stash(plan->vext[1][h], L[7], vext[1].data(), vext[1].size(), sizeof(NdVec));
    stash(plan->bg[h], L[8], bg.data(), bg.size(), sizeof(NdBg));
    stash(plan->bwd[h], L[9], bwd.data(), bwd.size(), sizeof(NdGemm));
    {
      std::vector<NdGemm> s1, s2, s3;
      std::vector<OzFixedGemm> t1, t2, t3;
      NdList l1, l2, l3;
      split_tc(fwd1, s1, l1, t1);
      split_tc(fwd2, s2, l2, t2);
      split_tc(bwd, s3, l3, t3);
      stash(plan->fwd1s[h], l1, s1.data(), s1.size(), sizeof(NdGemm));
      stash(plan->fwd2s[h], l2, s2.data(), s2.size(), sizeof(NdGemm));
      stash(plan->bwds[h], l3, s3.data(), s3.size(), sizeof(NdGemm));
      if (!t1.empty()) plan->g_fwd1[h] = plan->tc.add_group(t1);
      if (!t2.empty()) plan->g_fwd2[h] = plan->tc.add_group(t2);
      if (!t3.empty()) plan->g_bwd[h] = plan->tc.add_group(t3);
    }
  }
  if (bytes.empty()) bytes.push_back(0);
  LRFSI_TRY(plan->buf.alloc(bytes.size()));
  LRFSI_CUDA(cudaMemcpy(plan->buf.p, bytes.data(), bytes.size(), cudaMemcpyHostToDevice));
  // the tensor-core slices take about twice the bytes of the operands they
  // replace: built only within a quarter of the free device memory
  bool any = false;
  for (int h = 0; h < H; ++h) any = any || plan->g_fwd1[h] >= 0 || plan->g_fwd2[h] >= 0 || plan->g_bwd[h] >= 0;
  if (any) {
    size_t fr = 0, tot = 0;
    LRFSI_CUDA(cudaMemGetInfo(&fr, &tot));
    if (plan->tc.bytes_needed(ld) <= fr / 4) {
      LRFSI_TRY(plan->tc.build(ld, nprob));
      plan->tc_built = true;
    }
  }
  lu.plan = plan;
  return LRFSI_OK;
}

static int nd_gemm_launch(const NdPlan& pl, const NdList& L, int ncols, int nmax, const NdGates& gates, cudaStream_t s) {
  if (!L.count) return LRFSI_OK;
  const int nn = ncols > 0 ? ncols : nmax;
  const NdGemm* ds = reinterpret_cast<const NdGemm*>(pl.buf.p + L.off);
  // tile width: the next multiple of 16 up to 64 columns; 32 rows when no
  // GEMM of the list has more
  const int nc = nn >= 64 ? 4 : (nn + 15) / 16;
  const int rm = L.m <= 32 ? 2 : 4;
  dim3 grid(ceil_div(nn, 16 * nc), ceil_div(L.m, 16 * rm), L.count);
  switch (nc + 4 * (rm == 2)) {
    case 1: k_nd_gemm<1, 4><<<grid, 256, 0, s>>>(ds, ncols, gates); break;
    case 2: k_nd_gemm<2, 4><<<grid, 256, 0, s>>>(ds, ncols, gates); break;
    case 3: k_nd_gemm<3, 4><<<grid, 256, 0, s>>>(ds, ncols, gates); break;
    case 4: k_nd_gemm<4, 4><<<grid, 256, 0, s>>>(ds, ncols, gates); break;
    case 5: k_nd_gemm<1, 2><<<grid, 256, 0, s>>>(ds, ncols, gates); break;
    case 6: k_nd_gemm<2, 2><<<grid, 256, 0, s>>>(ds, ncols, gates); break;
    case 7: k_nd_gemm<3, 2><<<grid, 256, 0, s>>>(ds, ncols, gates); break;
    default: k_nd_gemm<4, 2><<<grid, 256, 0, s>>>(ds, ncols, gates); break;
  }
  return check_launch("k_nd_gemm");
}

int ndlu_factor(const lrfsi_mesh_s* m, NdLU& lu, const double* const* J3, const double* alpha, const double* beta,
                int nprob, cudaStream_t s) {
  if (nprob > lu.nprob || !lu.plan) return fail(LRFSI_EINVAL, "sparse LU: more problems than allocated");
  const NdSymbolic& sym = *lu.sym;
  const NdPlan& pl = *lu.plan;
  NdProbs pp{};
  for (int q = 0; q < nprob; ++q) {
    pp.ws[q] = lu.ws.p + lu.per_prob * q;
    pp.J3[q] = J3[q];
    pp.alpha[q] = alpha[q];
    pp.beta[q] = beta[q];
    LRFSI_CUDA(cudaMemsetAsync(pp.ws[q], 0, sizeof(double) * sym.ws_doubles, s));
  }
  LRFSI_CUDA(cudaMemsetAsync(lu.status.p, 0, sizeof(int) * nprob, s));
  TimedLaunch tl_all(KC_LU, s);
  const long nnz = (long)m->h.colidx.size();
  k_nd_extract<<<dim3(ceil_div(nnz, 256), nprob), 256, 0, s>>>(pp, lu.dsym->entry_off.p, nnz);
  LRFSI_TRY(check_launch("k_nd_extract"));
  NdGates open{};
  // the plan holds lu.nprob problems per height; factor the first nprob of them
  for (int h = 0; h < sym.heights; ++h) {
    const NdList& F = pl.fd[h];
    const int cnt = (int)((long)F.count * nprob / lu.nprob);
    if (!cnt) continue;
    const NdFD* fd = reinterpret_cast<const NdFD*>(pl.buf.p + F.off);
    int nbp = kNdNb;
    while (nbp > 8 && (size_t)F.f * (nbp + 1) * sizeof(double) > kNdSmem) nbp /= 2;
    for (int j0 = 0; j0 < F.f; j0 += nbp) {
      const int nb = std::min(nbp, F.f - j0);
      {
        account(KC_LUPANEL, 0, 0);
        TimedLaunch tk(KC_LUPANEL, s);
        k_nd_panel<<<cnt, kNdPanelThreads, sizeof(double) * (size_t)(F.f - j0) * (nbp + 1), s>>>(fd, j0, nbp);
        LRFSI_TRY(check_launch("k_nd_panel"));
        tk.end(s);
      }
      const int ncols = ceil_div(j0, kNdCols) + ceil_div(F.f - j0 - nb, kNdCols);
      if (ncols > 0) {
        account(KC_LUTRSM, 0, 0);
        TimedLaunch tk(KC_LUTRSM, s);
        const size_t smem = sizeof(double) * ((size_t)(F.f - j0) * kNdCols + 32 * 33) + sizeof(int) * (size_t)(F.f - j0);
        k_nd_update<<<dim3(ncols, cnt), kNdColThreads, smem, s>>>(fd, j0, nbp);
        LRFSI_TRY(check_launch("k_nd_update"));
        tk.end(s);
      }
    }
    {
      account(KC_LUTRSM, 0, 0);
      TimedLaunch tk(KC_LUTRSM, s);
      const size_t smem = sizeof(double) * ((size_t)F.f * kNdCols + 32 * 33) + sizeof(int) * (size_t)F.f;
      k_nd_rhs<<<dim3(ceil_div(F.m, kNdCols), cnt), kNdColThreads, smem, s>>>(fd);
      LRFSI_TRY(check_launch("k_nd_rhs"));
      tk.end(s);
    }
    const NdList& Sl = pl.schur[h];
    if (Sl.count) {
      NdList part = Sl;
      part.count = (int)((long)Sl.count * nprob / lu.nprob);
      if (part.count) {
        double fl = 0;
        for (int t : sym.by_height[h]) fl += 2.0 * sym.fr[t].b * sym.fr[t].b * sym.fr[t].f;
        account(KC_GEMM, fl * nprob, 0);
        TimedLaunch tk(KC_GEMM, s);
        LRFSI_TRY(nd_gemm_launch(pl, part, 0, Sl.n, open, s));
        tk.end(s);
      }
    }
    for (int slot = 0; slot < 2; ++slot) {
      const NdList& E = pl.ext[slot][h];
      const int ec = (int)((long)E.count * nprob / lu.nprob);
      if (!ec) continue;
      k_nd_extend<<<dim3(ceil_div((long)E.m * E.m, 256), ec), 256, 0, s>>>(
          reinterpret_cast<const NdExt*>(pl.buf.p + E.off));
      LRFSI_TRY(check_launch("k_nd_extend"));
    }
  }
  NdPlan& plw = *lu.plan;
  plw.tc_sliced = 0;
  if (plw.tc_built && gram_path() == 1) {
    LRFSI_TRY(plw.tc.slice(nprob, s));
    plw.tc_sliced = nprob;
  }
  account(KC_LU, sym.factor_flops * nprob, 0);
  tl_all.end(s);
  return LRFSI_OK;
}

int ndlu_solve(NdLU& lu, double* const* X, double* const* Y, const int* r, int ld, int nprob, cudaStream_t s,
               const Gate* gates) {
  if (nprob > lu.nprob || !lu.plan) return fail(LRFSI_EINVAL, "sparse LU solve: more problems than allocated");
  const NdSymbolic& sym = *lu.sym;
  const NdPlan& pl = *lu.plan;
  const long M = (long)sym.perm.size();
  int rmax = 0;
  NdSolvePtrs sp{};
  NdGates g{};
  int closed[kMaxGemmDescs];
  for (int q = 0; q < nprob; ++q) {
    if (r[q] < 0 || r[q] > lu.ld || (r[q] > 0 && r[q] > ld)) return fail(LRFSI_EINVAL, "sparse LU solve: r_q");
    rmax = std::max(rmax, r[q]);
    sp.X[q] = X[q];
    sp.Y[q] = Y[q];
    sp.r[q] = r[q];
    sp.zu[q] = lu.zu.p + (size_t)(M + sym.bsum) * lu.ld * q;
    sp.yp[q] = lu.yp.p + (size_t)M * lu.ld * q;
    g.g[q] = gates ? gates[q] : Gate{};
    closed[q] = r[q] == 0;
  }
  if (rmax == 0) return LRFSI_OK;
  // problems without columns: gated off with a device flag that is always zero
  {
    bool any_closed = false;
    for (int q = 0; q < nprob; ++q) any_closed = any_closed || closed[q];
    if (any_closed)
      for (int q = 0; q < nprob; ++q)
        if (closed[q]) g.g[q] = Gate{lu.zero.p, nullptr};
  }
  TimedLaunch tl_all(KC_LUSOLVE, s);
  const int ldl = lu.ld;
  k_nd_gather<<<dim3(ceil_div((M + sym.bsum) * rmax, 256), nprob), 256, 0, s>>>(
      sp, lu.dsym->perm.p, M, M + sym.bsum, rmax, ld, ldl, g);
  LRFSI_TRY(check_launch("k_nd_gather"));
  auto part = [&](const NdList& L) {
    NdList p = L;
    p.count = (int)((long)L.count * nprob / lu.nprob);
    return p;
  };
  double fl = 0;
  for (int h = 0; h < sym.heights; ++h) {
    for (int t : sym.by_height[h]) {
      const double f = sym.fr[t].f, b = sym.fr[t].b;
      fl += 2.0 * rmax * (f * f + 2.0 * f * b);
    }
  }
  // the sweep GEMMs: on the tensor cores where their slices are current (the
  // rest on the FP64 kernel), else all on the FP64 kernel
  // (a few right-hand sides: the FP64 kernel reads half the bytes)
  const bool tc = pl.tc_built && gram_path() == 1 && nprob <= pl.tc_sliced && rmax >= 8;
  int live = 0;
  for (int q = 0; q < nprob; ++q) live += (r[q] > 0 && gate_counts(g.g[q], s)) ? 1 : 0;
  if (!tc) account(KC_GEMM, fl * live, 0);
  auto sweep = [&](const std::vector<NdList>& all, const std::vector<NdList>& small, const std::vector<int>& grp,
                   int h) -> int {
    const NdList L = part(tc ? small[h] : all[h]);
    if (L.count) {
      if (tc) account(KC_GEMM, 2.0 * rmax * small[h].mk * live, 0);
      TimedLaunch tk(KC_GEMM, s);
      LRFSI_TRY(nd_gemm_launch(pl, L, rmax, rmax, g, s));
      tk.end(s);
    }
    return tc ? pl.tc.gemm(grp[h], rmax, nprob, g, s) : LRFSI_OK;
  };
  for (int h = 0; h < sym.heights; ++h) {  // forward: y_F = A_FF^{-1} z_F, z_B -= A_BF y_F, z_B to the parent
    LRFSI_TRY(sweep(pl.fwd1, pl.fwd1s, pl.g_fwd1, h));
    LRFSI_TRY(sweep(pl.fwd2, pl.fwd2s, pl.g_fwd2, h));
    for (int slot = 0; slot < 2; ++slot) {
      const NdList V = part(pl.vext[slot][h]);
      if (!V.count) continue;
      k_nd_vextend<<<dim3(ceil_div((long)V.m * rmax, 256), V.count), 256, 0, s>>>(
          reinterpret_cast<const NdVec*>(pl.buf.p + V.off), rmax, ldl, g);
      LRFSI_TRY(check_launch("k_nd_vextend"));
    }
  }
  for (int h = sym.heights - 1; h >= 0; --h) {  // backward: x_F = y_F - W x_B
    const NdList B = part(pl.bg[h]);
    if (B.count) {
      k_nd_bgather<<<dim3(ceil_div((long)B.m * rmax, 256), B.count), 256, 0, s>>>(
          reinterpret_cast<const NdBg*>(pl.buf.p + B.off), rmax, ldl, g);
      LRFSI_TRY(check_launch("k_nd_bgather"));
    }
    LRFSI_TRY(sweep(pl.bwd, pl.bwds, pl.g_bwd, h));
  }
  k_nd_scatter<<<dim3(ceil_div(M * rmax, 256), nprob), 256, 0, s>>>(sp, lu.dsym->perm.p, M, rmax, ld, ldl, g);
  LRFSI_TRY(check_launch("k_nd_scatter"));
  tl_all.end(s);
  return LRFSI_OK;
}

}  // namespace lrfsi
