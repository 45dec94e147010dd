// SpMM of the affine operators and the block-tridiagonal FP64 LU used for the
// mean-based preconditioner P_T^k = J(x~; mu_bar, nu_bar) (Sec. 4.2; the
// paper factors it with a permuted LU) and for the median Newton solves
// (Sec. 3.2).
//
// Fill-reducing ordering: the slab-major DOF order makes every operator block
// tridiagonal over the nx + 1 slabs of the channel, so the LU fills only the
// diagonal, first super- and first sub-diagonal blocks (block Thomas
// elimination).  Pivoting is partial pivoting inside each diagonal Schur
// block; its pivot threshold is reported through the status word.
#include <cmath>
#include <mutex>

#include "sparse_lu.h"

namespace lrfsi {

// ---------------------------------------------------------------------------
// SpMM: LPR lanes per row (256 / LPR rows per CTA), each lane CPL columns of
// U per pass; the (LPR, CPL) shape per precision and rank is picked by timing
// (spmm_variant below)
// ---------------------------------------------------------------------------
template <class T>
struct SpmmBatch {
  SpmmDesc<T> d[kMaxGemmDescs];
};

template <class T, int LPR, int CPL>
__global__ void __launch_bounds__(256) k_spmm(SpmmBatch<T> sb, const int* __restrict__ rowptr,
                                               const int* __restrict__ colidx, long M) {
  // The LPR lanes of a row load up to LPR nonzeros (index and the three
  // values) with one coalesced access and pass them around with shuffles, so
  // that the gathers of U rows for several nonzeros are in flight at once.
  // Trip counts are made uniform over the warp (rows of one warp differ in
  // length); lanes past their row's end only skip the arithmetic.
  const SpmmDesc<T>& dref = sb.d[blockIdx.y];
  if (!gate_open(dref.gate)) return;
  constexpr int RPB = 256 / LPR;
  const long row0 = (long)blockIdx.x * RPB + (threadIdx.x / LPR);
  const int lane = threadIdx.x % LPR;
  const bool valid = row0 < M;
  const long row = valid ? row0 : M - 1;
  const int r = dref.r;
  const T* __restrict__ U = dref.U;
  const T* __restrict__ J3 = dref.J3;
  const int ldu = dref.ldu;
  const bool combined = dref.o[1] < 0;
  const T a1 = dref.a1, a2 = dref.a2;
  const int k0 = rowptr[row], k1 = valid ? rowptr[row + 1] : k0;
  int nch = (k1 - k0 + LPR - 1) / LPR;
#pragma unroll
  for (int o = LPR; o < 32; o <<= 1) nch = max(nch, __shfl_xor_sync(0xffffffffu, nch, o));
  for (int c0 = 0; c0 < r; c0 += LPR * CPL) {
    T acc0[CPL], acc1[CPL], acc2[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) acc0[q] = acc1[q] = acc2[q] = T(0);
    for (int ch = 0; ch < nch; ++ch) {
      const int kb = k0 + ch * LPR, kk = kb + lane;
      const bool have = kk < k1;
      const int mc = have ? colidx[kk] : 0;
      const T w0 = have ? J3[3 * (size_t)kk] : T(0);
      const T w1 = have ? J3[3 * (size_t)kk + 1] : T(0);
      const T w2 = have ? J3[3 * (size_t)kk + 2] : T(0);
      const int nk = k1 - kb;
#pragma unroll 8
      for (int t = 0; t < LPR; ++t) {
        const int col = __shfl_sync(0xffffffffu, mc, t, LPR);
        const T v0 = __shfl_sync(0xffffffffu, w0, t, LPR);
        const T v1 = __shfl_sync(0xffffffffu, w1, t, LPR);
        const T v2 = __shfl_sync(0xffffffffu, w2, t, LPR);
        if (t < nk) {
          const T* ur = U + (size_t)col * ldu;
#pragma unroll
          for (int q = 0; q < CPL; ++q) {
            const int j = c0 + lane + LPR * q;
            if (j < r) {
              const T u = ur[j];
              if (combined) {
                acc0[q] += (v0 + a1 * v1 + a2 * v2) * u;
              } else {
                acc0[q] += v0 * u; acc1[q] += v1 * u; acc2[q] += v2 * u;
              }
            }
          }
        }
      }
    }
    if (valid) {
      T* yr = dref.Y + (size_t)row * dref.ldy;
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        const int j = c0 + lane + LPR * q;
        if (j < r) {
          yr[dref.o[0] + j] = dref.sc[0] * acc0[q];
          if (!combined) {
            yr[dref.o[1] + j] = dref.sc[1] * acc1[q];
            yr[dref.o[2] + j] = dref.sc[2] * acc2[q];
          }
        }
      }
    }
  }
}

// Windowed SpMM: CTA b takes rows [128 b, 128 b + 128) and first stages the
// rows of U its nonzeros touch (the column window of the row block; the slab
// ordering keeps it to about three slabs) in shared memory, in chunks of rc
// columns; the gathers then read shared memory.  LPR lanes per row, CPL
// columns per lane per pass.
template <class T, int LPR, int CPL>
__global__ void __launch_bounds__(256) k_spmm_win(SpmmBatch<T> sb, const int* __restrict__ rowptr,
                                                   const int* __restrict__ colidx, const int* __restrict__ win,
                                                   long M, int rc) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Us = reinterpret_cast<T*>(smraw);
  const SpmmDesc<T>& dref = sb.d[blockIdx.y];
  if (!gate_open(dref.gate)) return;
  const long rb0 = (long)blockIdx.x * kSpmmRowBlock;
  const int w0 = win[2 * blockIdx.x], w1 = win[2 * blockIdx.x + 1];
  const int wl = w1 - w0;
  const int r = dref.r, ldu = dref.ldu;
  const T* __restrict__ U = dref.U;
  const T* __restrict__ J3 = dref.J3;
  const bool combined = dref.o[1] < 0;
  const T a1 = dref.a1, a2 = dref.a2;
  const int lane = threadIdx.x % LPR, grp = threadIdx.x / LPR;
  constexpr int GROUPS = 256 / LPR;
  for (int cb = 0; cb < r; cb += rc) {
    const int nc = r - cb < rc ? r - cb : rc;
    __syncthreads();  // the previous chunk's gathers are done
    for (long e = threadIdx.x; e < (long)wl * nc; e += 256) {
      const int i = (int)(e / nc), c = (int)(e % nc);
      Us[e] = U[(size_t)(w0 + i) * ldu + cb + c];
    }
    __syncthreads();
    for (int rr = grp; rr < kSpmmRowBlock; rr += GROUPS) {
      const long row = rb0 + rr;
      if (row >= M) break;
      const int k0 = rowptr[row], k1 = rowptr[row + 1];
      for (int c0 = 0; c0 < nc; c0 += LPR * CPL) {
        T acc0[CPL], acc1[CPL], acc2[CPL];
#pragma unroll
        for (int q = 0; q < CPL; ++q) acc0[q] = acc1[q] = acc2[q] = T(0);
        for (int k = k0; k < k1; ++k) {
          const T* ur = Us + (size_t)(colidx[k] - w0) * nc;
          const T v0 = J3[3 * (size_t)k], v1 = J3[3 * (size_t)k + 1], v2 = J3[3 * (size_t)k + 2];
#pragma unroll
          for (int q = 0; q < CPL; ++q) {
            const int j = c0 + lane + LPR * q;
            if (j < nc) {
              const T u = ur[j];
              if (combined) {
                acc0[q] += (v0 + a1 * v1 + a2 * v2) * u;
              } else {
                acc0[q] += v0 * u; acc1[q] += v1 * u; acc2[q] += v2 * u;
              }
            }
          }
        }
        T* yr = dref.Y + (size_t)row * dref.ldy + cb;
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
          const int j = c0 + lane + LPR * q;
          if (j < nc) {
            yr[dref.o[0] + j] = dref.sc[0] * acc0[q];
            if (!combined) {
              yr[dref.o[1] + j] = dref.sc[1] * acc1[q];
              yr[dref.o[2] + j] = dref.sc[2] * acc2[q];
            }
          }
        }
      }
    }
  }
}

// The candidate shapes: lanes per row x columns per lane, U gathered from
// L2 (0-5) or from the shared-memory window (6-8).
constexpr int kSpmmVariants = 9;
constexpr size_t kSpmmWinSmem = 200 * 1024;
template <class T>
static int spmm_window_cols(const lrfsi_mesh_s* m, int rmax) {
  const long per_col = (long)m->spmm_winmax * (long)sizeof(T);
  if (per_col <= 0) return 0;
  int rc = (int)((long)kSpmmWinSmem / per_col);
  return rc < rmax ? rc : rmax;
}
template <class T>
static void spmm_launch(int v, const lrfsi_mesh_s* m, int cnt, int rmax, const SpmmBatch<T>& sb, cudaStream_t s) {
  const int* rp = m->rowptr.p;
  const int* ci = m->colidx.p;
  const long M = m->h.M;
  auto g = [&](int rpb) { return dim3(ceil_div(M, rpb), cnt); };
  if (v >= 6) {
    const int rc = spmm_window_cols<T>(m, rmax);
    const size_t smem = (size_t)m->spmm_winmax * rc * sizeof(T);
    const dim3 gw(ceil_div(M, kSpmmRowBlock), cnt);
    switch (v) {
      case 6: k_spmm_win<T, 32, 2><<<gw, 256, smem, s>>>(sb, rp, ci, m->spmm_win.p, M, rc); break;
      case 7: k_spmm_win<T, 16, 4><<<gw, 256, smem, s>>>(sb, rp, ci, m->spmm_win.p, M, rc); break;
      default: k_spmm_win<T, 8, 8><<<gw, 256, smem, s>>>(sb, rp, ci, m->spmm_win.p, M, rc); break;
    }
    return;
  }
  switch (v) {
    case 0: k_spmm<T, 32, 1><<<g(8), 256, 0, s>>>(sb, rp, ci, M); break;
    case 1: k_spmm<T, 32, 2><<<g(8), 256, 0, s>>>(sb, rp, ci, M); break;
    case 2: k_spmm<T, 16, 2><<<g(16), 256, 0, s>>>(sb, rp, ci, M); break;
    case 3: k_spmm<T, 16, 4><<<g(16), 256, 0, s>>>(sb, rp, ci, M); break;
    case 4: k_spmm<T, 8, 4><<<g(32), 256, 0, s>>>(sb, rp, ci, M); break;
    default: k_spmm<T, 8, 8><<<g(32), 256, 0, s>>>(sb, rp, ci, M); break;
  }
}

static int spmm_win_attrs() {
  static bool done = false;
  if (done) return LRFSI_OK;
  LRFSI_CUDA(cudaFuncSetAttribute(k_spmm_win<double, 32, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSpmmWinSmem));
  LRFSI_CUDA(cudaFuncSetAttribute(k_spmm_win<double, 16, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSpmmWinSmem));
  LRFSI_CUDA(cudaFuncSetAttribute(k_spmm_win<double, 8, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSpmmWinSmem));
  LRFSI_CUDA(cudaFuncSetAttribute(k_spmm_win<float, 32, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSpmmWinSmem));
  LRFSI_CUDA(cudaFuncSetAttribute(k_spmm_win<float, 16, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSpmmWinSmem));
  LRFSI_CUDA(cudaFuncSetAttribute(k_spmm_win<float, 8, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSpmmWinSmem));
  done = true;
  return LRFSI_OK;
}

// Autotuner: on the first batch of a given (precision, rank bucket) every
// shape is timed (CUDA events on the launching stream, best of 3 after one
// warm-up run) and the fastest is kept for the process.  The timed runs
// compute the same outputs, so the batch's result is unaffected.
struct SpmmChoice {
  int v = -1;
  float ms[kSpmmVariants] = {0};
};
static std::mutex g_spmm_mu;
static SpmmChoice g_spmm_choice[2][9];  // [FP64, FP32][rank bucket: ceil(rmax / 16), capped]

static int spmm_bucket(int rmax) {
  const int b = (rmax + 15) / 16;
  return b < 8 ? b : 8;
}

template <class T>
static int spmm_variant(const SpmmBatch<T>& sb, int cnt, int rmax, const lrfsi_mesh_s* m, cudaStream_t s) {
  const int pi = sizeof(T) == 8 ? 0 : 1, bk = spmm_bucket(rmax);
  {
    std::lock_guard<std::mutex> lk(g_spmm_mu);
    if (g_spmm_choice[pi][bk].v >= 0) return g_spmm_choice[pi][bk].v;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
    return rmax <= 32 ? 0 : 1;  // no timing while a stream is being captured
  cudaEvent_t e0, e1;
  LRFSI_CUDA(cudaEventCreate(&e0));
  LRFSI_CUDA(cudaEventCreate(&e1));
  SpmmChoice ch;
  float best = 1e30f;
  LRFSI_TRY(spmm_win_attrs());
  const bool win_ok = spmm_window_cols<T>(m, rmax) >= 1;
  for (int v = 0; v < kSpmmVariants; ++v) {
    float bv = 1e30f;
    if (v >= 6 && !win_ok) { ch.ms[v] = 0; continue; }
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(e0, s);
      spmm_launch<T>(v, m, cnt, rmax, sb, s);
      cudaEventRecord(e1, s);
      LRFSI_TRY(check_launch("k_spmm (autotune)"));
      LRFSI_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < bv) bv = ms;
    }
    ch.ms[v] = bv;
    if (bv < best) { best = bv; ch.v = v; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_spmm_mu);
  g_spmm_choice[pi][bk] = ch;
  return ch.v;
}

template <class T>
int spmm_batched(const lrfsi_mesh_s* m, const SpmmDesc<T>* d, int n, cudaStream_t s) {
  const long M = m->h.M;
  for (int i = 0; i < n;) {  // chunks of up to kMaxGemmDescs non-empty products
    SpmmBatch<T> sb;
    int cnt = 0, rmax = 0;
    for (; i < n && cnt < kMaxGemmDescs; ++i) {
      if (d[i].r <= 0) continue;
      sb.d[cnt++] = d[i];
      rmax = rmax > d[i].r ? rmax : d[i].r;
    }
    if (!cnt) continue;
    const int v = spmm_variant<T>(sb, cnt, rmax, m, s);
    {
      // algorithmic: CSR index + 3 value arrays once, U gathered once per row
      // of the pattern (L2-resident reuse not counted), outputs written once
      const double nnz = (double)m->h.colidx.size();
      double fl = 0, by = 0;
      for (int q = 0; q < cnt; ++q) {
        if (!gate_counts(sb.d[q].gate, s)) continue;
        const bool comb = sb.d[q].o[1] < 0;
        fl += nnz * sb.d[q].r * (comb ? 2.0 : 6.0);
        by += nnz * (4.0 + 3.0 * sizeof(T)) + 4.0 * (M + 1) + (double)M * sb.d[q].r * sizeof(T) * (comb ? 2.0 : 4.0);
      }
      account(sizeof(T) == 8 ? KC_SPMM : KC_SPMM32, fl, by);
    }
    TimedLaunch tl(sizeof(T) == 8 ? KC_SPMM : KC_SPMM32, s);
    spmm_launch<T>(v, m, cnt, rmax, sb, s);
    LRFSI_TRY(check_launch("k_spmm"));
    tl.end(s);
  }
  return LRFSI_OK;
}

int spmm_autotune_table(int precision, int bucket, int* variant, float* ms) {
  if (precision < 0 || precision > 1 || bucket < 0 || bucket > 8) return LRFSI_EINVAL;
  std::lock_guard<std::mutex> lk(g_spmm_mu);
  *variant = g_spmm_choice[precision][bucket].v;
  for (int v = 0; v < kSpmmVariants; ++v) ms[v] = g_spmm_choice[precision][bucket].ms[v];
  return LRFSI_OK;
}
template int spmm_batched<double>(const lrfsi_mesh_s*, const SpmmDesc<double>*, int, cudaStream_t);
template int spmm_batched<float>(const lrfsi_mesh_s*, const SpmmDesc<float>*, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Block LU
// ---------------------------------------------------------------------------
constexpr int kNb = 32;  // panel width

struct ProbPtrs {
  double* ws[kMaxGemmDescs];
  const double* J3[kMaxGemmDescs];
  int* piv[kMaxGemmDescs];
  int* status[kMaxGemmDescs];
  double alpha[kMaxGemmDescs], beta[kMaxGemmDescs];
  const double* b[kMaxGemmDescs];  // single-solve mode: right-hand side (stride ldb)
  double* y[kMaxGemmDescs];        // single-solve mode: solution (stride ldb)
  int ldb;
};

__global__ void k_lu_extract(ProbPtrs pp, const long long* __restrict__ dense_off, long nnz) {
  const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  const int b = blockIdx.y;
  const double* J = pp.J3[b];
  pp.ws[b][dense_off[k]] = J[3 * k] + pp.alpha[b] * J[3 * k + 1] + pp.beta[b] * J[3 * k + 2];
}

// Right-hand side of slab s (n rows, width w): RHS = [Up_s | I] (w = n_next + n,
// the inverse is kept) or, in single-solve mode, [Up_s | b_s] (w = n_next + 1).
__global__ void k_lu_rhs(ProbPtrs pp, size_t off_up_s, size_t off_rhs, int n, int nnext, int nmax, int w, long o,
                         int single) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)n * w) return;
  const int i = (int)(e / w), j = (int)(e % w);
  double* R = pp.ws[blockIdx.y] + off_rhs;
  double v;
  if (j < nnext) v = pp.ws[blockIdx.y][off_up_s + (size_t)i * nmax + j];
  else if (single) v = pp.b[blockIdx.y][(size_t)(o + i) * pp.ldb];
  else v = (j - nnext == i) ? 1.0 : 0.0;
  R[(size_t)i * w + j] = v;
}

// Panel factorization with partial pivoting of columns [j0, j0 + nb) of the
// n x n block A (ld) (rows j0..n-1); pivots are absolute row indices.  The
// panel ((n - j0) x nb) is staged in shared memory.  Two barriers per column:
// the search for the next pivot is fused into the rank-1 update (each thread
// tracks the largest |entry| of the next column among its rows, warps reduce
// with shuffles), and every thread finishes the reduction over the warps'
// candidates itself.  Ties go to the smallest row.
constexpr int kPanelSmem = 220 * 1024;  // dynamic shared memory for the staged panel
constexpr int kPanelThreads = 256;
// Candidates are compared as the bit patterns of |x| (unsigned integers order
// non-negative doubles like their values), which keeps the search off the
// FP64 pipe; a NaN compares above every number and is flagged as singular.
__device__ __forceinline__ unsigned long long abs_key(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
}
__device__ __forceinline__ void argmax_merge(unsigned long long& v, int& i, unsigned long long v2, int i2) {
  if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
}
__global__ void __launch_bounds__(kPanelThreads) k_lu_panel(ProbPtrs pp, size_t off_blk, int piv_off, int n, int ld,
                                                            int j0, int nb) {
  constexpr int kWarps = kPanelThreads / 32;
  const int b = blockIdx.x;
  double* A = pp.ws[b] + off_blk;
  int* piv = pp.piv[b] + piv_off;
  extern __shared__ double sp[];  // (n - j0) x nb, row-major with stride nb + 1 (no bank conflicts)
  __shared__ unsigned long long s_val[kWarps];
  __shared__ int s_idx[kWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rows = n - j0, sl = nb + 1;
  for (long e = tid; e < (long)rows * nb; e += kPanelThreads) {
    const int i = (int)(e / nb), c = (int)(e % nb);
    sp[(size_t)i * sl + c] = A[(size_t)(j0 + i) * ld + j0 + c];
  }
  __syncthreads();
  auto warp_argmax = [&](unsigned long long best, int bi) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v2 = __shfl_xor_sync(0xffffffffu, best, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      argmax_merge(best, bi, v2, i2);
    }
    if (lane == 0) { s_val[warp] = best; s_idx[warp] = bi; }
  };
  {  // candidates for column 0
    unsigned long long best = 0;
    int bi = 0x7fffffff;
    for (int i = tid; i < rows; i += kPanelThreads) argmax_merge(best, bi, abs_key(sp[(size_t)i * sl]), i);
    warp_argmax(best, bi);
  }
  __syncthreads();
  for (int jj = 0; jj < nb; ++jj) {
    unsigned long long pk = 0;
    int pr = 0x7fffffff;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) argmax_merge(pk, pr, s_val[w], s_idx[w]);
    double pv = __longlong_as_double((long long)pk);
    if (pr >= rows) { pr = jj; pv = 0.0; }
    if (tid == 0) {
      piv[j0 + jj] = j0 + pr;
      if (!(pv > 0.0)) *pp.status[b] = LRFSI_ESINGULAR;
    }
    if (pr != jj)
      for (int c = tid; c < nb; c += kPanelThreads) {
        const double t = sp[(size_t)jj * sl + c];
        sp[(size_t)jj * sl + c] = sp[(size_t)pr * sl + c];
        sp[(size_t)pr * sl + c] = t;
      }
    __syncthreads();
    const double* rj = sp + (size_t)jj * sl;
    double dgn = rj[jj];
    if (dgn == 0.0) dgn = 1e-300;  // singular: flagged above, keep going without NaNs
    const double inv = 1.0 / dgn;
    const int w = nb - jj - 1;
    unsigned long long best = 0;
    int bi = 0x7fffffff;
    for (int i = jj + 1 + tid; i < rows; i += kPanelThreads) {
      double* ri = sp + (size_t)i * sl;
      const double l = ri[jj] * inv;
      ri[jj] = l;
      for (int c = 0; c < w; ++c) ri[jj + 1 + c] = fma(-l, rj[jj + 1 + c], ri[jj + 1 + c]);
      if (w > 0) argmax_merge(best, bi, abs_key(ri[jj + 1]), i);
    }
    warp_argmax(best, bi);
    __syncthreads();
  }
  for (long e = tid; e < (long)rows * nb; e += kPanelThreads) {
    const int i = (int)(e / nb), c = (int)(e % nb);
    A[(size_t)(j0 + i) * ld + j0 + c] = sp[(size_t)i * sl + c];
  }
}



constexpr int kRhsCols = 8;      // columns per CTA of the column-parallel kernels
constexpr int kRhsThreads = 512;
// After the panel [j0, j0 + nb) of the slab block A (n x n, ld) is factored:
// the row interchanges of the panel applied to every other column, then for
// the columns right of the panel U12 = L11^{-1} A12 and A22 -= L21 U12.  The
// columns are independent: CTA t takes 8 columns (the first ceil(j0 / 8) CTAs
// the columns left of the panel, which only take the interchanges), stages
// rows [j0, n) of its columns in shared memory, one warp solves the unit lower
// diagonal block (four lanes per column) and all threads update the rows below.
__global__ void __launch_bounds__(kRhsThreads) k_lu_panel_update(ProbPtrs pp, size_t off_lu, int ld, int piv_off, int n,
                                                                 int j0, int nb) {
  extern __shared__ double usm[];
  const int q = blockIdx.y;
  double* A = pp.ws[q] + off_lu;
  const int* piv = pp.piv[q] + piv_off;
  const int nleft = (j0 + kRhsCols - 1) / kRhsCols;
  const bool left = (int)blockIdx.x < nleft;
  const int cb = left ? blockIdx.x * kRhsCols : j0 + nb + (blockIdx.x - nleft) * kRhsCols;
  const int ce = left ? min(cb + kRhsCols, j0) : min(cb + kRhsCols, n);
  const int tid = threadIdx.x;
  if (left) {  // interchanges only
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
  double* Bt = usm;                                  // rows x 8 tile (rows j0..n-1)
  double* Ls = usm + (size_t)rows * kRhsCols;        // 32 x 33: L11
  int* idx = reinterpret_cast<int*>(Ls + 32 * 33);   // row permutation of rows j0..n-1
  if (tid == 0) {
    for (int i = 0; i < rows; ++i) idx[i] = i;
    for (int j = j0; j < j0 + nb; ++j) {
      const int p = piv[j];
      if (p != j && p >= j0 && p < n) { const int t = idx[j - j0]; idx[j - j0] = idx[p - j0]; idx[p - j0] = t; }
    }
  }
  for (int e = tid; e < 32 * 32; e += kRhsThreads) {
    const int i = e >> 5, l = e & 31;
    Ls[i * 33 + l] = (i < nb && l < nb) ? A[(size_t)(j0 + i) * ld + j0 + l] : 0.0;
  }
  __syncthreads();
  for (int e = tid; e < rows * kRhsCols; e += kRhsThreads) {
    const int r = e / kRhsCols, c = e % kRhsCols;
    Bt[e] = cb + c < ce ? A[(size_t)(j0 + idx[r]) * ld + cb + c] : 0.0;
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  if (warp == 0) {  // U12 = L11^{-1} A12 (unit lower)
    const int lq = lane & 3, lbase = lane & ~3, lc = lane >> 2;
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int i = lq + 4 * k;
      x[k] = i < nb ? Bt[(size_t)i * kRhsCols + lc] : 0.0;
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
      if (i < nb) Bt[(size_t)i * kRhsCols + lc] = x[k];
    }
  }
  __syncthreads();
  {  // A22 -= L21 U12 on the tile (L21 = rows j0 + nb.. of the panel, already swapped by the panel kernel)
    const int c = tid % kRhsCols;
    for (int r = nb + tid / kRhsCols; r < rows; r += kRhsThreads / kRhsCols) {
      const double* ar = A + (size_t)(j0 + r) * ld + j0;
      double acc = Bt[(size_t)r * kRhsCols + c];
#pragma unroll 8
      for (int l = 0; l < nb; ++l) acc = fma(-ar[l], Bt[(size_t)l * kRhsCols + c], acc);
      Bt[(size_t)r * kRhsCols + c] = acc;
    }
  }
  __syncthreads();
  for (int e = tid; e < rows * kRhsCols; e += kRhsThreads) {
    const int r = e / kRhsCols, c = e % kRhsCols;
    if (cb + c < ce) A[(size_t)(j0 + r) * ld + cb + c] = Bt[e];
  }
}

// The right-hand-side phase of a slab in one launch: CTA (t, q) takes columns
// [8t, 8t + 8) of problem q's right-hand side R (n x w), applies the row
// interchanges, solves L (unit lower) then U (upper) of P S_s = L U, and
// writes the columns to their destinations (W_s to the Up slot; S_s^{-1} to the
// inverse slot or, in single-solve mode, y_s to the solution).  The columns
// are independent, so the two triangular solves need no grid-wide step: per
// 32-row block one warp solves the diagonal block (four lanes per column) and
// then all threads update the remaining rows of the tile in shared memory.
__global__ void __launch_bounds__(kRhsThreads) k_lu_rhs_solve(ProbPtrs pp, size_t off_lu, int ld, int piv_off,
                                                              size_t off_rhs, int w, int n, int nnext, size_t off_w,
                                                              size_t off_inv, long o, int single) {
  extern __shared__ double rsm[];
  double* Bt = rsm;                                  // n x kRhsCols tile
  double* Ls = rsm + (size_t)n * kRhsCols;           // 32 x 33 diagonal block
  int* idx = reinterpret_cast<int*>(Ls + 32 * 33);   // row permutation (n)
  const int q = blockIdx.y;
  const double* A = pp.ws[q] + off_lu;
  const double* R = pp.ws[q] + off_rhs;
  const int* piv = pp.piv[q] + piv_off;
  const int c0 = blockIdx.x * kRhsCols;
  const int tid = threadIdx.x;
  if (tid == 0) {  // the interchanges, applied in order, as one permutation
    for (int i = 0; i < n; ++i) idx[i] = i;
    for (int j = 0; j < n; ++j) {
      const int p = piv[j];
      if (p != j && p >= 0 && p < n) { const int t = idx[j]; idx[j] = idx[p]; idx[p] = t; }
    }
  }
  __syncthreads();
  for (int e = tid; e < n * kRhsCols; e += kRhsThreads) {
    const int r = e / kRhsCols, c = e % kRhsCols;
    Bt[e] = c0 + c < w ? R[(size_t)idx[r] * w + c0 + c] : 0.0;
  }
  const int lane = tid & 31, warp = tid >> 5;
  const int lq = lane & 3, lbase = lane & ~3, lc = lane >> 2;  // diagonal solve: 4 lanes per column
  for (int pass = 0; pass < 2; ++pass) {
    const bool upper = pass == 1;
    const int nblk = (n + 31) / 32;
    for (int bb = 0; bb < nblk; ++bb) {
      const int blk = upper ? nblk - 1 - bb : bb;
      const int i0 = blk * 32, nb = n - i0 < 32 ? n - i0 : 32;
      __syncthreads();  // the tile rows of this block are final
      for (int e = tid; e < 32 * 32; e += kRhsThreads) {
        const int i = e >> 5, l = e & 31;
        Ls[i * 33 + l] = (i < nb && l < nb) ? A[(size_t)(i0 + i) * ld + i0 + l] : 0.0;
      }
      __syncthreads();
      if (warp == 0) {
        double x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int i = lq + 4 * k;
          x[k] = i < nb ? Bt[(size_t)(i0 + i) * kRhsCols + lc] : 0.0;
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
              x[l >> 2] = (l < nb) ? x[l >> 2] / (dg == 0.0 ? 1e-300 : dg) : 0.0;
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
          if (i < nb) Bt[(size_t)(i0 + i) * kRhsCols + lc] = x[k];
        }
      }
      __syncthreads();
      // the rest of the tile: rows below (L) or above (U) the block
      const int rlo = upper ? 0 : i0 + nb, rhi = upper ? i0 : n;
      const int c = tid % kRhsCols;
      for (int r = rlo + tid / kRhsCols; r < rhi; r += kRhsThreads / kRhsCols) {
        const double* ar = A + (size_t)r * ld + i0;
        double acc = Bt[(size_t)r * kRhsCols + c];
#pragma unroll 8
        for (int l = 0; l < nb; ++l) acc = fma(-ar[l], Bt[(size_t)(i0 + l) * kRhsCols + c], acc);
        Bt[(size_t)r * kRhsCols + c] = acc;
      }
    }
  }
  __syncthreads();
  double* ws = pp.ws[q];
  for (int e = tid; e < n * kRhsCols; e += kRhsThreads) {
    const int r = e / kRhsCols, c = e % kRhsCols, j = c0 + c;
    if (j >= w) continue;
    const double v = Bt[e];
    if (j < nnext) ws[off_w + (size_t)r * ld + j] = v;
    else if (single) pp.y[q][(size_t)(o + r) * pp.ldb] = v;
    else ws[off_inv + (size_t)r * ld + (j - nnext)] = v;
  }
}


static int launch_panel(const ProbPtrs& pp, size_t offD, int poff, int n, int nmax, int j0, int nb, int nprob,
                        cudaStream_t s) {
  k_lu_panel<<<nprob, kPanelThreads, sizeof(double) * (size_t)(n - j0) * (nb + 1), s>>>(pp, offD, poff, n, nmax, j0, nb);
  return check_launch("k_lu_panel");
}

int blocklu_alloc(const lrfsi_mesh_s* m, int nprob, BlockLU& lu) {
  if (nprob < 1 || nprob > kMaxGemmDescs) return fail(LRFSI_EINVAL, "block LU: 1..32 problems per batch");
  if ((size_t)m->h.nmax * 9 * sizeof(double) > (size_t)kPanelSmem ||
      sizeof(double) * ((size_t)m->h.nmax * kRhsCols + 32 * 33) + sizeof(int) * (size_t)m->h.nmax > (size_t)kPanelSmem)
    return fail(LRFSI_EINVAL, "block LU: slab larger than the panel kernels support");
  {
    static bool attr = false;
    if (!attr) {
      LRFSI_CUDA(cudaFuncSetAttribute(k_lu_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPanelSmem));
      LRFSI_CUDA(cudaFuncSetAttribute(k_lu_rhs_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, kPanelSmem));
      LRFSI_CUDA(cudaFuncSetAttribute(k_lu_panel_update, cudaFuncAttributeMaxDynamicSharedMemorySize, kPanelSmem));
      attr = true;
    }
  }
  lu.nslab = m->h.nslab;
  lu.nmax = m->h.nmax;
  lu.nprob = nprob;
  lu.off = m->h.slab_off;
  const size_t nb2 = (size_t)lu.nmax * lu.nmax;
  lu.off_up = nb2 * lu.nslab;
  lu.off_lo = lu.off_up + nb2 * (lu.nslab - 1);
  lu.off_inv = lu.off_lo + nb2 * (lu.nslab - 1);
  lu.off_rhs = lu.off_inv + nb2 * lu.nslab;
  lu.per_prob = lu.off_rhs + 2 * nb2;
  LRFSI_TRY(lu.ws.alloc(lu.per_prob * nprob));
  LRFSI_TRY(lu.piv.alloc((size_t)lu.nslab * lu.nmax * nprob));
  LRFSI_TRY(lu.status.alloc(nprob));
  return LRFSI_OK;
}

static ProbPtrs make_ptrs(BlockLU& lu, int nprob) {
  ProbPtrs pp;
  for (int b = 0; b < nprob; ++b) {
    pp.ws[b] = lu.ws.p + lu.per_prob * b;
    pp.piv[b] = lu.piv.p + (size_t)lu.nslab * lu.nmax * b;
    pp.status[b] = lu.status.p + b;
    pp.J3[b] = nullptr;
    pp.alpha[b] = pp.beta[b] = 0;
  }
  return pp;
}

int blocklu_factor(const lrfsi_mesh_s* m, BlockLU& lu, const double* const* J3, const double* alpha,
                   const double* beta, int nprob, cudaStream_t s, const double* const* b, double* const* y, int ldb) {
  if (nprob > lu.nprob) return fail(LRFSI_EINVAL, "block LU: more problems than allocated");
  ProbPtrs pp = make_ptrs(lu, nprob);
  const int single = b != nullptr;
  pp.ldb = ldb;
  for (int q = 0; q < nprob; ++q) {
    pp.b[q] = single ? b[q] : nullptr;
    pp.y[q] = single ? y[q] : nullptr;
  }
  for (int b = 0; b < nprob; ++b) {
    pp.J3[b] = J3[b];
    pp.alpha[b] = alpha[b];
    pp.beta[b] = beta[b];
  }
  const int nmax = lu.nmax;
  const size_t nb2 = (size_t)nmax * nmax;
  for (int b = 0; b < nprob; ++b) LRFSI_CUDA(cudaMemsetAsync(pp.ws[b], 0, sizeof(double) * lu.off_inv, s));
  LRFSI_CUDA(cudaMemsetAsync(lu.status.p, 0, sizeof(int) * nprob, s));
  const long nnz = (long)m->h.colidx.size();
  TimedLaunch tl_all(KC_LU, s);  // the whole factorisation is one timed region of class KC_LU
  k_lu_extract<<<dim3(ceil_div(nnz, 256), nprob), 256, 0, s>>>(pp, m->dense_off.p, nnz);
  LRFSI_TRY(check_launch("k_lu_extract"));
  std::vector<GemmDesc<double>> gd(nprob);
  for (int sl = 0; sl < lu.nslab; ++sl) {
    const int n = (int)(lu.off[sl + 1] - lu.off[sl]);
    const int nnext = sl + 1 < lu.nslab ? (int)(lu.off[sl + 2] - lu.off[sl + 1]) : 0;
    const size_t offD = nb2 * sl;
    const int poff = sl * nmax;
    // blocked right-looking LU of the Schur block S_s; the panel width keeps
    // the staged panel within shared memory
    int nbp = kNb;
    while (nbp > 8 && (size_t)n * (nbp + 1) * sizeof(double) > (size_t)kPanelSmem) nbp /= 2;
    for (int j0 = 0; j0 < n; j0 += nbp) {
      const int nb = j0 + nbp < n ? nbp : n - j0;
      {
        account(KC_LUPANEL, (double)nprob * ((double)(n - j0) * nb * nb - (double)nb * nb * nb / 3.0), 0);
        TimedLaunch tk(KC_LUPANEL, s);
        LRFSI_TRY(launch_panel(pp, offD, poff, n, nmax, j0, nb, nprob, s));
        tk.end(s);
      }
      // interchanges left and right of the panel, U12 and the trailing update, columns in parallel
      {
        const int ncols = ceil_div(j0, kRhsCols) + ceil_div(n - j0 - nb, kRhsCols);
        if (ncols > 0) {
          account(KC_LUTRSM, (double)nprob * ((double)nb * nb * (n - j0 - nb) +
                                              2.0 * (double)(n - j0 - nb) * (n - j0 - nb) * nb), 0);
          TimedLaunch tk(KC_LUTRSM, s);
          const size_t smem = sizeof(double) * ((size_t)(n - j0) * kRhsCols + 32 * 33) + sizeof(int) * (size_t)(n - j0);
          k_lu_panel_update<<<dim3(ncols, nprob), kRhsThreads, smem, s>>>(pp, offD, nmax, poff, n, j0, nb);
          LRFSI_TRY(check_launch("k_lu_panel_update"));
          tk.end(s);
        }
      }
    }
    // RHS = P [Up_s | I];  L solve;  U solve  ->  [W_s | S_s^{-1}]; in
    // single-solve mode RHS = P [Up_s | b_s - Lo_{s-1} y_{s-1}] -> [W_s | y_s]
    const int ldr = nnext + (single ? 1 : n);
    const long o = lu.off[sl];
    k_lu_rhs<<<dim3(ceil_div((long)n * ldr, 256), nprob), 256, 0, s>>>(pp, lu.off_up + nb2 * sl, lu.off_rhs, n, nnext,
                                                                       nmax, ldr, o, single);
    LRFSI_TRY(check_launch("k_lu_rhs"));
    if (single && sl > 0) {
      const long op = lu.off[sl - 1];
      const int np = (int)(o - op);
      for (int q = 0; q < nprob; ++q) {
        double* ws = pp.ws[q];
        gd[q] = GemmDesc<double>{n, 1, np, ws + lu.off_lo + nb2 * (sl - 1), nmax, 1, y[q] + op * ldb, ldb, 1,
                                 ws + lu.off_rhs + nnext, ldr, 1, -1.0, 1.0};
      }
      LRFSI_TRY(gemm_grouped<double>(gd.data(), nprob, s));
    }
    {  // interchanges, L and U solves and the copy-out, columns in parallel
      account(KC_LUTRSM, (double)nprob * n * n * ldr, 0);
      TimedLaunch tk(KC_LUTRSM, s);
      const size_t smem = sizeof(double) * ((size_t)n * kRhsCols + 32 * 33) + sizeof(int) * (size_t)n;
      k_lu_rhs_solve<<<dim3(ceil_div(ldr, kRhsCols), nprob), kRhsThreads, smem, s>>>(
          pp, offD, nmax, poff, lu.off_rhs, ldr, n, nnext, lu.off_up + nb2 * sl, lu.off_inv + nb2 * sl, o, single);
      LRFSI_TRY(check_launch("k_lu_rhs_solve"));
      tk.end(s);
    }
    // Schur complement of the next slab: D_{s+1} -= Lo_s W_s
    if (nnext > 0) {
      for (int b = 0; b < nprob; ++b) {
        double* ws = pp.ws[b];
        gd[b] = GemmDesc<double>{nnext, nnext, n, ws + lu.off_lo + nb2 * sl, nmax, 1, ws + lu.off_up + nb2 * sl, nmax,
                                 1, ws + nb2 * (sl + 1), nmax, 1, -1.0, 1.0};
      }
      LRFSI_TRY(gemm_grouped<double>(gd.data(), nprob, s));
    }
  }
  if (single) {  // backward sweep: x_s = y_s - W_s x_{s+1}
    for (int sl = lu.nslab - 2; sl >= 0; --sl) {
      const long o = lu.off[sl], on = lu.off[sl + 1];
      const int n = (int)(on - o), nn = (int)(lu.off[sl + 2] - on);
      for (int q = 0; q < nprob; ++q) {
        double* ws = pp.ws[q];
        gd[q] = GemmDesc<double>{n, 1, nn, ws + lu.off_up + nb2 * sl, nmax, 1, y[q] + on * ldb, ldb, 1,
                                 y[q] + o * ldb, ldb, 1, -1.0, 1.0};
      }
      LRFSI_TRY(gemm_grouped<double>(gd.data(), nprob, s));
    }
  }
  {
    double fl = 0;
    for (int sl = 0; sl < lu.nslab; ++sl) {
      const double n = (double)(lu.off[sl + 1] - lu.off[sl]);
      const double nn = sl + 1 < lu.nslab ? (double)(lu.off[sl + 2] - lu.off[sl + 1]) : 0.0;
      // LU, the triangular solves on the right-hand side, the Schur update
      fl += (2.0 / 3.0) * n * n * n + 2.0 * n * n * (nn + (single ? 1.0 : n)) + 2.0 * nn * nn * n;
    }
    account(KC_LU, fl * nprob, 0);
  }
  tl_all.end(s);
  return LRFSI_OK;
}

int blocklu_solve(BlockLU& lu, double* const* X, double* const* Y, const int* r, int ld, int nprob, cudaStream_t s,
                  const Gate* gates) {
  TimedLaunch tl_all(KC_LUSOLVE, s);  // the whole solve is one timed region (its GEMMs are class KC_GEMM)
  const int nmax = lu.nmax;
  const size_t nb2 = (size_t)nmax * nmax;
  std::vector<GemmDesc<double>> gd(nprob);
  for (int sl = 0; sl < lu.nslab; ++sl) {
    const long o = lu.off[sl];
    const int n = (int)(lu.off[sl + 1] - o);
    if (sl > 0) {  // X_s -= Lo_{s-1} Y_{s-1}
      const long op = lu.off[sl - 1];
      const int np = (int)(o - op);
      for (int b = 0; b < nprob; ++b) {
        double* ws = lu.ws.p + lu.per_prob * b;
        gd[b] = GemmDesc<double>{n, r[b], np, ws + lu.off_lo + nb2 * (sl - 1), nmax, 1, Y[b] + op * ld, ld, 1,
                                 X[b] + o * ld, ld, 1, -1.0, 1.0};
        if (gates) gd[b].gate = gates[b];
      }
      LRFSI_TRY(gemm_grouped<double>(gd.data(), nprob, s));
    }
    for (int b = 0; b < nprob; ++b) {  // Y_s = S_s^{-1} X_s
      double* ws = lu.ws.p + lu.per_prob * b;
      gd[b] = GemmDesc<double>{n, r[b], n, ws + lu.off_inv + nb2 * sl, nmax, 1, X[b] + o * ld, ld, 1, Y[b] + o * ld,
                               ld, 1, 1.0, 0.0};
      if (gates) gd[b].gate = gates[b];
    }
    LRFSI_TRY(gemm_grouped<double>(gd.data(), nprob, s));
  }
  for (int sl = lu.nslab - 2; sl >= 0; --sl) {  // Y_s -= W_s Y_{s+1}
    const long o = lu.off[sl], on = lu.off[sl + 1];
    const int n = (int)(on - o), nn = (int)(lu.off[sl + 2] - on);
    for (int b = 0; b < nprob; ++b) {
      double* ws = lu.ws.p + lu.per_prob * b;
      gd[b] = GemmDesc<double>{n, r[b], nn, ws + lu.off_up + nb2 * sl, nmax, 1, Y[b] + on * ld, ld, 1, Y[b] + o * ld,
                               ld, 1, -1.0, 1.0};
      if (gates) gd[b].gate = gates[b];
    }
    LRFSI_TRY(gemm_grouped<double>(gd.data(), nprob, s));
  }
  tl_all.end(s);
  return LRFSI_OK;
}

int blocklu_status(BlockLU& lu, int nprob, std::vector<int>& out, cudaStream_t s) {
  out.assign(nprob, 0);
  LRFSI_CUDA(cudaMemcpyAsync(out.data(), lu.status.p, sizeof(int) * nprob, cudaMemcpyDeviceToHost, s));
  LRFSI_CUDA(cudaStreamSynchronize(s));
  return LRFSI_OK;
}

}  // namespace lrfsi
