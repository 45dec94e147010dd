// Dense FP64 building blocks: grouped GEMM, split-row Gram products and the
// small per-subset steps of the rank truncation.
//
// Truncation T (the paper's truncation operator, Sec. 5: for an order-2
// tensor the best approximation of rank <= R, Eckart-Young) of S = X Vc^T,
// X tall (M x p), Vc small (m x p), by two Cholesky-QR passes on X and a
// one-sided Jacobi SVD of the small core:
//   pass 1: G = X^T X scaled to unit diagonal, Cholesky with dependent-column
//           dropping (pivot <= drop), Q1 = X T1;
//   pass 2: G2 = Q1^T Q1 = R2^T R2, C = R2 R1 D^{-1} Vc^T (k x m),
//           C = W diag(s) Z^T (one-sided Jacobi), rank r by the tolerance rule,
//           U' = Q1 R2^{-1} W_r (orthonormal), V' = Z_r diag(s_r).
// The factorisations run in one CTA per problem, the SVD on a thread-block
// cluster per problem, and every product with O(p^2 m) or more work (the core
// products, T2 W_r) in the grouped GEMM.
#include <cooperative_groups.h>

#include <atomic>
#include <type_traits>
#include <vector>
#include <cmath>

#include "dense.h"
#include "ozaki.h"

namespace lrfsi {

// ---------------------------------------------------------------------------
// Grouped GEMM (SIMT; FP64 issue rate bounds it on this GPU)
// ---------------------------------------------------------------------------
template <class T>
struct GemmBatch {
  GemmDesc<T> d[kMaxGemmDescs];
};

constexpr int GBM = 64, GBN = 64, GBK = 16;

// Tile BM x BN, 256 threads, (BM/16) x (BN/16) outputs per thread.  With
// ks > 1 the k range is split: chunk c of descriptor z writes alpha * A B over
// its k slice to part[z][c] (m x n dense) and k_gemm_reduce adds the chunks in
// order (deterministic) together with beta * C.
template <class T, int BM, int BN>
__global__ void __launch_bounds__(256) k_gemm(GemmBatch<T> gb, int ks, T* __restrict__ part, long part_stride) {
  const int z = blockIdx.z / ks, chunk = blockIdx.z % ks;
  GemmDesc<T> g = gb.d[z];
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (m0 >= g.m || n0 >= g.n || !gate_open(g.gate)) return;
  if (g.sel && *g.sel) g.A = g.A_alt;
  constexpr int RM = BM / 16, RN = BN / 16;
  __shared__ T As[GBK][BM + 1];
  __shared__ T Bs[GBK][BN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[RM][RN];
#pragma unroll
  for (int r = 0; r < RM; ++r)
#pragma unroll
    for (int c = 0; c < RN; ++c) acc[r][c] = 0;
  const bool a_kfast = g.a_cs == 1, b_nfast = g.b_cs == 1;
  const int kc = (g.k + ks - 1) / ks;
  const int kbeg = chunk * kc, kend = kbeg + kc < g.k ? kbeg + kc : g.k;
  for (int k0 = kbeg; k0 < kend; k0 += GBK) {
    for (int idx = threadIdx.x; idx < BM * GBK; idx += 256) {
      int i, l;
      if (a_kfast) { l = idx % GBK; i = idx / GBK; } else { i = idx % BM; l = idx / BM; }
      const int gi = m0 + i, gl = k0 + l;
      As[l][i] = (gi < g.m && gl < kend) ? g.A[(long)gi * g.a_rs + (long)gl * g.a_cs] : T(0);
    }
    for (int idx = threadIdx.x; idx < BN * GBK; idx += 256) {
      int j, l;
      if (b_nfast) { j = idx % BN; l = idx / BN; } else { l = idx % GBK; j = idx / GBK; }
      const int gj = n0 + j, gl = k0 + l;
      Bs[l][j] = (gj < g.n && gl < kend) ? g.B[(long)gl * g.b_rs + (long)gj * g.b_cs] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < GBK; ++l) {
      T a[RM], bb[RN];
#pragma unroll
      for (int r = 0; r < RM; ++r) a[r] = As[l][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < RN; ++c) bb[c] = Bs[l][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int c = 0; c < RN; ++c) acc[r][c] = fma(a[r], bb[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < RM; ++r) {
    const int gi = m0 + ty + 16 * r;
    if (gi >= g.m) continue;
#pragma unroll
    for (int c = 0; c < RN; ++c) {
      const int gj = n0 + tx + 16 * c;
      if (gj >= g.n) continue;
      if (ks > 1) {
        part[(long)blockIdx.z * part_stride + (long)gi * g.n + gj] = g.alpha * acc[r][c];
      } else {
        T* cp = g.C + (long)gi * g.c_rs + (long)gj * g.c_cs;
        T v = g.alpha * acc[r][c];
        if (g.beta != T(0)) v += g.beta * *cp;
        *cp = v;
      }
    }
  }
}

template <class T>
__global__ void k_gemm_reduce(GemmBatch<T> gb, int ks, const T* __restrict__ part, long part_stride) {
  const GemmDesc<T> g = gb.d[blockIdx.y];
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)g.m * g.n || !gate_open(g.gate)) return;
  const int i = (int)(e / g.n), j = (int)(e % g.n);
  T v = 0;
  for (int c = 0; c < ks; ++c) v += part[((long)blockIdx.y * ks + c) * part_stride + e];
  T* cp = g.C + (long)i * g.c_rs + (long)j * g.c_cs;
  if (g.beta != T(0)) v += g.beta * *cp;
  *cp = v;
}

// the calling thread's workspace of the grouped GEMMs (split-K partial sums,
// tensor-core slices; grown on demand, freed when the thread exits), so that
// handles driven from different host threads on their own streams never share
// it, and the thread's bound workspace, if any
struct GemmWs {
  void* p = nullptr;
  size_t bytes = 0;
  ~GemmWs() {
    if (p) cudaFree(p);
  }
};
static thread_local GemmWs t_gemm_ws;
static thread_local void* t_ws_bound = nullptr;
static thread_local size_t t_ws_bound_bytes = 0;
static thread_local size_t t_ws_peak = 0;
void gemm_ws_bind(void* p, size_t bytes) { t_ws_bound = p; t_ws_bound_bytes = p ? bytes : 0; }
size_t gemm_ws_peak() { return t_ws_peak; }
void gemm_ws_peak_reset() { t_ws_peak = 0; }

// workspace of a grouped-GEMM call: the bound one, else the thread's one
// grown on demand; records the peak need
static int gemm_ws_get(size_t need, void** ws, size_t* bytes) {
  if (need > t_ws_peak) t_ws_peak = need;
  if (t_ws_bound) {
    if (need > t_ws_bound_bytes) return fail(LRFSI_EINVAL, "gemm_grouped: bound workspace too small");
    *ws = t_ws_bound;
    *bytes = t_ws_bound_bytes;
    return LRFSI_OK;
  }
  if (need > t_gemm_ws.bytes) {
    if (t_gemm_ws.p) cudaFree(t_gemm_ws.p);
    t_gemm_ws.p = nullptr;
    t_gemm_ws.bytes = 0;
    LRFSI_CUDA(cudaMalloc(&t_gemm_ws.p, need));
    t_gemm_ws.bytes = need;
  }
  *ws = t_gemm_ws.p;
  *bytes = t_gemm_ws.bytes;
  return LRFSI_OK;
}

template <class T>
static int gemm_grouped_simt(const GemmDesc<T>* descs, int n, cudaStream_t s);

template <class T>
int gemm_grouped(const GemmDesc<T>* descs, int n, cudaStream_t s) {
  if constexpr (std::is_same<T, double>::value) {
    if (gram_path() == 1) {
      std::vector<GemmDesc<double>> tcd, rest;
      for (int i = 0; i < n; ++i) (ozaki_gemm_eligible(descs[i]) ? tcd : rest).push_back(descs[i]);
      if (!tcd.empty()) {
        double fl = 0, by = 0;
        for (const GemmDesc<double>& g : tcd) {
          if (!gate_counts(g.gate, s)) continue;
          fl += 2.0 * g.m * g.n * g.k;
          by += 8.0 * ((double)g.m * g.k + (double)g.k * g.n + (g.beta != 0.0 ? 2.0 : 1.0) * g.m * g.n);
        }
        account(KC_GEMM_TC, fl, by);
        TimedLaunch tl(KC_GEMM_TC, s);
        void* ws = nullptr;
        size_t wsb = 0;
        LRFSI_TRY(gemm_ws_get(ozaki_gemm_work_bytes(tcd.data(), (int)tcd.size()), &ws, &wsb));
        LRFSI_TRY(ozaki_gemm(tcd.data(), (int)tcd.size(), ws, wsb, s));
        tl.end(s);
        return rest.empty() ? LRFSI_OK : gemm_grouped_simt<double>(rest.data(), (int)rest.size(), s);
      }
    }
  }
  return gemm_grouped_simt<T>(descs, n, s);
}

template <class T>
static int gemm_grouped_simt(const GemmDesc<T>* descs, int n, cudaStream_t s) {
  constexpr int kTarget = 2 * 152;  // enough CTAs to occupy every SM's FP64 unit twice
  for (int i = 0; i < n;) {  // chunks of up to kMaxGemmDescs non-empty products
    GemmBatch<T> gb;
    int cnt = 0, mm = 0, nn = 0, kk = 0;
    for (; i < n && cnt < kMaxGemmDescs; ++i) {
      if (descs[i].m <= 0 || descs[i].n <= 0) continue;
      gb.d[cnt] = descs[i];
      if (descs[i].k <= 0) gb.d[cnt].k = 0;
      mm = mm > descs[i].m ? mm : descs[i].m;
      nn = nn > descs[i].n ? nn : descs[i].n;
      kk = kk > descs[i].k ? kk : descs[i].k;
      ++cnt;
    }
    if (!cnt) continue;
    {
      double fl = 0, by = 0;
      for (int q = 0; q < cnt; ++q) {
        const GemmDesc<T>& g = gb.d[q];
        if (!gate_counts(g.gate, s)) continue;
        fl += 2.0 * g.m * g.n * g.k;
        by += sizeof(T) * ((double)g.m * g.k + (double)g.k * g.n + (g.beta != T(0) ? 2.0 : 1.0) * g.m * g.n);
      }
      account(sizeof(T) == 8 ? KC_GEMM : KC_GEMM32, fl, by);
    }
    TimedLaunch tl(sizeof(T) == 8 ? KC_GEMM : KC_GEMM32, s);
    const long tiles64 = (long)ceil_div(nn, 64) * ceil_div(mm, 64) * cnt;
    if (tiles64 >= kTarget) {  // enough 64x64 tiles to fill the GPU; else 32x32 tiles with split-K
      dim3 grid(ceil_div(nn, 64), ceil_div(mm, 64), cnt);
      k_gemm<T, 64, 64><<<grid, 256, 0, s>>>(gb, 1, (T*)nullptr, 0);
      LRFSI_TRY(check_launch("k_gemm"));
      tl.end(s);
      continue;
    }
    const long tiles32 = (long)ceil_div(nn, 32) * ceil_div(mm, 32) * cnt;
    int ks = 1;
    if (tiles32 < kTarget && kk >= 4 * GBK) {
      ks = (int)((kTarget + tiles32 - 1) / tiles32);
      const int kmax = kk / (2 * GBK);
      if (ks > kmax) ks = kmax;
      if (ks > 16) ks = 16;
      if (ks < 1) ks = 1;
    }
    const long pstride = (long)mm * nn;
    void* ws = nullptr;
    if (ks > 1) {
      size_t wsb = 0;
      LRFSI_TRY(gemm_ws_get(sizeof(T) * (size_t)cnt * ks * pstride, &ws, &wsb));
    }
    dim3 grid(ceil_div(nn, 32), ceil_div(mm, 32), cnt * ks);
    k_gemm<T, 32, 32><<<grid, 256, 0, s>>>(gb, ks, (T*)ws, pstride);
    LRFSI_TRY(check_launch("k_gemm"));
    if (ks > 1) {
      dim3 g2(ceil_div(pstride, 256), cnt);
      k_gemm_reduce<T><<<g2, 256, 0, s>>>(gb, ks, (const T*)ws, pstride);
      LRFSI_TRY(check_launch("k_gemm_reduce"));
    }
    tl.end(s);
  }
  return LRFSI_OK;
}
template int gemm_grouped<double>(const GemmDesc<double>*, int, cudaStream_t);
template int gemm_grouped<float>(const GemmDesc<float>*, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Gram products, split over rows
// ---------------------------------------------------------------------------
struct GramBatch {
  GramDesc d[kMaxGemmDescs];
};
constexpr int kGramRowsMin = 256;

__global__ void __launch_bounds__(256) k_gram_partial(GramBatch gb, long M, int nsplit, int pmax, int qmax,
                                                     double* __restrict__ work, int upper) {
  const GramDesc g = gb.d[blockIdx.z];
  const int tiles_q = (qmax + GBN - 1) / GBN;
  int ti = blockIdx.x / tiles_q, tj = blockIdx.x % tiles_q;
  if (upper) {  // blockIdx.x enumerates the tiles ti <= tj row by row
    int t = blockIdx.x;
    ti = 0;
    while (t >= tiles_q - ti) { t -= tiles_q - ti; ++ti; }
    tj = ti + t;
  }
  const int i0 = ti * GBM, j0 = tj * GBN;
  const int split = blockIdx.y;
  double* out = work + ((size_t)blockIdx.z * nsplit + split) * (size_t)pmax * qmax;
  if (i0 >= g.p || j0 >= g.q || !gate_open(g.gate)) return;
  const long chunk = (M + nsplit - 1) / nsplit;
  const long r0 = split * chunk, r1 = r0 + chunk < M ? r0 + chunk : M;
  __shared__ double As[GBK][GBM + 1];
  __shared__ double Bs[GBK][GBN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0;
  for (long k0 = r0; k0 < r1; k0 += GBK) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = threadIdx.x + 256 * e;
      const int i = idx % GBM, l = idx / GBM;  // rows of the tall matrices are contiguous in i
      const long gl = k0 + l;
      As[l][i] = (i0 + i < g.p && gl < r1) ? g.A[gl * g.lda + i0 + i] : 0.0;
      Bs[l][i] = (j0 + i < g.q && gl < r1) ? g.B[gl * g.ldb + j0 + i] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < GBK; ++l) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[l][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[l][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int gi = i0 + ty + 16 * r;
    if (gi >= g.p) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gj = j0 + tx + 16 * c;
      if (gj < g.q) out[(size_t)gi * qmax + gj] = acc[r][c];
    }
  }
}

__global__ void k_gram_reduce(GramBatch gb, int nsplit, int pmax, int qmax, const double* __restrict__ work,
                              int upper) {
  const GramDesc g = gb.d[blockIdx.y];
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)g.p * g.q || !gate_open(g.gate)) return;
  int i = (int)(idx / g.q), j = (int)(idx % g.q);
  const int oi = i, oj = j;
  // symmetric products: tiles below the diagonal were not computed, read the mirror
  if (upper && i / GBM > j / GBN) { const int t = i; i = j; j = t; }
  const double* w = work + (size_t)blockIdx.y * nsplit * (size_t)pmax * qmax + (size_t)i * qmax + j;
  double s = 0;
  for (int t = 0; t < nsplit; ++t) s += w[(size_t)t * pmax * qmax];
  g.G[(size_t)oi * g.ldg + oj] = s;
}

static int gram_nsplit(int nbatch, long M, int pmax, int qmax) {
  int tiles = ceil_div(pmax, GBM) * ceil_div(qmax, GBN);
  long want = 4L * 152 / ((long)tiles * nbatch);
  long maxs = (M + kGramRowsMin - 1) / kGramRowsMin;
  if (want < 1) want = 1;
  if (want > maxs) want = maxs;
  if (want > 256) want = 256;
  return (int)want;
}

size_t gram_work_len(int nbatch, long M, int pmax, int qmax) {
  const size_t simt = (size_t)nbatch * gram_nsplit(nbatch, M, pmax, qmax) * (size_t)pmax * qmax;
  const size_t oz = (ozaki_work_bytes(nbatch, M, pmax, qmax) + sizeof(double) - 1) / sizeof(double);
  return simt > oz ? simt : oz;
}

int gram_batched(const GramDesc* d, int nbatch, long M, double* work, size_t work_len, cudaStream_t s) {
  if (gram_path() == 1 && nbatch > 0) return ozaki_gram(d, nbatch, M, work, work_len * sizeof(double), s);
  for (int base = 0; base < nbatch; base += kMaxGemmDescs) {
    GramBatch gb;
    int cnt = 0, pmax = 1, qmax = 1;
    for (int i = base; i < nbatch && cnt < kMaxGemmDescs; ++i, ++cnt) {
      gb.d[cnt] = d[i];
      pmax = pmax > d[i].p ? pmax : d[i].p;
      qmax = qmax > d[i].q ? qmax : d[i].q;
    }
    // all products symmetric (A^T A): only the tiles on and above the diagonal
    bool upper = pmax == qmax;
    for (int i = 0; i < cnt; ++i)
      upper = upper && gb.d[i].A == gb.d[i].B && gb.d[i].lda == gb.d[i].ldb && gb.d[i].p == gb.d[i].q;
    const int T = ceil_div(pmax, GBM);
    const int ntiles = upper ? T * (T + 1) / 2 : ceil_div(pmax, GBM) * ceil_div(qmax, GBN);
    int nsplit = gram_nsplit(cnt, M, pmax, qmax);
    if (upper) {  // the same number of CTAs for fewer tiles: more row splits
      long want = 4L * 152 / ((long)ntiles * cnt);
      const long maxs = (M + kGramRowsMin - 1) / kGramRowsMin;
      if (want < 1) want = 1;
      if (want > maxs) want = maxs;
      if (want > 256) want = 256;
      nsplit = (int)want;
    }
    const size_t fit = work_len / ((size_t)cnt * pmax * qmax);
    if (fit < 1) return fail(LRFSI_EINVAL, "gram workspace too small");
    if ((size_t)nsplit > fit) nsplit = (int)fit;
    {
      double fl = 0, by = 0;
      for (int i = 0; i < cnt; ++i) {
        if (!gate_counts(gb.d[i].gate, s)) continue;
        // symmetric products: the algorithmic work is the upper triangle
        const bool sym = gb.d[i].A == gb.d[i].B && gb.d[i].p == gb.d[i].q;
        fl += sym ? 1.0 * M * gb.d[i].p * (gb.d[i].p + 1) : 2.0 * M * gb.d[i].p * gb.d[i].q;
        by += 8.0 * M * (gb.d[i].A == gb.d[i].B ? gb.d[i].p : gb.d[i].p + gb.d[i].q);
      }
      account(KC_GRAM, fl, by);
    }
    TimedLaunch tl(KC_GRAM, s);
    dim3 grid(ntiles, nsplit, cnt);
    k_gram_partial<<<grid, 256, 0, s>>>(gb, M, nsplit, pmax, qmax, work, upper ? 1 : 0);
    LRFSI_TRY(check_launch("k_gram_partial"));
    dim3 g2(ceil_div((long)pmax * qmax, 256), cnt);
    k_gram_reduce<<<g2, 256, 0, s>>>(gb, nsplit, pmax, qmax, work, upper ? 1 : 0);
    LRFSI_TRY(check_launch("k_gram_reduce"));
    tl.end(s);
  }
  return LRFSI_OK;
}

// ---------------------------------------------------------------------------
// Small per-problem kernels (one CTA of 1024 threads per problem)
// ---------------------------------------------------------------------------
constexpr int kSmallThreads = 1024;

// Inverse of the k x k upper triangular R (row-major, ldr) into Ri (row-major,
// ldi): the diagonal reciprocals first (in parallel), then the rows from the
// bottom up; in row a thread b computes Ri[a][b] = -(sum_{l=a+1..b} R[a][l]
// Ri[l][b]) Ri[a][a] with four independent partial sums (no cross-lane
// reductions: every FP64 instruction of a warp costs the SM's FP64 pipe a
// full warp).  Must be called by the whole block.
__device__ void upper_inverse(const double* R, int ldr, double* Ri, int ldi, int k) {
  for (long e = threadIdx.x; e < (long)k * k; e += blockDim.x) {
    const int i = (int)(e / k), j = (int)(e % k);
    if (j < i) Ri[(size_t)i * ldi + j] = 0.0;
    else if (j == i) Ri[(size_t)i * ldi + i] = 1.0 / R[(size_t)i * ldr + i];
  }
  __syncthreads();
  for (int a = k - 2; a >= 0; --a) {
    const double inv = Ri[(size_t)a * ldi + a];
    const double* Ra = R + (size_t)a * ldr;
    for (int b = a + 1 + threadIdx.x; b < k; b += blockDim.x) {
      double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
      int l = a + 1;
      for (; l + 3 <= b; l += 4) {
        s0 = fma(Ra[l], Ri[(size_t)l * ldi + b], s0);
        s1 = fma(Ra[l + 1], Ri[(size_t)(l + 1) * ldi + b], s1);
        s2 = fma(Ra[l + 2], Ri[(size_t)(l + 2) * ldi + b], s2);
        s3 = fma(Ra[l + 3], Ri[(size_t)(l + 3) * ldi + b], s3);
      }
      for (; l <= b; ++l) s0 = fma(Ra[l], Ri[(size_t)l * ldi + b], s0);
      Ri[(size_t)a * ldi + b] = -((s0 + s1) + (s2 + s3)) * inv;
    }
    __syncthreads();
  }
}

// Right-looking Cholesky G = R^T R in place (upper triangle holds R), rows with
// pivot <= drop are marked dropped (keep[i] = 0) and do not update the rest.
// Thread 0 takes the pivot's root and its reciprocal; in the update thread b
// owns column b of the trailing upper triangle.
__device__ void chol_drop(double* G, int ld, int p, double drop, int* keep) {
  __shared__ double s_piv, s_rinv;
  for (int i = 0; i < p; ++i) {
    if (threadIdx.x == 0) {
      double piv = G[(size_t)i * ld + i];
      keep[i] = (piv > drop && isfinite(piv)) ? 1 : 0;
      s_piv = keep[i] ? sqrt(piv) : 0.0;
      s_rinv = keep[i] ? 1.0 / s_piv : 0.0;
    }
    __syncthreads();
    const double r = s_piv, rinv = s_rinv;
    double* Gi = G + (size_t)i * ld;
    if (r > 0) {
      for (int j = i + threadIdx.x; j < p; j += blockDim.x) Gi[j] = (j == i) ? r : Gi[j] * rinv;
      __syncthreads();
      for (int b = i + 1 + threadIdx.x; b < p; b += blockDim.x) {
        const double gib = Gi[b];
        for (int a = i + 1; a <= b; ++a) G[(size_t)a * ld + b] = fma(-Gi[a], gib, G[(size_t)a * ld + b]);
      }
    } else {
      for (int j = i + threadIdx.x; j < p; j += blockDim.x) Gi[j] = 0.0;
    }
    __syncthreads();
  }
}

size_t trunc_small_work(int p, int m) {
  const size_t n = (size_t)(p > m ? p : m);
  return 4 * (size_t)p * p + 3 * n * n + 2 * (size_t)p * m + 4 * n + 64 + trunc_svd_global_len(p, m, 16) +
         trunc_qr_len(p, m);
}

// Pass 1: unit-diagonal scaling and a diagonally pivoted (rank-revealing)
// Cholesky of the Gram: at every step the column with the largest remaining
// Schur diagonal is taken; the factorisation stops when that diagonal is
// <= drop (the remaining columns lie in the span of the chosen ones up to a
// relative remainder sqrt(drop)).  Outputs T1 (Q1 = X T1, k columns), the
// scaled factor Rs = R1 D^{-1} (p x p in work Rk, rows >= k zero; the core
// Y = Rs Vc^T is a GEMM after this kernel) and info[0] = k.
// The Schur complements live in shared memory as the packed upper triangle
// (original column order) when p (p + 1) / 2 + 2 p doubles fit the dynamic
// shared memory of the launch (smem_doubles), else in d.G (full square).
__device__ __forceinline__ int packed_idx(int a, int b, int p) {
  if (a > b) { const int t = a; a = b; b = t; }
  return a * p - (a * (a - 1)) / 2 + (b - a);
}
__global__ void __launch_bounds__(kSmallThreads) k_trunc_pass1(TruncDesc* descs, int smem_doubles) {
  const TruncDesc d = descs[blockIdx.x];
  const int p = d.p, m = d.m;
  if (!gate_open(d.gate)) return;
  if (p <= 0) {
    if (threadIdx.x == 0) { d.info[0] = 0; d.info[1] = 0; d.info[2] = 0; d.info[4] = 0; *d.frob2 = 0.0; }
    return;
  }
  TruncWork W(d.work, p, m);
  double* G = d.G;         // p x p, original column order; Schur complements in place
  double* R = W.Rk;        // k x p, R[a][b] = R1 entry for permuted columns a, b (b >= a)
  int* perm = d.iwork;
  __shared__ double s_val[33], s_root, s_rinv;
  __shared__ int s_idx[33];
  __shared__ int s_k;
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    const double g = G[(size_t)i * p + i];
    W.Dsc[i] = (g > 0 && isfinite(g)) ? 1.0 / sqrt(g) : 0.0;
    perm[i] = i;
  }
  __syncthreads();
  extern __shared__ double psm[];
  const bool packed = (long)p * (p + 1) / 2 + 2L * p <= (long)smem_doubles;
  double* Pk = psm;                            // packed Schur complements
  double* rrow = psm + (size_t)p * (p + 1) / 2;  // row i of R (original order)
  int* sperm = (int*)(rrow + p);               // the permutation (shared copy)
  if (packed) {
    for (long e = threadIdx.x; e < (long)p * p; e += blockDim.x) {
      const int a = (int)(e / p), b = (int)(e % p);
      if (b >= a) Pk[packed_idx(a, b, p)] = (W.Dsc[a] > 0 && W.Dsc[b] > 0) ? G[e] * W.Dsc[a] * W.Dsc[b] : 0.0;
    }
    for (int i = threadIdx.x; i < p; i += blockDim.x) sperm[i] = i;
    perm = sperm;
  } else {
    for (long e = threadIdx.x; e < (long)p * p; e += blockDim.x) {
      const int a = (int)(e / p), b = (int)(e % p);
      G[e] = (W.Dsc[a] > 0 && W.Dsc[b] > 0) ? G[e] * W.Dsc[a] * W.Dsc[b] : 0.0;
    }
  }
  if (threadIdx.x == 0) s_k = p;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // per-warp pivot candidates (largest remaining diagonal; ties: the smallest
  // position) in s_val[w], s_idx[w]: a scan here for the first pivot and on the
  // global path; on the packed path the update of a row leaves its new diagonal
  // with lane 0 of the row's warp, which keeps the warp's candidate
  auto scan = [&](int from) {
    double best = -1.0;
    int bj = 0x7fffffff;
    for (int j = from + threadIdx.x; j < p; j += blockDim.x) {
      const int pj = perm[j];
      const double v = packed ? Pk[packed_idx(pj, pj, p)] : G[(size_t)pj * p + pj];
      if (v > best) { best = v; bj = j; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double v2 = __shfl_xor_sync(0xffffffffu, best, o);
      const int j2 = __shfl_xor_sync(0xffffffffu, bj, o);
      if (v2 > best || (v2 == best && j2 < bj)) { best = v2; bj = j2; }
    }
    if (lane == 0) { s_val[wp] = best; s_idx[wp] = bj; }
  };
  __syncthreads();
  scan(0);
  __syncthreads();
  for (int i = 0; i < p; ++i) {
    // the pivot from the warps' candidates; thread 0 takes its root and
    // reciprocal and moves it to position i of the permutation
    if (threadIdx.x < 32) {
      double best = lane < nw ? s_val[lane] : -1.0;
      int bj = lane < nw ? s_idx[lane] : 0x7fffffff;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, best, o);
        const int j2 = __shfl_xor_sync(0xffffffffu, bj, o);
        if (v2 > best || (v2 == best && j2 < bj)) { best = v2; bj = j2; }
      }
      if (threadIdx.x == 0) {
        s_val[32] = best;
        s_idx[32] = bj;
        s_root = best > 0 ? sqrt(best) : 0.0;
        s_rinv = s_root > 0 ? 1.0 / s_root : 0.0;
        if (best > d.drop && isfinite(best) && bj < p) {
          const int t = perm[i];
          perm[i] = perm[bj];
          perm[bj] = t;
        }
      }
    }
    __syncthreads();
    const double piv = s_val[32];
    if (!(piv > d.drop) || !isfinite(piv)) {
      if (threadIdx.x == 0) s_k = i;
      break;  // uniform: every thread read the same s_val[32]
    }
    const int pi = perm[i];
    const double r = s_root, rinv = s_rinv;
    // row i of R, indexed by ORIGINAL column (no swaps of earlier rows needed)
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
      const int pj = perm[j];
      const double gij = packed ? Pk[packed_idx(pi, pj, p)] : G[(size_t)pi * p + pj];
      const double v = j < i ? 0.0 : (j == i ? r : gij * rinv);
      R[(size_t)i * p + pj] = v;
      if (packed) rrow[pj] = v;
    }
    __syncthreads();
    const int nt = p - i - 1;
    if (packed) {  // the upper triangle of the trailing block: a warp per row
      double best = -1.0;
      int bj = 0x7fffffff;
      for (int ra = i + 1 + wp; ra < p; ra += nw) {
        const int pa = perm[ra];
        const double ua = rrow[pa];
        for (int rb = ra + lane; rb < p; rb += 32) {
          const int pb = perm[rb];
          const double v = Pk[packed_idx(pa, pb, p)] - ua * rrow[pb];
          Pk[packed_idx(pa, pb, p)] = v;
          if (rb == ra && v > best) { best = v; bj = ra; }  // lane 0: the new diagonal
        }
      }
      if (lane == 0) { s_val[wp] = best; s_idx[wp] = bj; }
    } else {
      for (long e = threadIdx.x; e < (long)nt * nt; e += blockDim.x) {
        const int pa = perm[i + 1 + (int)(e / nt)], pb = perm[i + 1 + (int)(e % nt)];
        G[(size_t)pa * p + pb] -= R[(size_t)i * p + pa] * R[(size_t)i * p + pb];
      }
      __syncthreads();
      scan(i + 1);
    }
    __syncthreads();
  }
  __syncthreads();
  if (packed) {  // the permutation for the later kernels
    for (int i = threadIdx.x; i < p; i += blockDim.x) d.iwork[i] = sperm[i];
    __syncthreads();
  }
  const int k = s_k;
  if (threadIdx.x == 0) { d.info[0] = k; d.info[1] = 0; d.info[2] = 0; d.info[3] = 0; d.info[4] = 0; }
  // R_kk[a][b] = R[a][perm[b]] (upper triangular in pivot order) into T2 (ld k), inverse into Rki (ld k)
  for (long e = threadIdx.x; e < (long)k * k; e += blockDim.x) {
    const int a = (int)(e / k), b = (int)(e % k);
    d.T2[e] = R[(size_t)a * p + perm[b]];
  }
  __syncthreads();
  upper_inverse(d.T2, k, W.Rki, k, k);
  __syncthreads();
  for (long e = threadIdx.x; e < (long)p * p; e += blockDim.x) d.T1[e] = 0.0;
  __syncthreads();
  for (long e = threadIdx.x; e < (long)k * k; e += blockDim.x) {
    const int a = (int)(e / k), b = (int)(e % k);
    d.T1[(size_t)perm[a] * p + b] = W.Dsc[perm[a]] * W.Rki[(size_t)a * k + b];
  }
  // Rs = R D^{-1} (p x p, rows >= k zero): the core Y = Rs Vc^T is formed by
  // a grouped GEMM after this kernel.  (R[a][o] = 0 before a in pivot order.)
  __syncthreads();
  for (long e = threadIdx.x; e < (long)p * p; e += blockDim.x) {
    const int a = (int)(e / p), o = (int)(e % p);
    const double db = W.Dsc[o];
    R[e] = (a < k && db > 0) ? R[e] / db : 0.0;
  }
}

// One Cholesky-QR pass on the k x k Gram Gq (ld p) of the current basis:
// Gq = R^T R, T2 = R^{-1} (k x k, ld p), R zero-padded to p x p in work Rki
// (the core update Y <- R Y is a GEMM after this kernel).  info[4] = 1 when the
// basis was far from orthonormal (max |Gq_ij - delta_ij| > 0.1), so that one
// more pass is needed before the SVD.
__global__ void __launch_bounds__(kSmallThreads) k_trunc_qr(TruncDesc* descs, int write_third, int smem_doubles) {
  const TruncDesc d = descs[blockIdx.x];
  const int p = d.p, m = d.m;
  if (!gate_open(d.gate)) return;
  __shared__ int s_k, s_bad;
  __shared__ double s_dev;
  if (threadIdx.x == 0) { s_k = p > 0 ? d.info[0] : 0; s_bad = 0; s_dev = 0.0; }
  __syncthreads();
  const int k = s_k;
  if (k <= 0 || m <= 0) return;
  TruncWork W(d.work, p, m);
  extern __shared__ double qrsm[];
  // k x k (ld k): in shared memory when it fits the launch's dynamic shared memory
  double* R = (long)k * k <= (long)smem_doubles ? qrsm : W.Rk;
  for (long e = threadIdx.x; e < (long)k * k; e += blockDim.x) {
    const int a = (int)(e / k), b = (int)(e % k);
    const double g = d.G2[(size_t)a * p + b];
    R[e] = g;
    const double dev = fabs(g - (a == b ? 1.0 : 0.0));
    if (dev > 0.1) s_dev = dev;  // benign race: any large value sets the flag
  }
  __syncthreads();
  int* flags = (int*)W.Vm;
  chol_drop(R, k, k, 1e-300, flags);
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < k; ++i)
      if (!flags[i]) s_bad = 1;
    if (write_third) d.info[4] = (s_dev > 0.1) ? 1 : 0;
    if (s_bad) {
      d.info[2] = LRFSI_EBREAKDOWN;
      if (d.broke) *d.broke = 1;
    }
  }
  __syncthreads();
  if (s_bad) return;
  upper_inverse(R, k, W.Rki, k, k);
  __syncthreads();
  // T2 = R^{-1} in the leading k x k block of a zero p x p block (ld p)
  for (long e = threadIdx.x; e < (long)p * p; e += blockDim.x) {
    const int a = (int)(e / p), b = (int)(e % p);
    d.T2[e] = (a < k && b < k) ? W.Rki[(size_t)a * k + b] : 0.0;
  }
  __syncthreads();
  // R (upper triangle of the k x k factor) zero-padded to p x p into Rki: the
  // core update Y <- R Y is a grouped GEMM after this kernel
  for (long e = threadIdx.x; e < (long)p * p; e += blockDim.x) {
    const int a = (int)(e / p), b = (int)(e % p);
    W.Rki[e] = (a < k && b < k && b >= a) ? R[(size_t)a * k + b] : 0.0;
  }
}

// ---------------------------------------------------------------------------
// QR preconditioning of the SVD (Drmac and Veselic, "New fast and accurate
// Jacobi SVD algorithm", SIAM J. Matrix Anal. Appl. 29, 2008): the Jacobi
// matrix A (L x n, L >= n: A = C if m < k, else C^T) is factored as
// A P = Q R by Householder reflections with column pivoting, and the one-sided
// Jacobi iteration then runs on X = R^T, which converges in a few sweeps
// (the rows of R are graded by the pivoting).  With X W = Y (orthogonal
// columns, norms sigma): A = (Q W) (P Y)^T, so Q W holds the left and P Y the
// (sigma-scaled) right singular vectors of A.
// ---------------------------------------------------------------------------
// One CTA per problem.  The matrix is worked on in shared memory when it fits
// the launch's dynamic shared memory (smem_bytes), else in Aw.  Aw ends as the column-major reflectors (v_j in rows
// j.. of column j, its leading entry explicit) and R above the diagonal;
// Rt = R^T; tau_j; perm (A P = A[:, perm]).  The trailing norms of the
// columns are downdated by the squared entry that each reflector moves into
// R, and recomputed exactly where the downdated value has lost more than a
// sqrt(eps) fraction of the last exact one (the safeguard of Drmac and
// Bujanovic, "On the failure of rank-revealing QR factorization software",
// ACM TOMS 35, 2008).
constexpr int kQrSmem = 200 * 1024;
__global__ void __launch_bounds__(kSmallThreads) k_trunc_qrcp(TruncDesc* descs, int smem_bytes) {
  const TruncDesc d = descs[blockIdx.x];
  if (!gate_open(d.gate)) return;
  const int p = d.p, m = d.m;
  const int k = p > 0 ? d.info[0] : 0;
  if (k <= 0 || m <= 0 || d.info[2] != 0) return;  // the SVD kernel handles these
  const bool cols_of_C = m < k;
  const int n = cols_of_C ? m : k, L = cols_of_C ? k : m;
  const TruncWork W(d.work, p, m);
  const QrWork Q(W, p, m);
  extern __shared__ double qsm[];
  const bool in_smem = (size_t)L * n * sizeof(double) <= (size_t)smem_bytes;
  double* A = in_smem ? qsm : Q.Aw;
  const double* core = (d.sel && *d.sel) ? d.core_alt : d.core;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  __shared__ double s_val[32], s_nrm[1024], s_nrm0[1024];
  __shared__ int s_idx[32];
  __shared__ int s_piv;
  __shared__ double s_tau;
  double* nrm = n <= 1024 ? s_nrm : Q.nrm;
  double* nrm0 = n <= 1024 ? s_nrm0 : Q.scr;  // the last exact value (scr is free until the SVD)
  for (long e = tid; e < (long)L * n; e += blockDim.x) {
    const int c = (int)(e / L), i = (int)(e % L);
    A[e] = cols_of_C ? core[(size_t)i * m + c] : core[(size_t)c * m + i];
  }
  for (int c = tid; c < n; c += blockDim.x) Q.perm[c] = c;
  __syncthreads();
  for (int c = warp; c < n; c += nw) {
    double t = 0;
    for (int i = lane; i < L; i += 32) t = fma(A[(size_t)c * L + i], A[(size_t)c * L + i], t);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) nrm[c] = nrm0[c] = t;
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    // pivot: the largest trailing norm (ties: the smallest column)
    {
      double best = -1.0;
      int bc = 0x7fffffff;
      for (int c = j + tid; c < n; c += blockDim.x)
        if (nrm[c] > best) { best = nrm[c]; bc = c; }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, best, o);
        const int c2 = __shfl_xor_sync(0xffffffffu, bc, o);
        if (v2 > best || (v2 == best && c2 < bc)) { best = v2; bc = c2; }
      }
      if (lane == 0) { s_val[warp] = best; s_idx[warp] = bc; }
      __syncthreads();
      if (warp == 0) {
        best = lane < nw ? s_val[lane] : -1.0;
        bc = lane < nw ? s_idx[lane] : 0x7fffffff;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const double v2 = __shfl_xor_sync(0xffffffffu, best, o);
          const int c2 = __shfl_xor_sync(0xffffffffu, bc, o);
          if (v2 > best || (v2 == best && c2 < bc)) { best = v2; bc = c2; }
        }
        if (lane == 0) s_piv = bc;
      }
      __syncthreads();
    }
    // every trailing norm NaN (a non-finite core): no pivoting, tau = 0 below
    const int pv = s_piv < n ? s_piv : j;
    if (pv != j) {
      for (int i = tid; i < L; i += blockDim.x) {
        const double t = A[(size_t)j * L + i];
        A[(size_t)j * L + i] = A[(size_t)pv * L + i];
        A[(size_t)pv * L + i] = t;
      }
    }
    __syncthreads();
    // reflector H = I - tau v v^T with H x = alpha e_1, alpha = -sign(x_0) |x|,
    // |x| computed exactly (rows j..; the downdated norms only choose the pivot:
    // H is orthogonal only with the exact |x|)
    if (warp == 0) {
      double sg = 0;
      for (int i = j + lane; i < L; i += 32) sg = fma(A[(size_t)j * L + i], A[(size_t)j * L + i], sg);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sg += __shfl_xor_sync(0xffffffffu, sg, o);
      if (lane == 0) {
        if (pv != j) {
          const int t = Q.perm[j];
          Q.perm[j] = Q.perm[pv];
          Q.perm[pv] = t;
          nrm[pv] = nrm[j];
          nrm0[pv] = nrm0[j];
        }
        const double x0 = A[(size_t)j * L + j];
        const double nx = sqrt(sg);
        double alpha = 0.0, tau = 0.0;
        if (nx > 0.0) {
          alpha = x0 >= 0 ? -nx : nx;
          const double v0 = x0 - alpha;
          tau = -1.0 / (alpha * v0);
          A[(size_t)j * L + j] = v0;
        }
        Q.tau[j] = tau;
        Q.Rt[(size_t)j * n + j] = alpha;
        s_tau = tau;
      }
    }
    __syncthreads();
    // apply H to the columns j+1..: w = v . a_c, a_c -= tau w v (rows j..);
    // the trailing norm of a_c (rows j+1..) = that of rows j.. (H keeps it)
    // minus the new a_c[j]^2, recomputed where that cancels
    const double tau = s_tau;
    const double* v = A + (size_t)j * L;
    for (int c = j + 1 + warp; c < n; c += nw) {
      double* a = A + (size_t)c * L;
      if (tau != 0.0) {
        double t = 0;
        for (int i = j + lane; i < L; i += 32) t = fma(v[i], a[i], t);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        t *= tau;
        for (int i = j + lane; i < L; i += 32) a[i] = fma(-t, v[i], a[i]);
      }
      int again = 0;
      if (lane == 0) {  // lane 0 holds row j
        const double aj = a[j], t2 = nrm[c] - aj * aj;
        if (t2 > 1.4901161193847656e-8 * nrm0[c]) nrm[c] = t2;
        else again = 1;
      }
      again = __shfl_sync(0xffffffffu, again, 0);
      if (again) {
        double q = 0;
        for (int i = j + 1 + lane; i < L; i += 32) q = fma(a[i], a[i], q);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
        if (lane == 0) nrm[c] = nrm0[c] = q;
      }
    }
    __syncthreads();
  }
  // X = R^T: column c of X is row c of R (R[c][i] = A[i][c] for i > c)
  for (long e = tid; e < (long)n * n; e += blockDim.x) {
    const int c = (int)(e / n), i = (int)(e % n);
    if (i != c) Q.Rt[e] = i > c ? A[(size_t)i * L + c] : 0.0;
  }
  if (in_smem)  // the reflectors, for the output stage of the SVD
    for (long e = tid; e < (long)L * n; e += blockDim.x) Q.Aw[e] = A[e];
}

// ---------------------------------------------------------------------------
// SVD of the core by one-sided Jacobi on a thread-block cluster
// ---------------------------------------------------------------------------
// The core C (k x m, rows of d.core, ld m) gives the Jacobi matrix A = C
// (k x m) if m < k, else A = C^T (m x k); k_trunc_qrcp factors A P = Q R and
// the iteration orthogonalises the n columns of X = R^T (n x n): X W = Y
// with orthogonal columns, W accumulated.  Every column is stored with its W
// column appended (length LV = 2n), so one rotation updates both (column
// stride LS = LV + 2).  The kept singular vectors follow from Y and W (see the
// output stage).
//
// Parallel block ordering: the n columns form nb = 2 C blocks of b columns; CTA
// c of the cluster owns blocks 2c, 2c+1 in its shared memory.  A sweep is
//   (i) every CTA orthogonalises all pairs inside its own 2b columns, then
//  (ii) nb - 1 rounds of the round-robin tournament on blocks: in each round
//       CTA c copies its pair of blocks (from the owners, through distributed
//       shared memory) into local memory, rotates all b^2 cross pairs (b
//       sub-rounds of b disjoint pairs, one warp per pair), and writes them
//       back, followed by a cluster barrier.
// Every block pair meets once per sweep, so every column pair is visited; the
// pairing and the order of rotations are fixed, so the result does not depend
// on timing.  A pair is rotated when |a_x . a_y| > 2e-15 sqrt(|a_x|^2
// |a_y|^2) and neither column is below max(1e-16, 1e-2 tol) times the largest
// column norm (such columns lie below what the truncation keeps).
// Stops after a sweep without rotations (info[3] = sweeps) or at 40 sweeps
// (info[2] = LRFSI_ENOCONV).  The FP64 rate of one SM is the bound here, hence
// the cluster: the rotations of one problem run on C SMs.
constexpr int kSvdThreads = 256;
constexpr int kSvdWarps = kSvdThreads / 32;

// The pair test computes |a_x|^2, |a_y|^2 and a_x . a_y together (interleaved
// chains, two partial sums each): a sub-round's time is the latency of this
// chain, not its FP64 count.
__device__ __forceinline__ bool jacobi_pair(double* __restrict__ cx, double* __restrict__ cy, int L, int LV,
                                            double small2, int lane) {
  double al0 = 0, be0 = 0, ga0 = 0, al1 = 0, be1 = 0, ga1 = 0;
  int i = lane;
  for (; i + 32 < L; i += 64) {
    const double u0 = cx[i], v0 = cy[i], u1 = cx[i + 32], v1 = cy[i + 32];
    al0 = fma(u0, u0, al0);
    be0 = fma(v0, v0, be0);
    ga0 = fma(u0, v0, ga0);
    al1 = fma(u1, u1, al1);
    be1 = fma(v1, v1, be1);
    ga1 = fma(u1, v1, ga1);
  }
  if (i < L) {
    const double u0 = cx[i], v0 = cy[i];
    al0 = fma(u0, u0, al0);
    be0 = fma(v0, v0, be0);
    ga0 = fma(u0, v0, ga0);
  }
  double al = al0 + al1, be = be0 + be1, ga = ga0 + ga1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    al += __shfl_xor_sync(0xffffffffu, al, o);
    be += __shfl_xor_sync(0xffffffffu, be, o);
    ga += __shfl_xor_sync(0xffffffffu, ga, o);
  }
  // rotate when |a_x . a_y| > 2e-15 |a_x| |a_y| (squared: no square root)
  if (!(al > small2 && be > small2 && ga * ga > 4e-30 * al * be)) return false;
  // the rotation with t = tan theta the smaller root of t^2 + 2 zeta t - 1 = 0,
  // zeta = (be - al) / (2 ga): with tau = be - al, g2 = 2 ga,
  // r = sqrt(tau^2 + g2^2) and d = |tau| + r, t = sign(tau) g2 / d, so
  // cos theta = sqrt(d / (2 r)) = d q and sin theta = sign(tau) g2 q with
  // q = 1 / sqrt(2 r d) (no division)
  const double tau = be - al, g2 = 2.0 * ga;
  const double r = sqrt(fma(tau, tau, g2 * g2)), d = fabs(tau) + r;
  const double q = rsqrt(2.0 * r * d);
  const double c = d * q, sn = (tau >= 0 ? g2 : -g2) * q;
  for (int j = lane; j < LV; j += 32) {
    const double u = cx[j], v = cy[j];
    cx[j] = c * u - sn * v;
    cy[j] = sn * u + c * v;
  }
  return true;
}

// largest squared column norm (A part) of the 2b columns at cols (stride LS;
// global column index of slot 0 = j0; columns >= n are padding)
__device__ double local_cmax(double* cols, int nslot, int j0, int n, int L, int LV, int LS) {
  __shared__ double s_red[kSvdWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double mx = 0;
  for (int h = warp; h < nslot; h += kSvdWarps) {
    if (j0 + h >= n) continue;
    double t = 0;
    for (int i = lane; i < L; i += 32) t = fma(cols[(size_t)h * LS + i], cols[(size_t)h * LS + i], t);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    (void)LV;
    mx = fmax(mx, t);
  }
  if (lane == 0) s_red[warp] = mx;
  __syncthreads();
  double r = 0;
  for (int w = 0; w < kSvdWarps; ++w) r = fmax(r, s_red[w]);
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kSvdThreads) k_trunc_svd(TruncDesc* descs, int global_blocks) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), crank = (int)cl.block_rank();
  const TruncDesc d = descs[blockIdx.y];
  const int p = d.p, m = d.m;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ double s_ex[2][2];  // per sweep parity: {rotations, max column norm^2}
  __shared__ double s_tot, s_cm;
  __shared__ int s_rot, s_r;
  // uniform across the cluster: every CTA reads the same descriptor and info
  if (!gate_open(d.gate)) return;
  const int k = p > 0 ? d.info[0] : 0;
  TruncWork W(d.work, p, m);
  // outputs beyond the chosen rank are zero (up to the rank cap), so that a
  // launch sequence of fixed widths can read rank_cap columns
  const int wcols = d.rank_cap < p ? d.rank_cap : p;
  auto zero_tail = [&](int r) {
    const long stride = (long)C * kSvdThreads;
    for (long e = (long)crank * kSvdThreads + tid; e < (long)p * wcols; e += stride) {
      const int a = (int)(e / wcols), j = (int)(e % wcols);
      if (a >= k || j >= r) W.Rk[(size_t)a * p + j] = 0.0;
    }
    const int vc = d.rank_cap - r;
    for (long e = (long)crank * kSvdThreads + tid; e < (long)m * (vc > 0 ? vc : 0); e += stride) {
      const int c = (int)(e / vc), j = r + (int)(e % vc);
      d.Vout[(size_t)c * d.ldvo + j] = 0.0;
    }
  };
  if (k <= 0 || m <= 0 || d.info[2] != 0) {
    if (crank == 0 && tid == 0) {
      d.info[1] = 0; d.info[3] = 0; *d.frob2 = 0.0;
      if (d.rank_out) *d.rank_out = 0;
      if (d.count) *d.count += 1;
    }
    if (m > 0) zero_tail(0);
    return;
  }
  // Jacobi on X = R^T (n x n) of the QR of A = C (if m < k) or C^T (k_trunc_qrcp)
  const bool cols_of_C = m < k;
  const int n = cols_of_C ? m : k, La = cols_of_C ? k : m, L = n, LV = 2 * n, LS = LV + 2;
  const QrWork Q(W, p, m);
  const int nb = 2 * C, b = (n + nb - 1) / nb;
  // the CTA's column blocks and round buffers: shared memory, or (problems
  // too large for it) a slice of the global work array per CTA
  extern __shared__ double smd[];
  const size_t per_cta = (size_t)4 * b * LS;
  double* sm = global_blocks ? W.Jg + (size_t)crank * per_cta : smd;
  auto owner_blocks = [&](int r) -> double* {
    return global_blocks ? W.Jg + (size_t)r * per_cta : cl.map_shared_rank(smd, r);
  };
  double* home = sm;                    // 2b columns: global columns 2 crank b + h
  double* work = sm + (size_t)2 * b * LS;  // the two blocks of a tournament round
  const int j0 = 2 * crank * b;
  for (long e = tid; e < (long)2 * b * LS; e += kSvdThreads) {
    const int h = (int)(e / LS), i = (int)(e % LS), j = j0 + h;
    double v = 0;
    if (j < n && i < LV) v = i < L ? Q.Rt[(size_t)j * n + i] : ((i - L == j) ? 1.0 : 0.0);
    home[e] = v;
  }
  __syncthreads();
  // exchange of {rotations, largest column norm} over the cluster
  auto csync = [&]() {
    if (global_blocks) __threadfence();
    cl.sync();
  };
  auto exchange = [&](int slot, double rot, double cm) {
    if (tid == 0) { s_ex[slot][0] = rot; s_ex[slot][1] = cm; }
    csync();
    if (tid == 0) {
      double tr = 0, tc = 0;
      for (int r = 0; r < C; ++r) {
        const double* ex = cl.map_shared_rank(&s_ex[slot][0], r);
        tr += ex[0];
        tc = fmax(tc, ex[1]);
      }
      s_tot = tr;
      s_cm = tc;
    }
    __syncthreads();
  };
  exchange(1, 0.0, local_cmax(home, 2 * b, j0, n, L, LV, LS));
  // columns below 1e-2 tol of the largest column norm cannot affect what the
  // truncation keeps (its tail is measured at tol): they are not rotated
  const double zfac = fmax(1e-32, (1e-2 * d.tol) * (1e-2 * d.tol));
  double small2 = s_cm * zfac;
  int sweeps = -1;
  for (int t = 0; t < 40; ++t) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    int nrot = 0;
    {  // (i) all pairs inside this CTA's 2b columns: tournament on 2b slots
      const int np = 2 * b;
      for (int round = 0; round < np - 1; ++round) {
        for (int q = warp; q < b; q += kSvdWarps) {
          auto pos = [&](int u) { return u == 0 ? 0 : ((round + u - 1) % (np - 1)) + 1; };
          int x = pos(q), y = pos(np - 1 - q);
          if (x > y) { const int tt = x; x = y; y = tt; }
          if (j0 + y >= n) continue;
          if (jacobi_pair(home + (size_t)x * LS, home + (size_t)y * LS, L, LV, small2, lane)) ++nrot;
        }
        __syncthreads();
      }
    }
    csync();
    for (int round = 0; round < nb - 1; ++round) {  // (ii) cross pairs of the block tournament
      auto bpos = [&](int u) { return u == 0 ? 0 : ((round + u - 1) % (nb - 1)) + 1; };
      int X = bpos(crank), Y = bpos(nb - 1 - crank);
      if (X > Y) { const int tt = X; X = Y; Y = tt; }
      double* hx = owner_blocks(X >> 1) + (size_t)(X & 1) * b * LS;
      double* hy = owner_blocks(Y >> 1) + (size_t)(Y & 1) * b * LS;
      const bool any = X * b < n && Y * b < n;
      if (any) {
        for (long e = tid; e < (long)b * LS; e += kSvdThreads) {
          work[e] = hx[e];
          work[(size_t)b * LS + e] = hy[e];
        }
        __syncthreads();
        for (int sr = 0; sr < b; ++sr) {
          for (int q = warp; q < b; q += kSvdWarps) {
            const int xi = q, yi = (q + sr) % b;
            if (X * b + xi >= n || Y * b + yi >= n) continue;
            if (jacobi_pair(work + (size_t)xi * LS, work + (size_t)(b + yi) * LS, L, LV, small2, lane)) ++nrot;
          }
          __syncthreads();
        }
        for (long e = tid; e < (long)b * LS; e += kSvdThreads) {
          hx[e] = work[e];
          hy[e] = work[(size_t)b * LS + e];
        }
      }
      csync();
    }
    if (lane == 0 && nrot) atomicAdd(&s_rot, nrot);
    __syncthreads();
    exchange(t & 1, (double)s_rot, local_cmax(home, 2 * b, j0, n, L, LV, LS));
    small2 = s_cm * zfac;
    if (s_tot == 0.0) { sweeps = t + 1; break; }
  }
  // unsorted singular values (column norms of Y = X W) into Dsc
  for (int h = warp; h < 2 * b; h += kSvdWarps) {
    const int j = j0 + h;
    if (j >= n) continue;
    const double* col = home + (size_t)h * LS;
    double t = 0;
    for (int i = lane; i < L; i += 32) t = fma(col[i], col[i], t);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) W.Dsc[j] = sqrt(t);
  }
  __threadfence();
  cl.sync();
  // every CTA: descending order (ties by index), rank rule (identical results)
  double* sig = work;
  int* order = (int*)(work + n);
  const double* sraw = W.Dsc;
  for (int j = tid; j < n; j += kSvdThreads) {
    const double v = __ldcg(sraw + j);
    int rk = 0;
    for (int l = 0; l < n; ++l) {
      const double w = __ldcg(sraw + l);
      rk += (w > v) || (w == v && l < j);
    }
    order[rk] = j;
    sig[rk] = v;
  }
  __syncthreads();
  if (tid == 0) {
    double tot = 0;
    for (int j = 0; j < n; ++j) tot += sig[j] * sig[j];
    double tail = 0;
    int r = n;
    for (int j = n - 1; j >= 0; --j) {  // smallest r with ||s[r:]|| <= tol ||s||
      const double t2 = tail + sig[j] * sig[j];
      if (sqrt(t2) <= d.tol * sqrt(tot)) { tail = t2; r = j; } else break;
    }
    if (tot == 0.0) r = 0;
    if (r > d.rank_cap) r = d.rank_cap;
    s_r = r;
    if (crank == 0) {
      d.info[1] = r;
      d.info[3] = sweeps;
      if (sweeps < 0) d.info[2] = LRFSI_ENOCONV;
      *d.frob2 = tot;
      if (d.rank_out) *d.rank_out = r;
      if (d.count) *d.count += 1;
    }
  }
  __syncthreads();
  if (crank == 0)
    for (int j = tid; j < n; j += kSvdThreads) d.sv[j] = sig[j];
  const int r = s_r;
  // outputs of the CTA's own columns that rank below r: with Y = X W,
  //   left singular vector of A  u = Q [w; 0]   (reflectors applied in reverse)
  //   right singular vector x sigma of A        = P y   (y[i] -> row perm[i])
  // C's left vectors (W_r into Rk, ld p) and sigma-scaled right vectors (Vout)
  // are u, P y (A = C) or P y / sigma, sigma u (A = C^T).
  for (int h = warp; h < 2 * b; h += kSvdWarps) {
    const int j = j0 + h;
    if (j >= n) continue;
    int pos = -1;
    for (int q = 0; q < r; ++q)
      if (order[q] == j) pos = q;
    if (pos < 0) continue;
    const double sg = sig[pos];
    const double* y = home + (size_t)h * LS;
    const double* w = y + L;
    double* u = Q.scr + (size_t)(crank * kSvdWarps + warp) * La;
    for (int i = lane; i < La; i += 32) u[i] = i < n ? w[i] : 0.0;
    __syncwarp();
    for (int jj = n - 1; jj >= 0; --jj) {
      const double tau = Q.tau[jj];
      if (tau == 0.0) continue;
      const double* v = Q.Aw + (size_t)jj * La;
      double t = 0;
      for (int i = jj + lane; i < La; i += 32) t = fma(v[i], u[i], t);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      t *= tau;
      for (int i = jj + lane; i < La; i += 32) u[i] = fma(-t, v[i], u[i]);
      __syncwarp();
    }
    if (cols_of_C) {
      for (int a = lane; a < k; a += 32) W.Rk[(size_t)a * p + pos] = u[a];
      for (int i = lane; i < n; i += 32) d.Vout[(size_t)Q.perm[i] * d.ldvo + pos] = y[i];
    } else {
      const double inv = sg > 0 ? 1.0 / sg : 0.0;
      for (int i = lane; i < n; i += 32) W.Rk[(size_t)Q.perm[i] * p + pos] = y[i] * inv;
      for (int c = lane; c < m; c += 32) d.Vout[(size_t)c * d.ldvo + pos] = u[c] * sg;
    }
  }
  __syncthreads();
  zero_tail(r);
}

constexpr int kPass1Smem = 220 * 1024;
int trunc_pass1(const TruncDesc* d, int n, cudaStream_t s, TruncDesc* d_dev, bool upload) {
  if (upload) LRFSI_CUDA(cudaMemcpyAsync(d_dev, d, sizeof(TruncDesc) * n, cudaMemcpyHostToDevice, s));
  static bool attr = false;
  if (!attr) {
    LRFSI_CUDA(cudaFuncSetAttribute(k_trunc_pass1, cudaFuncAttributeMaxDynamicSharedMemorySize, kPass1Smem));
    attr = true;
  }
  // packed Schur complements in shared memory when every problem of the launch fits
  size_t need = 0;
  for (int i = 0; i < n; ++i) {
    const size_t p = d[i].p > 0 ? (size_t)d[i].p : 0;
    const size_t b = sizeof(double) * (p * (p + 1) / 2 + 2 * p);
    need = b > need ? b : need;
  }
  const size_t smem = need <= (size_t)kPass1Smem ? need : 0;
  account(KC_TRUNC, 0, 0);
  TimedLaunch tl(KC_TRUNC, s);
  k_trunc_pass1<<<n, kSmallThreads, smem, s>>>(d_dev, (int)(smem / sizeof(double)));
  LRFSI_TRY(check_launch("k_trunc_pass1"));
  tl.end(s);
  return LRFSI_OK;
}

int trunc_qr(int n, cudaStream_t s, TruncDesc* d_dev, int write_third, int pmax) {
  static bool attr = false;
  if (!attr) {
    LRFSI_CUDA(cudaFuncSetAttribute(k_trunc_qr, cudaFuncAttributeMaxDynamicSharedMemorySize, kPass1Smem));
    attr = true;
  }
  const size_t need = sizeof(double) * (size_t)pmax * pmax;
  const size_t smem = need <= (size_t)kPass1Smem ? need : 0;
  account(KC_TRUNC, 0, 0);
  TimedLaunch tl(KC_TRUNC, s);
  k_trunc_qr<<<n, kSmallThreads, smem, s>>>(d_dev, write_third, (int)(smem / sizeof(double)));
  LRFSI_TRY(check_launch("k_trunc_qr"));
  tl.end(s);
  return LRFSI_OK;
}

// Cluster size for the SVD: the problems' clusters together should cover the
// SMs about once (16 needs the non-portable cluster size; fall back to 8 if
// the device cannot co-schedule it).
static std::atomic<int> g_svd_cluster{0};  // 0: by the rule below
int svd_cluster(int c) {
  const int old = g_svd_cluster.load();
  if (c >= 0) g_svd_cluster.store(c);
  return old;
}
static int svd_cluster_size(int nprob, size_t smem) {
  static int max16 = -1;
  if (max16 < 0) {
    max16 = 0;
    if (cudaFuncSetAttribute(k_trunc_svd, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 16;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(16, 1, 1);
      cfg.blockDim = dim3(kSvdThreads, 1, 1);
      cfg.dynamicSmemBytes = 16 * 1024;  // within the default dynamic limit (48 KB)
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int ncl = 0;
      if (cudaOccupancyMaxActiveClusters(&ncl, k_trunc_svd, &cfg) == cudaSuccess && ncl > 0) max16 = 1;
    }
    cudaGetLastError();
  }
  (void)smem;
  const int forced = g_svd_cluster.load();
  if (forced == 16 && max16) return 16;
  if (forced >= 2 && forced <= 8) return forced;
  if (nprob <= 9 && max16) return 16;
  if (nprob <= 19) return 8;
  if (nprob <= 38) return 4;
  return 2;
}

int trunc_svd(const TruncDesc* d, int n, cudaStream_t s, TruncDesc* d_dev, bool upload) {
  if (n <= 0) return LRFSI_OK;
  if (upload) LRFSI_CUDA(cudaMemcpyAsync(d_dev, d, sizeof(TruncDesc) * n, cudaMemcpyHostToDevice, s));
  int nmax = 1;
  for (int i = 0; i < n; ++i) {
    const int lo = d[i].p < d[i].m ? d[i].p : d[i].m;
    nmax = nmax > lo ? nmax : lo;
  }
  const int Lmax = nmax;  // the Jacobi matrix is R^T of the QR preconditioning (n x n)
  int C = svd_cluster_size(n, 0);
  size_t smem = 0;
  for (;;) {
    const int b = (nmax + 2 * C - 1) / (2 * C);
    smem = sizeof(double) * (size_t)4 * b * (Lmax + nmax + 2);
    if (smem <= 200 * 1024 || C >= 16) break;
    C *= 2;  // more CTAs per problem: smaller blocks
  }
  // beyond shared memory the column blocks live in the problem's global work
  // array (sized for 16 CTAs by trunc_small_work)
  const int global_blocks = smem > 200 * 1024 ? 1 : 0;
  if (global_blocks) {
    if (C < 16 && svd_cluster_size(1, 0) == 16) C = 16;
    smem = 0;
  }
  static size_t smem_set = 0;
  if (smem > 48 * 1024 && smem > smem_set) {
    LRFSI_CUDA(cudaFuncSetAttribute(k_trunc_svd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(200 * 1024)));
    smem_set = 200 * 1024;
  }
  account(KC_SVD, 0, 0);
  TimedLaunch tl(KC_SVD, s);
  static bool qr_attr = false;
  if (!qr_attr) {
    LRFSI_CUDA(cudaFuncSetAttribute(k_trunc_qrcp, cudaFuncAttributeMaxDynamicSharedMemorySize, kQrSmem));
    qr_attr = true;
  }
  // p x m bounds the Jacobi matrix (L x n from the pass-1 rank k <= p, known
  // only on the device): the launch gets that bound, at most kQrSmem, and the
  // kernel works in shared memory only where its matrix fits what it got
  size_t qsm = 0;
  for (int i = 0; i < n; ++i) {
    const size_t need = (size_t)d[i].p * d[i].m * sizeof(double);
    const size_t got = need < (size_t)kQrSmem ? need : (size_t)kQrSmem;
    if (got > qsm) qsm = got;
  }
  k_trunc_qrcp<<<n, kSmallThreads, qsm, s>>>(d_dev, (int)qsm);
  LRFSI_TRY(check_launch("k_trunc_qrcp"));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(C, n, 1);
  cfg.blockDim = dim3(kSvdThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  LRFSI_CUDA(cudaLaunchKernelEx(&cfg, k_trunc_svd, d_dev, global_blocks));
  LRFSI_TRY(check_launch("k_trunc_svd"));
  tl.end(s);
  return LRFSI_OK;
}

}  // namespace lrfsi
