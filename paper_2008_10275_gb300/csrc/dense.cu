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
#include <cmath>

#include "dense.h"

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
  const GemmDesc<T> g = gb.d[z];
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (m0 >= g.m || n0 >= g.n) return;
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
  if (e >= (long)g.m * g.n) return;
  const int i = (int)(e / g.n), j = (int)(e % g.n);
  T v = 0;
  for (int c = 0; c < ks; ++c) v += part[((long)blockIdx.y * ks + c) * part_stride + e];
  T* cp = g.C + (long)i * g.c_rs + (long)j * g.c_cs;
  if (g.beta != T(0)) v += g.beta * *cp;
  *cp = v;
}

// process-wide split-K workspace (grown on demand, never shrunk)
static void* g_gemm_ws = nullptr;
static size_t g_gemm_ws_bytes = 0;

template <class T>
int gemm_grouped(const GemmDesc<T>* descs, int n, cudaStream_t s) {
  constexpr int kTarget = 2 * 152;  // enough CTAs to occupy every SM's FP64 unit twice
  for (int base = 0; base < n; base += kMaxGemmDescs) {
    GemmBatch<T> gb;
    int cnt = 0, mm = 0, nn = 0, kk = 0;
    for (int i = base; i < n && cnt < kMaxGemmDescs; ++i) {
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
      for (int i = 0; i < cnt; ++i) {
        const GemmDesc<T>& g = gb.d[i];
        fl += 2.0 * g.m * g.n * g.k;
        by += sizeof(T) * ((double)g.m * g.k + (double)g.k * g.n + (g.beta != T(0) ? 2.0 : 1.0) * g.m * g.n);
      }
      account(sizeof(T) == 8 ? KC_GEMM : KC_GEMM32, fl, by);
    }
    TimedLaunch tl(sizeof(T) == 8 ? KC_GEMM : KC_GEMM32, s);
    const long tiles64 = (long)ceil_div(nn, 64) * ceil_div(mm, 64) * cnt;
    if (tiles64 >= kTarget || (mm >= 1024 && nn >= 64)) {
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
    if (ks > 1) {
      const size_t need = sizeof(T) * (size_t)cnt * ks * pstride;
      if (need > g_gemm_ws_bytes) {
        if (g_gemm_ws) cudaFree(g_gemm_ws);
        g_gemm_ws = nullptr;
        g_gemm_ws_bytes = 0;
        LRFSI_CUDA(cudaMalloc(&g_gemm_ws, need));
        g_gemm_ws_bytes = need;
      }
    }
    dim3 grid(ceil_div(nn, 32), ceil_div(mm, 32), cnt * ks);
    k_gemm<T, 32, 32><<<grid, 256, 0, s>>>(gb, ks, (T*)g_gemm_ws, pstride);
    LRFSI_TRY(check_launch("k_gemm"));
    if (ks > 1) {
      dim3 g2(ceil_div(pstride, 256), cnt);
      k_gemm_reduce<T><<<g2, 256, 0, s>>>(gb, ks, (const T*)g_gemm_ws, pstride);
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
                                                     double* __restrict__ work) {
  const GramDesc g = gb.d[blockIdx.z];
  const int tiles_q = (qmax + GBN - 1) / GBN;
  const int ti = blockIdx.x / tiles_q, tj = blockIdx.x % tiles_q;
  const int i0 = ti * GBM, j0 = tj * GBN;
  const int split = blockIdx.y;
  double* out = work + ((size_t)blockIdx.z * nsplit + split) * (size_t)pmax * qmax;
  if (i0 >= g.p || j0 >= g.q) return;
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

__global__ void k_gram_reduce(GramBatch gb, int nsplit, int pmax, int qmax, const double* __restrict__ work) {
  const GramDesc g = gb.d[blockIdx.y];
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)g.p * g.q) return;
  const int i = (int)(idx / g.q), j = (int)(idx % g.q);
  const double* w = work + (size_t)blockIdx.y * nsplit * (size_t)pmax * qmax + (size_t)i * qmax + j;
  double s = 0;
  for (int t = 0; t < nsplit; ++t) s += w[(size_t)t * pmax * qmax];
  g.G[(size_t)i * g.ldg + j] = s;
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
  return (size_t)nbatch * gram_nsplit(nbatch, M, pmax, qmax) * (size_t)pmax * qmax;
}

int gram_batched(const GramDesc* d, int nbatch, long M, double* work, size_t work_len, cudaStream_t s) {
  for (int base = 0; base < nbatch; base += kMaxGemmDescs) {
    GramBatch gb;
    int cnt = 0, pmax = 1, qmax = 1;
    for (int i = base; i < nbatch && cnt < kMaxGemmDescs; ++i, ++cnt) {
      gb.d[cnt] = d[i];
      pmax = pmax > d[i].p ? pmax : d[i].p;
      qmax = qmax > d[i].q ? qmax : d[i].q;
    }
    int nsplit = gram_nsplit(cnt, M, pmax, qmax);
    const size_t fit = work_len / ((size_t)cnt * pmax * qmax);
    if (fit < 1) return fail(LRFSI_EINVAL, "gram workspace too small");
    if ((size_t)nsplit > fit) nsplit = (int)fit;
    {
      double fl = 0, by = 0;
      for (int i = 0; i < cnt; ++i) {
        fl += 2.0 * M * gb.d[i].p * gb.d[i].q;
        by += 8.0 * M * (gb.d[i].A == gb.d[i].B ? gb.d[i].p : gb.d[i].p + gb.d[i].q);
      }
      account(KC_GRAM, fl, by);
    }
    TimedLaunch tl(KC_GRAM, s);
    dim3 grid(ceil_div(pmax, GBM) * ceil_div(qmax, GBN), nsplit, cnt);
    k_gram_partial<<<grid, 256, 0, s>>>(gb, M, nsplit, pmax, qmax, work);
    LRFSI_TRY(check_launch("k_gram_partial"));
    dim3 g2(ceil_div((long)pmax * qmax, 256), cnt);
    k_gram_reduce<<<g2, 256, 0, s>>>(gb, nsplit, pmax, qmax, work);
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
// ldi): rows from the bottom up; in row a every warp computes entries
// Ri[a][b] = -(sum_{l=a+1..b} R[a][l] Ri[l][b]) / R[a][a] with a lane-split dot
// product.  Must be called by the whole block.
__device__ void upper_inverse(const double* R, int ldr, double* Ri, int ldi, int k) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (long e = threadIdx.x; e < (long)k * k; e += blockDim.x) {
    const int i = (int)(e / k), j = (int)(e % k);
    if (j < i) Ri[(size_t)i * ldi + j] = 0.0;
  }
  for (int a = k - 1; a >= 0; --a) {
    const double inv = 1.0 / R[(size_t)a * ldr + a];
    for (int b = a + warp; b < k; b += nw) {
      double sacc = 0;
      for (int l = a + 1 + lane; l <= b; l += 32) sacc += R[(size_t)a * ldr + l] * Ri[(size_t)l * ldi + b];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
      if (lane == 0) Ri[(size_t)a * ldi + b] = (b == a) ? inv : -sacc * inv;
    }
    __syncthreads();
  }
}

// Right-looking Cholesky G = R^T R in place (upper triangle holds R), rows with
// pivot <= drop are marked dropped (keep[i] = 0) and do not update the rest.
__device__ void chol_drop(double* G, int ld, int p, double drop, int* keep) {
  __shared__ double s_piv;
  for (int i = 0; i < p; ++i) {
    if (threadIdx.x == 0) {
      double piv = G[(size_t)i * ld + i];
      keep[i] = (piv > drop && isfinite(piv)) ? 1 : 0;
      s_piv = keep[i] ? sqrt(piv) : 0.0;
    }
    __syncthreads();
    const double r = s_piv;
    if (r > 0) {
      for (int j = i + threadIdx.x; j < p; j += blockDim.x) G[(size_t)i * ld + j] = (j == i) ? r : G[(size_t)i * ld + j] / r;
      __syncthreads();
      const int nt = p - i - 1;
      for (long e = threadIdx.x; e < (long)nt * nt; e += blockDim.x) {
        const int a = i + 1 + (int)(e / nt), b = i + 1 + (int)(e % nt);
        if (b >= a) G[(size_t)a * ld + b] -= G[(size_t)i * ld + a] * G[(size_t)i * ld + b];
      }
    } else {
      for (int j = i + threadIdx.x; j < p; j += blockDim.x) G[(size_t)i * ld + j] = 0.0;
    }
    __syncthreads();
  }
}

size_t trunc_small_work(int p, int m) {
  const size_t n = (size_t)(p > m ? p : m);
  return 4 * (size_t)p * p + 3 * n * n + 2 * (size_t)p * m + 4 * n + 64;
}

// One-sided Jacobi on A (L x n, column-major, n <= L), accumulating the n x n
// rotation Vm (column-major): A_out = A_in Vm with orthogonal columns.  Pairs
// follow a round-robin tournament, one half-warp per pair.  A pair is rotated
// when |a_x . a_y| > 4 eps sqrt(|a_x|^2 |a_y|^2) and neither column is below
// eps times the largest column norm (such columns carry no information at
// working precision).  Returns the sweeps used (or -1 if not converged).
__device__ int jacobi_onesided(double* A, int L, int n, double* Vm, int max_sweeps) {
  const int hl = threadIdx.x & 15, half = threadIdx.x >> 4, nh = blockDim.x >> 4;
  const unsigned mask = (threadIdx.x & 16) ? 0xffff0000u : 0x0000ffffu;
  __shared__ int s_rot;
  __shared__ double s_cmax;
  for (long e = threadIdx.x; e < (long)n * n; e += blockDim.x) Vm[e] = ((e / n) == (e % n)) ? 1.0 : 0.0;
  if (threadIdx.x == 0) s_cmax = 0.0;
  __syncthreads();
  const int np = n + (n & 1);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    // largest squared column norm (for the negligible-column test)
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      double t = 0;
      for (int i = 0; i < L; ++i) t += A[(size_t)j * L + i] * A[(size_t)j * L + i];
      atomicMax((unsigned long long*)&s_cmax, (unsigned long long)__double_as_longlong(t));
    }
    __syncthreads();
    const double small2 = s_cmax * 1e-32;
    for (int round = 0; round < np - 1; ++round) {
      for (int k = half; k < np / 2; k += nh) {
        auto pos = [&](int t) { return t == 0 ? 0 : ((round + t - 1) % (np - 1)) + 1; };
        int x = pos(k), y = pos(np - 1 - k);
        if (x >= n || y >= n) continue;
        if (x > y) { const int t = x; x = y; y = t; }
        double* ax = A + (size_t)x * L;
        double* ay = A + (size_t)y * L;
        double al = 0, be = 0, ga = 0;
        for (int i = hl; i < L; i += 16) {
          const double u = ax[i], v = ay[i];
          al += u * u; be += v * v; ga += u * v;
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          al += __shfl_xor_sync(mask, al, o);
          be += __shfl_xor_sync(mask, be, o);
          ga += __shfl_xor_sync(mask, ga, o);
        }
        if (al > small2 && be > small2 && fabs(ga) > 4.4e-16 * sqrt(al * be)) {
          const double zeta = (be - al) / (2.0 * ga);
          const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
          for (int i = hl; i < L; i += 16) {
            const double u = ax[i], v = ay[i];
            ax[i] = c * u - sn * v;
            ay[i] = sn * u + c * v;
          }
          double* vx = Vm + (size_t)x * n;
          double* vy = Vm + (size_t)y * n;
          for (int i = hl; i < n; i += 16) {
            const double u = vx[i], v = vy[i];
            vx[i] = c * u - sn * v;
            vy[i] = sn * u + c * v;
          }
          if (hl == 0) atomicAdd(&s_rot, 1);
        }
      }
      __syncthreads();
    }
    if (s_rot == 0) return sweep + 1;
    __syncthreads();
  }
  return -1;
}

// Work layout per problem (doubles): Dsc (p) | Rk (p*p) | Rki (p*p) | Y (p*m) |
// C (p*m) | A (n'*n') | Vm (n'*n'), n' = max(p, m).
struct TruncWork {
  double *Dsc, *Rk, *Rki, *Y, *C, *A, *Vm;
  __device__ TruncWork(double* w, int p, int m) {
    const size_t n = (size_t)(p > m ? p : m);
    Dsc = w;
    Rk = Dsc + p;
    Rki = Rk + (size_t)p * p;
    Y = Rki + (size_t)p * p;
    C = Y + (size_t)p * m;
    A = C + (size_t)p * m;
    Vm = A + n * n;
  }
};

// Pass 1: unit-diagonal scaling and a diagonally pivoted (rank-revealing)
// Cholesky of the Gram: at every step the column with the largest remaining
// Schur diagonal is taken; the factorisation stops when that diagonal is
// <= drop (the remaining columns lie in the span of the chosen ones up to a
// relative remainder sqrt(drop)).  Outputs T1 (Q1 = X T1, k columns), the
// core Y = R1 D^{-1} Vc^T (k x m) and info[0] = k.
__global__ void __launch_bounds__(kSmallThreads) k_trunc_pass1(TruncDesc* descs) {
  const TruncDesc d = descs[blockIdx.x];
  const int p = d.p, m = d.m;
  if (p <= 0) {
    if (threadIdx.x == 0) { d.info[0] = 0; d.info[1] = 0; d.info[2] = 0; d.info[4] = 0; *d.frob2 = 0.0; }
    return;
  }
  TruncWork W(d.work, p, m);
  double* G = d.G;         // p x p, original column order; Schur complements in place
  double* R = W.Rk;        // k x p, R[a][b] = R1 entry for permuted columns a, b (b >= a)
  int* perm = d.iwork;
  __shared__ double s_val[33];
  __shared__ int s_idx[33];
  __shared__ int s_k;
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    const double g = G[(size_t)i * p + i];
    W.Dsc[i] = (g > 0 && isfinite(g)) ? 1.0 / sqrt(g) : 0.0;
    perm[i] = i;
  }
  __syncthreads();
  for (long e = threadIdx.x; e < (long)p * p; e += blockDim.x) {
    const int a = (int)(e / p), b = (int)(e % p);
    G[e] = (W.Dsc[a] > 0 && W.Dsc[b] > 0) ? G[e] * W.Dsc[a] * W.Dsc[b] : 0.0;
  }
  if (threadIdx.x == 0) s_k = p;
  __syncthreads();
  for (int i = 0; i < p; ++i) {
    // pivot: largest remaining diagonal (ties: smallest position)
    double best = -1.0;
    int bj = i;
    for (int j = i + threadIdx.x; j < p; j += blockDim.x) {
      const int pj = perm[j];
      const double v = G[(size_t)pj * p + pj];
      if (v > best) { best = v; bj = j; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double v2 = __shfl_xor_sync(0xffffffffu, best, o);
      const int j2 = __shfl_xor_sync(0xffffffffu, bj, o);
      if (v2 > best || (v2 == best && j2 < bj)) { best = v2; bj = j2; }
    }
    if ((threadIdx.x & 31) == 0) { s_val[threadIdx.x >> 5] = best; s_idx[threadIdx.x >> 5] = bj; }
    __syncthreads();
    if (threadIdx.x < 32) {
      const int nw = blockDim.x >> 5;
      best = threadIdx.x < nw ? s_val[threadIdx.x] : -1.0;
      bj = threadIdx.x < nw ? s_idx[threadIdx.x] : 0x7fffffff;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, best, o);
        const int j2 = __shfl_xor_sync(0xffffffffu, bj, o);
        if (v2 > best || (v2 == best && j2 < bj)) { best = v2; bj = j2; }
      }
      if (threadIdx.x == 0) { s_val[32] = best; s_idx[32] = bj; }
    }
    __syncthreads();
    const double piv = s_val[32];
    const int jm = s_idx[32];
    if (!(piv > d.drop) || !isfinite(piv)) {
      if (threadIdx.x == 0) s_k = i;
      break;  // uniform: every thread read the same s_val[0]
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const int t = perm[i];
      perm[i] = perm[jm];
      perm[jm] = t;
    }
    __syncthreads();
    const int pi = perm[i];
    const double r = sqrt(piv);
    // row i of R, indexed by ORIGINAL column (no swaps of earlier rows needed)
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
      const int pj = perm[j];
      R[(size_t)i * p + pj] = j < i ? 0.0 : (j == i ? r : G[(size_t)pi * p + pj] / r);
    }
    __syncthreads();
    const int nt = p - i - 1;
    for (long e = threadIdx.x; e < (long)nt * nt; e += blockDim.x) {
      const int pa = perm[i + 1 + (int)(e / nt)], pb = perm[i + 1 + (int)(e % nt)];
      G[(size_t)pa * p + pb] -= R[(size_t)i * p + pa] * R[(size_t)i * p + pb];
    }
    __syncthreads();
  }
  __syncthreads();
  const int k = s_k;
  if (threadIdx.x == 0) { d.info[0] = k; d.info[4] = 0; }
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
  // Y[a, c] = sum_o R[a][o] ||x_o|| Vc[c, o]   (k x m; R[a][o] = 0 before a in pivot order)
  for (long e = threadIdx.x; e < (long)k * m; e += blockDim.x) {
    const int a = (int)(e / m), c = (int)(e % m);
    double sacc = 0;
    for (int o = 0; o < p; ++o) {
      const double db = W.Dsc[o];
      if (db > 0) sacc += R[(size_t)a * p + o] / db * d.Vc[(size_t)c * d.ldv + o];
    }
    W.Y[(size_t)a * m + c] = sacc;
  }
}

// One Cholesky-QR pass on the k x k Gram Gq (ld p) of the current basis:
// Gq = R^T R, T2 = R^{-1} (k x k, ld p), Y <- R Y.  info[4] = 1 when the
// basis was far from orthonormal (max |Gq_ij - delta_ij| > 0.1), so that one
// more pass is needed before the SVD.
__global__ void __launch_bounds__(kSmallThreads) k_trunc_qr(TruncDesc* descs) {
  const TruncDesc d = descs[blockIdx.x];
  const int p = d.p, m = d.m;
  __shared__ int s_k, s_bad;
  __shared__ double s_dev;
  if (threadIdx.x == 0) { s_k = p > 0 ? d.info[0] : 0; s_bad = 0; s_dev = 0.0; }
  __syncthreads();
  const int k = s_k;
  if (k <= 0 || m <= 0) return;
  TruncWork W(d.work, p, m);
  double* R = W.Rk;  // k x k (ld k)
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
    d.info[4] = (s_dev > 0.1) ? 1 : 0;
    if (s_bad) d.info[2] = LRFSI_EBREAKDOWN;
  }
  __syncthreads();
  if (s_bad) return;
  upper_inverse(R, k, W.Rki, k, k);
  __syncthreads();
  for (long e = threadIdx.x; e < (long)k * k; e += blockDim.x) {
    const int a = (int)(e / k), b = (int)(e % k);
    d.T2[(size_t)a * p + b] = W.Rki[e];
  }
  // Y <- R Y (k x m), via C
  for (long e = threadIdx.x; e < (long)k * m; e += blockDim.x) {
    const int a = (int)(e / m), c = (int)(e % m);
    double sacc = 0;
    for (int l = a; l < k; ++l) sacc += R[(size_t)a * k + l] * W.Y[(size_t)l * m + c];
    W.C[e] = sacc;
  }
  __syncthreads();
  for (long e = threadIdx.x; e < (long)k * m; e += blockDim.x) W.Y[e] = W.C[e];
}

// SVD of the core C = Y (k x m) by one-sided Jacobi, rank rule, output
// T1 <- T2 W_r (k x r, ld p; the tall result is Q_last T1) and
// Vout = Z_r diag(s_r).
__global__ void __launch_bounds__(kSmallThreads) k_trunc_svd(TruncDesc* descs) {
  const TruncDesc d = descs[blockIdx.x];
  const int p = d.p, m = d.m;
  __shared__ int s_k, s_r;
  if (threadIdx.x == 0) s_k = p > 0 ? d.info[0] : 0;
  __syncthreads();
  const int k = s_k;
  if (k <= 0 || m <= 0 || d.info[2] != 0) {
    if (threadIdx.x == 0) { d.info[1] = 0; d.info[3] = 0; *d.frob2 = 0.0; }
    return;
  }
  TruncWork W(d.work, p, m);
  const int n = k < m ? k : m, L = k < m ? m : k;
  const bool cols_of_C = m <= k;  // A = C (L = k, n = m) else A = C^T (L = m, n = k)
  for (long e = threadIdx.x; e < (long)L * n; e += blockDim.x) {
    const int col = (int)(e / L), i = (int)(e % L);
    W.A[e] = cols_of_C ? W.Y[(size_t)i * m + col] : W.Y[(size_t)col * m + i];
  }
  __syncthreads();
  const int sweeps = jacobi_onesided(W.A, L, n, W.Vm, 40);
  __syncthreads();
  double* sraw = W.C;  // n unsorted singular values
  double* sig = d.sv;
  int* order = d.iwork;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double sacc = 0;
    for (int i = 0; i < L; ++i) sacc += W.A[(size_t)j * L + i] * W.A[(size_t)j * L + i];
    sraw[j] = sqrt(sacc);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    int rank = 0;
    for (int l = 0; l < n; ++l) rank += (sraw[l] > sraw[j]) || (sraw[l] == sraw[j] && l < j);
    order[rank] = j;
    sig[rank] = sraw[j];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
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
    d.info[1] = r;
    d.info[3] = sweeps;
    if (sweeps < 0) d.info[2] = LRFSI_ENOCONV;
    *d.frob2 = tot;
  }
  __syncthreads();
  const int r = s_r;
  double* Wr = W.Rk;  // k x r
  for (long e = threadIdx.x; e < (long)k * r; e += blockDim.x) {
    const int a = (int)(e / r), j = (int)(e % r);
    const int col = order[j];
    Wr[e] = cols_of_C ? (sig[j] > 0 ? W.A[(size_t)col * L + a] / sig[j] : 0.0) : W.Vm[(size_t)col * n + a];
  }
  for (long e = threadIdx.x; e < (long)m * r; e += blockDim.x) {
    const int c = (int)(e / r), j = (int)(e % r);
    const int col = order[j];
    d.Vout[(size_t)c * d.ldvo + j] = cols_of_C ? W.Vm[(size_t)col * n + c] * sig[j] : W.A[(size_t)col * L + c];
  }
  __syncthreads();
  // T1 = T2 W_r with T2 upper triangular (k x k, ld p)
  for (long e = threadIdx.x; e < (long)k * r; e += blockDim.x) {
    const int a = (int)(e / r), j = (int)(e % r);
    double sacc = 0;
    for (int l = a; l < k; ++l) sacc += d.T2[(size_t)a * p + l] * Wr[(size_t)l * r + j];
    d.T1[(size_t)a * p + j] = sacc;
  }
}

int trunc_pass1(const TruncDesc* d, int n, cudaStream_t s, TruncDesc* d_dev) {
  LRFSI_CUDA(cudaMemcpyAsync(d_dev, d, sizeof(TruncDesc) * n, cudaMemcpyHostToDevice, s));
  account(KC_TRUNC, 0, 0);
  TimedLaunch tl(KC_TRUNC, s);
  k_trunc_pass1<<<n, kSmallThreads, 0, s>>>(d_dev);
  LRFSI_TRY(check_launch("k_trunc_pass1"));
  tl.end(s);
  return LRFSI_OK;
}

int trunc_qr(int n, cudaStream_t s, TruncDesc* d_dev) {
  account(KC_TRUNC, 0, 0);
  TimedLaunch tl(KC_TRUNC, s);
  k_trunc_qr<<<n, kSmallThreads, 0, s>>>(d_dev);
  LRFSI_TRY(check_launch("k_trunc_qr"));
  tl.end(s);
  return LRFSI_OK;
}

int trunc_svd(int n, cudaStream_t s, TruncDesc* d_dev) {
  account(KC_TRUNC, 0, 0);
  TimedLaunch tl(KC_TRUNC, s);
  k_trunc_svd<<<n, kSmallThreads, 0, s>>>(d_dev);
  LRFSI_TRY(check_launch("k_trunc_svd"));
  tl.end(s);
  return LRFSI_OK;
}

}  // namespace lrfsi
