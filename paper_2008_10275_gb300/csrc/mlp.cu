// Learned initial guess: an MLP (mu_s, nu_f) -> 128 -> 128 -> k with exact-erf
// GELU, BF16 weights, FP32 biases and FP32 accumulation; its gradients, Adam,
// and the start x0 = offset + s .* (Phi c) with Dirichlet rows set to b_D.
// (Not a method of the paper: a serving-style start for the median Newton
// iteration of Algorithm 1.)
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>

#include "dense.h"
#include "mesh.h"

namespace lrfsi {

constexpr int kMlpLayers = 3;

struct MlpDims {
  int n[kMlpLayers + 1];
  long woff[kMlpLayers], boff[kMlpLayers];  // offsets into the packed parameter vector
  long total;
};

static MlpDims mlp_dims(int n0, int n1, int n2, int n3) {
  MlpDims d;
  d.n[0] = n0; d.n[1] = n1; d.n[2] = n2; d.n[3] = n3;
  long o = 0;
  for (int l = 0; l < kMlpLayers; ++l) {
    d.woff[l] = o;
    o += (long)d.n[l + 1] * d.n[l];
    d.boff[l] = o;
    o += d.n[l + 1];
  }
  d.total = o;
  return d;
}

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.3989422804014327f;
}

// out[b][j] = sum_i W[j][i] a[b][i] + bias[j]; z keeps the pre-activation,
// act applies GELU.  Thread per (b, j).
__global__ void k_dense_fwd(const __nv_bfloat16* __restrict__ W, const float* __restrict__ bias,
                            const float* __restrict__ a, int B, int nin, int nout, float* __restrict__ z,
                            float* __restrict__ out, int act) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)B * nout) return;
  const int b = (int)(e / nout), j = (int)(e % nout);
  float s = bias[j];
  const __nv_bfloat16* w = W + (long)j * nin;
  const float* ab = a + (long)b * nin;
  for (int i = 0; i < nin; ++i) s = fmaf(__bfloat162float(w[i]), ab[i], s);
  if (z) z[e] = s;
  out[e] = act ? gelu_f(s) : s;
}

// g_in[b][i] = (sum_j g[b][j] W[j][i]) * gelu'(z_prev[b][i])   (z_prev null: no GELU)
__global__ void k_dense_bwd_input(const __nv_bfloat16* __restrict__ W, const float* __restrict__ g, int B, int nin,
                                  int nout, const float* __restrict__ zprev, float* __restrict__ gin) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)B * nin) return;
  const int b = (int)(e / nin), i = (int)(e % nin);
  float s = 0.f;
  for (int j = 0; j < nout; ++j) s = fmaf(g[(long)b * nout + j], __bfloat162float(W[(long)j * nin + i]), s);
  gin[e] = zprev ? s * gelu_grad_f(zprev[e]) : s;
}

// dW[j][i] = sum_b g[b][j] a[b][i], db[j] = sum_b g[b][j]   (fixed order over b)
__global__ void k_dense_bwd_weight(const float* __restrict__ g, const float* __restrict__ a, int B, int nin,
                                   int nout, float* __restrict__ dW, float* __restrict__ db) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)nout * (nin + 1)) return;
  const int j = (int)(e / (nin + 1)), i = (int)(e % (nin + 1));
  float s = 0.f;
  if (i < nin)
    for (int b = 0; b < B; ++b) s = fmaf(g[(long)b * nout + j], a[(long)b * nin + i], s);
  else
    for (int b = 0; b < B; ++b) s += g[(long)b * nout + j];
  if (i < nin) dW[(long)j * nin + i] = s;
  else db[j] = s;
}

// g = 2 (y - t) / (B k); loss partial per block
__global__ void k_mse_grad(const float* __restrict__ y, const float* __restrict__ t, long n, float scale,
                           float* __restrict__ g, float* __restrict__ sq) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  float d = 0.f;
  if (e < n) {
    d = y[e] - t[e];
    g[e] = 2.0f * d * scale;
  }
  __shared__ float red[256];
  red[threadIdx.x] = d * d;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) sq[blockIdx.x] = red[0];
}

__global__ void k_sum(const float* __restrict__ x, int n, float scale, float* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += x[i];
    *out = s * scale;
  }
}

// Adam (Kingma & Ba) on the FP32 master parameters, then refresh the BF16
// copies (the forward pass reads BF16 weights and FP32 biases).
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long n, float lr, float b1, float b2, float eps, float c1, float c2,
                       __nv_bfloat16* __restrict__ pbf) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float ge = g[e];
  const float me = b1 * m[e] + (1.f - b1) * ge;
  const float ve = b2 * v[e] + (1.f - b2) * ge * ge;
  m[e] = me;
  v[e] = ve;
  const float pe = p[e] - lr * (me / c1) / (sqrtf(ve / c2) + eps);
  p[e] = pe;
  pbf[e] = __float2bfloat16_rn(pe);
}

__global__ void k_to_bf16(const float* __restrict__ p, long n, __nv_bfloat16* __restrict__ pbf) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) pbf[e] = __float2bfloat16_rn(p[e]);
}

// Box scaling of the parameters: z = 2 (p - lo) / (hi - lo) - 1 per coordinate.
__global__ void k_scale_params(const double* __restrict__ mu, const double* __restrict__ nu, int B, double mlo,
                               double mhi, double nlo, double nhi, float* __restrict__ Z) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  Z[2 * b] = (float)(2.0 * (mu[b] - mlo) / (mhi - mlo) - 1.0);
  Z[2 * b + 1] = (float)(2.0 * (nu[b] - nlo) / (nhi - nlo) - 1.0);
}

// Snapshot statistics per DOF: off[i] = mean_j X_j[i], ss[i] = sum_j (X_j[i] - off[i])^2.
// X: n problem-major rows of length ldx.
__global__ void k_snap_mean(const double* __restrict__ X, int ldx, int n, long M, double* __restrict__ off,
                            double* __restrict__ ss) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  double s = 0;
  for (int j = 0; j < n; ++j) s += X[(long)j * ldx + i];
  const double mean = s / n;
  double q = 0;
  for (int j = 0; j < n; ++j) {
    const double d = X[(long)j * ldx + i] - mean;
    q += d * d;
  }
  off[i] = mean;
  ss[i] = q;
}

// One block per field f: scale[f] = RMS of the centred snapshot values of that
// field (1 where the field does not vary), then fs[i] = scale[field[i]].
__global__ void k_field_scale(const double* __restrict__ ss, const int* __restrict__ field, long M, int n,
                              double* __restrict__ fscale) {
  const int f = blockIdx.x;
  double s = 0;
  long c = 0;
  for (long i = threadIdx.x; i < M; i += blockDim.x)
    if (field[i] == f) {
      s += ss[i];
      ++c;
    }
  __shared__ double rs[256];
  __shared__ long rc[256];
  rs[threadIdx.x] = s;
  rc[threadIdx.x] = c;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      rs[threadIdx.x] += rs[threadIdx.x + o];
      rc[threadIdx.x] += rc[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double v = rc[0] > 0 ? sqrt(rs[0] / ((double)rc[0] * n)) : 0.0;
    fscale[f] = v > 0 ? v : 1.0;
  }
}

__global__ void k_fill_field(const double* __restrict__ fscale, const int* __restrict__ field, long M,
                             double* __restrict__ fs) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) fs[i] = fscale[field[i]];
}

// Y (M x n, row-major) = (X_j[i] - off[i]) / fs[i]
__global__ void k_scale_snap(const double* __restrict__ X, int ldx, int n, long M, const double* __restrict__ off,
                             const double* __restrict__ fs, double* __restrict__ Y) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * n) return;
  const long i = e / n;
  const int j = (int)(e % n);
  Y[e] = (X[(long)j * ldx + i] - off[i]) / fs[i];
}

// Regression targets: cs[l] = RMS over snapshots of coefficient l (1 if zero),
// T[j][l] = C[j][l] / cs[l] in FP32.
__global__ void k_coef_targets(const double* __restrict__ Cc, int ldc, int n, int k, double* __restrict__ cs,
                               float* __restrict__ T) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= k) return;
  double q = 0;
  for (int j = 0; j < n; ++j) q += Cc[(long)j * ldc + l] * Cc[(long)j * ldc + l];
  double r = sqrt(q / n);
  if (!(r > 0)) r = 1.0;
  cs[l] = r;
  for (int j = 0; j < n; ++j) T[(long)j * k + l] = (float)(Cc[(long)j * ldc + l] / r);
}

// x0 = offset + fs .* (Phi (cs .* c_b)), Dirichlet rows -> b_D.  Writes the
// problem-major start X (B x M) and its column-major copy Xt (M x B) for the
// residual check.
__global__ void k_learned_start(const double* __restrict__ Phi, int ldphi, int k, const float* __restrict__ C,
                                const double* __restrict__ cs, const double* __restrict__ fs,
                                const double* __restrict__ off, const char* __restrict__ ident,
                                const double* __restrict__ bD, long M, int B, double* __restrict__ X,
                                double* __restrict__ Xt) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * B) return;
  const long i = e / B;
  const int b = (int)(e % B);
  double v;
  if (ident[i]) {
    v = bD[i];
  } else {
    double s = 0;
    for (int l = 0; l < k; ++l) s += Phi[i * ldphi + l] * (double)C[(long)b * k + l] * cs[l];
    v = off[i] + fs[i] * s;
  }
  Xt[e] = v;
  X[(long)b * M + i] = v;
}

// Columns whose start does not reduce the residual below that of b_D fall
// back to b_D: flag[b] = n2[b] >= n2D[b].
__global__ void k_start_fallback(const double* __restrict__ n2, const double* __restrict__ n2D,
                                 const double* __restrict__ bD, long M, int B, double* __restrict__ X,
                                 int* __restrict__ flag) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * B) return;
  const int b = (int)(e / M);
  const long i = e % M;
  const bool fb = !(n2[b] < n2D[b]);
  if (fb) X[e] = bD[i];
  if (i == 0) flag[b] = fb ? 1 : 0;
}

// Factors of the learned start relative to the median solution of subset k:
// X0 - x~_k 1^T = U0 V0^T with U0 = [offset - x~_k | diag(fs) Phi] (M x (k+1))
// and V0 = [1 | C diag(cs)] (m x (k+1)); Dirichlet rows of U0 are zero.
__global__ void k_learned_u0(const double* __restrict__ Phi, int ldphi, int k, const double* __restrict__ fs,
                             const double* __restrict__ off, const double* __restrict__ xt,
                             const char* __restrict__ ident, long M, double* __restrict__ U0, int ldu0) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * (k + 1)) return;
  const long i = e / (k + 1);
  const int l = (int)(e % (k + 1));
  double v = 0.0;
  if (!ident[i]) v = l == 0 ? off[i] - xt[i] : fs[i] * Phi[i * ldphi + l - 1];
  U0[i * ldu0 + l] = v;
}

__global__ void k_learned_v0(const float* __restrict__ C, int k, const double* __restrict__ cs, int B,
                             double* __restrict__ V0, int ldv0) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)B * (k + 1)) return;
  const int b = (int)(e / (k + 1)), l = (int)(e % (k + 1));
  V0[(size_t)b * ldv0 + l] = l == 0 ? 1.0 : cs[l - 1] * (double)C[(size_t)b * k + l - 1];
}

}  // namespace lrfsi

struct lrfsi_mlp_s {
  lrfsi::MlpDims d;
  lrfsi::DevBuf<float> p, g, m, v, act, z, gb, sq, loss;
  lrfsi::DevBuf<__nv_bfloat16> pbf;
  int t = 0;
  int cap_batch = 0;
};

using namespace lrfsi;

static int mlp_reserve(lrfsi_mlp_s* h, int B) {
  if (B <= h->cap_batch) return LRFSI_OK;
  long width = 0;
  for (int l = 0; l <= kMlpLayers; ++l) width += h->d.n[l];
  LRFSI_TRY(h->act.alloc((size_t)B * width));
  LRFSI_TRY(h->z.alloc((size_t)B * width));
  int wmax = 0;
  for (int l = 0; l <= kMlpLayers; ++l) wmax = wmax > h->d.n[l] ? wmax : h->d.n[l];
  LRFSI_TRY(h->gb.alloc((size_t)2 * B * wmax));
  LRFSI_TRY(h->sq.alloc((size_t)ceil_div((long)B * h->d.n[kMlpLayers], 256) + 1));
  h->cap_batch = B;
  return LRFSI_OK;
}

// activation offsets: layer l's input activations at act + B * sum_{i<l} n[i]
static long act_off(const MlpDims& d, int l, int B) {
  long o = 0;
  for (int i = 0; i < l; ++i) o += (long)B * d.n[i];
  return o;
}

static int mlp_forward_impl(lrfsi_mlp_s* h, const float* Z, int B, float* Y, cudaStream_t s, bool keep) {
  LRFSI_TRY(mlp_reserve(h, B));
  const MlpDims& d = h->d;
  LRFSI_CUDA(cudaMemcpyAsync(h->act.p, Z, sizeof(float) * B * d.n[0], cudaMemcpyDeviceToDevice, s));
  for (int l = 0; l < kMlpLayers; ++l) {
    const float* a = h->act.p + act_off(d, l, B);
    float* zo = h->z.p + act_off(d, l + 1, B);
    float* out = (l == kMlpLayers - 1 && !keep) ? Y : h->act.p + act_off(d, l + 1, B);
    const long n = (long)B * d.n[l + 1];
    k_dense_fwd<<<ceil_div(n, 128), 128, 0, s>>>(h->pbf.p + d.woff[l], h->p.p + d.boff[l], a, B, d.n[l], d.n[l + 1],
                                                  keep ? zo : nullptr, out, l < kMlpLayers - 1);
    LRFSI_TRY(check_launch("k_dense_fwd"));
  }
  if (keep && Y)
    LRFSI_CUDA(cudaMemcpyAsync(Y, h->act.p + act_off(d, kMlpLayers, B), sizeof(float) * B * d.n[kMlpLayers],
                               cudaMemcpyDeviceToDevice, s));
  return LRFSI_OK;
}

extern "C" {

int lrfsi_mlp_create(int n_in, int n_h1, int n_h2, int n_out, lrfsi_mlp_h* out) {
  if (!out || n_in < 1 || n_h1 < 1 || n_h2 < 1 || n_out < 1 || n_h1 > 4096 || n_h2 > 4096 || n_out > 4096)
    return fail(LRFSI_EINVAL, "lrfsi_mlp_create: bad sizes");
  lrfsi_mlp_s* h = new (std::nothrow) lrfsi_mlp_s();
  if (!h) return fail(LRFSI_ENOMEM, "lrfsi_mlp_create: host allocation");
  h->d = mlp_dims(n_in, n_h1, n_h2, n_out);
  int st = h->p.alloc(h->d.total);
  if (st == LRFSI_OK) st = h->g.alloc(h->d.total);
  if (st == LRFSI_OK) st = h->m.alloc(h->d.total);
  if (st == LRFSI_OK) st = h->v.alloc(h->d.total);
  if (st == LRFSI_OK) st = h->pbf.alloc(h->d.total);
  if (st == LRFSI_OK) st = h->loss.alloc(1);
  if (st == LRFSI_OK && cudaMemset(h->p.p, 0, sizeof(float) * h->d.total) != cudaSuccess) st = LRFSI_ECUDA;
  if (st == LRFSI_OK && cudaMemset(h->m.p, 0, sizeof(float) * h->d.total) != cudaSuccess) st = LRFSI_ECUDA;
  if (st == LRFSI_OK && cudaMemset(h->v.p, 0, sizeof(float) * h->d.total) != cudaSuccess) st = LRFSI_ECUDA;
  if (st != LRFSI_OK) {
    delete h;
    return st;
  }
  *out = h;
  return LRFSI_OK;
}

int lrfsi_mlp_destroy(lrfsi_mlp_h h) {
  delete h;
  return LRFSI_OK;
}

int64_t lrfsi_mlp_num_params(lrfsi_mlp_h h) { return h ? h->d.total : 0; }

int lrfsi_mlp_set_params(lrfsi_mlp_h h, const float* packed_host) {
  if (!h || !packed_host) return fail(LRFSI_EINVAL, "lrfsi_mlp_set_params: null argument");
  LRFSI_CUDA(cudaMemcpy(h->p.p, packed_host, sizeof(float) * h->d.total, cudaMemcpyHostToDevice));
  LRFSI_CUDA(cudaMemset(h->m.p, 0, sizeof(float) * h->d.total));
  LRFSI_CUDA(cudaMemset(h->v.p, 0, sizeof(float) * h->d.total));
  h->t = 0;
  k_to_bf16<<<ceil_div(h->d.total, 256), 256>>>(h->p.p, h->d.total, h->pbf.p);
  LRFSI_TRY(check_launch("k_to_bf16"));
  LRFSI_CUDA(cudaDeviceSynchronize());
  return LRFSI_OK;
}

int lrfsi_mlp_get_params(lrfsi_mlp_h h, float* packed_host) {
  if (!h || !packed_host) return fail(LRFSI_EINVAL, "lrfsi_mlp_get_params: null argument");
  LRFSI_CUDA(cudaDeviceSynchronize());
  LRFSI_CUDA(cudaMemcpy(packed_host, h->p.p, sizeof(float) * h->d.total, cudaMemcpyDeviceToHost));
  return LRFSI_OK;
}

int lrfsi_mlp_forward(lrfsi_mlp_h h, const float* Z, int B, float* Y, lrfsi_stream_t stream) {
  if (!h || !Z || !Y || B < 1) return fail(LRFSI_EINVAL, "lrfsi_mlp_forward: bad argument");
  return mlp_forward_impl(h, Z, B, Y, (cudaStream_t)stream, false);
}

int lrfsi_mlp_gradients(lrfsi_mlp_h h, const float* Z, const float* T, int B, float* grad, float* loss,
                        lrfsi_stream_t stream) {
  if (!h || !Z || !T || B < 1) return fail(LRFSI_EINVAL, "lrfsi_mlp_gradients: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  const MlpDims& d = h->d;
  LRFSI_TRY(mlp_forward_impl(h, Z, B, nullptr, s, true));
  float* G = grad ? grad : h->g.p;
  const int L = kMlpLayers;
  const long nout = (long)B * d.n[L];
  int wmax = 0;
  for (int l = 0; l <= kMlpLayers; ++l) wmax = wmax > d.n[l] ? wmax : d.n[l];
  float* gcur = h->gb.p;
  float* gnext = h->gb.p + (size_t)B * wmax;
  const int nblk = ceil_div(nout, 256);
  k_mse_grad<<<nblk, 256, 0, s>>>(h->act.p + act_off(d, L, B), T, nout, 1.0f / (float)nout, gcur, h->sq.p);
  LRFSI_TRY(check_launch("k_mse_grad"));
  k_sum<<<1, 32, 0, s>>>(h->sq.p, nblk, 1.0f / (float)nout, loss ? loss : h->loss.p);
  LRFSI_TRY(check_launch("k_sum"));
  for (int l = L - 1; l >= 0; --l) {
    const long nw = (long)d.n[l + 1] * (d.n[l] + 1);
    k_dense_bwd_weight<<<ceil_div(nw, 128), 128, 0, s>>>(gcur, h->act.p + act_off(d, l, B), B, d.n[l], d.n[l + 1],
                                                         G + d.woff[l], G + d.boff[l]);
    LRFSI_TRY(check_launch("k_dense_bwd_weight"));
    if (l > 0) {
      const long ni = (long)B * d.n[l];
      k_dense_bwd_input<<<ceil_div(ni, 128), 128, 0, s>>>(h->pbf.p + d.woff[l], gcur, B, d.n[l], d.n[l + 1],
                                                          h->z.p + act_off(d, l, B), gnext);
      LRFSI_TRY(check_launch("k_dense_bwd_input"));
      float* t = gcur;
      gcur = gnext;
      gnext = t;
    }
  }
  return LRFSI_OK;
}

int lrfsi_mlp_train(lrfsi_mlp_h h, const float* Z, const float* T, int B, int epochs, float lr, float* loss_host,
                    lrfsi_stream_t stream) {
  if (!h || !Z || !T || B < 1 || epochs < 0 || !(lr > 0)) return fail(LRFSI_EINVAL, "lrfsi_mlp_train: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  LRFSI_TRY(mlp_reserve(h, B));
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int e = 0; e < epochs; ++e) {
    LRFSI_TRY(lrfsi_mlp_gradients(h, Z, T, B, nullptr, h->loss.p, stream));
    h->t += 1;
    const float c1 = 1.f - powf(b1, (float)h->t), c2 = 1.f - powf(b2, (float)h->t);
    k_adam<<<ceil_div(h->d.total, 256), 256, 0, s>>>(h->p.p, h->g.p, h->m.p, h->v.p, h->d.total, lr, b1, b2, eps, c1,
                                                      c2, h->pbf.p);
    LRFSI_TRY(check_launch("k_adam"));
  }
  if (loss_host) {
    LRFSI_CUDA(cudaMemcpyAsync(loss_host, h->loss.p, sizeof(float), cudaMemcpyDeviceToHost, s));
    LRFSI_CUDA(cudaStreamSynchronize(s));
  }
  return LRFSI_OK;
}

int lrfsi_learned_fit(lrfsi_mesh_h mesh, lrfsi_mlp_h h, const double* mu_h, const double* nu_h, int n,
                      const double* box, const double* X, int ldx, int k, int epochs, float lr, double* Phi,
                      int ldphi, double* coef_scale, double* field_scale, double* offset, float* loss_host,
                      double* sigma_host, lrfsi_stream_t stream) {
  if (!mesh || !h || !mu_h || !nu_h || !box || !X || !Phi || !coef_scale || !field_scale || !offset || n < 1 ||
      k < 1 || k > n || ldx < mesh->h.M || ldphi < k || epochs < 0 || !(lr > 0) || h->d.n[0] != 2 ||
      h->d.n[kMlpLayers] != k || !(box[1] > box[0]) || !(box[3] > box[2]))
    return fail(LRFSI_EINVAL, "lrfsi_learned_fit: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  const long M = mesh->h.M;
  DevBuf<double> ss, fsc, Y, Cc, mu, nu;
  DevBuf<int> field;
  DevBuf<float> Z, T;
  LRFSI_TRY(ss.alloc(M));
  LRFSI_TRY(fsc.alloc(8));
  LRFSI_TRY(Y.alloc((size_t)M * n));
  LRFSI_TRY(Cc.alloc((size_t)n * k));
  LRFSI_TRY(Z.alloc((size_t)2 * n));
  LRFSI_TRY(T.alloc((size_t)n * k));
  LRFSI_TRY(field.upload(mesh->h.dof_field, s));
  std::vector<double> muv(mu_h, mu_h + n), nuv(nu_h, nu_h + n);
  LRFSI_TRY(mu.upload(muv, s));
  LRFSI_TRY(nu.upload(nuv, s));
  k_snap_mean<<<ceil_div(M, 256), 256, 0, s>>>(X, ldx, n, M, offset, ss.p);
  LRFSI_TRY(check_launch("k_snap_mean"));
  k_field_scale<<<5, 256, 0, s>>>(ss.p, field.p, M, n, fsc.p);
  LRFSI_TRY(check_launch("k_field_scale"));
  k_fill_field<<<ceil_div(M, 256), 256, 0, s>>>(fsc.p, field.p, M, field_scale);
  LRFSI_TRY(check_launch("k_fill_field"));
  k_scale_snap<<<ceil_div(M * n, 256), 256, 0, s>>>(X, ldx, n, M, offset, field_scale, Y.p);
  LRFSI_TRY(check_launch("k_scale_snap"));
  LRFSI_TRY(lrfsi_pod(mesh, Y.p, n, n, k, Phi, ldphi, Cc.p, k, sigma_host, stream));
  k_coef_targets<<<ceil_div(k, 64), 64, 0, s>>>(Cc.p, k, n, k, coef_scale, T.p);
  LRFSI_TRY(check_launch("k_coef_targets"));
  k_scale_params<<<ceil_div(n, 128), 128, 0, s>>>(mu.p, nu.p, n, box[0], box[1], box[2], box[3], Z.p);
  LRFSI_TRY(check_launch("k_scale_params"));
  // step schedule: a third of the epochs each at lr, lr / 4 and lr / 16
  const int e1 = epochs / 3, e2 = epochs / 3, e3 = epochs - e1 - e2;
  LRFSI_TRY(lrfsi_mlp_train(h, Z.p, T.p, n, e1, lr, nullptr, stream));
  LRFSI_TRY(lrfsi_mlp_train(h, Z.p, T.p, n, e2, lr * 0.25f, nullptr, stream));
  LRFSI_TRY(lrfsi_mlp_train(h, Z.p, T.p, n, e3, lr * 0.0625f, loss_host, stream));
  LRFSI_CUDA(cudaStreamSynchronize(s));
  return LRFSI_OK;
}

int lrfsi_learned_start(lrfsi_mesh_h mesh, lrfsi_mlp_h h, const double* mu_h, const double* nu_h, int B,
                        const double* box, const double* Phi, int ldphi, int k, const double* coef_scale,
                        const double* field_scale, const double* offset, double* X, int* fallback_host,
                        lrfsi_stream_t stream) {
  if (!mesh || !h || !mu_h || !nu_h || !box || !Phi || !coef_scale || !field_scale || !offset || !X || B < 1 ||
      k < 1 || ldphi < k || h->d.n[0] != 2 || h->d.n[kMlpLayers] != k || !(box[1] > box[0]) || !(box[3] > box[2]))
    return fail(LRFSI_EINVAL, "lrfsi_learned_start: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  const long M = mesh->h.M;
  DevBuf<float> Z, C;
  DevBuf<char> ident;
  DevBuf<double> mu, nu, Xt, R, n2, n2D, work;
  DevBuf<int> flag;
  LRFSI_TRY(Z.alloc((size_t)2 * B));
  LRFSI_TRY(C.alloc((size_t)B * k));
  LRFSI_TRY(Xt.alloc((size_t)M * B));
  LRFSI_TRY(R.alloc((size_t)M * B));
  LRFSI_TRY(n2.alloc(B));
  LRFSI_TRY(n2D.alloc(B));
  LRFSI_TRY(flag.alloc(B));
  LRFSI_TRY(work.alloc((size_t)ceil_div(M, 256) * B));
  std::vector<double> muv(mu_h, mu_h + B), nuv(nu_h, nu_h + B);
  LRFSI_TRY(mu.upload(muv, s));
  LRFSI_TRY(nu.upload(nuv, s));
  std::vector<char> id(mesh->h.ident.begin(), mesh->h.ident.end());
  LRFSI_TRY(ident.upload(id, s));
  k_scale_params<<<ceil_div(B, 128), 128, 0, s>>>(mu.p, nu.p, B, box[0], box[1], box[2], box[3], Z.p);
  LRFSI_TRY(check_launch("k_scale_params"));
  LRFSI_TRY(mlp_forward_impl(h, Z.p, B, C.p, s, false));
  k_learned_start<<<ceil_div(M * B, 256), 256, 0, s>>>(Phi, ldphi, k, C.p, coef_scale, field_scale, offset, ident.p,
                                                       mesh->bD.p, M, B, X, Xt.p);
  LRFSI_TRY(check_launch("k_learned_start"));
  // fallback test: residual of the learned start against that of b_D, per column
  LRFSI_TRY(launch_residual(mesh, Xt.p, B, B, nullptr, mu.p, nu.p, R.p, B, s));
  LRFSI_TRY(launch_colnorm2(R.p, M, B, B, n2.p, work.p, work.n, s));
  LRFSI_TRY(launch_residual(mesh, mesh->bD.p, 0, B, nullptr, mu.p, nu.p, R.p, B, s));
  LRFSI_TRY(launch_colnorm2(R.p, M, B, B, n2D.p, work.p, work.n, s));
  k_start_fallback<<<ceil_div(M * B, 256), 256, 0, s>>>(n2.p, n2D.p, mesh->bD.p, M, B, X, flag.p);
  LRFSI_TRY(check_launch("k_start_fallback"));
  if (fallback_host) LRFSI_CUDA(cudaMemcpyAsync(fallback_host, flag.p, sizeof(int) * B, cudaMemcpyDeviceToHost, s));
  LRFSI_CUDA(cudaStreamSynchronize(s));
  return LRFSI_OK;
}

int lrfsi_learned_factors(lrfsi_mesh_h mesh, lrfsi_mlp_h h, int K, const int* sizes_h, const double* mu_h,
                          const double* nu_h, const double* box, const double* Phi, int ldphi, int k,
                          const double* coef_scale, const double* field_scale, const double* offset,
                          const double* xt, double* U0, int ldu0, double* V0, int ldv0, lrfsi_stream_t stream) {
  if (!mesh || !h || K < 1 || !sizes_h || !mu_h || !nu_h || !box || !Phi || !coef_scale || !field_scale || !offset ||
      !xt || !U0 || !V0 || k < 1 || ldphi < k || ldu0 < k + 1 || ldv0 < k + 1 || h->d.n[0] != 2 ||
      h->d.n[kMlpLayers] != k || !(box[1] > box[0]) || !(box[3] > box[2]))
    return fail(LRFSI_EINVAL, "lrfsi_learned_factors: bad argument");
  int B = 0;
  for (int q = 0; q < K; ++q) {
    if (sizes_h[q] < 1) return fail(LRFSI_EINVAL, "lrfsi_learned_factors: empty subset");
    B += sizes_h[q];
  }
  cudaStream_t s = (cudaStream_t)stream;
  const long M = mesh->h.M;
  DevBuf<float> Z, C;
  DevBuf<char> ident;
  DevBuf<double> mu, nu;
  LRFSI_TRY(Z.alloc((size_t)2 * B));
  LRFSI_TRY(C.alloc((size_t)B * k));
  std::vector<double> muv(mu_h, mu_h + B), nuv(nu_h, nu_h + B);
  LRFSI_TRY(mu.upload(muv, s));
  LRFSI_TRY(nu.upload(nuv, s));
  std::vector<char> id(mesh->h.ident.begin(), mesh->h.ident.end());
  LRFSI_TRY(ident.upload(id, s));
  k_scale_params<<<ceil_div(B, 128), 128, 0, s>>>(mu.p, nu.p, B, box[0], box[1], box[2], box[3], Z.p);
  LRFSI_TRY(check_launch("k_scale_params"));
  LRFSI_TRY(mlp_forward_impl(h, Z.p, B, C.p, s, false));
  k_learned_v0<<<ceil_div((long)B * (k + 1), 256), 256, 0, s>>>(C.p, k, coef_scale, B, V0, ldv0);
  LRFSI_TRY(check_launch("k_learned_v0"));
  for (int q = 0; q < K; ++q) {
    k_learned_u0<<<ceil_div(M * (k + 1), 256), 256, 0, s>>>(Phi, ldphi, k, field_scale, offset, xt + (size_t)q * M,
                                                            ident.p, M, U0 + (size_t)q * M * ldu0, ldu0);
    LRFSI_TRY(check_launch("k_learned_u0"));
  }
  LRFSI_CUDA(cudaStreamSynchronize(s));
  return LRFSI_OK;
}

}  // extern "C"
