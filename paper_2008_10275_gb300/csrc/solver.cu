// The C ABI: mesh handles, assembly, batched residuals, the batched median
// Newton iteration (Sec. 3.2), and the subset Newton step solved on factors by
// the truncated preconditioned Chebyshev iteration (Sec. 3.4, Sec. 4.2,
// Algorithm 1).
#include <algorithm>
#include <climits>
#include <cstdint>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>

#include "dense.h"
#include "mesh.h"
#include "nd_lu.h"
#include "sparse_lu.h"

namespace lrfsi {

// ---------------------------------------------------------------------------
// errors and launch counting
// ---------------------------------------------------------------------------
static thread_local std::string g_err;
static std::atomic<uint64_t> g_launches{0};       // kernels launched (graph replays add their kernel nodes)
static std::atomic<uint64_t> g_host_launches{0};  // launch calls issued by the host (a graph replay is one)
void set_error(const std::string& msg) { g_err = msg; }
int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return LRFSI_ECUDA;
}
void count_launch(uint64_t n) {
  g_launches += n;
  g_host_launches += 1;
}

static std::mutex g_stat_mu;
static lrfsi_kernel_stat g_stat[LRFSI_NUM_KERNEL_CLASSES];
static bool g_timing = false;
struct PendingEv { int cls; cudaEvent_t a, b; };
static std::vector<PendingEv> g_pending;
bool timing_enabled() { return g_timing; }
bool gate_counts(const Gate& g, cudaStream_t s) {
  if (!g_timing || (!g.a && !g.b)) return true;
  int v[2] = {1, 1};
  if (g.a && cudaMemcpyAsync(&v[0], g.a, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return true;
  if (g.b && cudaMemcpyAsync(&v[1], g.b, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return true;
  if (cudaStreamSynchronize(s) != cudaSuccess) return true;
  return v[0] && v[1];
}
void account(int cls, double flops, double bytes) {
  std::lock_guard<std::mutex> lk(g_stat_mu);
  g_stat[cls].launches += 1;
  g_stat[cls].flops += flops;
  g_stat[cls].bytes += bytes;
}
TimedLaunch::TimedLaunch(int c, cudaStream_t s) : cls(c) {
  if (!g_timing) return;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) { a = b = nullptr; return; }
  cudaEventRecord(a, s);
}
void TimedLaunch::end(cudaStream_t s) {
  if (!a) return;
  cudaEventRecord(b, s);
  std::lock_guard<std::mutex> lk(g_stat_mu);
  g_pending.push_back(PendingEv{cls, a, b});
  a = b = nullptr;
}
static void collect_events() {
  std::lock_guard<std::mutex> lk(g_stat_mu);
  for (auto& e : g_pending) {
    float ms = 0;
    if (cudaEventSynchronize(e.b) == cudaSuccess && cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess)
      g_stat[e.cls].ms += ms;
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  g_pending.clear();
}

// ---------------------------------------------------------------------------
// small helper kernels
// ---------------------------------------------------------------------------
struct CopyDesc {
  const double* src;  // mode 0
  long lds;
  double* dst;
  long ldd;
  long rows;
  int ncols;
  int mode;            // 0: copy, 1: fill alpha * rowscale, 2: alpha * identity
  const double* rowscale;
  double alpha;
  Gate gate;
};
struct CopyBatch {
  CopyDesc d[kMaxGemmDescs];
};

__global__ void k_blockcopy(CopyBatch cb) {
  const CopyDesc& d = cb.d[blockIdx.y];
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.rows * d.ncols || !gate_open(d.gate)) return;
  const long i = e / d.ncols;
  const int j = (int)(e % d.ncols);
  double v;
  if (d.mode == 0) v = d.src[i * d.lds + j];
  else if (d.mode == 1) v = 1.0;
  else v = (i == j) ? 1.0 : 0.0;
  if (d.rowscale) v *= d.rowscale[i];
  d.dst[i * d.ldd + j] = d.alpha * v;
}

static int copy_batched(const std::vector<CopyDesc>& v, cudaStream_t s) {
  for (size_t i = 0; i < v.size();) {  // chunks of up to kMaxGemmDescs non-empty blocks
    CopyBatch cb;
    int cnt = 0;
    long mx = 0;
    for (; i < v.size() && cnt < kMaxGemmDescs; ++i) {
      if (v[i].rows <= 0 || v[i].ncols <= 0) continue;
      cb.d[cnt++] = v[i];
      mx = std::max(mx, v[i].rows * v[i].ncols);
    }
    if (!cnt) continue;
    k_blockcopy<<<dim3(ceil_div(mx, 256), cnt), 256, 0, s>>>(cb);
    LRFSI_TRY(check_launch("k_blockcopy"));
  }
  return LRFSI_OK;
}

// Block copy with precision conversion: dst[i*ldd + j] = (Tout) (alpha * rowscale[i] * src[i*lds + j])
struct ConvDesc {
  const void* src;
  long lds;
  void* dst;
  long ldd;
  long rows;
  int ncols;
  const double* rowscale;
  double alpha;
  Gate gate;
};
struct ConvBatch {
  ConvDesc d[kMaxGemmDescs];
};
template <class Tin, class Tout>
__global__ void k_convert(ConvBatch cb) {
  const ConvDesc& d = cb.d[blockIdx.y];
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.rows * d.ncols || !gate_open(d.gate)) return;
  const long i = e / d.ncols;
  const int j = (int)(e % d.ncols);
  double v = (double)((const Tin*)d.src)[i * d.lds + j] * d.alpha;
  if (d.rowscale) v *= d.rowscale[i];
  ((Tout*)d.dst)[i * d.ldd + j] = (Tout)v;
}
template <class Tin, class Tout>
static int convert_batched(const std::vector<ConvDesc>& v, cudaStream_t s) {
  for (size_t i = 0; i < v.size();) {  // chunks of up to kMaxGemmDescs non-empty blocks
    ConvBatch cb;
    int cnt = 0;
    long mx = 0;
    for (; i < v.size() && cnt < kMaxGemmDescs; ++i) {
      if (v[i].rows <= 0 || v[i].ncols <= 0) continue;
      cb.d[cnt++] = v[i];
      mx = std::max(mx, v[i].rows * v[i].ncols);
    }
    if (!cnt) continue;
    k_convert<Tin, Tout><<<dim3(ceil_div(mx, 256), cnt), 256, 0, s>>>(cb);
    LRFSI_TRY(check_launch("k_convert"));
  }
  return LRFSI_OK;
}

// problem-major (K x M) <-> column-major states (M x K row-major)
__global__ void k_transpose(const double* __restrict__ A, long rows, int cols, double* __restrict__ B) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const long i = e / cols;
  const int j = (int)(e % cols);
  B[(size_t)j * rows + i] = A[e];
}

// X[:, j] = Xold[:, j] + t[j] * dX[:, j]  (M x K row-major)
__global__ void k_newton_update(const double* __restrict__ Xold, const double* __restrict__ dX,
                                const double* __restrict__ t, long M, int K, double* __restrict__ X) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * K) return;
  const int j = (int)(e % K);
  X[e] = Xold[e] + t[j] * dX[e];
}

// Jacobian values at column j of an M x K state matrix: gather to a vector first
__global__ void k_gather_col(const double* __restrict__ X, long M, int K, int j, double* __restrict__ x) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) x[i] = X[i * K + j];
}

// Max-norm equilibration of P = J0 + a Jmu' + b Jnu' (values nnz x 3):
// r_i = 1 / max_j |P_ij|, c_j = 1 / max_i r_i |P_ij|.
__global__ void k_equil_rows(const double* __restrict__ J3, const int* __restrict__ rowptr, long M, double a,
                             double b, double* __restrict__ r) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  double mx = 0;
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
    mx = fmax(mx, fabs(J3[3 * (size_t)k] + a * J3[3 * (size_t)k + 1] + b * J3[3 * (size_t)k + 2]));
  r[i] = mx > 0 ? 1.0 / mx : 1.0;
}
__global__ void k_equil_colmax(const double* __restrict__ J3, const int* __restrict__ rowptr,
                               const int* __restrict__ colidx, long M, double a, double b,
                               const double* __restrict__ r, unsigned long long* __restrict__ cmax) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
    const double v = r[i] * fabs(J3[3 * (size_t)k] + a * J3[3 * (size_t)k + 1] + b * J3[3 * (size_t)k + 2]);
    atomicMax(cmax + colidx[k], (unsigned long long)__double_as_longlong(v));  // v >= 0: bit order = value order
  }
}
__global__ void k_equil_cols(const unsigned long long* __restrict__ cmax, long M, double* __restrict__ c) {
  const long j = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const double v = __longlong_as_double((long long)cmax[j]);
  c[j] = v > 0 ? 1.0 / v : 1.0;
}
__global__ void k_scale_vals(double* __restrict__ J3, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                             long M, const double* __restrict__ r, const double* __restrict__ c) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
    const double sc = r[i] * c[colidx[k]];
    J3[3 * (size_t)k] *= sc;
    J3[3 * (size_t)k + 1] *= sc;
    J3[3 * (size_t)k + 2] *= sc;
  }
}
// X[i, o + j] = x0[i] + s[i] * X[i, o + j]
__global__ void k_affine_cols(double* __restrict__ X, long ld, int o, int ncols, const double* __restrict__ x0,
                              const double* __restrict__ sc, long M) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * ncols) return;
  const long i = e / ncols;
  const int j = (int)(e % ncols);
  double* p = X + i * ld + o + j;
  *p = x0[i] + sc[i] * *p;
}

}  // namespace lrfsi

using namespace lrfsi;

// ---------------------------------------------------------------------------
// mesh API
// ---------------------------------------------------------------------------
extern "C" {

const char* lrfsi_last_error(void) { return g_err.c_str(); }

int lrfsi_stats(int cls, lrfsi_kernel_stat* out) {
  if (cls < 0 || cls >= LRFSI_NUM_KERNEL_CLASSES || !out) return fail(LRFSI_EINVAL, "lrfsi_stats: bad class");
  collect_events();
  std::lock_guard<std::mutex> lk(g_stat_mu);
  *out = g_stat[cls];
  return LRFSI_OK;
}
int lrfsi_stats_reset(void) {
  collect_events();
  std::lock_guard<std::mutex> lk(g_stat_mu);
  for (auto& st : g_stat) st = lrfsi_kernel_stat{0, 0, 0, 0};
  return LRFSI_OK;
}
int lrfsi_timing(int enable) {
  collect_events();
  g_timing = enable != 0;
  return LRFSI_OK;
}
uint64_t lrfsi_kernel_launches(void) { return g_launches.load(); }
uint64_t lrfsi_host_launches(void) { return g_host_launches.load(); }

int lrfsi_mesh_create(const lrfsi_problem* prob, lrfsi_mesh_h* out) {
  if (!prob || !out) return fail(LRFSI_EINVAL, "lrfsi_mesh_create: null argument");
  *out = nullptr;
  lrfsi_mesh_s* m = new (std::nothrow) lrfsi_mesh_s();
  if (!m) return fail(LRFSI_ENOMEM, "lrfsi_mesh_create: host allocation");
  int st = build_mesh(*prob, m->h);
  if (st == LRFSI_OK) st = m->rowptr.upload(m->h.rowptr);
  if (st == LRFSI_OK) st = m->colidx.upload(m->h.colidx);
  if (st == LRFSI_OK) st = m->cell_dof.upload(m->h.cell_dof);
  if (st == LRFSI_OK) st = m->cell_row.upload(m->h.cell_row);
  if (st == LRFSI_OK) st = m->slot.upload(m->h.slot);
  if (st == LRFSI_OK) st = m->color_cells.upload(m->h.color_cells);
  if (st == LRFSI_OK) st = m->ident_rows.upload(m->h.ident_rows);
  if (st == LRFSI_OK) st = m->ident_diag.upload(m->h.ident_diag);
  if (st == LRFSI_OK) st = m->cell_solid.upload(m->h.cell_solid);
  if (st == LRFSI_OK) st = m->bD.upload(m->h.bD);
  if (st == LRFSI_OK) st = m->dense_off.upload(m->h.dense_off);
  if (st == LRFSI_OK) {
    std::vector<long long> so(m->h.slab_off.begin(), m->h.slab_off.end());
    st = m->slab_off.upload(so);
  }
  if (st == LRFSI_OK) {  // SpMM column windows of the row blocks
    const long M = m->h.M;
    const long nb = (M + kSpmmRowBlock - 1) / kSpmmRowBlock;
    std::vector<int> win(2 * nb);
    for (long b = 0; b < nb; ++b) {
      int lo = INT32_MAX, hi = -1;
      for (long r = b * kSpmmRowBlock; r < std::min(M, (b + 1) * kSpmmRowBlock); ++r)
        for (int q = m->h.rowptr[r]; q < m->h.rowptr[r + 1]; ++q) {
          lo = std::min(lo, m->h.colidx[q]);
          hi = std::max(hi, m->h.colidx[q]);
        }
      if (hi < 0) { lo = 0; hi = -1; }
      win[2 * b] = lo;
      win[2 * b + 1] = hi + 1;
      m->spmm_winmax = std::max(m->spmm_winmax, hi + 1 - lo);
    }
    st = m->spmm_win.upload(win);
  }
  if (st == LRFSI_OK) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = cuda_fail(e, "lrfsi_mesh_create upload");
  }
  if (st != LRFSI_OK) {
    delete m;
    return st;
  }
  // the slot map is only needed on the device
  std::vector<int>().swap(m->h.slot);
  *out = m;
  return LRFSI_OK;
}

int lrfsi_mesh_destroy(lrfsi_mesh_h m) {
  delete m;
  return LRFSI_OK;
}

int lrfsi_mesh_info(lrfsi_mesh_h m, lrfsi_mesh_info_t* info) {
  if (!m || !info) return fail(LRFSI_EINVAL, "lrfsi_mesh_info: null argument");
  info->M = m->h.M;
  info->nnz = (int64_t)m->h.colidx.size();
  info->nslab = m->h.nslab;
  info->nmax = m->h.nmax;
  info->ncell = m->h.ncell;
  info->nsolid = m->h.nsolid;
  return LRFSI_OK;
}

int lrfsi_mesh_dofmap(lrfsi_mesh_h m, int32_t* field, int32_t* ix, int32_t* iy) {
  if (!m) return fail(LRFSI_EINVAL, "lrfsi_mesh_dofmap: null mesh");
  if (field) std::memcpy(field, m->h.dof_field.data(), sizeof(int32_t) * m->h.M);
  if (ix) std::memcpy(ix, m->h.dof_ix.data(), sizeof(int32_t) * m->h.M);
  if (iy) std::memcpy(iy, m->h.dof_iy.data(), sizeof(int32_t) * m->h.M);
  return LRFSI_OK;
}

int lrfsi_mesh_dirichlet(lrfsi_mesh_h m, double* bD) {
  if (!m || !bD) return fail(LRFSI_EINVAL, "lrfsi_mesh_dirichlet: null argument");
  std::memcpy(bD, m->h.bD.data(), sizeof(double) * m->h.M);
  return LRFSI_OK;
}

int lrfsi_mesh_pattern(lrfsi_mesh_h m, int32_t* rowptr, int32_t* colidx) {
  if (!m) return fail(LRFSI_EINVAL, "lrfsi_mesh_pattern: null mesh");
  if (rowptr) std::memcpy(rowptr, m->h.rowptr.data(), sizeof(int32_t) * (m->h.M + 1));
  if (colidx) std::memcpy(colidx, m->h.colidx.data(), sizeof(int32_t) * m->h.colidx.size());
  return LRFSI_OK;
}

size_t lrfsi_mesh_bytes(lrfsi_mesh_h m) {
  if (!m) return 0;
  return m->rowptr.bytes() + m->colidx.bytes() + m->cell_dof.bytes() + m->cell_row.bytes() + m->slot.bytes() +
         m->color_cells.bytes() + m->ident_rows.bytes() + m->ident_diag.bytes() + m->cell_solid.bytes() +
         m->bD.bytes() + m->dense_off.bytes() + m->slab_off.bytes();
}

int lrfsi_assemble_affine(lrfsi_mesh_h m, const double* x, double* J3, double* R3, lrfsi_stream_t stream) {
  if (!m || !x) return fail(LRFSI_EINVAL, "lrfsi_assemble_affine: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (J3) LRFSI_TRY(launch_jacobian(m, x, J3, s));
  if (R3) {
    // columns (rest, mu, nu) = (1,0,0), (0,1,0), (0,0,1)
    static const double h_coef[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    DevBuf<double> coef;
    LRFSI_TRY(coef.alloc(9));
    LRFSI_CUDA(cudaMemcpyAsync(coef.p, h_coef, sizeof(h_coef), cudaMemcpyHostToDevice, s));
    LRFSI_TRY(launch_residual(m, x, 0, 3, coef.p, coef.p + 3, coef.p + 6, R3, 3, s));
    LRFSI_CUDA(cudaStreamSynchronize(s));  // coef is freed on return
  }
  return LRFSI_OK;
}

}  // extern "C"

namespace lrfsi {
// J3a = (J0, Jmu', Jnurho'), J3b = (Jlam', Jrho', 0) from three assemblies at
// (rho_f, lambda_s) = (0, 0), (1, 0), (0, 1):  the rho and lambda parts are the
// differences of the J0 slots (they are zero at every entry the other terms fill).
__global__ void k_five_ops(const double* __restrict__ J00, const double* __restrict__ J10,
                           const double* __restrict__ J01, long nnz, double* __restrict__ Ja, double* __restrict__ Jb) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  const double j0 = J00[3 * e];
  Ja[3 * e] = j0;
  Ja[3 * e + 1] = J00[3 * e + 1];
  Ja[3 * e + 2] = J10[3 * e + 2];
  Jb[3 * e] = J01[3 * e] - j0;
  Jb[3 * e + 1] = J10[3 * e] - j0;
  Jb[3 * e + 2] = 0.0;
}
// R5 (M x 5: R0, Rmu, Rnurho, R0 + Rlam, R0 + Rrho) -> R3a = (R0, Rmu, Rnurho), R3b = (Rlam, Rrho, 0)
__global__ void k_five_res(const double* __restrict__ R5, long M, double* __restrict__ Ra, double* __restrict__ Rb) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const double* r = R5 + 5 * i;
  Ra[3 * i] = r[0];
  Ra[3 * i + 1] = r[1];
  Ra[3 * i + 2] = r[2];
  Rb[3 * i] = r[3] - r[0];
  Rb[3 * i + 1] = r[4] - r[0];
  Rb[3 * i + 2] = 0.0;
}

// The five affine pieces of the four-parameter problem at x (Sec. 4.4,
// Eq. (matrix_fourpars1) with the reference values set to 0):
//   J = J0 + mu Jmu' + (nu rho) Jnurho' + lam Jlam' + rho Jrho',  R likewise.
// J3a, J3b: nnz x 3 each (or NULL); R3a, R3b: M x 3 each (or NULL).
static int assemble_five(lrfsi_mesh_s* m, const double* x, double* J3a, double* J3b, double* R3a, double* R3b,
                         cudaStream_t s) {
  const long nnz = (long)m->h.colidx.size(), M = m->h.M;
  if (J3a || J3b) {
    DevBuf<double> J00, J10, J01;
    LRFSI_TRY(J00.alloc((size_t)3 * nnz));
    LRFSI_TRY(J10.alloc((size_t)3 * nnz));
    LRFSI_TRY(J01.alloc((size_t)3 * nnz));
    const double rl00[2] = {0.0, 0.0}, rl10[2] = {1.0, 0.0}, rl01[2] = {0.0, 1.0};
    LRFSI_TRY(launch_jacobian(m, x, J00.p, s, rl00));
    LRFSI_TRY(launch_jacobian(m, x, J10.p, s, rl10));
    LRFSI_TRY(launch_jacobian(m, x, J01.p, s, rl01));
    DevBuf<double> ta, tb;
    double* Ja = J3a;
    double* Jb = J3b;
    if (!Ja) { LRFSI_TRY(ta.alloc((size_t)3 * nnz)); Ja = ta.p; }
    if (!Jb) { LRFSI_TRY(tb.alloc((size_t)3 * nnz)); Jb = tb.p; }
    k_five_ops<<<ceil_div(nnz, 256), 256, 0, s>>>(J00.p, J10.p, J01.p, nnz, Ja, Jb);
    LRFSI_TRY(check_launch("k_five_ops"));
    LRFSI_CUDA(cudaStreamSynchronize(s));  // temporaries are freed on return
  }
  if (R3a || R3b) {
    // columns (rest, mu, nu, rho, lam):
    //   R0 (1,0,0,0,0), Rmu (0,1,0,0,0), Rnurho (0,0,1,1,0), R0 + Rlam (1,0,0,0,1), R0 + Rrho (1,0,0,1,0)
    static const double h_coef[25] = {1, 0, 0, 1, 1,   0, 1, 0, 0, 0,   0, 0, 1, 0, 0,
                                      0, 0, 1, 0, 1,   0, 0, 0, 1, 0};
    DevBuf<double> coef, R5, ta, tb;
    LRFSI_TRY(coef.alloc(25));
    LRFSI_TRY(R5.alloc((size_t)5 * M));
    LRFSI_CUDA(cudaMemcpyAsync(coef.p, h_coef, sizeof(h_coef), cudaMemcpyHostToDevice, s));
    LRFSI_TRY(launch_residual(m, x, 0, 5, coef.p, coef.p + 5, coef.p + 10, R5.p, 5, s, coef.p + 15, coef.p + 20));
    double* Ra = R3a;
    double* Rb = R3b;
    if (!Ra) { LRFSI_TRY(ta.alloc((size_t)3 * M)); Ra = ta.p; }
    if (!Rb) { LRFSI_TRY(tb.alloc((size_t)3 * M)); Rb = tb.p; }
    k_five_res<<<ceil_div(M, 256), 256, 0, s>>>(R5.p, M, Ra, Rb);
    LRFSI_TRY(check_launch("k_five_res"));
    LRFSI_CUDA(cudaStreamSynchronize(s));
  }
  return LRFSI_OK;
}
}  // namespace lrfsi

extern "C" {

int lrfsi_assemble_affine4(lrfsi_mesh_h m, const double* x, double* J3a, double* J3b, double* R3a, double* R3b,
                           lrfsi_stream_t stream) {
  if (!m || !x) return fail(LRFSI_EINVAL, "lrfsi_assemble_affine4: null argument");
  return assemble_five(m, x, J3a, J3b, R3a, R3b, (cudaStream_t)stream);
}

int lrfsi_residual_batch4(lrfsi_mesh_h m, const double* X, int ldx, int ncol, const double* mu, const double* nu,
                          const double* lam, const double* rho, double* R, int ldr, double* norm2,
                          lrfsi_stream_t stream) {
  if (!m || !X || !mu || !nu || !lam || !rho || !R || ncol < 0 || ldx < ncol || ldr < ncol)
    return fail(LRFSI_EINVAL, "lrfsi_residual_batch4: bad argument");
  if (ncol == 0) return LRFSI_OK;
  cudaStream_t s = (cudaStream_t)stream;
  LRFSI_TRY(launch_residual(m, X, ldx, ncol, nullptr, mu, nu, R, ldr, s, rho, lam));
  if (norm2) {
    DevBuf<double> work;
    LRFSI_TRY(work.alloc(colnorm_work_len(m->h.M, ncol)));
    LRFSI_TRY(launch_colnorm2(R, m->h.M, ncol, ldr, norm2, work.p, work.n, s));
    LRFSI_CUDA(cudaStreamSynchronize(s));
  }
  return LRFSI_OK;
}

int lrfsi_residual_batch(lrfsi_mesh_h m, const double* X, int ldx, int ncol, const double* mu, const double* nu,
                         double* R, int ldr, double* norm2, lrfsi_stream_t stream) {
  if (!m || !X || !mu || !nu || ncol < 0 || ldx < ncol) return fail(LRFSI_EINVAL, "lrfsi_residual_batch: bad argument");
  if (ncol == 0) return LRFSI_OK;
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf<double> tmp, work;
  double* Rp = R;
  int ld = ldr;
  if (!Rp) {
    LRFSI_TRY(tmp.alloc((size_t)m->h.M * ncol));
    Rp = tmp.p;
    ld = ncol;
  } else if (ldr < ncol) {
    return fail(LRFSI_EINVAL, "lrfsi_residual_batch: ldr < ncol");
  }
  LRFSI_TRY(launch_residual(m, X, ldx, ncol, nullptr, mu, nu, Rp, ld, s));
  if (norm2) {
    size_t wl = (size_t)ceil_div(m->h.M, 256) * ncol;
    LRFSI_TRY(work.alloc(wl));
    LRFSI_TRY(launch_colnorm2(Rp, m->h.M, ncol, ld, norm2, work.p, wl, s));
  }
  LRFSI_CUDA(cudaStreamSynchronize(s));
  return LRFSI_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// internal: relative residuals of dense columns
// ---------------------------------------------------------------------------
namespace lrfsi {

struct ResidualCtx {
  DevBuf<double> R, norm2, norm2_bD, work;
  long M = 0;
  int ncol = 0;
  int init(long M_, int ncol_) {
    M = M_;
    ncol = ncol_;
    LRFSI_TRY(R.alloc((size_t)M * ncol));
    LRFSI_TRY(norm2.alloc(ncol));
    LRFSI_TRY(norm2_bD.alloc(ncol));
    LRFSI_TRY(work.alloc((size_t)ceil_div(M, 256) * ncol));
    return LRFSI_OK;
  }
};

// ||R(b_D; mu, nu)||^2 per column (denominator of the relative residual)
static int residual_bD_norms(lrfsi_mesh_s* m, ResidualCtx& c, const double* mu, const double* nu, cudaStream_t s,
                             const double* rho = nullptr, const double* lam = nullptr) {
  LRFSI_TRY(launch_residual(m, m->bD.p, 0, c.ncol, nullptr, mu, nu, c.R.p, c.ncol, s, rho, lam));
  return launch_colnorm2(c.R.p, m->h.M, c.ncol, c.ncol, c.norm2_bD.p, c.work.p, c.work.n, s);
}

}  // namespace lrfsi

extern "C" int lrfsi_residual(lrfsi_mesh_h m, const double* xt, const double* U, int ldu, const double* V, int ldv,
                              int r, const double* mu, const double* nu, int ncol, double* relres,
                              lrfsi_stream_t stream) {
  if (!m || !xt || !mu || !nu || !relres || ncol < 1 || r < 0 || (r > 0 && (!U || !V || ldu < r || ldv < r)))
    return fail(LRFSI_EINVAL, "lrfsi_residual: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  const long M = m->h.M;
  DevBuf<double> X;
  LRFSI_TRY(X.alloc((size_t)M * ncol));
  std::vector<CopyDesc> cd(1);
  cd[0] = CopyDesc{xt, 1, X.p, ncol, M, 1, 0, nullptr, 1.0};
  // broadcast xt into every column: copy column 0 then use ldx trick per column
  for (int j = 0; j < ncol; ++j) {
    cd[0].dst = X.p + j;
    LRFSI_TRY(copy_batched(cd, s));
  }
  if (r > 0) {
    // FP64 kernels: the columns whose residual is reported (no tensor path)
    GemmDesc<double> g{(int)M, ncol, r, U, ldu, 1, V, 1, ldv, X.p, ncol, 1, 1.0, 1.0};
    LRFSI_TRY(gemm_grouped<double>(&g, 1, s));
  }
  ResidualCtx c;
  LRFSI_TRY(c.init(M, ncol));
  LRFSI_TRY(residual_bD_norms(m, c, mu, nu, s));
  LRFSI_TRY(launch_residual(m, X.p, ncol, ncol, nullptr, mu, nu, c.R.p, ncol, s));
  LRFSI_TRY(launch_colnorm2(c.R.p, M, ncol, ncol, c.norm2.p, c.work.p, c.work.n, s));
  std::vector<double> a(ncol), b(ncol);
  LRFSI_CUDA(cudaMemcpyAsync(a.data(), c.norm2.p, sizeof(double) * ncol, cudaMemcpyDeviceToHost, s));
  LRFSI_CUDA(cudaMemcpyAsync(b.data(), c.norm2_bD.p, sizeof(double) * ncol, cudaMemcpyDeviceToHost, s));
  LRFSI_CUDA(cudaStreamSynchronize(s));
  for (int j = 0; j < ncol; ++j) relres[j] = b[j] > 0 ? std::sqrt(a[j] / b[j]) : std::sqrt(a[j]);
  return LRFSI_OK;
}

// ---------------------------------------------------------------------------
// The sparse LU of the Newton steps and preconditioners: nested dissection with
// dense fronts (default), or the slab-ordered block-tridiagonal LU
// ---------------------------------------------------------------------------
namespace lrfsi {
static std::atomic<int> g_lu_mode{1};  // 0: slab block LU, 1: nested dissection

struct PrecLU {
  int kind = 1;
  BlockLU blk;
  NdLU nd;
  size_t bytes() const { return blk.bytes() + nd.bytes(); }
  int alloc(lrfsi_mesh_s* m, int nprob, int ld) {
    kind = g_lu_mode.load();
    return kind == 1 ? ndlu_alloc(m, nprob, ld, nd) : blocklu_alloc(m, nprob, blk);
  }
  int factor(lrfsi_mesh_s* m, const double* const* J3, const double* a, const double* b, int nprob, cudaStream_t s) {
    return kind == 1 ? ndlu_factor(m, nd, J3, a, b, nprob, s) : blocklu_factor(m, blk, J3, a, b, nprob, s);
  }
  int status(int nprob, std::vector<int>& out, cudaStream_t s) {
    return kind == 1 ? ndlu_status(nd, nprob, out, s) : blocklu_status(blk, nprob, out, s);
  }
  // Y = A^{-1} X (r_q columns, ld); the block LU overwrites X, the ND LU does not
  int solve(double* const* X, double* const* Y, const int* r, int ld, int nprob, cudaStream_t s,
            const Gate* gates = nullptr) {
    if (kind == 1) return ndlu_solve(nd, X, Y, r, ld, nprob, s, gates);
    return blocklu_solve(blk, X, Y, r, ld, nprob, s, gates);
  }
  int max_cols() const { return kind == 1 ? nd.ld : 1 << 30; }
};
}  // namespace lrfsi

extern "C" int lrfsi_lu_mode(int mode, int* previous) {
  using namespace lrfsi;
  if (mode < -1 || mode > 1) return fail(LRFSI_EINVAL, "lrfsi_lu_mode: mode must be 0, 1 (or -1 to query)");
  const int old = mode >= 0 ? g_lu_mode.exchange(mode) : g_lu_mode.load();
  if (previous) *previous = old;
  return LRFSI_OK;
}

extern "C" int lrfsi_lu_info(const lrfsi_problem* prob, int64_t* out8) {
  using namespace lrfsi;
  if (!prob || !out8) return fail(LRFSI_EINVAL, "lrfsi_lu_info: null argument");
  MeshHost h;
  LRFSI_TRY(build_mesh(*prob, h));
  NdSymbolic y;
  LRFSI_TRY(nd_symbolic(h, y));
  double thomas = 0;
  for (int sl = 0; sl < h.nslab; ++sl) {
    const double n = (double)(h.slab_off[sl + 1] - h.slab_off[sl]);
    const double nn = sl + 1 < h.nslab ? (double)(h.slab_off[sl + 2] - h.slab_off[sl + 1]) : 0.0;
    thomas += (2.0 / 3.0) * n * n * n + 2.0 * n * n * (nn + n) + 2.0 * nn * nn * n;
  }
  out8[0] = (int64_t)y.fr.size();
  out8[1] = y.heights;
  out8[2] = y.maxf;
  out8[3] = y.maxb;
  out8[4] = (int64_t)(y.ws_doubles + y.inv_doubles);
  out8[5] = (int64_t)y.factor_flops;
  out8[6] = (int64_t)thomas;
  out8[7] = (int64_t)h.nslab * h.nmax * h.nmax * 4;
  return LRFSI_OK;
}

// ---------------------------------------------------------------------------
// Batched Newton iteration for independent problems (median solutions)
// ---------------------------------------------------------------------------
namespace lrfsi {
// The theta-scheme (Sec. 4.3): one time step's operators and residual.
// J3 <- (theta J0 + cm Mv, theta Jmu', theta Jnu'), cm = rho_f / dt.
__global__ void k_theta_ops(double* __restrict__ J3, long nnz, double theta, double cm, const double* __restrict__ Mv) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  J3[3 * e] = theta * J3[3 * e] + cm * Mv[e];
  J3[3 * e + 1] *= theta;
  J3[3 * e + 2] *= theta;
}
// D = X - Xp (M x n, ld n)
__global__ void k_diff(const double* X, const double* Xp, long count, double* D) {  // D may be X
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) D[e] = X[e] - Xp[e];
}
// R <- theta R + (1 - theta) Rp + cm Y (M x n, ld n)
__global__ void k_theta_combine(double* __restrict__ R, const double* __restrict__ Rp, const double* __restrict__ Y,
                                long count, double theta, double cm) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) R[e] = theta * R[e] + (1.0 - theta) * Rp[e] + cm * Y[e];
}
// (Mv, 0, 0) as an operator triple for the SpMM
__global__ void k_mass_triple(const double* __restrict__ Mv, long nnz, double* __restrict__ M3) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  M3[3 * e] = Mv[e];
  M3[3 * e + 1] = 0.0;
  M3[3 * e + 2] = 0.0;
}

// State of a time step: previous states, their residual R(X_prev), the mass
// triple and the scheme's constants.
struct TimeStep {
  const double* Xprev = nullptr;  // M x n (ld n)
  const double* Rprev = nullptr;  // M x n: R(X_prev; mu, nu)
  const double* M3 = nullptr;     // nnz x 3 (Mv, 0, 0)
  const double* Mv = nullptr;     // nnz
  double theta = 1.0, cm = 0.0;   // cm = rho_f / dt
};

// R (M x n, ld n) <- R_theta(X) = theta R(X) + (1 - theta) R(X_prev) + cm Mass (X - X_prev),
// with R(X) already in R; D, Y: M x n scratch.
static int theta_residual_cols(lrfsi_mesh_s* m, const TimeStep& ts, const double* X, int n, double* R, double* D,
                               double* Y, cudaStream_t s) {
  const long M = m->h.M, cnt = M * n;
  k_diff<<<ceil_div(cnt, 256), 256, 0, s>>>(X, ts.Xprev, cnt, D);
  LRFSI_TRY(check_launch("k_diff"));
  SpmmDesc<double> d;
  d.J3 = ts.M3; d.U = D; d.ldu = n; d.r = n; d.Y = Y; d.ldy = n;
  d.o[0] = 0; d.o[1] = -1; d.o[2] = -1;
  d.sc[0] = d.sc[1] = d.sc[2] = 1.0;
  d.a1 = d.a2 = 0.0;
  LRFSI_TRY(spmm_batched<double>(m, &d, 1, s));
  k_theta_combine<<<ceil_div(cnt, 256), 256, 0, s>>>(R, ts.Rprev, Y, cnt, ts.theta, ts.cm);
  return check_launch("k_theta_combine");
}
}  // namespace lrfsi

// lam_h, rho_h (host, K each, optional): lambda_s and rho_f per problem (the
// four-parameter problem, Sec. 4.4) in place of the mesh's constants.
// ts (optional): a theta-scheme time step (Sec. 4.3): the residual is
// R_theta and the Jacobian rho_f Mass / dt + theta J (previous states M x K).
static int newton_impl(lrfsi_mesh_h m, int K, double* Xpm, const double* mu_h, const double* nu_h, const double* lam_h,
                       const double* rho_h, double eps, int max_it, int* iters_h, double* res_h,
                       lrfsi_stream_t stream, const TimeStep* ts = nullptr) {
  if (!m || !Xpm || !mu_h || !nu_h || K < 1 || K > kMaxGemmDescs || max_it < 0)
    return fail(LRFSI_EINVAL, "lrfsi_newton_median: bad argument (1 <= K <= 32)");
  for (int k = 0; k < K; ++k)
    if (!std::isfinite(mu_h[k]) || !std::isfinite(nu_h[k]) || (lam_h && !std::isfinite(lam_h[k])) ||
        (rho_h && !std::isfinite(rho_h[k])))
      return fail(LRFSI_EINVAL, "lrfsi_newton_median: parameters must be finite");
  cudaStream_t s = (cudaStream_t)stream;
  const long M = m->h.M;
  const long nnz = (long)m->h.colidx.size();
  DevBuf<double> X, Xold, dX, Rb, J3, xcol, tdev, mu, nu, work, norm2;
  LRFSI_TRY(X.alloc((size_t)M * K));
  LRFSI_TRY(Xold.alloc((size_t)M * K));
  LRFSI_TRY(dX.alloc((size_t)M * K));
  LRFSI_TRY(Rb.alloc((size_t)M * K));
  LRFSI_TRY(J3.alloc((size_t)3 * nnz * K));
  LRFSI_TRY(xcol.alloc(M));
  LRFSI_TRY(tdev.alloc(K));
  LRFSI_TRY(mu.alloc(K));
  LRFSI_TRY(nu.alloc(K));
  LRFSI_TRY(norm2.alloc(K));
  LRFSI_TRY(work.alloc((size_t)ceil_div(M, 256) * K));
  LRFSI_CUDA(cudaMemcpyAsync(mu.p, mu_h, sizeof(double) * K, cudaMemcpyHostToDevice, s));
  LRFSI_CUDA(cudaMemcpyAsync(nu.p, nu_h, sizeof(double) * K, cudaMemcpyHostToDevice, s));
  DevBuf<double> lam, rho;
  if (lam_h && rho_h) {
    LRFSI_TRY(lam.alloc(K));
    LRFSI_TRY(rho.alloc(K));
    LRFSI_CUDA(cudaMemcpyAsync(lam.p, lam_h, sizeof(double) * K, cudaMemcpyHostToDevice, s));
    LRFSI_CUDA(cudaMemcpyAsync(rho.p, rho_h, sizeof(double) * K, cudaMemcpyHostToDevice, s));
  }
  k_transpose<<<ceil_div(M * K, 256), 256, 0, s>>>(Xpm, K, (int)M, X.p);  // (K x M) -> (M x K)
  LRFSI_TRY(check_launch("k_transpose"));
  PrecLU lu;
  LRFSI_TRY(lu.alloc(m, K, 1));
  DevBuf<double> tsD, tsY;
  if (ts) {
    LRFSI_TRY(tsD.alloc((size_t)M * K));
    LRFSI_TRY(tsY.alloc((size_t)M * K));
  }
  auto resid = [&](const double* Xs) -> int {
    LRFSI_TRY(launch_residual(m, Xs, K, K, nullptr, mu.p, nu.p, Rb.p, K, s, rho.p, lam.p));
    if (ts) LRFSI_TRY(theta_residual_cols(m, *ts, Xs, K, Rb.p, tsD.p, tsY.p, s));
    return LRFSI_OK;
  };
  auto norms = [&](const double* Xs, std::vector<double>& out) -> int {
    LRFSI_TRY(resid(Xs));
    LRFSI_TRY(launch_colnorm2(Rb.p, M, K, K, norm2.p, work.p, work.n, s));
    out.resize(K);
    LRFSI_CUDA(cudaMemcpyAsync(out.data(), norm2.p, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
    LRFSI_CUDA(cudaStreamSynchronize(s));
    for (auto& v : out) v = std::sqrt(v);
    return LRFSI_OK;
  };
  std::vector<double> r, rn, t(K, 1.0);
  std::vector<int> it(K, 0);
  LRFSI_TRY(norms(X.p, r));
  int status = LRFSI_OK;
  for (int iter = 0; iter < max_it; ++iter) {
    std::vector<int> act;
    for (int k = 0; k < K; ++k)
      if (!(r[k] <= eps)) act.push_back(k);
    if (act.empty()) break;
    // residual at the current iterate (Rb holds it for every column after norms())
    LRFSI_TRY(resid(X.p));
    std::vector<const double*> J3p;
    std::vector<double> al, be;
    for (int k : act) {
      k_gather_col<<<ceil_div(M, 256), 256, 0, s>>>(X.p, M, K, k, xcol.p);
      LRFSI_TRY(check_launch("k_gather_col"));
      double* Jk = J3.p + (size_t)3 * nnz * J3p.size();
      const double rl[2] = {rho_h ? rho_h[k] : 0.0, lam_h ? lam_h[k] : 0.0};
      LRFSI_TRY(launch_jacobian(m, xcol.p, Jk, s, (lam_h && rho_h) ? rl : nullptr));
      if (ts) {
        k_theta_ops<<<ceil_div(nnz, 256), 256, 0, s>>>(Jk, nnz, ts->theta, ts->cm, ts->Mv);
        LRFSI_TRY(check_launch("k_theta_ops"));
      }
      J3p.push_back(Jk);
      al.push_back(mu_h[k]);
      be.push_back(nu_h[k]);
    }
    const int na = (int)act.size();
    // dX = -J^{-1} R: the residual is negated in place and its forward sweep
    // runs inside the factorisation (single-solve mode: no explicit inverses)
    {
      std::vector<CopyDesc> cd;
      cd.push_back(CopyDesc{Rb.p, K, Rb.p, K, M, K, 0, nullptr, -1.0});
      LRFSI_TRY(copy_batched(cd, s));
    }
    LRFSI_CUDA(cudaMemsetAsync(dX.p, 0, sizeof(double) * M * K, s));
    std::vector<const double*> bs(na);
    std::vector<double*> ys(na);
    for (int a = 0; a < na; ++a) {
      bs[a] = Rb.p + act[a];
      ys[a] = dX.p + act[a];
    }
    if (lu.kind == 1) {
      LRFSI_TRY(lu.factor(m, J3p.data(), al.data(), be.data(), na, s));
      std::vector<double*> bx(na);
      for (int a = 0; a < na; ++a) bx[a] = const_cast<double*>(bs[a]);
      std::vector<int> one(na, 1);
      LRFSI_TRY(lu.solve(bx.data(), ys.data(), one.data(), K, na, s));
    } else {
      LRFSI_TRY(blocklu_factor(m, lu.blk, J3p.data(), al.data(), be.data(), na, s, bs.data(), ys.data(), K));
    }
    std::vector<int> lst;
    LRFSI_TRY(lu.status(na, lst, s));
    for (int a = 0; a < na; ++a)
      if (lst[a] != 0) status = LRFSI_ESINGULAR;
    LRFSI_CUDA(cudaMemcpyAsync(Xold.p, X.p, sizeof(double) * M * K, cudaMemcpyDeviceToDevice, s));
    // step with halving while the residual grows (the stationary problem); a
    // time step takes full steps: its first step from x_prev typically raises
    // ||R_theta|| before the quadratic phase, and halving would stall it
    std::fill(t.begin(), t.end(), 0.0);
    for (int k : act) t[k] = 1.0;
    const int max_halve = ts ? 0 : 8;
    for (int h = 0; h <= max_halve; ++h) {
      LRFSI_CUDA(cudaMemcpyAsync(tdev.p, t.data(), sizeof(double) * K, cudaMemcpyHostToDevice, s));
      k_newton_update<<<ceil_div(M * K, 256), 256, 0, s>>>(Xold.p, dX.p, tdev.p, M, K, X.p);
      LRFSI_TRY(check_launch("k_newton_update"));
      LRFSI_TRY(norms(X.p, rn));
      bool again = false;
      for (int k : act) {
        if (t[k] > 0 && !(rn[k] < r[k]) && h < max_halve) {
          t[k] *= 0.5;
          again = true;
        }
      }
      if (!again) break;
    }
    for (int k : act) {
      r[k] = rn[k];
      it[k] += 1;
    }
  }
  for (int k = 0; k < K; ++k) {
    if (iters_h) iters_h[k] = it[k];
    if (res_h) res_h[k] = r[k];
    if (!(r[k] <= eps) && status == LRFSI_OK) status = LRFSI_ENOCONV;
  }
  k_transpose<<<ceil_div(M * K, 256), 256, 0, s>>>(X.p, M, K, Xpm);
  LRFSI_TRY(check_launch("k_transpose"));
  LRFSI_CUDA(cudaStreamSynchronize(s));
  if (status == LRFSI_ENOCONV) return fail(status, "lrfsi_newton_median: eps not reached within max_it");
  if (status == LRFSI_ESINGULAR) return fail(status, "lrfsi_newton_median: zero pivot in the block LU");
  return LRFSI_OK;
}

extern "C" int lrfsi_newton_median(lrfsi_mesh_h m, int K, double* Xpm, const double* mu_h, const double* nu_h,
                                   double eps, int max_it, int* iters_h, double* res_h, lrfsi_stream_t stream) {
  return newton_impl(m, K, Xpm, mu_h, nu_h, nullptr, nullptr, eps, max_it, iters_h, res_h, stream);
}

extern "C" int lrfsi_newton_median4(lrfsi_mesh_h m, int K, double* Xpm, const double* mu_h, const double* nu_h,
                                    const double* lam_h, const double* rho_h, double eps, int max_it, int* iters_h,
                                    double* res_h, lrfsi_stream_t stream) {
  if (!lam_h || !rho_h) return fail(LRFSI_EINVAL, "lrfsi_newton_median4: null lambda_s / rho_f");
  return newton_impl(m, K, Xpm, mu_h, nu_h, lam_h, rho_h, eps, max_it, iters_h, res_h, stream);
}

extern "C" int lrfsi_newton_theta(lrfsi_mesh_h m, int K, double* Xpm, const double* Xprev_pm, const double* mu_h,
                                  const double* nu_h, double theta, double dt, double eps, int max_it, int* iters_h,
                                  double* res_h, lrfsi_stream_t stream) {
  if (!m || !Xpm || !Xprev_pm || !mu_h || !nu_h || K < 1 || K > kMaxGemmDescs || !(theta > 0 && theta <= 1) ||
      !(dt > 0))
    return fail(LRFSI_EINVAL, "lrfsi_newton_theta: bad argument (0 < theta <= 1, dt > 0)");
  cudaStream_t s = (cudaStream_t)stream;
  const long M = m->h.M, nnz = (long)m->h.colidx.size();
  DevBuf<double> Xp, Rp, Mv, M3, mu, nu;
  LRFSI_TRY(Xp.alloc((size_t)M * K));
  LRFSI_TRY(Rp.alloc((size_t)M * K));
  LRFSI_TRY(Mv.alloc(nnz));
  LRFSI_TRY(M3.alloc((size_t)3 * nnz));
  LRFSI_TRY(mu.alloc(K));
  LRFSI_TRY(nu.alloc(K));
  LRFSI_CUDA(cudaMemcpyAsync(mu.p, mu_h, sizeof(double) * K, cudaMemcpyHostToDevice, s));
  LRFSI_CUDA(cudaMemcpyAsync(nu.p, nu_h, sizeof(double) * K, cudaMemcpyHostToDevice, s));
  k_transpose<<<ceil_div(M * K, 256), 256, 0, s>>>(Xprev_pm, K, (int)M, Xp.p);  // (K x M) -> (M x K)
  LRFSI_TRY(check_launch("k_transpose"));
  LRFSI_TRY(launch_residual(m, Xp.p, K, K, nullptr, mu.p, nu.p, Rp.p, K, s));
  LRFSI_TRY(launch_mass_fluid(m, Mv.p, s));
  k_mass_triple<<<ceil_div(nnz, 256), 256, 0, s>>>(Mv.p, nnz, M3.p);
  LRFSI_TRY(check_launch("k_mass_triple"));
  TimeStep ts;
  ts.Xprev = Xp.p;
  ts.Rprev = Rp.p;
  ts.M3 = M3.p;
  ts.Mv = Mv.p;
  ts.theta = theta;
  ts.cm = m->h.prob.rho_f / dt;
  return newton_impl(m, K, Xpm, mu_h, nu_h, nullptr, nullptr, eps, max_it, iters_h, res_h, stream, &ts);
}

extern "C" int lrfsi_mass_fluid(lrfsi_mesh_h m, double* Mv, lrfsi_stream_t stream) {
  if (!m || !Mv) return fail(LRFSI_EINVAL, "lrfsi_mass_fluid: null argument");
  return launch_mass_fluid(m, Mv, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// Subsets
// ---------------------------------------------------------------------------
struct lrfsi_subset_s {
  lrfsi_mesh_s* mesh = nullptr;
  int K = 0;
  long M = 0;
  std::vector<int> m, off, cap;
  int mtot = 0, mmax = 0, Rmax = 0, ldP = 0, ldR = 0;
  std::vector<double> mu_h, nu_h, mubar, nubar;
  DevBuf<double> mu, nu, xt, J3, R3;
  // four-parameter problem (Sec. 4.4): nu holds the affine coefficient nu rho;
  // nu_raw, lam, rho the parameters themselves (for the nonlinear residuals);
  // J3x = (Jlam', Jrho', 0) and R3x = (Rlam, Rrho, 0) per subset
  bool four = false;
  // theta-scheme time step (Sec. 4.3): operators (theta J0 + rho_f Mass / dt,
  // theta Jmu', theta Jnu'), previous states and their residual, mass triple
  bool timestep = false;
  double theta = 1.0, cm = 0.0;
  DevBuf<double> Mv, M3, Xprev, Rprev, Yth;
  std::vector<double> lambar, rhobar;
  DevBuf<double> nu_raw, lam, rho, J3x, R3x;
  DevBuf<float> J3xf;
  const double* nu_res() const { return four ? nu_raw.p : nu.p; }
  const double* rho_res() const { return four ? rho.p : nullptr; }
  const double* lam_res() const { return four ? lam.p : nullptr; }
  DevBuf<double> rsc, csc;  // K x M equilibration scales (rows, columns)
  DevBuf<double> cinv;      // K x M reciprocal column scales (allocated on first use)
  DevBuf<float> J3f, USf, Yf, Xf, Vf;  // FP32 operator copies and inner-residual buffers (mixed mode)
  PrecLU lu;
  DevBuf<double> Xcat, Q1, Q2, US, UD, UR, UZ, UB, Ytmp, UC;  // K x M x ld
  DevBuf<double> Vcat, VS, VD, VR, VB, VC;                // mtot x ld
  DevBuf<double> G, G2, T1, T2, swork, sv, frob2, gramwork;
  DevBuf<int> iwork, info;
  DevBuf<TruncDesc> tdesc;
  size_t swork_per = 0;
  // GMREST Krylov basis (allocated on first use for gm_iters steps per cycle)
  DevBuf<double> GU, GZ, GV, Gu, Gv, Gh;
  DevBuf<int> Gn;
  int gm_iters = 0;
  // dense columns for the nonlinear residual (M x mtot)
  DevBuf<double> Xd;
  ResidualCtx rc;
  // ChebyshevT as a fixed launch sequence (cheb_fixed): per-subset device
  // state, the truncation descriptors of the sequence (host copies and device
  // array), subset offsets/sizes, the bound split-K workspace and the graph
  DevBuf<int> cgi, offm;
  DevBuf<double> cgd;
  DevBuf<TruncDesc> cgt;
  std::vector<TruncDesc> cgt_host;
  DevBuf<unsigned char> cgws;
  cudaStream_t cap_stream = nullptr;
  std::vector<cudaGraphExec_t> cg_exec;  // one graph per phase of the sequence
  std::vector<uint64_t> cg_nodes;        // kernel nodes per phase graph
  std::vector<double> cg_key;
  int* live_host = nullptr;              // pinned: the live flags read after a residual
  double* tall(DevBuf<double>& b, int k, int ld) { return b.p + (size_t)k * M * ld; }
  double* vside(DevBuf<double>& b, int k, int ld) { return b.p + (size_t)off[k] * ld; }
  void drop_graph() {
    for (cudaGraphExec_t e : cg_exec)
      if (e) cudaGraphExecDestroy(e);
    cg_exec.clear();
    cg_nodes.clear();
    cg_key.clear();
  }
  ~lrfsi_subset_s() {
    drop_graph();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (live_host) cudaFreeHost(live_host);
  }
};

namespace lrfsi {

// Truncation counters (process-wide): calls, SVD sweeps (sum, max), SVDs that
// hit the sweep limit, Cholesky-QR breakdowns, retries.
static std::atomic<long long> g_tr_calls{0}, g_tr_sweeps{0}, g_tr_maxsweeps{0}, g_tr_noconv{0}, g_tr_breakdown{0},
    g_tr_retry{0};

// T([X | ...], [V | ...]) for the listed subsets.  Inputs in Xcat (ld ldP) and
// Vcat (ld ldP) with p[k] columns; outputs U (tall, ld ldR) and V (ld ldR).

static int truncate_once(lrfsi_subset_s* S, const std::vector<int>& act, const std::vector<int>& p, double tol,
                         const std::vector<int>& cap, const std::vector<double*>& Uout, const std::vector<double*>& Vout,
                         std::vector<int>& rank, std::vector<double>& frob2, double drop, std::vector<int>& broke,
                         cudaStream_t s, std::vector<double>* kept2 = nullptr) {
  const int na = (int)act.size();
  rank.assign(S->K, 0);
  frob2.assign(S->K, 0.0);
  if (kept2) kept2->assign(S->K, 0.0);
  if (!na) return LRFSI_OK;
  const int ldP = S->ldP, ldR = S->ldR;
  const long M = S->M;
  std::vector<GramDesc> gd;
  std::vector<TruncDesc> td(na);
  for (int a = 0; a < na; ++a) {
    const int k = act[a];
    gd.push_back(GramDesc{S->tall(S->Xcat, k, ldP), ldP, p[k], S->tall(S->Xcat, k, ldP), ldP, p[k],
                          S->G.p + (size_t)k * ldP * ldP, p[k]});
    TruncDesc& d = td[a];
    d.p = p[k];
    d.m = S->m[k];
    d.Vc = S->vside(S->Vcat, k, ldP);
    d.ldv = ldP;
    d.G = S->G.p + (size_t)k * ldP * ldP;
    d.G2 = S->G2.p + (size_t)k * ldP * ldP;
    d.T1 = S->T1.p + (size_t)k * ldP * ldP;
    d.T2 = S->T2.p + (size_t)k * ldP * ldP;
    d.Vout = Vout[k];
    d.ldvo = ldR;
    d.work = S->swork.p + S->swork_per * k;
    d.iwork = S->iwork.p + (size_t)2 * ldP * k;
    d.info = S->info.p + 5 * k;
    d.sv = S->sv.p + (size_t)ldP * k;
    d.frob2 = S->frob2.p + k;
    d.tol = tol;
    d.rank_cap = cap[k];
    d.drop = drop;
  }
  LRFSI_TRY(gram_batched(gd.data(), na, M, S->gramwork.p, S->gramwork.n, s));
  LRFSI_TRY(trunc_pass1(td.data(), na, s, S->tdesc.p));
  // Q1 = X T1 (tall) and the core Y = Rs Vc^T (p x m; rows >= k are zero)
  std::vector<GemmDesc<double>> gm(na), gy;
  for (int a = 0; a < na; ++a) {
    const int k = act[a];
    const TruncWork W(td[a].work, p[k], S->m[k]);
    gm[a] = GemmDesc<double>{(int)M, p[k], p[k], S->tall(S->Xcat, k, ldP), ldP, 1, td[a].T1, p[k], 1,
                             S->tall(S->Q1, k, ldP), ldP, 1, 1.0, 0.0};
    gm[a].tc = 1;
    gy.push_back(gm[a]);
    gy.push_back(GemmDesc<double>{p[k], S->m[k], p[k], W.Rk, p[k], 1, td[a].Vc, 1, td[a].ldv, W.Y, S->m[k], 1, 1.0,
                                  0.0});
  }
  LRFSI_TRY(gemm_grouped<double>(gy.data(), (int)gy.size(), s));
  for (int a = 0; a < na; ++a) {
    const int k = act[a];
    gd[a] = GramDesc{S->tall(S->Q1, k, ldP), ldP, p[k], S->tall(S->Q1, k, ldP), ldP, p[k], td[a].G2, p[k]};
  }
  LRFSI_TRY(gram_batched(gd.data(), na, M, S->gramwork.p, S->gramwork.n, s));
  {
    int pmax = 0;
    for (int a = 0; a < na; ++a) pmax = std::max(pmax, td[a].p);
    LRFSI_TRY(trunc_qr(na, s, S->tdesc.p, 1, pmax));
  }
  {  // core C = R2 Y
    std::vector<GemmDesc<double>> gc;
    for (int a = 0; a < na; ++a) {
      const int k = act[a];
      const TruncWork W(td[a].work, p[k], S->m[k]);
      gc.push_back(GemmDesc<double>{p[k], S->m[k], p[k], W.Rki, p[k], 1, W.Y, S->m[k], 1, W.C, S->m[k], 1, 1.0, 0.0});
      td[a].core = W.C;
    }
    LRFSI_TRY(gemm_grouped<double>(gc.data(), (int)gc.size(), s));
  }
  std::vector<int> info((size_t)5 * S->K);
  auto read_info = [&]() -> int {
    LRFSI_CUDA(cudaMemcpyAsync(info.data(), S->info.p, sizeof(int) * 5 * S->K, cudaMemcpyDeviceToHost, s));
    LRFSI_CUDA(cudaStreamSynchronize(s));
    return LRFSI_OK;
  };
  LRFSI_TRY(read_info());
  // a third Cholesky-QR pass where the pass-1 basis was far from orthonormal:
  // Q2 = Q1 R2^{-1}, G3 = Q2^T Q2, R3, Y <- R3 C (the input X stays intact for a retry)
  std::vector<char> third(S->K, 0);
  std::vector<TruncDesc> td2;
  std::vector<GemmDesc<double>> g2, g3;
  std::vector<GramDesc> gd2;
  broke.clear();
  std::vector<char> bad(S->K, 0);
  for (int a = 0; a < na; ++a) {
    const int k = act[a];
    if (info[5 * k + 2] == LRFSI_EBREAKDOWN) { bad[k] = 1; continue; }
    if (info[5 * k + 4]) {
      third[k] = 1;
      const int kk = info[5 * k];
      const TruncWork W(td[a].work, p[k], S->m[k]);
      g2.push_back(GemmDesc<double>{(int)M, kk, kk, S->tall(S->Q1, k, ldP), ldP, 1, td[a].T2, p[k], 1,
                                    S->tall(S->Q2, k, ldP), ldP, 1, 1.0, 0.0});
      g2.back().tc = 1;
      gd2.push_back(GramDesc{S->tall(S->Q2, k, ldP), ldP, kk, S->tall(S->Q2, k, ldP), ldP, kk, td[a].G2, p[k]});
      g3.push_back(GemmDesc<double>{p[k], S->m[k], p[k], W.Rki, p[k], 1, W.C, S->m[k], 1, W.Y, S->m[k], 1, 1.0, 0.0});
      td[a].core = W.Y;
      td2.push_back(td[a]);
    }
  }
  if (!td2.empty()) {
    LRFSI_TRY(gemm_grouped<double>(g2.data(), (int)g2.size(), s));
    LRFSI_TRY(gram_batched(gd2.data(), (int)gd2.size(), M, S->gramwork.p, S->gramwork.n, s));
    LRFSI_CUDA(cudaMemcpyAsync(S->tdesc.p + S->K, td2.data(), sizeof(TruncDesc) * td2.size(), cudaMemcpyHostToDevice, s));
    int pmax2 = 0;
    for (const TruncDesc& t : td2) pmax2 = std::max(pmax2, t.p);
    LRFSI_TRY(trunc_qr((int)td2.size(), s, S->tdesc.p + S->K, 1, pmax2));
    LRFSI_TRY(gemm_grouped<double>(g3.data(), (int)g3.size(), s));
  }
  LRFSI_TRY(trunc_svd(td.data(), na, s, S->tdesc.p));
  std::vector<double> f2(S->K), svh;
  LRFSI_CUDA(cudaMemcpyAsync(f2.data(), S->frob2.p, sizeof(double) * S->K, cudaMemcpyDeviceToHost, s));
  if (kept2) {  // singular values, for the norm of the kept part
    svh.resize((size_t)S->K * ldP);
    LRFSI_CUDA(cudaMemcpyAsync(svh.data(), S->sv.p, sizeof(double) * svh.size(), cudaMemcpyDeviceToHost, s));
  }
  LRFSI_TRY(read_info());
  {  // algorithmic FP64 work of the small kernels (upper bound: every Jacobi pair rotated)
    double fl = 0, fj = 0;
    for (int a = 0; a < na; ++a) {
      const int k = act[a];
      const double P = p[k], kk = info[5 * k];
      const double mm = S->m[k];
      const double n = std::min(kk, mm), L = std::max(kk, mm), sw = std::max(info[5 * k + 3], 1);
      fl += 2.0 * P * P * P / 3.0 + kk * kk * kk / 3.0;                 // pass 1
      fl += (third[k] ? 2.0 : 1.0) * (2.0 * kk * kk * kk / 3.0);         // QR passes
      // QR with pivoting of the L x n Jacobi matrix (updates and trailing norms),
      // Jacobi on R^T (n x n, pairs rotated with their V columns), reflectors
      // applied to the r kept columns
      fj += 3.0 * L * n * n - n * n * n + sw * n * (n - 1) / 2.0 * (6.0 * n + 8.0 * n) +
            4.0 * L * n * info[5 * k + 1];
    }
    account(KC_TRUNC, fl, 0);
    account(KC_SVD, fj, 0);
  }
  // tall coefficients T1 = T2_last W_r (k x r)
  {
    std::vector<GemmDesc<double>> gt;
    for (int a = 0; a < na; ++a) {
      const int k = act[a];
      const int r = info[5 * k + 1], kk = info[5 * k];
      if (bad[k] || info[5 * k + 2] == LRFSI_EBREAKDOWN || r <= 0) continue;
      const TruncWork W(td[a].work, p[k], S->m[k]);
      gt.push_back(GemmDesc<double>{kk, r, kk, td[a].T2, p[k], 1, W.Rk, p[k], 1, td[a].T1, p[k], 1, 1.0, 0.0});
    }
    LRFSI_TRY(gemm_grouped<double>(gt.data(), (int)gt.size(), s));
  }
  for (int a = 0; a < na; ++a) {
    const int k = act[a];
    g_tr_calls += 1;
    const int sw = info[5 * k + 3];
    if (sw > 0) {
      g_tr_sweeps += sw;
      long long cur = g_tr_maxsweeps.load();
      while (sw > cur && !g_tr_maxsweeps.compare_exchange_weak(cur, sw)) {
      }
    }
    if (info[5 * k + 2] == LRFSI_ENOCONV) g_tr_noconv += 1;
    if (bad[k] || info[5 * k + 2] == LRFSI_EBREAKDOWN) g_tr_breakdown += 1;
    rank[k] = info[5 * k + 1];
    frob2[k] = f2[k];
    if (kept2) {
      double t = 0;
      for (int j = 0; j < rank[k]; ++j) t += svh[(size_t)ldP * k + j] * svh[(size_t)ldP * k + j];
      (*kept2)[k] = t;
    }
    if (bad[k] || info[5 * k + 2] == LRFSI_EBREAKDOWN) {
      bad[k] = 1;
      broke.push_back(k);
      rank[k] = 0;
      gm[a].n = 0;  // no output GEMM for this subset
      continue;
    }
    const double* Qlast = third[k] ? S->tall(S->Q2, k, ldP) : S->tall(S->Q1, k, ldP);
    gm[a] = GemmDesc<double>{(int)M, rank[k], info[5 * k], Qlast, ldP, 1, td[a].T1, p[k], 1, Uout[k], ldR, 1, 1.0,
                             0.0};
    gm[a].tc = 1;
  }
  LRFSI_TRY(gemm_grouped<double>(gm.data(), na, s));
  return LRFSI_OK;
}

// T with a retry: a Cholesky-QR breakdown (basis still too ill-conditioned
// after dropping) is retried with a 100x larger drop threshold, at most three
// times (the lost relative remainder grows from 1e-7 to 1e-4 of a column).
static int truncate_batch(lrfsi_subset_s* S, const std::vector<int>& act, const std::vector<int>& p, double tol,
                          const std::vector<int>& cap, const std::vector<double*>& Uout, const std::vector<double*>& Vout,
                          std::vector<int>& rank, std::vector<double>& frob2, cudaStream_t s, double drop0 = 1e-14,
                          std::vector<double>* kept2 = nullptr) {
  std::vector<int> broke, todo = act;
  rank.assign(S->K, 0);
  frob2.assign(S->K, 0.0);
  if (kept2) kept2->assign(S->K, 0.0);
  double drop = drop0;
  for (int attempt = 0; attempt < 4 && !todo.empty(); ++attempt, drop *= 100.0) {
    std::vector<int> rk;
    std::vector<double> f2, k2;
    LRFSI_TRY(truncate_once(S, todo, p, tol, cap, Uout, Vout, rk, f2, drop, broke, s, kept2 ? &k2 : nullptr));
    for (int k : todo) {
      rank[k] = rk[k];
      frob2[k] = f2[k];
      if (kept2) (*kept2)[k] = k2[k];
    }
    todo = broke;
    g_tr_retry += (long long)broke.size();
  }
  if (!todo.empty()) return fail(LRFSI_EBREAKDOWN, "truncation: Cholesky-QR breakdown after retries");
  return LRFSI_OK;
}

}  // namespace lrfsi

extern "C" int lrfsi_spmm(lrfsi_mesh_h m, const void* J3, const void* U, int ldu, int r, void* Y, int ldy,
                          int precision, lrfsi_stream_t stream) {
  if (!m || !J3 || !U || !Y || r < 0 || ldu < r || ldy < 3 * r || (precision != 0 && precision != 1))
    return fail(LRFSI_EINVAL, "lrfsi_spmm: bad argument (ldu >= r, ldy >= 3 r, precision 0 or 1)");
  if (r == 0) return LRFSI_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == 0) {
    SpmmDesc<double> d;
    d.J3 = (const double*)J3; d.U = (const double*)U; d.ldu = ldu; d.r = r; d.Y = (double*)Y; d.ldy = ldy;
    d.o[0] = 0; d.o[1] = r; d.o[2] = 2 * r;
    d.sc[0] = d.sc[1] = d.sc[2] = 1.0;
    d.a1 = d.a2 = 0.0;
    return spmm_batched<double>(m, &d, 1, s);
  }
  SpmmDesc<float> d;
  d.J3 = (const float*)J3; d.U = (const float*)U; d.ldu = ldu; d.r = r; d.Y = (float*)Y; d.ldy = ldy;
  d.o[0] = 0; d.o[1] = r; d.o[2] = 2 * r;
  d.sc[0] = d.sc[1] = d.sc[2] = 1.0f;
  d.a1 = d.a2 = 0.0f;
  return spmm_batched<float>(m, &d, 1, s);
}

extern "C" int lrfsi_spmm_tuning(int precision, int bucket, int* variant, float* ms9) {
  if (!variant || !ms9) return fail(LRFSI_EINVAL, "lrfsi_spmm_tuning: null argument");
  if (spmm_autotune_table(precision, bucket, variant, ms9) != LRFSI_OK)
    return fail(LRFSI_EINVAL, "lrfsi_spmm_tuning: precision 0/1, bucket 0..8");
  return LRFSI_OK;
}

extern "C" int lrfsi_truncation_counters(int64_t* out6, int reset) {
  if (!out6) return fail(LRFSI_EINVAL, "lrfsi_truncation_counters: null argument");
  out6[0] = g_tr_calls.load();
  out6[1] = g_tr_sweeps.load();
  out6[2] = g_tr_maxsweeps.load();
  out6[3] = g_tr_noconv.load();
  out6[4] = g_tr_breakdown.load();
  out6[5] = g_tr_retry.load();
  if (reset) {
    g_tr_calls = 0; g_tr_sweeps = 0; g_tr_maxsweeps = 0; g_tr_noconv = 0; g_tr_breakdown = 0; g_tr_retry = 0;
  }
  return LRFSI_OK;
}

extern "C" int lrfsi_subset_destroy(lrfsi_subset_h S) {
  delete S;
  return LRFSI_OK;
}

extern "C" size_t lrfsi_subset_bytes(lrfsi_subset_h S) {
  if (!S) return 0;
  size_t b = 0;
  for (DevBuf<double>* p : {&S->mu, &S->nu, &S->xt, &S->J3, &S->R3, &S->rsc, &S->csc, &S->cinv, &S->Xcat, &S->Q1, &S->Q2, &S->US, &S->UD, &S->UR, &S->UZ,
                            &S->UB, &S->Ytmp, &S->UC, &S->Vcat, &S->VS, &S->VD, &S->VR, &S->VB, &S->VC, &S->G, &S->G2,
                            &S->T1, &S->T2, &S->swork, &S->sv, &S->frob2, &S->gramwork, &S->GU, &S->GZ, &S->GV,
                            &S->Gu, &S->Gv, &S->Gh, &S->Xd, &S->rc.R,
                            &S->rc.norm2, &S->rc.norm2_bD, &S->rc.work})
    b += p->bytes();
  for (DevBuf<float>* p : {&S->J3f, &S->USf, &S->Yf, &S->Xf, &S->Vf}) b += p->bytes();
  return b + S->iwork.bytes() + S->info.bytes() + S->tdesc.bytes() + S->Gn.bytes() + S->lu.bytes();
}

namespace lrfsi {
// Workspace of a subset handle (factors, concatenation buffers, truncation
// scratch, dense residual columns); S->K, M, m, cap, off, mtot, mmax, Rmax set.
static int subset_alloc_ws(lrfsi_subset_s* S, cudaStream_t s) {
  const int K = S->K;
  const long M = S->M;
  // largest concatenation: residual [B | J0 U | Jmu U | Jnu U] with rank(B) <= max(R, m)
  S->ldR = std::max(std::max(S->Rmax, S->mmax), S->four ? 5 : 3);
  S->ldP = S->ldR + (S->four ? 6 : 3) * S->Rmax + 4;
  const int ldP = S->ldP, ldR = S->ldR;
  for (DevBuf<double>* b : {&S->Xcat, &S->Q1, &S->Q2}) LRFSI_TRY(b->alloc((size_t)K * M * ldP));
  for (DevBuf<double>* b : {&S->US, &S->UD, &S->UR, &S->UZ, &S->UB, &S->Ytmp, &S->UC})
    LRFSI_TRY(b->alloc((size_t)K * M * ldR));
  LRFSI_TRY(S->Vcat.alloc((size_t)S->mtot * ldP));
  for (DevBuf<double>* b : {&S->VS, &S->VD, &S->VR, &S->VB, &S->VC}) LRFSI_TRY(b->alloc((size_t)S->mtot * ldR));
  for (DevBuf<double>* b : {&S->G, &S->G2, &S->T1, &S->T2}) LRFSI_TRY(b->alloc((size_t)K * ldP * ldP));
  S->swork_per = trunc_small_work(ldP, S->mmax);
  LRFSI_TRY(S->swork.alloc(S->swork_per * K));
  LRFSI_TRY(S->sv.alloc((size_t)K * ldP));
  LRFSI_TRY(S->frob2.alloc(K));
  LRFSI_TRY(S->iwork.alloc((size_t)2 * ldP * K));
  LRFSI_TRY(S->info.alloc((size_t)5 * K));
  LRFSI_TRY(S->tdesc.alloc(2 * K));
  LRFSI_TRY(S->gramwork.alloc(gram_work_len(K, M, ldP, ldP)));
  LRFSI_TRY(S->Xd.alloc((size_t)M * S->mtot));
  LRFSI_TRY(S->rc.init(M, S->mtot));
  return LRFSI_OK;
}
}  // namespace lrfsi

namespace lrfsi {
// J0 slot of P's values for the four-parameter preconditioner:
// Jeff = (J0 + lam_bar Jlam' + rho_bar Jrho', Jmu', Jnurho')
__global__ void k_four_precond(const double* __restrict__ Ja, const double* __restrict__ Jb, long nnz, double lb,
                               double rb, double* __restrict__ Je) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  Je[3 * e] = Ja[3 * e] + lb * Jb[3 * e] + rb * Jb[3 * e + 1];
  Je[3 * e + 1] = Ja[3 * e + 1];
  Je[3 * e + 2] = Ja[3 * e + 2];
}
}  // namespace lrfsi

static int subset_create_impl(lrfsi_mesh_h mesh, int K, const double* xt, const double* mu_h, const double* nu_h,
                              const double* lam_h, const double* rho_h, const int* m_h, const int* cap_h,
                              lrfsi_subset_h* out, lrfsi_stream_t stream, double theta = 0.0, double dt = 0.0) {
  if (!mesh || !xt || !mu_h || !nu_h || !m_h || !cap_h || !out || K < 1 || K > kMaxGemmDescs)
    return fail(LRFSI_EINVAL, "lrfsi_subset_create: bad argument (1 <= K <= 32)");
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  lrfsi_subset_s* S = new (std::nothrow) lrfsi_subset_s();
  if (!S) return fail(LRFSI_ENOMEM, "lrfsi_subset_create: host allocation");
  std::unique_ptr<lrfsi_subset_s> guard(S);
  S->mesh = mesh;
  S->K = K;
  S->M = mesh->h.M;
  const long M = S->M;
  S->m.assign(m_h, m_h + K);
  S->cap.assign(cap_h, cap_h + K);
  S->off.assign(K, 0);
  for (int k = 0; k < K; ++k) {
    if (S->m[k] < 1 || S->cap[k] < 1) return fail(LRFSI_EINVAL, "lrfsi_subset_create: m_k and R_k must be >= 1");
    S->off[k] = S->mtot;
    S->mtot += S->m[k];
    S->mmax = std::max(S->mmax, S->m[k]);
    S->Rmax = std::max(S->Rmax, S->cap[k]);
  }
  for (int i = 0; i < S->mtot; ++i)
    if (!std::isfinite(mu_h[i]) || !std::isfinite(nu_h[i]) || (lam_h && !std::isfinite(lam_h[i])) ||
        (rho_h && !std::isfinite(rho_h[i])))
      return fail(LRFSI_EINVAL, "lrfsi_subset_create: parameters must be finite");
  S->four = lam_h && rho_h;
  LRFSI_TRY(subset_alloc_ws(S, s));
  const long nnz = (long)mesh->h.colidx.size();
  const int ldP = S->ldP, ldR = S->ldR;
  S->mu_h.assign(mu_h, mu_h + S->mtot);
  S->nu_h.assign(nu_h, nu_h + S->mtot);
  if (S->four) {  // the affine coefficient of A2 is nu rho
    std::vector<double> lam_v(lam_h, lam_h + S->mtot), rho_v(rho_h, rho_h + S->mtot);
    LRFSI_TRY(S->nu_raw.upload(S->nu_h, s));
    LRFSI_TRY(S->lam.upload(lam_v, s));
    LRFSI_TRY(S->rho.upload(rho_v, s));
    for (int i = 0; i < S->mtot; ++i) S->nu_h[i] *= rho_h[i];
    LRFSI_TRY(S->J3x.alloc((size_t)K * 3 * nnz));
    LRFSI_TRY(S->R3x.alloc((size_t)K * 3 * M));
  }
  LRFSI_TRY(S->mu.upload(S->mu_h, s));
  LRFSI_TRY(S->nu.upload(S->nu_h, s));
  LRFSI_TRY(S->xt.alloc((size_t)K * M));
  LRFSI_CUDA(cudaMemcpyAsync(S->xt.p, xt, sizeof(double) * K * M, cudaMemcpyDeviceToDevice, s));
  LRFSI_TRY(S->J3.alloc((size_t)K * 3 * nnz));
  LRFSI_TRY(S->R3.alloc((size_t)K * 3 * M));
  // operators at xt_k and the preconditioners at the midpoint parameters
  std::vector<const double*> J3p(K);
  for (int k = 0; k < K; ++k) {
    double* Jk = S->J3.p + (size_t)k * 3 * nnz;
    J3p[k] = Jk;
    if (S->four) {
      LRFSI_TRY(assemble_five(mesh, S->xt.p + (size_t)k * M, Jk, S->J3x.p + (size_t)k * 3 * nnz,
                              S->R3.p + (size_t)k * 3 * M, S->R3x.p + (size_t)k * 3 * M, s));
      double llo = 1e300, lhi = -1e300, rlo = 1e300, rhi = -1e300;
      for (int i = S->off[k]; i < S->off[k] + S->m[k]; ++i) {
        llo = std::min(llo, lam_h[i]); lhi = std::max(lhi, lam_h[i]);
        rlo = std::min(rlo, rho_h[i]); rhi = std::max(rhi, rho_h[i]);
      }
      S->lambar.push_back(0.5 * (llo + lhi));
      S->rhobar.push_back(0.5 * (rlo + rhi));
    } else {
      LRFSI_TRY(lrfsi_assemble_affine(mesh, S->xt.p + (size_t)k * M, Jk, S->R3.p + (size_t)k * 3 * M, stream));
    }
    double mlo = 1e300, mhi = -1e300, nlo = 1e300, nhi = -1e300;
    for (int i = S->off[k]; i < S->off[k] + S->m[k]; ++i) {
      mlo = std::min(mlo, S->mu_h[i]); mhi = std::max(mhi, S->mu_h[i]);
      nlo = std::min(nlo, S->nu_h[i]); nhi = std::max(nhi, S->nu_h[i]);
    }
    S->mubar.push_back(0.5 * (mlo + mhi));
    S->nubar.push_back(0.5 * (nlo + nhi));
  }
  if (theta > 0) {  // time step: (theta J0 + rho_f Mass / dt, theta Jmu', theta Jnu')
    S->timestep = true;
    S->theta = theta;
    S->cm = mesh->h.prob.rho_f / dt;
    LRFSI_TRY(S->Mv.alloc(nnz));
    LRFSI_TRY(S->M3.alloc((size_t)3 * nnz));
    LRFSI_TRY(S->Xprev.alloc((size_t)M * S->mtot));
    LRFSI_TRY(S->Rprev.alloc((size_t)M * S->mtot));
    LRFSI_TRY(S->Yth.alloc((size_t)M * S->mtot));
    LRFSI_TRY(launch_mass_fluid(mesh, S->Mv.p, s));
    k_mass_triple<<<ceil_div(nnz, 256), 256, 0, s>>>(S->Mv.p, nnz, S->M3.p);
    LRFSI_TRY(check_launch("k_mass_triple"));
    for (int k = 0; k < K; ++k) {
      k_theta_ops<<<ceil_div(nnz, 256), 256, 0, s>>>(S->J3.p + (size_t)k * 3 * nnz, nnz, theta, S->cm, S->Mv.p);
      LRFSI_TRY(check_launch("k_theta_ops"));
    }
  }
  // equilibrate P_k and scale the operator values: the iteration and the
  // truncation run on diag(r) F(diag(c) S~) = diag(r) B
  LRFSI_TRY(S->rsc.alloc((size_t)K * M));
  LRFSI_TRY(S->csc.alloc((size_t)K * M));
  DevBuf<double> Jeff;  // four parameters: P's values as one (J0, Jmu', Jnurho') triple per subset
  if (S->four) {
    LRFSI_TRY(Jeff.alloc((size_t)K * 3 * nnz));
    for (int k = 0; k < K; ++k) {
      k_four_precond<<<ceil_div(nnz, 256), 256, 0, s>>>(S->J3.p + (size_t)k * 3 * nnz, S->J3x.p + (size_t)k * 3 * nnz,
                                                         nnz, S->lambar[k], S->rhobar[k], Jeff.p + (size_t)k * 3 * nnz);
      LRFSI_TRY(check_launch("k_four_precond"));
      J3p[k] = Jeff.p + (size_t)k * 3 * nnz;
    }
  }
  {
    DevBuf<unsigned long long> cmax;
    LRFSI_TRY(cmax.alloc(M));
    for (int k = 0; k < K; ++k) {
      double* Jk = const_cast<double*>(J3p[k]);
      double* rk = S->rsc.p + (size_t)k * M;
      double* ck = S->csc.p + (size_t)k * M;
      k_equil_rows<<<ceil_div(M, 256), 256, 0, s>>>(Jk, mesh->rowptr.p, M, S->mubar[k], S->nubar[k], rk);
      LRFSI_TRY(check_launch("k_equil_rows"));
      LRFSI_CUDA(cudaMemsetAsync(cmax.p, 0, sizeof(unsigned long long) * M, s));
      k_equil_colmax<<<ceil_div(M, 256), 256, 0, s>>>(Jk, mesh->rowptr.p, mesh->colidx.p, M, S->mubar[k], S->nubar[k],
                                                       rk, cmax.p);
      LRFSI_TRY(check_launch("k_equil_colmax"));
      k_equil_cols<<<ceil_div(M, 256), 256, 0, s>>>(cmax.p, M, ck);
      LRFSI_TRY(check_launch("k_equil_cols"));
      k_scale_vals<<<ceil_div(M, 256), 256, 0, s>>>(Jk, mesh->rowptr.p, mesh->colidx.p, M, rk, ck);
      LRFSI_TRY(check_launch("k_scale_vals"));
      if (S->four) {  // the operators themselves
        k_scale_vals<<<ceil_div(M, 256), 256, 0, s>>>(S->J3.p + (size_t)k * 3 * nnz, mesh->rowptr.p, mesh->colidx.p, M,
                                                       rk, ck);
        LRFSI_TRY(check_launch("k_scale_vals"));
        k_scale_vals<<<ceil_div(M, 256), 256, 0, s>>>(S->J3x.p + (size_t)k * 3 * nnz, mesh->rowptr.p, mesh->colidx.p,
                                                       M, rk, ck);
        LRFSI_TRY(check_launch("k_scale_vals"));
      }
    }
    LRFSI_CUDA(cudaStreamSynchronize(s));
  }
  // FP32 copies for the mixed-precision inner iteration
  {
    LRFSI_TRY(S->J3f.alloc((size_t)K * 3 * nnz));
    std::vector<ConvDesc> cv;
    for (int k = 0; k < K; ++k)
      cv.push_back(ConvDesc{S->J3.p + (size_t)k * 3 * nnz, 0, S->J3f.p + (size_t)k * 3 * nnz, 0, 3 * nnz, 1, nullptr,
                            1.0});
    if (S->four) {
      LRFSI_TRY(S->J3xf.alloc((size_t)K * 3 * nnz));
      for (int k = 0; k < K; ++k)
        cv.push_back(ConvDesc{S->J3x.p + (size_t)k * 3 * nnz, 0, S->J3xf.p + (size_t)k * 3 * nnz, 0, 3 * nnz, 1,
                              nullptr, 1.0});
    }
    for (auto& c : cv) { c.lds = 1; c.ldd = 1; }
    LRFSI_TRY((convert_batched<double, float>(cv, s)));
    LRFSI_TRY(S->USf.alloc((size_t)K * M * ldR));
    LRFSI_TRY(S->Yf.alloc((size_t)K * M * ldP));
    LRFSI_TRY(S->Xf.alloc((size_t)K * M * ldP));
    LRFSI_TRY(S->Vf.alloc((size_t)S->mtot * ldP));
  }
  LRFSI_TRY(S->lu.alloc(mesh, K, ldR));
  LRFSI_TRY(S->lu.factor(mesh, J3p.data(), S->mubar.data(), S->nubar.data(), K, s));
  std::vector<int> st;
  LRFSI_TRY(S->lu.status(K, st, s));
  for (int k = 0; k < K; ++k)
    if (st[k]) return fail(LRFSI_ESINGULAR, "lrfsi_subset_create: zero pivot in a preconditioner LU");
  LRFSI_TRY(residual_bD_norms(mesh, S->rc, S->mu.p, S->nu_res(), s, S->rho_res(), S->lam_res()));
  LRFSI_CUDA(cudaStreamSynchronize(s));
  *out = guard.release();
  return LRFSI_OK;
}

extern "C" int lrfsi_subset_create(lrfsi_mesh_h mesh, int K, const double* xt, const double* mu_h, const double* nu_h,
                                   const int* m_h, const int* cap_h, lrfsi_subset_h* out, lrfsi_stream_t stream) {
  return subset_create_impl(mesh, K, xt, mu_h, nu_h, nullptr, nullptr, m_h, cap_h, out, stream);
}

extern "C" int lrfsi_subset_create_theta(lrfsi_mesh_h mesh, int K, const double* xt, const double* mu_h,
                                         const double* nu_h, const int* m_h, const int* cap_h, double theta, double dt,
                                         lrfsi_subset_h* out, lrfsi_stream_t stream) {
  if (!(theta > 0 && theta <= 1) || !(dt > 0))
    return fail(LRFSI_EINVAL, "lrfsi_subset_create_theta: need 0 < theta <= 1 and dt > 0");
  return subset_create_impl(mesh, K, xt, mu_h, nu_h, nullptr, nullptr, m_h, cap_h, out, stream, theta, dt);
}

extern "C" int lrfsi_subset_create4(lrfsi_mesh_h mesh, int K, const double* xt, const double* mu_h, const double* nu_h,
                                    const double* lam_h, const double* rho_h, const int* m_h, const int* cap_h,
                                    lrfsi_subset_h* out, lrfsi_stream_t stream) {
  if (!lam_h || !rho_h) return fail(LRFSI_EINVAL, "lrfsi_subset_create4: null lambda_s / rho_f");
  return subset_create_impl(mesh, K, xt, mu_h, nu_h, lam_h, rho_h, m_h, cap_h, out, stream);
}

namespace lrfsi {

// ||B_k||_F of the dense right-hand sides in UB (M x m_k), from column norms.
static int rhs_norms(lrfsi_subset_s* S, const std::vector<int>& act, std::vector<double>& nB, cudaStream_t s) {
  const int ldR = S->ldR;
  const long M = S->M;
  nB.assign(S->K, 0.0);
  for (int k : act)
    LRFSI_TRY(launch_colnorm2(S->tall(S->UB, k, ldR), M, S->m[k], ldR, S->rc.norm2.p + S->off[k], S->rc.work.p,
                              S->rc.work.n, s));
  std::vector<double> cn(S->mtot);
  LRFSI_CUDA(cudaMemcpyAsync(cn.data(), S->rc.norm2.p, sizeof(double) * S->mtot, cudaMemcpyDeviceToHost, s));
  LRFSI_CUDA(cudaStreamSynchronize(s));
  for (int k : act) {
    double t = 0;
    for (int i = S->off[k]; i < S->off[k] + S->m[k]; ++i) t += cn[i];
    nB[k] = std::sqrt(t);
  }
  return LRFSI_OK;
}

// Residual Res = B - F(S) of the subsets in L (B dense in UB, S = US VS^T of
// rank rS), formed densely in Xcat (M x m_k) and truncated into UR/VR (ranks
// rR); the dense form avoids cancellation between the factors of B and F(S).
// nres[k] = ||Res_k||_F; kept2[k] (optional) = ||T(Res_k)||_F^2.
static int lr_residual(lrfsi_subset_s* S, const lrfsi_cheb_options& o, const std::vector<int>& L,
                       const std::vector<int>& rS, const std::vector<double>& nB, std::vector<int>& rR,
                       std::vector<double>& nres, std::vector<lrfsi_cheb_stats>& st, cudaStream_t s,
                       std::vector<double>* kept2 = nullptr) {
  const int K = S->K, ldP = S->ldP, ldR = S->ldR;
  const long M = S->M;
  const long nnz = (long)S->mesh->h.colidx.size();
  std::vector<int> p(K, 0), rk;
  std::vector<double*> Uo(K), Vo(K);
  std::vector<double> f2;
  std::vector<CopyDesc> cd, cd2;
  std::vector<SpmmDesc<double>> sd;
  std::vector<GemmDesc<double>> gm;
  for (int k : L) {
    double* X = S->tall(S->Xcat, k, ldP);
    double* Vc = S->vside(S->Vcat, k, ldP);
    const int m = S->m[k];
    cd.push_back(CopyDesc{S->tall(S->UB, k, ldR), ldR, X, ldP, M, m, 0, nullptr, 1.0});
    const int r = rS[k];
    if (r > 0) {
      const double* mu = S->mu.p + S->off[k];
      const double* nu = S->nu.p + S->off[k];
      cd.push_back(CopyDesc{S->vside(S->VS, k, ldR), ldR, Vc, ldP, m, r, 0, nullptr, 1.0});
      cd.push_back(CopyDesc{S->vside(S->VS, k, ldR), ldR, Vc + r, ldP, m, r, 0, mu, 1.0});
      cd.push_back(CopyDesc{S->vside(S->VS, k, ldR), ldR, Vc + 2 * r, ldP, m, r, 0, nu, 1.0});
      SpmmDesc<double> d;
      d.J3 = S->J3.p + (size_t)k * 3 * nnz;
      d.U = S->tall(S->US, k, ldR);
      d.ldu = ldR;
      d.r = r;
      d.Y = S->tall(S->Q1, k, ldP);
      d.ldy = ldP;
      d.o[0] = 0; d.o[1] = r; d.o[2] = 2 * r;
      d.sc[0] = d.sc[1] = d.sc[2] = 1.0;
      d.a1 = d.a2 = 0.0;
      sd.push_back(d);
      if (S->four) {  // + Jlam' S D_lam + Jrho' S D_rho (Sec. 4.4)
        cd.push_back(CopyDesc{S->vside(S->VS, k, ldR), ldR, Vc + 3 * r, ldP, m, r, 0, S->lam.p + S->off[k], 1.0});
        cd.push_back(CopyDesc{S->vside(S->VS, k, ldR), ldR, Vc + 4 * r, ldP, m, r, 0, S->rho.p + S->off[k], 1.0});
        SpmmDesc<double> d2 = d;
        d2.J3 = S->J3x.p + (size_t)k * 3 * nnz;
        d2.o[0] = 3 * r; d2.o[1] = 4 * r; d2.o[2] = 5 * r;
        d2.sc[2] = 0.0;
        sd.push_back(d2);
      }
      gm.push_back(GemmDesc<double>{(int)M, m, (S->four ? 5 : 3) * r, S->tall(S->Q1, k, ldP), ldP, 1, Vc, 1, ldP, X,
                                    ldP, 1, -1.0, 1.0});
      gm.back().tc = 1;
    }
    cd2.push_back(CopyDesc{nullptr, 0, Vc, ldP, m, m, 2, nullptr, 1.0});
    p[k] = m;
    Uo[k] = S->tall(S->UR, k, ldR);
    Vo[k] = S->vside(S->VR, k, ldR);
  }
  LRFSI_TRY(copy_batched(cd, s));
  if (!sd.empty() && o.precision == 0) {
    LRFSI_TRY(spmm_batched<double>(S->mesh, sd.data(), (int)sd.size(), s));
    LRFSI_TRY(gemm_grouped<double>(gm.data(), (int)gm.size(), s));
  } else if (!sd.empty()) {
    // mixed: B - F(S) with an FP32 SpMM and an FP32 GEMM (FP32 accumulation);
    // the result is widened to FP64 for the truncation
    std::vector<ConvDesc> c1, c2;
    std::vector<SpmmDesc<float>> sdf;
    std::vector<GemmDesc<float>> gmf;
    for (size_t q = 0; q < sd.size(); ++q) {
      if (S->four && sd[q].o[0] != 0) continue;  // the second operator triple is added below
      // subset of this SpMM descriptor
      int k = -1;
      for (int kk : L)
        if (S->tall(S->US, kk, ldR) == sd[q].U) k = kk;
      const int r = rS[k], m = S->m[k];
      const int kc = (S->four ? 5 : 3) * r;
      float* Uf = S->USf.p + (size_t)k * M * ldR;
      float* Yf = S->Yf.p + (size_t)k * M * ldP;
      float* Xf = S->Xf.p + (size_t)k * M * ldP;
      float* Vf = S->Vf.p + (size_t)S->off[k] * ldP;
      c1.push_back(ConvDesc{S->tall(S->US, k, ldR), ldR, Uf, ldR, M, r, nullptr, 1.0});
      c1.push_back(ConvDesc{S->tall(S->Xcat, k, ldP), ldP, Xf, ldP, M, m, nullptr, 1.0});
      c1.push_back(ConvDesc{S->vside(S->Vcat, k, ldP), ldP, Vf, ldP, m, kc, nullptr, 1.0});
      SpmmDesc<float> d;
      d.J3 = S->J3f.p + (size_t)k * 3 * nnz;
      d.U = Uf; d.ldu = ldR; d.r = r; d.Y = Yf; d.ldy = ldP;
      d.o[0] = 0; d.o[1] = r; d.o[2] = 2 * r;
      d.sc[0] = d.sc[1] = d.sc[2] = 1.0f;
      d.a1 = d.a2 = 0.0f;
      sdf.push_back(d);
      if (S->four) {
        SpmmDesc<float> d2 = d;
        d2.J3 = S->J3xf.p + (size_t)k * 3 * nnz;
        d2.o[0] = 3 * r; d2.o[1] = 4 * r; d2.o[2] = 5 * r;
        d2.sc[2] = 0.0f;
        sdf.push_back(d2);
      }
      gmf.push_back(GemmDesc<float>{(int)M, m, kc, Yf, ldP, 1, Vf, 1, ldP, Xf, ldP, 1, -1.0f, 1.0f});
      c2.push_back(ConvDesc{Xf, ldP, S->tall(S->Xcat, k, ldP), ldP, M, m, nullptr, 1.0});
    }
    LRFSI_TRY((convert_batched<double, float>(c1, s)));
    LRFSI_TRY(spmm_batched<float>(S->mesh, sdf.data(), (int)sdf.size(), s));
    LRFSI_TRY(gemm_grouped<float>(gmf.data(), (int)gmf.size(), s));
    LRFSI_TRY((convert_batched<float, double>(c2, s)));
  }
  LRFSI_TRY(copy_batched(cd2, s));
  // a residual formed in FP32 carries rounding noise of ~1e-7 of its terms in
  // every direction: it is truncated at that level (tolerance 1e-6, pivoted
  // Cholesky remainder 1e-6) instead of resolving the noise
  if (o.precision == 1) {
    LRFSI_TRY(truncate_batch(S, L, p, std::max(o.tol, 1e-6), S->cap, Uo, Vo, rk, f2, s, 1e-12, kept2));
  } else {
    LRFSI_TRY(truncate_batch(S, L, p, o.tol, S->cap, Uo, Vo, rk, f2, s, 1e-14, kept2));
  }
  nres.assign(K, 0.0);
  for (int k : L) {
    rR[k] = rk[k];
    nres[k] = std::sqrt(f2[k]);
    st[k].rel_lin_res = nres[k] / nB[k];
    st[k].max_concat_rank = std::max(st[k].max_concat_rank, 3 * rS[k]);
  }
  return LRFSI_OK;
}

// Y_k = P_k^{-1} X_k on tall factors (M x r[k], ld ldR) for the subsets in L
// with r[k] > 0; X_k is first copied to Ytmp (the solve overwrites its input).
static int lr_precond(lrfsi_subset_s* S, const std::vector<int>& L, const std::vector<double*>& X,
                      const std::vector<double*>& Y, const std::vector<int>& r, cudaStream_t s) {
  const int K = S->K, ldR = S->ldR;
  const long M = S->M;
  std::vector<CopyDesc> cd;
  // the LU batch is indexed by subset: problems of the factorisation are the
  // K subsets in order; subsets without work get r = 0 (their GEMMs are skipped)
  std::vector<double*> X2(K), Y2(K);
  std::vector<int> r2(K, 0);
  bool any = false;
  for (int k = 0; k < K; ++k) {
    X2[k] = S->tall(S->Ytmp, k, ldR);
    Y2[k] = S->tall(S->UZ, k, ldR);
  }
  for (int k : L) {
    if (r[k] == 0) continue;
    cd.push_back(CopyDesc{X[k], ldR, S->tall(S->Ytmp, k, ldR), ldR, M, r[k], 0, nullptr, 1.0});
    Y2[k] = Y[k];
    r2[k] = r[k];
    any = true;
  }
  if (!any) return LRFSI_OK;
  LRFSI_TRY(copy_batched(cd, s));
  return S->lu.solve(X2.data(), Y2.data(), r2.data(), ldR, K, s);
}

// Chebyshev on factors for the subsets in `act`; B given densely in UB.
// Results in US/VS with rank rS[k].
static int cheb_run(lrfsi_subset_s* S, const lrfsi_cheb_options& o, std::vector<int> act, std::vector<int>& rS,
                    std::vector<lrfsi_cheb_stats>& st, cudaStream_t s) {
  const int K = S->K, ldP = S->ldP, ldR = S->ldR;
  const long M = S->M;
  rS.assign(K, 0);
  st.assign(K, lrfsi_cheb_stats{0, 0, 1.0, 0});
  std::vector<int> rD(K, 0), rR(K, 0), p(K, 0);
  std::vector<double> nB, rho(K, 0.0);
  std::vector<double*> Uo(K), Vo(K), UR(K), UZ(K);
  std::vector<int> rk;
  std::vector<double> f2;
  const double sigma = o.d / o.c;
  for (int k = 0; k < K; ++k) {
    UR[k] = S->tall(S->UR, k, ldR);
    UZ[k] = S->tall(S->UZ, k, ldR);
  }
  LRFSI_TRY(rhs_norms(S, act, nB, s));
  std::vector<int> live;
  for (int k : act)
    if (nB[k] > 0) live.push_back(k);
  for (int cyc = 0; cyc < o.cycles && !live.empty(); ++cyc) {
    std::vector<double> nres;
    LRFSI_TRY(lr_residual(S, o, live, rS, nB, rR, nres, st, s));
    std::vector<int> next;
    for (int k : live) {
      if (o.eta > 0 && nres[k] <= o.eta * nB[k]) continue;
      next.push_back(k);
    }
    live.swap(next);
    if (live.empty()) break;
    LRFSI_TRY(lr_precond(S, live, UR, UZ, rR, s));  // Z = P^{-1} U_R
    {  // Delta = Z / d
      std::vector<CopyDesc> cd;
      for (int k : live) {
        cd.push_back(CopyDesc{S->tall(S->UZ, k, ldR), ldR, S->tall(S->UD, k, ldR), ldR, M, rR[k], 0, nullptr, 1.0});
        cd.push_back(CopyDesc{S->vside(S->VR, k, ldR), ldR, S->vside(S->VD, k, ldR), ldR, S->m[k], rR[k], 0, nullptr,
                              1.0 / o.d});
        rD[k] = rR[k];
        rho[k] = 1.0 / sigma;
      }
      LRFSI_TRY(copy_batched(cd, s));
    }
    for (int j = 0; j < o.iters && !live.empty(); ++j) {
      // S <- T([U_S | U_D], [V_S | V_D])
      {
        std::vector<CopyDesc> cd;
        for (int k : live) {
          cd.push_back(CopyDesc{S->tall(S->US, k, ldR), ldR, S->tall(S->Xcat, k, ldP), ldP, M, rS[k], 0, nullptr, 1.0});
          cd.push_back(CopyDesc{S->tall(S->UD, k, ldR), ldR, S->tall(S->Xcat, k, ldP) + rS[k], ldP, M, rD[k], 0, nullptr,
                                1.0});
          cd.push_back(CopyDesc{S->vside(S->VS, k, ldR), ldR, S->vside(S->Vcat, k, ldP), ldP, S->m[k], rS[k], 0, nullptr,
                                1.0});
          cd.push_back(CopyDesc{S->vside(S->VD, k, ldR), ldR, S->vside(S->Vcat, k, ldP) + rS[k], ldP, S->m[k], rD[k], 0,
                                nullptr, 1.0});
          p[k] = rS[k] + rD[k];
          Uo[k] = S->tall(S->US, k, ldR);
          Vo[k] = S->vside(S->VS, k, ldR);
        }
        LRFSI_TRY(copy_batched(cd, s));
        LRFSI_TRY(truncate_batch(S, live, p, o.tol, S->cap, Uo, Vo, rk, f2, s));
        for (int k : live) {
          rS[k] = rk[k];
          st[k].steps += 1;
        }
      }
      if (j == o.iters - 1) break;
      std::vector<double> nres2;
      LRFSI_TRY(lr_residual(S, o, live, rS, nB, rR, nres2, st, s));
      std::vector<int> next2;
      for (int k : live)
        if (!(o.eta > 0 && nres2[k] <= o.eta * nB[k])) next2.push_back(k);
      live.swap(next2);
      if (live.empty()) break;
      LRFSI_TRY(lr_precond(S, live, UR, UZ, rR, s));
      // Delta <- T([U_D | U_Z], [rho' rho V_D | (2 rho' / c) V_R])
      {
        std::vector<CopyDesc> cd;
        for (int k : live) {
          const double rn = 1.0 / (2.0 * sigma - rho[k]);
          cd.push_back(CopyDesc{S->tall(S->UD, k, ldR), ldR, S->tall(S->Xcat, k, ldP), ldP, M, rD[k], 0, nullptr, 1.0});
          cd.push_back(CopyDesc{S->tall(S->UZ, k, ldR), ldR, S->tall(S->Xcat, k, ldP) + rD[k], ldP, M, rR[k], 0, nullptr,
                                1.0});
          cd.push_back(CopyDesc{S->vside(S->VD, k, ldR), ldR, S->vside(S->Vcat, k, ldP), ldP, S->m[k], rD[k], 0, nullptr,
                                rn * rho[k]});
          cd.push_back(CopyDesc{S->vside(S->VR, k, ldR), ldR, S->vside(S->Vcat, k, ldP) + rD[k], ldP, S->m[k], rR[k], 0,
                                nullptr, 2.0 * rn / o.c});
          p[k] = rD[k] + rR[k];
          Uo[k] = S->tall(S->UD, k, ldR);
          Vo[k] = S->vside(S->VD, k, ldR);
          rho[k] = rn;
        }
        LRFSI_TRY(copy_batched(cd, s));
        LRFSI_TRY(truncate_batch(S, live, p, o.tol, S->cap, Uo, Vo, rk, f2, s));
        for (int k : live) rD[k] = rk[k];
      }
    }
  }
  for (int k : act) st[k].rank = rS[k];
  return LRFSI_OK;
}

// ---------------------------------------------------------------------------
// ChebyshevT as a fixed launch sequence
// ---------------------------------------------------------------------------
// cheb_run above sizes every launch from ranks read back to the host (two
// round trips per truncation).  The fixed sequence below takes no host
// decision, so that one whole solve (cycles x iters steps of Algorithm 1 step
// 3, for all subsets of the handle) can be captured once into a CUDA graph and
// replayed with one launch:
// - widths are fixed per subset: the iterate S, the direction Delta and the
//   truncated residual have Rk = min(R_k, m_k) columns, zero beyond their
//   rank (the SVD writes zeros there); concatenations have 2 Rk columns, the
//   dense residual m_k.  Zero columns change nothing: the pivoted Cholesky
//   drops them and the products add zeros;
// - the eta test clears a per-subset device flag ("live") that gates every
//   later launch of the subset, and the third Cholesky-QR pass is gated by
//   the flag its first pass writes; the ranks stay on the device;
// - every descriptor lives at a fixed device address (the truncation
//   descriptors in S->cgt, uploaded before the first capture) or is passed by
//   value, and the split-K workspace of the GEMMs is bound to the handle.
// The result equals cheb_run's up to the summation order of the zero columns,
// i.e. exactly in exact arithmetic.
enum { CG_LIVE = 0, CG_RANK = 1, CG_STEPS = 2, CG_BROKE = 3, CG_ACT = 4, CG_NINT = 5 };
enum { CG_NB = 0, CG_REL = 1, CG_NDBL = 2 };
enum { TS_S = 0, TS_RES = 1, TS_D = 2, TS_NSITES = 3 };

static std::atomic<int> g_graph_mode{2};  // 0 host-sized launches, 1 fixed sequence, 2 fixed sequence in a graph

// ||B_k||_F from the column norms, the live flags of the solve and reset
// counters (one thread per subset).
__global__ void k_cheb_init(const double* __restrict__ norm2, const int* __restrict__ offm, int K, int* __restrict__ st,
                            double* __restrict__ dd) {
  const int k = threadIdx.x;
  if (k >= K) return;
  const int o = offm[2 * k], m = offm[2 * k + 1];
  double t = 0;
  for (int i = 0; i < m; ++i) t += norm2[o + i];
  const double nb = sqrt(t);
  st[CG_LIVE * K + k] = (st[CG_ACT * K + k] && nb > 0) ? 1 : 0;
  st[CG_RANK * K + k] = 0;
  st[CG_STEPS * K + k] = 0;
  st[CG_BROKE * K + k] = 0;
  dd[CG_NB * K + k] = nb;
  dd[CG_REL * K + k] = 1.0;
}

// After a residual truncation: relative linear residual and the eta test.
__global__ void k_cheb_eta(const double* __restrict__ frob2, int K, double eta, int* __restrict__ st,
                           double* __restrict__ dd) {
  const int k = threadIdx.x;
  if (k >= K || !st[CG_LIVE * K + k]) return;
  const double r = sqrt(frob2[k]), nb = dd[CG_NB * K + k];
  dd[CG_REL * K + k] = nb > 0 ? r / nb : 0.0;
  if (eta > 0 && r <= eta * nb) st[CG_LIVE * K + k] = 0;
}

static int fixed_rank(const lrfsi_subset_s* S, int k) { return std::min(S->cap[k], S->m[k]); }
static Gate live_gate(lrfsi_subset_s* S, int k) { return Gate{S->cgi.p + CG_LIVE * S->K + k, nullptr}; }

// Host copies of the truncation descriptors of the three sites of the
// sequence (S update, residual, direction update) and of their third passes.
static void fixed_descs(lrfsi_subset_s* S, const lrfsi_cheb_options& o, std::vector<TruncDesc>& out) {
  const int K = S->K, ldP = S->ldP, ldR = S->ldR;
  out.assign((size_t)2 * TS_NSITES * K, TruncDesc{});
  for (int site = 0; site < TS_NSITES; ++site)
    for (int k = 0; k < K; ++k) {
      const int Rk = fixed_rank(S, k);
      TruncDesc& d = out[(size_t)site * K + k];
      d.p = site == TS_RES ? S->m[k] : 2 * Rk;
      d.m = S->m[k];
      d.Vc = S->vside(S->Vcat, k, ldP);
      d.ldv = ldP;
      d.G = S->G.p + (size_t)k * ldP * ldP;
      d.G2 = S->G2.p + (size_t)k * ldP * ldP;
      d.T1 = S->T1.p + (size_t)k * ldP * ldP;
      d.T2 = S->T2.p + (size_t)k * ldP * ldP;
      double* Vout = site == TS_S ? S->vside(S->VS, k, ldR)
                                  : (site == TS_RES ? S->vside(S->VR, k, ldR) : S->vside(S->VD, k, ldR));
      d.Vout = Vout;
      d.ldvo = ldR;
      d.work = S->swork.p + S->swork_per * k;
      d.iwork = S->iwork.p + (size_t)2 * ldP * k;
      d.info = S->info.p + 5 * k;
      d.sv = S->sv.p + (size_t)ldP * k;
      d.frob2 = S->frob2.p + k;
      d.rank_cap = Rk;
      if (site == TS_RES && o.precision == 1) {  // FP32 residual: truncated at its noise level
        d.tol = std::max(o.tol, 1e-6);
        d.drop = 1e-12;
      } else {
        d.tol = o.tol;
        d.drop = 1e-14;
      }
      d.gate = live_gate(S, k);
      const TruncWork W(d.work, d.p, d.m);
      d.core = W.C;
      d.core_alt = W.Y;
      d.sel = d.info + 4;
      d.rank_out = site == TS_S ? S->cgi.p + CG_RANK * K + k : nullptr;
      d.count = site == TS_S ? S->cgi.p + CG_STEPS * K + k : nullptr;
      d.broke = S->cgi.p + CG_BROKE * K + k;
      TruncDesc& d3 = out[(size_t)(TS_NSITES + site) * K + k];
      d3 = d;
      d3.gate = Gate{d.gate.a, d.info + 4};
    }
}

// T of the concatenation in Xcat / Vcat for every subset, as a fixed sequence
// (the launches of truncate_once with widths p, gated per subset; see the
// header of dense.cu for the algorithm).  Outputs: the site's U buffer
// (Rk columns, zero beyond the rank) and V buffer (written by the SVD).
static int trunc_fixed(lrfsi_subset_s* S, int site, cudaStream_t s) {
  const int K = S->K, ldP = S->ldP, ldR = S->ldR;
  const long M = S->M;
  const TruncDesc* hd = S->cgt_host.data() + (size_t)site * K;
  TruncDesc* dd = S->cgt.p + (size_t)site * K;
  TruncDesc* dd3 = S->cgt.p + (size_t)(TS_NSITES + site) * K;
  std::vector<GramDesc> g1, g2, g3;
  std::vector<GemmDesc<double>> q1y, c2, q2, y3, t1, uo;
  for (int k = 0; k < K; ++k) {
    const TruncDesc& d = hd[k];
    const int p = d.p, m = d.m, w = d.rank_cap;
    const TruncWork W(d.work, p, m);
    const Gate live = d.gate, third{d.gate.a, d.info + 4};
    double* X = S->tall(S->Xcat, k, ldP);
    double* Q1 = S->tall(S->Q1, k, ldP);
    double* Q2 = S->tall(S->Q2, k, ldP);
    double* Uout = site == TS_S ? S->tall(S->US, k, ldR)
                                : (site == TS_RES ? S->tall(S->UR, k, ldR) : S->tall(S->UD, k, ldR));
    GramDesc g{X, ldP, p, X, ldP, p, d.G, p};
    g.gate = live;
    g1.push_back(g);
    GemmDesc<double> a{(int)M, p, p, X, ldP, 1, d.T1, p, 1, Q1, ldP, 1, 1.0, 0.0};
    a.gate = live;
    a.tc = 1;
    q1y.push_back(a);
    GemmDesc<double> b{p, m, p, W.Rk, p, 1, d.Vc, 1, d.ldv, W.Y, m, 1, 1.0, 0.0};
    b.gate = live;
    q1y.push_back(b);
    g = GramDesc{Q1, ldP, p, Q1, ldP, p, d.G2, p};
    g.gate = live;
    g2.push_back(g);
    GemmDesc<double> c{p, m, p, W.Rki, p, 1, W.Y, m, 1, W.C, m, 1, 1.0, 0.0};
    c.gate = live;
    c2.push_back(c);
    GemmDesc<double> e{(int)M, p, p, Q1, ldP, 1, d.T2, p, 1, Q2, ldP, 1, 1.0, 0.0};
    e.gate = third;
    e.tc = 1;
    q2.push_back(e);
    g = GramDesc{Q2, ldP, p, Q2, ldP, p, d.G2, p};
    g.gate = third;
    g3.push_back(g);
    GemmDesc<double> f{p, m, p, W.Rki, p, 1, W.C, m, 1, W.Y, m, 1, 1.0, 0.0};
    f.gate = third;
    y3.push_back(f);
    GemmDesc<double> t{p, w, p, d.T2, p, 1, W.Rk, p, 1, d.T1, p, 1, 1.0, 0.0};
    t.gate = live;
    t1.push_back(t);
    GemmDesc<double> u{(int)M, w, p, Q1, ldP, 1, d.T1, p, 1, Uout, ldR, 1, 1.0, 0.0};
    u.gate = live;
    u.tc = 1;
    u.A_alt = Q2;
    u.sel = d.info + 4;
    uo.push_back(u);
  }
  LRFSI_TRY(gram_batched(g1.data(), K, M, S->gramwork.p, S->gramwork.n, s));
  LRFSI_TRY(trunc_pass1(hd, K, s, dd, false));
  LRFSI_TRY(gemm_grouped<double>(q1y.data(), (int)q1y.size(), s));
  LRFSI_TRY(gram_batched(g2.data(), K, M, S->gramwork.p, S->gramwork.n, s));
  int pmaxf = 0;
  for (int k = 0; k < K; ++k) pmaxf = std::max(pmaxf, hd[k].p);
  LRFSI_TRY(trunc_qr(K, s, dd, 1, pmaxf));
  LRFSI_TRY(gemm_grouped<double>(c2.data(), K, s));
  LRFSI_TRY(gemm_grouped<double>(q2.data(), K, s));
  LRFSI_TRY(gram_batched(g3.data(), K, M, S->gramwork.p, S->gramwork.n, s));
  LRFSI_TRY(trunc_qr(K, s, dd3, 0, pmaxf));
  LRFSI_TRY(gemm_grouped<double>(y3.data(), K, s));
  LRFSI_TRY(trunc_svd(hd, K, s, dd, false));
  if (timing_enabled()) {  // algorithmic work of the small kernels of the live subsets (as truncate_once)
    std::vector<int> info((size_t)5 * K), live(K);
    LRFSI_CUDA(cudaMemcpyAsync(info.data(), S->info.p, sizeof(int) * 5 * K, cudaMemcpyDeviceToHost, s));
    LRFSI_CUDA(cudaMemcpyAsync(live.data(), S->cgi.p + CG_LIVE * K, sizeof(int) * K, cudaMemcpyDeviceToHost, s));
    LRFSI_CUDA(cudaStreamSynchronize(s));
    double fl = 0, fj = 0;
    for (int k = 0; k < K; ++k) {
      if (!live[k]) continue;
      const double P = hd[k].p, kk = info[5 * k], mm = hd[k].m;
      const double n = std::min(kk, mm), L = std::max(kk, mm), sw = std::max(info[5 * k + 3], 1);
      fl += 2.0 * P * P * P / 3.0 + (info[5 * k + 4] ? 2.0 : 1.0) * (2.0 * kk * kk * kk / 3.0) + kk * kk * kk / 3.0;
      fj += 3.0 * L * n * n - n * n * n + sw * n * (n - 1) / 2.0 * (6.0 * n + 8.0 * n) +
            4.0 * L * n * info[5 * k + 1];
    }
    account(KC_TRUNC, fl, 0);
    account(KC_SVD, fj, 0);
  }
  LRFSI_TRY(gemm_grouped<double>(t1.data(), K, s));
  LRFSI_TRY(gemm_grouped<double>(uo.data(), K, s));
  return LRFSI_OK;
}

// Res = T(B - F(S)) for every live subset as a fixed sequence (lr_residual's
// launches with S at Rk columns), then the eta test.
static int residual_fixed(lrfsi_subset_s* S, const lrfsi_cheb_options& o, cudaStream_t s) {
  const int K = S->K, ldP = S->ldP, ldR = S->ldR;
  const long M = S->M;
  const long nnz = (long)S->mesh->h.colidx.size();
  std::vector<CopyDesc> cd, cd2;
  std::vector<SpmmDesc<double>> sd;
  std::vector<GemmDesc<double>> gm;
  std::vector<ConvDesc> c1, c2;
  std::vector<SpmmDesc<float>> sdf;
  std::vector<GemmDesc<float>> gmf;
  for (int k = 0; k < K; ++k) {
    const Gate live = live_gate(S, k);
    const int m = S->m[k], r = fixed_rank(S, k);
    double* X = S->tall(S->Xcat, k, ldP);
    double* Vc = S->vside(S->Vcat, k, ldP);
    const double* mu = S->mu.p + S->off[k];
    const double* nu = S->nu.p + S->off[k];
    const double* VS = S->vside(S->VS, k, ldR);
    cd.push_back(CopyDesc{S->tall(S->UB, k, ldR), ldR, X, ldP, M, m, 0, nullptr, 1.0, live});
    cd.push_back(CopyDesc{VS, ldR, Vc, ldP, m, r, 0, nullptr, 1.0, live});
    cd.push_back(CopyDesc{VS, ldR, Vc + r, ldP, m, r, 0, mu, 1.0, live});
    cd.push_back(CopyDesc{VS, ldR, Vc + 2 * r, ldP, m, r, 0, nu, 1.0, live});
    cd2.push_back(CopyDesc{nullptr, 0, Vc, ldP, m, m, 2, nullptr, 1.0, live});
    const int kc = (S->four ? 5 : 3) * r;
    if (S->four) {  // + Jlam' S D_lam + Jrho' S D_rho (Sec. 4.4)
      cd.push_back(CopyDesc{VS, ldR, Vc + 3 * r, ldP, m, r, 0, S->lam.p + S->off[k], 1.0, live});
      cd.push_back(CopyDesc{VS, ldR, Vc + 4 * r, ldP, m, r, 0, S->rho.p + S->off[k], 1.0, live});
    }
    if (o.precision == 0) {
      SpmmDesc<double> d;
      d.J3 = S->J3.p + (size_t)k * 3 * nnz;
      d.U = S->tall(S->US, k, ldR);
      d.ldu = ldR;
      d.r = r;
      d.Y = S->tall(S->Q1, k, ldP);
      d.ldy = ldP;
      d.o[0] = 0; d.o[1] = r; d.o[2] = 2 * r;
      d.sc[0] = d.sc[1] = d.sc[2] = 1.0;
      d.a1 = d.a2 = 0.0;
      d.gate = live;
      sd.push_back(d);
      if (S->four) {
        SpmmDesc<double> d2 = d;
        d2.J3 = S->J3x.p + (size_t)k * 3 * nnz;
        d2.o[0] = 3 * r; d2.o[1] = 4 * r; d2.o[2] = 5 * r;
        d2.sc[2] = 0.0;
        sd.push_back(d2);
      }
      GemmDesc<double> g{(int)M, m, kc, S->tall(S->Q1, k, ldP), ldP, 1, Vc, 1, ldP, X, ldP, 1, -1.0, 1.0};
      g.gate = live;
      g.tc = 1;
      gm.push_back(g);
    } else {  // B - F(S) with an FP32 SpMM and GEMM, widened to FP64 for the truncation
      float* Uf = S->USf.p + (size_t)k * M * ldR;
      float* Yf = S->Yf.p + (size_t)k * M * ldP;
      float* Xf = S->Xf.p + (size_t)k * M * ldP;
      float* Vf = S->Vf.p + (size_t)S->off[k] * ldP;
      c1.push_back(ConvDesc{S->tall(S->US, k, ldR), ldR, Uf, ldR, M, r, nullptr, 1.0, live});
      c1.push_back(ConvDesc{X, ldP, Xf, ldP, M, m, nullptr, 1.0, live});
      c1.push_back(ConvDesc{Vc, ldP, Vf, ldP, m, kc, nullptr, 1.0, live});
      SpmmDesc<float> d;
      d.J3 = S->J3f.p + (size_t)k * 3 * nnz;
      d.U = Uf; d.ldu = ldR; d.r = r; d.Y = Yf; d.ldy = ldP;
      d.o[0] = 0; d.o[1] = r; d.o[2] = 2 * r;
      d.sc[0] = d.sc[1] = d.sc[2] = 1.0f;
      d.a1 = d.a2 = 0.0f;
      d.gate = live;
      sdf.push_back(d);
      if (S->four) {
        SpmmDesc<float> d2 = d;
        d2.J3 = S->J3xf.p + (size_t)k * 3 * nnz;
        d2.o[0] = 3 * r; d2.o[1] = 4 * r; d2.o[2] = 5 * r;
        d2.sc[2] = 0.0f;
        sdf.push_back(d2);
      }
      GemmDesc<float> g{(int)M, m, kc, Yf, ldP, 1, Vf, 1, ldP, Xf, ldP, 1, -1.0f, 1.0f};
      g.gate = live;
      gmf.push_back(g);
      c2.push_back(ConvDesc{Xf, ldP, X, ldP, M, m, nullptr, 1.0, live});
    }
  }
  LRFSI_TRY(copy_batched(cd, s));
  if (o.precision == 0) {
    LRFSI_TRY(spmm_batched<double>(S->mesh, sd.data(), (int)sd.size(), s));
    LRFSI_TRY(gemm_grouped<double>(gm.data(), (int)gm.size(), s));
  } else {
    LRFSI_TRY((convert_batched<double, float>(c1, s)));
    LRFSI_TRY(spmm_batched<float>(S->mesh, sdf.data(), (int)sdf.size(), s));
    LRFSI_TRY(gemm_grouped<float>(gmf.data(), (int)gmf.size(), s));
    LRFSI_TRY((convert_batched<float, double>(c2, s)));
  }
  LRFSI_TRY(copy_batched(cd2, s));
  LRFSI_TRY(trunc_fixed(S, TS_RES, s));
  k_cheb_eta<<<1, 32, 0, s>>>(S->frob2.p, K, o.eta, S->cgi.p, S->cgd.p);
  return check_launch("k_cheb_eta");
}

// UZ = P^{-1} UR (Rk columns) for every live subset.
static int precond_fixed(lrfsi_subset_s* S, cudaStream_t s) {
  const int K = S->K, ldR = S->ldR;
  const long M = S->M;
  std::vector<CopyDesc> cd;
  std::vector<double*> X(K), Y(K);
  std::vector<int> r(K);
  std::vector<Gate> gates(K);
  for (int k = 0; k < K; ++k) {
    r[k] = fixed_rank(S, k);
    gates[k] = live_gate(S, k);
    X[k] = S->tall(S->Ytmp, k, ldR);
    Y[k] = S->tall(S->UZ, k, ldR);
    cd.push_back(CopyDesc{S->tall(S->UR, k, ldR), ldR, X[k], ldR, M, r[k], 0, nullptr, 1.0, gates[k]});
  }
  LRFSI_TRY(copy_batched(cd, s));
  return S->lu.solve(X.data(), Y.data(), r.data(), ldR, K, s, gates.data());
}

// [A | B] -> Xcat and [a VA | b VB] -> Vcat (Rk columns each) for every subset.
static int concat_fixed(lrfsi_subset_s* S, DevBuf<double>& UA, DevBuf<double>& VA, double a, DevBuf<double>& UB_,
                        DevBuf<double>& VB_, double b, cudaStream_t s) {
  const int K = S->K, ldP = S->ldP, ldR = S->ldR;
  const long M = S->M;
  std::vector<CopyDesc> cd;
  for (int k = 0; k < K; ++k) {
    const Gate live = live_gate(S, k);
    const int r = fixed_rank(S, k), m = S->m[k];
    double* X = S->tall(S->Xcat, k, ldP);
    double* Vc = S->vside(S->Vcat, k, ldP);
    cd.push_back(CopyDesc{S->tall(UA, k, ldR), ldR, X, ldP, M, r, 0, nullptr, 1.0, live});
    cd.push_back(CopyDesc{S->tall(UB_, k, ldR), ldR, X + r, ldP, M, r, 0, nullptr, 1.0, live});
    cd.push_back(CopyDesc{S->vside(VA, k, ldR), ldR, Vc, ldP, m, r, 0, nullptr, a, live});
    cd.push_back(CopyDesc{S->vside(VB_, k, ldR), ldR, Vc + r, ldP, m, r, 0, nullptr, b, live});
  }
  return copy_batched(cd, s);
}

// The phases of the fixed sequence (options o) for the subsets flagged in
// cgi[CG_ACT]; B dense in UB, result in US/VS (Rk columns, zero beyond
// cgi[CG_RANK]).  A solve runs
//   INIT, then per cycle: RES, Z0, and for j = 0 .. iters-1: S, then (j < iters - 1) RES, D_j,
// and ends early once no subset is live after a RES (the one host read of a step).
enum { PH_INIT = 0, PH_RES = 1, PH_Z0 = 2, PH_S = 3, PH_D0 = 4 };

static int cheb_phase(lrfsi_subset_s* S, const lrfsi_cheb_options& o, int ph, cudaStream_t s) {
  const int K = S->K, ldR = S->ldR;
  const long M = S->M;
  const double sigma = o.d / o.c;
  switch (ph) {
    case PH_INIT: {
      LRFSI_CUDA(cudaMemsetAsync(S->US.p, 0, sizeof(double) * (size_t)K * M * ldR, s));
      LRFSI_CUDA(cudaMemsetAsync(S->VS.p, 0, sizeof(double) * (size_t)S->mtot * ldR, s));
      for (int k = 0; k < K; ++k)
        LRFSI_TRY(launch_colnorm2(S->tall(S->UB, k, ldR), M, S->m[k], ldR, S->rc.norm2.p + S->off[k], S->rc.work.p,
                                  S->rc.work.n, s));
      k_cheb_init<<<1, 32, 0, s>>>(S->rc.norm2.p, S->offm.p, K, S->cgi.p, S->cgd.p);
      return check_launch("k_cheb_init");
    }
    case PH_RES:
      return residual_fixed(S, o, s);
    case PH_Z0: {  // Z = P^{-1} U_R, Delta = Z / d
      LRFSI_TRY(precond_fixed(S, s));
      std::vector<CopyDesc> cd;
      for (int k = 0; k < K; ++k) {
        const Gate live = live_gate(S, k);
        const int r = fixed_rank(S, k);
        cd.push_back(CopyDesc{S->tall(S->UZ, k, ldR), ldR, S->tall(S->UD, k, ldR), ldR, M, r, 0, nullptr, 1.0, live});
        cd.push_back(CopyDesc{S->vside(S->VR, k, ldR), ldR, S->vside(S->VD, k, ldR), ldR, S->m[k], r, 0, nullptr,
                              1.0 / o.d, live});
      }
      return copy_batched(cd, s);
    }
    case PH_S:  // S <- T(S + Delta)
      LRFSI_TRY(concat_fixed(S, S->US, S->VS, 1.0, S->UD, S->VD, 1.0, s));
      return trunc_fixed(S, TS_S, s);
    default: {  // D_j: Z = P^{-1} U_R, Delta <- T(rho' rho Delta + (2 rho' / c) Z) with the rho of step j
      const int j = ph - PH_D0;
      double rho = 1.0 / sigma;
      for (int i = 0; i < j; ++i) rho = 1.0 / (2.0 * sigma - rho);
      const double rn = 1.0 / (2.0 * sigma - rho);
      LRFSI_TRY(precond_fixed(S, s));
      LRFSI_TRY(concat_fixed(S, S->UD, S->VD, rn * rho, S->UZ, S->VR, 2.0 * rn / o.c, s));
      return trunc_fixed(S, TS_D, s);
    }
  }
}

// Prepared state of the fixed sequence for these options and buffers: the key
// holds everything the descriptors and the captured launches depend on.
static std::vector<double> fixed_key(const lrfsi_subset_s* S, const lrfsi_cheb_options& o) {
  return {o.c, o.d, (double)o.iters, (double)o.cycles, o.tol, o.eta, (double)o.precision, (double)S->ldP,
          (double)(uintptr_t)S->Xcat.p, (double)(uintptr_t)S->swork.p};
}

static int fixed_prepare(lrfsi_subset_s* S, const lrfsi_cheb_options& o, cudaStream_t s) {
  const int K = S->K;
  if (!S->cgi.p) {
    LRFSI_TRY(S->cgi.alloc((size_t)CG_NINT * K));
    LRFSI_TRY(S->cgd.alloc((size_t)CG_NDBL * K));
    std::vector<int> om(2 * K);
    for (int k = 0; k < K; ++k) { om[2 * k] = S->off[k]; om[2 * k + 1] = S->m[k]; }
    LRFSI_TRY(S->offm.upload(om, s));
  }
  const std::vector<double> key = fixed_key(S, o);
  if (key != S->cg_key) {
    S->drop_graph();
    fixed_descs(S, o, S->cgt_host);
    LRFSI_TRY(S->cgt.upload(S->cgt_host, s));
    S->cg_key = key;
  }
  return LRFSI_OK;
}

static std::atomic<long long> g_graph_replays{0}, g_graph_captures{0}, g_graph_fallbacks{0};

// ChebyshevT for the subsets in act through the fixed sequence.  Graph mode 2:
// the first solve with these options runs the phases directly (which also
// sizes the split-K workspace), then captures every phase once on the handle's
// stream; later solves replay the phase graphs, one graph launch per phase and
// one 4-byte-per-subset read of the live flags after each residual (the solve
// ends when no subset is live).  Mode 1, or kernel timing on: the phases are
// launched directly.  A subset whose truncation broke down is solved again by
// cheb_run.
static int cheb_fixed(lrfsi_subset_s* S, const lrfsi_cheb_options& o, const std::vector<int>& act,
                      std::vector<int>& rS, std::vector<lrfsi_cheb_stats>& st, cudaStream_t s) {
  const int K = S->K;
  const int nph = PH_D0 + std::max(o.iters - 1, 0);
  LRFSI_TRY(fixed_prepare(S, o, s));
  if (!S->live_host) LRFSI_CUDA(cudaMallocHost((void**)&S->live_host, sizeof(int) * CG_NINT * K));
  {
    std::vector<int> a(K, 0);
    for (int k : act) a[k] = 1;
    LRFSI_CUDA(cudaMemcpyAsync(S->cgi.p + CG_ACT * K, a.data(), sizeof(int) * K, cudaMemcpyHostToDevice, s));
  }
  const bool use_graph = g_graph_mode.load() == 2 && !g_timing;
  const bool replay = use_graph && (int)S->cg_exec.size() == nph;
  if (!replay) gemm_ws_peak_reset();
  auto run = [&](int ph) -> int {
    if (replay) {
      LRFSI_CUDA(cudaGraphLaunch(S->cg_exec[ph], s));
      count_launch(S->cg_nodes[ph]);  // one host launch, cg_nodes kernels
      g_graph_replays += 1;
      return LRFSI_OK;
    }
    return cheb_phase(S, o, ph, s);
  };
  auto any_live = [&](bool& any) -> int {
    LRFSI_CUDA(cudaMemcpyAsync(S->live_host, S->cgi.p + CG_LIVE * K, sizeof(int) * K, cudaMemcpyDeviceToHost, s));
    LRFSI_CUDA(cudaStreamSynchronize(s));
    any = false;
    for (int k = 0; k < K; ++k) any = any || S->live_host[k];
    return LRFSI_OK;
  };
  LRFSI_TRY(run(PH_INIT));
  bool any = true, done = false;
  for (int cyc = 0; cyc < o.cycles && !done; ++cyc) {
    LRFSI_TRY(run(PH_RES));
    LRFSI_TRY(any_live(any));
    if (!any) break;
    LRFSI_TRY(run(PH_Z0));
    for (int j = 0; j < o.iters; ++j) {
      LRFSI_TRY(run(PH_S));
      if (j == o.iters - 1) break;
      LRFSI_TRY(run(PH_RES));
      LRFSI_TRY(any_live(any));
      if (!any) { done = true; break; }
      LRFSI_TRY(run(PH_D0 + j));
    }
  }
  if (use_graph && !replay) {  // capture every phase for the next solves
    const size_t need = std::max<size_t>(gemm_ws_peak(), 256);
    if (S->cgws.n < need) LRFSI_TRY(S->cgws.alloc(need));
    if (!S->cap_stream) LRFSI_CUDA(cudaStreamCreateWithFlags(&S->cap_stream, cudaStreamNonBlocking));
    std::vector<cudaGraphExec_t> execs;
    std::vector<uint64_t> nodes;
    bool ok = true;
    gemm_ws_bind(S->cgws.p, S->cgws.n);
    for (int ph = 0; ph < nph && ok; ++ph) {
      const uint64_t before = g_launches.load(), hbefore = g_host_launches.load();
      cudaGraph_t graph = nullptr;
      int st_cap = LRFSI_OK;
      cudaError_t e = cudaStreamBeginCapture(S->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        st_cap = cheb_phase(S, o, ph, S->cap_stream);
        e = cudaStreamEndCapture(S->cap_stream, &graph);
      }
      const uint64_t n = g_launches.load() - before;
      g_launches -= n;  // captured, not launched
      g_host_launches -= g_host_launches.load() - hbefore;
      cudaGraphExec_t exec = nullptr;
      if (e == cudaSuccess && st_cap == LRFSI_OK && graph) e = cudaGraphInstantiate(&exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess || st_cap != LRFSI_OK || !exec) {
        ok = false;
        if (exec) cudaGraphExecDestroy(exec);
      } else {
        execs.push_back(exec);
        nodes.push_back(n);
      }
    }
    gemm_ws_bind(nullptr, 0);
    if (ok) {
      S->cg_exec = execs;
      S->cg_nodes = nodes;
      g_graph_captures += 1;
    } else {  // capture failed: keep launching the phases directly
      for (cudaGraphExec_t e : execs) cudaGraphExecDestroy(e);
      cudaGetLastError();
      g_graph_fallbacks += 1;
      g_graph_mode = 1;
    }
  }
  std::vector<int> hi((size_t)CG_NINT * K);
  std::vector<double> hd((size_t)CG_NDBL * K);
  LRFSI_CUDA(cudaMemcpyAsync(hi.data(), S->cgi.p, sizeof(int) * hi.size(), cudaMemcpyDeviceToHost, s));
  LRFSI_CUDA(cudaMemcpyAsync(hd.data(), S->cgd.p, sizeof(double) * hd.size(), cudaMemcpyDeviceToHost, s));
  LRFSI_CUDA(cudaStreamSynchronize(s));
  rS.assign(K, 0);
  st.assign(K, lrfsi_cheb_stats{0, 0, 1.0, 0});
  std::vector<int> redo;
  for (int k : act) {
    rS[k] = hi[CG_RANK * K + k];
    st[k].steps = hi[CG_STEPS * K + k];
    st[k].rank = rS[k];
    st[k].rel_lin_res = hd[CG_REL * K + k];
    st[k].max_concat_rank = 3 * fixed_rank(S, k);
    if (hi[CG_BROKE * K + k]) redo.push_back(k);
  }
  if (!redo.empty()) {  // a Cholesky-QR breakdown: the host-sized path with its retries
    g_tr_breakdown += (long long)redo.size();
    std::vector<int> r2;
    std::vector<lrfsi_cheb_stats> st2;
    LRFSI_TRY(cheb_run(S, o, redo, r2, st2, s));
    for (int k : redo) {
      rS[k] = r2[k];
      st[k] = st2[k];
    }
  }
  return LRFSI_OK;
}

// Krylov basis storage of GMREST for `iters` steps per cycle: the tall
// factors of V_j and Z_j = P^{-1} V_j (K x M x ldR each), the parameter-side
// factors of V_j (sum m_k x ldR), the two Gram blocks of the inner products
// (K x iters blocks of ldR^2) and their sizes and results (K x iters).
static int gmres_alloc(lrfsi_subset_s* S, int iters) {
  if (S->gm_iters >= iters) return LRFSI_OK;
  S->gm_iters = 0;  // nothing usable until every buffer below exists
  const size_t tall = (size_t)S->K * S->M * S->ldR, side = (size_t)S->mtot * S->ldR;
  const size_t nblk = (size_t)S->K * iters;
  LRFSI_TRY(S->GU.alloc(tall * iters));
  LRFSI_TRY(S->GZ.alloc(tall * iters));
  LRFSI_TRY(S->GV.alloc(side * iters));
  LRFSI_TRY(S->Gu.alloc(nblk * S->ldR * S->ldR));
  LRFSI_TRY(S->Gv.alloc(nblk * S->ldR * S->ldR));
  LRFSI_TRY(S->Gh.alloc(nblk));
  LRFSI_TRY(S->Gn.alloc(nblk));
  S->gm_iters = iters;
  return LRFSI_OK;
}

// h[q] = sum_e A_q[e] B_q[e] over the first n[q] entries of block q (blocks of
// `blk` doubles): the Frobenius inner product <X, Y> = sum((U_X^T U_Y) .*
// (V_X^T V_Y)) from its two Gram blocks.  One CTA per block, fixed-order
// reduction.
constexpr int kDotThreads = 256;
__global__ void __launch_bounds__(kDotThreads) k_block_dot(const double* __restrict__ A, const double* __restrict__ B,
                                                           const int* __restrict__ n, size_t blk,
                                                           double* __restrict__ h) {
  __shared__ double red[kDotThreads / 32];
  const int q = blockIdx.x;
  const int nq = n[q];
  const double* a = A + (size_t)q * blk;
  const double* b = B + (size_t)q * blk;
  double t = 0.0;
  for (int e = threadIdx.x; e < nq; e += kDotThreads) t = fma(a[e], b[e], t);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0;
    for (int w = 0; w < kDotThreads / 32; ++w) u += red[w];
    h[q] = u;
  }
}

// Widens the concatenation buffers and the truncation scratch to `width`
// columns (a GMREST sum has up to iters + 1 terms of rank <= R_k and is
// truncated at once).  The widened buffers are scratch only: no state lives in
// them between operations.
static int widen_concat(lrfsi_subset_s* S, int width) {
  if (width <= S->ldP) return LRFSI_OK;
  const int K = S->K;
  const long M = S->M;
  const size_t w = (size_t)width;
  // allocate everything first: on failure the handle keeps its old buffers
  DevBuf<double> Xc, Q1, Q2, Vc, G, G2, T1, T2, sw, sv, gw;
  DevBuf<int> iw;
  DevBuf<float> Yf, Xf, Vf;
  const size_t swork_per = trunc_small_work(width, S->mmax);
  for (DevBuf<double>* b : {&Xc, &Q1, &Q2}) LRFSI_TRY(b->alloc((size_t)K * M * w));
  LRFSI_TRY(Vc.alloc((size_t)S->mtot * w));
  for (DevBuf<double>* b : {&G, &G2, &T1, &T2}) LRFSI_TRY(b->alloc((size_t)K * w * w));
  LRFSI_TRY(sw.alloc(swork_per * K));
  LRFSI_TRY(sv.alloc((size_t)K * w));
  LRFSI_TRY(iw.alloc((size_t)2 * w * K));
  LRFSI_TRY(gw.alloc(gram_work_len(K, M, width, width)));
  LRFSI_TRY(Yf.alloc((size_t)K * M * w));
  LRFSI_TRY(Xf.alloc((size_t)K * M * w));
  LRFSI_TRY(Vf.alloc((size_t)S->mtot * w));
  // the old buffers may still be read by queued work: swap, and let the
  // destructors free them (cudaFree waits for the device)
  S->Xcat.swap(Xc); S->Q1.swap(Q1); S->Q2.swap(Q2); S->Vcat.swap(Vc);
  S->G.swap(G); S->G2.swap(G2); S->T1.swap(T1); S->T2.swap(T2);
  S->swork.swap(sw); S->sv.swap(sv); S->gramwork.swap(gw); S->iwork.swap(iw);
  S->Yf.swap(Yf); S->Xf.swap(Xf); S->Vf.swap(Vf);
  S->swork_per = swork_per;
  S->ldP = width;
  return LRFSI_OK;
}

// T(sum of terms) for the subsets in L, one truncation per subset: per subset
// a list of terms (tall factor, ld ldR; parameter-side factor, ld ldR; rank;
// scale of the parameter side) concatenated in Xcat/Vcat; the result goes to
// Uo/Vo (ld ldR; may be the first term's buffers).
struct LrTerm {
  const double* U;
  const double* V;
  int r;
  double a;
};
static int truncate_sum(lrfsi_subset_s* S, const std::vector<int>& L, const std::vector<std::vector<LrTerm>>& terms,
                        double tol, const std::vector<double*>& Uo, const std::vector<double*>& Vo,
                        std::vector<int>& rank, std::vector<double>* kept2, cudaStream_t s) {
  const int K = S->K, ldP = S->ldP, ldR = S->ldR;
  const long M = S->M;
  std::vector<int> p(K, 0);
  std::vector<CopyDesc> cd;
  for (int k : L) {
    int c = 0;
    for (const LrTerm& t : terms[k]) {
      if (c + t.r > ldP) return fail(LRFSI_EINVAL, "truncate_sum: concatenation wider than its buffer");
      cd.push_back(CopyDesc{t.U, ldR, S->tall(S->Xcat, k, ldP) + c, ldP, M, t.r, 0, nullptr, 1.0});
      cd.push_back(CopyDesc{t.V, ldR, S->vside(S->Vcat, k, ldP) + c, ldP, S->m[k], t.r, 0, nullptr, t.a});
      c += t.r;
    }
    p[k] = c;
  }
  LRFSI_TRY(copy_batched(cd, s));
  std::vector<double> f2;
  return truncate_batch(S, L, p, tol, S->cap, Uo, Vo, rank, f2, s, 1e-14, kept2);
}

// GMREST on factors for the subsets in `act`: restarted GMRES with right
// preconditioning by P_k, Frobenius inner products (<X, Y> from the Gram
// blocks of the factors), classical Gram-Schmidt, and the truncation applied
// to the starting residual, to F(Z_j), to the orthogonalised vector and to
// the updated iterate (each sum truncated at once: the concatenation buffers
// are widened to (iters + 1) R_max columns).  B given densely in UB; results
// in US/VS (ranks rS).
static int gmres_run(lrfsi_subset_s* S, const lrfsi_cheb_options& o, std::vector<int> act, std::vector<int>& rS,
                     std::vector<lrfsi_cheb_stats>& st, cudaStream_t s) {
  const int K = S->K, ldR = S->ldR, nit = o.iters;
  const long M = S->M;
  const long nnz = (long)S->mesh->h.colidx.size();
  rS.assign(K, 0);
  st.assign(K, lrfsi_cheb_stats{0, 0, 1.0, 0});
  if (S->gm_iters < nit || S->ldP < (nit + 1) * S->Rmax)
    return fail(LRFSI_EINVAL, "GMREST: workspace not prepared for this iteration count");
  const int ldP = S->ldP;
  const size_t tall = (size_t)K * M * ldR, side = (size_t)S->mtot * ldR, gblk = (size_t)ldR * ldR;
  auto GU = [&](int j, int k) { return S->GU.p + tall * j + (size_t)k * M * ldR; };
  auto GZ = [&](int j, int k) { return S->GZ.p + tall * j + (size_t)k * M * ldR; };
  auto GV = [&](int j, int k) { return S->GV.p + side * j + (size_t)S->off[k] * ldR; };
  std::vector<double> nB;
  LRFSI_TRY(rhs_norms(S, act, nB, s));
  std::vector<int> live;
  for (int k : act)
    if (nB[k] > 0) live.push_back(k);
  std::vector<int> rR(K, 0), rW(K, 0), rk;
  std::vector<double> f2;
  std::vector<double*> Uo(K), Vo(K), Xb(K), Yb(K);
  for (int k = 0; k < K; ++k) {
    Uo[k] = S->tall(S->UD, k, ldR);
    Vo[k] = S->vside(S->VD, k, ldR);
  }
  std::vector<int> hn((size_t)K * nit);    // Gram block sizes of the inner products
  std::vector<double> hh((size_t)K * nit);  // the inner products
  for (int cyc = 0; cyc < o.cycles && !live.empty(); ++cyc) {
    std::vector<double> nres, beta;
    LRFSI_TRY(lr_residual(S, o, live, rS, nB, rR, nres, st, s, &beta));
    std::vector<int> arn;
    for (int k : live) {
      if (o.eta > 0 && nres[k] <= o.eta * nB[k]) continue;
      beta[k] = std::sqrt(beta[k]);
      if (rR[k] > 0 && beta[k] > 0) arn.push_back(k);
    }
    live = arn;
    if (arn.empty()) break;
    // V_0 = T(Res) / beta
    std::vector<std::vector<int>> rb(K, std::vector<int>(nit, 0));
    {
      std::vector<CopyDesc> cd;
      for (int k : arn) {
        cd.push_back(CopyDesc{S->tall(S->UR, k, ldR), ldR, GU(0, k), ldR, M, rR[k], 0, nullptr, 1.0});
        cd.push_back(CopyDesc{S->vside(S->VR, k, ldR), ldR, GV(0, k), ldR, S->m[k], rR[k], 0, nullptr, 1.0 / beta[k]});
        rb[k][0] = rR[k];
      }
      LRFSI_TRY(copy_batched(cd, s));
    }
    // Hessenberg columns reduced by Givens rotations: Rh (upper triangle), g
    std::vector<std::vector<double>> Rh(K, std::vector<double>((size_t)(nit + 1) * nit, 0.0));
    std::vector<std::vector<double>> g(K, std::vector<double>(nit + 1, 0.0)), cs(K, std::vector<double>(nit, 1.0)),
        sn(K, std::vector<double>(nit, 0.0));
    std::vector<int> nstep(K, 0);
    for (int k : arn) g[k][0] = beta[k];
    for (int j = 0; j < nit && !arn.empty(); ++j) {
      // Z_j = P^{-1} V_j (tall factor)
      std::vector<int> rj(K, 0);
      for (int k : arn) {
        Xb[k] = GU(j, k);
        Yb[k] = GZ(j, k);
        rj[k] = rb[k][j];
      }
      LRFSI_TRY(lr_precond(S, arn, Xb, Yb, rj, s));
      // W = T(F(Z_j)) = T([J0 Z | Jmu' Z | Jnu' Z] [V | D_mu V | D_nu V]^T)
      {
        std::vector<SpmmDesc<double>> sd;
        std::vector<CopyDesc> cd;
        std::vector<int> p(K, 0);
        for (int k : arn) {
          const int r = rj[k];
          SpmmDesc<double> d;
          d.J3 = S->J3.p + (size_t)k * 3 * nnz;
          d.U = GZ(j, k);
          d.ldu = ldR;
          d.r = r;
          d.Y = S->tall(S->Xcat, k, ldP);
          d.ldy = ldP;
          d.o[0] = 0; d.o[1] = r; d.o[2] = 2 * r;
          d.sc[0] = d.sc[1] = d.sc[2] = 1.0;
          d.a1 = d.a2 = 0.0;
          sd.push_back(d);
          double* Vc = S->vside(S->Vcat, k, ldP);
          cd.push_back(CopyDesc{GV(j, k), ldR, Vc, ldP, S->m[k], r, 0, nullptr, 1.0});
          cd.push_back(CopyDesc{GV(j, k), ldR, Vc + r, ldP, S->m[k], r, 0, S->mu.p + S->off[k], 1.0});
          cd.push_back(CopyDesc{GV(j, k), ldR, Vc + 2 * r, ldP, S->m[k], r, 0, S->nu.p + S->off[k], 1.0});
          p[k] = 3 * r;
          st[k].max_concat_rank = std::max(st[k].max_concat_rank, 3 * r);
        }
        LRFSI_TRY(spmm_batched<double>(S->mesh, sd.data(), (int)sd.size(), s));
        LRFSI_TRY(copy_batched(cd, s));
        LRFSI_TRY(truncate_batch(S, arn, p, o.tol, S->cap, Uo, Vo, rk, f2, s));
        for (int k : arn) rW[k] = rk[k];
      }
      // h_ij = <W, V_i>_F = sum((U_W^T U_i) .* (V_W^T V_i)), i <= j
      std::vector<std::vector<double>> h(K, std::vector<double>(j + 1, 0.0));
      {
        std::vector<GramDesc> gd;
        std::vector<GemmDesc<double>> gv;
        for (int k : arn) {
          if (rW[k] == 0) continue;
          for (int i = 0; i <= j; ++i) {
            double* Gu = S->Gu.p + ((size_t)k * nit + i) * gblk;
            double* Gv = S->Gv.p + ((size_t)k * nit + i) * gblk;
            gd.push_back(GramDesc{S->tall(S->UD, k, ldR), ldR, rW[k], GU(i, k), ldR, rb[k][i], Gu, rb[k][i]});
            gv.push_back(GemmDesc<double>{rW[k], rb[k][i], S->m[k], S->vside(S->VD, k, ldR), 1, ldR, GV(i, k), ldR, 1,
                                          Gv, rb[k][i], 1, 1.0, 0.0});
          }
        }
        if (!gd.empty()) {
          std::fill(hn.begin(), hn.end(), 0);
          for (int k : arn)
            if (rW[k] > 0)
              for (int i = 0; i <= j; ++i) hn[(size_t)k * nit + i] = rW[k] * rb[k][i];
          LRFSI_CUDA(cudaMemcpyAsync(S->Gn.p, hn.data(), sizeof(int) * hn.size(), cudaMemcpyHostToDevice, s));
          LRFSI_TRY(gram_batched(gd.data(), (int)gd.size(), M, S->gramwork.p, S->gramwork.n, s));
          LRFSI_TRY(gemm_grouped<double>(gv.data(), (int)gv.size(), s));
          k_block_dot<<<(int)hn.size(), kDotThreads, 0, s>>>(S->Gu.p, S->Gv.p, S->Gn.p, gblk, S->Gh.p);
          LRFSI_TRY(check_launch("k_block_dot"));
          LRFSI_CUDA(cudaMemcpyAsync(hh.data(), S->Gh.p, sizeof(double) * hh.size(), cudaMemcpyDeviceToHost, s));
          LRFSI_CUDA(cudaStreamSynchronize(s));
        }
        for (int k : arn)
          if (rW[k] > 0)
            for (int i = 0; i <= j; ++i) h[k][i] = hh[(size_t)k * nit + i];
      }
      // W <- T(W - sum_i h_ij V_i); h_{j+1,j} = ||W||_F
      std::vector<double> hnext(K, 0.0);
      {
        std::vector<int> L;
        std::vector<std::vector<LrTerm>> terms(K);
        for (int k : arn) {
          if (rW[k] == 0) continue;
          terms[k].push_back(LrTerm{S->tall(S->UD, k, ldR), S->vside(S->VD, k, ldR), rW[k], 1.0});
          for (int i = 0; i <= j; ++i) terms[k].push_back(LrTerm{GU(i, k), GV(i, k), rb[k][i], -h[k][i]});
          L.push_back(k);
        }
        std::vector<double> kw;
        LRFSI_TRY(truncate_sum(S, L, terms, o.tol, Uo, Vo, rk, &kw, s));
        for (int k : L) {
          rW[k] = rk[k];
          hnext[k] = std::sqrt(kw[k]);
        }
      }
      // Givens rotations on column j; g_{j+1} is the least-squares residual
      std::vector<int> cont;
      for (int k : arn) {
        std::vector<double> col(j + 2, 0.0);
        for (int i = 0; i <= j; ++i) col[i] = h[k][i];
        col[j + 1] = hnext[k];
        for (int i = 0; i < j; ++i) {
          const double a = col[i], b = col[i + 1];
          col[i] = cs[k][i] * a + sn[k][i] * b;
          col[i + 1] = -sn[k][i] * a + cs[k][i] * b;
        }
        const double den = std::hypot(col[j], col[j + 1]);
        cs[k][j] = den > 0 ? col[j] / den : 1.0;
        sn[k][j] = den > 0 ? col[j + 1] / den : 0.0;
        col[j] = den;
        g[k][j + 1] = -sn[k][j] * g[k][j];
        g[k][j] = cs[k][j] * g[k][j];
        for (int i = 0; i <= j; ++i) Rh[k][(size_t)i * nit + j] = col[i];
        nstep[k] = j + 1;
        st[k].steps += 1;
        const bool stop = hnext[k] == 0.0 || rW[k] == 0 || (o.eta > 0 && std::fabs(g[k][j + 1]) <= o.eta * nB[k]);
        if (!stop && j + 1 < nit) {
          cont.push_back(k);
          rb[k][j + 1] = rW[k];
        }
      }
      // V_{j+1} = W / h_{j+1,j}
      {
        std::vector<CopyDesc> cd;
        for (int k : cont) {
          cd.push_back(CopyDesc{S->tall(S->UD, k, ldR), ldR, GU(j + 1, k), ldR, M, rW[k], 0, nullptr, 1.0});
          cd.push_back(CopyDesc{S->vside(S->VD, k, ldR), ldR, GV(j + 1, k), ldR, S->m[k], rW[k], 0, nullptr,
                                1.0 / hnext[k]});
        }
        LRFSI_TRY(copy_batched(cd, s));
      }
      arn.swap(cont);
    }
    // y = Rh^{-1} g (n x n upper triangular), S <- T(S + sum_j y_j Z_j)
    {
      std::vector<int> L;
      std::vector<std::vector<LrTerm>> terms(K);
      std::vector<double*> Us(K), Vs(K);
      for (int k : live) {
        const int n = nstep[k];
        std::vector<double> y(n, 0.0);
        for (int i = n - 1; i >= 0; --i) {
          double t = g[k][i];
          for (int l = i + 1; l < n; ++l) t -= Rh[k][(size_t)i * nit + l] * y[l];
          const double dg = Rh[k][(size_t)i * nit + i];
          y[i] = dg != 0.0 ? t / dg : 0.0;
        }
        Us[k] = S->tall(S->US, k, ldR);
        Vs[k] = S->vside(S->VS, k, ldR);
        terms[k].push_back(LrTerm{Us[k], Vs[k], rS[k], 1.0});
        for (int i = 0; i < n; ++i) terms[k].push_back(LrTerm{GZ(i, k), GV(i, k), rb[k][i], y[i]});
        L.push_back(k);
      }
      LRFSI_TRY(truncate_sum(S, L, terms, o.tol, Us, Vs, rk, nullptr, s));
      for (int k : L) rS[k] = rk[k];
    }
  }
  for (int k : act) st[k].rank = rS[k];
  return LRFSI_OK;
}

// Workspace of the selected solver, set up at an entry point before anything
// takes the concatenation width (GMREST: Krylov basis, widened buffers).
static int solver_prepare(lrfsi_subset_s* S, const lrfsi_cheb_options& o) {
  if (o.solver != 1) return LRFSI_OK;
  if (S->four) return fail(LRFSI_EINVAL, "GMREST is not available for four-parameter subsets (use ChebyshevT)");
  LRFSI_TRY(gmres_alloc(S, o.iters));
  return widen_concat(S, (o.iters + 1) * S->Rmax);
}

// The low-rank solver the options select (0: ChebyshevT, 1: GMREST).
static int lr_solve(lrfsi_subset_s* S, const lrfsi_cheb_options& o, const std::vector<int>& act,
                    std::vector<int>& rS, std::vector<lrfsi_cheb_stats>& st, cudaStream_t s) {
  if (o.solver == 1) return gmres_run(S, o, act, rS, st, s);
  return g_graph_mode.load() > 0 ? cheb_fixed(S, o, act, rS, st, s) : cheb_run(S, o, act, rS, st, s);
}

static int check_opts(const lrfsi_cheb_options* o) {
  if (!o || o->solver < 0 || o->solver > 1 || o->iters < 1 || o->cycles < 1 || o->rank_cap < 1 || !(o->tol >= 0) ||
      o->precision < 0 || o->precision > 1 || !(o->tol_sol >= 0))
    return fail(LRFSI_EINVAL, "lrfsi_cheb_options: need solver 0 or 1, iters, cycles, rank_cap >= 1, tol >= 0");
  if (o->solver == 0 && !(o->c > 0 && o->d > o->c))
    return fail(LRFSI_EINVAL, "lrfsi_cheb_options: ChebyshevT needs 0 < c < d");
  return LRFSI_OK;
}

}  // namespace lrfsi

// F_k(S_k) = UB_k VB_k^T by the given solver (0: ChebyshevT, 1: GMREST).
static int lowrank_solve(lrfsi_subset_h S, const double* UB, int lduB, const double* VB, int ldvB, const int* rB_h,
                         const lrfsi_cheb_options* opt_in, int solver, double* U, int ldu, double* V, int ldv,
                         int* rank_h, lrfsi_cheb_stats* stats, lrfsi_stream_t stream) {
  if (!S || !UB || !VB || !rB_h || !U || !V || !rank_h || !opt_in)
    return fail(LRFSI_EINVAL, "lrfsi_chebyshevT / lrfsi_gmresT: null argument");
  lrfsi_cheb_options o = *opt_in;
  o.solver = solver;
  const lrfsi_cheb_options* opt = &o;
  LRFSI_TRY(check_opts(opt));
  LRFSI_TRY(solver_prepare(S, *opt));
  cudaStream_t s = (cudaStream_t)stream;
  const int K = S->K, ldR = S->ldR;
  const long M = S->M;
  std::vector<int> act, rB(K);
  std::vector<GemmDesc<double>> gm;
  for (int k = 0; k < K; ++k) {
    rB[k] = rB_h[k];
    if (rB[k] < 1 || rB[k] > lduB || rB[k] > ldvB || ldu < S->cap[k] || ldv < S->cap[k])
      return fail(LRFSI_EINVAL, "lrfsi_chebyshevT: rank / leading dimension mismatch");
    act.push_back(k);
    // dense B_k = UB_k VB_k^T (M x m_k)
    gm.push_back(GemmDesc<double>{(int)M, S->m[k], rB[k], UB + (size_t)k * M * lduB, lduB, 1,
                                  VB + (size_t)S->off[k] * ldvB, 1, ldvB, S->tall(S->UB, k, ldR), ldR, 1, 1.0, 0.0});
    gm.back().tc = 1;
  }
  LRFSI_TRY(gemm_grouped<double>(gm.data(), (int)gm.size(), s));
  {
    std::vector<CopyDesc> sc;
    for (int k = 0; k < K; ++k)
      sc.push_back(CopyDesc{S->tall(S->UB, k, ldR), ldR, S->tall(S->UB, k, ldR), ldR, M, S->m[k], 0,
                            S->rsc.p + (size_t)k * M, 1.0});
    LRFSI_TRY(copy_batched(sc, s));
  }
  std::vector<int> rS;
  std::vector<lrfsi_cheb_stats> st;
  LRFSI_TRY(lr_solve(S, *opt, act, rS, st, s));
  std::vector<CopyDesc> cd;
  for (int k = 0; k < K; ++k) {
    rank_h[k] = rS[k];
    if (stats) stats[k] = st[k];
    cd.push_back(CopyDesc{S->tall(S->US, k, ldR), ldR, U + (size_t)k * M * ldu, ldu, M, rS[k], 0,
                          S->csc.p + (size_t)k * M, 1.0});
    cd.push_back(CopyDesc{S->vside(S->VS, k, ldR), ldR, V + (size_t)S->off[k] * ldv, ldv, S->m[k], rS[k], 0, nullptr, 1.0});
  }
  LRFSI_TRY(copy_batched(cd, s));
  LRFSI_CUDA(cudaStreamSynchronize(s));
  return LRFSI_OK;
}

using namespace lrfsi;

extern "C" int lrfsi_graph_mode(int mode, int* previous) {
  if (mode < -1 || mode > 2) return fail(LRFSI_EINVAL, "lrfsi_graph_mode: mode must be 0, 1, 2 (or -1 to query)");
  const int old = mode >= 0 ? g_graph_mode.exchange(mode) : g_graph_mode.load();
  if (previous) *previous = old;
  return LRFSI_OK;
}

extern "C" int lrfsi_graph_counters(int64_t* out3, int reset) {
  if (!out3) return fail(LRFSI_EINVAL, "lrfsi_graph_counters: null output");
  out3[0] = g_graph_replays.load();
  out3[1] = g_graph_captures.load();
  out3[2] = g_graph_fallbacks.load();
  if (reset) {
    g_graph_replays = 0;
    g_graph_captures = 0;
    g_graph_fallbacks = 0;
  }
  return LRFSI_OK;
}

extern "C" int lrfsi_chebyshevT(lrfsi_subset_h S, const double* UB, int lduB, const double* VB, int ldvB,
                                const int* rB_h, const lrfsi_cheb_options* opt, double* U, int ldu, double* V, int ldv,
                                int* rank_h, lrfsi_cheb_stats* stats, lrfsi_stream_t stream) {
  return lowrank_solve(S, UB, lduB, VB, ldvB, rB_h, opt, 0, U, ldu, V, ldv, rank_h, stats, stream);
}

extern "C" int lrfsi_gmresT(lrfsi_subset_h S, const double* UB, int lduB, const double* VB, int ldvB, const int* rB_h,
                            const lrfsi_cheb_options* opt, double* U, int ldu, double* V, int ldv, int* rank_h,
                            lrfsi_cheb_stats* stats, lrfsi_stream_t stream) {
  return lowrank_solve(S, UB, lduB, VB, ldvB, rB_h, opt, 1, U, ldu, V, ldv, rank_h, stats, stream);
}

__global__ void k_recip(const double* __restrict__ x, long n, double* __restrict__ y) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) y[e] = x[e] != 0.0 ? 1.0 / x[e] : 0.0;
}

// rows i of V (ld) with flag[i] != 0 set to zero (columns 0..r-1)
__global__ void k_zero_flagged_rows(double* __restrict__ V, int ld, int r, const int* __restrict__ flag, int n) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)n * r) return;
  const int i = (int)(e / r), j = (int)(e % r);
  if (flag[i]) V[(size_t)i * ld + j] = 0.0;
}

// Nonlinear residuals of X = xt 1^T + diag(c) U_C V_C^T (UC/VC, ranks rC) and
// chord corrections (right-hand side -R(X_i) per column, operators and
// preconditioner kept at xt) until every column's relative residual is <=
// target or max_outer corrections were made (LRFSI_ENOCONV).  rel receives the
// last relative residuals, outer the corrections per subset.
static int outer_corrections(lrfsi_subset_s* S, const lrfsi_cheb_options& o, double target, int max_outer,
                             std::vector<int>& rC, std::vector<int>& outer, std::vector<double>& rel, cudaStream_t s) {
  const int K = S->K, ldR = S->ldR, ldP = S->ldP;
  const long M = S->M;
  std::vector<CopyDesc> cd;
  std::vector<int> rS;
  std::vector<lrfsi_cheb_stats> st;
  int status = LRFSI_OK;
  for (int it = 0;; ++it) {
    // X = xt 1^T + diag(c) U_C V_C^T (dense columns, M x mtot) and its nonlinear residual
    std::vector<GemmDesc<double>> gm;
    for (int k = 0; k < K; ++k) {
      if (rC[k] > 0)  // FP64 kernels: these columns' residuals are the reported ones
        gm.push_back(GemmDesc<double>{(int)M, S->m[k], rC[k], S->tall(S->UC, k, ldR), ldR, 1,
                                      S->vside(S->VC, k, ldR), 1, ldR, S->Xd.p + S->off[k], S->mtot, 1, 1.0, 0.0});
      else
        LRFSI_CUDA(cudaMemset2DAsync(S->Xd.p + S->off[k], sizeof(double) * S->mtot, 0, sizeof(double) * S->m[k], M, s));
    }
    if (!gm.empty()) LRFSI_TRY(gemm_grouped<double>(gm.data(), (int)gm.size(), s));
    for (int k = 0; k < K; ++k) {
      k_affine_cols<<<ceil_div(M * S->m[k], 256), 256, 0, s>>>(S->Xd.p, S->mtot, S->off[k], S->m[k],
                                                              S->xt.p + (size_t)k * M, S->csc.p + (size_t)k * M, M);
      LRFSI_TRY(check_launch("k_affine_cols"));
    }
    LRFSI_TRY(launch_residual(S->mesh, S->Xd.p, S->mtot, S->mtot, nullptr, S->mu.p, S->nu_res(), S->rc.R.p, S->mtot, s,
                              S->rho_res(), S->lam_res()));
    if (S->timestep) {  // R_theta of the time step (Sec. 4.3); Xd becomes X - X_prev
      TimeStep ts;
      ts.Xprev = S->Xprev.p;
      ts.Rprev = S->Rprev.p;
      ts.M3 = S->M3.p;
      ts.Mv = S->Mv.p;
      ts.theta = S->theta;
      ts.cm = S->cm;
      LRFSI_TRY(theta_residual_cols(S->mesh, ts, S->Xd.p, S->mtot, S->rc.R.p, S->Xd.p, S->Yth.p, s));
    }
    LRFSI_TRY(launch_colnorm2(S->rc.R.p, M, S->mtot, S->mtot, S->rc.norm2.p, S->rc.work.p, S->rc.work.n, s));
    std::vector<double> a(S->mtot), b(S->mtot);
    LRFSI_CUDA(cudaMemcpyAsync(a.data(), S->rc.norm2.p, sizeof(double) * S->mtot, cudaMemcpyDeviceToHost, s));
    LRFSI_CUDA(cudaMemcpyAsync(b.data(), S->rc.norm2_bD.p, sizeof(double) * S->mtot, cudaMemcpyDeviceToHost, s));
    LRFSI_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < S->mtot; ++i) rel[i] = b[i] > 0 ? std::sqrt(a[i] / b[i]) : std::sqrt(a[i]);
    if (target <= 0) break;
    std::vector<int> need;
    for (int k = 0; k < K; ++k) {
      double mx = 0;
      for (int i = S->off[k]; i < S->off[k] + S->m[k]; ++i) mx = std::max(mx, rel[i]);
      if (mx > target) need.push_back(k);
    }
    if (need.empty()) break;
    if (it >= max_outer) {
      status = LRFSI_ENOCONV;
      break;
    }
    // correction: B = -R(X) (dense, rank <= m_k as factors (R_k, I))
    cd.clear();
    for (int k : need) {
      const int m = S->m[k];
      // UB must hold m columns: ldR >= mmax by construction
      cd.push_back(CopyDesc{S->rc.R.p + S->off[k], S->mtot, S->tall(S->UB, k, ldR), ldR, M, m, 0,
                            S->rsc.p + (size_t)k * M, -1.0});
    }
    LRFSI_TRY(copy_batched(cd, s));
    LRFSI_TRY(lr_solve(S, o, need, rS, st, s));
    // accumulate: C <- T([U_C | U_S], [V_C | V_S])
    cd.clear();
    std::vector<int> p(K, 0);
    std::vector<double*> Uo(K), Vo(K);
    for (int k : need) {
      cd.push_back(CopyDesc{S->tall(S->UC, k, ldR), ldR, S->tall(S->Xcat, k, ldP), ldP, M, rC[k], 0, nullptr, 1.0});
      cd.push_back(CopyDesc{S->tall(S->US, k, ldR), ldR, S->tall(S->Xcat, k, ldP) + rC[k], ldP, M, rS[k], 0, nullptr, 1.0});
      cd.push_back(CopyDesc{S->vside(S->VC, k, ldR), ldR, S->vside(S->Vcat, k, ldP), ldP, S->m[k], rC[k], 0, nullptr, 1.0});
      cd.push_back(CopyDesc{S->vside(S->VS, k, ldR), ldR, S->vside(S->Vcat, k, ldP) + rC[k], ldP, S->m[k], rS[k], 0,
                            nullptr, 1.0});
      p[k] = rC[k] + rS[k];
      Uo[k] = S->tall(S->UC, k, ldR);
      Vo[k] = S->vside(S->VC, k, ldR);
      outer[k] += 1;
    }
    LRFSI_TRY(copy_batched(cd, s));
    std::vector<int> rk;
    std::vector<double> f2;
    const double tol_sol = o.tol_sol > 0 ? o.tol_sol : 1e-6 * o.tol;
    LRFSI_TRY(truncate_batch(S, need, p, tol_sol, S->cap, Uo, Vo, rk, f2, s));
    for (int k : need) rC[k] = rk[k];
  }
  return status;
}

extern "C" int lrfsi_subset_step(lrfsi_subset_h S, const lrfsi_cheb_options* opt, double target, int max_outer,
                                 double* U, int ldu, double* V, int ldv, int* rank_h, double* relres_h, int* outer_h,
                                 lrfsi_stream_t stream) {
  if (!S || !U || !V || !rank_h || max_outer < 0) return fail(LRFSI_EINVAL, "lrfsi_subset_step: bad argument");
  LRFSI_TRY(check_opts(opt));
  LRFSI_TRY(solver_prepare(S, *opt));
  cudaStream_t s = (cudaStream_t)stream;
  const int K = S->K, ldR = S->ldR;
  const long M = S->M;
  for (int k = 0; k < K; ++k)
    if (ldu < S->cap[k] || ldv < S->cap[k]) return fail(LRFSI_EINVAL, "lrfsi_subset_step: ldu/ldv < rank cap");
  // B_k = -(R0 1^T + Rmu mu^T + Rnu nu^T), dense M x m_k in UB
  std::vector<CopyDesc> cd;
  std::vector<GemmDesc<double>> gb;
  std::vector<int> act;
  for (int k = 0; k < K; ++k) {
    act.push_back(k);
    double* vb = S->vside(S->VB, k, ldR);
    cd.push_back(CopyDesc{nullptr, 0, vb, ldR, S->m[k], 1, 1, nullptr, -1.0});
    cd.push_back(CopyDesc{nullptr, 0, vb + 1, ldR, S->m[k], 1, 1, S->mu.p + S->off[k], -1.0});
    cd.push_back(CopyDesc{nullptr, 0, vb + 2, ldR, S->m[k], 1, 1, S->nu.p + S->off[k], -1.0});
    gb.push_back(GemmDesc<double>{(int)M, S->m[k], 3, S->R3.p + (size_t)k * 3 * M, 3, 1, vb, 1, ldR,
                                  S->tall(S->UB, k, ldR), ldR, 1, 1.0, 0.0});
    if (S->four) {  // B^{mu,nu,lambda,rho}: -(... + Rlam lam^T + Rrho rho^T) (Sec. 4.4)
      cd.push_back(CopyDesc{nullptr, 0, vb + 3, ldR, S->m[k], 1, 1, S->lam.p + S->off[k], -1.0});
      cd.push_back(CopyDesc{nullptr, 0, vb + 4, ldR, S->m[k], 1, 1, S->rho.p + S->off[k], -1.0});
    }
  }
  LRFSI_TRY(copy_batched(cd, s));
  LRFSI_TRY(gemm_grouped<double>(gb.data(), (int)gb.size(), s));
  if (S->four) {
    std::vector<GemmDesc<double>> g2;
    for (int k = 0; k < K; ++k)
      g2.push_back(GemmDesc<double>{(int)M, S->m[k], 2, S->R3x.p + (size_t)k * 3 * M, 3, 1, S->vside(S->VB, k, ldR) + 3,
                                    1, ldR, S->tall(S->UB, k, ldR), ldR, 1, 1.0, 1.0});
    LRFSI_TRY(gemm_grouped<double>(g2.data(), (int)g2.size(), s));
  }
  cd.clear();
  for (int k = 0; k < K; ++k)
    cd.push_back(CopyDesc{S->tall(S->UB, k, ldR), ldR, S->tall(S->UB, k, ldR), ldR, M, S->m[k], 0,
                          S->rsc.p + (size_t)k * M, 1.0});
  LRFSI_TRY(copy_batched(cd, s));
  std::vector<int> rS;
  std::vector<lrfsi_cheb_stats> st;
  LRFSI_TRY(lr_solve(S, *opt, act, rS, st, s));
  // keep the accumulated update in UC/VC
  std::vector<int> rC = rS;
  cd.clear();
  for (int k = 0; k < K; ++k) {
    cd.push_back(CopyDesc{S->tall(S->US, k, ldR), ldR, S->tall(S->UC, k, ldR), ldR, M, rC[k], 0, nullptr, 1.0});
    cd.push_back(CopyDesc{S->vside(S->VS, k, ldR), ldR, S->vside(S->VC, k, ldR), ldR, S->m[k], rC[k], 0, nullptr, 1.0});
  }
  LRFSI_TRY(copy_batched(cd, s));
  std::vector<int> outer(K, 0);
  std::vector<double> rel(S->mtot, 0.0);
  const int status = outer_corrections(S, *opt, target, max_outer, rC, outer, rel, s);
  if (status != LRFSI_OK && status != LRFSI_ENOCONV) return status;
  cd.clear();
  for (int k = 0; k < K; ++k) {
    rank_h[k] = rC[k];
    if (outer_h) outer_h[k] = outer[k];
    cd.push_back(CopyDesc{S->tall(S->UC, k, ldR), ldR, U + (size_t)k * M * ldu, ldu, M, rC[k], 0,
                          S->csc.p + (size_t)k * M, 1.0});
    cd.push_back(CopyDesc{S->vside(S->VC, k, ldR), ldR, V + (size_t)S->off[k] * ldv, ldv, S->m[k], rC[k], 0, nullptr, 1.0});
  }
  LRFSI_TRY(copy_batched(cd, s));
  LRFSI_CUDA(cudaStreamSynchronize(s));
  if (relres_h) std::memcpy(relres_h, rel.data(), sizeof(double) * S->mtot);
  if (status != LRFSI_OK) return fail(status, "lrfsi_subset_step: target not reached within max_outer corrections");
  return LRFSI_OK;
}

extern "C" int lrfsi_subset_step_theta(lrfsi_subset_h S, const lrfsi_cheb_options* opt, const double* Xprev, int ldx,
                                       double target, int max_outer, double* U, int ldu, double* V, int ldv,
                                       int* rank_h, double* relres_h, int* outer_h, lrfsi_stream_t stream) {
  if (!S || !Xprev || !U || !V || !rank_h || max_outer < 1 || ldx < S->mtot)
    return fail(LRFSI_EINVAL, "lrfsi_subset_step_theta: bad argument (max_outer >= 1, ldx >= sum m_k)");
  if (!S->timestep) return fail(LRFSI_EINVAL, "lrfsi_subset_step_theta: handle not made by lrfsi_subset_create_theta");
  LRFSI_TRY(check_opts(opt));
  LRFSI_TRY(solver_prepare(S, *opt));
  cudaStream_t s = (cudaStream_t)stream;
  const int K = S->K, ldR = S->ldR;
  const long M = S->M;
  for (int k = 0; k < K; ++k)
    if (ldu < S->cap[k] || ldv < S->cap[k]) return fail(LRFSI_EINVAL, "lrfsi_subset_step_theta: ldu/ldv < rank cap");
  LRFSI_CUDA(cudaMemcpy2DAsync(S->Xprev.p, sizeof(double) * S->mtot, Xprev, sizeof(double) * ldx,
                               sizeof(double) * S->mtot, M, cudaMemcpyDeviceToDevice, s));
  LRFSI_TRY(launch_residual(S->mesh, S->Xprev.p, S->mtot, S->mtot, nullptr, S->mu.p, S->nu.p, S->Rprev.p, S->mtot, s));
  // from X = x~ 1^T: the first correction is the Newton step of Eq. (timedep_matrix1)
  std::vector<int> rC(K, 0), outer(K, 0);
  std::vector<double> rel(S->mtot, 0.0);
  const int status = outer_corrections(S, *opt, target, max_outer, rC, outer, rel, s);
  if (status != LRFSI_OK && status != LRFSI_ENOCONV) return status;
  std::vector<CopyDesc> cd;
  for (int k = 0; k < K; ++k) {
    rank_h[k] = rC[k];
    if (outer_h) outer_h[k] = outer[k];
    cd.push_back(CopyDesc{S->tall(S->UC, k, ldR), ldR, U + (size_t)k * M * ldu, ldu, M, rC[k], 0,
                          S->csc.p + (size_t)k * M, 1.0});
    cd.push_back(CopyDesc{S->vside(S->VC, k, ldR), ldR, V + (size_t)S->off[k] * ldv, ldv, S->m[k], rC[k], 0, nullptr, 1.0});
  }
  LRFSI_TRY(copy_batched(cd, s));
  LRFSI_CUDA(cudaStreamSynchronize(s));
  if (relres_h) std::memcpy(relres_h, rel.data(), sizeof(double) * S->mtot);
  if (status != LRFSI_OK) return fail(status, "lrfsi_subset_step_theta: target not reached within max_outer corrections");
  return LRFSI_OK;
}

extern "C" int lrfsi_subset_step_init(lrfsi_subset_h S, const lrfsi_cheb_options* opt, double target,
                                      int max_outer, const double* U0, int ldu0, const double* V0, int ldv0,
                                      const int* r0_h, double* U, int ldu, double* V, int ldv, int* rank_h,
                                      double* relres_h, int* outer_h, int* fallback_h, lrfsi_stream_t stream) {
  if (!S || !U0 || !V0 || !r0_h || !U || !V || !rank_h || max_outer < 0)
    return fail(LRFSI_EINVAL, "lrfsi_subset_step_init: bad argument");
  LRFSI_TRY(check_opts(opt));
  LRFSI_TRY(solver_prepare(S, *opt));
  cudaStream_t s = (cudaStream_t)stream;
  const int K = S->K, ldR = S->ldR, ldP = S->ldP;
  const long M = S->M;
  for (int k = 0; k < K; ++k) {
    if (ldu < S->cap[k] || ldv < S->cap[k]) return fail(LRFSI_EINVAL, "lrfsi_subset_step_init: ldu/ldv < rank cap");
    if (r0_h[k] < 0 || r0_h[k] > ldu0 || r0_h[k] > ldv0 || r0_h[k] > ldP)
      return fail(LRFSI_EINVAL, "lrfsi_subset_step_init: initial rank r0_k out of range");
  }
  if (!S->cinv.p) {
    LRFSI_TRY(S->cinv.alloc((size_t)K * M));
    k_recip<<<ceil_div((long)K * M, 256), 256, 0, s>>>(S->csc.p, (long)K * M, S->cinv.p);
    LRFSI_TRY(check_launch("k_recip"));
  }
  // C = T(diag(c)^{-1} U0, V0): the start in the scaled coordinates, at most cap_k
  std::vector<CopyDesc> cd;
  std::vector<int> act, p(K, 0), rC(K, 0);
  std::vector<double*> Uo(K), Vo(K);
  for (int k = 0; k < K; ++k) {
    if (r0_h[k] == 0) continue;
    act.push_back(k);
    cd.push_back(CopyDesc{U0 + (size_t)k * M * ldu0, ldu0, S->tall(S->Xcat, k, ldP), ldP, M, r0_h[k], 0,
                          S->cinv.p + (size_t)k * M, 1.0});
    cd.push_back(CopyDesc{V0 + (size_t)S->off[k] * ldv0, ldv0, S->vside(S->Vcat, k, ldP), ldP, S->m[k], r0_h[k], 0,
                          nullptr, 1.0});
    p[k] = r0_h[k];
    Uo[k] = S->tall(S->UC, k, ldR);
    Vo[k] = S->vside(S->VC, k, ldR);
  }
  LRFSI_TRY(copy_batched(cd, s));
  if (!act.empty()) {
    std::vector<int> rk;
    std::vector<double> f2;
    const double tol_sol = opt->tol_sol > 0 ? opt->tol_sol : 1e-6 * opt->tol;
    LRFSI_TRY(truncate_batch(S, act, p, tol_sol, S->cap, Uo, Vo, rk, f2, s));
    for (int k : act) rC[k] = rk[k];
  }
  // fallback: columns whose start does not cut the residual of the median
  // solution x~_k restart from x~_k (their row of V_C is zeroed)
  std::vector<int> fb(S->mtot, 0);
  {
    std::vector<GemmDesc<double>> gm;
    for (int k = 0; k < K; ++k) {
      if (rC[k] > 0)  // FP64 kernels: these columns' residuals are the reported ones
        gm.push_back(GemmDesc<double>{(int)M, S->m[k], rC[k], S->tall(S->UC, k, ldR), ldR, 1,
                                      S->vside(S->VC, k, ldR), 1, ldR, S->Xd.p + S->off[k], S->mtot, 1, 1.0, 0.0});
      else
        LRFSI_CUDA(cudaMemset2DAsync(S->Xd.p + S->off[k], sizeof(double) * S->mtot, 0, sizeof(double) * S->m[k], M, s));
    }
    if (!gm.empty()) LRFSI_TRY(gemm_grouped<double>(gm.data(), (int)gm.size(), s));
    for (int k = 0; k < K; ++k) {
      k_affine_cols<<<ceil_div(M * S->m[k], 256), 256, 0, s>>>(S->Xd.p, S->mtot, S->off[k], S->m[k],
                                                              S->xt.p + (size_t)k * M, S->csc.p + (size_t)k * M, M);
      LRFSI_TRY(check_launch("k_affine_cols"));
    }
    LRFSI_TRY(launch_residual(S->mesh, S->Xd.p, S->mtot, S->mtot, nullptr, S->mu.p, S->nu_res(), S->rc.R.p, S->mtot, s,
                              S->rho_res(), S->lam_res()));
    LRFSI_TRY(launch_colnorm2(S->rc.R.p, M, S->mtot, S->mtot, S->rc.norm2.p, S->rc.work.p, S->rc.work.n, s));
    std::vector<double> a(S->mtot), b(S->mtot);
    LRFSI_CUDA(cudaMemcpyAsync(a.data(), S->rc.norm2.p, sizeof(double) * S->mtot, cudaMemcpyDeviceToHost, s));
    // the median solutions themselves: Xd columns = x~_k
    LRFSI_CUDA(cudaMemsetAsync(S->Xd.p, 0, sizeof(double) * (size_t)M * S->mtot, s));
    for (int k = 0; k < K; ++k) {
      k_affine_cols<<<ceil_div(M * S->m[k], 256), 256, 0, s>>>(S->Xd.p, S->mtot, S->off[k], S->m[k],
                                                              S->xt.p + (size_t)k * M, S->csc.p + (size_t)k * M, M);
      LRFSI_TRY(check_launch("k_affine_cols"));
    }
    LRFSI_TRY(launch_residual(S->mesh, S->Xd.p, S->mtot, S->mtot, nullptr, S->mu.p, S->nu_res(), S->rc.R.p, S->mtot, s,
                              S->rho_res(), S->lam_res()));
    LRFSI_TRY(launch_colnorm2(S->rc.R.p, M, S->mtot, S->mtot, S->rc.norm2.p, S->rc.work.p, S->rc.work.n, s));
    LRFSI_CUDA(cudaMemcpyAsync(b.data(), S->rc.norm2.p, sizeof(double) * S->mtot, cudaMemcpyDeviceToHost, s));
    LRFSI_CUDA(cudaStreamSynchronize(s));
    bool any = false;
    for (int i = 0; i < S->mtot; ++i) {
      fb[i] = !(a[i] < b[i]);
      any = any || fb[i];
    }
    if (any) {
      DevBuf<int> fdev;
      LRFSI_TRY(fdev.upload(fb, s));
      for (int k = 0; k < K; ++k) {
        if (rC[k] <= 0) continue;
        k_zero_flagged_rows<<<ceil_div((long)S->m[k] * rC[k], 256), 256, 0, s>>>(
            S->vside(S->VC, k, ldR), ldR, rC[k], fdev.p + S->off[k], S->m[k]);
        LRFSI_TRY(check_launch("k_zero_flagged_rows"));
      }
      LRFSI_CUDA(cudaStreamSynchronize(s));
    }
  }
  std::vector<int> outer(K, 0);
  std::vector<double> rel(S->mtot, 0.0);
  const int status = outer_corrections(S, *opt, target, max_outer, rC, outer, rel, s);
  if (status != LRFSI_OK && status != LRFSI_ENOCONV) return status;
  cd.clear();
  for (int k = 0; k < K; ++k) {
    rank_h[k] = rC[k];
    if (outer_h) outer_h[k] = outer[k];
    cd.push_back(CopyDesc{S->tall(S->UC, k, ldR), ldR, U + (size_t)k * M * ldu, ldu, M, rC[k], 0,
                          S->csc.p + (size_t)k * M, 1.0});
    cd.push_back(CopyDesc{S->vside(S->VC, k, ldR), ldR, V + (size_t)S->off[k] * ldv, ldv, S->m[k], rC[k], 0, nullptr, 1.0});
  }
  LRFSI_TRY(copy_batched(cd, s));
  LRFSI_CUDA(cudaStreamSynchronize(s));
  if (relres_h) std::memcpy(relres_h, rel.data(), sizeof(double) * S->mtot);
  if (fallback_h) std::memcpy(fallback_h, fb.data(), sizeof(int) * S->mtot);
  if (status != LRFSI_OK) return fail(status, "lrfsi_subset_step_init: target not reached within max_outer corrections");
  return LRFSI_OK;
}

extern "C" int lrfsi_precond_apply(lrfsi_subset_h S, const double* X, int ldx, const int* r_h, double* Y, int ldy,
                                   lrfsi_stream_t stream) {
  if (!S || !X || !Y || !r_h) return fail(LRFSI_EINVAL, "lrfsi_precond_apply: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int K = S->K, ldP = S->ldP;
  const long M = S->M;
  std::vector<CopyDesc> cd;
  std::vector<double*> Xs(K), Ys(K);
  std::vector<int> rr(K);
  for (int k = 0; k < K; ++k) {
    rr[k] = r_h[k];
    if (rr[k] < 0 || rr[k] > ldx || rr[k] > ldy || rr[k] > ldP) return fail(LRFSI_EINVAL, "lrfsi_precond_apply: r_k");
    // scaled right-hand side diag(r) X into Xcat, solve into Q1, unscale by c
    cd.push_back(CopyDesc{X + (size_t)k * M * ldx, ldx, S->tall(S->Xcat, k, ldP), ldP, M, rr[k], 0,
                          S->rsc.p + (size_t)k * M, 1.0});
    Xs[k] = S->tall(S->Xcat, k, ldP);
    Ys[k] = S->tall(S->Q1, k, ldP);
  }
  LRFSI_TRY(copy_batched(cd, s));
  {  // in chunks of at most the LU's solve width
    const int w = S->lu.max_cols();
    int rmax = 0;
    for (int k = 0; k < K; ++k) rmax = std::max(rmax, rr[k]);
    for (int c0 = 0; c0 < rmax; c0 += w) {
      std::vector<double*> Xc(K), Yc(K);
      std::vector<int> rc(K);
      for (int k = 0; k < K; ++k) {
        Xc[k] = Xs[k] + c0;
        Yc[k] = Ys[k] + c0;
        rc[k] = std::max(0, std::min(w, rr[k] - c0));
      }
      LRFSI_TRY(S->lu.solve(Xc.data(), Yc.data(), rc.data(), ldP, K, s));
    }
  }
  cd.clear();
  for (int k = 0; k < K; ++k)
    cd.push_back(CopyDesc{S->tall(S->Q1, k, ldP), ldP, Y + (size_t)k * M * ldy, ldy, M, rr[k], 0,
                          S->csc.p + (size_t)k * M, 1.0});
  LRFSI_TRY(copy_batched(cd, s));
  LRFSI_CUDA(cudaStreamSynchronize(s));
  return LRFSI_OK;
}

extern "C" int lrfsi_truncate(lrfsi_subset_h S, const double* X, int ldx, const double* V, int ldv, const int* p_h,
                              double tol, const int* cap_h, double* U, int ldu, double* Vo, int ldvo, int* rank_h,
                              lrfsi_stream_t stream) {
  if (!S || !X || !V || !p_h || !cap_h || !U || !Vo || !rank_h || !(tol >= 0))
    return fail(LRFSI_EINVAL, "lrfsi_truncate: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int K = S->K, ldP = S->ldP, ldR = S->ldR;
  const long M = S->M;
  std::vector<CopyDesc> cd;
  std::vector<int> act, p(K), cap(K);
  std::vector<double*> Uo(K), Vout(K);
  for (int k = 0; k < K; ++k) {
    p[k] = p_h[k];
    cap[k] = std::min(cap_h[k], ldR);
    if (p[k] < 1 || p[k] > ldx || p[k] > ldv || p[k] > ldP || cap[k] < 1 || ldu < cap[k] || ldvo < cap[k])
      return fail(LRFSI_EINVAL, "lrfsi_truncate: rank / leading dimension mismatch");
    act.push_back(k);
    cd.push_back(CopyDesc{X + (size_t)k * M * ldx, ldx, S->tall(S->Xcat, k, ldP), ldP, M, p[k], 0, nullptr, 1.0});
    cd.push_back(CopyDesc{V + (size_t)S->off[k] * ldv, ldv, S->vside(S->Vcat, k, ldP), ldP, S->m[k], p[k], 0, nullptr,
                          1.0});
    Uo[k] = S->tall(S->UR, k, ldR);
    Vout[k] = S->vside(S->VR, k, ldR);
  }
  LRFSI_TRY(copy_batched(cd, s));
  std::vector<int> rk;
  std::vector<double> f2;
  LRFSI_TRY(truncate_batch(S, act, p, tol, cap, Uo, Vout, rk, f2, s));
  cd.clear();
  for (int k = 0; k < K; ++k) {
    rank_h[k] = rk[k];
    cd.push_back(CopyDesc{S->tall(S->UR, k, ldR), ldR, U + (size_t)k * M * ldu, ldu, M, rk[k], 0, nullptr, 1.0});
    cd.push_back(CopyDesc{S->vside(S->VR, k, ldR), ldR, Vo + (size_t)S->off[k] * ldvo, ldvo, S->m[k], rk[k], 0,
                          nullptr, 1.0});
  }
  LRFSI_TRY(copy_batched(cd, s));
  LRFSI_CUDA(cudaStreamSynchronize(s));
  return LRFSI_OK;
}

extern "C" int lrfsi_pod(lrfsi_mesh_h mesh, const double* X, int ldx, int n, int k, double* Phi, int ldphi, double* C,
                         int ldc, double* sigma, lrfsi_stream_t stream) {
  if (!mesh || !X || !Phi || !C || n < 1 || k < 1 || k > n || ldx < n || ldphi < k || ldc < k)
    return fail(LRFSI_EINVAL, "lrfsi_pod: bad argument (1 <= k <= n, ldx >= n, ldphi, ldc >= k)");
  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<lrfsi_subset_s> S(new (std::nothrow) lrfsi_subset_s());
  if (!S) return fail(LRFSI_ENOMEM, "lrfsi_pod: host allocation");
  S->mesh = mesh;
  S->K = 1;
  S->M = mesh->h.M;
  S->m = {n};
  S->cap = {k};
  S->off = {0};
  S->mtot = n;
  S->mmax = n;
  S->Rmax = k;
  LRFSI_TRY(subset_alloc_ws(S.get(), s));
  const long M = S->M;
  const int ldP = S->ldP, ldR = S->ldR;
  std::vector<CopyDesc> cd;
  cd.push_back(CopyDesc{X, ldx, S->Xcat.p, ldP, M, n, 0, nullptr, 1.0});
  cd.push_back(CopyDesc{nullptr, 0, S->Vcat.p, ldP, n, n, 2, nullptr, 1.0});
  LRFSI_TRY(copy_batched(cd, s));
  std::vector<int> act{0}, p{n}, rank;
  std::vector<double*> Uo{S->UR.p}, Vo{S->VR.p};
  std::vector<double> f2;
  LRFSI_TRY(truncate_batch(S.get(), act, p, 0.0, S->cap, Uo, Vo, rank, f2, s));
  // below the numerical rank the basis and coefficients are zero-filled
  const int kr = rank[0] < k ? rank[0] : k;
  cd.clear();
  if (kr > 0) {
    cd.push_back(CopyDesc{S->UR.p, ldR, Phi, ldphi, M, kr, 0, nullptr, 1.0});
    cd.push_back(CopyDesc{S->VR.p, ldR, C, ldc, n, kr, 0, nullptr, 1.0});
  }
  if (kr < k) {
    cd.push_back(CopyDesc{nullptr, 0, Phi + kr, ldphi, M, k - kr, 1, nullptr, 0.0});
    cd.push_back(CopyDesc{nullptr, 0, C + kr, ldc, n, k - kr, 1, nullptr, 0.0});
  }
  LRFSI_TRY(copy_batched(cd, s));
  if (sigma) {
    std::vector<double> sv(k, 0.0);
    if (kr > 0) LRFSI_CUDA(cudaMemcpyAsync(sv.data(), S->sv.p, sizeof(double) * kr, cudaMemcpyDeviceToHost, s));
    LRFSI_CUDA(cudaStreamSynchronize(s));
    std::memcpy(sigma, sv.data(), sizeof(double) * k);
  }
  LRFSI_CUDA(cudaStreamSynchronize(s));
  return LRFSI_OK;
}
