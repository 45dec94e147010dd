// FP64 Gram products on the BF16 tensor cores (tcgen05) by error-free
// splitting; see ozaki.h for the method.
//
// Layout of the slices in the workspace (per operand of a product): the rows
// are cut into chunks of 16 (one K step of a BF16 MMA), the columns into
// tiles of 128.  For chunk c, column tile T and slice t the 128 x 16 block is
// stored in the no-swizzle K-major canonical layout of tcgen05 operands:
// core matrices of 8 columns x 8 rows (16 bytes per column), the core
// matrix of column group g and row group k at byte g * 256 + k * 128.  The
// 8 slices of (c, T) are contiguous (32 KB), so the A operand of a chunk is
// one bulk copy; a B operand of 32 columns is the quarter of a block (1 KB).
//
// Kernels:
//   k_oz_exp    largest biased exponent of every column (atomicMax)
//   k_oz_split  the 8 digit slices of every entry, in the layout above
//   k_oz_gram   one CTA per (product, 128 x 32 output tile, row split):
//               4-stage bulk-copy pipeline, 36 MMAs per 16-row chunk into 8
//               level accumulators (tensor memory, double buffered per
//               256-row window), integer read-out by 8 warps into int32
//               sums, added to the tile's int64 level totals (atomics)
//   k_oz_reduce combines the 8 int64 level totals of an entry in FP64
#include <cuda_bf16.h>

#include <atomic>

#include "ozaki.h"

namespace lrfsi {

namespace {
constexpr int kSl = 8;            // slices per entry
constexpr int kLv = 8;            // levels t + u = 0 .. 7 (0-based slices)
constexpr int kChunk = 16;        // rows per chunk (K of one MMA)
constexpr int kWin = 256;         // rows per exact accumulation window
constexpr int kChunksPerWin = kWin / kChunk;
constexpr int kTA = 128;          // output rows per tile (MMA M)
constexpr int kTB = 32;           // output columns per tile (MMA N)
constexpr int kStages = 4;
constexpr int kABytes = kTA * kChunk * 2 * kSl;   // 32 KB: A operand of a chunk, all slices
constexpr int kBBytes = kTB * kChunk * 2 * kSl;   // 8 KB
constexpr int kStageBytes = kABytes + kBBytes;
constexpr int kGramThreads = 288;  // 8 read-out warps + 1 issuing warp
constexpr int kMaxWinPerSplit = 128;  // int32 read-out sums stay below 2^31
constexpr int kMaxOz = 16;        // products per launch

std::atomic<int> g_gram_path{1};
int* g_oz_err = nullptr;  // set by a pipeline wait of k_oz_gram that ran out

__host__ __device__ inline long ceil_div_l(long a, long b) { return (a + b - 1) / b; }
}  // namespace

int gram_path() { return g_gram_path.load(); }
void set_gram_path(int p) { g_gram_path.store(p ? 1 : 0); }

// ---------------------------------------------------------------------------
// PTX helpers (tcgen05, bulk copies, mbarriers)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t sm_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sm_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sm_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sm_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(sm_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of the given parity, at most ~2^31 clock cycles (about a
// second); false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity))
    if (clock64() - t0 > (1LL << 31)) return false;
  return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   sm_addr(dst)),
               "l"(src), "r"(bytes), "r"(sm_addr(bar))
               : "memory");
}
// shared-memory matrix descriptor: no swizzle, K-major canonical layout;
// lbo = byte distance of core matrices along K, sbo = along M / N
__device__ __forceinline__ uint64_t sm_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 D, M x N
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dt),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sm_addr(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's tensor-memory lane, loaded and
// waited for in one statement (the registers are valid only after
// tcgen05.wait::ld)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
}

// v 2^e: within the normal exponent range one multiplication by the power of
// two built from its IEEE-754 exponent field (exact, or rounded once where the
// product is subnormal: the same result as ldexp); ldexp outside it
__device__ __forceinline__ double oz_scale2(double v, int e) {
  if (e >= -1022 && e <= 1023) return v * __longlong_as_double((long long)(e + 1023) << 52);
  return ldexp(v, e);
}

// ---------------------------------------------------------------------------
// Launch parameters
// ---------------------------------------------------------------------------
// One operand (A or B of a product): its columns, slices and exponents.
struct OzOp {
  const double* X;   // rows x n: entry (l, i) at X[l * rs + i * cs]
  long rs, cs;
  long rows;         // rows (the contraction length) and
  long nch;          // 16-row chunks of slices written (zeros beyond rows)
  const int* lsc;    // optional per-row scale: entry (l, i) is taken times
  int lsign;         // 2^(lsign (lsc[l] - 1022)); lsc[l] == 0: the row is zero
  const double* Xalt;  // read instead of X when sel != nullptr && *sel != 0
  const int* sel;
  int n;             // columns
  int nt;            // 128-column tiles
  __nv_bfloat16* sl; // slices: nchunks x nt x 8 x 2048
  int* ex;           // nt * 128 biased exponents (max over the column; 0: zero column)
  Gate gate;
  int q;             // >= 0: the gate is the launch's gate q instead (descriptors on the device)
};
struct OzOps {
  OzOp op[2 * kMaxOz];
  int cnt;
};
// One product for the MMA and reduction kernels.
struct OzProd {
  int a, b;          // operand indices (b == a: symmetric, upper tiles only)
  int tiles;         // output tiles computed
  int ntb;           // 32-column tiles of B
  int first;         // first CTA (tile-major, split-minor) of this product
  unsigned long long* acc;  // tiles x kLv x kTB x kTA int64 level sums (two's complement)
  double* G;
  int ldg, p, q;
  Gate gate;
};
struct OzProds {
  OzProd pr[kMaxOz];
  OzOp op[2 * kMaxOz];
  int cnt;
  int nsplit;        // row splits per tile
  int wins;          // 256-row windows of the whole M
};

__device__ __forceinline__ void oz_tile_of(const OzProd& P, int t, int& ta, int& tb) {
  // symmetric: the tiles (ta, tb) with tb * 32 + 31 >= ta * 128, row by row;
  // otherwise all na x ntb tiles
  if (P.a == P.b) {
    int r = t;
    ta = 0;
    for (;;) {
      const int first_tb = (ta * kTA) / kTB;
      const int in_row = P.ntb - first_tb;
      if (r < in_row) { tb = first_tb + r; return; }
      r -= in_row;
      ++ta;
    }
  }
  ta = t / P.ntb;
  tb = t % P.ntb;
}

// ---------------------------------------------------------------------------
// Column exponents and digit slices
// ---------------------------------------------------------------------------
constexpr int kExpRows = 64;

// ex[i] = largest biased exponent field over column i < n (2047 if the column
// holds an Inf or NaN); ex must be zeroed first.  CTA (row block, 256 columns).
__device__ __forceinline__ void oz_exp_cols(const OzOp& op, int n) {
  const double* X = (op.sel && *op.sel) ? op.Xalt : op.X;
  const long rows = op.rows;
  const long r0 = (long)blockIdx.x * kExpRows, r1 = r0 + kExpRows < rows ? r0 + kExpRows : rows;
  const int i = blockIdx.y * 256 + threadIdx.x;
  if (i >= n) return;
  int mx = 0;
  for (long l = r0; l < r1; ++l) {
    int be = (int)((__double_as_longlong(X[l * op.rs + i * op.cs]) >> 52) & 0x7FF);
    if (op.lsc && be != 0 && be != 0x7FF) {
      const int ls = op.lsc[l];
      be = ls == 0 ? 0 : be + op.lsign * (ls - 1022);
      be = be < 1 ? 0 : (be > 0x7FE ? 0x7FE : be);
    }
    mx = be > mx ? be : mx;
  }
  if (mx) atomicMax(op.ex + i, mx);
}
__global__ void __launch_bounds__(256) k_oz_exp(const __grid_constant__ OzOps O, long M) {
  const OzOp& op = O.op[blockIdx.z];
  (void)M;
  if (!gate_open(op.gate)) return;
  oz_exp_cols(op, op.n);
}

// The 8 balanced base-128 digits of x as a 56-bit fixed-point number in units
// of 2^(e - 56), e = bexp_max - 1022 (so |x| < 2^e): a[0] in [-128, 128],
// a[1..7] in [-64, 63], x = sum_t a[t] 2^(e - 7 (t + 1)) up to 2^(e - 57).
__device__ __forceinline__ void oz_digits(double x, int bexp_max, int shift, int (&a)[kSl]) {
  const long long bits = __double_as_longlong(x);
  const int be = (int)((bits >> 52) & 0x7FF);
  long long v = 0;
  if (be != 0 && be != 0x7FF && bexp_max != 0x7FF) {
    const long long mant = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
    const int sh = be + shift - 1019 - (bexp_max - 1022);  // v = mant 2^sh, sh <= 3
    if (sh >= 0) v = mant << sh;
    else if (sh > -62) v = (mant + (1LL << (-sh - 1))) >> (-sh);
    if (bits < 0) v = -v;
  }
#pragma unroll
  for (int t = kSl - 1; t >= 1; --t) {
    const long long d = ((v + 64) & 127) - 64;
    a[t] = (int)d;
    v = (v - d) >> 7;
  }
  a[0] = (int)v;
}

// CTA = (16-row chunk, group of two 128-column tiles): every (column, 8-row
// half) item writes 16 bytes (8 rows of one column) of each slice; n columns
// in opnt tiles of 128 (columns >= n are zero).
__device__ __forceinline__ void oz_split_cols(const OzOp& op, int n, int opnt) {
  const double* X = (op.sel && *op.sel) ? op.Xalt : op.X;
  const long c = blockIdx.x;
  const int t0 = blockIdx.y * 2, nt = opnt - t0 < 2 ? opnt - t0 : 2;
  const long M = op.rows;
  if (nt <= 0 || c >= op.nch) return;
  const int items = nt * kTA * 2;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int i = t0 * kTA + it % (nt * kTA), kg = it / (nt * kTA);
    const int ti = i / kTA, il = i % kTA;
    const int bx = i < n ? op.ex[i] : 0;
    int dig[8][kSl];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const long l = c * kChunk + kg * 8 + e;
      double x = (i < n && l < M) ? X[l * op.rs + (long)i * op.cs] : 0.0;
      int shift = 0;
      if (op.lsc && l < M) {
        const int ls = op.lsc[l];
        if (ls == 0) x = 0.0;
        else shift = op.lsign * (ls - 1022);
      }
      oz_digits(x, bx, shift, dig[e]);
    }
    __nv_bfloat16* base = op.sl + ((size_t)(c * opnt + ti) * kSl) * (kTA * kChunk) + (il >> 3) * 128 + kg * 64 +
                          (il & 7) * 8;
#pragma unroll
    for (int t = 0; t < kSl; ++t) {
      __align__(16) __nv_bfloat16 v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = __float2bfloat16_rn((float)dig[e][t]);
      *reinterpret_cast<uint4*>(base + (size_t)t * (kTA * kChunk)) = *reinterpret_cast<const uint4*>(v);
    }
  }
}
__global__ void __launch_bounds__(256) k_oz_split(const __grid_constant__ OzOps O, long M) {
  const OzOp& op = O.op[blockIdx.z];
  (void)M;
  if (!gate_open(op.gate)) return;
  oz_split_cols(op, op.n, op.nt);
}

// ---------------------------------------------------------------------------
// Slice products on the tensor cores
// ---------------------------------------------------------------------------
// CTA = (product, output tile of 128 rows x 32 columns, row split).  Warp 8
// lane 0 issues the bulk copies and the MMAs; warps 0-7 read the level sums
// out of tensor memory after every 256-row window (warp w reads lanes
// 32 (w % 4) .. +31 and levels 4 (w / 4) .. +3) and keep them as int32.
// Tensor memory: 2 buffers x 8 levels x 32 FP32 columns = 512 columns.
__global__ void __launch_bounds__(kGramThreads, 1) k_oz_gram(const __grid_constant__ OzProds P, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], win[2], freeb[2], fin;
  __shared__ uint32_t s_tmem;
  const int cta = blockIdx.x;
  int pi = 0;
  while (pi + 1 < P.cnt && cta >= P.pr[pi + 1].first) ++pi;
  const OzProd& pr = P.pr[pi];
  if (!gate_open(pr.gate)) return;  // uniform over the CTA, before any barrier or allocation
  const int local = cta - pr.first;
  const int tile = local / P.nsplit, split = local % P.nsplit;
  int ta, tb;
  oz_tile_of(pr, tile, ta, tb);
  const OzOp& A = P.op[pr.a];
  const OzOp& B = P.op[pr.b];
  const int w0 = (int)((long)P.wins * split / P.nsplit), w1 = (int)((long)P.wins * (split + 1) / P.nsplit);
  const int nwin = w1 - w0, nch = nwin * kChunksPerWin;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&win[b], 1);
      mbar_init(&freeb[b], 8);
    }
    mbar_init(&fin, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(sm_addr(&s_tmem))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  int acc[4][32];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[k][j] = 0;

  if (warp == 8) {
    if (lane == 0) {
      constexpr uint32_t idesc = mma_idesc(kTA, kTB);
      const size_t cbase = (size_t)w0 * kChunksPerWin;
      auto load = [&](int c) {
        const int st = c % kStages;
        unsigned char* sa = smem + (size_t)st * kStageBytes;
        unsigned char* sb = sa + kABytes;
        const size_t cc = cbase + c;
        const __nv_bfloat16* ga = A.sl + (cc * A.nt + ta) * kSl * (kTA * kChunk);
        const __nv_bfloat16* gb = B.sl + (cc * B.nt + tb / 4) * kSl * (kTA * kChunk) + (tb % 4) * (kTB * kChunk);
        mbar_expect_tx(&full[st], kStageBytes);
        bulk_g2s(sa, ga, kABytes, &full[st]);
        for (int t = 0; t < kSl; ++t) bulk_g2s(sb + t * (kTB * kChunk * 2), gb + t * (kTA * kChunk), kTB * kChunk * 2, &full[st]);
      };
      int issued = 0, consumed = 0;
      for (; issued < nch && issued < kStages; ++issued) load(issued);
      bool ok = true;
      for (int c = 0; c < nch && ok; ++c) {
        const int st = c % kStages;
        if (!mbar_wait(&full[st], (uint32_t)(c / kStages) & 1)) { ok = false; break; }
        consumed = c + 1;
        const int w = c / kChunksPerWin, buf = w & 1;
        const bool first = (c % kChunksPerWin) == 0;
        if (first && w >= 2 && !mbar_wait(&freeb[buf], (uint32_t)((w - 2) >> 1) & 1)) { ok = false; break; }
        tc_fence_after();
        const uint32_t sa = sm_addr(smem + (size_t)st * kStageBytes), sb = sa + kABytes;
        // descriptors of slice 0; slice t starts t * 4 KB (A) / 1 KB (B) later,
        // i.e. t * 256 / t * 64 in the address field (smem addresses < 2^18)
        const uint64_t a0 = sm_desc(sa, 128, 256), b0 = sm_desc(sb, 128, 256);
        const uint32_t d0 = tmem + (uint32_t)(buf * (kLv * kTB));
        const uint32_t acc0 = first ? 0u : 1u;
#pragma unroll
        for (int lv = 0; lv < kLv; ++lv) {
#pragma unroll
          for (int t = 0; t <= lv; ++t)
            mma_bf16(d0 + lv * kTB, a0 + (uint64_t)(t * ((kTA * kChunk * 2) >> 4)),
                     b0 + (uint64_t)((lv - t) * ((kTB * kChunk * 2) >> 4)), idesc, t == 0 ? acc0 : 1u);
        }
        mma_commit(&empty[st]);
        if (c % kChunksPerWin == kChunksPerWin - 1) mma_commit(&win[buf]);
        if (c >= 1 && issued < nch) {  // refill the stage of chunk c - 1 once its MMAs are done
          const int ps = (c - 1) % kStages;
          if (!mbar_wait(&empty[ps], (uint32_t)((c - 1) / kStages) & 1)) { ok = false; break; }
          load(issued++);
        }
      }
      if (!ok) atomicExch(err, 1);
      // every MMA of this thread done, every issued copy landed, before the
      // tensor memory and the shared memory are released
      mma_commit(&fin);
      mbar_wait(&fin, 0);
      for (int c = consumed; c < issued; ++c) mbar_wait(&full[c % kStages], (uint32_t)(c / kStages) & 1);
    }
  } else {
    const int q = warp & 3, h = warp >> 2;
    for (int w = 0; w < nwin; ++w) {
      const int buf = w & 1;
      // one lane waits, the warp follows its result (tcgen05.ld is warp-aligned)
      int ok = 1;
      if (lane == 0) ok = mbar_wait(&win[buf], (uint32_t)(w >> 1) & 1) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) atomicExch(err, 1);
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * (kLv * kTB) + (4 * h + k) * kTB), v);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[k][j] += __float2int_rn(__uint_as_float(v[j]));
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&freeb[buf]);
    }
    // add this split's level sums into the tile's int64 totals
    // [tile][level][column][row] (integer adds: the order does not matter)
    unsigned long long* out = pr.acc + (size_t)tile * (kLv * kTB * kTA) + 32 * q + lane;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (acc[k][j]) atomicAdd(out + ((size_t)(4 * h + k) * kTB + j) * kTA, (unsigned long long)(long long)acc[k][j]);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// G[i][j] from the int64 level totals of its tile: the 8 levels combined in
// FP64 with the column scales.
__global__ void __launch_bounds__(256) k_oz_reduce(const __grid_constant__ OzProds P) {
  const OzProd& pr = P.pr[blockIdx.y];
  if (!gate_open(pr.gate)) return;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)pr.p * pr.q) return;
  const int i0 = (int)(e % pr.p), j0 = (int)(e / pr.p);
  int i = i0, j = j0;
  const bool sym = pr.a == pr.b;
  if (sym && (j / kTB) * kTB + kTB - 1 < (i / kTA) * kTA) { const int t = i; i = j; j = t; }
  const int ta = i / kTA, tb = j / kTB;
  int tile;
  if (sym) {
    tile = 0;
    for (int r = 0; r < ta; ++r) tile += pr.ntb - (r * kTA) / kTB;
    tile += tb - (ta * kTA) / kTB;
  } else {
    tile = ta * pr.ntb + tb;
  }
  const int ea = P.op[pr.a].ex[i], eb = P.op[pr.b].ex[j];
  double g;
  if (ea == 0x7FF || eb == 0x7FF) {
    g = __longlong_as_double(0x7FF8000000000000LL);
  } else {
    long long S[kLv];
#pragma unroll
    for (int lv = 0; lv < kLv; ++lv) S[lv] = 0;
    const unsigned long long* src = pr.acc + (size_t)tile * (kLv * kTB * kTA) + (j % kTB) * kTA + (i % kTA);
#pragma unroll
    for (int lv = 0; lv < kLv; ++lv) S[lv] = (long long)src[(size_t)lv * (kTB * kTA)];
    // x = sum_t a_t 2^(e - 7 (t + 1)), e = ex - 1022: level lv scales by 2^(ea + eb - 7 (lv + 2))
    const int sc = (ea ? ea - 1022 : 0) + (eb ? eb - 1022 : 0);
    g = 0.0;
#pragma unroll
    for (int lv = kLv - 1; lv >= 0; --lv) g += oz_scale2((double)S[lv], sc - 7 * (lv + 2));
  }
  pr.G[(size_t)i0 * pr.ldg + j0] = g;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {
struct OzPlan {
  int nsplit = 1, wins = 0;
  long nchunks = 0;
  size_t ex_bytes = 0, sl_bytes = 0, part_bytes = 0;
  size_t total() const { return ex_bytes + sl_bytes + part_bytes; }
};
inline size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }
inline int sym_tiles(int p) {
  const int nta = (int)ceil_div_l(p, kTA), ntb = (int)ceil_div_l(p, kTB);
  int t = 0;
  for (int r = 0; r < nta; ++r) t += ntb - (r * kTA) / kTB;
  return t;
}
// the split count for T output tiles: about two CTAs per SM, windows of a
// split at most kMaxWinPerSplit
inline int choose_nsplit(long T, int wins) {
  // whole waves of one CTA per SM (152 SMs), windows of a split at most
  // kMaxWinPerSplit
  long ns = (2L * 152) / (T > 0 ? T : 1);
  const long lo = (wins + kMaxWinPerSplit - 1) / kMaxWinPerSplit;
  if (ns < lo) ns = lo;
  if (ns > wins) ns = wins;
  if (ns < 1) ns = 1;
  return (int)ns;
}
// layout for cnt products: nops operands of nt_op tiles each and T tiles in total
OzPlan plan_for(long M, int nops, long sum_nt, long T) {
  OzPlan pl;
  pl.wins = (int)ceil_div_l(M, kWin);
  pl.nchunks = (long)pl.wins * kChunksPerWin;
  pl.nsplit = choose_nsplit(T, pl.wins);
  pl.ex_bytes = round256(sizeof(int) * (size_t)sum_nt * kTA);
  pl.sl_bytes = round256((size_t)pl.nchunks * sum_nt * kSl * kTA * kChunk * 2);
  pl.part_bytes = round256(sizeof(unsigned long long) * (size_t)T * kLv * kTB * kTA);
  (void)nops;
  return pl;
}
}  // namespace

// exponents and slices of every operand of a launch
static int oz_exp(const OzOps& ops, cudaStream_t s) {
  int nmax = 1;
  long rmax = 1;
  for (int o = 0; o < ops.cnt; ++o) {
    nmax = ops.op[o].n > nmax ? ops.op[o].n : nmax;
    rmax = ops.op[o].rows > rmax ? ops.op[o].rows : rmax;
  }
  k_oz_exp<<<dim3((unsigned)ceil_div_l(rmax, kExpRows), (unsigned)ceil_div_l(nmax, 256), ops.cnt), 256, 0, s>>>(ops,
                                                                                                          rmax);
  return check_launch("k_oz_exp");
}
// exponents and slices of every operand of a launch
static int oz_slice(const OzOps& ops, cudaStream_t s) {
  LRFSI_TRY(oz_exp(ops, s));
  int ntmax = 1;
  long rmax = 1, cmax = 1;
  for (int o = 0; o < ops.cnt; ++o) {
    ntmax = ops.op[o].nt > ntmax ? ops.op[o].nt : ntmax;
    rmax = ops.op[o].rows > rmax ? ops.op[o].rows : rmax;
    cmax = ops.op[o].nch > cmax ? ops.op[o].nch : cmax;
  }
  k_oz_split<<<dim3((unsigned)cmax, (unsigned)ceil_div_l(ntmax, 2), ops.cnt), 256, 0, s>>>(ops, rmax);
  return check_launch("k_oz_split");
}

// products per launch are limited by kMaxOz and by a workspace budget of
// 1 GiB (a single product may exceed it)
constexpr size_t kOzBudget = (size_t)1 << 30;

size_t ozaki_work_bytes(int nbatch, long M, int pmax, int qmax) {
  if (nbatch <= 0 || M <= 0) return 0;
  const long nta = ceil_div_l(pmax, kTA), ntq = ceil_div_l(qmax, kTA), ntb = ceil_div_l(qmax, kTB);
  // worst case per product: unsymmetric (two operands, all tiles)
  auto need = [&](int cnt) { return plan_for(M, 2 * cnt, (long)cnt * (nta + ntq), (long)cnt * nta * ntb).total(); };
  int cnt = nbatch < kMaxOz ? nbatch : kMaxOz;
  while (cnt > 1 && need(cnt) > kOzBudget) --cnt;
  return need(cnt) + 1024;
}

int ozaki_gram(const GramDesc* d, int nbatch, long M, void* work, size_t work_bytes, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    LRFSI_CUDA(cudaFuncSetAttribute(k_oz_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, kStages * kStageBytes));
    attr = true;
  }
  if (!g_oz_err) {
    LRFSI_CUDA(cudaMalloc(&g_oz_err, sizeof(int)));
    LRFSI_CUDA(cudaMemset(g_oz_err, 0, sizeof(int)));
  }
  for (int base = 0; base < nbatch;) {
    // the largest group of products from base that fits the workspace
    int cnt = 0;
    {
      long snt = 0, tt = 0;
      int nop = 0;
      while (base + cnt < nbatch && cnt < kMaxOz) {
        const GramDesc& g = d[base + cnt];
        const bool sym = g.A == g.B && g.lda == g.ldb && g.p == g.q;
        const long nt = ceil_div_l(g.p, kTA) + (sym ? 0 : ceil_div_l(g.q, kTA));
        const long tl = sym ? sym_tiles(g.p) : ceil_div_l(g.p, kTA) * ceil_div_l(g.q, kTB);
        if (cnt > 0 && plan_for(M, nop + (sym ? 1 : 2), snt + nt, tt + tl).total() > work_bytes) break;
        snt += nt;
        tt += tl;
        nop += sym ? 1 : 2;
        ++cnt;
      }
    }
    OzOps ops{};
    OzProds P{};
    P.cnt = cnt;
    long sum_nt = 0, T = 0;
    for (int b = 0; b < cnt; ++b) {
      const GramDesc& g = d[base + b];
      const bool sym = g.A == g.B && g.lda == g.ldb && g.p == g.q;
      OzProd& pr = P.pr[b];
      pr.a = ops.cnt;
      OzOp& oa = ops.op[ops.cnt++];
      oa.X = g.A; oa.rs = g.lda; oa.cs = 1; oa.rows = M; oa.nch = (long)ceil_div_l(M, kWin) * kChunksPerWin; oa.n = g.p; oa.nt = (int)ceil_div_l(g.p, kTA); oa.gate = g.gate;
      sum_nt += oa.nt;
      if (sym) {
        pr.b = pr.a;
      } else {
        pr.b = ops.cnt;
        OzOp& ob = ops.op[ops.cnt++];
        ob.X = g.B; ob.rs = g.ldb; ob.cs = 1; ob.rows = M; ob.nch = (long)ceil_div_l(M, kWin) * kChunksPerWin; ob.n = g.q; ob.nt = (int)ceil_div_l(g.q, kTA); ob.gate = g.gate;
        sum_nt += ob.nt;
      }
      pr.ntb = (int)ceil_div_l(g.q, kTB);
      pr.tiles = sym ? sym_tiles(g.p) : (int)ceil_div_l(g.p, kTA) * pr.ntb;
      pr.G = g.G; pr.ldg = g.ldg; pr.p = g.p; pr.q = g.q; pr.gate = g.gate;
      T += pr.tiles;
    }
    const OzPlan pl = plan_for(M, ops.cnt, sum_nt, T);
    if (pl.total() > work_bytes) return fail(LRFSI_EINVAL, "tensor-core Gram: workspace too small");
    unsigned char* w = (unsigned char*)work;
    int* ex = (int*)w;
    __nv_bfloat16* sl = (__nv_bfloat16*)(w + pl.ex_bytes);
    unsigned long long* part = (unsigned long long*)(w + pl.ex_bytes + pl.sl_bytes);
    size_t o_ex = 0, o_sl = 0;
    for (int o = 0; o < ops.cnt; ++o) {
      ops.op[o].ex = ex + o_ex;
      ops.op[o].sl = sl + o_sl;
      o_ex += (size_t)ops.op[o].nt * kTA;
      o_sl += (size_t)pl.nchunks * ops.op[o].nt * kSl * kTA * kChunk;
    }
    size_t o_part = 0;
    int first = 0;
    for (int b = 0; b < cnt; ++b) {
      P.pr[b].acc = part + o_part;
      P.pr[b].first = first;
      o_part += (size_t)P.pr[b].tiles * kLv * kTB * kTA;
      first += P.pr[b].tiles * pl.nsplit;
    }
    for (int o = 0; o < ops.cnt; ++o) P.op[o] = ops.op[o];
    P.nsplit = pl.nsplit;
    P.wins = pl.wins;
    {  // algorithmic FP64 work, as the FP64 Gram kernels count it
      double fl = 0, by = 0;
      for (int b = 0; b < cnt; ++b) {
        const GramDesc& g = d[base + b];
        if (!gate_counts(g.gate, s)) continue;
        const bool sym = P.pr[b].a == P.pr[b].b;
        fl += sym ? 1.0 * M * g.p * (g.p + 1) : 2.0 * M * g.p * g.q;
        by += 8.0 * M * (sym ? g.p : g.p + g.q);
      }
      account(KC_GRAM_TC, fl, by);
    }
    TimedLaunch tl(KC_GRAM_TC, s);
    LRFSI_CUDA(cudaMemsetAsync(ex, 0, pl.ex_bytes, s));
    LRFSI_CUDA(cudaMemsetAsync(part, 0, pl.part_bytes, s));
    LRFSI_TRY(oz_slice(ops, s));
    if (first > 0) {
      double mf = 0, mb = 0;  // BF16 MMA work actually issued (36 slice products per chunk and tile)
      for (int b = 0; b < cnt; ++b)
        if (gate_counts(P.pr[b].gate, s)) {
          mf += (double)P.pr[b].tiles * pl.wins * kChunksPerWin * 36.0 * 2.0 * kTA * kTB * kChunk;
          mb += (double)P.pr[b].tiles * pl.wins * kChunksPerWin * kStageBytes;
        }
      account(KC_TCMMA, mf, mb);
      TimedLaunch tm(KC_TCMMA, s);
      k_oz_gram<<<first, kGramThreads, kStages * kStageBytes, s>>>(P, g_oz_err);
      LRFSI_TRY(check_launch("k_oz_gram"));
      tm.end(s);
    }
    long pq = 1;
    for (int b = 0; b < cnt; ++b) pq = std::max(pq, (long)P.pr[b].p * P.pr[b].q);
    k_oz_reduce<<<dim3((unsigned)ceil_div_l(pq, 256), cnt), 256, 0, s>>>(P);
    LRFSI_TRY(check_launch("k_oz_reduce"));
    tl.end(s);
    base += cnt;
  }
  return LRFSI_OK;
}

int ozaki_error(cudaStream_t s, int* flag) {
  *flag = 0;
  if (!g_oz_err) return LRFSI_OK;
  LRFSI_CUDA(cudaMemcpyAsync(flag, g_oz_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  LRFSI_CUDA(cudaStreamSynchronize(s));
  if (*flag) LRFSI_CUDA(cudaMemsetAsync(g_oz_err, 0, sizeof(int), s));
  return LRFSI_OK;
}

}  // namespace lrfsi

extern "C" int lrfsi_gram_path(int path, int* previous) {
  using namespace lrfsi;
  if (path < -1 || path > 1) return fail(LRFSI_EINVAL, "lrfsi_gram_path: path must be 0, 1 (or -1 to query)");
  const int old = gram_path();
  if (path >= 0) set_gram_path(path);
  if (previous) *previous = old;
  return LRFSI_OK;
}

extern "C" int lrfsi_gram(const double* A, int lda, int p, const double* B, int ldb, int q, int64_t M, double* G,
                          int ldg, lrfsi_stream_t stream) {
  using namespace lrfsi;
  if (!A || !B || !G || M < 1 || p < 1 || q < 1 || lda < p || ldb < q || ldg < q)
    return fail(LRFSI_EINVAL, "lrfsi_gram: bad argument (M, p, q >= 1, lda >= p, ldb >= q, ldg >= q)");
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf<double> work;
  LRFSI_TRY(work.alloc(gram_work_len(1, (long)M, p, q)));
  GramDesc g{A, lda, p, B, ldb, q, G, ldg};
  LRFSI_TRY(gram_batched(&g, 1, (long)M, work.p, work.n, s));
  int flag = 0;
  LRFSI_TRY(ozaki_error(s, &flag));
  if (flag) return fail(LRFSI_ENOCONV, "lrfsi_gram: a pipeline wait of the tensor-core Gram ran out");
  return LRFSI_OK;
}

extern "C" int lrfsi_svd_cluster(int size, int* previous) {
  using namespace lrfsi;
  if (!(size == -1 || size == 0 || size == 2 || size == 4 || size == 8 || size == 16))
    return fail(LRFSI_EINVAL, "lrfsi_svd_cluster: size must be 0, 2, 4, 8 or 16 (or -1 to query)");
  const int old = svd_cluster(size);
  if (previous) *previous = old;
  return LRFSI_OK;
}

// ---------------------------------------------------------------------------
// Tall FP64 GEMMs C = alpha A B + beta C on the tensor cores (contraction
// K <= kOzMaxK: one exact window).  A is sliced by rows (A^T as the operand,
// one exponent per row of A over K), B by columns; the 8 levels of an entry
// are combined as two exact int64 groups (levels 0-3 and 4-7, each below
// 2^45.1) and one FP64 fma.  Used for the products whose left factor has
// orthonormal or comparable columns (the caller marks them, GemmDesc::tc):
// there the error follows |A| |B| like that of an FP64 GEMM.
// ---------------------------------------------------------------------------
namespace lrfsi {
namespace {
constexpr int kOzMaxK = 400;      // level sums over <= 409 rows stay below 2^24
constexpr int kGStages = 2;
constexpr int kGThreads = 288;
struct OzG {
  int a, b;          // operand indices: a = A^T (rows K, columns = rows of A), b = B
  int m, n, k;
  int ntn;           // 32-column tiles of C
  int first;         // first CTA (row tile major)
  double* C;
  long c_rs, c_cs;
  double alpha, beta;
  Gate gate;
};
struct OzGs {
  OzG g[kMaxOz];
  OzOp op[2 * kMaxOz];
  int cnt;
};
}  // namespace

// 8 consecutive FP32 columns of this thread's lane at 4 column offsets (4
// levels), loaded and waited for in one statement (the registers are valid
// only after tcgen05.wait::ld)
__device__ __forceinline__ void tmem_ld8x4(uint32_t t0, uint32_t t1, uint32_t t2, uint32_t t3,
                                           uint32_t (&v)[4][8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%32];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%33];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%34];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24,%25,%26,%27,%28,%29,%30,%31}, [%35];\n\t"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(v[0][0]), "=r"(v[0][1]), "=r"(v[0][2]), "=r"(v[0][3]), "=r"(v[0][4]), "=r"(v[0][5]), "=r"(v[0][6]),
        "=r"(v[0][7]), "=r"(v[1][0]), "=r"(v[1][1]), "=r"(v[1][2]), "=r"(v[1][3]), "=r"(v[1][4]), "=r"(v[1][5]),
        "=r"(v[1][6]), "=r"(v[1][7]), "=r"(v[2][0]), "=r"(v[2][1]), "=r"(v[2][2]), "=r"(v[2][3]), "=r"(v[2][4]),
        "=r"(v[2][5]), "=r"(v[2][6]), "=r"(v[2][7]), "=r"(v[3][0]), "=r"(v[3][1]), "=r"(v[3][2]), "=r"(v[3][3]),
        "=r"(v[3][4]), "=r"(v[3][5]), "=r"(v[3][6]), "=r"(v[3][7])
      : "r"(t0), "r"(t1), "r"(t2), "r"(t3)
      : "memory");
}

// One 128 x 32 tile (ta, tb) of C = alpha A B + beta C (m x n, contraction
// k <= kOzMaxK) from the slices of A^T (asl: nch x ant x 8 x 2048, row
// exponents aex) and of B (bsl: nch x bnt x 8 x 2048, column exponents bex).
// Warp 8 lane 0 issues the bulk copies and the 36 MMAs per 16-row chunk of K
// into 8 level accumulators (256 tensor-memory columns); warps 0-7 read all 8
// levels of 8 columns at a time (warp w: lanes 32 (w % 4) .., columns
// 16 (w / 4) ..) and write C.  Called by all kGThreads threads of the CTA,
// which must not have returned before.
template <int STAGES>
__device__ __forceinline__ void oz_gemm_tile(const __nv_bfloat16* __restrict__ asl, int ant, const int* __restrict__ aex,
                                             const __nv_bfloat16* __restrict__ bsl, int bnt,
                                             const int* __restrict__ bex, int m, int n, int k, int ta, int tb,
                                             double* C, long c_rs, long c_cs, double alpha, double beta, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done, fin;
  __shared__ uint32_t s_tmem;
  const int nch = (k + kChunk - 1) / kChunk;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    mbar_init(&fin, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(sm_addr(&s_tmem))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  if (warp == 8) {
    if (lane == 0) {
      constexpr uint32_t idesc = mma_idesc(kTA, kTB);
      auto load = [&](int c) {
        const int st = c % STAGES;
        unsigned char* sa = smem + (size_t)st * kStageBytes;
        unsigned char* sb = sa + kABytes;
        const __nv_bfloat16* ga = asl + ((size_t)c * ant + ta) * kSl * (kTA * kChunk);
        const __nv_bfloat16* gb = bsl + ((size_t)c * bnt + tb / 4) * kSl * (kTA * kChunk) + (tb % 4) * (kTB * kChunk);
        mbar_expect_tx(&full[st], kStageBytes);
        bulk_g2s(sa, ga, kABytes, &full[st]);
        for (int u = 0; u < kSl; ++u) bulk_g2s(sb + u * (kTB * kChunk * 2), gb + u * (kTA * kChunk), kTB * kChunk * 2, &full[st]);
      };
      int issued = 0, consumed = 0;
      for (; issued < nch && issued < STAGES; ++issued) load(issued);
      bool ok = true;
      for (int c = 0; c < nch && ok; ++c) {
        const int st = c % STAGES;
        if (!mbar_wait(&full[st], (uint32_t)(c / STAGES) & 1)) { ok = false; break; }
        consumed = c + 1;
        tc_fence_after();
        const uint32_t sa = sm_addr(smem + (size_t)st * kStageBytes), sb = sa + kABytes;
        const uint64_t a0 = sm_desc(sa, 128, 256), b0 = sm_desc(sb, 128, 256);
        const uint32_t acc0 = c == 0 ? 0u : 1u;
#pragma unroll
        for (int lv = 0; lv < kLv; ++lv) {
#pragma unroll
          for (int u = 0; u <= lv; ++u)
            mma_bf16(tmem + lv * kTB, a0 + (uint64_t)(u * ((kTA * kChunk * 2) >> 4)),
                     b0 + (uint64_t)((lv - u) * ((kTB * kChunk * 2) >> 4)), idesc, u == 0 ? acc0 : 1u);
        }
        mma_commit(&empty[st]);
        if (c == nch - 1) mma_commit(&done);
        if (c >= 1 && issued < nch) {
          const int ps = (c - 1) % STAGES;
          if (!mbar_wait(&empty[ps], (uint32_t)((c - 1) / STAGES) & 1)) { ok = false; break; }
          load(issued++);
        }
      }
      if (!ok) atomicExch(err, 1);
      mma_commit(&fin);
      mbar_wait(&fin, 0);
      for (int c = consumed; c < issued; ++c) mbar_wait(&full[c % STAGES], (uint32_t)(c / STAGES) & 1);
    }
  } else {
    const int q = warp & 3, h = warp >> 2;
    int ok = 1;
    if (lane == 0) ok = mbar_wait(&done, 0) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) {
      if (lane == 0) atomicExch(err, 1);
    } else {
      tc_fence_after();
      const int i = ta * kTA + 32 * q + lane;
      const int ea = i < m ? aex[i] : 0;
#pragma unroll 1
      for (int half = 0; half < 2; ++half) {
        const int jc = 16 * h + 8 * half;  // first column of these 8 in the tile
        uint32_t v[kLv][8];
        const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)jc;
        tmem_ld8x4(tl, tl + kTB, tl + 2 * kTB, tl + 3 * kTB, *reinterpret_cast<uint32_t(*)[4][8]>(&v[0][0]));
        tmem_ld8x4(tl + 4 * kTB, tl + 5 * kTB, tl + 6 * kTB, tl + 7 * kTB,
                   *reinterpret_cast<uint32_t(*)[4][8]>(&v[4][0]));
        if (i < m) {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const int j = tb * kTB + jc + jj;
            if (j >= n) continue;
            const int eb = bex[j];
            double val;
            if (ea == 0x7FF || eb == 0x7FF) {
              val = __longlong_as_double(0x7FF8000000000000LL);
            } else {
              long long Hs = 0, Ls = 0;
#pragma unroll
              for (int lv = 0; lv < 4; ++lv) Hs = Hs * 128 + __float2int_rn(__uint_as_float(v[lv][jj]));
#pragma unroll
              for (int lv = 4; lv < 8; ++lv) Ls = Ls * 128 + __float2int_rn(__uint_as_float(v[lv][jj]));
              const int sc = (ea ? ea - 1022 : 0) + (eb ? eb - 1022 : 0);
              val = oz_scale2(fma((double)Ls, 0x1p-28, (double)Hs), sc - 35);
            }
            double* cp = C + (size_t)i * c_rs + (size_t)j * c_cs;
            *cp = beta != 0.0 ? fma(alpha, val, beta * *cp) : alpha * val;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
  }
}

// CTA = (GEMM, 128 x 32 tile of C).
__global__ void __launch_bounds__(kGThreads) k_oz_gemm(const __grid_constant__ OzGs P, int* err) {
  const int cta = blockIdx.x;
  int gi = 0;
  while (gi + 1 < P.cnt && cta >= P.g[gi + 1].first) ++gi;
  const OzG& G = P.g[gi];
  if (!gate_open(G.gate)) return;  // uniform over the CTA, before any barrier or allocation
  const int t = cta - G.first, ta = t / G.ntn, tb = t % G.ntn;
  const OzOp& A = P.op[G.a];
  const OzOp& B = P.op[G.b];
  oz_gemm_tile<kGStages>(A.sl, A.nt, A.ex, B.sl, B.nt, B.ex, G.m, G.n, G.k, ta, tb, G.C, G.c_rs, G.c_cs, G.alpha,
                         G.beta, err);
}

bool ozaki_gemm_eligible(const GemmDesc<double>& g) {
  return gram_path() == 1 && g.tc && g.m >= 2048 && g.k >= 1 && g.k <= kOzMaxK && g.n >= 1;
}

namespace {
// bytes of the operands of GEMMs d[0..cnt) (exponents + slices), 256-aligned pieces
size_t gemm_ops_bytes(const GemmDesc<double>* d, int cnt) {
  size_t b = 0;
  for (int i = 0; i < cnt; ++i) {
    const long nch = ceil_div_l(d[i].k, kChunk);
    const long nta = ceil_div_l(d[i].m, kTA), ntb = ceil_div_l(d[i].n, kTA);
    b += round256(sizeof(int) * ((size_t)(nta + ntb) * kTA + d[i].k));
    b += round256((size_t)nch * nta * kSl * kTA * kChunk * 2) + round256((size_t)nch * ntb * kSl * kTA * kChunk * 2);
  }
  return b;
}
}  // namespace

size_t ozaki_gemm_work_bytes(const GemmDesc<double>* d, int n) {
  size_t mx = 0;
  for (int base = 0; base < n; base += kMaxOz) {
    const int cnt = n - base < kMaxOz ? n - base : kMaxOz;
    const size_t b = gemm_ops_bytes(d + base, cnt);
    mx = b > mx ? b : mx;
  }
  return mx + 1024;
}

int ozaki_gemm(const GemmDesc<double>* d, int n, void* work, size_t work_bytes, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    LRFSI_CUDA(cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kGStages * kStageBytes));
    attr = true;
  }
  if (!g_oz_err) {
    LRFSI_CUDA(cudaMalloc(&g_oz_err, sizeof(int)));
    LRFSI_CUDA(cudaMemset(g_oz_err, 0, sizeof(int)));
  }
  for (int base = 0; base < n; base += kMaxOz) {
    const int cnt = n - base < kMaxOz ? n - base : kMaxOz;
    if (gemm_ops_bytes(d + base, cnt) > work_bytes) return fail(LRFSI_EINVAL, "tensor-core GEMM: workspace too small");
    OzOps ops{}, eops{};
    OzGs P{};
    P.cnt = cnt;
    unsigned char* w = (unsigned char*)work;
    size_t off = 0;
    int first = 0;
    for (int b = 0; b < cnt; ++b) {
      const GemmDesc<double>& g = d[base + b];
      const long nch = ceil_div_l(g.k, kChunk);
      // the contraction index is equilibrated: column k of A is scaled by a
      // power of two to a largest entry in [1/2, 1), row k of B by the inverse
      OzOp& oe = eops.op[eops.cnt++];
      oe.X = g.A; oe.Xalt = g.A_alt; oe.sel = g.sel; oe.rs = g.a_rs; oe.cs = g.a_cs; oe.rows = g.m; oe.nch = 0;
      oe.n = g.k; oe.nt = 0; oe.gate = g.gate;
      OzOp& oa = ops.op[ops.cnt];
      oa.X = g.A; oa.Xalt = g.A_alt; oa.sel = g.sel; oa.rs = g.a_cs; oa.cs = g.a_rs; oa.rows = g.k; oa.nch = nch;
      oa.n = g.m; oa.nt = (int)ceil_div_l(g.m, kTA); oa.gate = g.gate;
      OzOp& ob = ops.op[ops.cnt + 1];
      ob.X = g.B; ob.rs = g.b_rs; ob.cs = g.b_cs; ob.rows = g.k; ob.nch = nch;
      ob.n = g.n; ob.nt = (int)ceil_div_l(g.n, kTA); ob.gate = g.gate;
      oe.ex = (int*)(w + off);
      oa.ex = oe.ex + g.k;
      ob.ex = oa.ex + (size_t)oa.nt * kTA;
      oa.lsc = ob.lsc = oe.ex;
      oa.lsign = -1;
      ob.lsign = 1;
      LRFSI_CUDA(cudaMemsetAsync(oe.ex, 0, sizeof(int) * ((size_t)(oa.nt + ob.nt) * kTA + g.k), s));
      off += round256(sizeof(int) * ((size_t)(oa.nt + ob.nt) * kTA + g.k));
      oa.sl = (__nv_bfloat16*)(w + off);
      off += round256((size_t)nch * oa.nt * kSl * kTA * kChunk * 2);
      ob.sl = (__nv_bfloat16*)(w + off);
      off += round256((size_t)nch * ob.nt * kSl * kTA * kChunk * 2);
      OzG& G = P.g[b];
      G.a = ops.cnt; G.b = ops.cnt + 1;
      ops.cnt += 2;
      G.m = g.m; G.n = g.n; G.k = g.k;
      G.ntn = (int)ceil_div_l(g.n, kTB);
      G.first = first;
      first += (int)ceil_div_l(g.m, kTA) * G.ntn;
      G.C = g.C; G.c_rs = g.c_rs; G.c_cs = g.c_cs; G.alpha = g.alpha; G.beta = g.beta; G.gate = g.gate;
    }
    for (int o = 0; o < ops.cnt; ++o) P.op[o] = ops.op[o];
    LRFSI_TRY(oz_exp(eops, s));   // column maxima of A (the contraction scales)
    LRFSI_TRY(oz_slice(ops, s));
    if (first > 0) {
      double mf = 0, mb = 0;  // BF16 MMA work actually issued
      for (int b = 0; b < cnt; ++b) {
        const GemmDesc<double>& g = d[base + b];
        if (!gate_counts(g.gate, s)) continue;
        const double tiles = (double)ceil_div_l(g.m, kTA) * ceil_div_l(g.n, kTB), nch = (double)ceil_div_l(g.k, kChunk);
        mf += tiles * nch * 36.0 * 2.0 * kTA * kTB * kChunk;
        mb += tiles * nch * kStageBytes;
      }
      account(KC_TCMMA, mf, mb);
      TimedLaunch tm(KC_TCMMA, s);
      k_oz_gemm<<<first, kGThreads, kGStages * kStageBytes, s>>>(P, g_oz_err);
      LRFSI_TRY(check_launch("k_oz_gemm"));
      tm.end(s);
    }
  }
  return LRFSI_OK;
}

// ---------------------------------------------------------------------------
// GEMMs with fixed left operands (OzFixedPlan)
// ---------------------------------------------------------------------------
namespace {
// One GEMM of a group: the A^T operand (slices made by slice()) and the B
// operand (sliced at every call, n = the call's columns), both with the
// contraction scales of A.
struct OzNdG {
  OzOp A, B;
  double* C;
  long c_rs;
  int m, k;
  double alpha, beta;
};
constexpr int kGridZ = 65535;
}  // namespace

// exponents / slices of the device-resident operands ops[0 .. cnt)
__global__ void __launch_bounds__(256) k_oz_exp_d(const OzOp* __restrict__ ops, int cnt) {
  for (int z = blockIdx.z; z < cnt; z += gridDim.z) oz_exp_cols(ops[z], ops[z].n);
}
__global__ void __launch_bounds__(256) k_oz_split_d(const OzOp* __restrict__ ops, int cnt) {
  for (int z = blockIdx.z; z < cnt; z += gridDim.z) oz_split_cols(ops[z], ops[z].n, ops[z].nt);
}
// The B operands of a group with ncols columns (gated per problem).  CTA =
// (128-column tile, GEMM), 512 threads: the exponents of its columns over the
// k rows (scaled by the contraction scales; 4 row groups reduced in shared
// memory), then the 8 slices of the 16-row chunks, two chunks at a time (one
// (column, 8-row half) item per thread and chunk).
constexpr int kBsThreads = 512;
__global__ void __launch_bounds__(kBsThreads) k_oz_bslice(const OzNdG* __restrict__ ds, int cnt, int ncols,
                                                          const __grid_constant__ OzGates G) {
  __shared__ int s_ex[kBsThreads / kTA][kTA];
  constexpr int kRowGroups = kBsThreads / kTA;
  const int ti = blockIdx.x, opnt = (int)ceil_div_l(ncols, kTA);
  const int il = threadIdx.x & (kTA - 1), grp = threadIdx.x >> 7;
  const int half = grp & 1, csub = grp >> 1;  // chunk phase: 8-row half, chunk of the pair
  const int i = ti * kTA + il;
  for (int z = blockIdx.z; z < cnt; z += gridDim.z) {
    const OzOp& op = ds[z].B;
    if (!gate_open(G.g[op.q])) continue;  // uniform over the CTA
    const double* X = op.X;
    const long k = op.rows;
    int mx = 0;
    if (i < ncols) {
#pragma unroll 4
      for (long l = grp; l < k; l += kRowGroups) {
        int be = (int)((__double_as_longlong(X[l * op.rs + i]) >> 52) & 0x7FF);
        if (be != 0 && be != 0x7FF) {
          const int ls = op.lsc[l];
          be = ls == 0 ? 0 : be + (ls - 1022);
          be = be < 1 ? 0 : (be > 0x7FE ? 0x7FE : be);
        }
        mx = be > mx ? be : mx;
      }
    }
    s_ex[grp][il] = mx;
    __syncthreads();
    int bx = 0;
#pragma unroll
    for (int g = 0; g < kRowGroups; ++g) bx = max(bx, s_ex[g][il]);
    if (grp == 0 && i < ncols) op.ex[i] = bx;
    for (long c = csub; c < op.nch; c += 2) {
      int dig[8][kSl];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const long l = c * kChunk + half * 8 + e;
        double x = 0.0;
        int shift = 0;
        if (i < ncols && l < k) {
          const int ls = op.lsc[l];
          if (ls != 0) {
            x = X[l * op.rs + i];
            shift = ls - 1022;
          }
        }
        oz_digits(x, bx, shift, dig[e]);
      }
      __nv_bfloat16* base = op.sl + ((size_t)(c * opnt + ti) * kSl) * (kTA * kChunk) + (il >> 3) * 128 + half * 64 +
                            (il & 7) * 8;
#pragma unroll
      for (int t = 0; t < kSl; ++t) {
        __align__(16) __nv_bfloat16 v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = __float2bfloat16_rn((float)dig[e][t]);
        *reinterpret_cast<uint4*>(base + (size_t)t * (kTA * kChunk)) = *reinterpret_cast<const uint4*>(v);
      }
    }
    __syncthreads();  // s_ex is rewritten by the next GEMM of this CTA
  }
}

// CTA = (32-column tile, 128-row tile, GEMM); STAGES pipeline stages (4 for
// long contractions: fewer CTAs, each with more copies in flight)
template <int STAGES>
__global__ void __launch_bounds__(kGThreads) k_oz_ndgemm(const OzNdG* __restrict__ ds, int ncols,
                                                         const __grid_constant__ OzGates G, int* err) {
  const OzNdG* d = ds + blockIdx.z;
  const int ta = blockIdx.y, tb = blockIdx.x;
  // uniform over the CTA, before any barrier or allocation
  if (ta >= d->A.nt || tb * kTB >= ncols || !gate_open(G.g[d->A.q])) return;
  oz_gemm_tile<STAGES>(d->A.sl, d->A.nt, d->A.ex, d->B.sl, (int)ceil_div_l(ncols, kTA), d->B.ex, d->m, ncols, d->k, ta, tb,
               d->C, d->c_rs, 1, d->alpha, d->beta, err);
}

bool ozaki_fixed_eligible(int m, int k) {
  return gram_path() == 1 && k >= 16 && k <= kOzMaxK && m >= 32 && (long)m * k >= 2048;
}

int OzFixedPlan::add_group(const std::vector<OzFixedGemm>& g) {
  Group G;
  G.gemms = g;
  groups_.push_back(std::move(G));
  return (int)groups_.size() - 1;
}

namespace {
// byte layout of an OzFixedPlan (dry run when base == nullptr)
struct FixedLayout {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off = round256(off + bytes);
    return o;
  }
};
inline size_t a_slice_bytes(int m, int k) {
  return (size_t)ceil_div_l(k, kChunk) * ceil_div_l(m, kTA) * kSl * kTA * kChunk * sizeof(__nv_bfloat16);
}
inline size_t a_exp_ints(int m, int k) { return (size_t)k + (size_t)ceil_div_l(m, kTA) * kTA; }
}  // namespace

size_t OzFixedPlan::bytes_needed(int max_cols) const {
  const int ntb = (int)ceil_div_l(max_cols, kTA);
  FixedLayout L;
  size_t total = 0, bex = 0, bsl = 0, aex = 0, asl = 0;
  for (const Group& G : groups_) {
    L.take(sizeof(OzNdG) * G.gemms.size());
    total += G.gemms.size();
    size_t be = 0, bs = 0;
    for (const OzFixedGemm& g : G.gemms) {
      be += (size_t)ntb * kTA;
      bs += round256((size_t)ceil_div_l(g.k, kChunk) * ntb * kSl * kTA * kChunk * sizeof(__nv_bfloat16));
      aex += a_exp_ints(g.m, g.k);
      asl += round256(a_slice_bytes(g.m, g.k));
    }
    bex = std::max(bex, be);
    bsl = std::max(bsl, bs);
  }
  L.take(sizeof(OzOp) * total);
  L.take(sizeof(OzOp) * total);
  L.take(sizeof(int) * aex);
  L.take(asl);
  L.take(sizeof(int) * bex);
  L.take(bsl);
  return L.off;
}

int OzFixedPlan::build(int max_cols, int nprob) {
  if (max_cols < 1 || nprob < 1 || nprob > kMaxGemmDescs) return fail(LRFSI_EINVAL, "tensor GEMM plan: bad sizes");
  nprob_ = nprob;
  max_cols_ = max_cols;
  // kernel attributes and the error flag, here and not in gemm(): gemm() may
  // run inside a stream capture
  {
    static bool attr = false;
    if (!attr) {
      LRFSI_CUDA(cudaFuncSetAttribute(k_oz_ndgemm<kGStages>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kGStages * kStageBytes));
      LRFSI_CUDA(cudaFuncSetAttribute(k_oz_ndgemm<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * kStageBytes));
      attr = true;
    }
    if (!g_oz_err) {
      LRFSI_CUDA(cudaMalloc(&g_oz_err, sizeof(int)));
      LRFSI_CUDA(cudaMemset(g_oz_err, 0, sizeof(int)));
    }
  }
  const int ntb = (int)ceil_div_l(max_cols, kTA);
  LRFSI_TRY(buf_.alloc(bytes_needed(max_cols)));
  unsigned char* base = buf_.p;
  FixedLayout L;
  size_t total = 0;
  for (Group& G : groups_) {
    G.d_off = L.take(sizeof(OzNdG) * G.gemms.size());
    total += G.gemms.size();
  }
  e_off_ = L.take(sizeof(OzOp) * total);
  a_off_ = L.take(sizeof(OzOp) * total);
  // slicing order: problem-major (prefixes of problems), groups in order within
  std::vector<std::pair<int, int>> order;  // (group, index)
  sl_prefix_.assign(nprob + 1, 0);
  for (int q = 0; q < nprob; ++q) {
    for (int gi = 0; gi < (int)groups_.size(); ++gi)
      for (int i = 0; i < (int)groups_[gi].gemms.size(); ++i)
        if (groups_[gi].gemms[i].q == q) order.push_back({gi, i});
    sl_prefix_[q + 1] = (int)order.size();
  }
  if (order.size() != total) return fail(LRFSI_EINVAL, "tensor GEMM plan: a problem index outside [0, nprob)");
  size_t aex_ints = 0, asl_bytes = 0;
  for (auto& o : order) {
    const OzFixedGemm& g = groups_[o.first].gemms[o.second];
    aex_ints += a_exp_ints(g.m, g.k);
    asl_bytes += round256(a_slice_bytes(g.m, g.k));
  }
  aex_off_ = L.take(sizeof(int) * aex_ints);
  const size_t asl_off = L.take(asl_bytes);
  size_t bex_max = 0, bsl_max = 0;
  for (Group& G : groups_) {
    size_t be = 0, bs = 0;
    for (const OzFixedGemm& g : G.gemms) {
      be += (size_t)ntb * kTA;
      bs += round256((size_t)ceil_div_l(g.k, kChunk) * ntb * kSl * kTA * kChunk * sizeof(__nv_bfloat16));
    }
    bex_max = std::max(bex_max, be);
    bsl_max = std::max(bsl_max, bs);
  }
  bex_off_ = L.take(sizeof(int) * bex_max);
  bsl_off_ = L.take(bsl_max);
  if (L.off > buf_.bytes()) return fail(LRFSI_EINVAL, "tensor GEMM plan: layout exceeds its buffer");
  // A operands in slicing order
  std::vector<OzOp> E(total), A(total);
  std::vector<std::vector<OzOp>> Aof(groups_.size());
  for (size_t gi = 0; gi < groups_.size(); ++gi) Aof[gi].resize(groups_[gi].gemms.size());
  aex_prefix_.assign(nprob + 1, 0);
  int* aex = (int*)(base + aex_off_);
  unsigned char* asl = base + asl_off;
  size_t ie = 0, is = 0;
  sl_rows_max_ = sl_n_max_ = sl_nch_max_ = sl_nt_max_ = 1;
  for (int q = 0, j = 0; q < nprob; ++q) {
    for (; j < sl_prefix_[q + 1]; ++j) {
      const OzFixedGemm& g = groups_[order[j].first].gemms[order[j].second];
      OzOp e{}, a{};
      e.X = g.A; e.rs = g.lda; e.cs = 1; e.rows = g.m; e.n = g.k; e.ex = aex + ie; e.q = -1;
      a.X = g.A; a.rs = 1; a.cs = g.lda; a.rows = g.k; a.nch = ceil_div_l(g.k, kChunk);
      a.lsc = aex + ie; a.lsign = -1; a.n = g.m; a.nt = (int)ceil_div_l(g.m, kTA);
      a.ex = aex + ie + g.k; a.sl = (__nv_bfloat16*)(asl + is); a.q = -1;
      ie += a_exp_ints(g.m, g.k);
      is += round256(a_slice_bytes(g.m, g.k));
      E[j] = e;
      A[j] = a;
      Aof[order[j].first][order[j].second] = a;
      sl_rows_max_ = std::max(sl_rows_max_, std::max(g.m, g.k));
      sl_n_max_ = std::max(sl_n_max_, std::max(g.m, g.k));
      sl_nch_max_ = std::max(sl_nch_max_, (int)a.nch);
      sl_nt_max_ = std::max(sl_nt_max_, a.nt);
    }
    aex_prefix_[q + 1] = sizeof(int) * ie;
  }
  LRFSI_CUDA(cudaMemcpy(base + e_off_, E.data(), sizeof(OzOp) * total, cudaMemcpyHostToDevice));
  LRFSI_CUDA(cudaMemcpy(base + a_off_, A.data(), sizeof(OzOp) * total, cudaMemcpyHostToDevice));
  // group descriptors; every group's B operands reuse the same workspace
  for (size_t gi = 0; gi < groups_.size(); ++gi) {
    Group& G = groups_[gi];
    std::vector<OzNdG> d(G.gemms.size());
    G.prefix.assign(nprob + 1, 0);
    size_t be = 0, bs = 0;
    for (size_t i = 0; i < G.gemms.size(); ++i) {
      const OzFixedGemm& g = G.gemms[i];
      if (i > 0 && g.q < G.gemms[i - 1].q) return fail(LRFSI_EINVAL, "tensor GEMM plan: a group not ordered by problem");
      OzNdG& x = d[i];
      x.A = Aof[gi][i];
      x.A.q = g.q;
      x.B = OzOp{};
      x.B.X = g.B; x.B.rs = g.ldb; x.B.cs = 1; x.B.rows = g.k; x.B.nch = ceil_div_l(g.k, kChunk);
      x.B.lsc = x.A.lsc; x.B.lsign = 1; x.B.n = max_cols; x.B.nt = ntb; x.B.q = g.q;
      x.B.ex = (int*)(base + bex_off_) + be;
      x.B.sl = (__nv_bfloat16*)(base + bsl_off_ + bs);
      be += (size_t)ntb * kTA;
      bs += round256((size_t)ceil_div_l(g.k, kChunk) * ntb * kSl * kTA * kChunk * sizeof(__nv_bfloat16));
      x.C = g.C; x.c_rs = g.ldc; x.m = g.m; x.k = g.k; x.alpha = g.alpha; x.beta = g.beta;
      G.mmax = std::max(G.mmax, g.m);
      G.kmax = std::max(G.kmax, g.k);
      G.ntmax = std::max(G.ntmax, x.A.nt);
      for (int q = g.q + 1; q <= nprob; ++q) G.prefix[q] = (int)i + 1;
    }
    if (!d.empty()) LRFSI_CUDA(cudaMemcpy(base + G.d_off, d.data(), sizeof(OzNdG) * d.size(), cudaMemcpyHostToDevice));
  }
  return LRFSI_OK;
}

int OzFixedPlan::slice(int nprob, cudaStream_t s) const {
  if (!buf_.p || nprob < 1) return LRFSI_OK;
  if (nprob > nprob_) return fail(LRFSI_EINVAL, "tensor GEMM plan: more problems than built");
  const int cnt = sl_prefix_[nprob];
  if (!cnt) return LRFSI_OK;
  const OzOp* E = (const OzOp*)(buf_.p + e_off_);
  const OzOp* A = (const OzOp*)(buf_.p + a_off_);
  const unsigned gz = (unsigned)std::min(cnt, kGridZ);
  LRFSI_CUDA(cudaMemsetAsync(buf_.p + aex_off_, 0, aex_prefix_[nprob], s));
  // contraction scales (column maxima of A), then the row exponents and slices of A^T
  k_oz_exp_d<<<dim3((unsigned)ceil_div_l(sl_rows_max_, kExpRows), (unsigned)ceil_div_l(sl_n_max_, 256), gz), 256, 0,
               s>>>(E, cnt);
  LRFSI_TRY(check_launch("k_oz_exp_d"));
  k_oz_exp_d<<<dim3((unsigned)ceil_div_l(sl_rows_max_, kExpRows), (unsigned)ceil_div_l(sl_n_max_, 256), gz), 256, 0,
               s>>>(A, cnt);
  LRFSI_TRY(check_launch("k_oz_exp_d"));
  k_oz_split_d<<<dim3((unsigned)sl_nch_max_, (unsigned)ceil_div_l(sl_nt_max_, 2), gz), 256, 0, s>>>(A, cnt);
  LRFSI_TRY(check_launch("k_oz_split_d"));
  return LRFSI_OK;
}

int OzFixedPlan::gemm(int gi, int ncols, int nprob, const OzGates& gates, cudaStream_t s) const {
  if (empty(gi) || ncols < 1 || nprob < 1) return LRFSI_OK;
  if (!buf_.p || ncols > max_cols_ || nprob > nprob_ || !g_oz_err)
    return fail(LRFSI_EINVAL, "tensor GEMM plan: call beyond its build");
  const Group& G = groups_[gi];
  const int cnt = G.prefix[nprob];
  if (!cnt) return LRFSI_OK;
  const OzNdG* d = (const OzNdG*)(buf_.p + G.d_off);
  {  // algorithmic FP64 work and the BF16 MMA work issued, for the live problems
    bool live[kMaxGemmDescs];
    for (int q = 0; q < nprob; ++q) live[q] = gate_counts(gates.g[q], s);
    double fl = 0, by = 0, mf = 0, mb = 0;
    for (int i = 0; i < cnt; ++i) {
      const OzFixedGemm& g = G.gemms[i];
      if (!live[g.q]) continue;
      fl += 2.0 * g.m * g.k * ncols;
      by += 8.0 * ((double)g.m * g.k + (double)g.k * ncols + (g.beta != 0.0 ? 2.0 : 1.0) * g.m * ncols);
      const double tiles = (double)ceil_div_l(g.m, kTA) * ceil_div_l(ncols, kTB), nch = (double)ceil_div_l(g.k, kChunk);
      mf += tiles * nch * 36.0 * 2.0 * kTA * kTB * kChunk;
      mb += tiles * nch * kStageBytes;
    }
    account(KC_GEMM_TC, fl, by);
    account(KC_TCMMA, mf, mb);
  }
  TimedLaunch tl(KC_GEMM_TC, s);
  const unsigned gz = (unsigned)std::min(cnt, kGridZ);
  k_oz_bslice<<<dim3((unsigned)ceil_div_l(ncols, kTA), 1, gz), kBsThreads, 0, s>>>(d, cnt, ncols, gates);
  LRFSI_TRY(check_launch("k_oz_bslice"));
  TimedLaunch tm(KC_TCMMA, s);
  const bool deep = G.kmax >= 8 * kChunk;
  for (int z0 = 0; z0 < cnt; z0 += kGridZ) {
    const int z = std::min(kGridZ, cnt - z0);
    const dim3 grid((unsigned)ceil_div_l(ncols, kTB), (unsigned)G.ntmax, (unsigned)z);
    if (deep)
      k_oz_ndgemm<4><<<grid, kGThreads, 4 * kStageBytes, s>>>(d + z0, ncols, gates, g_oz_err);
    else
      k_oz_ndgemm<kGStages><<<grid, kGThreads, kGStages * kStageBytes, s>>>(d + z0, ncols, gates, g_oz_err);
    LRFSI_TRY(check_launch("k_oz_ndgemm"));
  }
  tm.end(s);
  tl.end(s);
  return LRFSI_OK;
}
}  // namespace lrfsi

extern "C" int lrfsi_gemm(int m, int n, int k, const double* A, int lda, const double* B, int ldb, double* C, int ldc,
                          double alpha, double beta, int tensor, lrfsi_stream_t stream) {
  using namespace lrfsi;
  if (!A || !B || !C || m < 1 || n < 1 || k < 1 || lda < k || ldb < n || ldc < n)
    return fail(LRFSI_EINVAL, "lrfsi_gemm: bad argument (m, n, k >= 1, lda >= k, ldb >= n, ldc >= n)");
  cudaStream_t s = (cudaStream_t)stream;
  GemmDesc<double> g{m, n, k, A, lda, 1, B, ldb, 1, C, ldc, 1, alpha, beta};
  g.tc = tensor ? 1 : 0;
  LRFSI_TRY(gemm_grouped<double>(&g, 1, s));
  int flag = 0;
  LRFSI_TRY(ozaki_error(s, &flag));
  if (flag) return fail(LRFSI_ENOCONV, "lrfsi_gemm: a pipeline wait of the tensor-core GEMM ran out");
  return LRFSI_OK;
}
