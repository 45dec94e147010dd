// Algorithm 1's parameter bookkeeping (host code, no device work): the
// little-endian order of a parameter grid (Sec. 3.3, Def. 1), the order of an
// unstructured parameter set, the clustering into K contiguous subsets
// (Eq. (clustering1)), the upper median of every subset (Sec. 3.3, Def.
// "Upper Median Index"), and the split of the subsets over processes (Sec. 2:
// the K subsets are independent, so whole subsets go to one process each).
#include <algorithm>
#include <numeric>
#include <vector>

#include "common.h"
#include "lrfsi.h"

using namespace lrfsi;

extern "C" int lrfsi_order_grid(int m1, int m2, const double* mu_values_host, const double* nu_values_host,
                                int nu_fastest, double* mu_out_host, double* nu_out_host) {
  if (m1 < 1 || m2 < 1 || !mu_values_host || !nu_values_host || !mu_out_host || !nu_out_host)
    return fail(LRFSI_EINVAL, "lrfsi_order_grid: need m1, m2 >= 1 and non-null arrays");
  // Def. 1: (i1, i2) -> position i1 + (i2 - 1) m1 (1-based): the mu index runs
  // fastest.  nu_fastest swaps the roles (the cut of a two-subset split then
  // runs along mu).
  for (int i2 = 0; i2 < m2; ++i2)
    for (int i1 = 0; i1 < m1; ++i1) {
      const long p = nu_fastest ? (long)i1 * m2 + i2 : (long)i2 * m1 + i1;
      mu_out_host[p] = mu_values_host[i1];
      nu_out_host[p] = nu_values_host[i2];
    }
  return LRFSI_OK;
}

extern "C" int lrfsi_order_set(int m, const double* mu_host, const double* nu_host, int32_t* perm_host) {
  if (m < 0 || (m > 0 && (!mu_host || !nu_host || !perm_host)))
    return fail(LRFSI_EINVAL, "lrfsi_order_set: bad argument");
  for (int i = 0; i < m; ++i)
    if (!(mu_host[i] == mu_host[i]) || !(nu_host[i] == nu_host[i]))
      return fail(LRFSI_EINVAL, "lrfsi_order_set: NaN parameter");
  std::vector<int32_t> p(m);
  std::iota(p.begin(), p.end(), 0);
  // the grids' little-endian order carried over to a scattered set: sorted by
  // nu_f, then by mu_s (mu fastest); ties keep the input order
  std::stable_sort(p.begin(), p.end(), [&](int32_t a, int32_t b) {
    if (nu_host[a] != nu_host[b]) return nu_host[a] < nu_host[b];
    return mu_host[a] < mu_host[b];
  });
  std::copy(p.begin(), p.end(), perm_host);
  return LRFSI_OK;
}

extern "C" int lrfsi_cluster(int m, int K, int32_t* sizes_host, int32_t* offsets_host, int32_t* medians_host) {
  if (K < 1 || m < K || !sizes_host)
    return fail(LRFSI_EINVAL, "lrfsi_cluster: need 1 <= K <= m and a sizes array");
  // Eq. (clustering1): |I_k| = floor(m / K) for k < K, the remainder for k = K
  const int base = m / K;
  int off = 0;
  for (int k = 0; k < K; ++k) {
    const int sz = k < K - 1 ? base : m - (K - 1) * base;
    sizes_host[k] = sz;
    if (offsets_host) offsets_host[k] = off;
    // upper median: 1-based position floor(n / 2) + 1 of the ordered subset
    if (medians_host) medians_host[k] = off + sz / 2;
    off += sz;
  }
  return LRFSI_OK;
}

extern "C" int lrfsi_medians(int K, const int32_t* sizes_host, int32_t* offsets_host, int32_t* medians_host) {
  if (K < 1 || !sizes_host || !medians_host) return fail(LRFSI_EINVAL, "lrfsi_medians: bad argument");
  int off = 0;
  for (int k = 0; k < K; ++k) {
    if (sizes_host[k] < 1) return fail(LRFSI_EINVAL, "lrfsi_medians: empty subset");
    if (offsets_host) offsets_host[k] = off;
    medians_host[k] = off + sizes_host[k] / 2;
    off += sizes_host[k];
  }
  return LRFSI_OK;
}

extern "C" int lrfsi_partition(int K, const int64_t* weights_host, int nproc, int32_t* first_host) {
  if (K < 0 || nproc < 1 || (K > 0 && !weights_host) || !first_host)
    return fail(LRFSI_EINVAL, "lrfsi_partition: bad argument");
  for (int k = 0; k < K; ++k)
    if (weights_host[k] < 0) return fail(LRFSI_EINVAL, "lrfsi_partition: negative weight");
  // contiguous blocks minimising the largest block weight: binary search on
  // that bound with a greedy fill (a block is closed when the next subset
  // would exceed the bound), then the blocks are spread so that no process is
  // left empty while another holds more than one subset
  auto blocks_for = [&](int64_t cap) {
    int n = 1;
    int64_t s = 0;
    for (int k = 0; k < K; ++k) {
      if (s + weights_host[k] > cap && s > 0) {
        ++n;
        s = 0;
      }
      s += weights_host[k];
    }
    return n;
  };
  int64_t lo = 0, hi = 0;
  for (int k = 0; k < K; ++k) {
    lo = std::max(lo, weights_host[k]);
    hi += weights_host[k];
  }
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (blocks_for(mid) <= nproc) hi = mid;
    else lo = mid + 1;
  }
  // greedy fill at the optimal bound, keeping enough subsets for the
  // processes still to come
  int k = 0;
  for (int p = 0; p < nproc; ++p) {
    first_host[p] = k;
    int64_t s = 0;
    const int left_after = nproc - p - 1;
    while (k < K && (K - k) > left_after && (s == 0 || s + weights_host[k] <= lo)) {
      s += weights_host[k];
      ++k;
    }
  }
  first_host[nproc] = K;
  return LRFSI_OK;
}
