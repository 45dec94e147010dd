// Mesh / DOF layout (host) and FP64 finite element assembly kernels.
//
// Weak form: Sec. 2, Eq. (fsi_problem_weak1) of the paper (stationary
// Navier-Stokes in F, the paper's nonlinear solid stress in S, harmonic
// deformation extension in F); Jacobians of Sec. 3.1; affine split of
// Sec. 3, Eq. (pardep_matrix1).  Q2 velocity/deformation, Q1 pressure,
// 3 x 3 Gauss points per cell.
//
// DOF order ("slab-major"): slab s < nx holds the Q2 node columns 2s, 2s+1
// and the Q1 vertex column s; the last slab holds node column 2 nx and vertex
// column nx.  Inside a slab: node columns in order, nodes bottom to top, four
// unknowns (v_x, v_y, u_x, u_y) per node, then the slab's pressures.  A Q2
// cell couples node columns 2c..2c+2, so every operator is block tridiagonal
// over slabs.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "mesh.h"

namespace lrfsi {

namespace {

struct Tables {
  double N[9][kNq];
  double dN[9][kNq][2];  // physical gradients
  double P[4][kNq];
  double w[kNq];         // physical weights
  double rho, lam;
};

void make_tables(double hx, double hy, double rho, double lam, Tables& T) {
  const double g[3] = {0.5 - 0.5 * std::sqrt(0.6), 0.5, 0.5 + 0.5 * std::sqrt(0.6)};
  const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  auto L = [](int k, double t) { return k == 0 ? (2 * t - 1) * (t - 1) : k == 1 ? 4 * t * (1 - t) : t * (2 * t - 1); };
  auto dL = [](int k, double t) { return k == 0 ? 4 * t - 3 : k == 1 ? 4 - 8 * t : 4 * t - 1; };
  auto L1 = [](int k, double t) { return k == 0 ? 1 - t : t; };
  for (int qy = 0; qy < 3; ++qy)
    for (int qx = 0; qx < 3; ++qx) {
      int q = qx + 3 * qy;
      double tx = g[qx], ty = g[qy];
      T.w[q] = gw[qx] * gw[qy] * hx * hy;
      for (int ay = 0; ay < 3; ++ay)
        for (int ax = 0; ax < 3; ++ax) {
          int a = ax + 3 * ay;
          T.N[a][q] = L(ax, tx) * L(ay, ty);
          T.dN[a][q][0] = dL(ax, tx) * L(ay, ty) / hx;
          T.dN[a][q][1] = L(ax, tx) * dL(ay, ty) / hy;
        }
      for (int by = 0; by < 2; ++by)
        for (int bx = 0; bx < 2; ++bx) T.P[bx + 2 * by][q] = L1(bx, tx) * L1(by, ty);
    }
  T.rho = rho;
  T.lam = lam;
}

}  // namespace

int build_mesh(const lrfsi_problem& p, MeshHost& h) {
  if (p.nx < 1 || p.ny < 1 || !(p.Lx > 0) || !(p.Ly > 0))
    return fail(LRFSI_EINVAL, "lrfsi_mesh_create: need nx, ny >= 1 and positive lengths");
  if ((long)p.nx * p.ny > 4000000) return fail(LRFSI_EINVAL, "lrfsi_mesh_create: mesh too large");
  h.prob = p;
  const int nx = p.nx, ny = p.ny;
  h.nx = nx; h.ny = ny; h.nnx = 2 * nx + 1; h.nny = 2 * ny + 1;
  h.hx = p.Lx / nx; h.hy = p.Ly / ny;
  const int nnx = h.nnx, nny = h.nny;
  h.nslab = nx + 1;
  auto ncol = [&](int s) { return s < nx ? 2 : 1; };
  h.slab_off.assign(h.nslab + 1, 0);
  h.nmax = 0;
  for (int s = 0; s < h.nslab; ++s) {
    long n = (long)ncol(s) * nny * 4 + (ny + 1);
    h.slab_off[s + 1] = h.slab_off[s] + n;
    h.nmax = std::max<int>(h.nmax, (int)n);
  }
  const long M = h.slab_off[h.nslab];
  h.M = M;
  auto node_dof = [&](int i, int j, int f) -> long {
    int s = std::min(i / 2, nx);
    int c = i - 2 * s;
    return h.slab_off[s] + ((long)c * nny + j) * 4 + f;
  };
  auto vert_dof = [&](int a, int b) -> long { return h.slab_off[a] + (long)ncol(a) * nny * 4 + b; };

  h.dof_field.assign(M, -1); h.dof_ix.assign(M, -1); h.dof_iy.assign(M, -1);
  for (int j = 0; j < nny; ++j)
    for (int i = 0; i < nnx; ++i)
      for (int f = 0; f < 4; ++f) {
        long d = node_dof(i, j, f);
        h.dof_field[d] = f; h.dof_ix[d] = i; h.dof_iy[d] = j;
      }
  for (int b = 0; b <= ny; ++b)
    for (int a = 0; a <= nx; ++a) {
      long d = vert_dof(a, b);
      h.dof_field[d] = 4; h.dof_ix[d] = 2 * a; h.dof_iy[d] = 2 * b;
    }

  // cells and the closed solid
  h.ncell = nx * ny;
  h.cell_solid.assign(h.ncell, 0);
  const bool has_solid = p.flap[1] > p.flap[0] && p.flap[3] > p.flap[2];
  std::vector<char> in_sbar((size_t)nnx * nny, 0), vert_fluid((size_t)(nx + 1) * (ny + 1), 0);
  h.nsolid = 0;
  for (int cy = 0; cy < ny; ++cy)
    for (int cx = 0; cx < nx; ++cx) {
      int c = cx + nx * cy;
      double xc = (cx + 0.5) * h.hx, yc = (cy + 0.5) * h.hy;
      bool s = has_solid && xc > p.flap[0] && xc < p.flap[1] && yc > p.flap[2] && yc < p.flap[3];
      h.cell_solid[c] = s;
      if (s) {
        ++h.nsolid;
        for (int ay = 0; ay < 3; ++ay)
          for (int ax = 0; ax < 3; ++ax) in_sbar[(size_t)(2 * cx + ax) + (size_t)nnx * (2 * cy + ay)] = 1;
      } else {
        for (int by = 0; by < 2; ++by)
          for (int bx = 0; bx < 2; ++bx) vert_fluid[(size_t)(cx + bx) + (size_t)(nx + 1) * (cy + by)] = 1;
      }
    }
  // row ownership (coupling conditions built into the rows, see the header)
  auto node_flags = [&](int i, int j, bool& sbar, bool& bnd, bool& vdir) {
    sbar = in_sbar[(size_t)i + (size_t)nnx * j];
    bool inflow = i == 0, outflow = i == nnx - 1, wall = j == 0 || j == nny - 1;
    bnd = inflow || outflow || wall;
    vdir = inflow || wall || sbar;
  };
  auto mom_row = [&](int i, int j, int comp) -> long {
    bool sbar, bnd, vdir;
    node_flags(i, j, sbar, bnd, vdir);
    if (!vdir) return node_dof(i, j, comp);
    if (sbar && !bnd) return node_dof(i, j, 2 + comp);
    return -1;
  };
  auto ext_row = [&](int i, int j, int comp) -> long {
    bool sbar, bnd, vdir;
    node_flags(i, j, sbar, bnd, vdir);
    return (!bnd && !sbar) ? node_dof(i, j, 2 + comp) : -1;
  };
  auto div_row = [&](int a, int b) -> long { return vert_fluid[(size_t)a + (size_t)(nx + 1) * b] ? vert_dof(a, b) : -1; };

  std::vector<char> owned(M, 0);
  for (int j = 0; j < nny; ++j)
    for (int i = 0; i < nnx; ++i)
      for (int comp = 0; comp < 2; ++comp) {
        long r = mom_row(i, j, comp);
        if (r >= 0) { if (owned[r]) return fail(LRFSI_EINVAL, "row owned twice"); owned[r] = 1; }
        r = ext_row(i, j, comp);
        if (r >= 0) { if (owned[r]) return fail(LRFSI_EINVAL, "row owned twice"); owned[r] = 1; }
      }
  for (int b = 0; b <= ny; ++b)
    for (int a = 0; a <= nx; ++a) {
      long r = div_row(a, b);
      if (r >= 0) { if (owned[r]) return fail(LRFSI_EINVAL, "row owned twice"); owned[r] = 1; }
    }
  h.ident.assign(M, 0);
  h.bD.assign(M, 0.0);
  for (long d = 0; d < M; ++d) h.ident[d] = !owned[d];
  for (int j = 0; j < nny; ++j) {
    double y = j * 0.5 * h.hy;
    long d = node_dof(0, j, 0);
    if (h.ident[d]) h.bD[d] = p.v_mean * 6.0 / (p.Ly * p.Ly) * y * (p.Ly - y);
  }

  // per-cell DOF and test-row maps
  h.cell_dof.assign((size_t)h.ncell * kLoc, -1);
  h.cell_row.assign((size_t)h.ncell * kLoc, -1);
  for (int cy = 0; cy < ny; ++cy)
    for (int cx = 0; cx < nx; ++cx) {
      int c = cx + nx * cy;
      bool solid = h.cell_solid[c];
      int* dof = &h.cell_dof[(size_t)c * kLoc];
      int* row = &h.cell_row[(size_t)c * kLoc];
      for (int ay = 0; ay < 3; ++ay)
        for (int ax = 0; ax < 3; ++ax) {
          int a = ax + 3 * ay, i = 2 * cx + ax, j = 2 * cy + ay;
          for (int f = 0; f < 4; ++f) {
            dof[4 * a + f] = (int)node_dof(i, j, f);
            if (f < 2) row[4 * a + f] = (int)mom_row(i, j, f);
            else row[4 * a + f] = solid ? -1 : (int)ext_row(i, j, f - 2);
          }
        }
      for (int by = 0; by < 2; ++by)
        for (int bx = 0; bx < 2; ++bx) {
          int b = bx + 2 * by;
          dof[36 + b] = (int)vert_dof(cx + bx, cy + by);
          row[36 + b] = solid ? -1 : (int)div_row(cx + bx, cy + by);
        }
    }
  // active (test, trial) blocks: fluid mom x {v, p}, ext x u, div x v; solid mom x u
  auto active = [](bool solid, int t, int tt) {
    int tk = t >= 36 ? 2 : ((t & 3) < 2 ? 0 : 1);    // 0 mom, 1 ext, 2 div
    int uk = tt >= 36 ? 2 : ((tt & 3) < 2 ? 0 : 1);   // 0 v, 1 u, 2 p
    if (solid) return tk == 0 && uk == 1;
    return (tk == 0 && (uk == 0 || uk == 2)) || (tk == 1 && uk == 1) || (tk == 2 && uk == 0);
  };
  std::vector<std::vector<int>> cols(M);
  for (int c = 0; c < h.ncell; ++c) {
    bool solid = h.cell_solid[c];
    for (int t = 0; t < kLoc; ++t) {
      int r = h.cell_row[(size_t)c * kLoc + t];
      if (r < 0) continue;
      for (int tt = 0; tt < kLoc; ++tt)
        if (active(solid, t, tt)) cols[r].push_back(h.cell_dof[(size_t)c * kLoc + tt]);
    }
  }
  for (long d = 0; d < M; ++d)
    if (h.ident[d]) cols[d].push_back((int)d);
  h.rowptr.assign(M + 1, 0);
  for (long d = 0; d < M; ++d) {
    auto& v = cols[d];
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    h.rowptr[d + 1] = h.rowptr[d] + (int)v.size();
  }
  if ((long)h.rowptr[M] > 2000000000L) return fail(LRFSI_EINVAL, "pattern too large for int32 CSR");
  h.colidx.resize(h.rowptr[M]);
  for (long d = 0; d < M; ++d) std::copy(cols[d].begin(), cols[d].end(), h.colidx.begin() + h.rowptr[d]);
  std::vector<std::vector<int>>().swap(cols);
  auto find = [&](long r, int col) -> int {
    auto b = h.colidx.begin() + h.rowptr[r], e = h.colidx.begin() + h.rowptr[r + 1];
    auto it = std::lower_bound(b, e, col);
    return (it != e && *it == col) ? (int)(it - h.colidx.begin()) : -1;
  };
  h.slot.assign((size_t)h.ncell * kLoc * kLoc, -1);
  for (int c = 0; c < h.ncell; ++c) {
    bool solid = h.cell_solid[c];
    for (int t = 0; t < kLoc; ++t) {
      int r = h.cell_row[(size_t)c * kLoc + t];
      if (r < 0) continue;
      for (int tt = 0; tt < kLoc; ++tt)
        if (active(solid, t, tt))
          h.slot[((size_t)c * kLoc + t) * kLoc + tt] = find(r, h.cell_dof[(size_t)c * kLoc + tt]);
    }
  }
  h.ident_rows.clear(); h.ident_diag.clear();
  for (long d = 0; d < M; ++d)
    if (h.ident[d]) { h.ident_rows.push_back((int)d); h.ident_diag.push_back(find(d, (int)d)); }
  // colours: cells of one colour share no node
  h.color_cells.clear();
  for (int col = 0; col < 4; ++col) {
    h.color_start[col] = (int)h.color_cells.size();
    for (int cy = 0; cy < ny; ++cy)
      for (int cx = 0; cx < nx; ++cx)
        if ((cx & 1) + 2 * (cy & 1) == col) h.color_cells.push_back(cx + nx * cy);
  }
  h.color_start[4] = (int)h.color_cells.size();
  // CSR entry -> dense slab block offset (diag blocks, then upper, then lower)
  std::vector<int> slab_of(M);
  for (int s = 0; s < h.nslab; ++s)
    for (long d = h.slab_off[s]; d < h.slab_off[s + 1]; ++d) slab_of[d] = s;
  const long long nb2 = (long long)h.nmax * h.nmax;
  const long long Dsz = nb2 * h.nslab, Usz = nb2 * (h.nslab - 1);
  h.dense_off.resize(h.colidx.size());
  for (long r = 0; r < M; ++r)
    for (int k = h.rowptr[r]; k < h.rowptr[r + 1]; ++k) {
      int cidx = h.colidx[k];
      int si = slab_of[r], sj = slab_of[cidx];
      long long li = r - h.slab_off[si], lj = cidx - h.slab_off[sj];
      if (si == sj) h.dense_off[k] = si * nb2 + li * h.nmax + lj;
      else if (sj == si + 1) h.dense_off[k] = Dsz + si * nb2 + li * h.nmax + lj;
      else if (sj == si - 1) h.dense_off[k] = Dsz + Usz + sj * nb2 + li * h.nmax + lj;
      else return fail(LRFSI_EINVAL, "pattern is not block tridiagonal over slabs");
    }
  return LRFSI_OK;
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// Affine Jacobian values of one cell colour.  One block per cell.
__global__ void k_jacobian(Tables T, const int* __restrict__ cells, int ncells, const int* __restrict__ cell_dof,
                           const char* __restrict__ cell_solid, const int* __restrict__ slot,
                           const double* __restrict__ x, double* __restrict__ J3) {
  const int ci = blockIdx.x;
  if (ci >= ncells) return;
  const int c = cells[ci];
  __shared__ double xl[kLoc];
  __shared__ double sv[kNq][2], sGv[kNq][2][2], sGu[kNq][2][2];
  const int tid = threadIdx.x;
  if (tid < kLoc) xl[tid] = x[cell_dof[(size_t)c * kLoc + tid]];
  __syncthreads();
  if (tid < kNq) {
    const int q = tid;
    double v0 = 0, v1 = 0, g[2][2] = {{0, 0}, {0, 0}}, gu[2][2] = {{0, 0}, {0, 0}};
    for (int a = 0; a < 9; ++a) {
      double n = T.N[a][q], dx = T.dN[a][q][0], dy = T.dN[a][q][1];
      double va0 = xl[4 * a], va1 = xl[4 * a + 1], ua0 = xl[4 * a + 2], ua1 = xl[4 * a + 3];
      v0 += va0 * n; v1 += va1 * n;
      g[0][0] += va0 * dx; g[0][1] += va0 * dy; g[1][0] += va1 * dx; g[1][1] += va1 * dy;
      gu[0][0] += ua0 * dx; gu[0][1] += ua0 * dy; gu[1][0] += ua1 * dx; gu[1][1] += ua1 * dy;
    }
    sv[q][0] = v0; sv[q][1] = v1;
    for (int i = 0; i < 2; ++i)
      for (int k = 0; k < 2; ++k) { sGv[q][i][k] = g[i][k]; sGu[q][i][k] = gu[i][k]; }
  }
  __syncthreads();
  const bool solid = cell_solid[c];
  const int* sl = slot + (size_t)c * kLoc * kLoc;
  for (int idx = tid; idx < kLoc * kLoc; idx += blockDim.x) {
    const int e = sl[idx];
    if (e < 0) continue;
    const int t = idx / kLoc, tt = idx % kLoc;
    double j0 = 0, jm = 0, jn = 0;
    if (t < 36 && (t & 3) < 2) {
      const int a = t >> 2, i = t & 3;
      if (tt < 36) {
        const int b = tt >> 2, fk = tt & 3;
        if (!solid) {  // momentum test x velocity trial: convection (J_rho) and viscosity (A2)
          const int k = fk;
          for (int q = 0; q < kNq; ++q) {
            double gb_ga = T.dN[b][q][0] * T.dN[a][q][0] + T.dN[b][q][1] * T.dN[a][q][1];
            double vgb = sv[q][0] * T.dN[b][q][0] + sv[q][1] * T.dN[b][q][1];
            j0 += T.w[q] * T.N[a][q] * (T.N[b][q] * sGv[q][i][k] + (i == k ? vgb : 0.0));
            jn += T.w[q] * ((i == k ? gb_ga : 0.0) + T.dN[b][q][i] * T.dN[a][q][k]);
          }
          j0 *= T.rho; jn *= T.rho;
        } else {  // solid momentum x deformation trial: A1 + J_mu (mu) and J_lambda
          const int k = fk - 2;
          for (int q = 0; q < kNq; ++q) {
            double gb_ga = T.dN[b][q][0] * T.dN[a][q][0] + T.dN[b][q][1] * T.dN[a][q][1];
            double Gk_ga = sGu[q][k][0] * T.dN[a][q][0] + sGu[q][k][1] * T.dN[a][q][1];
            double Gk_gb = sGu[q][k][0] * T.dN[b][q][0] + sGu[q][k][1] * T.dN[b][q][1];
            jm += T.w[q] * ((i == k ? gb_ga : 0.0) + T.dN[b][q][i] * T.dN[a][q][k] +
                            T.dN[b][q][i] * Gk_ga + sGu[q][k][i] * gb_ga);
            j0 += T.w[q] * (T.dN[b][q][k] + Gk_gb) * T.dN[a][q][i];
          }
          j0 *= T.lam;
        }
      } else {  // momentum test x pressure trial
        const int b = tt - 36;
        for (int q = 0; q < kNq; ++q) j0 -= T.w[q] * T.P[b][q] * T.dN[a][q][i];
      }
    } else if (t < 36) {  // extension test x deformation trial
      const int a = t >> 2, i = (t & 3) - 2, b = tt >> 2, k = (tt & 3) - 2;
      if (i == k)
        for (int q = 0; q < kNq; ++q)
          j0 += T.w[q] * (T.dN[b][q][0] * T.dN[a][q][0] + T.dN[b][q][1] * T.dN[a][q][1]);
    } else {  // divergence test x velocity trial
      const int a = t - 36, b = tt >> 2, k = tt & 3;
      for (int q = 0; q < kNq; ++q) j0 += T.w[q] * T.dN[b][q][k] * T.P[a][q];
    }
    J3[3 * (size_t)e + 0] += j0;
    J3[3 * (size_t)e + 1] += jm;
    J3[3 * (size_t)e + 2] += jn;
  }
}

// Fluid velocity mass <v, phi>_F on the pattern (the theta-scheme's A_t^f,
// Sec. 4.3): momentum test (a, i) x velocity trial (b, i) of fluid cells.
__global__ void k_mass_fluid(Tables T, const int* __restrict__ cells, int ncells, const char* __restrict__ cell_solid,
                             const int* __restrict__ slot, double* __restrict__ Mv) {
  const int ci = blockIdx.x;
  if (ci >= ncells) return;
  const int c = cells[ci];
  if (cell_solid[c]) return;
  const int* sl = slot + (size_t)c * kLoc * kLoc;
  for (int idx = threadIdx.x; idx < kLoc * kLoc; idx += blockDim.x) {
    const int e = sl[idx];
    if (e < 0) continue;
    const int t = idx / kLoc, tt = idx % kLoc;
    if (t >= 36 || tt >= 36 || (t & 3) >= 2 || (tt & 3) != (t & 3)) continue;
    const int a = t >> 2, b = tt >> 2;
    double v = 0;
    for (int q = 0; q < kNq; ++q) v += T.w[q] * T.N[a][q] * T.N[b][q];
    Mv[e] += v;
  }
}

__global__ void k_ident_diag(const int* __restrict__ diag, int n, double* __restrict__ J3) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) J3[3 * (size_t)diag[i]] = 1.0;
}

// Residual of one colour for a block of columns; thread = column.
constexpr int kResCols = 64;
__global__ void __launch_bounds__(kResCols) k_residual(Tables T, const int* __restrict__ cells, int ncells,
                                                       const int* __restrict__ cell_dof, const int* __restrict__ cell_row,
                                                       const char* __restrict__ cell_solid, const double* __restrict__ X,
                                                       int ldx, int ncol, const double* __restrict__ c_rest,
                                                       const double* __restrict__ c_mu, const double* __restrict__ c_nu,
                                                       const double* __restrict__ c_rho,
                                                       const double* __restrict__ c_lam, double* __restrict__ R,
                                                       int ldr) {
  const int ci = blockIdx.x;
  const int j = blockIdx.y * kResCols + threadIdx.x;
  if (ci >= ncells || j >= ncol) return;
  const int c = cells[ci];
  const int* dof = cell_dof + (size_t)c * kLoc;
  const int* row = cell_row + (size_t)c * kLoc;
  const bool solid = cell_solid[c];
  const double cr = c_rest ? c_rest[j] : 1.0, cm = c_mu ? c_mu[j] : 0.0, cn = c_nu ? c_nu[j] : 0.0;
  // rho_f and lambda_s of this column (Sec. 4.4 varies them per parameter)
  const double rho = c_rho ? c_rho[j] : T.rho, lam = c_lam ? c_lam[j] : T.lam;
  // ldx == 0: every column reads the same state
  const size_t xs = ldx ? (size_t)ldx : 1, xj = ldx ? (size_t)j : 0;
  double xl[kLoc];
#pragma unroll
  for (int t = 0; t < kLoc; ++t) xl[t] = X[(size_t)dof[t] * xs + xj];
  double acc[kLoc];
#pragma unroll
  for (int t = 0; t < kLoc; ++t) acc[t] = 0.0;
  for (int q = 0; q < kNq; ++q) {
    double v0 = 0, v1 = 0, p = 0, g00 = 0, g01 = 0, g10 = 0, g11 = 0, u00 = 0, u01 = 0, u10 = 0, u11 = 0;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const double n = T.N[a][q], dx = T.dN[a][q][0], dy = T.dN[a][q][1];
      v0 += xl[4 * a] * n; v1 += xl[4 * a + 1] * n;
      g00 += xl[4 * a] * dx; g01 += xl[4 * a] * dy; g10 += xl[4 * a + 1] * dx; g11 += xl[4 * a + 1] * dy;
      u00 += xl[4 * a + 2] * dx; u01 += xl[4 * a + 2] * dy; u10 += xl[4 * a + 3] * dx; u11 += xl[4 * a + 3] * dy;
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) p += xl[36 + b] * T.P[b][q];
    const double w = T.w[q];
    if (!solid) {
      // momentum: rho (v.grad)v . phi - p div phi + nu rho (grad v + grad v^T) : grad phi
      const double c0 = rho * (v0 * g00 + v1 * g01), c1 = rho * (v0 * g10 + v1 * g11);
      const double s00 = 2 * g00, s01 = g01 + g10, s11 = 2 * g11;
      const double dv = g00 + g11;
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        const double n = T.N[a][q], dx = T.dN[a][q][0], dy = T.dN[a][q][1];
        acc[4 * a + 0] += w * (cr * (c0 * n - p * dx) + cn * rho * (s00 * dx + s01 * dy));
        acc[4 * a + 1] += w * (cr * (c1 * n - p * dy) + cn * rho * (s01 * dx + s11 * dy));
        acc[4 * a + 2] += w * cr * (u00 * dx + u01 * dy);  // extension
        acc[4 * a + 3] += w * cr * (u10 * dx + u11 * dy);
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[36 + b] += w * cr * dv * T.P[b][q];
    } else {
      // mu <G + G^T + G^T G, grad phi> + lambda <tr(G + G^T G / 2), div phi>
      const double e00 = 2 * u00 + u00 * u00 + u10 * u10;
      const double e01 = u01 + u10 + u00 * u01 + u10 * u11;
      const double e11 = 2 * u11 + u01 * u01 + u11 * u11;
      const double tr = u00 + u11 + 0.5 * (u00 * u00 + u01 * u01 + u10 * u10 + u11 * u11);
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        const double dx = T.dN[a][q][0], dy = T.dN[a][q][1];
        acc[4 * a + 0] += w * (cm * (e00 * dx + e01 * dy) + cr * lam * tr * dx);
        acc[4 * a + 1] += w * (cm * (e01 * dx + e11 * dy) + cr * lam * tr * dy);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < kLoc; ++t) {
    const int r = row[t];
    if (r >= 0) R[(size_t)r * ldr + j] += acc[t];
  }
}

__global__ void k_residual_ident(const int* __restrict__ rows, int nrows, const double* __restrict__ X, int ldx,
                                 const double* __restrict__ bD, int ncol, const double* __restrict__ c_rest,
                                 double* __restrict__ R, int ldr) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)nrows * ncol) return;
  const int i = (int)(idx / ncol), j = (int)(idx % ncol);
  const int r = rows[i];
  const double cr = c_rest ? c_rest[j] : 1.0;
  const size_t xs = ldx ? (size_t)ldx : 1, xj = ldx ? (size_t)j : 0;
  R[(size_t)r * ldr + j] = cr * (X[(size_t)r * xs + xj] - bD[r]);
}

constexpr int kNormRows = 256;
__global__ void k_colnorm_partial(const double* __restrict__ R, long M, int ncol, int ldr, double* __restrict__ part) {
  const int j = blockIdx.y * blockDim.x + threadIdx.x;
  if (j >= ncol) return;
  const long r0 = (long)blockIdx.x * kNormRows;
  const long r1 = r0 + kNormRows < M ? r0 + kNormRows : M;
  double s = 0;
  for (long r = r0; r < r1; ++r) {
    double v = R[r * ldr + j];
    s += v * v;
  }
  part[(size_t)blockIdx.x * ncol + j] = s;
}

__global__ void k_colnorm_reduce(const double* __restrict__ part, int nblk, int ncol, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncol) return;
  double s = 0;
  for (int b = 0; b < nblk; ++b) s += part[(size_t)b * ncol + j];
  out[j] = s;
}

// ---------------------------------------------------------------------------
// Launch wrappers
// ---------------------------------------------------------------------------

static Tables tables_of(const lrfsi_mesh_s* m) {
  Tables T;
  make_tables(m->h.hx, m->h.hy, m->h.prob.rho_f, m->h.prob.lam_s, T);
  return T;
}

int launch_jacobian(lrfsi_mesh_s* m, const double* x, double* J3, cudaStream_t s, const double* rho_lam) {
  Tables T = tables_of(m);
  if (rho_lam) {
    T.rho = rho_lam[0];
    T.lam = rho_lam[1];
  }
  LRFSI_CUDA(cudaMemsetAsync(J3, 0, sizeof(double) * 3 * m->h.colidx.size(), s));
  for (int col = 0; col < 4; ++col) {
    int n = m->h.color_start[col + 1] - m->h.color_start[col];
    if (n == 0) continue;
    k_jacobian<<<n, 128, 0, s>>>(T, m->color_cells.p + m->h.color_start[col], n, m->cell_dof.p, m->cell_solid.p,
                                 m->slot.p, x, J3);
    LRFSI_TRY(check_launch("k_jacobian"));
  }
  int ni = (int)m->h.ident_rows.size();
  if (ni) {
    k_ident_diag<<<ceil_div(ni, 256), 256, 0, s>>>(m->ident_diag.p, ni, J3);
    LRFSI_TRY(check_launch("k_ident_diag"));
  }
  return LRFSI_OK;
}

int launch_mass_fluid(lrfsi_mesh_s* m, double* Mv, cudaStream_t s) {
  const Tables T = tables_of(m);
  LRFSI_CUDA(cudaMemsetAsync(Mv, 0, sizeof(double) * m->h.colidx.size(), s));
  for (int col = 0; col < 4; ++col) {
    int n = m->h.color_start[col + 1] - m->h.color_start[col];
    if (n == 0) continue;
    k_mass_fluid<<<n, 128, 0, s>>>(T, m->color_cells.p + m->h.color_start[col], n, m->cell_solid.p, m->slot.p, Mv);
    LRFSI_TRY(check_launch("k_mass_fluid"));
  }
  return LRFSI_OK;
}

int launch_residual(lrfsi_mesh_s* m, const double* X, int ldx, int ncol, const double* c_rest,
                    const double* c_mu, const double* c_nu, double* R, int ldr, cudaStream_t s, const double* c_rho,
                    const double* c_lam) {
  if (ncol <= 0) return LRFSI_OK;
  const Tables T = tables_of(m);
  LRFSI_CUDA(cudaMemsetAsync(R, 0, sizeof(double) * (size_t)m->h.M * ldr, s));
  for (int col = 0; col < 4; ++col) {
    int n = m->h.color_start[col + 1] - m->h.color_start[col];
    if (n == 0) continue;
    dim3 grid(n, ceil_div(ncol, kResCols));
    k_residual<<<grid, kResCols, 0, s>>>(T, m->color_cells.p + m->h.color_start[col], n, m->cell_dof.p,
                                         m->cell_row.p, m->cell_solid.p, X, ldx, ncol, c_rest, c_mu, c_nu, c_rho, c_lam,
                                         R, ldr);
    LRFSI_TRY(check_launch("k_residual"));
  }
  long ni = (long)m->h.ident_rows.size();
  if (ni) {
    long tot = ni * ncol;
    k_residual_ident<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(m->ident_rows.p, (int)ni, X, ldx, m->bD.p, ncol,
                                                                  c_rest, R, ldr);
    LRFSI_TRY(check_launch("k_residual_ident"));
  }
  return LRFSI_OK;
}

size_t colnorm_work_len(long M, int ncol) { return (size_t)ceil_div(M, kNormRows) * (size_t)(ncol > 0 ? ncol : 0); }

int launch_colnorm2(const double* R, long M, int ncol, int ldr, double* out, double* work, size_t work_len,
                    cudaStream_t s) {
  if (ncol <= 0) return LRFSI_OK;
  int nblk = ceil_div(M, kNormRows);
  if ((size_t)nblk * ncol > work_len) return fail(LRFSI_EINVAL, "colnorm workspace too small");
  dim3 grid(nblk, ceil_div(ncol, 128));
  k_colnorm_partial<<<grid, 128, 0, s>>>(R, M, ncol, ldr, work);
  LRFSI_TRY(check_launch("k_colnorm_partial"));
  k_colnorm_reduce<<<ceil_div(ncol, 128), 128, 0, s>>>(work, nblk, ncol, out);
  return check_launch("k_colnorm_reduce");
}

}  // namespace lrfsi
