// Mesh, DOF layout and assembly data of the channel-with-flap FSI problem.
#pragma once

#include <memory>

#include "common.h"

namespace lrfsi {

// Local DOF numbering of a cell: Q2 node a = ax + 3 ay (ax, ay in 0..2), its
// four unknowns (v_x, v_y, u_x, u_y) at 4 a + f; the four Q1 vertices
// b = bx + 2 by at 36 + b.  Test functions use the same numbering: t < 36
// with f < 2 is the momentum test phi_a e_f, f >= 2 the extension test
// psi_a e_{f-2}; t >= 36 the divergence test xi_b.
constexpr int kLoc = 40;
constexpr int kNq = 9;  // 3 x 3 Gauss points

struct MeshHost {
  lrfsi_problem prob;
  int nx, ny, nnx, nny;
  double hx, hy;
  long M = 0;
  int nslab = 0, nmax = 0;
  std::vector<long> slab_off;         // nslab + 1
  std::vector<int> dof_field, dof_ix, dof_iy;
  std::vector<double> bD;
  std::vector<char> ident;            // identity (Dirichlet) rows
  std::vector<int> rowptr, colidx;    // CSR union pattern
  std::vector<int> cell_dof;          // ncell x 40
  std::vector<int> cell_row;          // ncell x 40 test -> row (-1: none)
  std::vector<char> cell_solid;
  std::vector<int> slot;              // ncell x 40 x 40 -> CSR entry (-1)
  std::vector<int> color_cells;       // cells sorted by colour
  int color_start[5];
  std::vector<int> ident_rows, ident_diag;  // identity rows and their diagonal CSR entry
  std::vector<long long> dense_off;   // CSR entry -> offset in the slab block workspace
  int ncell = 0, nsolid = 0;
};

}  // namespace lrfsi

namespace lrfsi {
struct NdSymbolic;
struct NdDevice;
}

// The opaque handle.
struct lrfsi_mesh_s {
  lrfsi::MeshHost h;
  lrfsi::DevBuf<int> rowptr, colidx, cell_dof, cell_row, slot, color_cells, ident_rows, ident_diag;
  lrfsi::DevBuf<char> cell_solid;
  lrfsi::DevBuf<double> bD;
  lrfsi::DevBuf<long long> dense_off;
  lrfsi::DevBuf<long long> slab_off;
  // SpMM windows: for row block b (kSpmmRowBlock rows) the column range
  // [win[2b], win[2b+1]) its nonzeros touch; winmax = the widest window
  lrfsi::DevBuf<int> spmm_win;
  int spmm_winmax = 0;
  // nested-dissection structure of the sparse LU (built on first use)
  std::shared_ptr<lrfsi::NdSymbolic> nd;
  std::shared_ptr<lrfsi::NdDevice> ndd;
};

namespace lrfsi {
constexpr int kSpmmRowBlock = 128;
}

namespace lrfsi {
int build_mesh(const lrfsi_problem& prob, MeshHost& h);

// Assembly launches (mesh.cu).
// Residual of ncol states: X (M x ldx, row-major; ldx = 0 broadcasts one
// state), output R (M x ldr).  Column j combines the terms as
//   c_rest[j] * (everything but the mu- and nu-terms, incl. x - b_D rows)
//   + c_mu[j] * <G + G^T + G^T G, grad phi>_S + c_nu[j] * rho_f <grad v + grad v^T, grad phi>_F
// c_rho, c_lam (per column, optional): rho_f and lambda_s of each column in
// place of the mesh's constants (the four-parameter problem, Sec. 4.4); they
// scale the convection and viscous terms (rho) and the lambda term.
int launch_residual(lrfsi_mesh_s* m, const double* X, int ldx, int ncol, const double* c_rest,
                    const double* c_mu, const double* c_nu, double* R, int ldr, cudaStream_t s,
                    const double* c_rho = nullptr, const double* c_lam = nullptr);
// Fluid velocity mass values <v, phi>_F on the pattern (nnz; the theta-scheme's A_t^f).
int launch_mass_fluid(lrfsi_mesh_s* m, double* Mv, cudaStream_t s);
// Affine Jacobian values (nnz x 3 interleaved) at state x; rho_lam (host,
// optional): {rho_f, lambda_s} in place of the mesh's constants.
int launch_jacobian(lrfsi_mesh_s* m, const double* x, double* J3, cudaStream_t s, const double* rho_lam = nullptr);
// Column squared norms of an M x ncol row-major block (ldr), accumulated in
// fixed order: out[j] = sum_i R[i, j]^2.  work: >= ceil(M/rows_per_block) * ncol doubles.
// Doubles of workspace launch_colnorm2 needs for M rows and ncol columns (one
// partial sum per column per block of rows).
size_t colnorm_work_len(long M, int ncol);
int launch_colnorm2(const double* R, long M, int ncol, int ldr, double* out, double* work,
                    size_t work_len, cudaStream_t s);
}  // namespace lrfsi
