"""Shared fixtures for the GPU parity tests: the library's DOF order is mapped
to the oracle's through lrfsi_mesh_dofmap (an interface fact, no shared code)."""
import numpy as np
import scipy.sparse as sp

from oracle import fsi


def perm_lib_to_oracle(lib_mesh, om):
    f, ix, iy = lib_mesh.dofmap()
    nnx = 2 * om.nx + 1
    perm = np.where(f < 4, f.astype(np.int64) * om.NQ2 + ix + nnx * iy,
                    4 * om.NQ2 + ix // 2 + (om.nx + 1) * (iy // 2))
    assert len(np.unique(perm)) == om.M
    return perm


def lib_csr(lib_mesh, vals):
    rp, ci = lib_mesh.pattern()
    return sp.csr_matrix((vals, ci, rp), shape=(lib_mesh.M, lib_mesh.M))


def rel_max(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
