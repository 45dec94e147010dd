"""Python binding of the lrfsi C ABI (include/lrfsi.h): argument marshalling only.

Every computation runs in the CUDA library ``liblrfsi.so`` built from
``csrc/``; this module converts torch tensors (device memory) and numpy arrays
(host memory) to pointers and checks status codes.  There is no fallback: if
the library is missing, importing the binding raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblrfsi.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "lrfsi.h")

OK, EINVAL, ENOMEM, ECUDA, ESINGULAR, ENOCONV, EBREAKDOWN, ETIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7


class LrfsiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lrfsi error {code}: {msg}")
        self.code = code


class lrfsi_problem(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("Lx", C.c_double), ("Ly", C.c_double),
                ("flap", C.c_double * 4), ("rho_f", C.c_double), ("lam_s", C.c_double), ("v_mean", C.c_double)]


class lrfsi_mesh_info_t(C.Structure):
    _fields_ = [("M", C.c_int64), ("nnz", C.c_int64), ("nslab", C.c_int), ("nmax", C.c_int),
                ("ncell", C.c_int), ("nsolid", C.c_int)]


class lrfsi_cheb_options(C.Structure):
    _fields_ = [("c", C.c_double), ("d", C.c_double), ("iters", C.c_int), ("cycles", C.c_int),
                ("rank_cap", C.c_int), ("tol", C.c_double), ("eta", C.c_double), ("precision", C.c_int),
                ("tol_sol", C.c_double), ("solver", C.c_int)]


class lrfsi_kernel_stat(C.Structure):
    _fields_ = [("launches", C.c_uint64), ("flops", C.c_double), ("bytes", C.c_double), ("ms", C.c_double)]


KERNEL_CLASSES = ("gemm_fp64", "spmm_fp64", "gram_fp64", "block_lu", "fe_assembly", "gemm_fp32", "spmm_fp32",
                  "trunc_small", "lu_panel", "lu_trsm", "lu_solve", "trunc_svd", "tc_mma", "gemm_tc", "gram_tc")
# classes that time whole regions containing launches of other classes, and the
# tensor-core slice products (inside gemm_tc / gram_tc)
REGION_CLASSES = ("block_lu", "lu_solve", "tc_mma")
# FP64 products on the tensor cores (FP64 algorithmic FLOPs over the whole
# splitting pipeline: not FP64-unit work)
TENSOR_CLASSES = ("gemm_tc", "gram_tc")


class lrfsi_cheb_stats(C.Structure):
    _fields_ = [("steps", C.c_int), ("rank", C.c_int), ("rel_lin_res", C.c_double), ("max_concat_rank", C.c_int)]


_lib = None


def load():
    """Load liblrfsi.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"liblrfsi.so not built ({LIB_PATH}); run paper_2008_10275_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i, d, i64p = C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_int64)
    sig = {
        "lrfsi_mesh_create": [C.POINTER(lrfsi_problem), C.POINTER(vp)],
        "lrfsi_mesh_destroy": [vp],
        "lrfsi_mesh_info": [vp, C.POINTER(lrfsi_mesh_info_t)],
        "lrfsi_mesh_dofmap": [vp, vp, vp, vp],
        "lrfsi_mesh_dirichlet": [vp, vp],
        "lrfsi_mesh_pattern": [vp, vp, vp],
        "lrfsi_assemble_affine": [vp, vp, vp, vp, vp],
        "lrfsi_residual_batch": [vp, vp, i, i, vp, vp, vp, i, vp, vp],
        "lrfsi_residual": [vp, vp, vp, i, vp, i, i, vp, vp, i, vp, vp],
        "lrfsi_residual_batch_noalloc": [vp, vp, i, i, vp, vp, vp, i, vp, vp],
        "lrfsi_mlp_create": [i, i, i, i, C.POINTER(vp)],
        "lrfsi_mlp_destroy": [vp],
        "lrfsi_mlp_set_params": [vp, vp],
        "lrfsi_mlp_get_params": [vp, vp],
        "lrfsi_mlp_forward": [vp, vp, i, vp, vp],
        "lrfsi_mlp_gradients": [vp, vp, vp, i, vp, vp, vp],
        "lrfsi_mlp_train": [vp, vp, vp, i, i, C.c_float, vp, vp],
        "lrfsi_learned_fit": [vp, vp, vp, vp, i, vp, vp, i, i, i, C.c_float, vp, i, vp, vp, vp, vp, vp, vp],
        "lrfsi_learned_start": [vp, vp, vp, vp, i, vp, vp, i, i, vp, vp, vp, vp, vp, vp],
        "lrfsi_truncation_counters": [vp, i],
        "lrfsi_spmm": [vp, vp, vp, i, i, vp, i, i, vp],
        "lrfsi_spmm_tuning": [i, i, vp, vp],
        "lrfsi_pod": [vp, vp, i, i, i, vp, i, vp, i, vp, vp],
        "lrfsi_newton_median": [vp, i, vp, vp, vp, d, i, vp, vp, vp],
        "lrfsi_subset_create": [vp, i, vp, vp, vp, vp, vp, C.POINTER(vp), vp],
        "lrfsi_subset_destroy": [vp],
        "lrfsi_chebyshevT": [vp, vp, i, vp, i, vp, C.POINTER(lrfsi_cheb_options), vp, i, vp, i, vp, vp, vp],
        "lrfsi_gmresT": [vp, vp, i, vp, i, vp, C.POINTER(lrfsi_cheb_options), vp, i, vp, i, vp, vp, vp],
        "lrfsi_subset_step": [vp, C.POINTER(lrfsi_cheb_options), d, i, vp, i, vp, i, vp, vp, vp, vp],
        "lrfsi_subset_step_init": [vp, C.POINTER(lrfsi_cheb_options), d, i, vp, i, vp, i, vp, vp, i, vp, i, vp, vp,
                                   vp, vp, vp],
        "lrfsi_learned_factors": [vp, vp, i, vp, vp, vp, vp, vp, i, i, vp, vp, vp, vp, vp, i, vp, i, vp],
        "lrfsi_precond_apply": [vp, vp, i, vp, vp, i, vp],
        "lrfsi_truncate": [vp, vp, i, vp, i, vp, d, vp, vp, i, vp, i, vp, vp],
        "lrfsi_graph_mode": [i, vp],
        "lrfsi_mass_fluid": [vp, vp, vp],
        "lrfsi_newton_theta": [vp, i, vp, vp, vp, vp, d, d, d, i, vp, vp, vp],
        "lrfsi_subset_create_theta": [vp, i, vp, vp, vp, vp, vp, d, d, C.POINTER(vp), vp],
        "lrfsi_subset_step_theta": [vp, C.POINTER(lrfsi_cheb_options), vp, i, d, i, vp, i, vp, i, vp, vp, vp, vp],
        "lrfsi_assemble_affine4": [vp, vp, vp, vp, vp, vp, vp],
        "lrfsi_residual_batch4": [vp, vp, i, i, vp, vp, vp, vp, vp, i, vp, vp],
        "lrfsi_newton_median4": [vp, i, vp, vp, vp, vp, vp, d, i, vp, vp, vp],
        "lrfsi_subset_create4": [vp, i, vp, vp, vp, vp, vp, vp, vp, C.POINTER(vp), vp],
        "lrfsi_lu_mode": [i, vp],
        "lrfsi_lu_info": [C.POINTER(lrfsi_problem), vp],
        "lrfsi_graph_counters": [vp, i],
        "lrfsi_order_grid": [i, i, vp, vp, i, vp, vp],
        "lrfsi_order_set": [i, vp, vp, vp],
        "lrfsi_cluster": [i, i, vp, vp, vp],
        "lrfsi_medians": [i, vp, vp, vp],
        "lrfsi_partition": [i, vp, i, vp],
        "lrfsi_gram": [vp, i, i, vp, i, i, C.c_int64, vp, i, vp],
        "lrfsi_gram_path": [i, vp],
        "lrfsi_svd_cluster": [i, vp],
        "lrfsi_gemm": [i, i, i, vp, i, vp, i, vp, i, d, d, i, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.lrfsi_last_error.restype = C.c_char_p
    lib.lrfsi_kernel_launches.restype = C.c_uint64
    lib.lrfsi_host_launches.restype = C.c_uint64
    lib.lrfsi_mesh_bytes.restype = C.c_size_t
    lib.lrfsi_mesh_bytes.argtypes = [vp]
    lib.lrfsi_subset_bytes.restype = C.c_size_t
    lib.lrfsi_subset_bytes.argtypes = [vp]
    lib.lrfsi_mlp_num_params.argtypes = [vp]
    lib.lrfsi_mlp_num_params.restype = C.c_int64
    lib.lrfsi_stats.argtypes = [i, C.POINTER(lrfsi_kernel_stat)]
    lib.lrfsi_stats.restype = C.c_int
    lib.lrfsi_stats_reset.restype = C.c_int
    lib.lrfsi_timing.argtypes = [i]
    lib.lrfsi_timing.restype = C.c_int
    _lib = lib
    return lib


def declared_symbols():
    """Names of the functions declared in include/lrfsi.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lrfsi_[a-zA-Z0-9_]+)\s*\(", txt)))


def _check(code, allow=()):
    if code != OK and code not in allow:
        raise LrfsiError(code, load().lrfsi_last_error().decode())
    return code


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(int(stream))


def lrfsi_order_grid(mu_values, nu_values, nu_fastest=False):
    """Little-endian order of the grid (Def. 1); returns (mu, nu) of length m1 m2."""
    a = np.ascontiguousarray(mu_values, np.float64)
    b = np.ascontiguousarray(nu_values, np.float64)
    mu = np.zeros(len(a) * len(b))
    nu = np.zeros(len(a) * len(b))
    _check(load().lrfsi_order_grid(len(a), len(b), _ptr(a), _ptr(b), int(bool(nu_fastest)), _ptr(mu), _ptr(nu)))
    return mu, nu


def lrfsi_order_set(mu, nu):
    """Order of a scattered parameter set (nu_f, then mu_s); returns the permutation."""
    a = np.ascontiguousarray(mu, np.float64)
    b = np.ascontiguousarray(nu, np.float64)
    perm = np.zeros(len(a), np.int32)
    _check(load().lrfsi_order_set(len(a), _ptr(a), _ptr(b), _ptr(perm)))
    return perm


def lrfsi_cluster(m, K):
    """Eq. (clustering1) subsets and upper medians: (sizes, offsets, medians)."""
    sizes = np.zeros(max(K, 1), np.int32); offs = np.zeros(max(K, 1), np.int32); med = np.zeros(max(K, 1), np.int32)
    _check(load().lrfsi_cluster(int(m), int(K), _ptr(sizes), _ptr(offs), _ptr(med)))
    return sizes, offs, med


def lrfsi_medians(sizes):
    """Offsets and upper medians of given subset sizes: (offsets, medians)."""
    sz = np.ascontiguousarray(sizes, np.int32)
    offs = np.zeros(max(len(sz), 1), np.int32); med = np.zeros(max(len(sz), 1), np.int32)
    _check(load().lrfsi_medians(len(sz), _ptr(sz), _ptr(offs), _ptr(med)))
    return offs, med


def lrfsi_partition(weights, nproc):
    """Contiguous balanced split of the subsets over nproc processes: first[nproc + 1]."""
    w = np.ascontiguousarray(weights, np.int64)
    first = np.zeros(nproc + 1, np.int32)
    _check(load().lrfsi_partition(len(w), _ptr(w) if len(w) else None, int(nproc), _ptr(first)))
    return first


def graph_mode(mode=-1):
    """Set the ChebyshevT launch mode (0 host-sized, 1 fixed sequence, 2 CUDA
    graph; -1 queries); returns the previous mode."""
    prev = C.c_int(0)
    _check(load().lrfsi_graph_mode(int(mode), C.byref(prev)))
    return prev.value


def gram_path(path=-1):
    """Set the Gram product path (1 tensor cores by error-free splitting, 0
    FP64 FMA; -1 queries); returns the previous path."""
    prev = C.c_int(0)
    _check(load().lrfsi_gram_path(int(path), C.byref(prev)))
    return prev.value


def lrfsi_gemm(m, n, k, A, lda, B, ldb, C, ldc, alpha=1.0, beta=0.0, tensor=True, stream=None):
    """C = alpha A B + beta C for row-major device matrices (tall products on the
    tensor cores when ``tensor`` and the tensor path is on, else FP64 kernels)."""
    for t in (A, B, C):
        if not t.is_contiguous():
            raise ValueError("lrfsi_gemm: A, B and C must be row-major contiguous tensors")
    _check(load().lrfsi_gemm(int(m), int(n), int(k), _ptr(A), lda, _ptr(B), ldb, _ptr(C), ldc, float(alpha),
                             float(beta), int(bool(tensor)), _stream(stream)))


def svd_cluster(size=-1):
    """Set the cluster size of the truncation SVD (0 automatic, 2, 4, 8, 16;
    -1 queries); returns the previous setting."""
    prev = C.c_int(0)
    _check(load().lrfsi_svd_cluster(int(size), C.byref(prev)))
    return prev.value


def lrfsi_gram(A, lda, p, B, ldb, q, M, G, ldg, stream=None):
    """G = A^T B of tall row-major device factors (M x p, M x q) into G (p x q, ldg)."""
    _check(load().lrfsi_gram(_ptr(A), lda, p, _ptr(B), ldb, q, int(M), _ptr(G), ldg, _stream(stream)))


def lu_mode(mode=-1):
    """Set the sparse LU (1 nested dissection, 0 slab block LU; -1 queries);
    returns the previous mode."""
    prev = C.c_int(0)
    _check(load().lrfsi_lu_mode(int(mode), C.byref(prev)))
    return prev.value


def lu_info(nx, ny, Lx=2.0, Ly=0.4, flap=(0.6, 0.7, 0.0, 0.2), rho_f=1e3, lam_s=2e6, v_mean=0.2):
    """Host-only nested-dissection analysis of a mesh (no GPU needed)."""
    p = lrfsi_problem(nx, ny, Lx, Ly, (C.c_double * 4)(*flap), rho_f, lam_s, v_mean)
    out = np.zeros(8, np.int64)
    _check(load().lrfsi_lu_info(C.byref(p), _ptr(out)))
    keys = ("fronts", "heights", "max_separator", "max_boundary", "factor_doubles", "factor_flops",
            "slab_lu_flops", "slab_lu_doubles")
    return dict(zip(keys, (int(v) for v in out)))


def graph_counters(reset=False):
    """(replays, captures, capture failures) of the ChebyshevT graphs."""
    out = np.zeros(3, np.int64)
    _check(load().lrfsi_graph_counters(_ptr(out), int(bool(reset))))
    return dict(replays=int(out[0]), captures=int(out[1]), failures=int(out[2]))


def kernel_launches():
    return int(load().lrfsi_kernel_launches())


def host_launches():
    return int(load().lrfsi_host_launches())


class Mesh:
    """A mesh handle (lrfsi_mesh)."""

    def __init__(self, nx, ny, Lx=2.0, Ly=0.4, flap=(0.6, 0.7, 0.0, 0.2), rho_f=1e3, lam_s=2e6, v_mean=0.2):
        lib = load()
        p = lrfsi_problem(nx, ny, Lx, Ly, (C.c_double * 4)(*(flap if flap is not None else (0, 0, 0, 0))),
                          rho_f, lam_s, v_mean)
        self.h = C.c_void_p()
        _check(lib.lrfsi_mesh_create(C.byref(p), C.byref(self.h)))
        info = lrfsi_mesh_info_t()
        _check(lib.lrfsi_mesh_info(self.h, C.byref(info)))
        self.M, self.nnz, self.nslab, self.nmax = int(info.M), int(info.nnz), info.nslab, info.nmax
        self.ncell, self.nsolid = info.ncell, info.nsolid
        self.nx, self.ny = nx, ny

    def close(self):
        if self.h:
            load().lrfsi_mesh_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dofmap(self):
        f = np.zeros(self.M, np.int32); ix = np.zeros(self.M, np.int32); iy = np.zeros(self.M, np.int32)
        _check(load().lrfsi_mesh_dofmap(self.h, _ptr(f), _ptr(ix), _ptr(iy)))
        return f, ix, iy

    def dirichlet(self):
        b = np.zeros(self.M)
        _check(load().lrfsi_mesh_dirichlet(self.h, _ptr(b)))
        return b

    def pattern(self):
        rp = np.zeros(self.M + 1, np.int32); ci = np.zeros(self.nnz, np.int32)
        _check(load().lrfsi_mesh_pattern(self.h, _ptr(rp), _ptr(ci)))
        return rp, ci

    def device_bytes(self):
        return int(load().lrfsi_mesh_bytes(self.h))


def lrfsi_mesh(nx, ny, **kw):
    return Mesh(nx, ny, **kw)


def lrfsi_assemble_affine(mesh, x, J3=None, R3=None, stream=None):
    _check(load().lrfsi_assemble_affine(mesh.h, _ptr(x), _ptr(J3), _ptr(R3), _stream(stream)))


def lrfsi_residual_batch(mesh, X, ldx, m, mu, nu, R=None, ldr=0, norm2=None, stream=None):
    _check(load().lrfsi_residual_batch(mesh.h, _ptr(X), ldx, m, _ptr(mu), _ptr(nu), _ptr(R), ldr, _ptr(norm2),
                                       _stream(stream)))


def lrfsi_residual_batch_noalloc(mesh, X, ldx, m, mu, nu, R, ldr, norm2=None, stream=None):
    """lrfsi_residual_batch without device allocation (R is required)."""
    _check(load().lrfsi_residual_batch_noalloc(mesh.h, _ptr(X), ldx, m, _ptr(mu), _ptr(nu), _ptr(R), ldr,
                                               _ptr(norm2), _stream(stream)))


def lrfsi_residual(mesh, xt, U, ldu, V, ldv, r, mu, nu, m, stream=None):
    out = np.zeros(m)
    _check(load().lrfsi_residual(mesh.h, _ptr(xt), _ptr(U), ldu, _ptr(V), ldv, r, _ptr(mu), _ptr(nu), m,
                                 _ptr(out), _stream(stream)))
    return out


def lrfsi_newton_median(mesh, X, mu, nu, eps, max_it, stream=None, allow_noconv=False):
    """X: K x M device tensor (in: start, out: solution).  Returns (iters, res, status)."""
    K = len(mu)
    mu = np.ascontiguousarray(mu, np.float64); nu = np.ascontiguousarray(nu, np.float64)
    it = np.zeros(K, np.int32); res = np.zeros(K)
    st = load().lrfsi_newton_median(mesh.h, K, _ptr(X), _ptr(mu), _ptr(nu), eps, max_it, _ptr(it), _ptr(res),
                                    _stream(stream))
    _check(st, (ENOCONV,) if allow_noconv else ())
    return it, res, st


def lrfsi_newton_median4(mesh, X, mu, nu, lam, rho, eps, max_it, stream=None, allow_noconv=False):
    """Four-parameter median Newton (Sec. 4.4); X: K x M device tensor."""
    K = len(mu)
    a = [np.ascontiguousarray(v, np.float64) for v in (mu, nu, lam, rho)]
    it = np.zeros(K, np.int32); res = np.zeros(K)
    st = load().lrfsi_newton_median4(mesh.h, K, _ptr(X), *[_ptr(v) for v in a], eps, max_it, _ptr(it), _ptr(res),
                                     _stream(stream))
    _check(st, (ENOCONV,) if allow_noconv else ())
    return it, res, st


def lrfsi_assemble_affine4(mesh, x, J3a=None, J3b=None, R3a=None, R3b=None, stream=None):
    _check(load().lrfsi_assemble_affine4(mesh.h, _ptr(x), _ptr(J3a), _ptr(J3b), _ptr(R3a), _ptr(R3b),
                                         _stream(stream)))


def lrfsi_residual_batch4(mesh, X, ldx, m, mu, nu, lam, rho, R, ldr, norm2=None, stream=None):
    _check(load().lrfsi_residual_batch4(mesh.h, _ptr(X), ldx, m, _ptr(mu), _ptr(nu), _ptr(lam), _ptr(rho), _ptr(R),
                                        ldr, _ptr(norm2), _stream(stream)))


def lrfsi_mass_fluid(mesh, Mv, stream=None):
    _check(load().lrfsi_mass_fluid(mesh.h, _ptr(Mv), _stream(stream)))


def lrfsi_newton_theta(mesh, X, Xprev, mu, nu, theta, dt, eps, max_it, stream=None, allow_noconv=False):
    """One theta-scheme time step of K problems (Sec. 4.3); X, Xprev: K x M."""
    K = len(mu)
    mu = np.ascontiguousarray(mu, np.float64); nu = np.ascontiguousarray(nu, np.float64)
    it = np.zeros(K, np.int32); res = np.zeros(K)
    st = load().lrfsi_newton_theta(mesh.h, K, _ptr(X), _ptr(Xprev), _ptr(mu), _ptr(nu), theta, dt, eps, max_it,
                                   _ptr(it), _ptr(res), _stream(stream))
    _check(st, (ENOCONV,) if allow_noconv else ())
    return it, res, st


def lrfsi_subset_step_theta(sub, opt, Xprev, ldx, target, max_outer, U, ldu, V, ldv, stream=None,
                            allow_noconv=True):
    ranks = np.zeros(sub.K, np.int32)
    rel = np.zeros(int(sub.sizes.sum()))
    outer = np.zeros(sub.K, np.int32)
    st = load().lrfsi_subset_step_theta(sub.h, C.byref(opt), _ptr(Xprev), ldx, target, max_outer, _ptr(U), ldu,
                                        _ptr(V), ldv, _ptr(ranks), _ptr(rel), _ptr(outer), _stream(stream))
    _check(st, (ENOCONV,) if allow_noconv else ())
    return ranks, rel, outer, st


SOLVERS = {"chebyshev": 0, "gmres": 1}


def cheb_options(c, d, iters=6, cycles=2, rank_cap=20, tol=1e-8, eta=0.0, precision=0, tol_sol=0.0,
                 solver="chebyshev"):
    return lrfsi_cheb_options(c, d, iters, cycles, rank_cap, tol, eta, precision, tol_sol, SOLVERS[solver])


class Subsets:
    """K subsets sharing one mesh (lrfsi_subset_create; with lam and rho the
    four-parameter problem, lrfsi_subset_create4)."""

    def __init__(self, mesh, xt, mu, nu, sizes, caps, stream=None, lam=None, rho=None, theta=None, dt=None):
        self.mesh = mesh
        self.K = len(sizes)
        self.mu = np.ascontiguousarray(mu, np.float64)
        self.nu = np.ascontiguousarray(nu, np.float64)
        self.sizes = np.ascontiguousarray(sizes, np.int32)
        self.caps = np.ascontiguousarray(caps, np.int32)
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)[:-1]]).astype(np.int64)
        self.h = C.c_void_p()
        if theta is not None:
            _check(load().lrfsi_subset_create_theta(mesh.h, self.K, _ptr(xt), _ptr(self.mu), _ptr(self.nu),
                                                    _ptr(self.sizes), _ptr(self.caps), float(theta), float(dt),
                                                    C.byref(self.h), _stream(stream)))
        elif lam is not None:
            self.lam = np.ascontiguousarray(lam, np.float64)
            self.rho = np.ascontiguousarray(rho, np.float64)
            _check(load().lrfsi_subset_create4(mesh.h, self.K, _ptr(xt), _ptr(self.mu), _ptr(self.nu), _ptr(self.lam),
                                               _ptr(self.rho), _ptr(self.sizes), _ptr(self.caps), C.byref(self.h),
                                               _stream(stream)))
        else:
            _check(load().lrfsi_subset_create(mesh.h, self.K, _ptr(xt), _ptr(self.mu), _ptr(self.nu),
                                              _ptr(self.sizes), _ptr(self.caps), C.byref(self.h), _stream(stream)))

    def close(self):
        if self.h:
            load().lrfsi_subset_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_bytes(self):
        return int(load().lrfsi_subset_bytes(self.h))


def lrfsi_subset_create(mesh, xt, mu, nu, sizes, caps, stream=None):
    return Subsets(mesh, xt, mu, nu, sizes, caps, stream)


def _lowrank_solve(fn, sub, UB, lduB, VB, ldvB, rB, opt, U, ldu, V, ldv, stream):
    rB = np.ascontiguousarray(rB, np.int32)
    ranks = np.zeros(sub.K, np.int32)
    stats = (lrfsi_cheb_stats * sub.K)()
    _check(fn(sub.h, _ptr(UB), lduB, _ptr(VB), ldvB, _ptr(rB), C.byref(opt), _ptr(U), ldu, _ptr(V), ldv,
              _ptr(ranks), C.cast(stats, C.c_void_p), _stream(stream)))
    return ranks, [dict(steps=s.steps, rank=s.rank, rel_lin_res=s.rel_lin_res, max_concat_rank=s.max_concat_rank)
                   for s in stats]


def lrfsi_chebyshevT(sub, UB, lduB, VB, ldvB, rB, opt, U, ldu, V, ldv, stream=None):
    return _lowrank_solve(load().lrfsi_chebyshevT, sub, UB, lduB, VB, ldvB, rB, opt, U, ldu, V, ldv, stream)


def lrfsi_gmresT(sub, UB, lduB, VB, ldvB, rB, opt, U, ldu, V, ldv, stream=None):
    return _lowrank_solve(load().lrfsi_gmresT, sub, UB, lduB, VB, ldvB, rB, opt, U, ldu, V, ldv, stream)


def lrfsi_subset_step(sub, opt, target, max_outer, U, ldu, V, ldv, stream=None, allow_noconv=True):
    ranks = np.zeros(sub.K, np.int32)
    rel = np.zeros(int(sub.sizes.sum()))
    outer = np.zeros(sub.K, np.int32)
    st = load().lrfsi_subset_step(sub.h, C.byref(opt), target, max_outer, _ptr(U), ldu, _ptr(V), ldv, _ptr(ranks),
                                  _ptr(rel), _ptr(outer), _stream(stream))
    _check(st, (ENOCONV,) if allow_noconv else ())
    return ranks, rel, outer, st


def lrfsi_subset_step_init(sub, opt, target, max_outer, U0, ldu0, V0, ldv0, r0, U, ldu, V, ldv, stream=None,
                           allow_noconv=True):
    """lrfsi_subset_step from X0_k = x~_k 1^T + U0_k V0_k^T.  Returns
    (ranks, relres, outer, fallback flags, status)."""
    ranks = np.zeros(sub.K, np.int32)
    rel = np.zeros(int(sub.sizes.sum()))
    outer = np.zeros(sub.K, np.int32)
    fb = np.zeros(int(sub.sizes.sum()), np.int32)
    r0 = np.ascontiguousarray(np.broadcast_to(r0, (sub.K,)), np.int32)
    st = load().lrfsi_subset_step_init(sub.h, C.byref(opt), target, max_outer, _ptr(U0), ldu0, _ptr(V0), ldv0,
                                       _ptr(r0), _ptr(U), ldu, _ptr(V), ldv, _ptr(ranks), _ptr(rel), _ptr(outer),
                                       _ptr(fb), _stream(stream))
    _check(st, (ENOCONV,) if allow_noconv else ())
    return ranks, rel, outer, fb, st


def lrfsi_precond_apply(sub, X, ldx, r, Y, ldy, stream=None):
    r = np.ascontiguousarray(np.broadcast_to(r, (sub.K,)), np.int32)
    _check(load().lrfsi_precond_apply(sub.h, _ptr(X), ldx, _ptr(r), _ptr(Y), ldy, _stream(stream)))


def lrfsi_truncate(sub, X, ldx, V, ldv, p, tol, cap, U, ldu, Vo, ldvo, stream=None):
    p = np.ascontiguousarray(np.broadcast_to(p, (sub.K,)), np.int32)
    cap = np.ascontiguousarray(np.broadcast_to(cap, (sub.K,)), np.int32)
    ranks = np.zeros(sub.K, np.int32)
    _check(load().lrfsi_truncate(sub.h, _ptr(X), ldx, _ptr(V), ldv, _ptr(p), tol, _ptr(cap), _ptr(U), ldu, _ptr(Vo),
                                 ldvo, _ptr(ranks), _stream(stream)))
    return ranks


def kernel_stats():
    """{class name: dict(launches, flops, bytes, ms)} accumulated since the last reset."""
    out = {}
    for i, name in enumerate(KERNEL_CLASSES):
        st = lrfsi_kernel_stat()
        _check(load().lrfsi_stats(i, C.byref(st)))
        out[name] = dict(launches=int(st.launches), flops=st.flops, bytes=st.bytes, ms=st.ms)
    return out


def lrfsi_spmm(mesh, J3, U, ldu, r, Y, ldy, stream=None):
    """Y = [J0 U | Jmu' U | Jnu' U]; FP64 or FP32 tensors (all the same dtype)."""
    import torch
    prec = {torch.float64: 0, torch.float32: 1}[U.dtype]
    _check(load().lrfsi_spmm(mesh.h, _ptr(J3), _ptr(U), ldu, r, _ptr(Y), ldy, prec, _stream(stream)))


def spmm_tuning(precision, bucket):
    v = np.zeros(1, np.int32)
    ms = np.zeros(9, np.float32)
    _check(load().lrfsi_spmm_tuning(precision, bucket, _ptr(v), _ptr(ms)))
    return int(v[0]), ms


def truncation_counters(reset=False):
    out = np.zeros(6, np.int64)
    _check(load().lrfsi_truncation_counters(_ptr(out), int(reset)))
    return dict(zip(("calls", "sweeps_sum", "sweeps_max", "svd_noconv", "breakdowns", "retries"), out.tolist()))


def stats_reset():
    _check(load().lrfsi_stats_reset())


def timing(enable):
    _check(load().lrfsi_timing(1 if enable else 0))


class MLP:
    """The learned-start network (lrfsi_mlp_*): n_in -> n_h1 -> n_h2 -> n_out."""

    def __init__(self, sizes=(2, 128, 128, 64)):
        self.sizes = tuple(sizes)
        self.h = C.c_void_p()
        _check(load().lrfsi_mlp_create(*self.sizes, C.byref(self.h)))
        self.n = int(load().lrfsi_mlp_num_params(self.h))

    def close(self):
        if self.h:
            load().lrfsi_mlp_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, packed):
        packed = np.ascontiguousarray(packed, np.float32)
        assert packed.size == self.n
        _check(load().lrfsi_mlp_set_params(self.h, _ptr(packed)))

    def get_params(self):
        out = np.zeros(self.n, np.float32)
        _check(load().lrfsi_mlp_get_params(self.h, _ptr(out)))
        return out

    def forward(self, Z, Y, B, stream=None):
        _check(load().lrfsi_mlp_forward(self.h, _ptr(Z), B, _ptr(Y), _stream(stream)))

    def gradients(self, Z, T, B, grad, loss=None, stream=None):
        _check(load().lrfsi_mlp_gradients(self.h, _ptr(Z), _ptr(T), B, _ptr(grad), _ptr(loss), _stream(stream)))

    def train(self, Z, T, B, epochs, lr, stream=None):
        loss = np.zeros(1, np.float32)
        _check(load().lrfsi_mlp_train(self.h, _ptr(Z), _ptr(T), B, epochs, C.c_float(lr), _ptr(loss),
                                      _stream(stream)))
        return float(loss[0])


def pack_params(params):
    """Packed layout of lrfsi_mlp_*: W_0, b_0, W_1, b_1, ... (row-major)."""
    return np.concatenate([np.asarray(p, np.float32).ravel() for p in params])


def unpack_params(packed, sizes=(2, 128, 128, 64)):
    out, o = [], 0
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        out.append(packed[o:o + n_in * n_out].reshape(n_out, n_in)); o += n_in * n_out
        out.append(packed[o:o + n_out]); o += n_out
    return out


class LearnedStart:
    """Device state of the learned start: the MLP, Phi, the scales and offset
    (torch tensors on the mesh's device)."""

    def __init__(self, mesh, k=64, hidden=(128, 128), box=None, seed=0, init=None):
        import torch
        from . import inputs
        self.mesh, self.k = mesh, k
        self.box = np.array(box if box is not None else (*inputs.MU_RANGE, *inputs.NU_RANGE), np.float64)
        self.mlp = MLP((2, hidden[0], hidden[1], k))
        if init is None:
            init = inputs.mlp_init((2, hidden[0], hidden[1], k), seed)
        self.mlp.set_params(init)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.Phi = torch.zeros(mesh.M, k, dtype=torch.float64, device=dev)
        self.cs = torch.zeros(k, dtype=torch.float64, device=dev)
        self.fs = torch.zeros(mesh.M, dtype=torch.float64, device=dev)
        self.off = torch.zeros(mesh.M, dtype=torch.float64, device=dev)
        self.loss = None
        self.sigma = None

    def fit(self, X, mu, nu, epochs=500, lr=1e-3, stream=None):
        """X: n x M device tensor of solutions (problem-major)."""
        n = len(mu)
        mu = np.ascontiguousarray(mu, np.float64); nu = np.ascontiguousarray(nu, np.float64)
        loss = np.zeros(1, np.float32); sigma = np.zeros(self.k)
        _check(load().lrfsi_learned_fit(self.mesh.h, self.mlp.h, _ptr(mu), _ptr(nu), n, _ptr(self.box), _ptr(X),
                                        X.stride(0), self.k, epochs, C.c_float(lr), _ptr(self.Phi), self.k,
                                        _ptr(self.cs), _ptr(self.fs), _ptr(self.off), _ptr(loss), _ptr(sigma),
                                        _stream(stream)))
        self.loss, self.sigma = float(loss[0]), sigma
        return self.loss

    def factors(self, sizes, mu, nu, xt, U0, V0, stream=None):
        """Start factors relative to the K median solutions xt (K x M tensor):
        U0 (K*M x (k+1)) and V0 (sum(sizes) x (k+1)) device tensors."""
        sizes = np.ascontiguousarray(sizes, np.int32)
        mu = np.ascontiguousarray(mu, np.float64); nu = np.ascontiguousarray(nu, np.float64)
        _check(load().lrfsi_learned_factors(self.mesh.h, self.mlp.h, len(sizes), _ptr(sizes), _ptr(mu), _ptr(nu),
                                            _ptr(self.box), _ptr(self.Phi), self.k, self.k, _ptr(self.cs),
                                            _ptr(self.fs), _ptr(self.off), _ptr(xt), _ptr(U0), self.k + 1,
                                            _ptr(V0), self.k + 1, _stream(stream)))

    def start(self, mu, nu, X, stream=None):
        """Fill X (B x M device tensor) with the start; returns the fallback flags."""
        B = len(mu)
        mu = np.ascontiguousarray(mu, np.float64); nu = np.ascontiguousarray(nu, np.float64)
        fb = np.zeros(B, np.int32)
        _check(load().lrfsi_learned_start(self.mesh.h, self.mlp.h, _ptr(mu), _ptr(nu), B, _ptr(self.box),
                                          _ptr(self.Phi), self.k, self.k, _ptr(self.cs), _ptr(self.fs),
                                          _ptr(self.off), _ptr(X), _ptr(fb), _stream(stream)))
        return fb


def lrfsi_pod(mesh, X, ldx, n, k, Phi, ldphi, Cm, ldc, stream=None):
    sigma = np.zeros(k)
    _check(load().lrfsi_pod(mesh.h, _ptr(X), ldx, n, k, _ptr(Phi), ldphi, _ptr(Cm), ldc, _ptr(sigma),
                            _stream(stream)))
    return sigma
