"""Learned initial guess on the GPU (lrfsi_mlp_*, lrfsi_pod, lrfsi_learned_*)
against the oracle (oracle/mlp.py) and against properties of the method.

Tolerances: the MLP runs in FP32 with BF16 weights on both sides (the oracle
rounds the same weights to BF16, ties to even, and accumulates in FP64), so
outputs and gradients agree to FP32 accumulation error over <= 128 terms:
1e-4 relative to the largest entry.  POD singular values are an FP64
Cholesky-QR + Jacobi result: 1e-10 relative."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fsi, mlp as omlp  # noqa: E402
from paper_2008_10275_gb300 import build, inputs, lrfsi  # noqa: E402
from tests.gpu_common import perm_lib_to_oracle  # noqa: E402

DEV = "cuda:0"
SIZES = (2, 128, 128, 64)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    lrfsi.load()


def _f32(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32), device=DEV)


def _params(seed=1):
    packed = inputs.mlp_init(SIZES, seed)
    rng = np.random.default_rng(seed + 100)
    ps = lrfsi.unpack_params(packed.copy(), SIZES)
    for i in range(1, len(ps), 2):  # nonzero biases so the bias path is exercised
        ps[i][:] = 0.1 * rng.standard_normal(ps[i].shape)
    return lrfsi.pack_params(ps)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_mlp_forward_parity():
    packed = _params()
    net = lrfsi.MLP(SIZES)
    net.set_params(packed)
    assert np.array_equal(net.get_params(), packed)
    for B in (1, 37, 300):
        Z = np.random.default_rng(B).uniform(-1, 1, (B, 2)).astype(np.float32)
        Y = torch.zeros(B, SIZES[-1], dtype=torch.float32, device=DEV)
        net.forward(_f32(Z), Y, B)
        Yo, _ = omlp.forward(lrfsi.unpack_params(packed, SIZES), Z, dtype=np.float64, bf16=True)
        assert _rel(Y.cpu().numpy(), Yo) <= 1e-4


def test_mlp_gradients_parity():
    packed = _params(2)
    net = lrfsi.MLP(SIZES)
    net.set_params(packed)
    B = 53
    rng = np.random.default_rng(4)
    Z = rng.uniform(-1, 1, (B, 2)).astype(np.float32)
    T = rng.standard_normal((B, SIZES[-1])).astype(np.float32)
    G = torch.zeros(net.n, dtype=torch.float32, device=DEV)
    L = torch.zeros(1, dtype=torch.float32, device=DEV)
    net.gradients(_f32(Z), _f32(T), B, G, L)
    Yo, cache = omlp.forward(lrfsi.unpack_params(packed, SIZES), Z, dtype=np.float64, bf16=True)
    go = omlp.backward(cache, Yo, T)
    gg = lrfsi.unpack_params(G.cpu().numpy(), SIZES)
    for a, b in zip(gg, go):
        assert _rel(a, b) <= 1e-4
    assert float(L.cpu()[0]) == pytest.approx(omlp.loss(Yo, T), rel=1e-5)


def test_mlp_first_adam_step_matches_oracle():
    packed = _params(3)
    net = lrfsi.MLP(SIZES)
    net.set_params(packed)
    B = 40
    rng = np.random.default_rng(5)
    Z = rng.uniform(-1, 1, (B, 2)).astype(np.float32)
    T = rng.standard_normal((B, SIZES[-1])).astype(np.float32)
    lr = 1e-3
    net.train(_f32(Z), _f32(T), B, 1, lr)
    p1 = net.get_params()
    ps = [p.astype(np.float64) for p in lrfsi.unpack_params(packed, SIZES)]
    Yo, cache = omlp.forward(ps, Z, dtype=np.float64, bf16=True)
    go = omlp.backward(cache, Yo, T)
    state = ([np.zeros_like(p) for p in ps], [np.zeros_like(p) for p in ps], 0)
    po, _ = omlp.adam_step(ps, go, state, lr=lr)
    d_gpu = p1 - packed
    d_ora = lrfsi.pack_params(po).astype(np.float64) - packed
    g = np.abs(lrfsi.pack_params(go))
    sel = g > 1e-3 * g.max()  # the first Adam step is ~ -lr sign(g): compare where the sign is decided
    assert sel.sum() > 0.5 * g.size
    assert np.max(np.abs(d_gpu[sel] - d_ora[sel])) <= 1e-3 * lr + 2e-7


def test_mlp_training_reduces_loss():
    net = lrfsi.MLP((2, 32, 32, 4))
    net.set_params(inputs.mlp_init((2, 32, 32, 4), 0))
    B = 128
    rng = np.random.default_rng(6)
    Z = rng.uniform(-1, 1, (B, 2)).astype(np.float32)
    T = np.stack([np.sin(2 * Z[:, 0]), Z[:, 0] * Z[:, 1], np.cos(Z[:, 1]), Z[:, 0] ** 2], 1).astype(np.float32)
    l0 = net.train(_f32(Z), _f32(T), B, 1, 1e-3)
    l1 = net.train(_f32(Z), _f32(T), B, 800, 3e-3)
    assert l1 < 0.05 * l0


def test_pod_matches_dense_svd():
    mesh = lrfsi.Mesh(20, 4)
    M, n, k = mesh.M, 48, 12
    rng = np.random.default_rng(7)
    Q1, _ = np.linalg.qr(rng.standard_normal((M, n)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = 10.0 ** (-0.25 * np.arange(n))
    X = (Q1 * s) @ Q2.T
    Xd = torch.as_tensor(X, device=DEV)
    Phi = torch.zeros(M, k, dtype=torch.float64, device=DEV)
    Cm = torch.zeros(n, k, dtype=torch.float64, device=DEV)
    sig = lrfsi.lrfsi_pod(mesh, Xd, n, n, k, Phi, k, Cm, k)
    assert np.allclose(sig, s[:k], rtol=1e-10, atol=0)
    P = Phi.cpu().numpy()
    assert np.max(np.abs(P.T @ P - np.eye(k))) <= 1e-12
    # the projector onto the leading k left singular vectors (gap 10^0.25).
    # The truncation drops directions whose pivoted-Cholesky remainder is below
    # sqrt(1e-14) of the column norm (E with ||E|| ~ 1e-7 sigma_1); E lies in
    # the trailing singular directions, so it moves the leading subspace only
    # in second order, ~ (||E|| / gap)^2 ~ 1e-8.
    Pe = Q1[:, :k] @ Q1[:, :k].T
    assert np.max(np.abs(P @ P.T - Pe)) <= 1e-6
    err = np.linalg.norm(X - P @ Cm.cpu().numpy().T)
    assert err == pytest.approx(np.sqrt(np.sum(s[k:] ** 2)), rel=1e-8)


@pytest.mark.parametrize("k", [20, 40])
def test_pod_many_snapshots_of_low_rank(k):
    """400 snapshots of exact rank 30: the p x m bound of the Jacobi matrix
    (400 x 400) is far beyond shared memory while the matrix of the pass-1
    rank (30 x 400) fits it, so the QR preconditioning works in shared memory
    sized by the launch; k = 40 asks for more than the rank (zero-filled)."""
    mesh = lrfsi.Mesh(40, 8)
    M, n, r = mesh.M, 400, 30
    rng = np.random.default_rng(17)
    Q1, _ = np.linalg.qr(rng.standard_normal((M, r)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, r)))
    s = 10.0 ** (-0.1 * np.arange(r))
    X = (Q1 * s) @ Q2.T
    Xd = torch.as_tensor(X, device=DEV)
    Phi = torch.zeros(M, k, dtype=torch.float64, device=DEV)
    Cm = torch.zeros(n, k, dtype=torch.float64, device=DEV)
    sig = lrfsi.lrfsi_pod(mesh, Xd, n, n, k, Phi, k, Cm, k)
    kr = min(k, r)
    assert np.allclose(sig[:kr], s[:kr], rtol=1e-10, atol=0)
    assert np.all(sig[kr:] == 0)
    P = Phi.cpu().numpy()
    assert np.max(np.abs(P[:, :kr].T @ P[:, :kr] - np.eye(kr))) <= 1e-12
    assert np.all(P[:, kr:] == 0)
    err = np.linalg.norm(X - P @ Cm.cpu().numpy().T)
    assert err <= 1e-9 * s[0] + 1.000001 * np.sqrt(np.sum(s[kr:] ** 2))


def _newton(mesh, mus, nus, X0):
    """GPU Newton in chunks of <= 32 parameters; returns solutions and steps."""
    X = X0.clone()
    its = []
    for a in range(0, len(mus), 32):
        it, res, _ = lrfsi.lrfsi_newton_median(mesh, X[a:a + 32], mus[a:a + 32], nus[a:a + 32], 1e-9, 30)
        assert np.all(res <= 1e-9)
        its.append(it)
    return X, np.concatenate(its)


def test_learned_start_fit_and_start():
    mesh = lrfsi.Mesh(20, 4)
    M = mesh.M
    bD = torch.as_tensor(mesh.dirichlet(), device=DEV)
    mu_t, nu_t = inputs.latin_hypercube(64, seed=11)
    Xs, it_train = _newton(mesh, mu_t, nu_t, bD.repeat(64, 1))
    k = 16
    ls = lrfsi.LearnedStart(mesh, k=k, seed=0)
    loss = ls.fit(Xs, mu_t, nu_t, epochs=1500, lr=2e-3)
    assert np.isfinite(loss) and loss < 0.05
    # the fitted pieces follow their definitions
    Xh = Xs.cpu().numpy()
    off = Xh.mean(0)
    assert np.allclose(ls.off.cpu().numpy(), off, rtol=0, atol=1e-12 * np.abs(Xh).max())
    field, _, _ = mesh.dofmap()
    fs = ls.fs.cpu().numpy()
    for f in range(5):
        sel = field == f
        rms = np.sqrt(np.mean((Xh[:, sel] - off[sel]) ** 2))
        assert fs[sel][0] == pytest.approx(rms if rms > 0 else 1.0, rel=1e-10)
        assert np.all(fs[sel] == fs[sel][0])
    Y = (Xh - off) / fs
    sv = np.linalg.svd(Y.T, compute_uv=False)
    assert np.allclose(ls.sigma, sv[:k], rtol=1e-9)
    Phi = ls.Phi.cpu().numpy()
    assert np.max(np.abs(Phi.T @ Phi - np.eye(k))) <= 1e-12

    # the start: its formula against the oracle MLP, then fewer Newton steps
    mu_e, nu_e = inputs.uniform_parameters(24, seed=12)
    X0 = torch.zeros(24, M, dtype=torch.float64, device=DEV)
    fb = ls.start(mu_e, nu_e, X0)
    Z = omlp.scale_params(mu_e, nu_e, inputs.MU_RANGE, inputs.NU_RANGE)
    c, _ = omlp.forward(lrfsi.unpack_params(ls.mlp.get_params(), (2, 128, 128, k)), Z, np.float64, True)
    x_ref = off + fs * ((c * ls.cs.cpu().numpy()) @ Phi.T)
    bDh = mesh.dirichlet()
    om = fsi.Mesh(fsi.Problem(20, 4))
    inv = np.argsort(perm_lib_to_oracle(mesh, om))  # oracle index -> library index
    ident = inv[om.ident_rows]
    x_ref[:, ident] = bDh[ident]
    X0h = X0.cpu().numpy()
    for b in range(24):
        if fb[b]:
            assert np.array_equal(X0h[b], bDh)
        else:
            assert _rel(X0h[b], x_ref[b]) <= 1e-4
    # the residual norm weighs displacement errors by lambda_s: a column may
    # keep b_D (exact zero displacement) although its learned start is closer
    # in the solution; such columns fall back, most do not
    assert fb.sum() <= len(fb) // 4
    Xl, it_l = _newton(mesh, mu_e, nu_e, X0)
    Xb, it_b = _newton(mesh, mu_e, nu_e, bD.repeat(24, 1))
    assert it_l.sum() < it_b.sum()
    assert np.all(it_l <= it_b)
    # Newton's solution does not depend on the start
    assert _rel(Xl.cpu().numpy(), Xb.cpu().numpy()) <= 1e-7


def test_learned_start_of_the_subset_step_saves_corrections():
    """What the trained network gains: the subset step started from the
    learned start (lrfsi_subset_step_init) needs fewer correction steps than
    the plain step from the median solution, reaches the same target in every
    column and lands on the same solutions."""
    mesh = lrfsi.Mesh(20, 4)
    M = mesh.M
    bD = torch.as_tensor(mesh.dirichlet(), device=DEV)
    mu_t, nu_t = inputs.latin_hypercube(96, seed=21)
    Xs, _ = _newton(mesh, mu_t, nu_t, bD.repeat(96, 1))
    k = 16
    ls = lrfsi.LearnedStart(mesh, k=k, seed=1)
    ls.fit(Xs, mu_t, nu_t, epochs=2000, lr=2e-3)
    # evaluation: 3 subsets of 16 held-out parameters (ordered by mu_s) in the
    # middle of the box, where the chord corrections of the plain step
    # converge in a few steps
    mu_e, nu_e = inputs.uniform_parameters(48, seed=22)
    mu_e = 8e5 + (mu_e - inputs.MU_RANGE[0]) / (inputs.MU_RANGE[1] - inputs.MU_RANGE[0]) * 6e5
    nu_e = 2.5e-3 + (nu_e - inputs.NU_RANGE[0]) / (inputs.NU_RANGE[1] - inputs.NU_RANGE[0]) * 1e-3
    o = np.argsort(mu_e)
    mu_e, nu_e = mu_e[o], nu_e[o]
    K, m, R = 3, 16, 20
    sizes = [m] * K
    med = [q * m + m // 2 for q in range(K)]
    X = bD.repeat(K, 1)
    lrfsi.lrfsi_newton_median(mesh, X, mu_e[med], nu_e[med], 1e-10, 30)
    opt = lrfsi.cheb_options(0.65, 1.0, iters=6, cycles=2, rank_cap=R, tol=1e-8, eta=0.05)
    target = 1e-6
    res = {}
    for mode in ("plain", "learned"):
        sub = lrfsi.Subsets(mesh, X, mu_e, nu_e, sizes, [R] * K)
        U = torch.zeros(K * M * R, dtype=torch.float64, device=DEV)
        V = torch.zeros(K * m * R, dtype=torch.float64, device=DEV)
        if mode == "plain":
            ranks, rel, outer, st = lrfsi.lrfsi_subset_step(sub, opt, target, 40, U, R, V, R)
            fb = None
        else:
            U0 = torch.zeros(K * M * (k + 1), dtype=torch.float64, device=DEV)
            V0 = torch.zeros(K * m * (k + 1), dtype=torch.float64, device=DEV)
            ls.factors(sizes, mu_e, nu_e, X, U0, V0)
            ranks, rel, outer, fb, st = lrfsi.lrfsi_subset_step_init(sub, opt, target, 40, U0, k + 1, V0, k + 1,
                                                                     k + 1, U, R, V, R)
        assert st == 0 and np.all(rel <= target), (mode, outer, rel.max())
        cols = []
        for q in range(K):
            Uq = U[q * M * R:(q + 1) * M * R].view(M, R)[:, :ranks[q]]
            Vq = V[q * m * R:(q + 1) * m * R].view(m, R)[:, :ranks[q]]
            cols.append(X[q][:, None] + Uq @ Vq.T)
        res[mode] = (outer.copy(), torch.cat(cols, 1).cpu().numpy(), fb)
        sub.close()
    # the plain step counts its first Newton step as a ChebyshevT solve plus
    # the corrections; the learned step replaces that first step
    plain_solves = res["plain"][0].sum() + K
    learned_solves = res["learned"][0].sum()
    assert learned_solves < plain_solves, (res["plain"][0], res["learned"][0])
    assert res["learned"][2].sum() <= len(mu_e) // 4
    Xp, Xl = res["plain"][1], res["learned"][1]
    # both solve R(x_i) = 0 to a relative residual of 1e-6; the solutions agree
    # to that order relative to the size of the correction from b_D
    d = np.abs(Xp - Xl).max() / np.abs(Xp - mesh.dirichlet()[:, None]).max()
    assert d <= 1e-4
