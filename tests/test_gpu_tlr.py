"""GPU parity of the CUDA path against the CPU oracle (through the C ABI)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense as DN
from oracle import matern as M
from oracle import tlr as TL
from paper_1804_09137_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    from paper_1804_09137_gb300 import tlr

    return tlr


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def problem(side, theta, n=None):
    x, y = inputs.jittered_grid(side, n=n)
    z = DN.sample(x, y, theta, inputs.standard_normal(len(x)))
    return x, y, z


@pytest.mark.parametrize("theta", [(1.0, 0.1, 0.5), (1.0, 0.3, 1.0), (1.7, 0.05, 1.5), (0.6, 0.2, 0.8)])
def test_generation_matches_oracle(T, theta):
    x, y = inputs.jittered_grid(20)  # n = 400, tiles of 96 (last ragged: 16)
    h = T.Handle(dev(x), dev(y), nb=96, eps=1e-9)
    h.matern_generate(theta)
    p = h.get_perm().cpu().numpy()
    xs, ys = x[p], y[p]
    S = DN.covariance(xs, ys, theta)
    nb = 96
    for i in range(h.nt):
        D, _ = h.get_tile(i, i)
        D = D.cpu().numpy()
        m = min(nb, len(x) - i * nb)
        ref = S[i * nb:i * nb + m, i * nb:i * nb + m]
        assert np.max(np.abs(D[:m, :m] - ref)) <= 1e-13 * theta[0]
        # padded points are identity points
        assert np.allclose(D[m:, m:], np.eye(nb - m)) and np.all(D[:m, m:] == 0)


@pytest.mark.parametrize("theta,eps", [((1.0, 0.1, 0.5), 1e-9), ((1.0, 0.3, 1.0), 1e-7), ((1.0, 0.03, 0.5), 1e-5)])
def test_compression_error_bound(T, theta, eps):
    x, y = inputs.jittered_grid(24)  # n = 576, 5 tiles of 128 (last 64)
    nb = 128
    h = T.Handle(dev(x), dev(y), nb=nb, eps=eps, rank_cap=nb)
    h.matern_generate(theta)
    h.compress()
    h.check()
    p = h.get_perm().cpu().numpy()
    S = DN.covariance(x[p], y[p], theta)
    n = len(x)
    for i in range(h.nt):
        for j in range(i):
            U, V = h.get_tile(i, j)
            A = np.zeros((nb, nb))
            ri, rj = min(nb, n - i * nb), min(nb, n - j * nb)
            A[:ri, :rj] = S[i * nb:i * nb + ri, j * nb:j * nb + rj]
            if V is None:  # stored dense: exact generation
                assert np.max(np.abs(U.cpu().numpy() - A)) <= 1e-13
                continue
            U, V = U.cpu().numpy(), V.cpu().numpy()
            err = np.linalg.norm(A - U @ V.T, 2)
            assert err <= 2.0 * eps, (i, j, err)
            s = np.linalg.svd(A, compute_uv=False)
            k_opt = int(np.sum(s > eps))
            assert U.shape[1] <= k_opt + 3, (i, j, U.shape[1], k_opt)  # pivoted-QR truncation is near optimal


@pytest.mark.parametrize("theta", [(1.0, 0.1, 0.5), (1.0, 0.3, 1.0)])
def test_loglik_small_eps_matches_dense(T, theta):
    x, y, z = problem(30, theta, n=880)  # 7 tiles of 128, last ragged
    ll, ld, q = DN.loglik(x, y, z, theta)
    h = T.Handle(dev(x), dev(y), nb=128, eps=1e-12, rank_cap=128)
    h.factor(theta)
    out = h.loglik(dev(z)).cpu().numpy()
    h.check()
    assert abs(out[0] - ll) <= 1e-9 * abs(ll)
    assert abs(out[1] - ld) <= 1e-9 * abs(ld)
    assert abs(out[2] - q) <= 1e-8 * abs(q)


def test_arena_grows_and_results_stay_exact(T):
    """At eps = 1e-13 with dense_rank 80 the ranks outgrow the low-rank arena's starting size (32 columns a
    tile): compression and the factorization enlarge it and repeat, and l and the gradient still match
    the exact oracle."""
    theta = (1.0, 0.1, 0.5)
    x, y, z = problem(26, theta, n=650)
    ll_ref, g_ref = DN.loglik_grad(x, y, z, theta)
    h = T.Handle(dev(x), dev(y), nb=96, eps=1e-13, rank_cap=96, dense_rank=80)
    m0 = h.memory()
    h.factor(theta)
    ll, g = h.loglik_grad(dev(z))
    h.check()
    m1 = h.memory()
    assert h.rank_stats()["kmax"] > 32 and m1["arenas"] > m0["arenas"], (h.rank_stats(), m0, m1)
    assert 0 < m1["arena_used"] <= m1["arenas"] < m1["total"]
    ll, g = ll.cpu().numpy()[0], g.cpu().numpy()
    assert abs(ll - ll_ref) <= 1e-9 * abs(ll_ref)
    np.testing.assert_allclose(g, g_ref, rtol=1e-6, atol=1e-6 * np.max(np.abs(g_ref)))
    # a second evaluation on the enlarged arena gives the same numbers bit for bit
    h.factor(theta)
    ll2, g2 = h.loglik_grad(dev(z))
    assert ll2.cpu().numpy()[0] == ll and np.array_equal(g2.cpu().numpy(), g)
    h.close()


@pytest.mark.parametrize("dense_rank", [4, 16, 120])
def test_dense_threshold_does_not_change_result(T, dense_rank):
    theta = (1.0, 0.3, 1.0)
    x, y, z = problem(30, theta, n=850)
    ll = DN.loglik(x, y, z, theta)[0]
    h = T.Handle(dev(x), dev(y), nb=128, eps=1e-11, rank_cap=128, dense_rank=dense_rank)
    h.factor(theta)
    out = h.loglik(dev(z)).cpu().numpy()
    h.check()
    cnt = h.tile_counts()
    assert cnt["dense"] + cnt["lowrank"] == h.nt * (h.nt - 1) // 2
    assert abs(out[0] - ll) <= 1e-8 * abs(ll), (out[0], ll, cnt)


@pytest.mark.parametrize("theta", [(1.0, 0.1, 0.5), (1.0, 0.3, 1.0)])
def test_dense_mode_matches_oracle(T, theta):
    # eps < 0: every tile dense, the exact full-tile comparator
    x, y, z = problem(30, theta, n=870)
    ll, ld, q = DN.loglik(x, y, z, theta)
    h = T.Handle(dev(x), dev(y), nb=96, eps=-1.0)
    h.factor(theta)
    out = h.loglik(dev(z)).cpu().numpy()
    h.check()
    assert h.tile_counts()["lowrank"] == 0
    assert abs(out[0] - ll) <= 1e-10 * abs(ll)
    assert abs(out[1] - ld) <= 1e-10 * abs(ld)


def test_single_tile_is_dense(T):
    theta = (1.3, 0.2, 0.7)
    x, y, z = problem(15, theta)
    ll = DN.loglik(x, y, z, theta)[0]
    h = T.Handle(dev(x), dev(y), nb=256, eps=1e-3)
    h.factor(theta)
    out = h.loglik(dev(z)).cpu().numpy()
    assert abs(out[0] - ll) <= 1e-11 * abs(ll)


def test_full_rank_equals_dense(T):
    # eps = 0 with rank_cap = nb keeps every nonzero singular value
    theta = (1.0, 0.1, 0.5)
    x, y, z = problem(16, theta)
    ll = DN.loglik(x, y, z, theta)[0]
    h = T.Handle(dev(x), dev(y), nb=64, eps=0.0, rank_cap=64)
    h.factor(theta)
    out = h.loglik(dev(z)).cpu().numpy()
    h.check()
    assert abs(out[0] - ll) <= 1e-11 * abs(ll)


@pytest.mark.parametrize("eps", [1e-5, 1e-7])
def test_loglik_matches_cpu_tlr_reference(T, eps):
    theta = (1.0, 0.3, 1.0)
    x, y, z = problem(32, theta)
    nb = 128
    ll_cpu = TL.loglik(x, y, z, theta, nb=nb, eps=eps)[0]
    ll_d = DN.loglik(x, y, z, theta)[0]
    h = T.Handle(dev(x), dev(y), nb=nb, eps=eps, rank_cap=nb)
    h.factor(theta)
    out = h.loglik(dev(z)).cpu().numpy()
    h.check()
    # both approximations sit within the same eps-driven distance of the exact value
    tol = max(5 * abs(ll_cpu - ll_d), 1e-9 * abs(ll_d))
    assert abs(out[0] - ll_d) <= tol, (out[0], ll_cpu, ll_d)


def test_kriging_matches_oracle(T):
    theta = (1.0, 0.1, 0.5)
    x, y, z = problem(30, theta)
    obs, held = inputs.holdout(len(x), 90)
    want = DN.krige(x[obs], y[obs], z[obs], x[held], y[held], theta)
    h = T.Handle(dev(x[obs]), dev(y[obs]), nb=128, eps=1e-12, rank_cap=128)
    h.factor(theta)
    got = h.predict(dev(z[obs]), dev(x[held]), dev(y[held])).cpu().numpy()
    h.check()
    np.testing.assert_allclose(got, want, rtol=1e-8, atol=1e-9)


def test_prediction_variance_matches_oracle(T):
    """Multi-right-hand-side solve: 810 observed points in 7 tiles of 128 (ragged last), 90 new points
    (two column chunks would be the same code path); TLR at eps = 1e-12 and the dense path."""
    theta = (1.0, 0.1, 0.5)
    x, y = inputs.jittered_grid(30)
    obs, held = inputs.holdout(len(x), 90)
    want = DN.krige_var(x[obs], y[obs], x[held], y[held], theta)
    for eps, cap in ((1e-12, 128), (-1.0, 0)):
        h = T.Handle(dev(x[obs]), dev(y[obs]), nb=128, eps=eps, rank_cap=cap)
        h.factor(theta)
        got = h.predict_var(dev(x[held]), dev(y[held])).cpu().numpy()
        h.check()
        np.testing.assert_allclose(got, want, rtol=1e-7, atol=1e-9)
        # at observed locations the variance vanishes (no nugget)
        v0 = h.predict_var(dev(x[obs[:7]]), dev(y[obs[:7]])).cpu().numpy()
        assert np.all(np.abs(v0) <= 1e-7)
        h.close()


def test_batched_prediction_variance_dense_tiles_matches_oracle(T):
    """The batched multi-right-hand-side forward solve at tile size 256 with dense off-diagonal tiles
    (dense_rank 24): 2,500 observed points in 10 tiles, 1,500 new points (two batches of right-hand sides,
    the second ragged), against the exact conditional variance; a second call gives the same bits."""
    theta = (1.0, 0.1, 0.5)
    x, y = inputs.jittered_grid(50)
    xn, yn = inputs.uniform_points(1500)
    want = DN.krige_var(x, y, xn, yn, theta)
    h = T.Handle(dev(x), dev(y), nb=256, eps=1e-11, rank_cap=256, dense_rank=24)
    h.factor(theta)
    cnt = h.tile_counts()
    assert cnt["dense"] > 0 and cnt["lowrank"] > 0, cnt
    got = h.predict_var(dev(xn), dev(yn)).cpu().numpy()
    again = h.predict_var(dev(xn), dev(yn)).cpu().numpy()
    h.check()
    np.testing.assert_allclose(got, want, rtol=1e-6, atol=1e-8)
    assert np.array_equal(got, again)
    h.close()


def test_sample_is_cholesky_times_e(T):
    theta = (1.0, 0.1, 0.5)
    x, y = inputs.jittered_grid(18)
    e = inputs.standard_normal(len(x))
    want = DN.sample(x, y, theta, e)
    h = T.Handle(dev(x), dev(y), nb=100, eps=1e-13, rank_cap=100, order=False)
    h.factor(theta)
    got = h.sample(dev(e)).cpu().numpy()
    np.testing.assert_allclose(got, want, atol=1e-9)


def test_not_spd_reported(T):
    x, y = inputs.jittered_grid(10)
    x = np.concatenate([x, x[:3]])  # duplicated locations: singular Sigma
    y = np.concatenate([y, y[:3]])
    h = T.Handle(dev(x), dev(y), nb=64, eps=1e-12, rank_cap=64)
    h.factor((1.0, 0.1, 0.5))
    rc, info = h.status()
    assert rc == T.TLR_ERR_NOT_SPD and info >= 1


def test_rank_cap_reported(T):
    # eps-ranks 10..42 (oracle SVD), several in 13..20: low rank allowed above 12 but storage capped at 12
    x, y = inputs.jittered_grid(24)
    h = T.Handle(dev(x), dev(y), nb=64, eps=1e-6, rank_cap=12, dense_rank=16)
    h.matern_generate((1.0, 0.3, 1.0))
    h.compress()
    rc, _ = h.status()
    assert rc == T.TLR_ERR_RANK_CAP


def test_calls_out_of_order(T):
    x, y = inputs.jittered_grid(8)
    h = T.Handle(dev(x), dev(y), nb=32, eps=1e-9)
    z = dev(np.ones(len(x)))
    with pytest.raises(T.TlrError):
        h.loglik(z)
    with pytest.raises(T.TlrError):
        h.potrf()


@pytest.mark.parametrize("theta", [(1.0, 0.1, 0.5), (1.0, 0.3, 1.0), (0.7, 0.15, 1.4)])
def test_gradient_matches_oracle(T, theta):
    x, y, z = problem(26, theta, n=650)
    ll_ref, g_ref = DN.loglik_grad(x, y, z, theta)
    h = T.Handle(dev(x), dev(y), nb=96, eps=1e-12, rank_cap=96)
    h.factor(theta)
    ll, g = h.loglik_grad(dev(z))
    h.check()
    ll, g = ll.cpu().numpy()[0], g.cpu().numpy()
    assert abs(ll - ll_ref) <= 1e-9 * abs(ll_ref)
    np.testing.assert_allclose(g, g_ref, rtol=1e-6, atol=1e-6 * np.max(np.abs(g_ref)))


def test_gradient_dense_mode(T):
    theta = (1.0, 0.3, 1.0)
    x, y, z = problem(24, theta, n=560)
    _, g_ref = DN.loglik_grad(x, y, z, theta)
    h = T.Handle(dev(x), dev(y), nb=80, eps=-1.0)
    h.factor(theta)
    _, g = h.loglik_grad(dev(z))
    h.check()
    np.testing.assert_allclose(g.cpu().numpy(), g_ref, rtol=1e-8, atol=1e-8 * np.max(np.abs(g_ref)))


def test_gradient_finite_differences_of_gpu_loglik(T):
    theta = np.array([1.0, 0.2, 0.8])
    x, y, z = problem(30, tuple(theta), n=880)
    h = T.Handle(dev(x), dev(y), nb=128, eps=1e-12, rank_cap=128)
    zt = dev(z)
    h.factor(theta)
    _, g = h.loglik_grad(zt)
    g = g.cpu().numpy()
    for p in range(3):
        hp = 1e-6 * theta[p]
        vals = []
        for sgn in (1, -1):
            th = theta.copy()
            th[p] += sgn * hp
            h.factor(th)
            vals.append(h.loglik(zt).cpu().numpy()[0])
        fd = (vals[0] - vals[1]) / (2 * hp)
        assert abs(g[p] - fd) <= 1e-5 * max(abs(fd), 1.0), (p, g[p], fd)


def test_great_circle_distance_matches_oracle(T):
    """Eq. 6 distances (x = longitude, y = latitude in degrees, radius 6371 km): l in dense mode and in
    TLR form, and kriging, against the oracle on 576 points of a 20 x 20 degree region."""
    theta, radius = (1.0, 400.0, 1.0), 6371.0
    u, v = inputs.jittered_grid(24)
    lon, lat = 30.0 + 20.0 * u, 10.0 + 20.0 * v
    z = DN.sample(lon, lat, theta, inputs.standard_normal(len(lon)), radius=radius)
    obs, held = inputs.holdout(len(lon), 40)
    want, _, _ = DN.loglik(lon[obs], lat[obs], z[obs], theta, radius=radius)
    kw = DN.krige(lon[obs], lat[obs], z[obs], lon[held], lat[held], theta, radius=radius)
    for eps, cap, tol in ((-1.0, 0, 1e-10), (1e-12, 96, 1e-9)):
        h = T.Handle(dev(lon[obs]), dev(lat[obs]), nb=96, eps=eps, rank_cap=cap, radius=radius)
        h.factor(theta)
        got = h.loglik(dev(z[obs]))[0].item()
        h.check()
        assert abs(got - want) <= tol * abs(want)
        kg = h.predict(dev(z[obs]), dev(lon[held]), dev(lat[held])).cpu().numpy()
        np.testing.assert_allclose(kg, kw, rtol=1e-7, atol=1e-8)
        h.close()


_CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1804_09137_gb300 import inputs, tlr as T
from oracle import dense as DN
theta = (1.0, 0.1, 0.5)
x, y = inputs.jittered_grid(50)
z = DN.sample(x, y, theta, inputs.standard_normal(len(x)))
d = lambda a: torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")
h = T.Handle(d(x), d(y), nb=256, eps=1e-9, rank_cap=128, dense_rank=48)
h.factor(theta)
ll, g = h.loglik_grad(d(z))
h.check()
print(" ".join(float(v).hex() for v in [ll.item(), *g.cpu().numpy()]))
"""


def test_cluster_split_equals_one_cta_bit_for_bit(T):
    """The low-rank update items split over two-CTA clusters (default) and on one CTA each (the environment
    variable TLR_UPD_PAIR=0, read once per process) run the same arithmetic: l and the gradient agree bit for
    bit (n = 2,500, 10 tiles, eps = 1e-9)."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = []
    for mode in ("1", "0"):
        env = dict(os.environ, TLR_UPD_PAIR=mode)
        r = subprocess.run([sys.executable, "-c", _CHILD, root], env=env, capture_output=True, text=True,
                           timeout=600, cwd=root)
        assert r.returncode == 0, r.stderr[-2000:]
        out.append(r.stdout.strip().splitlines()[-1])
    assert out[0] == out[1], out


def test_lauum_overlapped_reduction_matches_epilogue_reduction(T):
    """The gradient's reduction of each LAUUM batch by its own kernel beside the next batch's products
    (default) and inside the tensor-core epilogue (TLR_LAUUM_OVERLAP=0) sum the same entries in another
    order, the first with double-float derivative polynomials: l and dl/dsigma2 agree bit for bit, dl/dbeta
    and dl/dnu to 1e-9 relative (n = 2,500, 10 tiles, eps = 1e-9)."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    vals = []
    for mode in ("1", "0"):
        env = dict(os.environ, TLR_LAUUM_OVERLAP=mode)
        r = subprocess.run([sys.executable, "-c", _CHILD, root], env=env, capture_output=True, text=True,
                           timeout=600, cwd=root)
        assert r.returncode == 0, r.stderr[-2000:]
        vals.append([float.fromhex(v) for v in r.stdout.strip().splitlines()[-1].split()])
    (l1, s1, b1, n1), (l0, s0, b0, n0) = vals
    assert l1 == l0 and s1 == s0
    assert abs(b1 - b0) <= 1e-9 * abs(b0) and abs(n1 - n0) <= 1e-9 * abs(n0), vals
