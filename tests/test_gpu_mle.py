"""autograd.Function gradient and the L-BFGS-B MLE loop against the oracle (GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense as DN
from paper_1804_09137_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    from paper_1804_09137_gb300 import mle, tlr

    return mle, tlr


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def test_autograd_function_backward(M):
    mle, T = M
    theta = (1.0, 0.2, 0.8)
    x, y = inputs.jittered_grid(20)
    z = DN.sample(x, y, theta, inputs.standard_normal(len(x)))
    h = T.Handle(dev(x), dev(y), nb=100, eps=1e-12, rank_cap=100)
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    ll = mle.loglik(th, h, dev(z))
    ll.backward()
    ll_ref, g_ref = DN.loglik_grad(x, y, z, theta)
    assert abs(ll.item() - ll_ref) <= 1e-9 * abs(ll_ref)
    np.testing.assert_allclose(th.grad.numpy(), g_ref, rtol=1e-6, atol=1e-6 * np.abs(g_ref).max())


def test_mle_matches_oracle_mle(M):
    # n = 400 from theta0 = (1, 0.1, 0.5); both optimisers start at (0.5, 0.05, 0.8)
    from scipy.optimize import minimize

    mle, T = M
    truth = (1.0, 0.1, 0.5)
    x, y = inputs.jittered_grid(20)
    z = DN.sample(x, y, truth, inputs.standard_normal(len(x)))
    start = (0.5, 0.05, 0.8)

    def f(th):
        ll, g = DN.loglik_grad(x, y, z, th)
        return -ll, -g

    ref = minimize(f, np.array(start), jac=True, method="L-BFGS-B", bounds=mle.DEFAULT_BOUNDS,
                   options={"ftol": 1e-12, "gtol": 1e-8, "maxiter": 200})
    h = T.Handle(dev(x), dev(y), nb=100, eps=1e-11, rank_cap=100)
    th, ll, info = mle.fit(h, dev(z), start, ftol=1e-12, gtol=1e-8, maxiter=200)
    assert info["evals"] > 3
    np.testing.assert_allclose(th, ref.x, rtol=1e-3)
    assert abs(ll + ref.fun) <= 1e-7 * abs(ref.fun)


def test_tlr_mle_within_one_percent_of_dense_mle(M):
    mle, T = M
    truth = (1.0, 0.3, 1.0)
    x, y = inputs.jittered_grid(48)  # n = 2304, tiles of 256
    hd = T.Handle(dev(x), dev(y), nb=256, eps=-1.0)
    hs = T.Handle(dev(x), dev(y), nb=256, eps=1e-12, rank_cap=256)
    hs.factor(truth)
    z = hs.sample(dev(inputs.standard_normal(len(x))))
    start = (0.5, 0.05, 0.8)
    th_d, ll_d, _ = mle.fit(hd, z, start)
    h = T.Handle(dev(x), dev(y), nb=256, eps=1e-7)
    th_t, ll_t, info = mle.fit(h, z, start)
    np.testing.assert_allclose(th_t, th_d, rtol=1e-2)
    assert abs(ll_t - ll_d) <= 1e-6 * abs(ll_d)
