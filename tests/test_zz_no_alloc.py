"""The allocation-free entry point (tlr_loglik_dense_noalloc) against the handle path and the oracle.

tlr_loglik_dense_noalloc serves callers that cannot call cudaMalloc: it keeps
all of its workspace in a static device array of the library.  It must give the
log-likelihood that the ordinary entry points (tlr_create, tlr_matern_generate,
tlr_compress, tlr_potrf, tlr_loglik with one tile covering every point) give,
and the oracle's dense value, on consecutive calls that reuse the same static
workspace: a larger problem first, then a smaller one (stale contents left
behind), and a failing call (not positive definite) followed by a valid one
(the status words start from zero again).
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense as DN
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


def _dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _call(T, xd, yd, zd, theta, out):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return T.lib().tlr_loglik_dense_noalloc(int(xd.numel()), _ptr(xd), _ptr(yd), _ptr(zd), T.TlrTheta(*theta),
                                            _ptr(out), stream)


def test_no_alloc_matches_handle_path_on_two_calls(T):
    cases = [(31, (1.3, 0.25, 1.1), 1), (20, (1.0, 0.1, 0.5), 0)]  # n = 961, then n = 400
    for side, theta, seed in cases:
        x, y = inputs.jittered_grid(side)
        n = len(x)
        z = np.random.default_rng(seed).standard_normal(n)
        xd, yd, zd = _dev(x), _dev(y), _dev(z)
        out = torch.zeros(3, dtype=torch.float64, device="cuda")
        assert _call(T, xd, yd, zd, theta, out) == 0
        h = T.Handle(xd, yd, nb=n, eps=1e-9, order=False)  # a single tile: the dense path
        h.factor(theta)
        ref = h.loglik(zd)
        h.check()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref.cpu().numpy(), rtol=1e-11, atol=0)
        want = np.array(DN.loglik(x, y, z, theta))
        np.testing.assert_allclose(got, want, rtol=1e-10, atol=0)
        h.close()


def test_no_alloc_reports_not_spd_then_recovers(T):
    x, y = inputs.jittered_grid(12)
    x = np.concatenate([x, x[:2]])  # repeated locations: a singular covariance
    y = np.concatenate([y, y[:2]])
    z = np.random.default_rng(3).standard_normal(len(x))
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    assert _call(T, _dev(x), _dev(y), _dev(z), (1.0, 0.1, 0.5), out) == T.TLR_ERR_NOT_SPD
    x, y = inputs.jittered_grid(12)
    z = z[: len(x)]
    assert _call(T, _dev(x), _dev(y), _dev(z), (1.0, 0.1, 0.5), out) == 0
    np.testing.assert_allclose(out.cpu().numpy(), np.array(DN.loglik(x, y, z, (1.0, 0.1, 0.5))), rtol=1e-10)


def test_no_alloc_rejects_sizes_beyond_its_workspace(T):
    one = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    rc = T.lib().tlr_loglik_dense_noalloc(1025, _ptr(one), _ptr(one), _ptr(one), T.TlrTheta(1.0, 0.1, 0.5),
                                          _ptr(out), None)
    assert rc == -1
