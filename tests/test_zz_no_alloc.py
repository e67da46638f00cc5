"""The allocation-free entry point (tlr_loglik_dense_noalloc) against the handle path.

tlr_loglik_dense_noalloc serves callers that cannot call cudaMalloc: it keeps
all of its workspace in a static device array of the library.  It must give the
log-likelihood that the ordinary entry points (tlr_create, tlr_matern_generate,
tlr_compress, tlr_potrf, tlr_loglik with one tile covering every point) give,
on consecutive calls that reuse the same static workspace.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def test_no_alloc_matches_handle_path_on_two_calls(T):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [(20, (1.0, 0.1, 0.5), 0), (31, (1.3, 0.25, 1.1), 1)]  # n = 400, then n = 961
    for side, theta, seed in cases:
        x, y = inputs.jittered_grid(side)
        n = len(x)
        z = np.random.default_rng(seed).standard_normal(n)
        xd, yd, zd = _dev(x), _dev(y), _dev(z)
        out = torch.zeros(3, dtype=torch.float64, device="cuda")
        rc = T.lib().tlr_loglik_dense_noalloc(n, _ptr(xd), _ptr(yd), _ptr(zd), T.TlrTheta(*theta), _ptr(out), stream)
        assert rc == 0
        h = T.Handle(xd, yd, nb=n, eps=1e-9, order=False)  # a single tile: the dense path
        h.factor(theta)
        ref = h.loglik(zd)
        h.check()
        np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=1e-11, atol=0)


def test_no_alloc_rejects_sizes_beyond_its_workspace(T):
    one = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    rc = T.lib().tlr_loglik_dense_noalloc(1025, _ptr(one), _ptr(one), _ptr(one), T.TlrTheta(1.0, 0.1, 0.5),
                                          _ptr(out), None)
    assert rc == -1
