"""Batched independent regions (GPU) against one handle per region and the oracle."""
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


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def test_batched_regions_match_single_handles(T):
    sizes = [300, 450, 700, 900, 1200, 1500, 640]
    thetas = [(1.0, 0.1, 0.5), (0.7, 0.2, 1.0), (1.5, 0.05, 1.5), (1.0, 0.3, 1.0), (2.0, 0.15, 0.5),
              (0.5, 0.25, 1.5), (1.2, 0.08, 1.0)]
    nbs = [300, 128, 256, 256, 384, 256, 640]  # mixed: single tiles and TLR, shared tile sizes
    xs, ys, zs, opts = [], [], [], []
    for r, (n, th, nb) in enumerate(zip(sizes, thetas, nbs)):
        x, y = inputs.locations(n, seed=100 + r)
        z = inputs.standard_normal(n, seed=200 + r)
        xs.append(dev(x)); ys.append(dev(y)); zs.append(dev(z))
        opts.append(T.TlrOpts(nb, 1e-11, nb, 0, 1, 0, 0.0))
    ll, grad, st = T.loglik_grad_batched(xs, ys, zs, thetas, opts, nworkers=3)
    assert st == [0] * len(sizes)
    for r in range(len(sizes)):
        h = T.Handle(xs[r], ys[r], nb=nbs[r], eps=1e-11, rank_cap=nbs[r])
        h.factor(thetas[r])
        l1, g1 = h.loglik_grad(zs[r])
        assert abs(ll[r].item() - l1.item()) <= 1e-11 * abs(l1.item())
        np.testing.assert_allclose(grad[r].cpu().numpy(), g1.cpu().numpy(), rtol=1e-8, atol=1e-9)
    # the smallest region against the oracle
    x, y = inputs.locations(300, seed=100)
    l_ref, g_ref = DN.loglik_grad(x, y, inputs.standard_normal(300, seed=200), thetas[0])
    assert abs(ll[0].item() - l_ref) <= 1e-9 * abs(l_ref)
    np.testing.assert_allclose(grad[0].cpu().numpy(), g_ref, rtol=1e-6, atol=1e-6 * np.abs(g_ref).max())


def test_batched_reports_per_region_failure(T):
    x, y = inputs.locations(200, seed=5)
    xd = np.concatenate([x, x[:2]]); yd = np.concatenate([y, y[:2]])  # duplicated points: not SPD
    xs = [dev(x), dev(xd)]; ys = [dev(y), dev(yd)]
    zs = [dev(inputs.standard_normal(200)), dev(inputs.standard_normal(202))]
    opts = [T.TlrOpts(64, 1e-10, 64, 0, 1, 0, 0.0)] * 2
    ll, grad, st = T.loglik_grad_batched(xs, ys, zs, [(1.0, 0.1, 0.5)] * 2, opts, nworkers=2)
    assert st[0] == 0 and st[1] == T.TLR_ERR_NOT_SPD


def test_autotuner_picks_a_measured_candidate(T):
    from paper_1804_09137_gb300 import regions

    choice = regions.autotune_nb([900, 1100, 2600], eps=1e-8, candidates=(0, 256, 512), edges=(2000,))
    assert set(choice) == {0, 1}
    for c, (nb, cap, secs, timings) in choice.items():
        assert (nb, cap) in timings and secs == min(timings.values())
        # every tile size was tried with both rank caps
        for b in {b for b, _ in timings if b > 0}:
            assert (b, max(b // 4, 16)) in timings and (b, b // 2) in timings
