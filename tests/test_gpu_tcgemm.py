"""The float64-accurate tensor-core GEMM (tlr_gemm_tc: bf16 digit slices on tcgen05) against float64 products.

Element by element against numpy's float64 product on the CPU, for the four transpose combinations, ragged
sizes (m, n, k not multiples of the 128 x 64 x 32 tiles, several exact-accumulation chunks along k), rows
and columns spread over twelve decades (one scale per row of op(A) and column of op(B)), zero rows and
k = 0.  The bound is the one stated for the method: with 2^sa_i (2^sb_j) the power of two above the
largest magnitude in row i of op(A) (column j of op(B)),
    |C - C_ref| <= |alpha| k 2^sa_i 2^sb_j ((S + 4) 2^-8S + 2^-38) + float64 rounding of the reference.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    from paper_1804_09137_gb300 import tlr

    return tlr


def colmajor(X):
    """A column-major CUDA tensor holding X (shape kept)."""
    return torch.tensor(np.ascontiguousarray(X.T), dtype=torch.float64, device="cuda").T


def pow2_above(v):
    _, e = np.frexp(v)  # v = f 2^e, 0.5 <= f < 1
    return np.where(v > 0, np.ldexp(1.0, e), 0.0)


def run(T, opA, opB, C0, tA, tB, alpha, beta, slices):
    A = opA.T if tA else opA
    B = opB.T if tB else opB
    Cd = colmajor(C0)
    T.gemm_tc(colmajor(A), colmajor(B), Cd, tA=tA, tB=tB, alpha=alpha, beta=beta, slices=slices)
    got = Cd.cpu().numpy()
    ref = beta * C0 + alpha * (opA @ opB)
    k = opA.shape[1]
    sa = pow2_above(np.max(np.abs(opA), axis=1)) if k else np.zeros(opA.shape[0])
    sb = pow2_above(np.max(np.abs(opB), axis=0)) if k else np.zeros(opB.shape[1])
    bound = abs(alpha) * k * np.outer(sa, sb) * ((slices + 4) * 2.0 ** (-8 * slices) + 2.0 ** -38)
    bound += 1e-15 * (np.abs(beta * C0) + abs(alpha) * (np.abs(opA) @ np.abs(opB)))
    return got, ref, bound


def operands(m, n, k, seed):
    rng = np.random.default_rng(seed)
    opA = rng.standard_normal((m, k)) * 10.0 ** rng.uniform(-6, 6, size=(m, 1))
    opB = rng.standard_normal((k, n)) * 10.0 ** rng.uniform(-6, 6, size=(1, n))
    return opA, opB, rng.standard_normal((m, n))


@pytest.mark.parametrize("slices", [4, 5, 6])
@pytest.mark.parametrize("m,n,k,tA,tB", [(300, 200, 700, False, False), (128, 64, 32, False, True),
                                          (257, 65, 33, True, False), (900, 900, 1000, True, True)])
def test_gemm_tc_matches_float64(T, m, n, k, tA, tB, slices):
    opA, opB, C0 = operands(m, n, k, m + n + k)
    got, ref, bound = run(T, opA, opB, C0, tA, tB, -1.3, 0.7, slices)
    err = np.abs(got - ref)
    assert np.all(err <= bound), (float(np.max(err / bound)), float(np.max(err)))


def test_gemm_tc_special_rows_and_depths(T):
    m, n, k = 150, 70, 130
    opA, opB, C0 = operands(m, n, k, 3)
    opA[5] = 0.0                 # a zero row
    opA[7, :] *= 1e-30           # tiny row: its own scale
    opA[9, 3] = 1e20             # one huge entry: the rest of its row falls below the digits (bounded error)
    opB[:, 11] = 0.0             # a zero column
    got, ref, bound = run(T, opA, opB, C0, False, False, 1.0, 0.0, 6)
    assert np.all(np.abs(got - ref) <= bound)
    assert np.all(got[5] == 0.0) and np.all(got[:, 11] == 0.0)
    # k = 1 and k = 0 (C = beta C)
    for kk in (1, 0):
        a, b = opA[:, :kk].copy(), opB[:kk, :].copy()
        got, ref, bound = run(T, a, b, C0, False, False, 2.0, -0.5, 6)
        assert np.all(np.abs(got - ref) <= bound + 1e-15 * np.abs(ref))
