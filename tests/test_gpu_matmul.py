"""GPU parity of the library's dense product (cpinv_matmul) in both
arithmetics, against the oracle's correctly rounded product X'Y
(oracle.exact_cross: exact integer-slice sums, one rounding)."""
import numpy as np
import pytest

import oracle
from paper_0804_4809_gb300 import inputs

from gpu_util import dev, to_dev

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def cp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0804_4809_gb300 import build
    build.build()
    from paper_0804_4809_gb300 import cpinv
    return cpinv


def _exact(opA, opB):
    # op(A) op(B) = (op(A)')' op(B): exact_cross(X, Y) = X'Y
    return oracle.exact_cross(opA.T, opB)


def _run(cp, A, B, ta, tb, mode, bits=0, alpha=1.0, beta=0.0, C=None):
    import torch
    Cd = None if C is None else to_dev(C)
    out = cp.matmul(to_dev(A), to_dev(B), ta, tb, mode=mode, bits=bits, alpha=alpha, beta=beta, C=Cd)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
@pytest.mark.parametrize("M,N,K", [(130, 70, 300), (256, 384, 1024), (1, 129, 64), (200, 1, 4096),
                                   (129, 257, 65)])
def test_exact_slice_is_correctly_rounded(cp, ta, tb, M, N, K):
    g = np.random.default_rng(M * 31 + N * 7 + K)
    opA = g.standard_normal((M, K)) * np.exp2(g.integers(-20, 20, (M, 1)))
    opB = g.standard_normal((K, N)) * np.exp2(g.integers(-20, 20, (1, N)))
    A = opA.T.copy() if ta else opA
    B = opB.T.copy() if tb else opB
    C = _run(cp, A, B, ta, tb, "exact", bits=62)
    X = _exact(opA, opB)
    bound = np.abs(opA) @ np.abs(opB)
    err = np.abs(C - X)
    assert np.all(err <= 4 * U * bound), float(np.max(err / np.maximum(bound, 1e-300)))
    # one rounding: almost every entry is the correctly rounded value
    assert np.mean(C == X) > 0.97


def test_fp64_mode_error_is_fp64_sized(cp):
    g = np.random.default_rng(5)
    A = g.standard_normal((300, 200))
    B = g.standard_normal((300, 150))
    C = _run(cp, A, B, True, False, "fp64")
    X = _exact(A.T, B)
    bound = np.abs(A.T) @ np.abs(B)
    assert np.all(np.abs(C - X) <= 300 * U * bound)


def test_exact_slice_extreme_sums(cp):
    """Constant operands make every residue product of a modulus equal, so the
    FP32 tensor-core sums reach K * 64^2 = 2^24 for the largest residues: the
    result must still be exact."""
    K = 4096
    for x in [1.0 - 2.0 ** -52, 0.7500000000000002, 3.0, -1.2345678901234567]:
        A = np.full((128, K), x)
        B = np.full((K, 128), x)
        C = _run(cp, A, B, False, False, "exact", bits=62)
        X = _exact(A, B)
        assert np.array_equal(C, X), (x, float(np.max(np.abs(C - X))))


def test_exact_slice_chunked_k_and_alpha_beta(cp):
    g = np.random.default_rng(9)
    A = g.standard_normal((96, 9000))
    B = g.standard_normal((9000, 40))
    C0 = g.standard_normal((96, 40))
    C = _run(cp, A, B, False, False, "exact", bits=53, alpha=-0.5, beta=2.0, C=C0)
    X = -0.5 * _exact(A, B) + 2.0 * C0
    bound = 0.5 * (np.abs(A) @ np.abs(B)) + 2.0 * np.abs(C0)
    assert np.all(np.abs(C - X) <= 8 * U * bound)


def test_exact_slice_symmetric_operand(cp):
    G = inputs.rank_deficient(500, 300, 200, seed=3)
    Gd = to_dev(G)
    import torch
    C = cp.matmul(Gd, Gd, True, False, mode="exact", bits=62)
    torch.cuda.synchronize()
    X = oracle.gram(G)
    assert np.mean(C.cpu().numpy() == X) > 0.97
    assert np.max(np.abs(C.cpu().numpy() - X)) <= 4 * U * np.max(np.abs(X))


def test_exact_slice_nonfinite(cp):
    A = np.ones((64, 64))
    A[3, 5] = np.inf
    with pytest.raises(cp.CpinvError) as e:
        _run(cp, A, A, False, False, "exact")
    assert e.value.status == 2


@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True)])
@pytest.mark.parametrize("M,N,K", [(130, 70, 300), (256, 384, 5000), (129, 257, 65)])
def test_split_bf16x3_error_bound(cp, ta, tb, M, N, K):
    """BF16x3 split precision: hi*hi + hi*lo + lo*hi with hi, lo the BF16
    parts of each scaled operand and FP32 sums; |error| <= 2^-13 (|A| |B|)."""
    g = np.random.default_rng(M + 3 * N + 5 * K)
    opA = g.standard_normal((M, K))
    opB = g.standard_normal((K, N))
    A = opA.T.copy() if ta else opA
    B = opB.T.copy() if tb else opB
    C = _run(cp, A, B, ta, tb, "bf16x3")
    X = _exact(opA, opB)
    bound = np.abs(opA) @ np.abs(opB)
    assert np.all(np.abs(C - X) <= 2.0 ** -13 * bound)
    # and it is not secretly an FP64 product: the error is far above FP64's
    assert np.max(np.abs(C - X) / bound) > 1e-10


@pytest.mark.parametrize("ta,tb", [(False, False), (True, True)])
@pytest.mark.parametrize("M,N,K", [(300, 260, 1000), (257, 513, 2048), (1030, 70, 333)])
def test_exact_slice_53bit_outputs_correctly_rounded(cp, ta, tb, M, N, K):
    """53-bit operands (the chain's products: fewer moduli, the 128-bit
    reconstruction).  Integer entries below 2^40 times a power of two per
    row are exact in 53-bit fixed point, so the product is exact before its
    one rounding."""
    g = np.random.default_rng(M + 3 * N + 7 * K)
    opA = g.integers(-2 ** 40, 2 ** 40, (M, K)).astype(np.float64) * np.exp2(g.integers(-30, 30, (M, 1)))
    opB = g.integers(-2 ** 40, 2 ** 40, (K, N)).astype(np.float64) * np.exp2(g.integers(-30, 30, (1, N)))
    A = opA.T.copy() if ta else opA
    B = opB.T.copy() if tb else opB
    C = _run(cp, A, B, ta, tb, "exact", bits=53)
    X = _exact(opA, opB)
    assert np.array_equal(C, X), float(np.max(np.abs(C - X) / np.maximum(np.abs(X), 1e-300)))


def test_exact_slice_53bit_symmetric_and_alpha_beta(cp):
    import torch
    g = np.random.default_rng(77)
    G = g.integers(-2 ** 30, 2 ** 30, (700, 400)).astype(np.float64) * np.exp2(g.integers(-8, 8, (1, 400)))
    Gd = to_dev(G)
    C = cp.matmul(Gd, Gd, True, False, mode="exact", bits=53)
    torch.cuda.synchronize()
    X = _exact(G.T, G)
    assert np.array_equal(C.cpu().numpy(), X)
    A = g.standard_normal((500, 300))
    B = g.standard_normal((300, 280))
    C0 = g.standard_normal((500, 280))
    C = _run(cp, A, B, False, False, "exact", bits=53, alpha=-0.5, beta=2.0, C=C0)
    Xc = -0.5 * _exact(A, B) + 2.0 * C0
    bound = 0.5 * (np.abs(A) @ np.abs(B)) + 2.0 * np.abs(C0)
    assert np.all(np.abs(C - Xc) <= 8 * U * bound)
