"""The FP64-accurate digit-split product (elm_ddm_fp64_gemm: the split kernels and the
tensor-core products the solver's dense updates run on) against an extended-precision
reference, kernel by kernel.

Bound under test (include/elm_ddm.h): each row of A and B loses less than 2^-54 of its
largest magnitude to the digit truncation, the digit pairs of weight below 2^-62 that
are not formed add at most 6 * 2^-54 max_k|A_ik| max_k|B_jk| per term, and each element
is rounded once, so
    |C_ij - (A B^T)_ij| <= 2^-53 |(A B^T)_ij|
                           + 2^-54 (max_k|A_ik| sum_k|B_jk| + max_k|B_jk| sum_k|A_ik|)
                           + 6 K 2^-54 max_k|A_ik| max_k|B_jk|.
This is normwise per row and column: entries far below their row's largest one get no
componentwise guarantee, which the test shows on rows spanning more than 40 binades and
on an upper-triangular factor with kappa ~ 1e14 (the shape of the local R factors).
The reference is numpy's long double (IEEE quad on the Arm GPU hosts, 64-bit-mantissa
extended on x86): every product of two doubles is exact or within 2^-64 there.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2406_15959_gb300 import elm_ddm as E

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
if np.finfo(np.longdouble).nmant < 63:
    pytest.skip("long double is no wider than double here", allow_module_level=True)

DEV = torch.device("cuda:0")
RNG = np.random.default_rng(2024)


def _exact(A, B):
    return A.astype(np.longdouble) @ B.astype(np.longdouble).T


def _bound(A, B, exact):
    amax, asum = np.abs(A).max(1), np.abs(A).sum(1)
    bmax, bsum = np.abs(B).max(1), np.abs(B).sum(1)
    trunc = 2.0 ** -54 * (amax[:, None] * bsum[None, :] + bmax[None, :] * asum[:, None])
    dropped = 6.0 * A.shape[1] * 2.0 ** -54 * amax[:, None] * bmax[None, :]
    # beyond 62 chunks of 128 the two int64 sums are rounded once each when converted
    rounds = 1.0 if A.shape[1] <= 62 * 128 else 3.0
    return rounds * 2.0 ** -53 * np.abs(exact.astype(np.float64)) + 1.0001 * (trunc + dropped) + 1e-300


def _check(kernel, A, B, alpha=1.0, beta=0.0, C0=None, a_layout="row", b_layout="row"):
    M, K = A.shape
    N = B.shape[0]
    # a_layout "col": A stored column-major (stride (1, M)); "row": row-major
    At = torch.as_tensor(A, device=DEV)
    if a_layout == "col":
        At = torch.as_tensor(np.asfortranarray(A), device=DEV).t().contiguous().t()
    Bt = torch.as_tensor(B, device=DEV)
    if b_layout == "col":
        Bt = torch.as_tensor(np.asfortranarray(B), device=DEV).t().contiguous().t()
    C = torch.as_tensor(C0 if C0 is not None else np.zeros((M, N)), device=DEV).t().contiguous().t()
    E.fp64_gemm(At, Bt, C, alpha, beta, kernel)
    got = C.cpu().numpy()
    ex = _exact(A, B)
    ref = np.longdouble(alpha) * ex
    if C0 is not None:
        ref = ref + np.longdouble(beta) * C0.astype(np.longdouble)
    err = np.abs(got.astype(np.longdouble) - ref).astype(np.float64)
    bnd = abs(alpha) * _bound(A, B, ex)
    if C0 is not None or abs(alpha) != 1.0:
        bnd = bnd + 2.0 ** -52 * (np.abs(alpha * ex.astype(np.float64)) + np.abs(beta * (C0 if C0 is not None else 0)))
    ok = err <= bnd
    assert ok.all(), (kernel, float((err / bnd).max()), np.argwhere(~ok)[:3])
    return float((err / bnd).max())


def _wide_rows(M, K, binades=44):
    return RNG.standard_normal((M, K)) * 2.0 ** -RNG.uniform(0, binades, size=(M, K))


@pytest.mark.parametrize("kernel,K", [(E.GEMM_TILE32, 300), (E.GEMM_TILE32, 2048),
                                      (E.GEMM_TILE64, 128), (E.GEMM_PERSISTENT, 96),
                                      (E.GEMM_FUSED_SPLIT, 700), (E.GEMM_TILE32, 9000),
                                      (E.GEMM_FUSED_SPLIT, 9000), (E.GEMM_FUSED_SPLIT, 2400),
                                      (E.GEMM_FUSED_SPLIT_B, 700),
                                      (E.GEMM_FUSED_SPLIT_B, 2400), (E.GEMM_FUSED_SPLIT_B, 9000)])
def test_random_operands_within_the_bound(kernel, K):
    # (M <= 128 for the fused A split at K = 2400: one tile, K split over 4 CTAs)
    M, N = {E.GEMM_FUSED_SPLIT: (120 if K == 2400 else 200, 32),
            E.GEMM_FUSED_SPLIT_B: (120, 350)}.get(kernel, (200, 70))
    A, B = RNG.standard_normal((M, K)), RNG.standard_normal((N, K))
    _check(kernel, A, B)
    # the bound is also tight enough to mean FP64 accuracy for well-scaled data
    got = torch.zeros((M, N), dtype=torch.float64, device=DEV)
    E.fp64_gemm(torch.as_tensor(A, device=DEV), torch.as_tensor(B, device=DEV), got, kernel=kernel)
    ex = _exact(A, B).astype(np.float64)
    assert np.abs(got.cpu().numpy() - ex).max() <= 1e-14 * np.abs(A).sum(1).max() * np.abs(B).max()


@pytest.mark.parametrize("kernel", [E.GEMM_TILE32, E.GEMM_PERSISTENT, E.GEMM_FUSED_SPLIT,
                                    E.GEMM_FUSED_SPLIT_B])
def test_rows_spanning_forty_binades(kernel):
    K = 128 if kernel == E.GEMM_PERSISTENT else 520
    N = 32 if kernel == E.GEMM_FUSED_SPLIT else 45
    M = 128 if kernel == E.GEMM_FUSED_SPLIT_B else 150
    A, B = _wide_rows(M, K), _wide_rows(N, K)
    _check(kernel, A, B, a_layout="col" if kernel != E.GEMM_FUSED_SPLIT else "row",
           b_layout="row" if kernel == E.GEMM_FUSED_SPLIT_B else "col")


def test_upper_triangular_factor_with_kappa_1e14():
    """R-shaped operand: upper triangular, columns scaled from 1 down to 1e-14, as the
    local R^s of the paper's initialisation; the product R R^T has entries that span the
    same range, and the small ones carry only the normwise guarantee."""
    K = 256
    R = np.triu(RNG.standard_normal((K, K))) * np.logspace(0, -14, K)[None, :]
    _check(E.GEMM_TILE32, R, R, a_layout="col", b_layout="col")
    # against an FP64 GEMM on the same data: no worse than a few times its componentwise error
    ex = _exact(R, R).astype(np.float64)
    got = torch.zeros((K, K), dtype=torch.float64, device=DEV)
    E.fp64_gemm(torch.as_tensor(R, device=DEV), torch.as_tensor(R, device=DEV), got)
    big = np.abs(ex) > 1e-3 * np.abs(ex).max()
    assert (np.abs(got.cpu().numpy() - ex)[big] <= 1e-13 * np.abs(ex)[big]).all()


@pytest.mark.parametrize("kernel,alpha,beta", [(E.GEMM_TILE32, -1.0, 1.0), (E.GEMM_PERSISTENT, -1.0, 1.0),
                                               (E.GEMM_PERSISTENT, 0.75, -2.0), (E.GEMM_TILE32, 1.0, 0.0),
                                               (E.GEMM_PERSISTENT_WIDE, -1.0, 1.0),
                                               (E.GEMM_PERSISTENT_WIDE, 1.0, 1.0)])
def test_alpha_beta_update(kernel, alpha, beta):
    M, N, K = (300, 150, 128) if kernel == E.GEMM_PERSISTENT_WIDE else (260, 66, 64)
    A, B = RNG.standard_normal((M, K)), RNG.standard_normal((N, K))
    C0 = RNG.standard_normal((M, N))
    _check(kernel, A, B, alpha, beta, C0)


def test_zero_and_subnormal_rows():
    K = 64
    A = RNG.standard_normal((140, K))
    A[3] = 0.0
    A[7, 5] = 5e-320          # subnormal entry in an otherwise normal row
    A[9] = -0.0
    B = RNG.standard_normal((33, K))
    B[0] = 0.0
    _check(E.GEMM_TILE32, A, B)
    _check(E.GEMM_PERSISTENT, A, B)
    _check(E.GEMM_PERSISTENT_WIDE, A, B, beta=1.0, C0=RNG.standard_normal((140, 33)))


def test_rejects_unsupported_shapes():
    lib = E.load()
    assert lib.elm_ddm_fp64_gemm_workspace(E.GEMM_PERSISTENT, 10, 10, 129) == 0
    assert lib.elm_ddm_fp64_gemm_workspace(E.GEMM_FUSED_SPLIT, 10, 33, 10) == 0
    assert lib.elm_ddm_fp64_gemm_workspace(E.GEMM_FUSED_SPLIT_B, 129, 10, 10) == 0
    assert lib.elm_ddm_fp64_gemm_workspace(E.GEMM_PERSISTENT_WIDE, 10, 10, 129) == 0
    assert lib.elm_ddm_fp64_gemm_workspace(9, 10, 10, 10) == 0
    with pytest.raises(E.ElmDdmError):   # the wide update is C += +-A B^T
        E.fp64_gemm(torch.zeros((4, 4), dtype=torch.float64, device=DEV),
                    torch.zeros((4, 4), dtype=torch.float64, device=DEV),
                    torch.zeros((4, 4), dtype=torch.float64, device=DEV), 0.5, 1.0, E.GEMM_PERSISTENT_WIDE)
    A = torch.zeros((4, 4), dtype=torch.float64, device=DEV)
    with pytest.raises(E.ElmDdmError):   # fused split needs beta = 0
        E.fp64_gemm(A, A, A.clone(), 1.0, 1.0, E.GEMM_FUSED_SPLIT)


def test_cholesky_pivot_reciprocal_within_two_ulp():
    """The Schur Cholesky's pivots use a Newton reciprocal from an FP32 seed instead of a
    division: within two units in the last place of the correctly rounded 1/x over the
    normal range (and the division itself at the ends of it)."""
    x = np.concatenate([RNG.uniform(1.0, 2.0, 4000),
                        2.0 ** RNG.uniform(-1020, 1020, 4000),
                        np.nextafter(2.0 ** np.arange(-1022, 1023, 7), 0.0),
                        [1.0, 2.0, 3.0, 1.5, np.nextafter(1.0, 2.0), np.nextafter(2.0, 1.0),
                         2.0 ** -1021, 2.0 ** -1022, 2.0 ** 1023]])
    y = E.selftest(E.SELFTEST_PIVOT_RCP, torch.as_tensor(x, device=DEV)).cpu().numpy()
    ref = 1.0 / x.astype(np.longdouble)
    ulp = np.spacing(np.abs(ref.astype(np.float64)))
    err = np.abs((y.astype(np.longdouble) - ref)).astype(np.float64) / ulp
    assert err.max() <= 2.0, (float(err.max()), x[np.argmax(err)])
