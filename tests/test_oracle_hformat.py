"""Pins for blockwise truncation, formatting and the H-inverse (Sec. 3.1.5,
Sec. 4.3 H_eps, Sec. 4 approximate inverse)."""
import numpy as np
import pytest

from oracle.assembly import stencil_poisson, plane_blocks
from oracle.hformat import truncate_block, fmt, hinv
from oracle.hstructure import Structure
from inputs import gaussian_field_kappa


def _with_spectrum(m, n, sig, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, len(sig))))
    V, _ = np.linalg.qr(rng.standard_normal((n, len(sig))))
    return (U * sig) @ V.T


@pytest.mark.parametrize("eps,expect", [(1e-1, 3), (1e-3, 5), (1e-6, 7), (1e-7, 8),
                                        (0.5, 1), (2.0, 0)])
def test_truncation_rank_and_eckart_young(eps, expect):
    sig = np.array([4.0, 2.0, 1.0, 0.3, 0.01, 0.001, 2e-5, 1e-6, 0.0][:8])
    sig = sig / sig[0] * 7.0
    B = _with_spectrum(40, 30, sig, 0)
    Bk, k = truncate_block(B, eps)
    if eps < 1.0:
        assert k == expect
        err = np.linalg.norm(B - Bk, 2)
        want = sig[k] if k < len(sig) else 0.0
        assert abs(err - want) <= 1e-12 * sig[0]
    else:
        assert k == 0 and not Bk.any()


def test_threshold_tie_is_dropped():
    sig = np.array([1.0, 0.5, 0.25])
    B = _with_spectrum(10, 10, sig, 1)
    _, k = truncate_block(B, 0.25 * (1 + 1e-9))
    assert k == 2


def test_fmt_keeps_dense_and_bounds_lowrank_error():
    st = Structure(8, 1.0, 8)
    rng = np.random.default_rng(2)
    M = rng.standard_normal((64, 64))
    eps = 0.2
    ranks = {}
    F = fmt(M, st, 0, 0, eps, ranks)
    for a, b, kind in st.leaves():
        ra, rb = st.rng(a), st.rng(b)
        if kind == "D":
            assert np.array_equal(F[ra, rb], M[ra, rb])
        else:
            s1 = np.linalg.svd(M[ra, rb], compute_uv=False)[0]
            assert np.linalg.norm(M[ra, rb] - F[ra, rb], 2) <= eps * s1 + 1e-12
            assert np.linalg.matrix_rank(F[ra, rb], tol=1e-10) == ranks[(a, b)]
    assert ranks  # the case has admissible blocks


@pytest.mark.parametrize("n,eta,leaf", [(8, 1.0, 8), (12, 2.0, 16), (16, 2.0, 32)])
def test_hinv_eps_to_zero_is_exact_inverse(n, eta, leaf):
    kap = gaussian_field_kappa(n, 5)
    D, _, _ = plane_blocks(stencil_poisson(kap, n), n)
    st = Structure(n, eta, leaf)
    p = np.asarray(st.perm)
    A = fmt(D[n // 2][np.ix_(p, p)], st, 0, 0, 1e-15)
    X = hinv(A, st, 1e-15)
    Xe = np.linalg.inv(A)
    assert np.linalg.norm(X - Xe) <= 1e-10 * np.linalg.norm(Xe)


def test_hinv_accuracy_improves_with_eps():
    n = 16
    kap = gaussian_field_kappa(n, 6)
    D, _, _ = plane_blocks(stencil_poisson(kap, n), n)
    st = Structure(n, 2.0, 16)
    p = np.asarray(st.perm)
    A = D[3][np.ix_(p, p)]
    errs = []
    for eps in (1e-1, 1e-3, 1e-5):
        X = hinv(fmt(A, st, 0, 0, eps), st, eps)
        errs.append(np.linalg.norm(A @ X - np.eye(len(A))))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-3
