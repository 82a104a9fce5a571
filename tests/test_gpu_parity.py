"""GPU parity tests: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances:
* assembly, SpMV: FP64 with a different rounding order -> 1e-14 relative;
* ACR apply, FP64 form: the GPU formats every block exactly like the
  oracle (exact result, then truncation at eps) except that its range finder
  discards directions below tau = max(1e-3 eps, 1e-7) of the sketch before
  the final truncation; allowed difference 10 tau relative;
* ACR apply, FP32 form: 1e-5 relative (factors in float, FP64 vectors), or,
  where float arithmetic itself cannot reach that, 5 e32: e32 is the
  difference between the oracle and its own float32 arithmetic model
  (cr_setup(arith=float32): float32 products and sums, float32 storage,
  FP64 SVDs and leaf inverses) -- the device's float arithmetic rounds in a
  different order, hence the factor;
* ACR apply, BF16 form: every stored factor entry carries a relative rounding
  error of at most u = 2^-9 (8 significant bits, round to nearest even).  A
  path from r to z multiplies 4L + 1 factors (forward: X and a coupling per
  level, X_0, backward: a coupling and X per level); the roundings of
  different entries are independent and of either sign, so their effects add
  in quadrature rather than linearly (the probabilistic rounding-error
  bound of Higham and Mary, 2019): allowed sqrt(4L + 1) u relative, about
  7e-3 to 9e-3 at L = 3..5.  The FP64 Krylov solve must still reach its full
  tolerance, which the solve tests check;
* both the norm-wise error ||z - z_o|| / ||z_o|| and the element-wise one
  max |z - z_o| / max |z_o| are gated: FP32 and BF16 at the same rule (FP32
  with the model's element-wise error), FP64 at 10x the norm-wise bound
  (the sub-tau differences of the range finder sit in individual blocks, so
  they concentrate in few entries);
* Krylov solutions: the oracle's own SpMV must confirm ||f - A u|| <= rtol
  ||f||, and ||u - u_ref|| <= 10 cond(A) rtol ||u_ref|| for the exact u_ref.
"""
import functools

import numpy as np
import pytest
import scipy.sparse.linalg as sla

from inputs import (workload, codi_beta, uniform_rhs, gaussian_field_kappa, layered_speed,
                    helmholtz_omega)
from oracle.assembly import (stencil_poisson, stencil_codi, stencil_helmholtz, stencil_apply,
                             stencil_matrix, plane_blocks, NAMES)
from oracle.cr import cr_setup, cr_apply
from oracle.hstructure import Structure

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def acr():
    from paper_1712_08872_gb300 import _build
    _build.build()
    import paper_1712_08872_gb300 as pkg
    pkg.load_library()
    return pkg


def T(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda:0")


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def operator(acr, kind, n, seed=0):
    if kind == "poisson":
        kap = gaussian_field_kappa(n, seed)
        st = stencil_poisson(kap, n)
        coef = torch.empty(7 * n ** 3, dtype=torch.float64, device="cuda:0")
        acr.acr_stencil_poisson(n, T(kap), coef)
    elif kind == "helmholtz":
        sig = (helmholtz_omega(n) / layered_speed(n, 30)) ** 2
        st = stencil_helmholtz(sig, n)
        coef = torch.empty(7 * n ** 3, dtype=torch.float64, device="cuda:0")
        acr.acr_stencil_helmholtz(n, T(sig), coef)
    else:
        beta = codi_beta(n)
        st = stencil_codi(beta, n)
        coef = torch.empty(7 * n ** 3, dtype=torch.float64, device="cuda:0")
        acr.acr_stencil_codi(n, T(beta), coef)
    return st, coef


@pytest.mark.parametrize("kind,n", [("poisson", 7), ("poisson", 16), ("codi", 9), ("codi", 32),
                                    ("helmholtz", 9), ("helmholtz", 32)])
def test_assembly_and_spmv(acr, kind, n):
    st, coef = operator(acr, kind, n)
    ref = np.concatenate([st[k] for k in NAMES])
    assert rel(coef.cpu().numpy(), ref) <= 1e-14
    x = np.random.default_rng(1).standard_normal(n ** 3)
    y = torch.empty(n ** 3, dtype=torch.float64, device="cuda:0")
    acr.acr_spmv(n, coef, T(x), y)
    assert rel(y.cpu().numpy(), stencil_apply(st, n, x)) <= 1e-14


@pytest.mark.parametrize("kind,method", [("poisson", 0), ("codi", 1)])
def test_plain_krylov(acr, kind, method):
    n = 10
    st, coef = operator(acr, kind, n)
    f = uniform_rhs(n, 3)
    u = torch.zeros(n ** 3, dtype=torch.float64, device="cuda:0")
    info, status = acr.acr_krylov_solve_plain(n, coef, method, 20, 1e-10, 3000, T(f), u)
    assert status == 0 and info.converged
    uh = u.cpu().numpy()
    assert rel(stencil_apply(st, n, uh), f) <= 1e-10 * 1.0001
    A = stencil_matrix(st, n)
    ue = sla.spsolve(A.tocsc(), f)
    cond = np.linalg.cond(A.toarray())
    assert rel(uh, ue) <= 10 * cond * 1e-10


def cond_estimate(A, its=40):
    """2-norm condition number estimate: power iteration on A^T A for
    sigma_max, inverse power iteration with a sparse LU for sigma_min."""
    lu = sla.splu(A.tocsc())
    luT = sla.splu(A.T.tocsc())
    x = np.random.default_rng(0).standard_normal(A.shape[0])
    y = x.copy()
    smax = smin_inv = 0.0
    for _ in range(its):
        x = A.T @ (A @ x)
        smax = np.sqrt(np.linalg.norm(x))
        x /= np.linalg.norm(x)
        y = lu.solve(luT.solve(y))
        smin_inv = np.sqrt(np.linalg.norm(y))
        y /= np.linalg.norm(y)
    return smax * smin_inv


def tau(eps):
    return max(1e-3 * eps, 1e-7)


BF16_U = 2.0 ** -9


def apply_tol(prec, eps, levels, e32=0.0):
    """Allowed relative difference of a GPU apply from the oracle's (e32:
    the oracle's float32-arithmetic model error, FP32 form only)."""
    if prec == 0:
        return 10 * tau(eps)
    if prec == 1:
        return max(1e-5, 5 * e32)
    return np.sqrt(4 * levels + 1) * BF16_U


@functools.lru_cache(maxsize=None)
def float32_model_errors(kind, n, eta, leaf, eps, seed):
    """(norm-wise, element-wise) difference between the oracle's apply and
    that of its float32 arithmetic model, same input as the parity test."""
    st = {"poisson": lambda: stencil_poisson(gaussian_field_kappa(n, seed), n),
          "helmholtz": lambda: stencil_helmholtz((helmholtz_omega(n) / layered_speed(n, 30)) ** 2, n),
          "codi": lambda: stencil_codi(codi_beta(n), n)}[kind]()
    D, Ld, Ud = plane_blocks(st, n)
    S = Structure(n, eta, leaf)
    f = uniform_rhs(n, 4)
    z = cr_apply(cr_setup(D, Ld, Ud, S, eps), f)
    z32 = cr_apply(cr_setup(D, Ld, Ud, S, eps, arith=np.float32), f)
    return errors(z32, z)


def errors(z, zo):
    """(norm-wise, element-wise) relative differences."""
    return rel(z, zo), np.max(np.abs(z - zo)) / max(np.max(np.abs(zo)), 1e-300)


APPLY_CASES = [("poisson", 8, 1.0, 16, 1e-10), ("codi", 8, 2.0, 8, 1e-3),
               ("poisson", 16, 1.0, 32, 1e-6), ("codi", 16, 2.0, 32, 1e-2),
               ("poisson", 16, 2.0, 16, 1e-2)]
# indefinite Helmholtz (10 points per wavelength, 8-layer medium), FP64
APPLY_CASES_HELM = [("helmholtz", 8, 2.0, 16, 1e-5), ("helmholtz", 16, 2.0, 32, 1e-5)]
# eta = 16 puts plane couplings inside admissible blocks (exact ranks up to
# the interface length) and deepens the H-arithmetic.
APPLY_CASES_FP64 = APPLY_CASES + [("codi", 16, 16.0, 32, 1e-2)] + APPLY_CASES_HELM
APPLY_CASES_FP32 = APPLY_CASES_FP64


# the BF16 form is meant for coarse preconditioners (eps >= 1e-3)
APPLY_CASES_BF16 = [c for c in APPLY_CASES if c[4] >= 1e-3]


@pytest.mark.parametrize("kind,n,eta,leaf,eps,prec",
                         [c + (0,) for c in APPLY_CASES_FP64] + [c + (1,) for c in APPLY_CASES_FP32]
                         + [c + (2,) for c in APPLY_CASES_BF16])
def test_acr_apply_matches_oracle(acr, parity_log, kind, n, eta, leaf, eps, prec):
    st, coef = operator(acr, kind, n, seed=2)
    f = uniform_rhs(n, 4)
    D, Ld, Ud = plane_blocks(st, n)
    F = cr_setup(D, Ld, Ud, Structure(n, eta, leaf), eps)
    zo = cr_apply(F, f)
    h = acr.Handle(n, coef, eps, eta, leaf, prec, 32)
    z = torch.empty(n ** 3, dtype=torch.float64, device="cuda:0")
    h.apply(T(f), z)
    torch.cuda.synchronize()
    e2, einf = errors(z.cpu().numpy(), zo)
    m2 = minf = 0.0
    if prec == 1:
        m2, minf = float32_model_errors(kind, n, eta, leaf, eps, 2)
    tol, tolinf = apply_tol(prec, eps, len(F.levels), m2), apply_tol(prec, eps, len(F.levels), minf)
    if prec == 0:
        tolinf = 10 * tol
    info = h.info()
    h.close()
    parity_log(test="apply", kind=kind, n=n, eta=eta, leaf=leaf, eps=eps, prec=prec,
               rank_cap=32, tol=tol, tolinf=tolinf, err2=e2, errinf=einf, model32=m2,
               model32inf=minf, max_rank=info.max_rank, avg_rank=info.avg_rank,
               lr_truncations=info.lr_truncations, sketch_overflows=info.sketch_overflows)
    assert e2 <= tol and einf <= tolinf, (e2, einf, tol, tolinf)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_acr_apply_transpose_matches_oracle(acr, parity_log, prec):
    n, eta, leaf, eps = 8, 2.0, 8, 1e-3
    st, coef = operator(acr, "codi", n)
    D, Ld, Ud = plane_blocks(st, n)
    F = cr_setup(D, Ld, Ud, Structure(n, eta, leaf), eps)
    N = n ** 3
    Minv = np.stack([cr_apply(F, e) for e in np.eye(N)], axis=1)   # columns M^-1 e_j
    r = uniform_rhs(n, 5)
    want = Minv.T @ r
    h = acr.Handle(n, coef, eps, eta, leaf, prec, 32)
    z = torch.empty(N, dtype=torch.float64, device="cuda:0")
    h.apply_transpose(T(r), z)
    torch.cuda.synchronize()
    e2, einf = errors(z.cpu().numpy(), want)
    h.close()
    tol = apply_tol(prec, eps, len(F.levels))
    tolinf = 10 * tol if prec == 0 else tol
    parity_log(test="apply_transpose", kind="codi", n=n, eta=eta, leaf=leaf, eps=eps, prec=prec,
               tol=tol, err2=e2, errinf=einf)
    assert e2 <= tol and einf <= tolinf, (e2, einf, tol)


def test_fp32_form_eta16_solves_to_fp64_accuracy(acr):
    n = 16
    st, coef = operator(acr, "codi", n)
    f = uniform_rhs(n, 8)
    h = acr.Handle(n, coef, 1e-2, 16.0, 32, 1, 32)
    u = torch.zeros(n ** 3, dtype=torch.float64, device="cuda:0")
    info, status = acr.acr_krylov_solve(h.h, coef, acr.ACR_GMRES, 30, 1e-8, 100, T(f), u)
    torch.cuda.synchronize()
    h.close()
    assert status == 0 and info.iterations <= 6
    assert rel(stencil_apply(st, n, u.cpu().numpy()), f) <= 1e-8 * 1.0001


def test_exact_limit_equals_direct_solve(acr):
    n = 16
    st, coef = operator(acr, "codi", n)
    f = uniform_rhs(n, 6)
    ue = sla.spsolve(stencil_matrix(st, n).tocsc(), f)
    h = acr.Handle(n, coef, 1e-10, 2.0, 16, 0, 48)
    z = torch.empty(n ** 3, dtype=torch.float64, device="cuda:0")
    h.apply(T(f), z)
    torch.cuda.synchronize()
    h.close()
    assert rel(z.cpu().numpy(), ue) <= 1e-8


def _solve_case(acr, name, n, prec, eta=2.0):
    spec, cin, f = workload(name, n=n)
    if spec["pde"] == "codi":
        st = stencil_codi(cin, n)
        coef = torch.empty(7 * n ** 3, dtype=torch.float64, device="cuda:0")
        acr.acr_stencil_codi(n, T(cin), coef)
    else:
        st = stencil_poisson(cin, n)
        coef = torch.empty(7 * n ** 3, dtype=torch.float64, device="cuda:0")
        acr.acr_stencil_poisson(n, T(cin), coef)
    h = acr.Handle(n, coef, spec["eps"], eta, spec["leaf"], prec, 32)
    u = torch.zeros(n ** 3, dtype=torch.float64, device="cuda:0")
    method = acr.ACR_GMRES if spec["krylov"] == "gmres" else acr.ACR_PCG
    info, status = acr.acr_krylov_solve(h.h, coef, method, spec.get("restart", 30), spec["rtol"],
                                        1000, T(f), u)
    torch.cuda.synchronize()
    h.close()
    return spec, st, f, u.cpu().numpy(), info


def test_config_poisson_grf_n16_dense_lu(acr):
    """kappa = exp(GRF), n = 16, leaf 32, eta 1, eps 1e-6, PCG to 1e-10,
    checked against a dense LU solve."""
    spec, st, f, u, info = _solve_case(acr, "poisson_grf_n16", 16, 0, eta=1.0)
    A = stencil_matrix(st, 16).toarray()
    ue = np.linalg.solve(A, f)
    assert rel(A @ u, f) <= spec["rtol"] * 1.0001
    assert rel(u, ue) <= 10 * np.linalg.cond(A) * spec["rtol"]
    assert info.iterations <= 5


# BF16-stored factors are checked on the convection-diffusion recipe only: on
# the kappa-contrast-1e4 boxes their rounding leaves ||I - M^-1 A|| at 2.5
# (n = 32) and the FP64 Krylov iteration stalls; the FP32 form is the mixed
# form for that recipe.
@pytest.mark.parametrize("name,n,prec", [("poisson_boxes_n64", 32, 0), ("poisson_boxes_n64", 32, 1),
                                         ("codi_n128", 32, 0), ("codi_n128", 32, 1),
                                         ("codi_n128", 32, 2)])
def test_config_recipes_small_grid(acr, name, n, prec):
    spec, st, f, u, info = _solve_case(acr, name, n, prec)
    A = stencil_matrix(st, n)
    assert rel(A @ u, f) <= spec["rtol"] * 1.0001
    ue, cond = _direct_and_cond(name, n)
    assert rel(u, ue) <= 10 * cond * spec["rtol"]


@functools.lru_cache(maxsize=None)
def _direct_and_cond(name, n):
    spec, cin, f = workload(name, n=n)
    st = stencil_codi(cin, n) if spec["pde"] == "codi" else stencil_poisson(cin, n)
    A = stencil_matrix(st, n)
    return sla.splu(A.tocsc()).solve(f), cond_estimate(A, its=25)


@pytest.mark.parametrize("prec", [0, 1])
def test_helmholtz_recipe_small_grid(acr, prec):
    """The indefinite Helmholtz recipe at n = 32 (eps 1e-5, GMRES(30) to
    1e-8), first right-hand side: the oracle's SpMV confirms the residual and
    the solution is within 10 cond rtol of the direct solve; unpreconditioned
    GMRES(30) does not converge on it."""
    n = 32
    spec, sig, F = workload("helmholtz_n64", n=n)
    f = F[0]
    st = stencil_helmholtz(sig, n)
    coef = torch.empty(7 * n ** 3, dtype=torch.float64, device="cuda:0")
    acr.acr_stencil_helmholtz(n, T(sig), coef)
    h = acr.Handle(n, coef, spec["eps"], spec["eta"], 32, prec, 48)
    u = torch.zeros(n ** 3, dtype=torch.float64, device="cuda:0")
    info, status = acr.acr_krylov_solve(h.h, coef, acr.ACR_GMRES, 30, spec["rtol"], 300, T(f), u)
    torch.cuda.synchronize()
    h.close()
    A = stencil_matrix(st, n)
    uh = u.cpu().numpy()
    assert rel(A @ uh, f) <= spec["rtol"] * 1.0001
    assert info.iterations <= (5 if prec == 0 else 12)
    ue = sla.splu(A.tocsc()).solve(f)
    assert rel(uh, ue) <= 10 * cond_estimate(A, its=25) * spec["rtol"]
    u0 = torch.zeros(n ** 3, dtype=torch.float64, device="cuda:0")
    info0, st0 = acr.acr_krylov_solve_plain(n, coef, acr.ACR_GMRES, 30, spec["rtol"], 300,
                                            T(f), u0, check=False)
    assert st0 != 0


def test_full_size_codi_n128_fp32(acr):
    """The benchmark workload at full size (n = 128, FP32 factors, GMRES(30)):
    the oracle's own SpMV confirms the relative residual."""
    spec, st, f, u, info = _solve_case(acr, "codi_n128", 128, 1)
    assert info.converged
    assert rel(stencil_apply(st, 128, u), f) <= spec["rtol"] * 1.0001


def test_full_size_codi_n128_bf16(acr):
    """The benchmark workload at full size with BF16-stored factors: the FP64
    GMRES reaches the full tolerance (checked by the oracle's SpMV)."""
    spec, st, f, u, info = _solve_case(acr, "codi_n128", 128, 2)
    assert info.converged
    assert rel(stencil_apply(st, 128, u), f) <= spec["rtol"] * 1.0001


def test_bf16_form_halves_factor_bytes(acr):
    n, eta, leaf, eps = 16, 2.0, 32, 1e-2
    st, coef = operator(acr, "codi", n)
    infos = []
    for prec in (1, 2):
        h = acr.Handle(n, coef, eps, eta, leaf, prec, 32)
        infos.append(h.info())
        h.close()
    diag = 2 * n ** 3 * 8   # level-0 couplings stay FP64
    assert (infos[1].factor_bytes - diag) * 2 == infos[0].factor_bytes - diag
    assert infos[1].max_rank == infos[0].max_rank


def test_edge_cases(acr):
    # n = 1 (one plane, one point) and n = 2
    for n in (1, 2, 4):
        st, coef = operator(acr, "poisson", n)
        f = uniform_rhs(n, 7) if n > 1 else np.array([0.5])
        h = acr.Handle(n, coef, 1e-8, 2.0, 4, 0, 8)
        z = torch.empty(n ** 3, dtype=torch.float64, device="cuda:0")
        h.apply(T(f), z)
        torch.cuda.synchronize()
        A = stencil_matrix(st, n).toarray()
        assert rel(z.cpu().numpy(), np.linalg.solve(A, f)) <= 1e-10
        # zero right-hand side
        u = torch.ones(n ** 3, dtype=torch.float64, device="cuda:0")
        info, status = acr.acr_krylov_solve(h.h, coef, 0, 0, 1e-8, 10,
                                            torch.zeros_like(u), u)
        assert status == 0 and float(u.abs().max()) == 0.0
        h.close()


def test_error_statuses(acr):
    import ctypes
    n = 16
    st, coef = operator(acr, "codi", n)
    with pytest.raises(acr.AcrError) as e:
        acr.Handle(n, coef, 0.0, 2.0, 16)
    assert e.value.status == 1
    with pytest.raises(acr.AcrError) as e:
        acr.Handle(n, coef, 1e-2, 2.0, 16, 0, 49)
    assert e.value.status == 1
    with pytest.raises(acr.AcrError) as e:          # no such precision form
        acr.Handle(n, coef, 1e-2, 2.0, 16, 3)
    assert e.value.status == 1
    with pytest.raises(acr.AcrError) as e:          # leaves above 64 points
        acr.Handle(n, coef, 1e-2, 2.0, 128)
    assert e.value.status == 8
    with pytest.raises(acr.AcrError) as e:          # rank cap 1 at eps 1e-10
        acr.Handle(n, coef, 1e-10, 2.0, 16, 0, 1)
    assert e.value.status == 5
    lib = acr.load_library()
    assert lib.acr_apply(None, None, None, 1, None) == 1
    # the library stays usable after the errors
    h = acr.Handle(n, coef, 1e-2, 2.0, 16)
    h.close()


def test_profile_counts(acr):
    n = 16
    st, coef = operator(acr, "codi", n)
    h = acr.Handle(n, coef, 1e-2, 2.0, 16, 1, 16, flags=acr.ACR_FLAG_PROFILE)
    p = h.profile()
    info = h.info()
    assert p.gemm.launches > 0 and p.gemm.flops > 0 and p.gemm.ms > 0
    assert p.leaf_inv.launches > 0 and p.eig.launches > 0
    assert info.apply_bytes > info.factor_bytes
    h.close()


def test_breakdown_from_pivot_growth(acr):
    """Indefinite Helmholtz plane blocks built on the host to be (nearly)
    singular: with a uniform shift sigma equal to the smallest eigenvalue of
    D_k = 2D Laplacian + (2/h^2) I - sigma I (closed form, DST eigenpairs),
    the first-level leaf inverses (n = 4, leaf 16: one leaf per plane) have
    growth max|A| max|A^-1| above the storage precision's bound (1e10 for
    FP64 factors, 1e6 for float factors, whose rounding already perturbs the
    leaf) and the setup reports BREAKDOWN; a shift half-way between two
    eigenvalues sets up normally."""
    n = 4
    h = 1.0 / (n + 1)
    lam = lambda a, b: (4 / h ** 2) * (np.sin(a * np.pi * h / 2) ** 2
                                       + np.sin(b * np.pi * h / 2) ** 2) + 2 / h ** 2
    good = 0.5 * (lam(1, 1) + lam(1, 2))
    growth = lambda M: np.max(np.abs(M)) * np.max(np.abs(np.linalg.inv(M)))
    bound = {0: 1e10, 1: 1e6}
    for sig, expect_ok in ((lam(1, 1), False), (lam(1, 1) * (1 - 1e-13), False), (good, True)):
        sigma = np.full(n ** 3, sig)
        st = stencil_helmholtz(sigma, n)
        D, Ld, Ud = plane_blocks(st, n)
        stored = {0: D[1], 1: D[1].astype(np.float32).astype(np.float64)}
        coef = torch.empty(7 * n ** 3, dtype=torch.float64, device="cuda:0")
        acr.acr_stencil_helmholtz(n, T(sigma), coef)
        for prec in (0, 1):
            # the host-side expectation, on the leaf as the precision stores it
            assert (growth(stored[prec]) <= bound[prec]) == expect_ok
            if expect_ok:
                h_ = acr.Handle(n, coef, 1e-8, 2.0, 16, prec, 16)
                h_.close()
            else:
                with pytest.raises(acr.AcrError) as e:
                    acr.Handle(n, coef, 1e-8, 2.0, 16, prec, 16)
                assert e.value.status == 4
    # the library stays usable after the breakdowns
    st, coef = operator(acr, "codi", 8)
    acr.Handle(8, coef, 1e-3, 2.0, 8, 0, 16).close()
