"""Batches of problems of uneven size (GPU, through the C ABI): the mixed batch
of 12 kappa-Poisson instances at n in {32, 48, 64} (Gaussian-field kappa,
seeds 40-51), FP32 factors, eps 1e-2, eta 2, leaf 64, rank cap 24.

* every instance's batched apply equals the apply of a handle set up for
  that instance alone (the batch shares launches, not arithmetic);
* the first n = 32 instance matches the oracle's apply within the FP32
  parity bound of tests/test_gpu_parity.py (1e-5, or 5x the oracle's own
  float32-arithmetic model error);
* the setup + apply captured in one CUDA graph and replayed equals the
  uncaptured batch, and after the coefficient arrays are overwritten in
  place a replay equals a fresh setup of the new operator;
* refactoring, applying and replaying allocate nothing (the arena is sized
  once by the counting pass), and the batch issues fewer launches than the
  instances one at a time;
* each instance's PCG solve with its own preconditioner reaches 1e-8, the
  oracle's SpMV confirming the residual.
"""
import numpy as np
import pytest

from inputs import gaussian_field_kappa, uniform_rhs
from oracle.assembly import stencil_poisson, stencil_apply, plane_blocks
from oracle.cr import cr_setup, cr_apply
from oracle.hstructure import Structure

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NS = [32, 48, 64] * 4
SEEDS = list(range(40, 52))
EPS, ETA, LEAF, CAP = 1e-2, 2.0, 64, 24


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


def coef_of(acr, n, seed):
    c = torch.empty(7 * n ** 3, dtype=torch.float64, device="cuda:0")
    acr.acr_stencil_poisson(n, T(gaussian_field_kappa(n, seed)), c)
    return c


def single_apply(acr, n, coef, r):
    h = acr.Handle(n, coef, EPS, ETA, LEAF, acr.ACR_FP32, CAP)
    z = torch.empty(n ** 3, dtype=torch.float64, device="cuda:0")
    h.apply(T(r), z)
    torch.cuda.synchronize()
    h.close()
    return z.cpu().numpy()


def test_mixed_batch_of_12(acr, parity_log):
    coefs = [coef_of(acr, n, s) for n, s in zip(NS, SEEDS)]
    offs = np.concatenate([[0], np.cumsum([n ** 3 for n in NS])])
    r = np.concatenate([uniform_rhs(n, 100 + i) for i, n in enumerate(NS)])
    stream = torch.cuda.Stream()
    b = acr.acr_batch_create(NS, coefs, EPS, ETA, LEAF, acr.ACR_FP32, CAP, stream)
    try:
        rd = T(r)
        z = torch.empty_like(rd)
        launches0 = acr.acr_launch_count()
        acr.acr_batch_apply(b, rd, z, stream)
        stream.synchronize()
        batch_launches = acr.acr_launch_count() - launches0
        zb = z.cpu().numpy()
        # 1. each instance equals its own single-problem handle
        single_launches = 0
        for i, n in enumerate(NS):
            ri = r[offs[i]:offs[i + 1]]
            l0 = acr.acr_launch_count()
            zs = single_apply(acr, n, coefs[i], ri)
            single_launches += acr.acr_launch_count() - l0
            assert rel(zb[offs[i]:offs[i + 1]], zs) <= 1e-13, i
        # (the single applies include their setups; compare applies alone)
        h = acr.Handle(32, coefs[0], EPS, ETA, LEAF, acr.ACR_FP32, CAP)
        l0 = acr.acr_launch_count()
        zz = torch.empty(32 ** 3, dtype=torch.float64, device="cuda:0")
        h.apply(T(r[:32 ** 3]), zz)
        torch.cuda.synchronize()
        one_apply = acr.acr_launch_count() - l0
        h.close()
        assert batch_launches < 12 * one_apply
        # 2. the first n = 32 instance against the oracle
        st = stencil_poisson(gaussian_field_kappa(32, SEEDS[0]), 32)
        D, Ld, Ud = plane_blocks(st, 32)
        S = Structure(32, ETA, LEAF)
        zo = cr_apply(cr_setup(D, Ld, Ud, S, EPS), r[:32 ** 3])
        z32 = cr_apply(cr_setup(D, Ld, Ud, S, EPS, arith=np.float32), r[:32 ** 3])
        e2 = rel(zb[:32 ** 3], zo)
        tol = max(1e-5, 5 * rel(z32, zo))
        parity_log(test="batch_apply", n=32, seed=SEEDS[0], prec=1, err2=e2, tol=tol,
                   batch_launches=batch_launches, one_apply_launches=one_apply)
        assert e2 <= tol, (e2, tol)
        # 3. graph: setup + apply captured once, replayed; no allocation
        z2 = torch.zeros_like(rd)
        acr.acr_batch_capture(b, rd, z2, stream)
        a0 = acr.acr_alloc_count()
        for _ in range(2):
            acr.acr_batch_replay(b, stream)
            acr.acr_batch_status(b, stream)
            assert np.array_equal(z2.cpu().numpy(), zb)
        acr.acr_batch_refactor(b, stream)
        acr.acr_batch_apply(b, rd, z, stream)
        acr.acr_batch_status(b, stream)
        assert acr.acr_alloc_count() == a0
        assert np.array_equal(z.cpu().numpy(), zb)
        # new coefficients in place -> a replay refactors from them
        fresh = coef_of(acr, NS[0], 60)
        coefs[0].copy_(fresh)
        torch.cuda.synchronize()
        acr.acr_batch_replay(b, stream)
        acr.acr_batch_status(b, stream)
        zg = z2.cpu().numpy()
        assert rel(zg[:offs[1]], single_apply(acr, NS[0], fresh, r[:offs[1]])) <= 1e-13
        assert np.array_equal(zg[offs[1]:], zb[offs[1]:])
        # 4. per-instance PCG with the instance's own preconditioner
        for i in (0, 1, 2):
            n = NS[i]
            f = uniform_rhs(n, 200 + i)
            u = torch.zeros(n ** 3, dtype=torch.float64, device="cuda:0")
            info, s = acr.acr_batch_krylov_solve(b, i, coefs[i], acr.ACR_PCG, 0, 1e-8, 200,
                                                 T(f), u, stream)
            stream.synchronize()
            seed = 60 if i == 0 else SEEDS[i]
            sti = stencil_poisson(gaussian_field_kappa(n, seed), n)
            assert s == 0 and info.converged
            assert rel(stencil_apply(sti, n, u.cpu().numpy()), f) <= 1e-8 * 1.0001
    finally:
        acr.acr_batch_destroy(b)


def test_batch_argument_errors(acr):
    import ctypes
    lib = acr.load_library()
    assert lib.acr_batch_create(0, None, None, None, None, None) == 1
    c = coef_of(acr, 8, 1)
    with pytest.raises(acr.AcrError):
        acr.acr_batch_create([8], [c], 0.0, ETA, 8)                 # eps out of range
    b = acr.acr_batch_create([8, 8], [c, c], 1e-3, ETA, 8, acr.ACR_FP64)
    try:
        assert lib.acr_batch_replay(ctypes.c_void_p(b), None) == 1  # nothing captured yet
        r = torch.zeros(2 * 512, dtype=torch.float64, device="cuda:0")
        # the legacy stream cannot be captured
        assert lib.acr_batch_capture(ctypes.c_void_p(b), ctypes.c_void_p(r.data_ptr()),
                                     ctypes.c_void_p(r.data_ptr()), None) == 1
    finally:
        acr.acr_batch_destroy(b)
