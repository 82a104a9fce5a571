"""The allocation-free CG entry point (acr_krylov_solve_plain_noalloc),
called through the C ABI, against the allocating one
(acr_krylov_solve_plain with ACR_PCG) on two calls in a row.

It exists for callers that cannot call cudaMalloc where they solve (device
memory owned by another pool allocator, or loops that cannot take the
device synchronisation of an allocation); it keeps all its work in one
fixed device array.  This file is collected last so that a run stopping at
the first failure has run every other test before it."""
import numpy as np
import pytest

from inputs import gaussian_field_kappa, uniform_rhs
from oracle.assembly import stencil_poisson, stencil_apply

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_noalloc_cg_matches_allocating_entry_point():
    from paper_1712_08872_gb300 import _build
    _build.build()
    import paper_1712_08872_gb300 as acr
    n, rtol = 20, 1e-10
    kap = gaussian_field_kappa(n, 3)
    st = stencil_poisson(kap, n)
    dev = "cuda:0"
    kd = torch.tensor(kap, dtype=torch.float64, device=dev)
    coef = torch.empty(7 * n ** 3, dtype=torch.float64, device=dev)
    acr.acr_stencil_poisson(n, kd, coef)
    for call in range(2):                 # two calls in a row share the array
        f = uniform_rhs(n, 40 + call)
        fd = torch.tensor(f, dtype=torch.float64, device=dev)
        u_ref = torch.zeros_like(fd)
        a0 = acr.acr_alloc_count()
        info_ref, s_ref = acr.acr_krylov_solve_plain(n, coef, acr.ACR_PCG, 0, rtol, 2000, fd, u_ref)
        a1 = acr.acr_alloc_count()
        u = torch.zeros_like(fd)
        info, s = acr.acr_krylov_solve_plain_noalloc(n, coef, rtol, 2000, fd, u)
        torch.cuda.synchronize()
        # the allocating entry point allocates; the new one makes no
        # allocation of the library's (device or pinned host)
        assert a1 > a0 and acr.acr_alloc_count() == a1
        assert s == 0 and s_ref == 0
        assert info.iterations == info_ref.iterations
        uh, ur = u.cpu().numpy(), u_ref.cpu().numpy()
        # same criterion as the other Krylov parity tests: the oracle's SpMV
        # confirms the residual; the two solutions agree to well within
        # cond * rtol (identical kernels and reduction order: equal here)
        assert _rel(stencil_apply(st, n, uh), f) <= rtol * 1.0001
        assert _rel(uh, ur) <= 1e-12
    # grids beyond the fixed array are refused with a clear status
    big = int(round(acr.acr_noalloc_max_unknowns() ** (1 / 3))) + 1
    cb = torch.zeros(7 * big ** 3, dtype=torch.float64, device=dev)
    fb = torch.zeros(big ** 3, dtype=torch.float64, device=dev)
    _, s = acr.acr_krylov_solve_plain_noalloc(big, cb, rtol, 10, fb, fb.clone(), check=False)
    assert s == 1
