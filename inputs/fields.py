"""Seeded coefficient fields and right-hand sides for the ACR workloads.

Every function returns float64 numpy arrays of length ``n**3`` (x fastest)
or ``(3, n**3)`` for a vector field.  Seeds go through
``numpy.random.default_rng`` so the same call gives the same bytes on any
machine.
"""
import numpy as np


def grid_coords(n):
    """Node coordinates (x, y, z), each of shape (n**3,), x fastest, h=1/(n+1)."""
    h = 1.0 / (n + 1)
    t = (np.arange(n) + 1.0) * h
    z, y, x = np.meshgrid(t, t, t, indexing="ij")
    return x.ravel(), y.ravel(), z.ravel()


def _se_sqrt_1d(n, length):
    """Symmetric square root of the 1D squared-exponential kernel matrix.

    K_ij = exp(-(x_i - x_j)^2 / (2 length^2)) on the interior nodes.  Negative
    eigenvalues (round-off of a numerically singular K) are clipped to zero.
    """
    h = 1.0 / (n + 1)
    t = (np.arange(n) + 1.0) * h
    d = t[:, None] - t[None, :]
    k = np.exp(-(d * d) / (2.0 * length * length))
    w, q = np.linalg.eigh(k)
    w = np.clip(w, 0.0, None)
    return (q * np.sqrt(w)) @ q.T


def gaussian_field_kappa(n, seed, length=0.2, variance=1.0):
    """kappa = exp(g), g a Gaussian random field with covariance
    variance * exp(-|r|^2 / (2 length^2)).

    The squared-exponential kernel factorises over the axes, so the 3D
    covariance on the grid is Kx (x) Ky (x) Kz and g = (Sx (x) Sy (x) Sz) xi with
    S the symmetric square root of the 1D kernel and xi ~ N(0, 1) iid; this
    samples the field exactly (no truncated expansion).
    """
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal((n, n, n))  # axes (z, y, x)
    s = _se_sqrt_1d(n, length)
    g = np.einsum("ai,bj,ck,ijk->abc", s, s, s, xi, optimize=True)
    return np.exp(np.sqrt(variance) * g).ravel()


def box_inclusions_kappa(n, seed, nbox=40, high=1.0e4, side=(0.05, 0.25)):
    """kappa = 1 with ``nbox`` axis-aligned boxes where kappa = ``high``.

    Each box side is U[side] per axis and its lower corner U[0, 1 - side];
    overlapping boxes stay at ``high``.  Evaluated at the grid nodes.
    """
    rng = np.random.default_rng(seed)
    x, y, z = grid_coords(n)
    kap = np.ones(n ** 3)
    for _ in range(nbox):
        sd = rng.uniform(side[0], side[1], size=3)
        lo = rng.uniform(0.0, 1.0 - sd)
        inside = ((x >= lo[0]) & (x <= lo[0] + sd[0]) &
                  (y >= lo[1]) & (y <= lo[1] + sd[1]) &
                  (z >= lo[2]) & (z <= lo[2] + sd[2]))
        kap[inside] = high
    return kap


def layered_speed(n, seed, layers=8, c_range=(1.0, 3.0)):
    """Piecewise-constant wave speed c(x) in ``layers`` slabs normal to x:
    the layers - 1 interfaces are sorted U(0, 1) positions, each slab's c is
    U[c_range].  Evaluated at the grid nodes, shape (n**3,)."""
    rng = np.random.default_rng(seed)
    cuts = np.sort(rng.uniform(0.0, 1.0, size=layers - 1))
    speeds = rng.uniform(c_range[0], c_range[1], size=layers)
    x, _, _ = grid_coords(n)
    return speeds[np.searchsorted(cuts, x)]


def helmholtz_omega(n, points_per_wavelength=10.0):
    """Angular frequency giving ``points_per_wavelength`` grid spacings per
    wavelength at c = 1: 2 pi / (ppw h), h = 1/(n+1)."""
    return 2.0 * np.pi * (n + 1) / points_per_wavelength


def codi_beta(n, magnitude=50.0):
    """Convection velocity beta = magnitude*(1,1,1)*(1 + 0.5 sin(2 pi x) sin(2 pi y))
    at the grid nodes, shape (3, n**3)."""
    x, y, _ = grid_coords(n)
    s = magnitude * (1.0 + 0.5 * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y))
    return np.stack([s, s, s])


def uniform_rhs(n, seed, nrhs=1):
    """f ~ U(-1, 1) iid per node; shape (n**3,) or (nrhs, n**3)."""
    rng = np.random.default_rng(seed)
    if nrhs == 1:
        return rng.uniform(-1.0, 1.0, size=n ** 3)
    return rng.uniform(-1.0, 1.0, size=(nrhs, n ** 3))


# Workloads of the benchmark suite: the PDE, its coefficient field and the
# preconditioner / Krylov settings.  eta = 2 (the paper's strong setting) for
# the cases that do not specify it; the n=16 case uses the eta it is
# specified with.  poisson_grad_n96 is the differentiable solve: kappa as in
# poisson_grf_n16, the observation u_obs solved from a second field (seed
# 100), finite-difference cells drawn with seed 101.
WORKLOADS = {
    "poisson_grf_n16": dict(pde="poisson", n=16, field="grf", field_seed=0,
                            rhs_seed=1, eps=1e-6, eta=1.0, leaf=32,
                            krylov="pcg", rtol=1e-10),
    "poisson_boxes_n64": dict(pde="poisson", n=64, field="boxes", field_seed=10,
                              rhs_seed=11, eps=1e-2, eta=2.0, leaf=64,
                              krylov="pcg", rtol=1e-8),
    "codi_n128": dict(pde="codi", n=128, field="codi", field_seed=None,
                      rhs_seed=20, eps=1e-2, eta=2.0, leaf=64,
                      krylov="gmres", rtol=1e-8, restart=30),
    "helmholtz_n64": dict(pde="helmholtz", n=64, field="layers", field_seed=30,
                          rhs_seed=31, nrhs=32, eps=1e-5, eta=2.0, leaf=64,
                          krylov="gmres", rtol=1e-8, restart=30),
    "poisson_grad_n96": dict(pde="poisson", n=96, field="grf", field_seed=0,
                             rhs_seed=1, obs_seed=100, fd_seed=101, fd_cells=20,
                             eps=1e-2, eta=2.0, leaf=64, krylov="pcg", rtol=1e-10),
}


def fd_cells(n, seed, count):
    """``count`` distinct node indices drawn uniformly (finite-difference
    checks of a gradient)."""
    return np.random.default_rng(seed).choice(n ** 3, size=count, replace=False)


def workload(name, n=None):
    """Return (spec, coefficient array, rhs) for a named workload.

    ``n`` overrides the grid size (same recipe, same seeds) for scaled-down
    parity cases.  The coefficient array is kappa (n**3,) for Poisson, beta
    (3, n**3) for convection-diffusion and the shift sigma = (omega/c)^2
    (n**3,) for Helmholtz; f is (nrhs, n**3) for multi-RHS workloads.
    """
    spec = dict(WORKLOADS[name])
    if n is not None:
        spec["n"] = n
    nn = spec["n"]
    if spec["field"] == "grf":
        coef = gaussian_field_kappa(nn, spec["field_seed"])
    elif spec["field"] == "layers":
        # the shift sigma = (omega / c)^2 of -Lap u - sigma u
        coef = (helmholtz_omega(nn) / layered_speed(nn, spec["field_seed"])) ** 2
    elif spec["field"] == "boxes":
        coef = box_inclusions_kappa(nn, spec["field_seed"])
    else:
        coef = codi_beta(nn)
    if spec.get("nrhs", 1) > 1:
        # seeds rhs_seed, rhs_seed + 1, ... one per right-hand side
        f = np.stack([uniform_rhs(nn, spec["rhs_seed"] + k) for k in range(spec["nrhs"])])
    else:
        f = uniform_rhs(nn, spec["rhs_seed"])
    return spec, coef, f
