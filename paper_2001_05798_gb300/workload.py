"""Seeded synthetic inputs for the steady groundwater flow solve.

This module only draws inputs: conductivity fields, well positions,
boundary descriptors.  It holds none of the solver's arithmetic, so both the
CUDA path and the CPU oracle take their inputs from here.

The paper's benchmarks use homogeneous K and synthetic lognormal K fields with
sigma^2_lnK = 10 on 2D (275,000 cells) and 3D (2.75M cells, 10 layers) grids
(Benchmarking Examples section); the fields themselves are not published, so
seeded Gaussian lnK fields of the stated shape stand in for them.

Layout: a field on an nx*ny*nz grid is a C-order array of shape (nz, ny, nx),
so cell (x, y, z) has flat index i = x + nx*(y + ny*z).
"""
import hashlib

import numpy as np

NOFLOW, DIRICHLET = 0, 1
# boundary faces in the order -x, +x, -y, +y, -z, +z
FACES = ("-x", "+x", "-y", "+y", "-z", "+z")


def lnk_field(nx, ny, nz, var, corr, seed):
    """Gaussian lnK field, mean 0, variance ``var``, exponential covariance
    C(r) = var * exp(-sqrt(sum_d (r_d / corr_d)^2)), drawn by circulant
    embedding (Dietrich & Newsam 1997): the covariance is evaluated at the
    minimum-image lags of a grid padded to twice the size on every axis with
    more than one cell, its FFT eigenvalues are clipped at zero, and
    real(IFFT(sqrt(eig) * FFT(W))) with W ~ N(0,1) (numpy default_rng(seed),
    C order on the padded grid) is cut back to the grid.  Not renormalised.

    Returns (lnK of shape (nz, ny, nx), clipped eigenvalue fraction)."""
    if np.isscalar(corr):
        corr = (corr, corr, corr)
    dims = (nz, ny, nx)
    lam = (float(corr[2]), float(corr[1]), float(corr[0]))
    m = tuple(1 if d == 1 else 2 * d for d in dims)
    axes = []
    for mi, li in zip(m, lam):
        k = np.arange(mi, dtype=np.float64)
        axes.append(np.minimum(k, mi - k) / li)
    r2 = axes[0][:, None, None] ** 2 + axes[1][None, :, None] ** 2 + axes[2][None, None, :] ** 2
    c = var * np.exp(-np.sqrt(r2))
    del r2
    eig = np.fft.rfftn(c).real
    del c
    clipped = float(np.count_nonzero(eig < 0)) / eig.size
    np.maximum(eig, 0.0, out=eig)
    np.sqrt(eig, out=eig)
    rng = np.random.default_rng(seed)
    W = rng.standard_normal(m)
    F = np.fft.rfftn(W)
    del W
    F *= eig
    del eig
    f = np.fft.irfftn(F, s=m, axes=(0, 1, 2))
    del F
    return np.ascontiguousarray(f[:nz, :ny, :nx]), clipped


def wells(nx, ny, nz, count, seed, rate):
    """Point sinks/sources: ``count`` distinct cells below the top layer drawn
    by default_rng(seed).choice(nx*ny*(nz-1), count, replace=False), each with
    source term ``rate`` (volume per time; negative = pumping)."""
    q = np.zeros(nx * ny * nz)
    pool = nx * ny * max(nz - 1, 1)
    idx = np.random.default_rng(seed).choice(pool, count, replace=False)
    q[idx] = rate
    return q, np.sort(idx)


def cells(n, count, seed):
    """``count`` distinct cell indices drawn by default_rng(seed)."""
    return np.sort(np.random.default_rng(seed).choice(n, count, replace=False))


def sha256(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def problem(nx, ny, nz, var=0.0, corr=8.0, seed=1, kz_ratio=1.0, bct=(DIRICHLET, DIRICHLET, 0, 0, 0, 0),
            bcv=(1.0, 0.0, 0.0, 0.0, 0.0, 0.0), wells_count=0, wells_seed=3, wells_rate=-1e-3):
    """One flow problem: dict with nx, ny, nz, Kx, Ky, Kz (flat float64), bct, bcv, q.
    var = 0 gives K = 1 everywhere.  Kz = K / kz_ratio (Kh/Kv anisotropy)."""
    n = nx * ny * nz
    if var > 0.0:
        lnk, clipped = lnk_field(nx, ny, nz, var, corr, seed)
        K = np.exp(lnk).ravel()
    else:
        K, clipped = np.ones(n), 0.0
    Kz = K if kz_ratio == 1.0 else K / kz_ratio
    q = None
    well_idx = None
    if wells_count:
        q, well_idx = wells(nx, ny, nz, wells_count, wells_seed, wells_rate)
    return dict(nx=nx, ny=ny, nz=nz, Kx=K, Ky=K, Kz=Kz, bct=tuple(bct), bcv=tuple(float(v) for v in bcv),
                q=q, wells=well_idx, clipped=clipped)


def homogeneous_2d_128():
    """2D homogeneous flow, 128x128 cells, K = 1, h = 1 on -x, h = 0 on +x, no-flow
    elsewhere; the head is linear in x."""
    return problem(128, 128, 1)


def heterogeneous_3d(side=128, var=4.0, corr=8.0, seed=1):
    """3D heterogeneous flow, side^3 cells, lnK variance ``var``, exponential
    covariance with correlation length ``corr`` cells, h = 1 / h = 0 on the
    x faces, no-flow elsewhere."""
    return problem(side, side, side, var=var, corr=corr, seed=seed)


def layered_wells_3d(nx=256, ny=256, nz=128, var=1.0, corr=(32.0, 32.0, 4.0), seed=2, kz_ratio=10.0,
                     wells_count=16, wells_seed=3, wells_rate=-1e-3):
    """3D layered anisotropic flow: lnK variance 1, correlation lengths 32/32/4
    cells, Kh/Kv = 10, pumping wells of -1e-3 per cell below the top layer,
    fixed head h = 0 on the top (+z) face, no-flow elsewhere."""
    return problem(nx, ny, nz, var=var, corr=corr, seed=seed, kz_ratio=kz_ratio,
                   bct=(0, 0, 0, 0, 0, DIRICHLET), bcv=(0, 0, 0, 0, 0, 0.0),
                   wells_count=wells_count, wells_seed=wells_seed, wells_rate=wells_rate)


def lnk_field_device(nx, ny, nz, var, corr, seed, device="cuda", pad=1):
    """The same circulant-embedding recipe as lnk_field, drawn on a torch
    device (white noise from torch.Generator(device).manual_seed(seed)), for
    request streams where thousands of fields are needed.  The padded grid is
    twice the size on every axis with more than one cell, rounded up to a
    multiple of ``pad``: any periodic domain of at least twice the size embeds
    the covariance at every lag of the grid, and a few padded sizes let the
    FFT plans be reused across requests of different sizes.  Returns a
    float64 tensor of nx*ny*nz values (C order (nz, ny, nx))."""
    import torch

    if np.isscalar(corr):
        corr = (corr, corr, corr)
    dims = (nz, ny, nx)
    lam = (float(corr[2]), float(corr[1]), float(corr[0]))
    m = tuple(1 if d == 1 else -(-2 * d // pad) * pad for d in dims)
    axes = []
    for mi, li in zip(m, lam):
        k = torch.arange(mi, dtype=torch.float64, device=device)
        axes.append(torch.minimum(k, mi - k) / li)
    r2 = axes[0][:, None, None] ** 2 + axes[1][None, :, None] ** 2 + axes[2][None, None, :] ** 2
    eig = torch.fft.rfftn(var * torch.exp(-torch.sqrt(r2))).real.clamp_min_(0.0).sqrt_()
    del r2
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    W = torch.randn(m, generator=gen, dtype=torch.float64, device=device)
    f = torch.fft.irfftn(torch.fft.rfftn(W) * eig, s=m, dim=(0, 1, 2))
    return f[:nz, :ny, :nx].contiguous().reshape(-1)


def serving_requests(count=2000, seed=4, side_range=(32, 160), var_range=(0.5, 4.0), corr_range=(4.0, 16.0),
                     field_seed0=1000):
    """The request mix of the serving stream: side = round(exp(U[ln a, ln b])),
    lnK variance ~ U[var_range], correlation length ~ U[corr_range], request r
    drawing its field with seed field_seed0 + r."""
    rng = np.random.default_rng(seed)
    sides = np.rint(np.exp(rng.uniform(np.log(side_range[0]), np.log(side_range[1]), count))).astype(int)
    var = rng.uniform(var_range[0], var_range[1], count)
    corr = rng.uniform(corr_range[0], corr_range[1], count)
    return [dict(id=r, side=int(sides[r]), var=float(var[r]), corr=float(corr[r]), seed=field_seed0 + r)
            for r in range(count)]


def poisson_arrivals(count, rate, seed=4):
    """Arrival times (s) of a Poisson process of the given rate."""
    return np.cumsum(np.random.default_rng(seed + 1).exponential(1.0 / rate, count))
