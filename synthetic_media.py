"""Seeded synthetic media and sources for periodic Helmholtz / Schroedinger solves.

This module only draws inputs: velocity fields c(x), potentials V(l*y) and
right-hand sides f on the periodic grid x_j = j*h, h = 1/n, of the unit torus
(Section 2.1 of the paper).  It holds none of the method's arithmetic (no shift
s, no q, no Green's function, no stencil): both the CPU oracle and the CUDA
library take these arrays as plain inputs.

Layout: every field is a flat float64 / complex128 array of length n**d with
axis 0 fastest, i.e. flat index j0 + n*j1 (+ n*n*j2).  As a numpy array of
shape (n,)*d in C order this is arr[j_{d-1}, ..., j_0].

Recipes (the paper leaves the media partly unspecified; the parameters below
are this project's choices and are listed with the configurations):
  * centre Gaussian: c = 1 + a*exp(-|x-x0|^2/(2 w^2)), periodic minimum image.
  * Gaussian random field (GRF): real part of ifft(sqrt(S_hat) * xi) with
    S_hat(k) = exp(-2 pi^2 lam^2 |k|^2) and xi complex normal, then shifted to
    zero mean and scaled to unit variance; c = 1 + 0.3*tanh(GRF).
  * lattice wells: V(x) = -sum_i d_i exp(-|x-x_i|^2/(2 w^2)) in l-units with
    one well at the centre of each unit cell of [0,l)^d, depths d_i ~ U[lo,hi].
  * Gaussian bump source: exp(-|x-x0|^2/(2 sigma^2)) times a phase e^{i theta}.
Seeds: medium seed 1000+i, right-hand-side seed 2000+i.
"""
from __future__ import annotations

import numpy as np

MEDIUM_SEED_BASE = 1000
RHS_SEED_BASE = 2000


def grid_coords(d: int, n: int) -> list[np.ndarray]:
    """Coordinates x_a = j_a / n of every grid point, as d arrays of shape (n,)*d.

    Returned in axis order (x_0, x_1, ...), each laid out as arr[j_{d-1},...,j_0].
    """
    one = np.arange(n, dtype=np.float64) / n
    mesh = np.meshgrid(*([one] * d), indexing="ij")  # mesh[a] varies along array axis a
    # array axis a corresponds to grid axis d-1-a
    return [mesh[d - 1 - a] for a in range(d)]


def _min_image_dist2(coords: list[np.ndarray], centre, period: float = 1.0) -> np.ndarray:
    r2 = np.zeros_like(coords[0])
    for a, xa in enumerate(coords):
        dx = xa - centre[a]
        dx -= period * np.round(dx / period)
        r2 += dx * dx
    return r2


def gaussian_bump(d: int, n: int, centre, width: float, amplitude: float = 1.0) -> np.ndarray:
    """Periodic (minimum image) Gaussian amplitude*exp(-|x-centre|^2/(2 width^2)), flat."""
    r2 = _min_image_dist2(grid_coords(d, n), centre)
    return (amplitude * np.exp(-r2 / (2.0 * width * width))).ravel()


def centre_gaussian_velocity(d: int, n: int, amplitude: float = -0.4, width: float = 0.1,
                             centre=None) -> np.ndarray:
    """c(x) = 1 + amplitude*exp(-|x-x0|^2/(2 width^2)), x0 the domain centre by default."""
    if centre is None:
        centre = [0.5] * d
    return 1.0 + gaussian_bump(d, n, centre, width, amplitude)


def gaussian_random_field(d: int, n: int, corr_len: float, seed: int) -> np.ndarray:
    """Zero-mean, unit-variance periodic Gaussian random field (flat float64)."""
    rng = np.random.default_rng(seed)
    shape = (n,) * d
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    ks = np.meshgrid(*([k1] * d), indexing="ij")
    k2 = sum(k * k for k in ks)
    spec = np.exp(-2.0 * np.pi ** 2 * corr_len ** 2 * k2)
    xi = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    field = np.fft.ifftn(np.sqrt(spec) * xi).real
    field -= field.mean()
    std = field.std()
    if std > 0:
        field /= std
    return field.ravel()


def grf_velocity(d: int, n: int, corr_len: float, seed: int, contrast: float = 0.3) -> np.ndarray:
    """c(x) = 1 + contrast*tanh(GRF(x))."""
    return 1.0 + contrast * np.tanh(gaussian_random_field(d, n, corr_len, seed))


def lattice_wells_potential(d: int, n: int, ell: float, seed: int, depth=(5.0, 15.0),
                            width: float = 0.15, missing_centre: bool = False) -> np.ndarray:
    """V(l*y) on the unit grid: one Gaussian well per unit cell of [0,l)^d (l-units).

    V(x) = -sum_i d_i exp(-|x - x_i|^2 / (2 width^2)), x_i = cell centres,
    d_i ~ U[depth], periodic minimum image with period l.  Returned as a flat
    array sampled at x = l * j / n.
    """
    rng = np.random.default_rng(seed)
    m = int(round(ell))
    coords = [c * ell for c in grid_coords(d, n)]
    V = np.zeros_like(coords[0])
    idx = np.indices((m,) * d).reshape(d, -1).T
    depths = rng.uniform(depth[0], depth[1], size=len(idx))
    centre_cell = tuple([m // 2] * d)
    for cell, dep in zip(idx, depths):
        if missing_centre and tuple(cell) == centre_cell:
            continue
        x0 = [(ci + 0.5) for ci in cell]
        r2 = _min_image_dist2(coords, x0, period=ell)
        V -= dep * np.exp(-r2 / (2.0 * width * width))
    return V.ravel()


def random_gaussian_source(d: int, n: int, seed: int, width: float = 0.05) -> np.ndarray:
    """Gaussian bump at a seeded uniform random centre times a seeded phase e^{i theta}."""
    rng = np.random.default_rng(seed)
    centre = rng.uniform(0.0, 1.0, size=d)
    theta = rng.uniform(0.0, 2.0 * np.pi)
    return gaussian_bump(d, n, centre, width).astype(np.complex128) * np.exp(1j * theta)


def random_complex_vector(N: int, seed: int) -> np.ndarray:
    """Complex normal test vector (real and imaginary parts N(0,1))."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(N) + 1j * rng.standard_normal(N)


# --------------------------------------------------------------------------------------
# Named workloads.  Each returns a dict of plain inputs: dimension d, grid n, leaf size b,
# the medium (kind + array + scalars) and the right-hand side f.
# --------------------------------------------------------------------------------------

def helmholtz_centre_gaussian_64(i: int = 0) -> dict:
    """2D 64x64, omega = 2 pi 8, c = 1 - 0.4 exp(-|x-(.5,.5)|^2/(2*0.1^2)),
    f = Gaussian of width 0.05 at (0.25, 0.25); leaf size b = 4."""
    d, n = 2, 64
    c = centre_gaussian_velocity(d, n, amplitude=-0.4, width=0.1)
    f = gaussian_bump(d, n, [0.25, 0.25], 0.05).astype(np.complex128)
    return dict(name="helmholtz2d_n64_centre_gaussian", d=d, n=n, b=4, kind="helmholtz",
                omega=2 * np.pi * 8, c=c, f=f)


def helmholtz_grf(d: int, n: int, b: int, omega: float, corr_len: float, i: int = 0) -> dict:
    c = grf_velocity(d, n, corr_len, MEDIUM_SEED_BASE + i)
    f = random_gaussian_source(d, n, RHS_SEED_BASE + i)
    return dict(name=f"helmholtz{d}d_n{n}_grf", d=d, n=n, b=b, kind="helmholtz",
                omega=omega, c=c, f=f)


def schrodinger_wells(d: int, n: int, b: int, ell: float, E: float, i: int = 0) -> dict:
    V = lattice_wells_potential(d, n, ell, MEDIUM_SEED_BASE + i)
    f = random_gaussian_source(d, n, RHS_SEED_BASE + i)
    return dict(name=f"schrodinger{d}d_n{n}_wells", d=d, n=n, b=b, kind="schrodinger",
                ell=ell, E=E, V=V, f=f)


def helmholtz_grf_512(i: int = 0) -> dict:
    """2D 512x512 Helmholtz, omega = 2 pi 64, c = 1 + 0.3 tanh(GRF, corr. length 0.05), b = 16."""
    return helmholtz_grf(2, 512, 16, 2 * np.pi * 64, 0.05, i)


def schrodinger_wells_512(i: int = 0) -> dict:
    """2D 512x512 Schroedinger, l = 16, E = 10, 16x16 lattice wells depth U[5,15] width 0.15, b = 16."""
    return schrodinger_wells(2, 512, 16, 16.0, 10.0, i)


def helmholtz_grf_3d(n: int = 128, b: int = 8, i: int = 0) -> dict:
    """3D Helmholtz on n^3, omega = 2 pi n/8, c = 1 + 0.3 tanh(GRF, corr. length 0.08)."""
    return helmholtz_grf(3, n, b, 2 * np.pi * n / 8, 0.08, i)


# ---------------------------------------------------------------- batched 2D problems
BATCH_SIZES = {128: 8, 192: 6, 256: 8, 384: 12, 512: 16}  # grid n -> leaf size b (n / b = 16 or 32)


def batched_2d_problems(count: int = 64, nrhs: int = 8, seed: int = 3000) -> list:
    """Heterogeneous 2D batch: grid sizes drawn uniformly from {128, 192, 256, 384, 512}
    (seeded), even-indexed problems Helmholtz (omega = 2 pi n / 8, c = 1 + 0.3 tanh(GRF,
    correlation length 0.05)), odd-indexed Schroedinger (an l x l lattice of Gaussian wells,
    l drawn from {4, 8, 16}, E = 10); nrhs random-centre, random-phase Gaussian sources
    each.  Problem i uses medium seed 1100 + i and source seeds 3000 + nrhs i + r."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice(sorted(BATCH_SIZES), size=count)
    ells = rng.choice([4.0, 8.0, 16.0], size=count)
    out = []
    for i in range(count):
        n = int(sizes[i])
        b = BATCH_SIZES[n]
        if i % 2 == 0:
            c = grf_velocity(2, n, 0.05, MEDIUM_SEED_BASE + 100 + i)
            p = dict(d=2, n=n, b=b, kind="helmholtz", omega=2 * np.pi * n / 8, c=c)
        else:
            V = lattice_wells_potential(2, n, float(ells[i]), MEDIUM_SEED_BASE + 100 + i)
            p = dict(d=2, n=n, b=b, kind="schrodinger", ell=float(ells[i]), E=10.0, V=V)
        p["rhs"] = [random_gaussian_source(2, n, RHS_SEED_BASE + 1000 + nrhs * i + r)
                    for r in range(nrhs)]
        out.append(p)
    return out



# ---------------------------------------------------------------- learned initial guess
def fno_initial_params(c_in: int = 3, width: int = 32, modes: int = 16, layers: int = 4,
                       hidden: int = 128, c_out: int = 2, seed: int = 4000) -> np.ndarray:
    """Seeded initial weights of the Fourier-layer network, flat float64 in the network's
    parameter order (lift P [W, c_in], p [W]; per layer R [2M, M, W, W, 2], W_l [W, W],
    b_l [W]; Q1 [H, W], c1 [H], Q2 [c_out, H], c2 [c_out]).  Pointwise weights and biases
    are uniform in +-1/sqrt(fan_in); the spectral weights' real and imaginary parts are
    uniform in [0, 1/W^2)."""
    rng = np.random.default_rng(seed)

    def lin(o, i):
        k = 1.0 / np.sqrt(i)
        return [rng.uniform(-k, k, size=(o, i)).ravel(), rng.uniform(-k, k, size=o)]

    W, M = width, modes
    parts = lin(W, c_in)
    for _ in range(layers):
        parts.append(rng.uniform(0.0, 1.0 / (W * W), size=(2 * M, M, W, W, 2)).ravel())
        parts += lin(W, W)
    parts += lin(hidden, W) + lin(c_out, hidden)
    return np.concatenate(parts)


def lattice_wells_potential_2d(n: int, ell: float, seed: int, depth=(5.0, 15.0),
                               width: float = 0.15) -> np.ndarray:
    """The 2D lattice_wells_potential in separable form: with the per-axis minimum image,
    exp(-r^2 / (2 w^2)) = ex(x) ey(y), so V = -ex^T D ey over the l x l cells (same seed,
    same depths, same values up to rounding; fast enough for thousands of media)."""
    rng = np.random.default_rng(seed)
    m = int(round(ell))
    depths = rng.uniform(depth[0], depth[1], size=m * m).reshape(m, m)  # [cell j1][cell j0]
    x = np.arange(n) * (ell / n)
    d = x[None, :] - (np.arange(m)[:, None] + 0.5)
    d = d - ell * np.round(d / ell)
    e = np.exp(-d * d / (2.0 * width * width))                           # [cell][point]
    # np.indices ordering: cell index (i0, i1) flattened with i1 fastest; i0 is axis 0 (j0)
    V = -np.einsum("ab,ay,bx->yx", depths.T, e, e)
    return V.ravel()


def lattice_wells_potential_3d(n: int, ell: float, seed: int, depth=(5.0, 15.0),
                               width: float = 0.15) -> np.ndarray:
    """The 3D lattice_wells_potential in separable form (per-axis minimum image:
    exp(-r^2 / (2 w^2)) = ex(x) ey(y) ez(z)); same seed, same depths, same values up to
    rounding, without one full-grid pass per well."""
    rng = np.random.default_rng(seed)
    m = int(round(ell))
    depths = rng.uniform(depth[0], depth[1], size=m ** 3).reshape(m, m, m)  # [i0][i1][i2]
    x = np.arange(n) * (ell / n)
    d = x[None, :] - (np.arange(m)[:, None] + 0.5)
    d = d - ell * np.round(d / ell)
    e = np.exp(-d * d / (2.0 * width * width))                              # [cell][point]
    V = -np.einsum("abc,ax,by,cz->zyx", depths, e, e, e, optimize=True)      # [j2][j1][j0]
    return V.ravel()


def schrodinger_wells_3d(n: int = 128, b: int = 8, ell: float = 8.0, E: float = 10.0,
                         i: int = 0) -> dict:
    """3D rescaled Schroedinger on n^3: an l x l x l lattice of Gaussian wells (depth
    U[5, 15], width 0.15 l-units, medium seed 1000 + i), E = 10, a random-centre,
    random-phase Gaussian source (seed 2000 + i)."""
    V = lattice_wells_potential_3d(n, ell, MEDIUM_SEED_BASE + i)
    f = random_gaussian_source(3, n, RHS_SEED_BASE + i)
    return dict(name=f"schrodinger3d_n{n}_wells", d=3, n=n, b=b, kind="schrodinger",
                ell=ell, E=E, V=V, f=f)
