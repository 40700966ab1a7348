"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This module holds none of the lattice Boltzmann arithmetic: it produces
velocity / density fields, random distribution arrays, body forces and block
refinement patterns from fixed seeds.  Every array is float64 and laid out
[z][y][x] (x fastest), with vector fields as [3][z][y][x].

The workloads stand in for the paper's turbulent jet (Section 3, whose
experimental data are not available): a Taylor-Green vortex, a decaying
random-phase turbulence field, and round jets on nested block grids.
"""
import math

import numpy as np

BLOCK = 8


def grid_coords(NX, NY, NZ):
    """Cell-centre coordinates (x+1/2, y+1/2, z+1/2) broadcastable to [z][y][x]."""
    x = (np.arange(NX) + 0.5)[None, None, :]
    y = (np.arange(NY) + 0.5)[None, :, None]
    z = (np.arange(NZ) + 0.5)[:, None, None]
    return x, y, z


def taylor_green_3d(N, u0, shape=None):
    """u = u0 (sin kx cos ky cos kz, -cos kx sin ky cos kz, 0), k = 2 pi / N, rho = 1."""
    NX, NY, NZ = shape if shape is not None else (N, N, N)
    x, y, z = grid_coords(NX, NY, NZ)
    k = 2.0 * math.pi / N
    u = np.zeros((3, NZ, NY, NX))
    u[0] = u0 * np.sin(k * x) * np.cos(k * y) * np.cos(k * z)
    u[1] = -u0 * np.cos(k * x) * np.sin(k * y) * np.cos(k * z)
    return np.ones((NZ, NY, NX)), u


def taylor_green_2d(N, u0, NZ=8):
    """2-D Taylor-Green vortex in the x-y plane, constant along z."""
    x, y, z = grid_coords(N, N, NZ)
    k = 2.0 * math.pi / N
    u = np.zeros((3, NZ, N, N))
    u[0] = u0 * np.sin(k * x) * np.cos(k * y) * np.ones_like(z)
    u[1] = -u0 * np.cos(k * x) * np.sin(k * y) * np.ones_like(z)
    return np.ones((NZ, N, N)), u


def shear_wave(NX, NY, NZ, amp, drift_y=0.0, ly=None):
    """u_x = amp sin(2 pi y / ly), u_y = drift_y, rho = 1 (cell centres)."""
    ly = NY if ly is None else ly
    x, y, z = grid_coords(NX, NY, NZ)
    u = np.zeros((3, NZ, NY, NX))
    u[0] = amp * np.sin(2.0 * math.pi * y / ly) * np.ones_like(x) * np.ones_like(z)
    u[1] = drift_y
    return np.ones((NZ, NY, NX)), u


def spectrum_field(N, k0=4.0, urms=0.04, seed=1206):
    """Random-phase solenoidal field with E(k) ~ k^4 exp(-2 (k/k0)^2).

    Built in Fourier space: random complex amplitudes are projected on the
    plane normal to k (divergence free), scaled to the target spectrum and
    transformed back; the real field is normalised to
    u_rms = sqrt(<|u|^2>/3) = urms.  rho = 1.
    """
    rng = np.random.default_rng(seed)
    kk = np.fft.fftfreq(N, d=1.0 / N)
    kz, ky, kx = np.meshgrid(kk, kk, kk, indexing="ij")
    kmag = np.sqrt(kx * kx + ky * ky + kz * kz)
    a = rng.standard_normal((3, N, N, N)) + 1j * rng.standard_normal((3, N, N, N))
    kvec = np.stack([kx, ky, kz])
    with np.errstate(invalid="ignore", divide="ignore"):
        khat = np.where(kmag > 0, kvec / kmag, 0.0)
    a = a - khat * (khat * a).sum(0)
    with np.errstate(divide="ignore"):
        E = kmag ** 4 * np.exp(-2.0 * (kmag / k0) ** 2)
        amp = np.where(kmag > 0, np.sqrt(E / (4.0 * math.pi * np.maximum(kmag, 1e-30) ** 2)), 0.0)
    a = a * amp
    u = np.real(np.fft.ifftn(a, axes=(1, 2, 3)))
    u -= u.mean(axis=(1, 2, 3), keepdims=True)
    u *= urms / math.sqrt((u * u).sum(0).mean() / 3.0)
    return np.ones((N, N, N)), u


def random_distributions(Q, shape, seed, amp=0.05, base=None):
    """Random distribution array (Q, NZ, NY, NX): base_i (1 + amp U[-1, 1)).

    base defaults to 1/Q for every i; these states are far from equilibrium,
    which exercises every moment of a collision.
    """
    rng = np.random.default_rng(seed)
    b = np.full(Q, 1.0 / Q) if base is None else np.asarray(base, dtype=np.float64)
    noise = rng.uniform(-1.0, 1.0, (Q,) + tuple(shape))
    return b[:, None, None, None] * (1.0 + amp * noise)


def random_fluctuations(Q, shape, seed, amp=0.01):
    """Random small values (Q, NZ, NY, NX) in [-amp/Q, amp/Q): a fluctuation state."""
    rng = np.random.default_rng(seed)
    return (amp / Q) * rng.uniform(-1.0, 1.0, (Q,) + tuple(shape))


def random_force(shape, seed, sigma=1e-6):
    """Body force (3, NZ, NY, NX) with N(0, sigma^2) entries."""
    rng = np.random.default_rng(seed)
    return sigma * rng.standard_normal((3,) + tuple(shape))


def random_directions(n, shape, seed):
    """n unit-norm Gaussian directions of shape (3, NZ, NY, NX)."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3) + tuple(shape))
    return d / np.sqrt((d * d).reshape(n, -1).sum(1))[:, None, None, None, None]


# ---------------------------------------------------------------- block grids

def refine_radial(nb, centre, radius):
    """Level-0 refine flags (nbz, nby, nbx): blocks whose centre (y, z) lies
    within `radius` coarse cells of the axis (y, z) = centre, along all of x."""
    nbx, nby, nbz = nb
    by = np.arange(nby) * BLOCK + BLOCK / 2.0
    bz = np.arange(nbz) * BLOCK + BLOCK / 2.0
    r2 = (by[None, :] - centre[0]) ** 2 + (bz[:, None] - centre[1]) ** 2
    col = r2 < radius * radius
    return np.repeat(col[:, :, None], nbx, axis=2)


def refine_ring(nb_level, scale, centre, r_in, r_out, x_range=None):
    """Refine flags of a level whose block grid is nb_level and whose cell size
    is 1/scale coarse cells: blocks with centre radius in [r_in, r_out)."""
    nbx, nby, nbz = nb_level
    h = BLOCK / scale
    by = (np.arange(nby) + 0.5) * h
    bz = (np.arange(nbz) + 0.5) * h
    r2 = (by[None, :] - centre[0]) ** 2 + (bz[:, None] - centre[1]) ** 2
    col = (r2 >= r_in * r_in) & (r2 < r_out * r_out)
    flags = np.repeat(col[:, :, None], nbx, axis=2)
    if x_range is not None:
        bx = (np.arange(nbx) + 0.5) * h
        flags &= ((bx >= x_range[0]) & (bx < x_range[1]))[None, None, :]
    return flags


def expand_children(flags):
    """Block flags of the children of flagged blocks (2x along each axis)."""
    return flags.repeat(2, 0).repeat(2, 1).repeat(2, 2)


def dilate_blocks(flags, periodic_x):
    out = flags.copy()
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                r = np.roll(flags, (dz, dy, dx), axis=(0, 1, 2))
                if not periodic_x and dx == 1:
                    r[:, :, 0] = False
                if not periodic_x and dx == -1:
                    r[:, :, -1] = False
                out |= r
    return out


def jet_two_level(nbx=48, nby=24, nbz=24, radius=24.0):
    """Round-jet grid: coarse blocks, one refined level covering the cylinder
    of the given radius around the axis through the centre of the y-z face."""
    centre = (nby * BLOCK / 2.0, nbz * BLOCK / 2.0)
    return [refine_radial((nbx, nby, nbz), centre, radius)], centre


def jet_three_level(nbx=64, nby=32, nbz=32, r1=(4.0, 36.0), r2=(12.0, 24.0), x1=None, x2=None):
    """Three-level jet grid: level 1 is a thick ring (r1, coarse cells) around
    the axis over x in x1 (coarse cells, default all), level 2 a thinner ring
    (r2) along the shear layer r ~ D/2 inside it over x in x2; level-2 flags
    are trimmed so every flagged level-1 block keeps a full ring of level-1
    neighbours (the nesting rule)."""
    centre = (nby * BLOCK / 2.0, nbz * BLOCK / 2.0)
    nb0 = (nbx, nby, nbz)
    f0 = refine_ring(nb0, 1, centre, r1[0], r1[1], x1)
    region1 = expand_children(f0)
    nb1 = (2 * nbx, 2 * nby, 2 * nbz)
    f1 = refine_ring(nb1, 2, centre, r2[0], r2[1], x2) & region1
    # nesting: a refined level-1 block needs all 26 neighbours inside level 1
    ok = ~dilate_blocks(~region1, periodic_x=False)
    f1 &= ok
    return [f0, f1], centre


def jet_paper_scale():
    """The 3-level jet at the paper's scale: coarse 512 x 256 x 256 in 8^3
    blocks, nozzle D = 32 at x = 0 on the axis; level 1 a ring 8 <= r < 24
    coarse cells over x < 192, level 2 a ring 12 <= r < 24 around the shear
    layer r = D/2 over x < 96.  Active cells 33.21 M + 2.16 M + 4.72 M =
    40.09 M (4.0e7 + 0.2 %, 1.08e9 D3Q27 values)."""
    return jet_three_level(64, 32, 32, r1=(8.0, 24.0), r2=(12.0, 24.0), x1=(0, 192), x2=(0, 96))
