"""Seeded synthetic inputs shared by the tests, the bench and the oracle legs.

This module holds input generators and workload parameters only (random
fields, the stencil offset tables with the workloads' coefficients, the
sparse SPD test matrix, right-hand sides).  It performs none of the method's
arithmetic and imports neither the CUDA library nor the oracle, so both sides
can draw identical inputs from it.

Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state_i = seed + (i+1)*gamma
with gamma = 0x9E3779B97F4A7C15, output = mix64(state_i) with the two
xor-shift-multiply rounds of the published finaliser.  A double in [0, 1) is
(output >> 11) * 2^-53.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM = 0x632BE59BD9B4E019  # separates sub-streams of one seed


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs start..start+n-1 of the SplitMix64 sequence seeded with ``seed``."""
    idx = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, start: int = 0) -> np.ndarray:
    """n doubles uniform in [0, 1) (53-bit mantissa)."""
    return (splitmix64(seed, n, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def substream(seed: int, k: int) -> int:
    return (seed + k * _STREAM) & 0xFFFFFFFFFFFFFFFF


# --------------------------------------------------------------------------
# Stencil shapes (offset tables) and the workloads' coefficients
# --------------------------------------------------------------------------

def star_offsets(ndim: int, radius: int) -> list[tuple[int, int, int]]:
    """Centre first, then -x,+x,-y,+y,-z,+z at distance 1, then distance 2..."""
    offs = [(0, 0, 0)]
    for d in range(1, radius + 1):
        for axis in range(ndim):
            for sgn in (-1, 1):
                o = [0, 0, 0]
                o[axis] = sgn * d
                offs.append(tuple(o))
    return offs


def box_offsets(ndim: int, radius: int) -> list[tuple[int, int, int]]:
    """All offsets with |d| <= radius in the active dims, row-major (x fastest)."""
    rz = range(-radius, radius + 1) if ndim >= 3 else range(0, 1)
    ry = range(-radius, radius + 1) if ndim >= 2 else range(0, 1)
    return [(dx, dy, dz) for dz in rz for dy in ry for dx in range(-radius, radius + 1)]


SHAPES = {
    # name: (kind, ndim, radius) -- the benchmark names of Table 3
    "2d5pt": ("star", 2, 1),
    "2ds9pt": ("star", 2, 2),
    "2d13pt": ("star", 2, 3),
    "2d17pt": ("star", 2, 4),
    "2d9pt": ("box", 2, 1),
    "2d25pt": ("box", 2, 2),
    "3d7pt": ("star", 3, 1),
    "3d13pt": ("star", 3, 2),
    "3d27pt": ("box", 3, 1),
    "poisson": ("box19", 3, 1),  # Table 3's 19-point stencil: centre, 6 faces, 12 edges
}


def shape_offsets(name: str) -> list[tuple[int, int, int]]:
    kind, ndim, r = SHAPES[name]
    if kind == "star":
        return star_offsets(ndim, r)
    offs = box_offsets(ndim, r)
    if kind == "box19":  # the box without its 8 corners
        offs = [o for o in offs if not all(abs(d) == r for d in o)]
    return offs


def workload_weights(name: str, seed: int = 0) -> np.ndarray:
    """Coefficients of the synthetic workloads.

    2d5pt: every weight 0.2; 3d7pt: centre 0.4, each neighbour 0.1; box
    stencils of radius 1: uniform 1/npts; radius-2 stencils: seeded positive
    weights (0.5 + U[0,1)) normalised to sum 1.
    """
    offs = shape_offsets(name)
    n = len(offs)
    kind, ndim, r = SHAPES[name]
    if name == "2d5pt":
        return np.full(n, 0.2)
    if name == "3d7pt":
        w = np.full(n, 0.1)
        w[0] = 0.4
        return w
    if r == 1:
        return np.full(n, 1.0 / n)
    u = 0.5 + uniform(substream(seed, 7), n)
    return u / u.sum()


def stencil_field(shape: tuple[int, ...], seed: int) -> np.ndarray:
    """Interior field uniform in [0, 1), filled in row-major (x fastest) order."""
    n = int(np.prod(shape))
    return uniform(seed, n).reshape(shape)


# --------------------------------------------------------------------------
# Sparse SPD matrix and right-hand side for CG
# --------------------------------------------------------------------------

def csr_spd_matrix(n: int, seed: int, kmin: int = 3, kmax: int = 31, diag_factor: float = 1.05):
    """Symmetric, strictly diagonally dominant (hence SPD) CSR matrix.

    Row i draws k_i ~ U{kmin..kmax} partner columns j != i uniformly and a
    value v ~ U[-1, 0) for each; the pair sets A_ij = A_ji = v.  A pair drawn
    more than once keeps its first draw.  The diagonal is diag_factor times
    the absolute sum of the row's off-diagonals.  Returns (rowptr int32,
    col int32, val float64) with columns sorted within each row.
    """
    if n < 2:
        raise ValueError("n must be >= 2")
    k = kmin + np.floor(uniform(substream(seed, 1), n) * (kmax - kmin + 1)).astype(np.int64)
    m = int(k.sum())
    rows = np.repeat(np.arange(n, dtype=np.int64), k)
    cols = np.floor(uniform(substream(seed, 2), m) * (n - 1)).astype(np.int64)
    cols += (cols >= rows)
    vals = uniform(substream(seed, 3), m) - 1.0
    lo = np.minimum(rows, cols)
    hi = np.maximum(rows, cols)
    _, first = np.unique(lo * n + hi, return_index=True)
    first.sort()
    i, j, v = rows[first], cols[first], vals[first]
    absrow = np.bincount(np.concatenate([i, j]), weights=np.abs(np.concatenate([v, v])),
                         minlength=n)
    diag = diag_factor * absrow
    r_all = np.concatenate([i, j, np.arange(n, dtype=np.int64)])
    c_all = np.concatenate([j, i, np.arange(n, dtype=np.int64)])
    v_all = np.concatenate([v, v, diag])
    order = np.argsort(r_all * n + c_all, kind="stable")
    r_all, c_all, v_all = r_all[order], c_all[order], v_all[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(r_all, minlength=n), out=rowptr[1:])
    if rowptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("nnz exceeds int32")
    return rowptr.astype(np.int32), c_all.astype(np.int32), v_all.astype(np.float64)


def cg_rhs(n: int, seed: int) -> np.ndarray:
    """b uniform in [-1, 1)."""
    return 2.0 * uniform(substream(seed, 4), n) - 1.0


# Seeds of the synthetic workloads (one offset per configuration).
SEED_2D = 0
SEED_3D = 1
SEED_BATCH = 2
SEED_CG = 3
SEED_POISSON = 4


# --------------------------------------------------------------------------
# Batched uneven 2-D domains
# --------------------------------------------------------------------------

def batch_domains(count: int = 64, seed: int = SEED_BATCH, lo: int = 128, hi: int = 2048,
                  multiple: int = 8):
    """Square 2-D domains with sides log-uniform in [lo, hi], rounded to a
    multiple of `multiple` cells (so rows split into 16-byte vectors for every
    storage type); odd-indexed domains use the 3x3 box with weights 1/9,
    even-indexed ones the 5x5 box with seeded positive weights summing to 1.
    Returns a list of dicts (shape, name, offsets, weights, seed)."""
    u = uniform(substream(seed, 11), count)
    sides = np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))
    sides = np.clip(np.round(sides / multiple) * multiple, lo, hi).astype(int)
    out = []
    for i, s in enumerate(sides):
        if i % 2 == 1:
            name, w = "2d9pt", workload_weights("2d9pt")
        else:
            name, w = "2d25pt", workload_weights("2d25pt", seed=substream(seed, 100 + i))
        out.append(dict(shape=(int(s), int(s)), name=name, offsets=shape_offsets(name), weights=w,
                        seed=substream(seed, 1000 + i)))
    return out


# --------------------------------------------------------------------------
# Variable-coefficient Poisson: Gaussian random fields
# --------------------------------------------------------------------------

def normal(seed: int, n: int) -> np.ndarray:
    """n standard normal doubles by Box-Muller from two SplitMix64 streams."""
    u1 = uniform(substream(seed, 21), n)
    u2 = uniform(substream(seed, 22), n)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


def _grf_spectrum(n: int, ell: float, sigma: float):
    """Square roots of the eigenvalues of the circulant embedding of the
    squared-exponential covariance sigma^2 exp(-r^2 / (2 ell^2)) on an M x M
    torus (M a power of two >= max(2n, n + 8 ell)), scaled by 1/M."""
    m = 1
    while m < max(2 * n, n + 8 * ell):
        m *= 2
    d = np.minimum(np.arange(m), m - np.arange(m)).astype(np.float64)
    c = sigma ** 2 * np.exp(-(d[:, None] ** 2 + d[None, :] ** 2) / (2.0 * ell ** 2))
    lam = np.maximum(np.fft.fft2(c).real, 0.0)
    return np.sqrt(lam) / m, m


def grf(n: int, count: int, seed: int, ell: float = 32.0, sigma: float = 1.0) -> np.ndarray:
    """`count` n x n samples of a zero-mean stationary Gaussian field with
    covariance sigma^2 exp(-r^2 / (2 ell^2)) (r in cells), by circulant
    embedding (Dietrich & Newsam 1997): F(sqrt(lambda / M^2) xi) for complex
    standard normal xi gives two independent fields (real and imaginary
    parts); each is cropped to its top-left n x n block."""
    sq, m = _grf_spectrum(n, ell, sigma)
    out = np.empty((count, n, n))
    for i in range((count + 1) // 2):
        s = substream(seed, 1000 + i)
        xi = normal(s, m * m).reshape(m, m) + 1j * normal(substream(s, 1), m * m).reshape(m, m)
        z = np.fft.fft2(sq * xi)
        out[2 * i] = z.real[:n, :n]
        if 2 * i + 1 < count:
            out[2 * i + 1] = z.imag[:n, :n]
    return out


def poisson_problems(n: int, count: int, seed: int = SEED_POISSON, ell: float = 32.0, sigma: float = 1.0):
    """(k, f): k = exp(GRF), f uniform in [-1, 1); arrays (count, n, n)."""
    k = np.exp(grf(n, count, substream(seed, 31), ell, sigma))
    f = 2.0 * uniform(substream(seed, 32), count * n * n).reshape(count, n, n) - 1.0
    return k, f


def poisson_problems_device(n: int, count: int, seed: int = SEED_POISSON, ell: float = 32.0, sigma: float = 1.0,
                            device: str = "cuda"):
    """The same construction drawn on the device for large batches: torch's
    seeded generator supplies the normals and uniforms, torch.fft the
    transform (input synthesis only; different numbers from `poisson_problems`
    with the same distribution)."""
    import torch
    sq, m = _grf_spectrum(n, ell, sigma)
    sq_t = torch.from_numpy(sq).to(device)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    k = torch.empty((count, n, n), dtype=torch.float64, device=device)
    chunk = 16
    for i0 in range(0, (count + 1) // 2, chunk):
        i1 = min((count + 1) // 2, i0 + chunk)
        xi = torch.complex(torch.randn((i1 - i0, m, m), generator=g, dtype=torch.float64, device=device),
                           torch.randn((i1 - i0, m, m), generator=g, dtype=torch.float64, device=device))
        z = torch.fft.fft2(sq_t * xi)[:, :n, :n]
        for j in range(i1 - i0):
            a = 2 * (i0 + j)
            k[a] = z[j].real
            if a + 1 < count:
                k[a + 1] = z[j].imag
    k.exp_()
    f = torch.rand((count, n, n), generator=g, dtype=torch.float64, device=device).mul_(2.0).sub_(1.0)
    return k, f
