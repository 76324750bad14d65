"""Seeded synthetic inputs shared by the CUDA path, the oracle-based tests and the bench.

This module draws random numbers and builds microstructures; it holds none of the
ADMM arithmetic.  Every array it returns is an *input* (phase maps, director
fields, macroscopic strains, request streams) that the caller hands, unchanged, to
both the CUDA library and the CPU oracle.

Randomness comes from one counter-based generator, SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), written
out here so that the streams are identical on every machine and numpy version.

Layout convention (shared with the C ABI): a scalar field on an N^d grid is a
C-ordered array of shape (N,)*d whose LAST axis is x (direction e_1), i.e.
``a[z, y, x]`` in 3D and ``a[y, x]`` in 2D.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TAGMUL = np.uint64(0xD1B54A32D192ED03)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (the 'mix' step of the published generator)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, tag: int, count: int, start: int = 0) -> np.ndarray:
    """Words start..start+count-1 of the stream (seed, tag): word i = mix(base + (i+1)*gamma)."""
    with np.errstate(over="ignore"):
        base = _mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(tag) * _TAGMUL))
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix64(base + idx * _GAMMA)


def uniform(seed: int, tag: int, count: int, start: int = 0) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits each."""
    return (splitmix64(seed, tag, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, tag: int, count: int) -> np.ndarray:
    """Standard normal deviates by the Box-Muller transform of two uniform streams."""
    u1 = uniform(seed, 2 * tag + 1, count)
    u2 = uniform(seed, 2 * tag + 2, count)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


# --------------------------------------------------------------------------- material maps

def laminate_phase(n: int, dim: int) -> np.ndarray:
    """Two-phase laminate with layers normal to e_1 and volume fraction 1/2.

    Phase 0 occupies voxels with x-index < n/2, phase 1 the rest.  One bilayer per
    cell.  With n divisible by 4 the exact laminate solution is representable on
    the central-difference grid.
    """
    ph = np.zeros((n,) * dim, dtype=np.uint8)
    ph[..., n // 2:] = 1
    return ph


def inclusion_phase(n: int, dim: int, seed: int, radius: int = 6,
                    target_fraction: float = 0.20, max_spheres: int = 1 << 20) -> np.ndarray:
    """Matrix (phase 0) with periodic spherical (circular in 2D) inclusions (phase 1).

    Centres are voxel centres drawn uniformly from the grid; a voxel belongs to an
    inclusion when its periodic integer distance to a centre is <= ``radius``
    voxels.  Spheres are added (overlap allowed) until the inclusion volume
    fraction reaches ``target_fraction``.  All geometry is integer arithmetic, so
    the map is bit-identical on every machine.
    """
    ph = np.zeros((n,) * dim, dtype=np.uint8)
    r = int(radius)
    off = np.arange(-r, r + 1)
    grids = np.meshgrid(*([off] * dim), indexing="ij")
    inside = sum(g * g for g in grids) <= r * r
    offs = [g[inside] for g in grids]           # offsets along axes 0..dim-1 (z,y,x order)
    target = int(np.ceil(target_fraction * ph.size))
    count = 0
    batch = 64
    drawn = 0
    while count < target and drawn < max_spheres:
        u = uniform(seed, 17, batch * dim, start=drawn * dim)   # sphere i uses words i*dim..i*dim+dim-1
        cs = np.minimum((u * n).astype(np.int64), n - 1).reshape(batch, dim)
        for c in cs:
            idx = tuple((c[a] + offs[a]) % n for a in range(dim))
            if n > 2 * r:  # the ball's voxels are distinct: count the new ones
                count += int(np.count_nonzero(ph[idx] == 0))
                ph[idx] = 1
            else:
                ph[idx] = 1
                count = int(np.count_nonzero(ph))
            drawn += 1
            if count >= target:
                break
    return ph


def disc_phase(n: int, dim: int, radius: float) -> np.ndarray:
    """One centred circular (spherical in 3D) inclusion (phase 1) of the given radius
    (in cell lengths) in a matrix (phase 0): a voxel is inside when its centre is."""
    c = (np.arange(n) + 0.5) / n - 0.5
    grids = np.meshgrid(*([c] * dim), indexing="ij")
    return (sum(g * g for g in grids) <= radius * radius).astype(np.uint8)


def director_grf(n: int, seed: int, corr: float = 8.0) -> np.ndarray:
    """Polydomain director field n0 on an n^3 grid, shape (3, n, n, n), unit length.

    Three i.i.d. standard-normal voxel fields are smoothed by periodic convolution
    with exp(-|x|^2 / (2 corr^2)) (x in voxel units) and normalised voxel by voxel
    (Section 5.3: a Gaussian random field filtered to a length scale).
    """
    g = normal(seed, 31, 3 * n ** 3).reshape(3, n, n, n)
    m = np.fft.fftfreq(n) * n
    d2 = m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2
    ker = np.exp(-d2 / (2.0 * corr * corr))
    kh = np.fft.rfftn(ker)
    f = np.fft.irfftn(np.fft.rfftn(g, axes=(1, 2, 3)) * kh[None], s=(n, n, n), axes=(1, 2, 3))
    nrm = np.sqrt(np.sum(f * f, axis=0))
    return f / nrm[None]


# --------------------------------------------------------------------------- macroscopic strains

def random_fbar(seed: int, tag: int, amp: float = 0.1) -> np.ndarray:
    """Fbar = I + sym(E) with E_ij ~ U[-amp, amp]; returned as a 3x3 row-major array."""
    e = (uniform(seed, tag, 9).reshape(3, 3) * 2.0 - 1.0) * amp
    return np.eye(3) + 0.5 * (e + e.T)


# --------------------------------------------------------------------------- Bloch-wave starts

def bloch_start(n: int, dim: int, seed: int) -> np.ndarray:
    """Start p_0 of the Bloch-wave iteration: complex (dim, n, ..., n) with independent
    standard-normal real and imaginary parts (tags 71 and 72)."""
    a = normal(seed, 71, dim * n ** dim).reshape((dim,) + (n,) * dim)
    b = normal(seed, 72, dim * n ** dim).reshape((dim,) + (n,) * dim)
    return a + 1j * b


# --------------------------------------------------------------------------- standard material tables

def lame_lambda(mu: float, nu: float) -> float:
    """Lame's first parameter from shear modulus and Poisson ratio."""
    return 2.0 * mu * nu / (1.0 - 2.0 * nu)


def two_phase_params(mu0: float, mu1: float, nu: float = 0.3) -> np.ndarray:
    """Per-phase (mu, lambda) table for a two-phase compressible neo-Hookean or linear cell."""
    return np.array([[mu0, lame_lambda(mu0, nu)], [mu1, lame_lambda(mu1, nu)]], dtype=np.float64)


# --------------------------------------------------------------------------- batch and serving streams

BATCH_SIZES = (32, 48, 64, 96, 128)


def batch_spec(count: int, seed: int):
    """Batch of RVEs of uneven sizes: N uniform over BATCH_SIZES, laminate when the
    per-RVE seed is even and inclusions when odd, Fbar = I + sym(E), |E_ij| <= 0.1."""
    u = uniform(seed, 41, count)
    out = []
    for i in range(count):
        n = BATCH_SIZES[min(int(u[i] * len(BATCH_SIZES)), len(BATCH_SIZES) - 1)]
        s = seed * 1000 + i
        kind = "laminate" if s % 2 == 0 else "inclusion"
        out.append({"n": n, "seed": s, "kind": kind, "Fbar": random_fbar(s, 43)})
    return out


def smooth_sizes(lo: int = 32, hi: int = 256):
    """Even integers in [lo, hi] of the form 2^a 3^b (a >= 1)."""
    out = []
    for a in range(1, 12):
        for b in range(0, 8):
            v = (2 ** a) * (3 ** b)
            if lo <= v <= hi:
                out.append(v)
    return sorted(out)


def serving_stream(count: int, seed: int, rate_hz: float = 200.0, lo: int = 32, hi: int = 256,
                   mix=(0.4, 0.4, 0.2)):
    """Poisson arrivals of RVE solve requests.

    Inter-arrival times are exponential with mean 1/rate_hz.  Grid sizes are
    log-uniform on [lo, hi] rounded (in log) to the nearest even 2^a 3^b.  The
    microstructure kind is laminate / inclusion / LCE with probabilities ``mix``.
    Fbar = I + sym(E) with |E_ij| <= 0.1.
    """
    u_t = uniform(seed, 51, count)
    u_n = uniform(seed, 52, count)
    u_k = uniform(seed, 53, count)
    sizes = np.array(smooth_sizes(lo, hi), dtype=np.float64)
    t = np.cumsum(-np.log1p(-u_t) / rate_hz)
    reqs = []
    for i in range(count):
        target = lo * (hi / lo) ** u_n[i]
        n = int(sizes[np.argmin(np.abs(np.log(sizes) - np.log(target)))])
        kind = "laminate" if u_k[i] < mix[0] else ("inclusion" if u_k[i] < mix[0] + mix[1] else "lce")
        reqs.append({"t": float(t[i]), "n": n, "kind": kind, "seed": seed * 100000 + i,
                     "Fbar": random_fbar(seed * 100000 + i, 54)})
    return reqs
