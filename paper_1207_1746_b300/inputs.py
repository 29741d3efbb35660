"""Seeded synthetic inputs for the five stencil workloads.

This module draws numbers and lays out dense host arrays; it holds none of
the stencil arithmetic.  Both the CUDA path (through the benchmark and the
tests) and the CPU oracle consume what it returns.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): the i-th draw of stream ``seed``
is the SplitMix64 finaliser applied to ``seed + (i + 1) * 0x9E3779B97F4A7C15``
(mod 2^64), and a uniform double in [0, 1) is its top 53 bits times 2^-53.

Every array returned is a dense float64 array of shape
``(nz + 2hz, ny + 2hy, nx + 2hx)`` (x fastest) that includes the halo, so the
same array can be uploaded to a device grid or wrapped by the oracle.
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Draws ``start .. start+count-1`` of stream ``seed`` as uint64."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    return (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(seed: int, count: int, lo: float, hi: float, start: int = 0) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, count, start)


def padded_shape(n, halo):
    nx, ny, nz = n
    hx, hy, hz = halo
    return (nz + 2 * hz, ny + 2 * hy, nx + 2 * hx)


def interior_view(a: np.ndarray, n, halo) -> np.ndarray:
    nx, ny, nz = n
    hx, hy, hz = halo
    return a[hz:hz + nz, hy:hy + ny, hx:hx + nx]


def random_interior(seed: int, n, halo, lo: float, hi: float, halo_value: float = 0.0) -> np.ndarray:
    """Interior uniform in [lo, hi) in (k, j, i) order from stream ``seed``; halo constant."""
    a = np.full(padded_shape(n, halo), halo_value, dtype=np.float64)
    nx, ny, nz = n
    interior_view(a, n, halo)[...] = uniform(seed, nx * ny * nz, lo, hi).reshape(nz, ny, nx)
    return a


# ---------------------------------------------------------------- workload 1
def laplace2d(seed: int = 101, n: int = 256) -> np.ndarray:
    """2D Laplace/Jacobi input: an n x n interior uniform in [0, 1) and a 1-cell halo
    holding sin(pi x) with x_i = (i + 1) / (n + 1), i = -1 .. n, on every halo cell
    (so the x = 0 and x = 1 edges hold sin(0) and sin(pi) as rounded by libm)."""
    a = random_interior(seed, (n, n, 1), (1, 1, 0), 0.0, 1.0)
    x = np.array([math.sin(math.pi * (i + 1) / (n + 1)) for i in range(-1, n + 1)])
    a[0, 0, :] = x
    a[0, -1, :] = x
    a[0, :, 0] = x[0]
    a[0, :, -1] = x[-1]
    return a


# ---------------------------------------------------------------- workload 2
def heat3d(seed: int = 202, n: int = 256):
    """3D heat / damped Jacobi inputs: u0 = 0 with a zero 1-cell halo and an RHS f
    uniform in [-1, 1) on the interior (zero halo).  Returns (u0, f)."""
    shape = (n, n, n)
    u0 = np.zeros(padded_shape(shape, (1, 1, 1)), dtype=np.float64)
    f = random_interior(seed, shape, (1, 1, 1), -1.0, 1.0)
    return u0, f


# ---------------------------------------------------------------- workload 3
CLIMATE_FIELDS = ("q0", "q1", "q2", "kappa", "w", "t0", "t1", "t2")


def smooth_field(seed: int, n, halo) -> np.ndarray:
    """Sum of three random-phase sinusoids, each of amplitude 1/3, plus 1e-3 uniform
    noise in [-1, 1), evaluated on every cell including the halo.  Wave numbers a, b, c
    are integers in [1, 4] and phases uniform in [0, 2 pi), drawn from stream ``seed``."""
    nx, ny, nz = n
    hx, hy, hz = halo
    p = uniform01(seed, 12)
    k = np.arange(-hz, nz + hz, dtype=np.float64)[:, None, None]
    j = np.arange(-hy, ny + hy, dtype=np.float64)[None, :, None]
    i = np.arange(-hx, nx + hx, dtype=np.float64)[None, None, :]
    a = np.zeros(padded_shape(n, halo), dtype=np.float64)
    for s in range(3):
        ka = 1 + int(4 * p[4 * s + 0])
        kb = 1 + int(4 * p[4 * s + 1])
        kc = 1 + int(4 * p[4 * s + 2])
        phi = 2.0 * math.pi * p[4 * s + 3]
        a += (1.0 / 3.0) * np.sin(2.0 * math.pi * (ka * i / nx + kb * j / ny + kc * k / nz) + phi)
    a += 1e-3 * uniform(seed, a.size, -1.0, 1.0, start=12).reshape(a.shape)
    return a


def climate(seed: int = 303, n=(256, 256, 80), halo=(2, 2, 1), kappa0: float = 1.0 / 256.0):
    """The eight input fields of the multi-grid operator, keyed by name.

    Field g uses stream ``seed * 16 + g``.  q0..q2 are smooth fields; kappa =
    kappa0 (1 + s/2) and w = 0.05 s with s a smooth field in [-1, 1]; t0..t2 are
    smooth fields scaled by 1e-2.  Halo cells hold the same formulas."""
    out = {}
    for g, name in enumerate(CLIMATE_FIELDS):
        s = smooth_field(seed * 16 + g, n, halo)
        if name == "kappa":
            s = kappa0 * (1.0 + 0.5 * s)
        elif name == "w":
            s = 0.05 * s
        elif name.startswith("t"):
            s = 1e-2 * s
        out[name] = s
    return out


# ---------------------------------------------------------------- workload 4
def batch_sides(seed: int = 4040, count: int = 96, lo: int = 32, hi: int = 224):
    """Per-instance (nx, ny, nz), each side uniform on the integers lo..hi."""
    u = uniform01(seed, 3 * count).reshape(count, 3)
    return [tuple(int(lo + math.floor((hi - lo + 1) * v)) for v in row) for row in u]


def batch_instance(index: int, n, base_seed: int = 404) -> np.ndarray:
    """Instance ``index`` of the batched heat workload: interior uniform in [-1, 1),
    zero 1-cell halo, stream ``base_seed + index``."""
    return random_interior(base_seed + index, n, (1, 1, 1), -1.0, 1.0)


# ---------------------------------------------------------------- workload 5
def poisson_request(request_id: int, base_seed: int = 505, lo: int = 64, hi: int = 256):
    """Request ``request_id`` of the serving workload: a cubic side n uniform on
    lo..hi and an RHS f uniform in [-1, 1) with a zero 1-cell halo.  The first
    draw of stream ``base_seed + request_id`` picks n; the interior follows."""
    seed = base_seed + request_id
    n = int(lo + math.floor((hi - lo + 1) * uniform01(seed, 1)[0]))
    f = np.zeros(padded_shape((n, n, n), (1, 1, 1)), dtype=np.float64)
    interior_view(f, (n, n, n), (1, 1, 1))[...] = uniform(seed, n ** 3, -1.0, 1.0, start=1).reshape(n, n, n)
    return n, f


def poisson_arrivals(rate: float, window_s: float, seed: int = 5050):
    """Arrival times (seconds) of a Poisson process of the given rate over [0, window_s)."""
    times = []
    t = 0.0
    i = 0
    while True:
        u = uniform01(seed, 1, start=i)[0]
        i += 1
        t += -math.log1p(-u) / rate
        if t >= window_s:
            return times
        times.append(t)
