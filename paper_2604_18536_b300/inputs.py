"""Seeded synthetic inputs shared by the CUDA path's callers and the oracle's tests.

This module holds no arithmetic of the method (no operator, no Poisson solve,
no time stepping). It only builds grids' face coordinates and raw initial
fields from seeds. Projection onto divergence-free fields and normalisation
are done afterwards by whichever implementation consumes the field.

Random numbers come from one counter-based generator: SplitMix64
(G. L. Steele, D. Lea, C. H. Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), output n of the stream with key k being
mix(k + (n + 1) * 0x9E3779B97F4A7C15), followed by the Box-Muller transform
for normal deviates. Every value is addressed by (seed, component, wavevector)
so any subset can be regenerated independently.
"""

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(key, counter):
    """Output ``counter`` (uint64 array) of the SplitMix64 stream with the given key."""
    with np.errstate(over="ignore"):
        z = np.uint64(key) + (np.asarray(counter, dtype=np.uint64) + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(key, counter):
    """Uniform deviates in (0, 1]: the top 53 bits of SplitMix64, plus one ulp."""
    bits = splitmix64(key, counter) >> np.uint64(11)
    return (bits.astype(np.float64) + 1.0) * (2.0 ** -53)


def normal_pair(key, counter):
    """Two independent standard normal deviates per counter (Box-Muller)."""
    c = np.asarray(counter, dtype=np.uint64)
    u1 = uniform01(key, c * np.uint64(2))
    u2 = uniform01(key, c * np.uint64(2) + np.uint64(1))
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)


# ------------------------------------------------------------------ grids
def uniform_faces(n, a, b):
    """n + 1 equally spaced face coordinates on [a, b]."""
    return a + (b - a) * np.arange(n + 1, dtype=np.float64) / n


def tanh_faces(n, a, b, gamma):
    """tanh-stretched faces clustered at both ends (the paper's tanh-grid formula)."""
    s = np.arange(n + 1, dtype=np.float64) / n
    return a + 0.5 * (b - a) * (1.0 + np.tanh(gamma * (2.0 * s - 1.0)) / np.tanh(gamma))


def centres(faces):
    f = np.asarray(faces, dtype=np.float64)
    return 0.5 * (f[:-1] + f[1:])


def periodic_box(n, dim, length=2.0 * np.pi):
    """Faces of a periodic uniform box [0, length]^dim with n cells per direction."""
    return [uniform_faces(n, 0.0, length) for _ in range(dim)]


def channel_faces(nx, ny, nz, lx=4.0 * np.pi, ly=2.0, lz=4.0 * np.pi / 3.0, gamma=1.5):
    """Channel box: uniform in x and z, tanh-stretched wall-normal y on [0, ly]."""
    return [uniform_faces(nx, 0.0, lx), tanh_faces(ny, 0.0, ly, gamma), uniform_faces(nz, 0.0, lz)]


def _mesh(faces, a):
    """Coordinates of the u^a positions as broadcastable arrays, x the last axis."""
    dim = len(faces)
    out = []
    for b in range(dim):
        v = np.asarray(faces[b], dtype=np.float64)[1:] if b == a else centres(faces[b])
        shp = [1] * dim
        shp[dim - 1 - b] = -1
        out.append(v.reshape(shp))
    return out


# ---------------------------------------------------------------- fields
def taylor_green_2d(faces, t=0.0, nu=0.0):
    """2-D Taylor-Green vortex u = sin x cos y, v = -cos x sin y, times exp(-2 nu t)."""
    ny, nx = len(faces[1]) - 1, len(faces[0]) - 1
    u = np.zeros((2, ny, nx))
    x, y = _mesh(faces, 0)
    u[0] = np.sin(x) * np.cos(y)
    x, y = _mesh(faces, 1)
    u[1] = -np.cos(x) * np.sin(y)
    return u * np.exp(-2.0 * nu * t)


def random_field(shape, seed, scale=1.0):
    """Plain seeded uniform(-scale, scale) field of any shape (test input)."""
    rng = np.random.default_rng(seed)
    return scale * (2.0 * rng.random(shape) - 1.0)


def spectrum_velocity_raw(n, dim, seed, k0=4.0, kmax=None):
    """Random Fourier velocity with energy spectrum E(k) ~ k^4 exp(-2 (k/k0)^2).

    For every integer wavevector with 0 < |k| <= kc (kc = N/2 - 1 with N the smallest
    resolution, or the given kmax if smaller) and every component a the coefficient is
    sqrt(E(|k|) / S(|k|)) (g1 + i g2) / sqrt(2), with S the shell area (4 pi k^2 in 3-D,
    2 pi k in 2-D) and (g1, g2) the Box-Muller pair of counter
    ((a * Nz + iz) * Ny + iy) * Nx + ix under key ``seed``. Only wavevectors inside the
    cutoff draw numbers (the counter makes every value independent of the others, so this
    changes nothing). The field is the real part of the inverse DFT, read as face values.
    It is NOT yet divergence free and NOT normalised: project it, then scale to unit energy.
    """
    import scipy.fft
    if isinstance(n, int):
        n = (n,) * dim
    n = tuple(n)
    shape = tuple(reversed(n))
    kax = [np.fft.fftfreq(nn, d=1.0 / nn) for nn in n]          # integer wavenumbers
    k2 = np.zeros(shape)
    for a in range(dim):
        shp = [1] * dim
        shp[dim - 1 - a] = -1
        k2 = k2 + (kax[a] ** 2).reshape(shp)
    kcut = min(n) // 2 - 1
    if kmax is not None:
        kcut = min(kcut, kmax)
    idx = np.nonzero((k2 > 0) & (k2 <= kcut * kcut))     # |k| <= kc exactly (integer k)
    km = np.sqrt(k2[idx])
    E = km ** 4 * np.exp(-2.0 * (km / k0) ** 2)
    shell = 4.0 * np.pi * km ** 2 if dim == 3 else 2.0 * np.pi * km
    amp = np.sqrt(E / shell)
    size = int(np.prod(shape))
    lin = np.ravel_multi_index(idx, shape).astype(np.uint64)
    u = np.zeros((dim,) + shape)
    for a in range(dim):
        g1, g2 = normal_pair(seed, np.uint64(a) * np.uint64(size) + lin)
        coef = np.zeros(shape, dtype=np.complex128)
        coef[idx] = amp * (g1 + 1j * g2) / np.sqrt(2.0)
        u[a] = np.real(scipy.fft.ifftn(coef, workers=-1)) * float(size)
    return u


def channel_velocity_raw(faces, seed, u_bulk=15.6, amplitude=0.1):
    """Laminar parabola plus a seeded perturbation for the channel (y in [0, 2]).

    u^x = 1.5 u_bulk y(2-y) + amplitude u_bulk y(2-y) g, u^y, u^z = amplitude u_bulk y(2-y) g
    with g standard normal deviates (counter = component * cells + linear index).
    The envelope vanishes on the walls, so the stored top-wall u^y is 0.
    NOT divergence free: project it with the wall Poisson solver.
    """
    dim = len(faces)
    n = tuple(len(f) - 1 for f in faces)
    shape = tuple(reversed(n))
    u = np.zeros((dim,) + shape)
    size = int(np.prod(shape))
    lin = np.arange(size, dtype=np.uint64).reshape(shape)
    for a in range(dim):
        pos = _mesh(faces, a)
        y = pos[1] - faces[1][0]
        env = y * (2.0 - y) * np.ones(shape)
        g1, _ = normal_pair(seed, np.uint64(a) * np.uint64(size) + lin)
        u[a] = amplitude * u_bulk * env * g1
        if a == 0:
            u[a] += 1.5 * u_bulk * env
    # exact zero on the stored top wall face of u^y
    idx = [slice(None)] * dim
    idx[dim - 2] = -1
    u[1][tuple(idx)] = 0.0
    return u
