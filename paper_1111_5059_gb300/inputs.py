"""Seeded synthetic inputs shared, as data, by the CPU oracle and the CUDA path.

This module holds no arithmetic of the domain-wall method: it only draws
random numbers and shapes them into the fields the method consumes.

Random numbers: SplitMix64 used as a counter-based generator (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the
i-th 64-bit output of a stream with key ``k`` is ``mix(k + (i+1)*GOLDEN)``
with the published finaliser ``mix``.  Uniforms take the top 53 bits;
normals come from the Box-Muller transform of consecutive uniform pairs.
Being counter based, any slice of a stream can be regenerated on its own,
which is what the large-size parity tests use.

Field shapes (the library's boundary layout):
  gauge links  complex128 [4][T][Z][Y][X][3][3]   (mu = x, y, z, t)
  5D spinor    complex128 [Ls][T][Z][Y][X][4][3]
  momenta      float64    [4][T][Z][Y][X][8]      (components on T_j)

Gauge links are the near-identity SU(3) matrices exp(i eps sum_k a_k lambda_k)
with a_k ~ N(0,1) (Gell-Mann lambda_k), computed by a scaled Taylor series and
re-unitarised to SU(3).  Spinors have Re, Im ~ N(0,1) independently.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22

# Stream identifiers: each field drawn for one seed uses its own stream.
STREAM_GAUGE = 1
STREAM_SOURCE = 2
STREAM_MOMENTA = 3
STREAM_GAUGE_TRANSFORM = 4
STREAM_NOISE = 5


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> int:
    """64-bit key of stream ``stream`` under ``seed`` (one SplitMix64 output)."""
    z = np.array([(int(seed) * 0x100000001B3 + int(stream)) & (2**64 - 1)], dtype=np.uint64)
    with np.errstate(over="ignore"):
        return int(_mix(z + GOLDEN)[0])


def splitmix64(key: int, start: int, count: int) -> np.ndarray:
    """Outputs start..start+count-1 of the counter-based SplitMix64 stream ``key``."""
    i = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(np.uint64(key) + i * GOLDEN)


def uniform(key: int, start: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each output."""
    return (splitmix64(key, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _normal_chunk(key: int, start_pair: int, npairs: int) -> np.ndarray:
    u = uniform(key, 2 * start_pair, 2 * npairs).reshape(npairs, 2)
    r = np.sqrt(-2.0 * np.log1p(-u[:, 0]))
    th = 2.0 * np.pi * u[:, 1]
    out = np.empty((npairs, 2))
    out[:, 0] = r * np.cos(th)
    out[:, 1] = r * np.sin(th)
    return out.reshape(-1)


def normal(key: int, count: int, start: int = 0) -> np.ndarray:
    """``count`` standard normals of stream ``key`` starting at normal ``start``.

    Normal 2k and 2k+1 come from uniform pair k (Box-Muller), so ``start``
    must be even.  Large draws are split into chunks over threads.
    """
    if start % 2:
        raise ValueError("normal(): start must be even")
    npairs = (count + 1) // 2
    p0 = start // 2
    out = np.empty(2 * npairs)
    nchunk = (npairs + _CHUNK - 1) // _CHUNK
    if nchunk <= 1:
        out[:] = _normal_chunk(key, p0, npairs)
    else:
        def work(c):
            a = c * _CHUNK
            b = min(npairs, a + _CHUNK)
            out[2 * a:2 * b] = _normal_chunk(key, p0 + a, b - a)
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            list(ex.map(work, range(nchunk)))
    return out[:count]


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3)."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1] = -1j
    l[1][1, 0] = 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2] = -1j
    l[4][2, 0] = 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2] = -1j
    l[6][2, 1] = 1j
    l[7][0, 0] = l[7][1, 1] = 1 / np.sqrt(3)
    l[7][2, 2] = -2 / np.sqrt(3)
    return l


def _mul3(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Product of two stacks of 3x3 matrices held as [3][3][N] arrays."""
    C = np.empty_like(A)
    for i in range(3):
        for j in range(3):
            C[i, j] = A[i, 0] * B[0, j] + A[i, 1] * B[1, j] + A[i, 2] * B[2, j]
    return C


def _expm_taylor(X: np.ndarray, squarings: int = 6, order: int = 10) -> np.ndarray:
    """exp of a stack of 3x3 matrices: Taylor series of X/2^s, squared s times."""
    Y = np.ascontiguousarray(np.moveaxis(X, 0, -1)) / (2.0 ** squarings)
    E = np.zeros_like(Y)
    for i in range(3):
        E[i, i] = 1.0
    term = E.copy()
    for k in range(1, order + 1):
        term = _mul3(term, Y) / k
        E += term
    for _ in range(squarings):
        E = _mul3(E, E)
    return np.moveaxis(E, -1, 0)


def reunitarize(U: np.ndarray) -> np.ndarray:
    """Gram-Schmidt on rows 0 and 1; row 2 = conj(row0 x row1), so det = 1."""
    r0 = U[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = U[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def su3_near_identity(key: int, count: int, eps: float) -> np.ndarray:
    """``count`` SU(3) matrices exp(i eps sum_k a_k lambda_k), a_k ~ N(0,1)."""
    lam = gell_mann()
    out = np.empty((count, 3, 3), dtype=np.complex128)
    step = 1 << 17

    def work(a):
        b = min(count, a + step)
        coef = normal(key, 8 * (b - a), start=8 * a).reshape(b - a, 8)
        H = np.einsum("nk,kab->nab", coef, lam)
        out[a:b] = reunitarize(_expm_taylor(1j * eps * H))

    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(work, range(0, count, step)))
    return out


def gauge_field(seed: int, dims, eps: float) -> np.ndarray:
    """Near-identity SU(3) links, complex128 [4][T][Z][Y][X][3][3]."""
    X, Y, Z, T = dims
    n = 4 * T * Z * Y * X
    U = su3_near_identity(stream_key(seed, STREAM_GAUGE), n, eps)
    return U.reshape(4, T, Z, Y, X, 3, 3)


def gauge_transform(seed: int, dims, eps: float = 1.0) -> np.ndarray:
    """Random SU(3) gauge transformation G(n), complex128 [T][Z][Y][X][3][3]."""
    X, Y, Z, T = dims
    G = su3_near_identity(stream_key(seed, STREAM_GAUGE_TRANSFORM), T * Z * Y * X, eps)
    return G.reshape(T, Z, Y, X, 3, 3)


def gaussian_spinor(seed: int, dims, Ls: int, stream: int = STREAM_SOURCE) -> np.ndarray:
    """Gaussian 5D spinor with Re, Im ~ N(0,1): complex128 [Ls][T][Z][Y][X][4][3]."""
    X, Y, Z, T = dims
    n = Ls * T * Z * Y * X * 12
    v = normal(stream_key(seed, stream), 2 * n)
    return v.view(np.complex128).reshape(Ls, T, Z, Y, X, 4, 3)


def gaussian_momenta(seed: int, dims) -> np.ndarray:
    """su(3) momenta components p^j ~ N(0,1): float64 [4][T][Z][Y][X][8]."""
    X, Y, Z, T = dims
    n = 4 * T * Z * Y * X * 8
    return normal(stream_key(seed, STREAM_MOMENTA), n).reshape(4, T, Z, Y, X, 8)
