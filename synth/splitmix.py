"""SplitMix64 as a counter-based generator, vectorised with numpy.

SplitMix64 is the generator of Steele, Lea and Flood ("Fast splittable
pseudorandom number generators", OOPSLA 2014) in the form popularised by
Vigna: the state advances by the odd constant gamma = 0x9E3779B97F4A7C15 and
each output is the state passed through a 64-bit finaliser (xor-shift 30,
multiply, xor-shift 27, multiply, xor-shift 31). Output number ``n`` (0-based)
of the stream started at ``seed`` is therefore mix(seed + (n + 1) * gamma),
which lets every cell draw its value from its own global linear index, so the
initial grid does not depend on how the grid is later split into blocks.

A uniform double in [0, 1) is the top 53 bits of the output times 2**-53.
"""

from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 24


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of the SplitMix64 stream at ``seed``."""
    with np.errstate(over="ignore"):
        n = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + n * GAMMA
        return _mix(z)


def uniform01(seed: int, start: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1): (output >> 11) * 2**-53, one per index."""
    z = splitmix64(seed, start, count)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def grid_uniform01(seed: int, nx: int, ny: int, nz: int, out: np.ndarray | None = None) -> np.ndarray:
    """Interior of an (nz, ny, nx) grid, x fastest, cell n = i + nx*(j + ny*k)
    drawing output n of the stream. Generated in chunks to bound host memory."""
    total = nx * ny * nz
    if out is None:
        out = np.empty(total, dtype=np.float64)
    flat = out.reshape(-1)
    for s in range(0, total, _CHUNK):
        c = min(_CHUNK, total - s)
        flat[s:s + c] = uniform01(seed, s, c)
    return out.reshape(nz, ny, nx)


def grid_uniform01_f32(seed: int, nx: int, ny: int, nz: int, out: np.ndarray | None = None) -> np.ndarray:
    """The same grid rounded to binary32 (round to nearest even)."""
    total = nx * ny * nz
    if out is None:
        out = np.empty(total, dtype=np.float32)
    flat = out.reshape(-1)
    for s in range(0, total, _CHUNK):
        c = min(_CHUNK, total - s)
        flat[s:s + c] = uniform01(seed, s, c).astype(np.float32)
    return out.reshape(nz, ny, nx)
