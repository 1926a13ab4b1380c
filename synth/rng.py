"""SplitMix64, counter-based, vectorised with numpy uint64 wrap-around arithmetic.

Value ``i`` of stream ``(seed, tag)`` is ``mix(key + (i + 1) * GAMMA)`` with
``key = mix(seed ^ (tag * TAG_MUL))``, where ``mix`` is the SplitMix64 output
function (Steele, Lea and Flood, OOPSLA 2014).  ``uniform`` maps a draw to
U[0,1) as ``(x >> 11) * 2**-53``.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)
TAG_MUL = np.uint64(0xD1B54A32D192ED03)

TAG_POLY = 1
TAG_WEIGHTS = 2
TAG_VECTOR = 3
TAG_MESH_JITTER = 4
TAG_STAR_RADII = 5
TAG_REQUESTS = 6


def mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        z = z ^ (z >> np.uint64(31))
    return z


def stream_key(seed: int, tag: int) -> np.uint64:
    with np.errstate(over="ignore"):
        k = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(tag) * TAG_MUL)
    return mix(np.array([k], dtype=np.uint64))[0]


def bits(seed: int, tag: int, n: int) -> np.ndarray:
    key = stream_key(seed, tag)
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix(key + i * GAMMA)


def uniform(seed: int, tag: int, n: int) -> np.ndarray:
    return (bits(seed, tag, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
