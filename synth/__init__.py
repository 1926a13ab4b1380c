"""Seeded synthetic inputs shared by the CUDA path's tests, the benchmark and the oracle.

This module draws random numbers and builds meshes; it holds none of the
method's arithmetic (no finite elements, no partitioning, no Schwarz or GNN
step).  Every random draw comes from one counter-based generator, SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014), mapped to U[0,1) as ``(x >> 11) * 2**-53``.

Workload shapes follow the paper's data recipe (Section IV-A): random 2D
domains meshed with unstructured triangles, forcing ``f`` and Dirichlet data
``g`` drawn as random quadratic polynomials with coefficients ``r_1..r_9`` in
U(-10, 10).  The paper's GMSH/Bezier meshes are replaced by two seeded
families: a jittered Delaunay grid on the unit square and a radially mapped
disk mesh on a random star-shaped 12-gon.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import rng
from .mesh import square_mesh, star_mesh, Mesh

__all__ = [
    "rng", "Mesh", "square_mesh", "star_mesh", "poly_coeffs", "dss_weights",
    "residual_vector", "n_weights_per_block", "workload", "request_stream",
]


def poly_coeffs(seed: int) -> np.ndarray:
    """r_1..r_9 ~ U(-10, 10) for the paper's f and g family (Section IV-A)."""
    return -10.0 + 20.0 * rng.uniform(seed, rng.TAG_POLY, 9)


def n_weights_per_block(d: int) -> int:
    """Length of one block's slice of the weight vector that ``dss_weights`` draws."""
    return 2 * ((2 * d + 3) * d + d + d * d + d) + ((3 * d + 1) * d + d + d * d + d) + (d * d + d + d + 1)


def dss_weights(kbar: int, d: int, seed: int, bias_scale: float = 0.0, gain: float = 1.0) -> np.ndarray:
    """Flat float32 weight vector, Xavier-uniform matrices and U(-bias_scale, bias_scale) biases.

    Layout per block (row-major W[out][in]): Phi_out W1[d][2d+3] b1[d] W2[d][d] b2[d];
    Phi_in (same); Psi W1[d][3d+1] b1[d] W2[d][d] b2[d]; D W1[d][d] b1[d] W2[1][d] b2[1].
    ``bias_scale = 0`` gives the paper's initialisation (Section IV-B: Xavier, biases 0).
    """
    shapes = []
    for _ in range(kbar):
        for _mlp in range(2):
            shapes += [("w", d, 2 * d + 3), ("b", d), ("w", d, d), ("b", d)]
        shapes += [("w", d, 3 * d + 1), ("b", d), ("w", d, d), ("b", d)]
        shapes += [("w", d, d), ("b", d), ("w", 1, d), ("b", 1)]
    total = sum(s[1] * s[2] if s[0] == "w" else s[1] for s in shapes)
    assert total == kbar * n_weights_per_block(d)
    u = rng.uniform(seed, rng.TAG_WEIGHTS, total)
    out = np.empty(total, dtype=np.float64)
    pos = 0
    for s in shapes:
        if s[0] == "w":
            fan_out, fan_in = s[1], s[2]
            a = gain * math.sqrt(6.0 / (fan_in + fan_out))
            cnt = fan_out * fan_in
            out[pos:pos + cnt] = -a + 2.0 * a * u[pos:pos + cnt]
        else:
            cnt = s[1]
            out[pos:pos + cnt] = -bias_scale + 2.0 * bias_scale * u[pos:pos + cnt]
        pos += cnt
    return out.astype(np.float32)


def residual_vector(n: int, seed: int) -> np.ndarray:
    """A residual-like FP64 vector, U(-1, 1) entries."""
    return -1.0 + 2.0 * rng.uniform(seed, rng.TAG_VECTOR, n)


@dataclass
class Workload:
    name: str
    mesh: Mesh
    coeffs: np.ndarray
    K: int
    overlap: int


def workload(name: str, seed: int = 0) -> Workload:
    """The named synthetic workloads.

    * ``square2k``: unit square, 45x45 jittered Delaunay grid (~2,000 nodes),
      K = 4 subdomains, 1-layer overlap.
    * ``star100k``: random star 12-gon, ~100k nodes, K = round(n_free/1000),
      2-layer overlap.
    * ``star1m``: the same family at ~1M nodes.
    * ``starN`` for any integer N (e.g. ``star20000``): the same family at ~N nodes.
    """
    coeffs = poly_coeffs(seed)
    if name == "square2k":
        m = square_mesh(45, seed=seed, jitter=0.3)
        return Workload(name, m, coeffs, 4, 1)
    if name == "star100k":
        target = 100_000
    elif name == "star1m":
        target = 1_000_000
    elif name.startswith("star"):
        target = int(name[4:])
    else:
        raise ValueError(name)
    m = star_mesh(target, seed=seed)
    n_free_est = m.n - m.n_boundary_ring
    K = max(1, int(round(n_free_est / 1000.0)))
    return Workload(name, m, coeffs, K, 2)


@dataclass
class Request:
    arrival_s: float      # seconds after the stream starts
    n_target: int         # requested mesh size (nodes)
    seed: int             # seed of its star domain, mesh jitter and f, g coefficients


def request_stream(n_requests: int, rate_per_s: float, n_min: int, n_max: int, seed: int) -> list[Request]:
    """A Poisson-process stream of independent solves with log-uniform mesh sizes.

    Inter-arrival gaps are exponential with mean ``1 / rate_per_s`` (inverse
    transform of U[0,1)); sizes are ``exp(U(log n_min, log n_max))``; request
    ``i`` gets the seed ``seed * 1_000_003 + 7919 * (i + 1)`` for its domain
    and data.
    """
    u = rng.uniform(seed, rng.TAG_REQUESTS, 2 * n_requests)
    t, out = 0.0, []
    for i in range(n_requests):
        t += -math.log1p(-u[2 * i]) / rate_per_s
        n = int(round(math.exp(math.log(n_min) + (math.log(n_max) - math.log(n_min)) * u[2 * i + 1])))
        out.append(Request(t, n, seed * 1_000_003 + 7919 * (i + 1)))
    return out
