"""Seeded synthetic workloads shaped like the paper's evaluation data (Sec. 5.1, Table 2).

The paper evaluates on public vector collections (SIFT, DEEP, GIST, BIGANN, ...).  None of
them is available here, so every workload below is a seeded synthetic stand-in with the
same size, dimensionality, value range and cluster structure.  No record of any of those
collections is reproduced.

This module holds only random-number recipes.  It contains none of the method's
arithmetic, so both the CUDA path and the CPU oracle may read its output.

Recipes (numpy ``Generator(PCG64(seed))``, rows generated in fixed chunks so the output
does not depend on memory limits).  Descriptor collections such as SIFT, DEEP and BIGANN lie
near a low-dimensional structure, so their mixtures live in one shared 16-dimensional
subspace: x = c0 + A (u_a + z) + e, with a shared loading matrix A (d x 16), cluster offsets
u_a ~ N(0, I_16) (the mixture's centres are c0 + A u_a), z ~ N(0, I_16) and a small isotropic
term e.  (Clusters given private subspaces, or centres spread wider than the clusters, turn
into islands that graphs built from exact neighbour lists cannot navigate between.)

* ``gauss``      i.i.d. N(0, 1) float32.
* ``sift``       64 centres; c0 uniform on the integers 112..143 per dimension; A entries
                 N(0, 25^2 / 16) (per-coordinate std about 25 per unit of u + z); e ~ N(0, 2^2);
                 clipped to [0, 255] and rounded to integers (float32).
* ``deep``       256 centres; c0 a random unit vector; A entries N(0, 0.25 / (16 d));
                 e ~ N(0, 0.05^2 / d); x normalised to unit length.
* ``sift_iso``   the isotropic alternative: 64 centres with coordinates uniform on the
                 integers 40..215, x = centre + N(0, 25^2 I) in all d dimensions, clipped to
                 [0, 255] and rounded (each cluster intrinsically d-dimensional).
* ``gist``       100 centres N(0, 0.1^2 I); per (centre, dimension) standard deviation
                 sqrt(v), v log-uniform on [0.01, 1] (diagonal covariance).
* ``bigann16``   1,024 centres; c0 = 0; A entries N(0, 0.25 / 16); e ~ N(0, 0.05^2); stored
                 as float16.
"""
from __future__ import annotations

import dataclasses
import numpy as np

_CHUNK = 1 << 16  # rows drawn per chunk; fixed so results are independent of memory


@dataclasses.dataclass(frozen=True)
class Workload:
    """One seeded workload: base points, query points and training queries."""

    name: str
    kind: str
    n: int
    d: int
    nq: int
    k: int
    alpha: float
    R: int
    L: int
    n_train: int
    seed: int
    dtype: str = "float32"
    repair_slots: int = 8  # phase-4 slots per row
    connect_L: int = 0  # phase-4 search beam (0: the library default, 32)

    def base(self, n: int | None = None) -> np.ndarray:
        return generate(self.kind, self.n if n is None else n, self.d, self.seed, self.dtype)

    def queries(self, nq: int | None = None) -> np.ndarray:
        return generate(self.kind, self.nq if nq is None else nq, self.d, 1000 + self.seed, self.dtype,
                        centre_seed=self.seed)

    def train_queries(self, nt: int | None = None) -> np.ndarray:
        return generate(self.kind, self.n_train if nt is None else nt, self.d, 2000 + self.seed,
                        self.dtype, centre_seed=self.seed)


# The five workloads: sizes and parameters of the hot-path scope table.
WORKLOADS = {
    "gauss10k": Workload("gauss10k", "gauss", 10_000, 32, 100, 10, 1.2, 32, 64, 2_000, 0),
    "sift1m": Workload("sift1m", "sift", 1_000_000, 128, 10_000, 10, 1.2, 32, 128, 20_000, 1),
    "deep1m": Workload("deep1m", "deep", 1_000_000, 96, 10_000, 10, 1.3, 48, 160, 20_000, 2),
    # at d = 960 many points get no in-edge from exact candidate lists; phase 4 needs room
    # and a wider search (a beam of 32 stalls with tens of thousands of points unreached)
    "gist1m": Workload("gist1m", "gist", 1_000_000, 960, 1_000, 10, 1.2, 32, 128, 2_000, 3,
                       repair_slots=32, connect_L=128),
    "bigann10m": Workload("bigann10m", "bigann16", 10_000_000, 128, 100_000, 10, 1.2, 32, 128,
                          200_000, 4, "float16"),
    # the SIFT-like shape with isotropic clusters (reported beside the low-rank recipe)
    "sift1m_iso": Workload("sift1m_iso", "sift_iso", 1_000_000, 128, 10_000, 10, 1.2, 32, 128,
                           20_000, 5),
}


LATENT = 16


def _centres(kind: str, d: int, seed: int):
    """(c0, A, U): base point, shared loading matrix and cluster offsets (own stream).  For
    ``gist``: (centres, per-centre scales, None)."""
    rng = np.random.Generator(np.random.PCG64(seed * 7919 + 17))
    m = LATENT
    if kind == "sift":
        c0 = rng.integers(112, 144, size=d).astype(np.float32)
        A = (rng.standard_normal((d, m)) * (25.0 / np.sqrt(m))).astype(np.float32)
        return c0, A, rng.standard_normal((64, m)).astype(np.float32)
    if kind == "deep":
        g = rng.standard_normal(d)
        c0 = (g / np.linalg.norm(g)).astype(np.float32)
        A = (rng.standard_normal((d, m)) * (0.5 / np.sqrt(m * d))).astype(np.float32)
        return c0, A, rng.standard_normal((256, m)).astype(np.float32)
    if kind == "sift_iso":
        return rng.integers(40, 216, size=(64, d)).astype(np.float32), None, None
    if kind == "gist":
        c = (0.1 * rng.standard_normal((100, d))).astype(np.float32)
        v = np.exp(rng.uniform(np.log(0.01), np.log(1.0), size=(100, d))).astype(np.float32)
        return c, np.sqrt(v).astype(np.float32), None
    if kind == "bigann16":
        A = (rng.standard_normal((d, m)) * (0.5 / np.sqrt(m))).astype(np.float32)
        return np.zeros(d, np.float32), A, rng.standard_normal((1024, m)).astype(np.float32)
    return None, None, None


def generate(kind: str, n: int, d: int, seed: int, dtype: str = "float32",
             centre_seed: int | None = None) -> np.ndarray:
    """Return ``n`` rows of workload ``kind`` in dimension ``d`` (C-contiguous)."""
    if n < 0 or d <= 0:
        raise ValueError("n must be >= 0 and d > 0")
    c0, A, U = _centres(kind, d, seed if centre_seed is None else centre_seed)
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((n, d), dtype=np.float16 if dtype == "float16" else np.float32)
    for r0 in range(0, n, _CHUNK):
        m = min(_CHUNK, n - r0)
        if kind == "gauss":
            blk = rng.standard_normal((m, d), dtype=np.float32)
        elif kind in ("sift", "deep", "bigann16"):
            a = rng.integers(0, U.shape[0], size=m)
            z = rng.standard_normal((m, U.shape[1]), dtype=np.float32)
            blk = c0 + (U[a] + z) @ A.T
            eps = {"sift": 2.0, "deep": 0.05 / np.sqrt(d), "bigann16": 0.05}[kind]
            blk += eps * rng.standard_normal((m, d), dtype=np.float32)
            if kind == "sift":
                blk = np.rint(np.clip(blk, 0.0, 255.0))
            elif kind == "deep":
                blk = blk / np.linalg.norm(blk, axis=1, keepdims=True)
        elif kind == "sift_iso":
            a = rng.integers(0, c0.shape[0], size=m)
            blk = c0[a] + 25.0 * rng.standard_normal((m, d), dtype=np.float32)
            blk = np.rint(np.clip(blk, 0.0, 255.0))
        elif kind == "gist":
            a = rng.integers(0, c0.shape[0], size=m)
            blk = c0[a] + A[a] * rng.standard_normal((m, d), dtype=np.float32)
        else:
            raise ValueError(f"unknown workload kind {kind!r}")
        out[r0:r0 + m] = blk
    return out


def small(kind: str, n: int, d: int, seed: int = 0) -> np.ndarray:
    """Convenience: ``n`` base rows of ``kind`` for parity tests at reduced size."""
    return generate(kind, n, d, seed)
