"""Seeded synthetic inputs shared by the CUDA path, the tests and the bench.

This module draws random numbers only; it holds none of the search
method's arithmetic.  It produces

* the sparse binary projection of FlyHash (Def. 7): for every output j, F
  distinct input dimensions, listed in ascending order (the random matrix
  W is an input of the hash, so it is drawn here and passed to both the
  CUDA path and the oracle);
* vector-set databases and query sets shaped like the paper's workloads
  (millions of small sets of unit-norm embeddings; the CS dataset has
  d = 384 and sets of a few to a few hundred vectors), drawn from a
  Gaussian mixture and rounded to multiples of 2^-8.

Mixture recipe (a reading: the workloads name only "a K-component
Gaussian mixture"):

* the K components are split into groups of ``group`` components; a group
  has a mean g ~ N(0, I_d), normalised, and component c of that group has
  mean mu_c = normalise(g + tau * e_c / sqrt(d)) with e_c ~ N(0, I_d);
* a set picks one group, then 1, 2 or 3 distinct components of it
  (uniformly), then each of its vectors picks one of those components
  uniformly and is normalise(mu_c + sigma * e / sqrt(d)), e ~ N(0, I_d);
* set sizes are uniform in [size_lo, size_hi];
* values are rounded to the nearest multiple of 2^-8 after normalising
  ("grid" values), so FP32 sums of a few of them are exact.

Queries are drawn the same way from another seed, over the same
components.
"""
from __future__ import annotations

import math

import numpy as np
import torch

GRID = 256.0


def projection(d: int, m: int, fanin: int, seed: int) -> np.ndarray:
    """(m, fanin) uint16: row j = ``fanin`` distinct dims of [0, d), ascending."""
    if not (1 <= fanin <= d):
        raise ValueError("need 1 <= fanin <= d")
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((m, fanin), np.uint16)
    chunk = 4096
    for j0 in range(0, m, chunk):
        j1 = min(m, j0 + chunk)
        keys = rng.random((j1 - j0, d))
        pick = np.argpartition(keys, fanin - 1, axis=1)[:, :fanin]
        out[j0:j1] = np.sort(pick, axis=1).astype(np.uint16)
    return out


def set_sizes(n_sets: int, lo: int, hi: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(lo, hi + 1, size=n_sets, dtype=np.int64)


def zipf_sizes(n_sets: int, lo: int, hi: int, seed: int, s: float = 1.0) -> np.ndarray:
    """Set sizes with P(size = k) proportional to k^-s on [lo, hi] (a truncated Zipf
    law; s = 1 is the classic one)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = np.arange(lo, hi + 1, dtype=np.float64)
    p = k ** -s
    return rng.choice(np.arange(lo, hi + 1, dtype=np.int64), size=n_sets, p=p / p.sum())


def offsets_from_sizes(sizes: np.ndarray) -> np.ndarray:
    off = np.zeros(sizes.shape[0] + 1, np.int64)
    np.cumsum(sizes, out=off[1:])
    return off


class Mixture:
    """Component means of the grouped Gaussian mixture (seeded)."""

    def __init__(self, d: int, n_components: int, seed: int, group: int = 16,
                 tau: float = 0.5, device="cpu"):
        self.d = d
        self.K = n_components
        self.group = max(1, min(group, n_components))
        self.n_groups = max(1, n_components // self.group)
        self.device = torch.device(device)
        g = torch.Generator(device="cpu").manual_seed(int(seed) * 7919 + 1)
        gm = torch.randn(self.n_groups, d, generator=g, dtype=torch.float64)
        gm = gm / gm.norm(dim=1, keepdim=True)
        e = torch.randn(self.n_groups * self.group, d, generator=g, dtype=torch.float64)
        mu = gm.repeat_interleave(self.group, dim=0) + tau * e / math.sqrt(d)
        self.mu = (mu / mu.norm(dim=1, keepdim=True)).to(torch.float32).to(self.device)

    def draw_sets(self, sizes: np.ndarray, seed: int, sigma: float = 0.5,
                  grid: bool = True, chunk_vectors: int = 1 << 21) -> torch.Tensor:
        """Vectors (sum(sizes), d) float32 on the mixture's device, set-contiguous."""
        n_sets = int(sizes.shape[0])
        dev = self.device
        gen = torch.Generator(device=dev).manual_seed(int(seed))
        sz = torch.as_tensor(sizes, dtype=torch.int64, device=dev)
        grp = torch.randint(0, self.n_groups, (n_sets,), generator=gen, device=dev)
        n_topics = torch.randint(1, min(3, self.group) + 1, (n_sets,), generator=gen,
                                 device=dev)
        keys = torch.rand(n_sets, self.group, generator=gen, device=dev)
        topics = keys.argsort(dim=1)[:, :3]                         # distinct picks
        total = int(sizes.sum())
        out = torch.empty(total, self.d, dtype=torch.float32, device=dev)
        set_of_vec = torch.repeat_interleave(torch.arange(n_sets, device=dev), sz)
        for v0 in range(0, total, chunk_vectors):
            v1 = min(total, v0 + chunk_vectors)
            s = set_of_vec[v0:v1]
            u = (torch.rand(v1 - v0, generator=gen, device=dev)
                 * n_topics[s].to(torch.float32)).to(torch.int64)
            u = torch.minimum(u, n_topics[s] - 1)
            comp = grp[s] * self.group + topics[s, u]
            e = torch.randn(v1 - v0, self.d, generator=gen, device=dev)
            x = self.mu[comp] + (sigma / math.sqrt(self.d)) * e
            x = x / x.norm(dim=1, keepdim=True)
            if grid:
                x = torch.round(x * GRID) / GRID
            out[v0:v1] = x
        return out


def workload(n_sets: int, size_lo: int, size_hi: int, d: int, n_components: int,
             n_queries: int, q_lo: int, q_hi: int, m: int, fanin: int,
             seed: int = 0, device="cpu", sigma: float = 0.5, tau: float = 0.5,
             group: int = 16, grid: bool = True, size_dist: str = "uniform",
             q_dist: str = "uniform"):
    """A database, its query sets and the FlyHash projection, all seeded.

    seed -> database, seed + 1 -> queries, seed + 2 -> projection.  Database set
    sizes are uniform or (size_dist="zipf") truncated Zipf with exponent 1 on
    [size_lo, size_hi]; query set sizes are uniform on [q_lo, q_hi] or (q_dist="zipf")
    truncated Zipf on it.
    Returns a dict of vectors / offsets (torch on ``device``; offsets also
    as numpy) and the projection (numpy uint16).
    """
    mix = Mixture(d, n_components, seed, group=group, tau=tau, device=device)
    if size_dist == "zipf":
        sizes = zipf_sizes(n_sets, size_lo, size_hi, seed * 1000 + 11)
    elif size_dist == "uniform":
        sizes = set_sizes(n_sets, size_lo, size_hi, seed * 1000 + 11)
    else:
        raise ValueError("size_dist must be 'uniform' or 'zipf'")
    if q_dist == "zipf":
        qsizes = zipf_sizes(n_queries, q_lo, q_hi, seed * 1000 + 12)
    elif q_dist == "uniform":
        qsizes = set_sizes(n_queries, q_lo, q_hi, seed * 1000 + 12)
    else:
        raise ValueError("q_dist must be 'uniform' or 'zipf'")
    vec = mix.draw_sets(sizes, seed * 1000 + 21, sigma=sigma, grid=grid)
    qvec = mix.draw_sets(qsizes, seed * 1000 + 22, sigma=sigma, grid=grid)
    proj = projection(d, m, fanin, seed + 2)
    return dict(vectors=vec, offsets=offsets_from_sizes(sizes), q_vectors=qvec,
                q_offsets=offsets_from_sizes(qsizes), proj=proj)


# The two sizes the tests and the bench use.
SMALL = dict(n_sets=2000, size_lo=4, size_hi=16, d=128, n_components=64,
             n_queries=100, q_lo=4, q_hi=16, m=2048, fanin=8, L=32, C=200, k=10)
LARGE = dict(n_sets=1_000_000, size_lo=8, size_hi=32, d=384, n_components=4096,
             n_queries=1000, q_lo=8, q_hi=32, m=4096, fanin=8, L=64, C=2000, k=10)
# The batched serving load: Zipf set sizes, d = 768 (values exact in BF16), 4096 query
# sets of 1-64 vectors per pass.  The load names neither the mixture, m, F, L, C nor k;
# they are taken from LARGE.
SERVING = dict(n_sets=200_000, size_lo=1, size_hi=128, d=768, n_components=4096,
               n_queries=4096, q_lo=1, q_hi=64, m=4096, fanin=8, L=64, C=2000, k=10,
               size_dist="zipf")
# The FP8 refine's load at high dimension: 500k sets of Zipf sizes 4-64, d = 1024, a
# 16,384-component mixture, 2000 query sets, C = 4000.  The load names neither m, F, L,
# A, M nor the query sets' sizes: m, F, L come from LARGE and the query sets follow the
# database's size law.
FP8_HIGH_D = dict(n_sets=500_000, size_lo=4, size_hi=64, d=1024, n_components=16384,
                  n_queries=2000, q_lo=4, q_hi=64, m=4096, fanin=8, L=64, C=4000, k=10,
                  size_dist="zipf", q_dist="zipf")
