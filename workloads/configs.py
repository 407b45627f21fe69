"""The five growth workloads, built from seeds.

1. S_8 with the 7 adjacent transpositions (Coxeter), full growth (40,320 states, diameter 28).
2. S_11 with LRX (L, R = L^-1, X), full growth (39,916,800 states).
3. S_14 pancake (13 prefix reversals), growth truncated at the first radius whose layer
   exceeds 2^31 states (that layer is computed and reported).
4. Batched: 4096 independent random groups, n ~ U{6..10}, k ~ U{2..5}; even-indexed groups
   get inverses appended (undirected), odd-indexed stay directed.
5. Serving: a Poisson stream of 20,000 growth jobs, n ~ U{8..16}, family ~ U{Coxeter, all
   transpositions, LRX, pancake, 2-5 random permutations with inverses}, radius cap
   ~ U{6..D_family}.

Draw order of the seeded generators is part of the input definition and must not change:
config 4 draws, per group in index order, n, then k, then k permutations (identity rejected);
config 5 draws, per job in index order, the inter-arrival gap, n, the family, the random
generators when the family is random (count, then permutations), then the radius cap.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import families as fam

BATCH_SEED = 20250919
SERVE_SEED = 20250920
TRUNCATE_ABOVE_2_31 = 1 << 31


@dataclass
class GrowthJob:
    """One growth problem: generators in one-line notation plus run limits."""
    n: int
    gens: List[List[int]]
    inverse_closed: bool
    max_radius: int = -1          # < 0: unlimited
    stop_above: int = 0           # > 0: stop after the first layer larger than this
    name: str = ""
    family: str = ""
    arrival: float = 0.0          # serving only: arrival time in units of 1/rate
    extra: dict = field(default_factory=dict)
    start: Optional[List[int]] = None   # central state of a Schreier coset graph (None: identity)

    @property
    def k(self) -> int:
        return len(self.gens)


def config_s8_coxeter() -> GrowthJob:
    return GrowthJob(8, fam.coxeter(8), True, name="S8-coxeter-k7-full", family="coxeter")


def config_s11_lrx() -> GrowthJob:
    return GrowthJob(11, fam.lrx(11), True, name="S11-LRX-k3-full", family="lrx")


def config_s14_pancake() -> GrowthJob:
    return GrowthJob(14, fam.pancake(14), True, stop_above=TRUNCATE_ABOVE_2_31,
                     name="S14-pancake-k13-trunc2^31", family="pancake")


def batch_groups(seed: int = BATCH_SEED, count: int = 4096) -> List[GrowthJob]:
    """Config 4: independent random groups; even index undirected, odd index directed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    jobs: List[GrowthJob] = []
    for g in range(count):
        n = int(rng.integers(6, 11))
        k = int(rng.integers(2, 6))
        gens = fam.random_perms(rng, n, k)
        undirected = (g % 2 == 0)
        if undirected:
            gens = fam.inverse_closure(gens)
        jobs.append(GrowthJob(n, gens, fam.is_inverse_closed(gens), name=f"batch{g}",
                              family="random+inv" if undirected else "random"))
    return jobs


SERVE_FAMILIES = ("coxeter", "all_transpositions", "lrx", "pancake", "random_inv")


def serve_diameter_guess(family: str, n: int) -> int:
    """Upper end D of the radius-cap range per family: n(n-1)/2 for Coxeter and LRX
    (their diameters, Section 3.3), n-1 for all transpositions, ceil(1.2 n) + 2 for pancake
    (the table gives only "about 1.2 n"), and n^2/2 + 4n for random sets (the conjectured
    bound of Section 3.6)."""
    if family in ("coxeter", "lrx"):
        return n * (n - 1) // 2
    if family == "all_transpositions":
        return n - 1
    if family == "pancake":
        return int(math.ceil(1.2 * n)) + 2
    return n * n // 2 + 4 * n


def serve_stream(seed: int = SERVE_SEED, count: int = 20000,
                 n_range=(8, 16)) -> List[GrowthJob]:
    """Config 5: Poisson arrivals (unit rate; scale by 1/rate), mixed families and caps."""
    rng = np.random.Generator(np.random.PCG64(seed))
    jobs: List[GrowthJob] = []
    t = 0.0
    for j in range(count):
        t += float(rng.exponential(1.0))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        family = SERVE_FAMILIES[int(rng.integers(0, len(SERVE_FAMILIES)))]
        if family == "random_inv":
            kk = int(rng.integers(2, 6))
            gens = fam.inverse_closure(fam.random_perms(rng, n, kk))
        else:
            gens = fam.FAMILIES[family](n)
        D = max(6, serve_diameter_guess(family, n))
        cap = int(rng.integers(6, D + 1))
        jobs.append(GrowthJob(n, gens, True, max_radius=cap, name=f"serve{j}",
                              family=family, arrival=t))
    return jobs


def describe(job: GrowthJob) -> dict:
    return {"name": job.name, "n": job.n, "k": job.k, "family": job.family,
            "inverse_closed": job.inverse_closed, "max_radius": job.max_radius}


def optional_int(x: Optional[int]) -> int:
    return -1 if x is None else int(x)
