"""Seeded synthetic case-control genotype data for the three-way epistasis scan.

This module only simulates inputs.  It contains none of the method's arithmetic
(no bit packing, no contingency counting, no K2), so both the CPU oracle and the
CUDA library can consume what it produces without sharing any code.

Data model (paper Sec. III): a data set of M SNPs x N samples, genotype values
0 (homozygous major), 1 (heterozygous), 2 (homozygous minor), and one phenotype
value per sample, 0 = control and 1 = case.  Genotypes are returned SNP-major,
``genotypes[m, s]``, as uint8; the phenotype is a separate uint8 vector.

Simulation recipe (the paper's own synthetic sets are not described, Sec. V):

* per SNP a minor-allele frequency p ~ U[a, b], genotypes ~ Binomial(2, p)
  (Hardy-Weinberg equilibrium);
* planted interacting triplets: each planted triplet uses three distinct SNPs
  whose MAF is drawn from U[0.25, 0.5] (or fixed), and an individual carrying
  the genotype combination (1, 1, 1) at those three SNPs has its disease odds
  multiplied by ``odds_ratio`` (3) over a baseline prevalence of 0.1;
* case-control ascertainment: individuals are simulated in order and kept as
  cases or controls until the exact quotas N1 = n_cases and N0 = N - N1 are
  filled.  Kept samples stay in simulation order, so cases and controls are
  interleaved.  SNPs outside planted triplets do not influence the phenotype,
  so they are drawn directly for the kept individuals.
* optional duplicated SNP columns copy the genotype row of a planted SNP into
  another column, which creates triplets with exactly equal tables (ties).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = ["Dataset", "make_dataset", "make_config", "make_batch", "CONFIGS",
           "n_triplets"]


@dataclass
class Dataset:
    genotypes: np.ndarray          # uint8 [M, N], values 0/1/2
    phenotype: np.ndarray          # uint8 [N], values 0/1
    maf: np.ndarray                # float64 [M]
    planted: list = field(default_factory=list)      # sorted (i, j, k) tuples
    duplicates: list = field(default_factory=list)   # (source, copy) columns
    name: str = ""
    seed: int = 0
    top_k: int = 10

    @property
    def n_snps(self) -> int:
        return int(self.genotypes.shape[0])

    @property
    def n_samples(self) -> int:
        return int(self.genotypes.shape[1])

    @property
    def n_cases(self) -> int:
        return int(self.phenotype.sum())


def n_triplets(m: int) -> int:
    return m * (m - 1) * (m - 2) // 6


def make_dataset(n_snps: int, n_samples: int, n_cases: int, maf_range=(0.05, 0.5),
                 n_planted: int = 1, seed: int = 1, planted_maf=None,
                 odds_ratio: float = 3.0, prevalence: float = 0.1,
                 n_duplicates: int = 0, name: str = "", top_k: int = 10,
                 rng: np.random.Generator | None = None) -> Dataset:
    """Simulate one case-control data set (see the module docstring)."""
    if n_snps < 1 or n_samples < 0 or not (0 <= n_cases <= n_samples):
        raise ValueError("bad shape")
    if 3 * n_planted + n_duplicates > n_snps:
        raise ValueError("not enough SNPs for the planted triplets and duplicates")
    rng = np.random.default_rng(seed) if rng is None else rng
    M, N, N1 = int(n_snps), int(n_samples), int(n_cases)
    N0 = N - N1
    maf = rng.uniform(maf_range[0], maf_range[1], size=M)

    planted_idx = rng.choice(M, size=3 * n_planted, replace=False) if n_planted else \
        np.zeros(0, dtype=np.int64)
    planted = [tuple(sorted(int(x) for x in planted_idx[3 * t:3 * t + 3]))
               for t in range(n_planted)]
    if n_planted:
        if planted_maf is None:
            maf[planted_idx] = rng.uniform(0.25, 0.5, size=planted_idx.size)
        else:
            maf[planted_idx] = float(planted_maf)

    odds0 = prevalence / (1.0 - prevalence)
    pl_cols = planted_idx  # order: triplet t uses columns 3t..3t+2 of this array
    kept_pl = np.zeros((N, pl_cols.size), dtype=np.uint8)
    kept_ph = np.zeros(N, dtype=np.uint8)
    n_ctrl = n_case = n_kept = 0
    batch = max(4096, 2 * N)
    while n_ctrl < N0 or n_case < N1:
        g = rng.binomial(2, maf[pl_cols][None, :], size=(batch, pl_cols.size)).astype(np.uint8)
        odds = np.full(batch, odds0)
        for t in range(n_planted):
            hit = np.all(g[:, 3 * t:3 * t + 3] == 1, axis=1)
            odds = np.where(hit, odds * odds_ratio, odds)
        is_case = rng.random(batch) < odds / (1.0 + odds)
        take_case = np.nonzero(is_case)[0][: N1 - n_case]
        take_ctrl = np.nonzero(~is_case)[0][: N0 - n_ctrl]
        take = np.sort(np.concatenate([take_case, take_ctrl]))
        kept_pl[n_kept:n_kept + take.size] = g[take]
        kept_ph[n_kept:n_kept + take.size] = is_case[take]
        n_case += take_case.size
        n_ctrl += take_ctrl.size
        n_kept += take.size

    geno = rng.binomial(2, maf[:, None], size=(M, N)).astype(np.uint8)
    if pl_cols.size:
        geno[pl_cols, :] = kept_pl.T

    duplicates = []
    if n_duplicates:
        free = np.setdiff1d(np.arange(M), pl_cols)
        dst = rng.choice(free, size=n_duplicates, replace=False)
        for d in range(n_duplicates):
            src = int(pl_cols[d % pl_cols.size]) if pl_cols.size else int(rng.integers(M))
            geno[int(dst[d])] = geno[src]
            maf[int(dst[d])] = maf[src]
            duplicates.append((src, int(dst[d])))

    return Dataset(genotypes=np.ascontiguousarray(geno), phenotype=kept_ph, maf=maf,
                   planted=planted, duplicates=duplicates, name=name, seed=seed,
                   top_k=top_k)


# The five workloads of the scan: (name, SNPs, samples, case fraction, MAF range,
# planted triplets, extra keyword arguments, top-k).
CONFIGS = {
    "tiny":   dict(n_snps=64, n_samples=512, case_fraction=0.5, maf_range=(0.05, 0.5),
                   n_planted=1, top_k=10),
    "medium": dict(n_snps=1024, n_samples=8192, case_fraction=0.5, maf_range=(0.05, 0.5),
                   n_planted=2, top_k=10),
    "large":  dict(n_snps=2048, n_samples=16384, case_fraction=0.4, maf_range=(0.01, 0.5),
                   n_planted=1, top_k=10),
    "stress": dict(n_snps=4096, n_samples=4096, case_fraction=0.5, maf_range=(0.02, 0.5),
                   n_planted=4, planted_maf=0.4, n_duplicates=2, top_k=64),
}


def make_config(name: str, seed: int = 1, n_snps: int | None = None) -> Dataset:
    """One of the named single-cohort workloads: tiny, medium, large, stress (optionally
    with another SNP count, everything else kept: a smaller case of the same shape)."""
    c = dict(CONFIGS[name])
    if n_snps is not None:
        c["n_snps"] = int(n_snps)
    frac = c.pop("case_fraction")
    n1 = int(round(frac * c["n_samples"]))
    return make_dataset(n_cases=n1, seed=seed, name=name, **c)


def make_batch(seed: int = 1, n_cohorts: int = 48, m_range=(96, 1024),
               n_range=(1000, 20000), frac_range=(0.2, 0.6), top_k: int = 5) -> list:
    """The many-cohort workload: independent data sets of uneven shape.

    SNP count ~ U{96..1024}, sample count ~ U{1000..20000}, case fraction
    ~ U[0.2, 0.6], MAF ~ U[0.05, 0.5], one planted triplet each, top-5.
    """
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_cohorts):
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        f = float(rng.uniform(frac_range[0], frac_range[1]))
        child = int(rng.integers(1 << 62))
        out.append(make_dataset(m, n, int(round(f * n)), (0.05, 0.5), 1, seed=child,
                                name=f"cohort{c}", top_k=top_k))
    return out


def total_sample_triplets(datasets) -> int:
    return sum(n_triplets(d.n_snps) * d.n_samples for d in datasets)


def random_triplets(m: int, n: int, seed: int = 0) -> np.ndarray:
    """n uniformly random sorted triplets i<j<k over m SNPs (int32 [n, 3])."""
    rng = np.random.default_rng(seed)
    out = np.empty((n, 3), dtype=np.int32)
    got = 0
    while got < n:
        t = np.sort(rng.integers(0, m, size=(2 * (n - got) + 16, 3)), axis=1)
        ok = (t[:, 0] < t[:, 1]) & (t[:, 1] < t[:, 2])
        t = t[ok][: n - got]
        out[got:got + len(t)] = t
        got += len(t)
    return out


def _self_check():  # pragma: no cover - manual use
    d = make_config("tiny")
    assert d.genotypes.shape == (64, 512) and d.n_cases == 256
    assert math.comb(64, 3) == n_triplets(64)
