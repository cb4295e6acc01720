"""Seeded synthetic sequencing reads for the five workloads.

This module only simulates input: a random genome with repeat families and
tandem arrays, reads sampled from either strand with substitution errors.  It
computes nothing of the graph construction (no k-mers, no canonical forms),
so both the CUDA path and the CPU oracle can consume what it produces.

Recipes (genome model, read model, seeds) are the five workloads of the
method's evaluation on one GPU:

  tiny       100 kbp uniform genome, 10,000 x 36 bp reads, 1 % errors, k = 21
  large      50 Mbp genome, >= 2 % covered by copies of 10 repeat families
             (1-5 kbp, 1 % diverged), 15 M x 100 bp reads (30x), 0.5 %, k = 31
  long_k     20 Mbp genome, repeats as above plus 0.5 % tandem arrays,
             4 M x 150 bp reads (30x), 0.3 % errors, k = 55
  batched    256 read sets: genome log-uniform on [10 kbp, 5 Mbp], coverage
             U[10, 60], read length in {36, 75, 100, 150}, errors U[0, 1 %],
             k in {21, 31}
  served     Poisson arrivals of requests drawn like ``batched``

Every read set is returned as (reads, lengths): ``reads`` a uint8 array of
ASCII 'A','C','G','T' with all reads back to back, ``lengths`` uint32.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

ALPHABET = np.frombuffer(b"ACGT", dtype=np.uint8)
# the other strand of DNA pairs A with T and C with G (a byte translation)
_PAIR = np.zeros(256, dtype=np.uint8)
for _a, _b in zip(b"ACGT", b"TGCA"):
    _PAIR[_a] = _b


@dataclasses.dataclass(frozen=True)
class ReadSetSpec:
    genome_len: int
    n_reads: int
    read_len: int
    error_rate: float
    k: int
    seed: int
    repeat_fraction: float = 0.0     # interspersed repeat coverage target
    tandem_fraction: float = 0.0     # tandem-array coverage target

    @property
    def raw_edges(self) -> int:
        return self.n_reads * max(0, self.read_len - self.k)


def tiny_spec(seed: int = 0) -> ReadSetSpec:
    return ReadSetSpec(100_000, 10_000, 36, 0.01, 21, seed)


def large_spec(scale: float = 1.0, seed: int = 1) -> ReadSetSpec:
    g = max(20_000, int(round(50_000_000 * scale)))
    n = int(round(15_000_000 * scale))
    return ReadSetSpec(g, max(1, n), 100, 0.005, 31, seed, repeat_fraction=0.02)


def long_k_spec(scale: float = 1.0, seed: int = 2) -> ReadSetSpec:
    g = max(20_000, int(round(20_000_000 * scale)))
    n = int(round(4_000_000 * scale))
    return ReadSetSpec(g, max(1, n), 150, 0.003, 55, seed,
                       repeat_fraction=0.02, tandem_fraction=0.005)


def batched_specs(n_sets: int = 256, seed: int = 3, max_genome: int = 5_000_000,
                  min_genome: int = 10_000) -> list[ReadSetSpec]:
    """Per-set recipe: genome log-uniform on [min_genome, max_genome],
    coverage U[10, 60], read length from {36, 75, 100, 150}, errors U[0, 1 %],
    k from {21, 31}; each set has its own sub-seed."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(n_sets):
        g = int(round(math.exp(rng.uniform(math.log(min_genome), math.log(max_genome)))))
        cov = rng.uniform(10.0, 60.0)
        L = int(rng.choice([36, 75, 100, 150]))
        err = float(rng.uniform(0.0, 0.01))
        k = int(rng.choice([21, 31]))
        n = max(1, int(round(cov * g / L)))
        specs.append(ReadSetSpec(max(g, L), n, L, err, k, seed * 1_000_003 + i + 1))
    return specs


# --------------------------------------------------------------------------
# genome model
# --------------------------------------------------------------------------

def _mutate(codes: np.ndarray, rate: float, rng: np.random.Generator) -> np.ndarray:
    """i.i.d. substitutions; the new base is uniform over the other three."""
    if rate <= 0 or codes.size == 0:
        return codes
    hit = rng.random(codes.shape, dtype=np.float32) < rate
    shift = rng.integers(1, 4, size=codes.shape, dtype=np.uint8)
    return np.where(hit, (codes + shift) & 3, codes).astype(np.uint8)


def _insertions(spec: ReadSetSpec, rng: np.random.Generator) -> list[np.ndarray]:
    """Repeat copies and tandem arrays to be written into the genome."""
    out = []
    g = spec.genome_len
    if spec.repeat_fraction > 0:
        # 10 families of 1-5 kbp, 20 copies each, then further copies
        # round-robin until the target fraction of the genome is covered
        fams = [rng.integers(0, 4, size=int(rng.integers(1000, 5001)), dtype=np.uint8)
                for _ in range(10)]
        copies, covered, i = [], 0, 0
        while i < 200 or covered < spec.repeat_fraction * g:
            f = fams[i % 10]
            copies.append(_mutate(f.copy(), 0.01, rng))
            covered += f.size
            i += 1
            if covered > 0.5 * g:
                break
        out.extend(copies)
    if spec.tandem_fraction > 0:
        covered = 0
        while covered < spec.tandem_fraction * g:
            unit = rng.integers(0, 4, size=int(rng.integers(2, 101)), dtype=np.uint8)
            length = int(rng.integers(500, 5001))
            arr = np.resize(unit, length)
            out.append(_mutate(arr, 0.01, rng))
            covered += length
    return out


def genome_codes(spec: ReadSetSpec, rng: np.random.Generator) -> tuple[np.ndarray, float]:
    """Random uniform genome (codes 0..3) with the spec's insertions written at
    uniform, non-overlapping positions; returns it and the covered fraction."""
    g = spec.genome_len
    genome = rng.integers(0, 4, size=g, dtype=np.uint8)
    ins = _insertions(spec, rng)
    if not ins:
        return genome, 0.0
    order = rng.permutation(len(ins))
    seg = g // len(ins)
    covered = 0
    for slot, idx in enumerate(order):
        piece = ins[idx]
        if piece.size >= seg:
            continue
        start = slot * seg + int(rng.integers(0, seg - piece.size + 1))
        genome[start:start + piece.size] = piece
        covered += piece.size
    return genome, covered / g


def _substitute(block: np.ndarray, rate: float, rng: np.random.Generator) -> None:
    """i.i.d. per-base substitutions in place: the number of errors is
    Binomial(size, rate), their positions a uniform subset, and each new base
    uniform over the other three."""
    flat = block.reshape(-1)
    count = int(rng.binomial(flat.size, rate))
    if count == 0:
        return
    pos = rng.choice(flat.size, size=count, replace=False)
    code_of = np.zeros(256, dtype=np.uint8)
    code_of[ALPHABET] = np.arange(4, dtype=np.uint8)
    shift = rng.integers(1, 4, size=count, dtype=np.uint8)
    flat[pos] = ALPHABET[(code_of[flat[pos]] + shift) & 3]


def sample_reads(spec: ReadSetSpec, genome_ascii: np.ndarray, rng: np.random.Generator,
                 chunk: int = 1 << 18) -> tuple[np.ndarray, np.ndarray]:
    """Reads of fixed length at uniform positions of a linear genome, each
    from the reverse strand with probability 1/2, with substitution errors."""
    L, n = spec.read_len, spec.n_reads
    out = np.empty(n * L, dtype=np.uint8)
    windows = np.lib.stride_tricks.sliding_window_view(genome_ascii, L)
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        m = c1 - c0
        starts = rng.integers(0, windows.shape[0], size=m, dtype=np.int64)
        block = windows[starts]
        reverse = rng.random(m) < 0.5
        block[reverse] = _PAIR[block[reverse][:, ::-1]]
        if spec.error_rate > 0:
            _substitute(block, spec.error_rate, rng)
        out[c0 * L:c1 * L] = block.reshape(-1)
    return out, np.full(n, L, dtype=np.uint32)


def generate(spec: ReadSetSpec) -> tuple[np.ndarray, np.ndarray]:
    """(reads, lengths) for one read set, deterministic in spec.seed."""
    rng = np.random.default_rng(spec.seed)
    codes, _ = genome_codes(spec, rng)
    return sample_reads(spec, ALPHABET[codes], rng)


def random_reads(rng: np.random.Generator, n: int, min_len: int, max_len: int,
                 alphabet: bytes = b"ACGT") -> tuple[np.ndarray, np.ndarray]:
    """Unrelated reads of uniform random lengths (for ragged-size tests)."""
    lengths = rng.integers(min_len, max_len + 1, size=n).astype(np.uint32)
    letters = np.frombuffer(alphabet, dtype=np.uint8)
    reads = letters[rng.integers(0, len(letters), size=int(lengths.sum()))]
    return reads.astype(np.uint8), lengths


def poisson_arrivals(rate_per_s: float, n: int, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson stream with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
