"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA-side tests/bench.

This module holds no Montgomery, multiplication or exponentiation code of the
method under test. It only draws random limbs, shapes them (bit length, odd
moduli, values below a modulus) and converts between limb arrays and Python
integers. Prime generation for the RSA-like moduli uses Python's built-in
``pow`` for Miller-Rabin, which is input generation, not the method.

Limb convention everywhere: little-endian uint32 words, ``n = ceil(bits/32)``
words per value, instance-major arrays of shape ``[batch, n]``.

Workload recipes (one independent stream per (seed, workload, field)):

* ``plain_small``   : batch 8, 1024-bit random odd moduli, bases < N, 1024-bit exponents.
* ``batch_2048``    : 2048-bit moduli, half random odd, half products of two 1024-bit
                      primes (top two bits set) drawn from a seeded prime pool.
* ``batch_4096``    : 4096-bit (and 4108/4154-bit edge sizes) random odd moduli.
* ``mixed``         : sizes drawn 40% 2048 / 25% 1024 / 20% 3072 / 15% 4096.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

FIELDS = {"modulus": 1, "base": 2, "exponent": 3, "prime": 4, "size": 5, "other": 6,
          "arrival": 7, "pool": 8}
WORKLOADS = {"plain_small": 1, "batch_2048": 2, "batch_4096": 3, "mixed": 4, "serving": 5, "lazy": 6,
             "test": 99}


def limbs_for(bits: int) -> int:
    """Number of 32-bit words for a ``bits``-bit value."""
    return (int(bits) + 31) // 32


def stream(seed: int, workload: str | int, field: str | int, sub: int = 0) -> np.random.Generator:
    """Independent PCG64 stream keyed by (seed, workload, field, sub)."""
    w = WORKLOADS[workload] if isinstance(workload, str) else int(workload)
    f = FIELDS[field] if isinstance(field, str) else int(field)
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), w, f, int(sub)])))


def random_bits(rng: np.random.Generator, batch: int, bits: int) -> np.ndarray:
    """Uniform ``bits``-bit strings (top bit not forced), shape [batch, n] uint32."""
    n = limbs_for(bits)
    x = rng.integers(0, 1 << 32, size=(batch, n), dtype=np.uint64).astype(np.uint32)
    top = bits - 32 * (n - 1)
    if top < 32:
        x[:, n - 1] &= np.uint32((1 << top) - 1)
    return x


def random_odd_moduli(rng: np.random.Generator, batch: int, bits: int) -> np.ndarray:
    """Random odd ``bits``-bit moduli with the top bit set."""
    x = random_bits(rng, batch, bits)
    n = x.shape[1]
    top = bits - 32 * (n - 1)
    x[:, n - 1] |= np.uint32(1 << (top - 1))
    x[:, 0] |= np.uint32(1)
    return x


def less_than(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Row-wise a < b for [batch, n] limb arrays (vectorised lexicographic compare)."""
    lt = np.zeros(a.shape[0], dtype=bool)
    decided = np.zeros(a.shape[0], dtype=bool)
    for i in range(a.shape[1] - 1, -1, -1):
        ai, bi = a[:, i], b[:, i]
        newly = ~decided & (ai != bi)
        lt |= newly & (ai < bi)
        decided |= newly
    return lt


def uniform_below(rng: np.random.Generator, N: np.ndarray, bits: int) -> np.ndarray:
    """Values uniform in [0, N) per row, by rejection sampling of ``bits``-bit strings."""
    out = np.zeros_like(N)
    todo = np.arange(N.shape[0])
    while todo.size:
        cand = random_bits(rng, todo.size, bits)
        ok = less_than(cand, N[todo])
        out[todo[ok]] = cand[ok]
        todo = todo[~ok]
    return out


def to_int(limbs) -> int:
    """One value's limbs (little-endian uint32) to a Python int."""
    return int.from_bytes(np.asarray(limbs, dtype="<u4").tobytes(), "little")


def to_ints(arr: np.ndarray) -> list[int]:
    return [to_int(r) for r in np.asarray(arr)]


def from_int(x: int, n: int) -> np.ndarray:
    """Python int to n little-endian uint32 limbs (x must fit)."""
    if x < 0 or x.bit_length() > 32 * n:
        raise ValueError("value does not fit")
    return np.frombuffer(int(x).to_bytes(4 * n, "little"), dtype="<u4").astype(np.uint32)


def from_ints(xs, n: int) -> np.ndarray:
    return np.stack([from_int(int(x), n) for x in xs]) if len(xs) else np.zeros((0, n), np.uint32)


# ----------------------------------------------------------------------------- primes

_SMALL_PRIMES = None


def _small_primes(limit: int = 20000) -> np.ndarray:
    global _SMALL_PRIMES
    if _SMALL_PRIMES is None:
        sieve = np.ones(limit, dtype=bool)
        sieve[:2] = False
        for p in range(2, int(limit ** 0.5) + 1):
            if sieve[p]:
                sieve[p * p::p] = False
        _SMALL_PRIMES = np.nonzero(sieve)[0][1:]  # odd primes
    return _SMALL_PRIMES


def _miller_rabin(x: int, rng: np.random.Generator, rounds: int) -> bool:
    d, s = x - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for _ in range(rounds):
        a = 2 + int(rng.integers(0, 1 << 62)) % (x - 3)
        y = pow(a, d, x)
        if y in (1, x - 1):
            continue
        for _ in range(s - 1):
            y = y * y % x
            if y == x - 1:
                break
        else:
            return False
    return True


def random_prime(rng: np.random.Generator, bits: int, rounds: int = 24) -> int:
    """Random prime of exactly ``bits`` bits with its top two bits set.

    Candidates are scanned upward from a random odd start; a sieve over small
    primes discards most of them before Miller-Rabin."""
    sp = _small_primes()
    span = 4 * bits
    while True:
        start = int.from_bytes(rng.bytes((bits + 7) // 8), "little")
        start &= (1 << bits) - 1
        start |= (3 << (bits - 2)) | 1
        # offsets k (candidate start + 2k) divisible by a small prime are removed
        alive = np.ones(span, dtype=bool)
        for p in sp:
            if p >= start:
                break
            r = start % int(p)
            # start + 2k == 0 mod p  <=>  k == -r * inv(2) mod p
            k0 = (-r * ((int(p) + 1) // 2)) % int(p)
            alive[k0::int(p)] = False
        for k in np.nonzero(alive)[0]:
            x = start + 2 * int(k)
            if x.bit_length() != bits:
                break
            if _miller_rabin(x, rng, rounds):
                return x


def _pool_prime(args):
    seed, workload, i, bits = args
    return random_prime(stream(seed, workload, "prime", i), bits)


def prime_pool(seed: int, workload: str, count: int, bits: int, procs: int = 0) -> list[int]:
    """``count`` primes; prime i comes from its own stream, so the pool is the same
    whether it is generated serially or by a (spawned) process pool."""
    jobs = [(seed, workload, i, bits) for i in range(count)]
    if procs and procs > 1 and count > 8:
        import multiprocessing as mproc
        with mproc.get_context("spawn").Pool(procs) as pool:
            return pool.map(_pool_prime, jobs, chunksize=max(1, count // (4 * procs)))
    return [_pool_prime(j) for j in jobs]


def rsa_moduli(seed: int, workload: str, batch: int, bits: int, pool_size: int | None = None,
               procs: int = 0) -> np.ndarray:
    """``batch`` products p*q of distinct primes of bits/2 bits (top two bits set),
    drawn as distinct pairs from a seeded pool of primes; each product has exactly
    ``bits`` bits. The pool is the smallest size whose pair count covers ``batch``
    (at least 2), so the cost of prime generation stays bounded."""
    if pool_size is None:
        pool_size = max(2, int(math.ceil((1 + math.sqrt(1 + 8 * batch)) / 2)))
    primes = prime_pool(seed, workload, pool_size, bits // 2, procs)
    rng = stream(seed, workload, "pool")
    pairs = set()
    out = []
    P = len(primes)
    while len(out) < batch:
        i, j = (int(v) for v in rng.integers(0, P, size=2))
        if i == j or (min(i, j), max(i, j)) in pairs:
            if len(pairs) >= P * (P - 1) // 2:
                pairs.clear()
            continue
        pairs.add((min(i, j), max(i, j)))
        out.append(primes[i] * primes[j])
    return from_ints(out, limbs_for(bits))


# ----------------------------------------------------------------------------- workloads


@dataclass
class Batch:
    """One fixed-size batch: moduli N, bases a < N and exponents e (all [batch, *] uint32)."""
    bits: int
    N: np.ndarray
    a: np.ndarray
    b: np.ndarray
    e: np.ndarray
    ebits: int

    @property
    def n(self) -> int:
        return self.N.shape[1]

    @property
    def batch(self) -> int:
        return self.N.shape[0]


def make_batch(seed: int, workload: str, batch: int, bits: int, ebits: int | None = None,
               rsa_fraction: float = 0.0, sub: int = 0, procs: int = 0) -> Batch:
    """Random odd moduli (a fraction of them RSA-like products), bases a, b < N and
    ``ebits``-bit exponents (default: full length, ``ebits = bits``)."""
    ebits = bits if ebits is None else ebits
    N = random_odd_moduli(stream(seed, workload, "modulus", sub), batch, bits)
    n_rsa = int(round(batch * rsa_fraction))
    if n_rsa:
        N[batch - n_rsa:] = rsa_moduli(seed, workload, n_rsa, bits, procs=procs)
    rb = stream(seed, workload, "base", sub)
    a = uniform_below(rb, N, bits)
    b = uniform_below(rb, N, bits)
    e = random_bits(stream(seed, workload, "exponent", sub), batch, ebits) if ebits > 0 \
        else np.zeros((batch, 1), np.uint32)
    return Batch(bits, N, a, b, e, ebits)


def plain_small(seed: int = 0) -> Batch:
    """8 instances, 1024-bit random odd moduli, uniform bases, 1024-bit exponents."""
    return make_batch(seed, "plain_small", 8, 1024)


def batch_2048(seed: int = 0, batch: int = 65536, procs: int = 0) -> Batch:
    """2048-bit moduli, half random odd, half products of two 1024-bit primes."""
    return make_batch(seed, "batch_2048", batch, 2048, rsa_fraction=0.5, procs=procs)


def batch_4096(seed: int = 0, batch: int = 16384, bits: int = 4096) -> Batch:
    return make_batch(seed, "batch_4096", batch, bits, sub=bits)


MIX = ((2048, 0.40), (1024, 0.25), (3072, 0.20), (4096, 0.15))


def mixed_sizes(seed: int, count: int) -> np.ndarray:
    """Per-instance bit sizes for the mixed workload, shuffled with the seed."""
    counts = [int(round(count * f)) for _, f in MIX]
    counts[0] += count - sum(counts)
    sizes = np.concatenate([np.full(c, b, dtype=np.int32) for (b, _), c in zip(MIX, counts)])
    stream(seed, "mixed", "size").shuffle(sizes)
    return sizes


# ----------------------------------------------------------------------------- serving traces


@dataclass
class Trace:
    """A request trace: arrival times (s, increasing), the pool entry each request uses,
    and its exponent words (full length for that entry's size, instance-major). bases:
    None for a fixed-base trace, else per request its own base words (below the entry's
    modulus) or None for a request on the entry's fixed base."""
    arrival: np.ndarray      # float64 [count]
    entry: np.ndarray        # int64 [count], index into the pool
    exponents: list          # per request: uint32 words
    bases: list | None = None


def pool_sizes(seed: int, count: int) -> np.ndarray:
    """Bit sizes of a resident pool of ``count`` moduli with the mixed-size distribution."""
    return mixed_sizes(seed + 1000, count)


@dataclass
class PoolInputs:
    """A resident serving pool: entry k has sizes[k] bits; moduli[bits] and bases[bits] list the
    moduli and fixed bases of the entries of that size in entry order."""
    sizes: np.ndarray
    moduli: dict
    bases: dict


def serving_pool(seed: int, count: int) -> PoolInputs:
    """``count`` pool entries with the mixed-size distribution: random odd moduli and one
    uniform fixed base below each."""
    sizes = pool_sizes(seed, count)
    moduli, bases = {}, {}
    for bits in sorted(set(int(b) for b in sizes)):
        cnt = int((sizes == bits).sum())
        b = make_batch(seed, "serving", cnt, bits, ebits=1, sub=bits)
        moduli[bits], bases[bits] = b.N, b.a
    return PoolInputs(sizes, moduli, bases)


def poisson_trace(seed: int, rate: float, count: int, sizes: np.ndarray) -> Trace:
    """``count`` requests with exponential inter-arrival gaps of mean 1/rate, each picking a
    pool entry uniformly and carrying a fresh full-length exponent for that entry's size."""
    r = stream(seed, "serving", "arrival", int(rate))
    gaps = r.exponential(1.0 / rate, size=count)
    arrival = np.cumsum(gaps)
    entry = r.integers(0, len(sizes), size=count)
    re = stream(seed, "serving", "exponent", int(rate))
    exps = []
    for k in entry:
        bits = int(sizes[k])
        exps.append(random_bits(re, 1, bits)[0])
    return Trace(arrival, entry, exps)


def with_bases(trace: Trace, pool: PoolInputs, fraction: float, seed: int = 0) -> Trace:
    """The same trace with a fraction of its requests (chosen with the seed) carrying their own
    base, uniform below the modulus of their pool entry."""
    r = stream(seed, "serving", "base", int(1e6 * fraction))
    pick = r.random(len(trace.arrival)) < fraction
    local = {}
    for bits in pool.moduli:
        ids = np.nonzero(pool.sizes == bits)[0]
        local.update({int(k): i for i, k in enumerate(ids)})
    bases = []
    for k, (e, v) in enumerate(zip(trace.entry, pick)):
        if not v:
            bases.append(None)
            continue
        bits = int(pool.sizes[e])
        N = pool.moduli[bits][local[int(e)]][None, :]
        bases.append(uniform_below(r, N, bits)[0])
    return Trace(trace.arrival, trace.entry, trace.exponents, bases)
