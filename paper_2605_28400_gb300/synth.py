"""Seeded synthetic triplet workloads (inputs only — no alignment arithmetic lives here).

The paper evaluates on AliSim-simulated triplets and on Illumina reads, neither of which is
available; these generators stand in for them with the same kind of structure: related
sequences derived from a common ancestor by substitutions and geometric-length indels, over the
DNA alphabet (match/mismatch scoring) or a 20-letter protein alphabet (seeded symmetric
substitution matrix).

Random numbers come from splitmix64 used as a counter-based generator (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): draw ``n`` of stream ``key`` is
``mix64(key + (n + 1) * 0x9E3779B97F4A7C15)``. Being counter based, any draw can be computed on
its own, which keeps the mutation process vectorisable and identical on every machine.

Both the CUDA path's tests/bench and the oracle consume what this module returns; neither
side's arithmetic is here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

DNA_ALPHABET = "ACGT"
PROTEIN_ALPHABET = "ACDEFGHIKLMNPQRSTVWY"

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1


def _mix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser on a uint64 array (wrap-around arithmetic)."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def _mix64_int(z: int) -> int:
    z &= _MASK
    z ^= z >> 30
    z = (z * 0xBF58476D1CE4E5B9) & _MASK
    z ^= z >> 27
    z = (z * 0x94D049BB133111EB) & _MASK
    z ^= z >> 31
    return z


def stream_key(*parts: int) -> int:
    """Derive an independent stream key from a seed and integer tags."""
    k = 0x243F6A8885A308D3
    for p in parts:
        k = _mix64_int(k ^ _mix64_int((int(p) + 0x632BE59BD9B4E019) & _MASK))
    return k


def draws_u64(key: int, counters: np.ndarray) -> np.ndarray:
    """uint64 draws of stream ``key`` at the given counters (random access)."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key) + (c + np.uint64(1)) * _GAMMA
    return _mix64(z)


def uniform(key: int, counters: np.ndarray) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each draw."""
    return (draws_u64(key, counters) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def categorical(key: int, counters: np.ndarray, cdf: np.ndarray) -> np.ndarray:
    u = uniform(key, counters)
    return np.minimum(np.searchsorted(cdf, u, side="right"), len(cdf) - 1).astype(np.uint8)


@dataclass
class Scoring:
    """Alphabet, symmetric int8 substitution matrix and linear gap alpha (<= 0)."""
    alphabet: str
    sub: np.ndarray          # (K, K) int32, symmetric
    gap: int
    freqs: np.ndarray        # background residue frequencies (for generation only)
    name: str = ""

    @property
    def K(self) -> int:
        return len(self.alphabet)


def dna_scoring() -> Scoring:
    """DNA: match +2, mismatch -1, gap -2 per residue-gap pair, uniform background."""
    K = 4
    sub = np.full((K, K), -1, dtype=np.int32)
    np.fill_diagonal(sub, 2)
    return Scoring(DNA_ALPHABET, sub, -2, np.full(K, 0.25), "dna")


def protein_scoring(seed: int) -> Scoring:
    """Protein: seeded symmetric matrix (diagonal U{4..11}, off-diagonal U{-4..2}), gap -4,
    background frequencies from weights U[0.5, 1.5] normalised."""
    K = 20
    key = stream_key(seed, 0x5C0)
    sub = np.zeros((K, K), dtype=np.int32)
    iu = np.triu_indices(K, 1)
    off = (draws_u64(key, np.arange(len(iu[0]))) % np.uint64(7)).astype(np.int64) - 4
    sub[iu] = off
    sub[(iu[1], iu[0])] = off
    diag = (draws_u64(key, np.arange(1000, 1000 + K)) % np.uint64(8)).astype(np.int64) + 4
    sub[np.arange(K), np.arange(K)] = diag
    w = 0.5 + uniform(key, np.arange(2000, 2000 + K))
    return Scoring(PROTEIN_ALPHABET, sub, -4, w / w.sum(), "protein")


def random_seq(key: int, n: int, freqs: np.ndarray) -> np.ndarray:
    cdf = np.cumsum(freqs)
    cdf[-1] = 1.0
    return categorical(key, np.arange(n, dtype=np.uint64), cdf)


_INDEL_CAP = 64  # geometric indel lengths are truncated here (tail mass < 1e-11 at mean 3)


def mutate(key: int, anc: np.ndarray, p_sub: float, p_indel: float, mean_len: float,
           freqs: np.ndarray) -> np.ndarray:
    """Descendant of ``anc``: at each ancestral position an indel event starts with probability
    ``p_indel`` (insertion or deletion with equal chance, length geometric on {1,2,...} with the
    given mean, truncated at 64); an insertion puts new background residues before the position,
    a deletion removes the position and the ones after it. A kept residue is substituted with
    probability ``p_sub`` by a uniformly chosen different residue."""
    L = len(anc)
    K = len(freqs)
    cdf = np.cumsum(freqs)
    cdf[-1] = 1.0
    pos = np.arange(L, dtype=np.uint64)
    u_ev = uniform(key, pos * np.uint64(8))
    u_sub = uniform(key, pos * np.uint64(8) + np.uint64(1))
    seq = anc.copy()
    subs = np.nonzero(u_sub < p_sub)[0]
    if len(subs):
        shift = 1 + (draws_u64(key, subs.astype(np.uint64) * np.uint64(8) + np.uint64(2))
                     % np.uint64(K - 1)).astype(np.int64)
        seq[subs] = ((seq[subs].astype(np.int64) + shift) % K).astype(np.uint8)
    keep = np.ones(L, dtype=bool)
    inserts: dict[int, np.ndarray] = {}
    events = np.nonzero(u_ev < p_indel)[0]
    q = 1.0 / mean_len
    deleted_until = -1
    for p in events:
        p = int(p)
        if p <= deleted_until:
            continue
        c = np.array([p * 8 + 3, p * 8 + 4], dtype=np.uint64)
        u_type, u_len = uniform(key, c)
        ell = 1 + int(math.floor(math.log(max(1.0 - u_len, 1e-300)) / math.log(1.0 - q))) \
            if q < 1.0 else 1
        ell = min(ell, _INDEL_CAP)
        if u_type < 0.5:
            ikey = stream_key(key, p)
            inserts[p] = categorical(ikey, np.arange(ell, dtype=np.uint64), cdf)
        else:
            keep[p:p + ell] = False
            deleted_until = p + ell - 1
    if not inserts:
        return seq[keep].copy()
    parts = []
    last = 0
    for p in sorted(inserts):
        parts.append(seq[last:p][keep[last:p]])
        parts.append(inserts[p])
        last = p
    parts.append(seq[last:][keep[last:]])
    return np.concatenate(parts).astype(np.uint8)


@dataclass
class Workload:
    name: str
    scoring: Scoring
    triplets: list            # list of (s0, s1, s2) uint8 code arrays
    traceback: bool
    meta: dict = field(default_factory=dict)

    @property
    def cells(self) -> int:
        """The paper's cell count: sum over triplets of |S0|*|S1|*|S2|."""
        return int(sum(len(a) * len(b) * len(c) for a, b, c in self.triplets))


def related_triplet(seed: int, idx: int, L: int, sc: Scoring, p_sub: float, p_indel: float,
                    mean_len: float):
    anc = random_seq(stream_key(seed, idx, 0xA), L, sc.freqs)
    return tuple(mutate(stream_key(seed, idx, q), anc, p_sub, p_indel, mean_len, sc.freqs)
                 for q in range(3))


def config0(seed: int = 1000) -> Workload:
    """Three independent uniform ACGT sequences of length 128; score + traceback."""
    sc = dna_scoring()
    t = tuple(random_seq(stream_key(seed, 0, q), 128, sc.freqs) for q in range(3))
    return Workload("dna_128_independent", sc, [t], True)


def config1(seed: int = 1001, L: int = 1000) -> Workload:
    """Related DNA triplet: ancestor length 1000, descendants 5% subs, 2% indels (mean 2)."""
    sc = dna_scoring()
    return Workload(f"dna_related_{L}", sc,
                    [related_triplet(seed, 0, L, sc, 0.05, 0.02, 2.0)], True)


def config2(seed: int = 1002, n: int = 4096, lo: int = 100, hi: int = 300) -> Workload:
    """Batch of related DNA triplets, ancestor lengths uniform in [100, 300]; score only."""
    sc = dna_scoring()
    lens = lo + (draws_u64(stream_key(seed, 0xB), np.arange(n)) %
                 np.uint64(hi - lo + 1)).astype(np.int64)
    trip = [related_triplet(seed, i, int(lens[i]), sc, 0.05, 0.02, 2.0) for i in range(n)]
    return Workload(f"dna_batch_{n}_{lo}_{hi}", sc, trip, False)


def config3(seed: int = 1003, L: int = 4000) -> Workload:
    """Large protein triplet: ancestor 4000, 15% subs, 3% indels (mean 3); score only."""
    sc = protein_scoring(seed)
    return Workload(f"protein_related_{L}", sc,
                    [related_triplet(seed, 0, L, sc, 0.15, 0.03, 3.0)], False)


def config4(seed: int = 1004, n: int = 10000, lo: int = 50, hi: int = 2000,
            mu: float = math.log(300.0), sdev: float = 0.8):
    """Serving stream: 70% DNA / 30% protein requests, ancestor length lognormal(mu, sdev)
    clipped to [50, 2000], 20% ask for traceback, unit-rate Poisson inter-arrival gaps (scale by
    1/lambda). Returns (dna_scoring, protein_scoring, requests) with each request a dict."""
    dna = dna_scoring()
    prot = protein_scoring(seed)
    key = stream_key(seed, 0xC)
    idx = np.arange(n, dtype=np.uint64)
    u_kind = uniform(key, idx * np.uint64(8))
    u1 = np.maximum(uniform(key, idx * np.uint64(8) + np.uint64(1)), 1e-300)
    u2 = uniform(key, idx * np.uint64(8) + np.uint64(2))
    u_tb = uniform(key, idx * np.uint64(8) + np.uint64(3))
    u_arr = np.maximum(uniform(key, idx * np.uint64(8) + np.uint64(4)), 1e-300)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)  # Box-Muller normal
    L = np.clip(np.round(np.exp(mu + sdev * z)), lo, hi).astype(np.int64)
    gaps = -np.log(u_arr)
    reqs = []
    for i in range(n):
        protein = bool(u_kind[i] >= 0.7)
        sc = prot if protein else dna
        if protein:
            trip = related_triplet(seed, i, int(L[i]), sc, 0.15, 0.03, 3.0)
        else:
            trip = related_triplet(seed, i, int(L[i]), sc, 0.05, 0.02, 2.0)
        reqs.append({"id": i, "protein": protein, "triplet": trip,
                     "traceback": bool(u_tb[i] < 0.2), "gap": float(gaps[i])})
    return dna, prot, reqs


def to_str(codes: np.ndarray, alphabet: str) -> str:
    table = np.frombuffer(alphabet.encode(), dtype=np.uint8)
    return table[np.asarray(codes, dtype=np.int64)].tobytes().decode()
