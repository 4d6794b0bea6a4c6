"""Digest of a pair set for the tests: (pairs, sum mod 2^64, xor) of
mix(r << 32 | s) over the pairs, mix being the output function of SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
2014), written here with numpy independently of the oracle's C version.  It
does not depend on the order of the pairs, so a GPU result of 1e9 pairs can be
compared with the oracle's digest chunk by chunk, without a sort."""
from __future__ import annotations

import numpy as np

_GOLD = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix(k: np.ndarray) -> np.ndarray:
    z = k.astype(np.uint64) + _GOLD              # numpy uint64 arithmetic wraps mod 2^64
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def digest(pairs) -> tuple[int, int, int]:
    """Digest of int32[n, 2] (r, s) rows."""
    a = np.asarray(pairs).reshape(-1, 2)
    k = (a[:, 0].astype(np.int64).astype(np.uint64) & np.uint64(0xFFFFFFFF)) << np.uint64(32)
    k |= a[:, 1].astype(np.int64).astype(np.uint64) & np.uint64(0xFFFFFFFF)
    h = mix(k)
    s = int(h.sum(dtype=np.uint64)) if len(h) else 0
    x = int(np.bitwise_xor.reduce(h)) if len(h) else 0
    return len(a), s, x


def combine(parts) -> tuple[int, int, int]:
    n, s, x = 0, 0, 0
    for pn, ps, px in parts:
        n += pn
        s = (s + ps) & 0xFFFFFFFFFFFFFFFF
        x ^= px
    return n, s, x


def digest_device(pairs, chunk: int = 1 << 24, threads: int = 8) -> tuple[int, int, int]:
    """Digest of a device tensor of pairs, copied to the host in chunks and
    digested by a few threads (numpy releases the GIL in its loops)."""
    from concurrent.futures import ThreadPoolExecutor

    starts = range(0, pairs.shape[0], chunk)
    with ThreadPoolExecutor(threads) as pool:
        parts = list(pool.map(lambda i: digest(pairs[i:i + chunk].cpu().numpy()), starts))
    return combine(parts)
