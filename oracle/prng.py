"""Counter-based random draws for the sketches (oracle side).

The paper's sparse embedding (Definition 2.1) needs, for every column of S, a
set of gamma distinct row indices drawn uniformly without replacement plus
independent signs. The paper fixes no generator; this module implements the
reading used by both sides of the parity test, each from the published
definitions (no code is shared with the CUDA path):

* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014). The generator seeded with
  ``seed`` returns, as its k-th output (k = 0, 1, ...),
  ``mix64(seed + (k + 1) * 0x9E3779B97F4A7C15 mod 2^64)``, where ``mix64`` is the
  finaliser  z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
  z *= 0x94D049BB133111EB; z ^= z >> 31  (all mod 2^64).
  Used here as a counter-based generator: the counter is
  ``k = (stream << 56) | (row << 8) | q`` with row < 2^48 and q < 256.
* A uniform integer in [0, m) is the high 64 bits of the 128-bit product u * m
  (multiply-shift; bias at most m / 2^64, no rejection loop).
* Floyd's algorithm (Bentley and Floyd, CACM 1987) draws gamma distinct values
  from {0, ..., s-1}: for t = s-gamma, ..., s-1 draw r uniform in {0, ..., t};
  keep r if it is new, else keep t. Draw q (q = t - (s - gamma)) uses counter q.
* After the gamma values are sorted ascending, the sign of the q-th smallest is
  negative iff the top bit of draw (stream + 1, row, q) is set.

Plain Python integers throughout: slow, but every step can be read against the
definitions above.
"""

from __future__ import annotations

MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


def mix64(z: int) -> int:
    """SplitMix64 output finaliser (the 'mix64' of Steele, Lea and Flood)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def splitmix64_output(seed: int, k: int) -> int:
    """The k-th output (k >= 0) of SplitMix64 seeded with ``seed``."""
    return mix64((seed + (k + 1) * GOLDEN_GAMMA) & MASK64)


def counter(stream: int, row: int, q: int) -> int:
    if not (0 <= stream < 256 and 0 <= row < (1 << 48) and 0 <= q < 256):
        raise ValueError("counter field out of range")
    return (stream << 56) | (row << 8) | q


def draw(seed: int, stream: int, row: int, q: int) -> int:
    return splitmix64_output(seed & MASK64, counter(stream, row, q))


def uniform_below(u: int, m: int) -> int:
    """Uniform integer in [0, m) from a 64-bit draw: floor(u * m / 2^64)."""
    return (u * m) >> 64


def floyd_sample(seed: int, stream: int, row: int, s: int, gamma: int) -> list[int]:
    """gamma distinct values of {0..s-1}, uniformly without replacement, sorted."""
    if not (1 <= gamma <= s):
        raise ValueError("need 1 <= gamma <= s")
    chosen: set[int] = set()
    for q, t in enumerate(range(s - gamma, s)):
        r = uniform_below(draw(seed, stream, row, q), t + 1)
        chosen.add(t if r in chosen else r)
    return sorted(chosen)


def signs_for_row(seed: int, stream: int, row: int, gamma: int) -> list[int]:
    """+1/-1 for the q-th smallest chosen index, q = 0..gamma-1."""
    return [-1 if (draw(seed, stream + 1, row, q) >> 63) else 1 for q in range(gamma)]
