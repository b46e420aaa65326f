"""Seeded synthetic inputs for the product C = A*B (holds none of the method's arithmetic).

This module is the only code that both the oracle-side checks and the GPU-side
calls consume: it makes the operands. It never touches the library or the
oracle.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used as a counter-based generator. With
GOLDEN = 0x9E3779B97F4A7C15 and all arithmetic modulo 2^64:

    mix(z)   = z1 ^ (z1 >> 31), where z0 = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
                                       z1 = (z0 ^ (z0 >> 27)) * 0x94D049BB133111EB
    base     = mix(seed + stream * GOLDEN)
    word(i)  = mix(base + (i + 1) * GOLDEN)
    unit(i)  = (word(i) >> 11) * 2^-53                  in [0, 1)
    sym(i)   = 2 * unit(i) - 1                           in [-1, 1), exact in double

Element (r, c) of a rows x cols matrix draws counter i = r * cols + c.
The library's device-side filler implements the same definition; the tests
check the two against each other bit for bit.

Workload recipes (the paper uses Box-Muller normal deviates from rand(),
Sec. IV; the benchmark configurations replace them with these):
  * uniform[-1, 1] entries                          -> ``uniform``
  * uniform[-1, 1] * 2^e, e an integer uniform on [-20, 20], one e per row of A
    (or per column of B)                            -> ``row_scaled`` / ``col_scaled``
  * dimensions log-uniform on [lo, hi]: round(exp(U(ln lo, ln hi)))
                                                    -> ``loguniform_dims``
  * the paper's Box-Muller transform on two unit draws (Sec. IV), with the
    first draw moved into (0, 1] so the logarithm is finite -> ``box_muller``
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_A = 1
STREAM_B = 2
STREAM_EXP_A = 3
STREAM_EXP_B = 4
STREAM_DIMS = 5
STREAM_ARRIVALS = 6
STREAM_CLASS = 7


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def words(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """word(i) for i in [start, start + count) as uint64."""
    with np.errstate(over="ignore"):
        base = _mix(np.array([(seed + stream * int(GOLDEN)) % (1 << 64)], dtype=np.uint64))[0]
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix(base + i * GOLDEN)


def sym_at(seed: int, stream: int, idx) -> np.ndarray:
    """sym(i) in [-1, 1) at arbitrary counters idx (uint64 array)."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        base = _mix(np.array([(seed + stream * int(GOLDEN)) % (1 << 64)], dtype=np.uint64))[0]
        w = _mix(base + (idx + np.uint64(1)) * GOLDEN)
    return 2.0 * ((w >> np.uint64(11)).astype(np.float64) * 2.0 ** -53) - 1.0


def slot_block(seed: int, stream: int, ld: int, rows: int, cols: int, row0: int = 0) -> np.ndarray:
    """Rows [row0, row0+rows) x columns [0, cols) of an ld x ld matrix filled by
    ``uniform(ld, ld, seed, stream)`` (element (r, c) draws counter r*ld + c)."""
    r = np.arange(row0, row0 + rows, dtype=np.uint64)[:, None]
    c = np.arange(cols, dtype=np.uint64)[None, :]
    return sym_at(seed, stream, r * np.uint64(ld) + c)


def unit(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """unit(i) in [0, 1)."""
    return (words(seed, stream, count, start) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def uniform(rows: int, cols: int, seed: int, stream: int) -> np.ndarray:
    """rows x cols matrix of sym(i) in [-1, 1), row-major counters."""
    u = unit(seed, stream, rows * cols)
    return (2.0 * u - 1.0).reshape(rows, cols)


def int_uniform(lo: int, hi: int, count: int, seed: int, stream: int) -> np.ndarray:
    """Integers uniform on [lo, hi]: lo + floor(unit * (hi - lo + 1))."""
    u = unit(seed, stream, count)
    return lo + np.floor(u * (hi - lo + 1)).astype(np.int64)


def row_scaled(m: int, k: int, seed: int, emin: int = -20, emax: int = 20) -> np.ndarray:
    """A with entries uniform[-1,1) * 2^(e_i), e_i uniform on [emin, emax] per row."""
    e = int_uniform(emin, emax, m, seed, STREAM_EXP_A)
    return np.ldexp(uniform(m, k, seed, STREAM_A), e[:, None])


def col_scaled(k: int, n: int, seed: int, emin: int = -20, emax: int = 20) -> np.ndarray:
    """B with entries uniform[-1,1) * 2^(f_j), f_j uniform on [emin, emax] per column."""
    f = int_uniform(emin, emax, n, seed, STREAM_EXP_B)
    return np.ldexp(uniform(k, n, seed, STREAM_B), f[None, :])


def loguniform_dims(count: int, lo: int, hi: int, seed: int, stream: int = STREAM_DIMS) -> np.ndarray:
    """round(exp(U(ln lo, ln hi))) as int64, clipped to [lo, hi]."""
    u = unit(seed, stream, count)
    v = np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))
    return np.clip(np.rint(v), lo, hi).astype(np.int64)


def box_muller(rows: int, cols: int, seed: int, stream: int) -> np.ndarray:
    """Normal deviates by the paper's Box-Muller transform (Sec. IV): from two
    unit draws u1, u2, z0 = sqrt(-2 ln u1) cos(2 pi u2), z1 = ... sin(...).
    Pairs (z0, z1) fill consecutive entries; u1 is taken as 1 - unit so it is
    never 0."""
    count = rows * cols
    pairs = (count + 1) // 2
    u = unit(seed, stream, 2 * pairs)
    u1 = 1.0 - u[0::2]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * pairs)
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:count].reshape(rows, cols)


def wide_spread(rows: int, cols: int, seed: int, stream: int, octaves: int = 16) -> np.ndarray:
    """Heavy spread within every row and column: sym(i) * 2^-g(i), with g(i) an
    integer uniform on [0, octaves] drawn from the stream after the values
    (counters rows*cols + i)."""
    v = uniform(rows, cols, seed, stream)
    g = np.floor(unit(seed, stream, rows * cols, rows * cols) * (octaves + 1)).astype(np.int64)
    return np.ldexp(v, -g.reshape(rows, cols))


def student_t3(rows: int, cols: int, seed: int, stream: int) -> np.ndarray:
    """Heavy-tailed deviates, Student's t with 3 degrees of freedom: z0 / sqrt((z1^2 + z2^2 + z3^2) / 3)
    from four Box-Muller normals of the stream (entry i takes normals 4i .. 4i+3)."""
    z = box_muller(4 * rows * cols, 1, seed, stream).reshape(rows * cols, 4)
    t = z[:, 0] / np.sqrt((z[:, 1] ** 2 + z[:, 2] ** 2 + z[:, 3] ** 2) / 3.0)
    return t.reshape(rows, cols)


def cauchy(rows: int, cols: int, seed: int, stream: int) -> np.ndarray:
    """Cauchy deviates (no finite mean): the ratio of two Box-Muller normals of the stream."""
    z = box_muller(2 * rows * cols, 1, seed, stream).reshape(rows * cols, 2)
    return (z[:, 0] / z[:, 1]).reshape(rows, cols)


def problem_set(count: int, lo: int, hi: int, seed: int):
    """(m, n, k) triples, each dimension log-uniform on [lo, hi] independently."""
    d = loguniform_dims(3 * count, lo, hi, seed)
    return d.reshape(count, 3)
