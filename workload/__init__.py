"""Seeded synthetic inputs for the dense N x N FP64 product C = A.B.

This module is the only code shared by the oracle tests and the GPU path.
It holds random-number generation and nothing of the product's arithmetic.

The paper fills its matrices with an unspecified ``RAND()`` (Alg. 2 and
Alg. 4, Sec. 3.1).  The distributions here are the synthetic stand-ins for
that: uniform [0, 1), uniform [-1, 1), log-uniform magnitude with a random
sign, and small integers in {-8..8} whose products are exact in FP64.

The generator is counter based: draw ``i`` of stream ``seed`` is
SplitMix64 (Steele, Lea, Flood 2014) evaluated at ``seed + (i + 1) * gamma``,
so any element can be reproduced without generating the ones before it.
"""
from __future__ import annotations

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
# Stream offset separating B from A for the same seed.
B_STREAM_OFFSET = 0x5851F42D4C957F2D
# Stream offset for the sign bits of log-uniform entries.
SIGN_STREAM_OFFSET = 0x2545F4914F6CDD1D

DISTRIBUTIONS = ("uniform01", "uniform11", "loguniform20", "int8")


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Draws ``start .. start+count-1`` of the SplitMix64 stream ``seed``."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix64_torch(seed: int, count: int, device):
    """The same draws as splitmix64 (start 0), generated by PyTorch on `device`
    as int64 bit patterns (wrapping multiplication, logical right shifts)."""
    import torch
    def s64(v):  # a uint64 constant as the int64 with the same bits
        v &= 0xFFFFFFFFFFFFFFFF
        return v - (1 << 64) if v >= 1 << 63 else v
    def srl(z, k):
        return (z >> k) & ((1 << (64 - k)) - 1)
    idx = torch.arange(1, count + 1, dtype=torch.int64, device=device)
    z = idx * s64(int(GOLDEN_GAMMA)) + s64(seed)
    z = (z ^ srl(z, 30)) * s64(int(_M1))
    z = (z ^ srl(z, 27)) * s64(int(_M2))
    return z ^ srl(z, 31)


def values_torch(dist: str, seed: int, count: int, device):
    """values() generated on a PyTorch device (uniform01 and loguniform20),
    equal to the host's draws up to the last bit of exp2 (exact for uniform01)."""
    import torch
    u = (torch.bitwise_right_shift(splitmix64_torch(seed, count, device), 11) & ((1 << 53) - 1)).double() * 2.0 ** -53
    if dist == "uniform01":
        return u
    if dist == "loguniform20":
        mag = torch.exp2(-20.0 + 40.0 * u)
        sign = splitmix64_torch(seed + SIGN_STREAM_OFFSET, count, device) < 0  # top bit set
        return torch.where(sign, -mag, mag)
    raise ValueError(f"values_torch supports uniform01 and loguniform20, not {dist!r}")


def pair_torch(dist: str, seed: int, n: int, device):
    """pair() generated on a PyTorch device (see values_torch)."""
    A = values_torch(dist, seed, n * n, device).reshape(n, n)
    B = values_torch(dist, seed + B_STREAM_OFFSET, n * n, device).reshape(n, n)
    return A, B


def uniform01(seed: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1): the top 53 bits of each draw times 2^-53."""
    z = splitmix64(seed, count)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def values(dist: str, seed: int, count: int) -> np.ndarray:
    """``count`` FP64 values of distribution ``dist`` from stream ``seed``."""
    if dist == "uniform01":
        return uniform01(seed, count)
    if dist == "uniform11":
        return 2.0 * uniform01(seed, count) - 1.0
    if dist == "loguniform20":
        u = uniform01(seed, count)
        mag = np.exp2(-20.0 + 40.0 * u)
        sign = (splitmix64(seed + SIGN_STREAM_OFFSET, count) >> np.uint64(63)).astype(np.int64)
        return np.where(sign == 1, -mag, mag)
    if dist == "int8":
        z = splitmix64(seed, count)
        return ((z % np.uint64(17)).astype(np.int64) - 8).astype(np.float64)
    raise ValueError(f"unknown distribution {dist!r}; expected one of {DISTRIBUTIONS}")


def matrix(dist: str, seed: int, n: int, which: str = "A") -> np.ndarray:
    """Row-major n x n FP64 matrix; ``which`` = "A" or "B" selects the stream."""
    s = seed if which == "A" else seed + B_STREAM_OFFSET
    return np.ascontiguousarray(values(dist, s, n * n).reshape(n, n))


def pair(dist: str, seed: int, n: int) -> tuple[np.ndarray, np.ndarray]:
    """The (A, B) operand pair of one product."""
    return matrix(dist, seed, n, "A"), matrix(dist, seed, n, "B")


def rect_pair(dist: str, seed: int, m: int, n: int, k: int) -> tuple[np.ndarray, np.ndarray]:
    """Operands of a rectangular product: A (m x k) and B (k x n), row-major,
    from the same streams as pair() (m = n = k gives pair()'s matrices)."""
    A = np.ascontiguousarray(values(dist, seed, m * k).reshape(m, k))
    B = np.ascontiguousarray(values(dist, seed + B_STREAM_OFFSET, k * n).reshape(k, n))
    return A, B


STRUCTURES = ("split_scales", "wide60", "outlier_column")


def structured_pair(kind: str, seed: int, n: int) -> tuple[np.ndarray, np.ndarray]:
    """Operand pairs whose rows and columns mix magnitudes far apart: the
    inputs on which an emulation that scales each row of A and column of B by
    its maximum loses accuracy relative to |A||B|.

    split_scales   a_i0 = u, a_ij = 2^-30 u (j > 0); b_0k = 2^-30 u, b_jk = u
                   (j > 0): each row's large entry meets the small ones of B,
                   and the reverse, so every c_ik is a sum of small terms
    wide60         entries of magnitude 2^U(-60, 60), random signs
    outlier_column uniform [-1, 1) with the first column of A scaled by 2^40
    (u uniform [1/2, 1) from stream ``seed``; B from the offset stream.)"""
    if kind == "wide60":
        def draw(s):
            u = uniform01(s, n * n)
            sign = (splitmix64(s + SIGN_STREAM_OFFSET, n * n) >> np.uint64(63)).astype(np.int64)
            mag = np.exp2(-60.0 + 120.0 * u)
            return np.where(sign == 1, -mag, mag).reshape(n, n)
        return np.ascontiguousarray(draw(seed)), np.ascontiguousarray(draw(seed + B_STREAM_OFFSET))
    if kind == "split_scales":
        A = (0.5 + 0.5 * uniform01(seed, n * n)).reshape(n, n) * 2.0 ** -30
        B = (0.5 + 0.5 * uniform01(seed + B_STREAM_OFFSET, n * n)).reshape(n, n)
        A[:, 0] *= 2.0 ** 30
        B[0, :] *= 2.0 ** -30
        return np.ascontiguousarray(A), np.ascontiguousarray(B)
    if kind == "outlier_column":
        A, B = pair("uniform11", seed, n)
        A[:, 0] *= 2.0 ** 40
        return A, B
    raise ValueError(f"unknown structure {kind!r}; expected one of {STRUCTURES}")


def loguniform_sizes(count: int, lo: int, hi: int, seed: int) -> list[int]:
    """``count`` sizes N log-uniform over the integers [lo, hi].

    N = clamp(floor(exp(ln lo + u (ln(hi + 1) - ln lo))), lo, hi), u uniform [0, 1).
    """
    u = uniform01(seed, count)
    n = np.floor(np.exp(np.log(lo) + u * (np.log(hi + 1.0) - np.log(lo)))).astype(np.int64)
    return [int(x) for x in np.clip(n, lo, hi)]


def batch(dist: str, seed: int, sizes: list[int]) -> list[tuple[np.ndarray, np.ndarray]]:
    """Operand pairs for a batch; problem p uses stream ``seed * 1000003 + p``."""
    return [pair(dist, seed * 1000003 + p, n) for p, n in enumerate(sizes)]


# Workloads by name.  Sizes follow the paper's sweep (N from 10 to 2000,
# Sec. 1.1 and Tables 1-3) and its larger extensions.
SWEEP_SIZES = (10, 100, 500, 1000, 1500, 2000)
PRECISION_SIZES = (2000, 4096, 8192)


def flops(n: int) -> int:
    """The paper's operation count for one N x N product: N^2 (2N - 1) = 2N^3 - N^2."""
    return 2 * n ** 3 - n ** 2
