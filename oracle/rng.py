"""Oracle-side random draws for the sketch S and the norm-estimate vectors W.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper leaves the random number generator open (MATLAB's).  The project
defines one counter-based generator, implemented independently here and in the
CUDA library's host code:

* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15; output is the state
  passed through xor-shift/multiply rounds with 0xBF58476D1CE4E5B9 and
  0x94D049BB133111EB (shifts 30, 27, 31).
* Stream (t, i) of seed `seed` starts from state mix64(seed ^ (t << 56) ^ i)
  where mix64 is the SplitMix64 output function applied to a raw word.
  t = 1: sketch rows of column i; t = 2: sketch signs of column i;
  t = 3: Gaussian entry i of W (column-major index).
* Sketch column i (Definition of the sparse sign embedding, Section 5.1):
  xi distinct rows in [0, s), each drawn as ((z >> 32) * s) >> 32 from stream
  (1, i), redrawing a row already taken; sign k is +1 when bit 63 of the k-th
  draw of stream (2, i) is clear, else -1.  Entries are +-xi^(-1/2).
* W entry i: two draws z1, z2 of stream (3, i); u1 = ((z1 >> 11) + 1) 2^-53,
  u2 = (z2 >> 11) 2^-53; value sqrt(-2 log u1) cos(2 pi u2) (Box-Muller),
  evaluated with the C library's log/cos/sqrt (Python's math module).
"""
from __future__ import annotations

import math

import numpy as np

MASK = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def mix64(z: int) -> int:
    """SplitMix64 output function of a 64-bit word."""
    z &= MASK
    z = ((z ^ (z >> 30)) * _M1) & MASK
    z = ((z ^ (z >> 27)) * _M2) & MASK
    return z ^ (z >> 31)


def splitmix64_sequence(state: int, count: int) -> list[int]:
    """The first `count` outputs of SplitMix64 started from `state`."""
    out = []
    for _ in range(count):
        state = (state + GOLDEN) & MASK
        out.append(mix64(state))
    return out


def stream_state(seed: int, t: int, i: int) -> int:
    return mix64((seed & MASK) ^ ((t & 0xFF) << 56) ^ (i & ((1 << 56) - 1)))


# ---- vectorised forms (numpy uint64 arithmetic wraps modulo 2^64) ----------------

def _mix64_np(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= np.uint64(_M1)
    z ^= z >> np.uint64(27)
    z *= np.uint64(_M2)
    z ^= z >> np.uint64(31)
    return z


def _stream_state_np(seed: int, t: int, idx: np.ndarray) -> np.ndarray:
    base = np.uint64((seed & MASK) ^ ((t & 0xFF) << 56))
    return _mix64_np(base ^ (idx.astype(np.uint64) & np.uint64((1 << 56) - 1)))


def sparse_sign(seed: int, s: int, m: int, xi: int) -> tuple[np.ndarray, np.ndarray]:
    """Rows (m, xi) int32 and signs (m, xi) int8 of the s x m sparse sign embedding."""
    if not 1 <= xi <= s:
        raise ValueError("need 1 <= xi <= s")
    idx = np.arange(m, dtype=np.uint64)
    state = _stream_state_np(seed, 1, idx)
    rows = np.full((m, xi), -1, dtype=np.int64)
    count = np.zeros(m, dtype=np.int64)
    active = np.arange(m)
    while active.size:
        state[active] += np.uint64(GOLDEN)
        z = _mix64_np(state[active])
        r = ((z >> np.uint64(32)) * np.uint64(s)) >> np.uint64(32)
        r = r.astype(np.int64)
        taken = np.any(rows[active] == r[:, None], axis=1)
        ok = ~taken
        a_ok = active[ok]
        rows[a_ok, count[a_ok]] = r[ok]
        count[a_ok] += 1
        active = active[count[active] < xi]
    sstate = _stream_state_np(seed, 2, idx)
    signs = np.empty((m, xi), dtype=np.int8)
    for k in range(xi):
        sstate += np.uint64(GOLDEN)
        z = _mix64_np(sstate)
        signs[:, k] = np.where((z >> np.uint64(63)) == 0, 1, -1)
    return rows.astype(np.int32), signs


def gaussian_w(seed: int, n: int, r: int) -> np.ndarray:
    """n x r standard Gaussian matrix (float64), column-major entry order."""
    total = n * r
    st = _stream_state_np(seed, 3, np.arange(total, dtype=np.uint64))
    st1 = st + np.uint64(GOLDEN)
    st2 = st1 + np.uint64(GOLDEN)
    z1 = _mix64_np(st1)
    z2 = _mix64_np(st2)
    u1 = ((z1 >> np.uint64(11)) + np.uint64(1)).astype(np.float64) * 2.0 ** -53
    u2 = (z2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    two_pi = 2.0 * math.pi
    # the C library's scalar log/cos (numpy's vector kernels may round differently)
    vals = np.fromiter((math.sqrt(-2.0 * math.log(a)) * math.cos(two_pi * c)
                        for a, c in zip(u1.tolist(), u2.tolist())), dtype=np.float64, count=total)
    return vals.reshape(r, n).T.copy()


# ---- dense sketching operators (Appendix "Sketch comparison": Gaussian and SRFT) -------
# Stream layout, continuing the one above:
#   t = 4: entry (r, c) of the Gaussian sketch G (s x m), index c * s + r (column-major);
#          value from two draws by Box-Muller as for W; S = G / sqrt(s).
#   t = 5: sign d_c of column c of the subsampled randomized Hadamard transform (bit 63 of
#          the first draw of stream (5, c): clear +1, set -1);
#   t = 6: its s sampled rows of the m' x m' Hadamard matrix (m' = the power of two >= m),
#          drawn one after another from stream (6, 0) as ((z >> 32) * m') >> 32, a row
#          already taken drawn again; rows kept in draw order.


def _gaussian_entries(seed: int, t: int, total: int) -> np.ndarray:
    st = _stream_state_np(seed, t, np.arange(total, dtype=np.uint64))
    st1 = st + np.uint64(GOLDEN)
    st2 = st1 + np.uint64(GOLDEN)
    z1 = _mix64_np(st1)
    z2 = _mix64_np(st2)
    u1 = ((z1 >> np.uint64(11)) + np.uint64(1)).astype(np.float64) * 2.0 ** -53
    u2 = (z2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    two_pi = 2.0 * math.pi
    return np.fromiter((math.sqrt(-2.0 * math.log(a)) * math.cos(two_pi * c)
                        for a, c in zip(u1.tolist(), u2.tolist())), dtype=np.float64, count=total)


def gaussian_sketch(seed: int, s: int, m: int) -> np.ndarray:
    """The s x m Gaussian embedding G / sqrt(s), G i.i.d. N(0, 1)."""
    g = _gaussian_entries(seed, 4, s * m)
    return g.reshape(m, s).T / math.sqrt(s)


def srht_rows_signs(seed: int, s: int, m: int):
    """(sampled Hadamard rows (s,), column signs (m,)) of the SRHT of m columns."""
    mp = 1
    while mp < m:
        mp *= 2
    if s > mp:
        raise ValueError("need s <= the padded length")
    st = stream_state(seed, 6, 0)
    rows, taken = [], set()
    while len(rows) < s:
        st = (st + GOLDEN) & MASK
        p = ((mix64(st) >> 32) * mp) >> 32
        if p not in taken:
            taken.add(p)
            rows.append(p)
    sst = _stream_state_np(seed, 5, np.arange(m, dtype=np.uint64)) + np.uint64(GOLDEN)
    signs = np.where((_mix64_np(sst) >> np.uint64(63)) == 0, 1.0, -1.0)
    return np.array(rows, dtype=np.int64), signs


def srht_sketch(seed: int, s: int, m: int) -> np.ndarray:
    """The s x m subsampled randomized Hadamard transform (1 / sqrt(s)) R H D: row r holds
    (-1)^popcount(p_r & c) d_c / sqrt(s), p_r the sampled row of the unnormalised m' x m'
    Walsh-Hadamard matrix (its columns beyond m meet the zero padding of A)."""
    rows, d = srht_rows_signs(seed, s, m)
    c = np.arange(m, dtype=np.int64)
    par = np.zeros((s, m), dtype=np.int64)
    x = rows[:, None] & c[None, :]
    while np.any(x):
        par ^= x & 1
        x >>= 1
    return np.where(par == 0, 1.0, -1.0) * d[None, :] / math.sqrt(s)


def round_bf16(x) -> np.ndarray:
    """Round to bfloat16 (round to nearest, ties to even) after rounding to FP32, returned as
    float64: the rounding of the tensor-core sketch operands (FP64 values go to FP32 first)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    return (u.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


def bf16_pieces(x, k: int) -> list:
    """The k-term bfloat16 expansion of fp32(x): p_0 = bf16(f), p_j = bf16(f - p_0 - ... -
    p_{j-1}) with every difference taken in FP32 (exact: each residual has at most 24 - 8 j
    significant bits left).  Three terms represent an FP32 value exactly (barring underflow
    below 2^-126); returned as float64 arrays.  The operand representation of A in the
    tensor-core sketch."""
    r = np.asarray(x, dtype=np.float32).copy()
    out = []
    for _ in range(k):
        p = round_bf16(r)
        out.append(p)
        r = (r - p.astype(np.float32)).astype(np.float32)
    return out
