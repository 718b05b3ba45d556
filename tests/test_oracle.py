"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself:
  * brute force from Eq. 1's element relations (Sec. 2.1) on tiny square matrices;
  * a schoolbook carry-less polynomial product, taking coefficients n-1 .. n+m-2
    (the coefficient selection of Step 3, Sec. 3, read 0-based with l for k);
  * linearity in the key and in the seed; the Toeplitz shift T[i+1][j+1] = T[i][j];
  * closed forms (single-bit seed or key, all-ones seed, n = 1, m = 1);
  * the XOR merge of any p x q split equals the unsplit hash (Eq. finalkey).
"""
import numpy as np
import pytest

from paper_1805_02372_gb300 import inputs

RNG = np.random.default_rng(12345)


def rand_bits(k):
    return RNG.integers(0, 2, size=k, dtype=np.uint8)


def oracle_bits(o, n, m, s_bits, x_bits, threads=None):
    return o.unpack(o.hash_full(n, m, o.pack(s_bits), o.pack(x_bits), threads=threads), m)


def to_int(bits):
    v = 0
    for i in np.flatnonzero(bits):
        v |= 1 << int(i)
    return v


def clmul(a, b):
    """Carry-less product of two non-negative ints (schoolbook, XOR of shifts)."""
    acc = 0
    j = 0
    while b:
        if b & 1:
            acc ^= a << j
        b >>= 1
        j += 1
    return acc


def eq1_matrix(t):
    """Square T from Eq. 1 literally: t_{i-j} on/below the diagonal, t_{j-i+n-1} above."""
    n = (len(t) + 1) // 2
    T = np.zeros((n, n), dtype=np.uint8)
    for i in range(n):
        for j in range(n):
            T[i, j] = t[i - j] if i >= j else t[j - i + n - 1]
    return T


@pytest.mark.parametrize("n", [1, 2, 3, 7, 16, 33, 64])
def test_eq1_bruteforce(oracle, n):
    t = rand_bits(2 * n - 1)
    T = eq1_matrix(t)
    # The printed matrix: first column t_0..t_{n-1}, first row t_0, t_n, ..., t_{2n-2}.
    assert list(T[:, 0]) == list(t[:n])
    assert list(T[0, 1:]) == list(t[n:])
    # Diagonal-constant.
    assert np.array_equal(T[1:, 1:], T[:-1, :-1])
    x = rand_bits(n)
    want = (T.astype(np.int64) @ x.astype(np.int64)) % 2
    s = oracle.seed_from_eq1(t)
    got = oracle_bits(oracle, n, n, s, x)
    assert np.array_equal(got, want.astype(np.uint8))


@pytest.mark.parametrize("n,m", [(1, 1), (1, 9), (9, 1), (63, 64), (64, 63), (65, 130),
                                 (1000, 333), (4097, 2049), (3000, 7000), (12345, 777)])
def test_schoolbook_carryless_product(oracle, n, m):
    x = rand_bits(n)
    s = rand_bits(n + m - 1)
    c = clmul(to_int(s), to_int(x))
    want = np.array([(c >> (n - 1 + i)) & 1 for i in range(m)], dtype=np.uint8)
    assert np.array_equal(oracle_bits(oracle, n, m, s, x), want)


@pytest.mark.parametrize("n,m", [(5, 4), (40, 23), (130, 70)])
def test_explicit_matrix_and_bitloop(oracle, n, m):
    x = rand_bits(n)
    s = rand_bits(n + m - 1)
    want = oracle.hash_explicit(n, m, s, x)
    assert np.array_equal(oracle_bits(oracle, n, m, s, x), want)
    rows = np.arange(m)
    assert np.array_equal(oracle.hash_rows(n, m, oracle.pack(s), oracle.pack(x), rows,
                                           bitloop=True), want)


@pytest.mark.parametrize("n,m", [(777, 555), (2048, 64), (5001, 4999)])
def test_linearity(oracle, n, m):
    s1, s2 = rand_bits(n + m - 1), rand_bits(n + m - 1)
    x1, x2 = rand_bits(n), rand_bits(n)
    h = lambda s, x: oracle_bits(oracle, n, m, s, x)
    assert np.array_equal(h(s1, x1 ^ x2), h(s1, x1) ^ h(s1, x2))
    assert np.array_equal(h(s1 ^ s2, x1), h(s1, x1) ^ h(s2, x1))
    assert not h(s1, np.zeros(n, np.uint8)).any()


@pytest.mark.parametrize("n,m", [(100, 80), (1031, 517)])
def test_shift_invariance(oracle, n, m):
    # T[i+1][j+1] = T[i][j]: shifting the key up one place shifts the output.
    x = rand_bits(n)
    x[n - 1] = 0
    xs = np.zeros(n, np.uint8)
    xs[1:] = x[:-1]
    s = rand_bits(n + m - 1)
    y = oracle_bits(oracle, n, m, s, x)
    ys = oracle_bits(oracle, n, m, s, xs)
    assert np.array_equal(ys[1:], y[:-1])


def test_closed_forms(oracle):
    n, m = 300, 211
    x = rand_bits(n)
    # Seed with one set bit at n-1+t: y_i = x_{i-t} (zero out of range).
    for t in (-50, -1, 0, 3, 150):
        s = np.zeros(n + m - 1, np.uint8)
        s[n - 1 + t] = 1
        want = np.array([x[i - t] if 0 <= i - t < n else 0 for i in range(m)], np.uint8)
        assert np.array_equal(oracle_bits(oracle, n, m, s, x), want)
    # All-ones seed: every output bit is the parity of the key.
    s = np.ones(n + m - 1, np.uint8)
    assert np.all(oracle_bits(oracle, n, m, s, x) == (int(x.sum()) & 1))
    # Key with one set bit j: y = column j of T = s[n-1-j .. n-2-j+m].
    s = rand_bits(n + m - 1)
    for j in (0, 17, n - 1):
        e = np.zeros(n, np.uint8)
        e[j] = 1
        assert np.array_equal(oracle_bits(oracle, n, m, s, e), s[n - 1 - j:n - 1 - j + m])
    # n = 1: y_i = x_0 AND s_i.
    s1 = rand_bits(m)
    for x0 in (0, 1):
        assert np.array_equal(oracle_bits(oracle, 1, m, s1, np.array([x0], np.uint8)), s1 * x0)
    # m = 1: y_0 = parity of sum_j x_j s_{n-1-j}.
    sm = rand_bits(n)
    want = int(sum(int(x[j]) * int(sm[n - 1 - j]) for j in range(n)) & 1)
    assert oracle_bits(oracle, n, 1, sm, x)[0] == want


@pytest.mark.parametrize("n,m,p,q", [(1000, 700, 3, 2), (4099, 1025, 5, 4), (640, 64, 10, 1)])
def test_split_xor_merge(oracle, n, m, p, q):
    # Eq. finalkey: split the key into p blocks and the output into q ranges; each
    # piece is again a Toeplitz hash over a shifted seed window; XOR merges them.
    x = rand_bits(n)
    s = rand_bits(n + m - 1)
    full = oracle_bits(oracle, n, m, s, x)
    jcut = sorted(set([0, n] + list(RNG.integers(1, n, size=p - 1))))
    icut = sorted(set([0, m] + list(RNG.integers(1, m, size=q - 1))))
    merged = np.zeros(m, np.uint8)
    for a, b in zip(icut[:-1], icut[1:]):
        for j0, j1 in zip(jcut[:-1], jcut[1:]):
            n2, m2 = j1 - j0, b - a
            off = n - j1 + a
            sub = oracle_bits(oracle, n2, m2, s[off:off + n2 + m2 - 1], x[j0:j1])
            merged[a:b] ^= sub
    assert np.array_equal(merged, full)


def test_threads_rows_and_tails(oracle):
    blk = inputs.single_block(20011, 3001, 77, 78)
    key, seed = blk.key(), blk.seed()
    n, m = blk.n, blk.m
    y1 = oracle.hash_full(n, m, seed, key, threads=1)
    y7 = oracle.hash_full(n, m, seed, key, threads=7)
    assert np.array_equal(y1, y7)
    # Output tail beyond m is zero.
    assert (int(y1[-1]) >> (m % 64)) == 0
    rows = RNG.integers(0, m, size=200)
    assert np.array_equal(oracle.hash_rows(n, m, seed, key, rows), oracle.unpack(y1, m)[rows])
    assert np.array_equal(oracle.hash_rows(n, m, seed, key, rows[:20], bitloop=True),
                          oracle.unpack(y1, m)[rows[:20]])
    # Bits past n (key) and past n+m-1 (seed) are ignored.
    k2, s2 = key.copy(), seed.copy()
    k2[-1] ^= np.uint64(~((1 << (n % 64)) - 1) & 0xFFFFFFFFFFFFFFFF)
    s2[-1] ^= np.uint64(~((1 << ((n + m - 1) % 64)) - 1) & 0xFFFFFFFFFFFFFFFF)
    assert np.array_equal(oracle.hash_full(n, m, s2, k2), y1)


def test_invalid_arguments(oracle):
    z = np.zeros(4, np.uint64)
    with pytest.raises(ValueError):
        oracle.hash_full(0, 5, z, z)
    with pytest.raises(ValueError):
        oracle.hash_rows(10, 5, z, z, [5])


def test_generator_is_splitmix64():
    # Published SplitMix64 first outputs from state 0 (reference values of the
    # generator's public definition, computed here with Python integers).
    def ref(state, k):
        z = (state + k * 0x9E3779B97F4A7C15) & (2**64 - 1)
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & (2**64 - 1)
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & (2**64 - 1)
        return z ^ (z >> 31)
    got = inputs.splitmix64(0, 3)
    assert [int(v) for v in got] == [ref(0, k) for k in (1, 2, 3)]
    assert int(got[0]) == 0xE220A8397B1DCDAF
    blocks = inputs.batched_blocks()
    assert len(blocks) == 256
    assert all(100_000 <= b.n <= 4_000_000 and 1 <= b.m <= b.n // 2 for b in blocks)
