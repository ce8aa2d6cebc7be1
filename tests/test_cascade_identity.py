"""The identity behind the integer image-moment kernel, in exact integers.

Running A_0 += I_i, A_1 += A_0, ..., A_K += A_(K-1) over a row segment of n
pixels gives A_j = sum_i C(n-1-i+j, j) I_i.  With w = n - i, the power sums
sum_w w^b I are sum_j (-1)^(b-j) S(b,j) j! A_j (S: Stirling numbers of the
second kind), and the Pascal recurrence m_b += D m_(b-1), applied K times
to m_k = (-1)^k Q_k, yields sum (D - w)^b I, the power sums in the signed
coordinate c = f - off_f with D = f_start + n - off_f (Eq. 1 with the
origin shift of Sec. 5).  The kernel does all of it modulo 2^128; the test
does the same and compares with the direct sums, and checks that A_0..A_6,
which the kernel keeps in signed 64-bit words, stay below 2^63 in magnitude
for segments of at most 64 pixels of 32-bit values (unsigned, or signed
limbs of magnitude at most 2^31).  The
batched kernel runs the same cascade over interleaved segments
(f = g, g + nseg, ...), scaling the Stirling step by (-nseg)^k, modulo 2^64
when the host's bound says the row power sums fit int64.
"""
import random
from math import comb, factorial

M128 = 1 << 128


def stirling2(n, k):
    table = [[0] * (n + 1) for _ in range(n + 1)]
    table[0][0] = 1
    for i in range(1, n + 1):
        for j in range(1, i + 1):
            table[i][j] = j * table[i - 1][j] + table[i - 1][j - 1]
    return table[n][k]


def segment_power_sums(I, K, f_start, off_f):
    """The kernel's steps for one segment, modulo 2^128."""
    A = [0] * (K + 1)
    for v in I:
        A[0] = (A[0] + v) % M128
        for j in range(1, K + 1):
            A[j] = (A[j] + A[j - 1]) % M128
    m = []
    for b in range(K + 1):
        q = sum((-1) ** (b - j) * stirling2(b, j) * factorial(j) * A[j] for j in range(b + 1))
        m.append((-q if b & 1 else q) % M128)
    D = f_start + len(I) - off_f
    for i in range(1, K + 1):
        for b in range(K, i - 1, -1):
            m[b] = (m[b] + D * m[b - 1]) % M128
    return A, m


def test_cascade_matches_direct_power_sums():
    rng = random.Random(11)
    for _ in range(200):
        K = rng.randint(0, 8)
        n = rng.randint(1, 128)
        f_start = rng.randint(0, 4000)
        off_f = rng.randint(0, 4000)
        I = [rng.choice([0, rng.randint(0, 2**32 - 1)]) for _ in range(n)]
        A, F = segment_power_sums(I, K, f_start, off_f)
        for b in range(K + 1):
            direct = sum((f_start + i - off_f) ** b * v for i, v in enumerate(I))
            assert F[b] == direct % M128, (K, n, b)
        for j in range(K + 1):
            assert A[j] == sum(comb(n - 1 - i + j, j) * v for i, v in enumerate(I)) % M128


def test_low_cascade_sums_fit_64_bits():
    # worst case: 64 pixels, every pixel 2^32 - 1 (or -2^31 for a limb)
    for top in (2**32 - 1, 2**31):
        for j in range(7):
            assert top * comb(64 + j, j + 1) < 2**63
    assert (2**32 - 1) * comb(64 + 7, 8) >= 2**63  # A_7 needs the 128-bit path
    # the bound is the largest A_j: every pixel at the maximum
    for n in (1, 17, 64):
        A, _ = segment_power_sums([2**32 - 1] * n, 6, 0, 0)
        assert all(A[j] == (2**32 - 1) * comb(n + j, j + 1) for j in range(7))


def test_summed_segments_give_the_row():
    """Segments of one row add up to the row's power sums (the CTA sums them)."""
    rng = random.Random(5)
    K, F, off_f, seg = 6, 300, 150, 32
    row = [rng.randint(0, 10**6) for _ in range(F)]
    tot = [0] * (K + 1)
    for fs in range(0, F, seg):
        _, Fs = segment_power_sums(row[fs:fs + seg], K, fs, off_f)
        tot = [(a + b) % M128 for a, b in zip(tot, Fs)]
    for b in range(K + 1):
        assert tot[b] == sum((f - off_f) ** b * v for f, v in enumerate(row)) % M128


def strided_segment_power_sums(I_row, K, g, nseg, off_f, modulus):
    """The batched kernel's steps for the interleaved segment f = g, g + nseg,
    ... of one row: the same cascade over its n pixels, then the Stirling
    conversion scaled by (-nseg)^k (the coordinate is D - nseg w with
    D = g + nseg n - off_f) and the Pascal recurrence, modulo `modulus`."""
    pix = I_row[g::nseg]
    n = len(pix)
    A = [0] * (K + 1)
    for v in pix:
        A[0] = (A[0] + v) % modulus
        for j in range(1, K + 1):
            A[j] = (A[j] + A[j - 1]) % modulus
    m, sc = [], 1
    for b in range(K + 1):
        q = sum((-1) ** (b - j) * stirling2(b, j) * factorial(j) * A[j] for j in range(b + 1))
        m.append(q * sc % modulus)
        sc = sc * (-nseg) % modulus
    D = g + nseg * n - off_f
    for i in range(1, K + 1):
        for b in range(K, i - 1, -1):
            m[b] = (m[b] + D * m[b - 1]) % modulus
    return m


def test_interleaved_segments_modulo_2_64():
    """Interleaved segments (the batched moment stage) computed modulo 2^64
    give the exact power sums whenever those fit int64, and the nseg
    segments of a row add up to the row's power sums."""
    rng = random.Random(23)
    M64 = 1 << 64
    for _ in range(150):
        K = rng.randint(0, 8)
        F = rng.randint(1, 400)
        nseg = rng.randint(1, min(F, 24))
        off_f = rng.randint(0, F)
        row = [rng.choice([0, rng.randint(0, 65535)]) for _ in range(F)]
        tot = [0] * (K + 1)
        for g in range(nseg):
            Fs = strided_segment_power_sums(row, K, g, nseg, off_f, M64)
            for b in range(K + 1):
                direct = sum((f - off_f) ** b * row[f] for f in range(g, F, nseg))
                if abs(direct) < 2**63:
                    signed = Fs[b] - M64 if Fs[b] >= 2**63 else Fs[b]
                    assert signed == direct, (K, F, nseg, g, b)
                else:
                    assert Fs[b] == direct % M64
            tot = [(a + c) % M64 for a, c in zip(tot, Fs)]
        for b in range(K + 1):
            assert tot[b] == sum((f - off_f) ** b * v for f, v in enumerate(row)) % M64


def test_segment_numbers_fit_32_bits_at_the_largest_dimensions():
    """Step 2 divides segment numbers in 32 bits: even at the largest
    dimensions (65536 on every axis) and the shortest segments (16 pixels),
    every image has fewer than 2^31 row segments."""
    import oracle
    for k in range(11):
        S, F, _, _ = oracle.image_geometry(k, 65536, 65536, 65536)
        assert S * ((F + 15) // 16) < 2**31, k
