"""The arithmetic behind the paired 64-bit reductions of the projection
kernel's segment-end flush, checked in exact integers on the CPU.

Two neighbouring image pixels at an 8-byte aligned address form one 64-bit
word (low word: the pixel at the aligned address).  The flush adds a pair
with one 64-bit addition while other code adds single pixels with 32-bit
additions that do not carry.  That is exact when the low word never leaves
[0, 2^32) in any order of the additions:
- unsigned integer images: every partial sum of a pixel lies between 0 and
  its final value, which is below 2^32;
- signed limb images (partial sums of magnitude below 2^30): the low word
  starts at the bias 2^31 and the low half of a pair addition is
  sign-extended.
"""
import random

M32, M64 = 1 << 32, 1 << 64
BIAS = 1 << 31


def run(contribs, bias, sign_extend, rng):
    """Apply (kind, lo, hi) additions in a random order to one pair word:
    kind 'pair' adds hi * 2^32 + lo as 64 bits, 'lo' / 'hi' add 32 bits to
    one half without carry.  Returns the decoded (lo, hi) as int32."""
    word = bias
    order = contribs[:]
    rng.shuffle(order)
    for kind, lo, hi in order:
        if kind == "pair":
            # the low half sign-extended to 64 bits (limb images) or not
            add = ((hi % M32) << 32) + (lo % M64 if sign_extend else lo % M32)
            word = (word + add) % M64
        elif kind == "lo":
            word = (word & ~(M32 - 1)) | (((word & (M32 - 1)) + lo) % M32)
        else:
            word = (word + ((hi % M32) << 32)) % M64
    lo_w, hi_w = word & (M32 - 1), word >> 32
    lo_v = (lo_w - bias) % M32
    to_i32 = lambda u: u - M32 if u >= 1 << 31 else u
    return to_i32(lo_v), to_i32(hi_w), lo_w


def contributions(rng, n, signed, cap):
    out = []
    for _ in range(n):
        kind = rng.choice(["pair", "lo", "hi"])
        lo = rng.randint(-cap, cap) if signed else rng.randint(0, cap)
        hi = rng.randint(-cap, cap) if signed else rng.randint(0, cap)
        out.append((kind, lo if kind != "hi" else 0, hi if kind != "lo" else 0))
    return out


def test_unsigned_pairs_never_carry():
    rng = random.Random(1)
    for _ in range(300):
        c = contributions(rng, rng.randint(1, 40), False, (M32 - 1) // 64)
        lo_sum = sum(x[1] for x in c)
        hi_sum = sum(x[2] for x in c)
        assert lo_sum < M32 and hi_sum < M32
        lo, hi, _ = run(c, 0, False, rng)
        assert lo % M32 == lo_sum % M32 and hi % M32 == hi_sum % M32


def test_signed_limb_pairs_with_bias():
    rng = random.Random(2)
    for _ in range(300):
        n = rng.randint(1, 40)
        c = contributions(rng, n, True, (1 << 30) // 64)
        lo_sum = sum(x[1] for x in c)
        hi_sum = sum(x[2] for x in c)
        lo, hi, lo_w = run(c, BIAS, True, rng)
        assert lo == lo_sum and hi == hi_sum
        assert 0 <= lo_w < M32


def test_signed_pairs_without_bias_go_wrong():
    """Without the bias a negative partial sum in the low word borrows from
    the high word: the scheme needs it."""
    rng = random.Random(3)
    c = [("pair", -5, 7), ("lo", 3, 0), ("hi", 0, 1)]
    lo, hi, _ = run(c, 0, True, rng)
    assert lo == -2
    assert hi != 8


def run_ops(W, o, lo, hi):
    """The reductions the projection kernel's red_add_run issues for window
    positions k of [lo, hi): ('pair', k) adds k and k + 1 with one 64-bit
    reduction (p + k 8-byte aligned, i.e. k + o even), ('one', k) a single
    pixel.  o = 1 when the run's first pixel is the high word of a pair."""
    ops = []
    inside = lambda k: lo <= k < hi
    if o == 1 and inside(0):
        ops.append(("one", 0))
    for k in range(o, W - 1, 2):
        if inside(k) and inside(k + 1):
            ops.append(("pair", k))
        else:
            ops += [("one", j) for j in (k, k + 1) if inside(j)]
    if (W - o) % 2 == 1 and inside(W - 1):
        ops.append(("one", W - 1))
    return ops


def test_runs_add_each_position_once_and_pair_only_aligned_words():
    for W in (4, 8):
        for o in (0, 1):
            for lo in range(-2, W + 2):
                for hi in range(lo, W + 3):
                    seen = []
                    for kind, k in run_ops(W, o, lo, hi):
                        if kind == "pair":
                            assert (k + o) % 2 == 0 and k + 1 < W
                            seen += [k, k + 1]
                        else:
                            seen.append(k)
                    want = [k for k in range(W) if lo <= k < hi]
                    assert sorted(seen) == want, (W, o, lo, hi)
