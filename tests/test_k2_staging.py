"""Index arithmetic of the step-2 kernel's shared-memory staging, checked on
the CPU: a CTA of 128 row segments copies the pixels from its first
segment's start to its last segment's end, pixel i at word i + i // seg.
For every image shape and CTA: the copied range holds each segment of the
CTA whole, the padded words stay inside the stage (128 * 64 + 128 words),
and with full segments the 32 lanes of a warp reading the i-th pixel of
their own segments hit 32 distinct banks."""
import random

UNITS = 128          # segments per CTA
SEG_MAX = 64         # pixels per segment at most
STAGE_WORDS = UNITS * SEG_MAX + UNITS


def cta_range(S, F, seg, chunk):
    nseg = (F + seg - 1) // seg
    units = S * nseg
    u_first = chunk * UNITS
    u_last = min(u_first + UNITS, units) - 1
    s0, sl = u_first // nseg, u_last // nseg
    gl = u_last - sl * nseg
    p0 = s0 * F + (u_first - s0 * nseg) * seg
    plen = sl * F + min((gl + 1) * seg, F) - p0
    segs = []
    for u in range(u_first, u_last + 1):
        s, g = divmod(u, nseg)
        fs = g * seg
        n = min(F - fs, seg)
        segs.append((s * F + fs - p0, n))
    return p0, plen, segs


def test_ranges_cover_segments_and_fit_the_stage():
    rng = random.Random(7)
    for _ in range(400):
        seg = rng.choice([32, 64])
        S, F = rng.randint(1, 300), rng.randint(1, 2100)
        nseg = (F + seg - 1) // seg
        nblk = (S * nseg + UNITS - 1) // UNITS
        for chunk in {0, nblk - 1, rng.randrange(nblk)}:
            p0, plen, segs = cta_range(S, F, seg, chunk)
            assert 0 < plen <= UNITS * seg
            last = plen - 1
            assert last + last // seg < STAGE_WORDS
            covered = [0] * plen
            for o, n in segs:
                assert 0 <= o and o + n <= plen and 1 <= n <= seg
                for i in range(o, o + n):
                    covered[i] += 1
            assert all(c == 1 for c in covered)   # contiguous, no overlap


def test_padding_spreads_full_segments_over_the_banks():
    for seg in (32, 64):
        for i in range(seg):
            banks = {((t * seg + i) + (t * seg + i) // seg) % 32 for t in range(32)}
            assert len(banks) == 32
