"""Statistics of the random bits that drive stochastic rounding of the 16-bit
stores, from a numpy restatement of the device generator: the counter-based
pair hash (a mix of the site pair and a key drawn from the step number) and
the per-direction word (the hash times an odd constant per direction, high
half folded into the low one).

The rounding is unbiased when every dropped-bit pattern is equally likely
and the bits of different stores are independent: FP16 uses the low 13 bits
of each half of a word, BF16 all 16.  Checked over 2^20 site pairs, nine
directions and three steps: uniform fields (chi^2 per degree of freedom over
256 bins), no correlation between directions, between the two halves of a
word or between steps beyond the sampling scale 1/sqrt(N), and no bias in
the mean.  The effect on the simulation (the decay that round-to-nearest
freezes, recovered without bias) is checked on the GPU in
test_gpu_precision.py."""
import numpy as np

M32 = np.uint64(0xFFFFFFFF)


def _mix32(x):
    x = x.astype(np.uint64)
    x ^= x >> np.uint64(16)
    x = (x * np.uint64(0x7FEB352D)) & M32
    x ^= x >> np.uint64(15)
    x = (x * np.uint64(0x846CA68B)) & M32
    x ^= x >> np.uint64(16)
    return x


def _step_key(step):
    return _mix32(np.array([(step * 0x9E3779B9 + 0x632BE5AB) & 0xFFFFFFFF], np.uint64))[0]


def _words(pairs, step):
    """[9, n] direction words of site pairs `pairs` at `step`."""
    base = _mix32(pairs.astype(np.uint64) ^ _step_key(step))
    out = []
    for i in range(9):
        c = np.uint64((0x9E3779B9 + 2 * i * 0x6A09E667) & 0xFFFFFFFF)
        x = (base * c) & M32
        out.append(x ^ (x >> np.uint64(16)))
    return np.stack(out)


def _fields(words, bits):
    lo = (words & np.uint64(0xFFFF)) & np.uint64((1 << bits) - 1)
    hi = (words >> np.uint64(16)) & np.uint64((1 << bits) - 1)
    return lo.astype(np.float64), hi.astype(np.float64)


def _chi2_per_dof(v, bits, bins=256):
    h = np.bincount((v.astype(np.int64) >> (bits - 8)), minlength=bins)
    e = v.size / bins
    return float(((h - e) ** 2 / e).sum() / (bins - 1))


def test_rounding_bits_uniform_and_independent():
    n = 1 << 20
    pairs = np.arange(n, dtype=np.uint64) * np.uint64(3) + np.uint64(12345)
    per_step = [_words(pairs, s) for s in (0, 1, 977)]
    tol_corr = 5.0 / np.sqrt(n)
    for bits in (13, 16):
        full = 1 << bits
        for w in per_step:
            lo, hi = _fields(w, bits)
            for i in range(9):
                for v in (lo[i], hi[i]):
                    assert _chi2_per_dof(v, bits) < 1.5
                    # mean of (r + 0.5)/2^bits is 1/2: no bias in the rounding
                    assert abs((v.mean() + 0.5) / full - 0.5) < 5 * np.sqrt(1 / 12 / n)
                assert abs(np.corrcoef(lo[i], hi[i])[0, 1]) < tol_corr
            for i in range(9):
                for j in range(i + 1, 9):
                    assert abs(np.corrcoef(lo[i], lo[j])[0, 1]) < tol_corr
                    assert abs(np.corrcoef(hi[i], hi[j])[0, 1]) < tol_corr
        a, _ = _fields(per_step[0], bits)
        b, _ = _fields(per_step[1], bits)
        for i in range(9):
            assert abs(np.corrcoef(a[i], b[i])[0, 1]) < tol_corr


def test_neighbouring_pairs_do_not_share_bits():
    """Adjacent site pairs (the lanes of one warp, the rows above and below)
    get unrelated words: no correlation between pair p and p + 1 or p + nx/2."""
    n = 1 << 18
    pairs = np.arange(n + 1024, dtype=np.uint64)
    w = _words(pairs, 5)
    lo, _ = _fields(w, 13)
    tol = 5.0 / np.sqrt(n)
    for d in (1, 2, 1024):
        for i in (0, 4, 8):
            assert abs(np.corrcoef(lo[i, :n], lo[i, d:n + d])[0, 1]) < tol
