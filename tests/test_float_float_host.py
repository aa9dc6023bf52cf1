"""Host checks of the float-float state arithmetic of the mixed-precision path.

The mixed path keeps each state value as a pair (hi, lo) of FP32 numbers,
advanced by Knuth's TwoSum followed by Dekker's FastTwoSum renormalisation
(ff_add in csrc/fdcgks_kernels.cuh), and moves it through FP64 buffers with
split (hi = fl32(d), lo = fl32(d - hi)) and join (d = hi + lo in FP64) in
csrc/fdcgks_api.cu.  The adjoint of a mixed run replays the run through such
FP64 buffers, one step at a time.  These tests emulate that arithmetic with
numpy's separately rounded FP32 operations (the device code has no
multiplications there, so nothing is contracted into a fused multiply-add)
and pin what the replay keeps:

* a pair joined to FP64 and split again has the same FP64 value;
* its low part changes only where hi + lo needs more than 53 bits, that is,
  where lo lies far below the last bit of hi;
* a run replayed through FP64 buffers follows the unbroken run to FP64
  rounding (1e-13 relative is asserted; about 1e-14 is seen).
"""
import numpy as np

F32, F64 = np.float32, np.float64


def two_sum(a, b):
    s = (a + b).astype(F32)
    v = (s - a).astype(F32)
    e = ((a - (s - v).astype(F32)).astype(F32) + (b - v).astype(F32)).astype(F32)
    return s, e


def ff_add(hi, lo, b):
    s, e = two_sum(hi, b)
    e = (e + lo).astype(F32)
    h = (s + e).astype(F32)
    return h, (e - (h - s).astype(F32)).astype(F32)


def split(d):
    h = d.astype(F32)
    return h, (d - h.astype(F64)).astype(F32)


def join(h, lo):
    return h.astype(F64) + lo.astype(F64)


def _increments(rng, n):
    """FP32 increments of the sizes an S2O4 stage adds (1e-9 to 1e-2 of O(1)
    state values, either sign)."""
    return (rng.standard_normal(n) * 10.0 ** rng.uniform(-9, -2, n)).astype(F32)


def _pairs(n, seed, steps=5):
    rng = np.random.default_rng(seed)
    d = rng.uniform(0.5, 2.5, n) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    hi, lo = split(d)
    for _ in range(steps):
        hi, lo = ff_add(hi, lo, _increments(rng, n))
    return hi, lo


def test_fast_two_sum_pairs_are_normalised():
    """|lo| <= ulp(hi) / 2 for every pair the update produces."""
    hi, lo = _pairs(200_000, 1)
    ulp = np.spacing(np.abs(hi)).astype(F64)
    assert np.all(np.abs(lo.astype(F64)) <= 0.5 * ulp)


def test_join_then_split_keeps_the_fp64_value():
    hi, lo = _pairs(200_000, 2)
    d = join(hi, lo)
    h2, l2 = split(d)
    assert np.array_equal(h2, hi)
    assert np.array_equal(join(h2, l2), d)
    changed = l2 != lo
    # the low part changes only where it lies more than 29 bits below the
    # last bit of hi (hi + lo then needs more than 53 bits), and then by less
    # than 2^-53 of the value
    assert changed.any()
    ulp = np.spacing(np.abs(hi[changed])).astype(F64)
    assert np.all(np.abs(lo[changed].astype(F64)) < ulp * 2.0 ** -5)
    assert np.all(np.abs((l2 - lo)[changed].astype(F64)) <= np.abs(d[changed]) * 2.0 ** -53)


def test_replay_through_fp64_buffers_follows_the_unbroken_run():
    """Three pair additions per step (the stage accumulations), the replayed
    copy joined and split again after every step, 30 steps."""
    n = 400_000
    rng = np.random.default_rng(3)
    d = rng.uniform(0.5, 2.5, n) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    hi, lo = split(d)
    rh, rl = hi.copy(), lo.copy()
    lossy = 0
    for _ in range(30):
        for _ in range(3):
            b = _increments(rng, n)
            hi, lo = ff_add(hi, lo, b)
            rh, rl = ff_add(rh, rl, b)
        j = join(rh, rl)
        nh, nl = split(j)
        lossy += int(np.count_nonzero(nl != rl))
        rh, rl = nh, nl
    a, b = join(hi, lo), join(rh, rl)
    rel = np.abs(a - b) / np.abs(a)
    assert 0 < lossy < 0.01 * 30 * n
    assert rel.max() <= 1e-13
    assert np.mean(rel > 0) < 0.01
