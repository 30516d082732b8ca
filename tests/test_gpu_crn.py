"""GPU common random numbers against the oracle's independent Philox4x32-10, word by word.

The filter kernels draw every random number from Philox4x32-10 (Salmon et al., SC'11) with
the key (seed_lo ^ iteration, seed_hi ^ row) and the counter (t, call, stream, 0) (Sec. I:
one fixed stream of numbers per sample and iteration).  smc2_selftest_crn runs the kernels'
own key expansion, rounds, uniform map and Box-Muller pair; the words and uniforms must be
bit-identical to the oracle's, the normals equal within FP32 rounding of the same formula.
Covered: all five streams (propagation, resampling uniforms, initial state, outer normals,
outer uniform), the batched systematic draw of 32 steps (counters (t + lane, 0, 1, 0)), the
multinomial uniforms (call i / 4, word i % 4), large counters and keys with high bits set.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

SEEDS = [12345, 777, (0xDEADBEEF << 32) | 0x01234567, 2 ** 64 - 1]


def _cases():
    rng = np.random.default_rng(5)
    ctr, key = [], []
    for seed in SEEDS:
        lo, hi = seed & 0xFFFFFFFF, seed >> 32
        for it, row in [(1, 0), (2, 1023), (7, 4095), (0xFFFFFFFF, 0x80000000)]:
            for stream in range(5):
                # t in the filters' range, calls of up to 16 normals a particle (d_x = 16)
                for t in list(range(0, 40)) + [250, 499, 1000]:
                    for call in (0, 1, 2, 255, 511, 4095):
                        ctr.append((t, call, stream, 0))
                        key.append((lo, hi, it, row))
            # the 32-step batched systematic draw: lane l takes counter (t + l, 0, 1, 0)
            for t0 in (1, 33, 225):
                for lane in range(32):
                    ctr.append((t0 + lane, 0, 1, 0))
                    key.append((lo, hi, it, row))
    # random counters and keys over the whole 32-bit range
    for _ in range(2000):
        ctr.append(tuple(int(v) for v in rng.integers(0, 2 ** 32, 4, dtype=np.uint64)))
        key.append(tuple(int(v) for v in rng.integers(0, 2 ** 32, 4, dtype=np.uint64)))
    return np.array(ctr, dtype=np.uint64).astype(np.uint32), np.array(key, dtype=np.uint64).astype(np.uint32)


def test_philox_words_and_uniforms_bit_exact():
    from paper_2407_17296_gb300 import binding
    ctr, key = _cases()
    out = binding.selftest_crn(ctr, key)
    words, u = out["words"], out["u"]
    assert len(words) > 10000
    for i in range(len(ctr)):
        ref = oracle.philox4x32_10(ctr[i], (int(key[i][0]) ^ int(key[i][2]), int(key[i][1]) ^ int(key[i][3])))
        assert list(words[i]) == ref, (i, ctr[i], key[i], list(words[i]), ref)
    # the map to (0, 1]: ((w >> 8) + 1) 2^-24, exact in FP32
    expect = ((words.astype(np.uint64) >> 8) + 1).astype(np.float64) * 2.0 ** -24
    np.testing.assert_array_equal(u.astype(np.float64), expect)


def test_normals_match_oracle_streams():
    """Box-Muller normals of the filters' streams: GPU FP32 against the oracle's FP64 draw of
    the same counters, including the multinomial uniforms of stream 1."""
    from paper_2407_17296_gb300 import binding
    worst = 0.0
    for seed in SEEDS[:3]:
        lo, hi = seed & 0xFFFFFFFF, seed >> 32
        for it, row in [(1, 0), (3, 517)]:
            for stream in (0, 2, 3):
                for t in (0, 1, 17, 250):
                    n_calls = 64
                    ctr = np.array([(t, c, stream, 0) for c in range(n_calls)], dtype=np.uint32)
                    key = np.array([(lo, hi, it, row)] * n_calls, dtype=np.uint32)
                    z = binding.selftest_crn(ctr, key, want=("z",))["z"].reshape(-1).astype(np.float64)
                    ref = oracle.normals(seed, it, row, t, stream, 4 * n_calls)
                    err = np.abs(z - ref) / np.maximum(1.0, np.abs(ref))
                    worst = max(worst, float(err.max()))
            # multinomial uniforms before step t: particle i -> call i/4, word i%4
            t = 9
            ctr = np.array([(t, c, 1, 0) for c in range(32)], dtype=np.uint32)
            key = np.array([(lo, hi, it, row)] * 32, dtype=np.uint32)
            u = binding.selftest_crn(ctr, key, want=("u",))["u"].reshape(-1)
            for i in range(128):
                assert float(u[i]) == oracle.uniform_open(seed, it, row, t, 1, call=i // 4, word=i % 4)
    # FP32 Box-Muller against FP64: the angle 2 pi U - pi is rounded to FP32 (3.7e-7 at pi) and
    # the hardware sine/cosine add ~2^-21 absolute; times a radius of at most 5.8 (U >= 2^-24)
    assert worst < 1e-5, worst
    print(f"\n[crn normals] largest |z_gpu - z_oracle| / max(1, |z|) = {worst:.2e}")
