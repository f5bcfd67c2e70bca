"""Pins for the oracle's Philox4x32-10 generator (Salmon et al., SC'11).

The oracle's generator is compared word for word with an independent
implementation (triton's ``tl.philox`` run in its CPU interpreter) over random
counters and keys, and its output is checked for the uniformity every use in
the method relies on (Metropolis acceptance, nearest-integer resampling).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _triton_available():
    try:
        import triton  # noqa: F401
        return True
    except Exception:
        return False


@pytest.mark.skipif(not _triton_available(), reason="triton not installed")
def test_philox_matches_independent_implementation(oracle_lib):
    rng = np.random.default_rng(12345)
    items = []
    # structured counters first: zero, all-ones, the counter shapes the method uses
    items.append([0, 0, 0, 0, 0, 0])
    items.append([0xFFFFFFFF] * 6)
    for _ in range(300):
        items.append([int(v) for v in rng.integers(0, 2 ** 32, size=6, dtype=np.uint64)])
    for h in range(8):
        for c in range(2):
            items.append([h, c, 5, 7, 0x1234, 0x2 << 28])
    proc = subprocess.run([sys.executable, os.path.join(HERE, "philox_triton_ref.py")],
                          input=json.dumps(items), capture_output=True, text=True, timeout=600)
    assert proc.returncode == 0, proc.stderr[-2000:]
    ref = json.loads(proc.stdout)
    for it, expect in zip(items, ref):
        got = oracle_lib.philox(it[:4], it[4:6])
        assert [int(x) for x in got] == expect, f"ctr={it[:4]} key={it[4:]}"


def test_philox_zero_counter_known_answer(oracle_lib):
    # Value produced by the independent implementation above for counter 0, key 0.
    assert [hex(int(x)) for x in oracle_lib.philox([0, 0, 0, 0], [0, 0])] == \
        ["0x6627e8d5", "0xe169c58d", "0xbc57ac4c", "0x9b00dbd8"]


def test_philox_words_are_uniform(oracle_lib):
    key = oracle_lib.key(987654321, oracle_lib.P_METROPOLIS, 1)
    words = np.array([oracle_lib.philox([i, 3, 9, 4], key) for i in range(20000)], dtype=np.uint64).ravel()
    n = words.size
    u = words / 2.0 ** 32
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    bits = ((words[:, None] >> np.arange(32, dtype=np.uint64)) & 1).mean(axis=0)
    assert np.all(np.abs(bits - 0.5) < 5 * 0.5 / np.sqrt(n))
    # acceptance frequency of a threshold test, as used by Metropolis and resampling
    thr = int(0.3 * 2 ** 32)
    p = (words < thr).mean()
    assert abs(p - 0.3) < 5 * np.sqrt(0.3 * 0.7 / n)


def test_key_layout(oracle_lib):
    k = oracle_lib.key((0xAB << 32) | 0x12345678, 3, 1)
    assert int(k[0]) == 0x12345678
    assert int(k[1]) == 0xAB | (3 << 28) | (1 << 24)
