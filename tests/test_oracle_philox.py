"""Pins of the oracle's Philox4x64-10 (Salmon et al., SC'11): published
known-answer vectors and numpy's independent implementation."""
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _kat():
    rows = []
    with open(os.path.join(HERE, "golden", "philox4x64_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            a, b = line.split("->")
            ins = [int(v, 16) for v in a.split()]
            outs = [int(v, 16) for v in b.split()]
            rows.append((ins[:4], ins[4:], outs))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_known_answers(ctr, key, out):
    assert oracle.philox(ctr, key) == out


def test_against_numpy_philox():
    rng = np.random.default_rng(12345)
    for _ in range(200):
        ctr = [int(v) for v in rng.integers(0, 2**63, 4, dtype=np.uint64)]
        key = [int(v) for v in rng.integers(0, 2**63, 2, dtype=np.uint64)]
        # numpy advances the 256-bit counter by one before producing a block
        start = (sum(c << (64 * i) for i, c in enumerate(ctr)) - 1) % 2**256
        words = np.array([(start >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64)
        bg = np.random.Philox(counter=words, key=np.array(key, dtype=np.uint64))
        assert oracle.philox(ctr, key) == [int(v) for v in bg.random_raw(4)]
