"""Pin of the oracle's Philox4x32-10 (oracle.philox) to an independent
implementation of the same published generator (Salmon, Moraes, Dror, Shaw,
SC'11): Triton's ``tl.philox``, run by Triton's CPU interpreter.

The oracle's other pins (a bijection, dependence on every word, moments of
the normals) would all pass with swapped multipliers, another key schedule or
another output order; equality with a separately written implementation on
many counters and keys would not.  Triton is only a test reference here and
appears nowhere else.  The interpreter runs in a child process, so its
environment switch does not reach the other tests.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import philox

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import json, sys
import torch
import triton
import triton.language as tl

@triton.jit
def k(c_ptr, out_ptr, seed, n: tl.constexpr):
    i = tl.arange(0, n)
    c0 = tl.load(c_ptr + 4 * i + 0)
    c1 = tl.load(c_ptr + 4 * i + 1)
    c2 = tl.load(c_ptr + 4 * i + 2)
    c3 = tl.load(c_ptr + 4 * i + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + 4 * i + 0, a)
    tl.store(out_ptr + 4 * i + 1, b)
    tl.store(out_ptr + 4 * i + 2, c)
    tl.store(out_ptr + 4 * i + 3, d)

cases = json.loads(sys.stdin.read())
res = []
for seed, ctrs in cases:
    c = torch.tensor(ctrs, dtype=torch.int64).to(torch.int32).reshape(-1)  # two's complement of the uint32s
    out = torch.zeros_like(c)
    k[(1,)](c, out, seed, len(ctrs))
    res.append([int(v) & 0xFFFFFFFF for v in out.tolist()])
print(json.dumps(res))
"""


def _triton_words(cases):
    env = dict(os.environ, TRITON_INTERPRET="1", CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", _CHILD], input=json.dumps(cases), capture_output=True, text=True,
                         env=env, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-3000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_philox_matches_independent_implementation():
    pytest.importorskip("triton")
    rng = np.random.default_rng(20240917)
    cases = []
    # seeds below 2^63 (Triton takes the key as one 64-bit seed: k0 = low word, k1 = high word)
    seeds = [0, 1, 12345, 0xFFFFFFFF, 0x7FFFFFFFFFFFFFFF, 0x243F6A8885A308D3 & 0x7FFFFFFFFFFFFFFF]
    seeds += [int(v) for v in rng.integers(0, 2 ** 63 - 1, size=4, dtype=np.int64)]
    for seed in seeds:
        ctrs = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 0, 0, 0], [0, 0, 0, 1]]
        ctrs += rng.integers(0, 2 ** 32, size=(12, 4), dtype=np.uint64).tolist()
        cases.append([seed, [[int(w) for w in c] for c in ctrs]])
    got = _triton_words(cases)
    n = 0
    for (seed, ctrs), words in zip(cases, got):
        c = np.array(ctrs, dtype=np.uint64)
        ours = philox.philox4x32_10(c[:, 0], c[:, 1], c[:, 2], c[:, 3], seed & 0xFFFFFFFF, seed >> 32)
        ours = np.stack(ours, axis=1).reshape(-1).astype(np.uint64)
        assert np.array_equal(ours, np.array(words, dtype=np.uint64)), hex(seed)
        n += len(ctrs)
    assert n == len(seeds) * 16


def test_probe_words_are_philox_blocks_in_counter_order():
    """probe_words lays the blocks of counters (i // 4, t, slice, 0) end to end,
    word i % 4 of each (so the pin above covers the probe stream too)."""
    seed, t, sl = 0x1234_5678_9ABC, 7, 3
    w = philox.probe_words(4 * 5 + 2, seed, t, sl)
    for g in range(6):
        blk = philox.philox4x32_10(np.array([g]), np.array([t]), np.array([sl]), np.array([0]),
                                   seed & 0xFFFFFFFF, seed >> 32)
        for j in range(4):
            if 4 * g + j < len(w):
                assert int(w[4 * g + j]) == int(blk[j][0])
