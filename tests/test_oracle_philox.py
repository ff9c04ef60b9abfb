"""Pins the oracle's Philox4x32-10 to two library implementations run on the CPU.

* triton's ``tl.philox`` (the interpreter, TRITON_INTERPRET=1), arbitrary counters and keys;
* cuRAND's host generator CURAND_RNG_PSEUDO_PHILOX4_32_10, whose block j for seed s is
  Philox(key = (s_lo, s_hi), counter = (0, 0, j, 0)) (mapping established by comparing outputs).
"""
import ctypes
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle

_TRITON_SCRIPT = r"""
import os, json, sys
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl

@triton.jit
def k(out_ptr, c_ptr, k_ptr, n: tl.constexpr):
    offs = tl.arange(0, n)
    c0 = tl.load(c_ptr + offs * 4 + 0); c1 = tl.load(c_ptr + offs * 4 + 1)
    c2 = tl.load(c_ptr + offs * 4 + 2); c3 = tl.load(c_ptr + offs * 4 + 3)
    k0 = tl.load(k_ptr + offs * 2 + 0); k1 = tl.load(k_ptr + offs * 2 + 1)
    seed = k0.to(tl.uint64) | (k1.to(tl.uint64) << 32)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + offs * 4 + 0, a); tl.store(out_ptr + offs * 4 + 1, b)
    tl.store(out_ptr + offs * 4 + 2, c); tl.store(out_ptr + offs * 4 + 3, d)

cases = json.loads(sys.stdin.read())
n = len(cases)
ctr = torch.tensor([v for c in cases for v in c[0]], dtype=torch.int64).to(torch.uint32)
key = torch.tensor([v for c in cases for v in c[1]], dtype=torch.int64).to(torch.uint32)
out = torch.zeros(4 * n, dtype=torch.uint32)
k[(1,)](out, ctr, key, n)
print(json.dumps([int(v) for v in out.to(torch.int64).tolist()]))
"""


def _cases():
    rng = np.random.default_rng(123)
    cases = [([0, 0, 0, 0], [0, 0]),
             ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2),
             ([1, 2, 3, 4], [5, 6])]
    while len(cases) < 16:
        cases.append((rng.integers(0, 2**32, 4).tolist(), rng.integers(0, 2**32, 2).tolist()))
    return cases


def test_philox_matches_triton_interpreter():
    pytest.importorskip("triton")
    cases = _cases()
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(cases),
                       capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + r.stderr.strip().splitlines()[-1])
    ref = np.array(json.loads(r.stdout.strip().splitlines()[-1]), dtype=np.uint64).reshape(-1, 4)
    for (ctr, key), want in zip(cases, ref):
        got = oracle.philox(ctr, key)
        assert got.tolist() == want.tolist(), (ctr, key)


def test_philox_matches_curand_host_generator():
    try:
        lib = ctypes.CDLL("libcurand.so.10")
    except OSError:
        pytest.skip("libcurand not present")
    for seed in (0, 0x0123456789ABCDEF):
        gen = ctypes.c_void_p()
        if lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:   # PHILOX4_32_10
            pytest.skip("cuRAND host generator unavailable")
        try:
            assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
            n = 4 * 8
            buf = (ctypes.c_uint32 * n)()
            assert lib.curandGenerate(gen, buf, ctypes.c_size_t(n)) == 0
        finally:
            lib.curandDestroyGenerator(gen)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for j in range(8):
            got = oracle.philox([0, 0, j, 0], key)
            assert got.tolist() == list(buf[4 * j:4 * j + 4]), (seed, j)
