"""Pins of the oracle's random-number path (CPU only).

- Philox4x32-10 words against an independent implementation run as a
  library (triton's CPU interpreter), on random counters and keys.
- The uniform map, Box-Muller normals and the Laplace/Gaussian mixture
  against scipy's distributions (KS tests, moments) and closed-form
  values.
"""

import json
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import stats

import ra_scenes as rs

_TRITON_SCRIPT = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl
from triton.language.random import philox

@triton.jit
def kern(out_ptr, c_ptr, seed, N: tl.constexpr):
    offs = tl.arange(0, N)
    c0 = tl.load(c_ptr + offs * 4 + 0); c1 = tl.load(c_ptr + offs * 4 + 1)
    c2 = tl.load(c_ptr + offs * 4 + 2); c3 = tl.load(c_ptr + offs * 4 + 3)
    a, b, c, d = philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + offs * 4 + 0, a); tl.store(out_ptr + offs * 4 + 1, b)
    tl.store(out_ptr + offs * 4 + 2, c); tl.store(out_ptr + offs * 4 + 3, d)

cases = json.loads(sys.stdin.read())
res = []
for ctr, key in cases:
    seed = key[0] | (key[1] << 32)
    if seed >= 2**63:
        seed -= 2**64
    c = torch.tensor([x - 2**32 if x >= 2**31 else x for x in ctr] + [0] * 4, dtype=torch.int32)
    out = torch.zeros(8, dtype=torch.int32)
    kern[(1,)](out, c, seed, 2)
    res.append([int(v) & 0xFFFFFFFF for v in out[:4]])
print(json.dumps(res))
"""


def test_philox_matches_independent_library(orc):
    pytest.importorskip("triton")
    rng = np.random.default_rng(7)
    cases = [([0, 0, 0, 0], [0, 0]), ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2)]
    for _ in range(30):
        cases.append((rng.integers(0, 2**32, 4).tolist(), rng.integers(0, 2**32, 2).tolist()))
    env = dict(os.environ, TRITON_INTERPRET="1", CUDA_VISIBLE_DEVICES="")
    proc = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(cases),
                          capture_output=True, text=True, env=env, timeout=600)
    if proc.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + proc.stderr[-300:])
    ref = json.loads(proc.stdout.strip().splitlines()[-1])
    for (ctr, key), want in zip(cases, ref):
        got = orc.philox(ctr, key).tolist()
        assert got == want, (ctr, key, got, want)


def test_philox_counter_sensitivity(orc):
    # every counter and key word changes the output (no word is dropped)
    base = orc.philox([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert not np.array_equal(orc.philox(c, [5, 6]), base)
    for i in range(2):
        k = [5, 6]
        k[i] ^= 1
        assert not np.array_equal(orc.philox([1, 2, 3, 4], k), base)


def test_uniform_map_endpoints(orc):
    assert orc.uniform(0) == 2.0**-33
    assert orc.uniform(2**32 - 1) == 1.0 - 2.0**-33
    assert orc.uniform(2**31) == 0.5 + 2.0**-33


def _words(orc, n, seed=3):
    out = []
    for i in range(n):
        out.append(orc.philox([i, 17, 23, 0], [seed, 99]))
    return np.array(out, dtype=np.uint64)


def test_box_muller_normals(orc):
    w = _words(orc, 20000)
    z = np.array([orc.box_muller(a, b) for a, b in w[:, :2]]).ravel()
    assert abs(z.mean()) < 4 / np.sqrt(z.size)
    assert abs(z.std() - 1.0) < 0.01
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # the pair is uncorrelated
    zz = np.array([orc.box_muller(a, b) for a, b in w[:, 2:]])
    assert abs(np.corrcoef(zz[:, 0], zz[:, 1])[0, 1]) < 4 / np.sqrt(len(zz))


def test_mix_laplace_branch(orc):
    b = 0.02
    w = _words(orc, 40000, seed=11)
    vals = np.array([orc.mix_value(0xFFFFFFFF, int(x), b, 0.0, 5.0) for x in w[:, 0]])
    assert stats.kstest(vals, stats.laplace(scale=b).cdf).pvalue > 1e-3
    assert abs(vals.std() - np.sqrt(2) * b) < 0.02 * np.sqrt(2) * b
    # sign convention: the smallest word is the most negative value
    assert orc.mix_value(0xFFFFFFFF, 0, b, 0.0, 5.0) < -20 * b
    assert orc.mix_value(0xFFFFFFFF, 0xFFFFFFFF, b, 0.0, 5.0) > 20 * b
    # inverse CDF at a = (x + 1/2) 2^-32 exactly
    x = 123456789
    a = (x + 0.5) / 2**32
    assert abs(orc.mix_value(0xFFFFFFFF, x, b, 0.0, 5.0) - stats.laplace(scale=b).ppf(a)) < 1e-15


def test_mix_gaussian_branch(orc):
    # p = 1: every selector word below 2^32 - 1 takes the Gaussian branch, and
    # the selector is the Box-Muller angle word
    b, s = 0.02, 5.0
    w = _words(orc, 40000, seed=12)
    vals = np.array([orc.mix_value(int(a), int(x), b, 1.0, s) for a, x in w[:, :2]])
    assert stats.kstest(vals, stats.norm(scale=s * b).cdf).pvalue > 1e-3
    assert abs(vals.std() - s * b) < 0.02 * s * b
    # the angle (sel + 1/2) / (2^32 - 1) is exactly 1/2 at sel = 2^31 - 1, so
    # cos = -1 and the value is the Rayleigh radius sqrt(-2 ln v) (word < 2^31
    # gives the negative sign, v = (word + 1/2) 2^-31)
    for x in (0, 5, 123456789, 2**31 - 1):
        v = (x + 0.5) / 2**31
        assert orc.mix_value(2**31 - 1, x, b, 1.0, s) == pytest.approx(s * b * np.sqrt(-2 * np.log(v)), rel=1e-14, abs=1e-18)
    # the radius does not depend on the sign word: words x and ~x mirror
    assert orc.mix_value(77, 1000, b, 1.0, s) == -orc.mix_value(77, 0xFFFFFFFF - 1000, b, 1.0, s)


def test_mixture_distribution(orc):
    b, s, p = 0.02, 5.0, float(np.float32(0.1))
    w = _words(orc, 40000, seed=13)
    vals = np.array([orc.mix_value(int(a), int(c), b, p, s) for a, c in w[:, :2]])

    def cdf(x):
        return (1 - p) * stats.laplace(scale=b).cdf(x) + p * stats.norm(scale=s * b).cdf(x)

    assert stats.kstest(vals, cdf).pvalue > 1e-3
    # the selector threshold is floor(p 2^32): an integer decision
    thr = int(np.floor(p * 2**32))
    v = (5 + 0.5) / 2**31
    gauss = -s * b * np.sqrt(-2 * np.log(v)) * np.cos(2 * np.pi * (thr - 0.5) / thr)
    assert orc.mix_value(thr - 1, 5, b, p, s) == pytest.approx(gauss, rel=1e-12)
    assert orc.mix_value(thr, 5, b, p, s) == pytest.approx(b * np.log((5 + 0.5) / 2**31), rel=1e-12)


def test_process_noise_kinematic_moments(orc):
    p = rs.preset("c1_plain")
    prob = orc.make_problem(p)
    w = np.array([orc.process_noise(prob, k, m, t) for k in range(4) for m in range(50) for t in range(50)])
    std = w.std(0)
    np.testing.assert_allclose(std, [0.05, 0.05, 0.02, 0.1], rtol=0.04)
    c = np.corrcoef(w.T)
    assert np.max(np.abs(c - np.eye(4))) < 4 / np.sqrt(len(w))


def test_control_noise_moments(orc):
    p = rs.preset("c1_plain")
    prob = orc.make_problem(p)
    e = np.array([orc.control_noise(prob, k, t) for k in range(200) for t in range(40)])
    np.testing.assert_allclose(e.std(0), [0.3, 1.0], rtol=0.03)
    assert stats.kstest(e[:, 0] / np.float32(0.3), "norm").pvalue > 1e-3
    # another iteration gives another stream
    prob2 = orc.make_problem(p, iteration=1)
    assert not np.allclose(orc.control_noise(prob, 0, 0), orc.control_noise(prob2, 0, 0))
