"""The integer float-pair split of the tree build (csrc/fsplit.cuh), compiled
for the host and checked against the conversions it replaces: hi = v rounded
to single precision (to nearest, ties to even), lo = (v - hi) rounded, on
random doubles over the exponent range the leaf frames use and on the cases
where the bit manipulation can go wrong (ties, carries into the next binade,
an exact zero rest, negative values, the out-of-range fallback)."""
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2507_21913_gb300", "csrc", "fsplit.cuh")

HARNESS = r"""
#include <stdio.h>
#include <inttypes.h>
#include "fsplit.cuh"
int main() {
  uint64_t u;
  while (scanf("%" SCNx64, &u) == 1) {
    double v;
    memcpy(&v, &u, 8);
    FsPair p = fs_split(v);
    float r = fs_round(v);
    uint32_t a, b, c;
    memcpy(&a, &p.hi, 4); memcpy(&b, &p.lo, 4); memcpy(&c, &r, 4);
    printf("%08x %08x %08x\n", a, b, c);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    d = tmp_path_factory.mktemp("fsplit")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I",
                        os.path.dirname(HDR), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return str(exe)


def run(exe, vals):
    vals = np.asarray(vals, np.float64)
    inp = "\n".join("%016x" % int(u) for u in vals.view(np.uint64)) + "\n"
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    w = np.array([[int(t, 16) for t in line.split()] for line in out.split("\n") if line],
                 np.uint32)
    return w[:, 0].view(np.float32), w[:, 1].view(np.float32), w[:, 2].view(np.float32)


def reference(vals):
    v = np.asarray(vals, np.float64)
    hi = v.astype(np.float32)                  # round to nearest, ties to even
    lo = (v - hi.astype(np.float64)).astype(np.float32)  # v - hi is exact in double here
    return hi, lo


def check(exe, vals):
    hi, lo, r = run(exe, vals)
    rh, rl = reference(vals)
    np.testing.assert_array_equal(hi.view(np.uint32), rh.view(np.uint32))
    np.testing.assert_array_equal(lo.view(np.uint32), rl.view(np.uint32))
    np.testing.assert_array_equal(r.view(np.uint32), rh.view(np.uint32))


def test_random_doubles(harness):
    g = np.random.Generator(np.random.PCG64(5))
    e = g.integers(-70, 100, 20000)
    m = g.uniform(1.0, 2.0, 20000)
    s = np.where(g.random(20000) < 0.5, -1.0, 1.0)
    check(harness, s * np.ldexp(m, e))


def test_ties_carries_and_exact(harness):
    g = np.random.Generator(np.random.PCG64(6))
    vals = []
    for e in (-70, -40, -3, 0, 1, 30, 99):
        for sgn in (1.0, -1.0):
            # exact ties: 24 significant bits then a single 1 at bit 25 (even and odd top)
            top = g.integers(1 << 23, 1 << 24, 8)
            vals += list(sgn * np.ldexp((2.0 * top + 1.0), e - 24))
            # a carry into the next binade: 2^e (1 - 2^-26)
            vals.append(sgn * np.ldexp(1.0 - 2.0 ** -26, e))
            vals.append(sgn * np.ldexp(1.0 - 2.0 ** -25, e))  # a tie that rounds up and carries
            # an exact float (zero rest) and the rest at its extremes
            vals.append(sgn * np.ldexp(float(top[0]), e - 23))
            vals.append(sgn * np.ldexp(float(top[0]) + 2.0 ** -29, e - 23))
            vals.append(sgn * np.ldexp(float(top[0]) + 0.5 - 2.0 ** -29, e - 23))
    check(harness, vals)


def test_outside_the_integer_range(harness):
    # zero and exponents outside [-70, 100] take the conversion instructions
    check(harness, [0.0, -0.0, 1e-30, -3e-25, 1e35, 2.0 ** 101, 2.0 ** -71])

