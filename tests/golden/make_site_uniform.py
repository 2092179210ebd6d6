#!/usr/bin/env python3
"""Writes site_uniform.txt: the uniform u of the random-phase initial state
(Sec. 2 of arXiv:1809.00995: phases alpha = 2 pi u drawn from Philox) for a few
(seed, site index) pairs, by the word-to-uniform definition this project uses:

    ctr = (0, 0, index lo, index hi), key = (seed lo, seed hi),
    (w0, w1, w2, w3) = Philox-4x32-10(ctr, key),
    u = (w0 * 2^21 + floor(w1 / 2^11)) / 2^53            in [0, 1).

The Philox words come from the oracle's block function (itself pinned by the
published known-answer vectors); the mapping is evaluated here in exact
rational arithmetic (Python integers and fractions), independently of the
oracle's C code.  Each line: seed, index, u as an exact hexadecimal double.
Run from the repository root:  python tests/golden/make_site_uniform.py
"""
import os
import sys
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402

CASES = [(1, 0), (1, 1), (1, 12345), (2, 1 << 20), (3, 1073741823), (3, 1073741824),
         (100, 5), (163, 16777215), (0xFFFFFFFF, 7), ((1 << 32) + 9, 42),
         (0xDEADBEEFCAFEF00D, (1 << 32) + 3), (12, (1 << 33) - 1)]


def exact_u(seed: int, idx: int) -> Fraction:
    ctr = [0, 0, idx & 0xFFFFFFFF, idx >> 32]
    key = [seed & 0xFFFFFFFF, seed >> 32]
    w = O.philox4x32_10(ctr, key)
    m = w[0] * 2 ** 21 + w[1] // 2 ** 11
    assert 0 <= m < 2 ** 53
    return Fraction(m, 2 ** 53)


def main():
    lines = ["# seed index u  (see make_site_uniform.py: exact rational u, written as a hex double)"]
    for seed, idx in CASES:
        u = exact_u(seed, idx)
        d = float(u)
        assert Fraction(d) == u           # 53 bits: exactly representable
        lines.append("%d %d %s" % (seed, idx, d.hex()))
    with open(os.path.join(HERE, "site_uniform.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
