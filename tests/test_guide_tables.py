"""Guide tables of the inverse-CDF search (host logic, no GPU).

The step kernel starts the search of a CDF row (Eq. 7, and the pair
spectrum) at an entry of a guide table instead of bisecting the row:
buckets of xi in (0, 1/2] (and of eta = 1 - xi above 1/2), four per octave;
the lower-half entry is the last node below the bucket's lower edge, the
upper-half entry the last node with 1 - C above the bucket's upper edge.  On
the oracle's CDF rows, entry + forward scan must find exactly the interval a
bisection finds, for every row and random xi, with short scans.
"""
import math

import numpy as np

import oracle as O

NB = 224


def bucket(x):
    m, e = math.frexp(x)           # x = m 2^e, m in [0.5, 1)
    e -= 1                         # x = (2m) 2^e, 2m in [1, 2)
    k = int((2 * m - 1.0) * 4)     # two leading mantissa bits
    return min(max(((-1 - e) << 2) | k, 0), NB - 1)


def guides(C):
    gl = np.zeros(NB, int)
    gu = np.zeros(NB, int)
    for m in range(NB):
        e, k = -1 - (m >> 2), m & 3
        lo, hi = math.ldexp(1 + k / 4, e), math.ldexp(1 + (k + 1) / 4, e)
        below = np.nonzero(C[:255] < lo * (1 - 1e-9))[0]
        above = np.nonzero(1.0 - C[:255] > hi * (1 + 1e-9))[0]
        gl[m] = below.max() if len(below) else 0
        gu[m] = above.max() if len(above) else 0
    return gl, gu


def bisect(C, xi):
    lo, hi = 0, 255
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if C[mid] < xi:
            lo = mid
        else:
            hi = mid
    return lo


def test_guide_entry_and_scan_find_the_bisection_interval():
    T = O.tables()
    rng = np.random.default_rng(7)
    worst = 0
    for table in (np.asarray(T.Cg).reshape(97, 256), np.asarray(T.Cp).reshape(97, 256)):
        for r in range(0, 97, 4):
            C = table[r]
            gl, gu = guides(C)
            # uniform xi, and xi concentrated in both tails
            xs = np.concatenate([rng.random(300), 10.0 ** -rng.uniform(1, 15, 150),
                                 1 - 10.0 ** -rng.uniform(1, 15, 150)])
            for xi in xs:
                if not (C[0] < xi < C[255]):
                    continue
                g = gl[bucket(xi)] if xi <= 0.5 else gu[bucket(1.0 - xi)]
                steps = 0
                while g < 254 and C[g + 1] < xi:
                    g += 1
                    steps += 1
                assert g == bisect(C, xi), (r, xi)
                worst = max(worst, steps)
    print(f"\nlongest forward scan: {worst} nodes")
    assert worst <= 24
