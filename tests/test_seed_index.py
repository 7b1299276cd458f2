"""The inflow seeding's first-seed index, taken in parallel.

A seed goes where the running inflow measure reaches (k + 1/2) h_s.  Walking
the boundary edge by edge, k is raised while the level (k + 1/2) h_s stays
below the measure after the edge.  The GPU instead sums the measure serially
and then gives every edge, independently, the smallest k whose level is not
below the measure before it.  Both give the same indices in floating point
because the running measure never decreases and the rounded level rises with
k.  This test checks that claim on random weights in IEEE doubles (Python
floats), including zero and negative weights and levels met exactly."""
import math
import random


def _serial(w, hs):
    k, cum, kf, cb = 0, 0.0, [], []
    for wv in w:
        kf.append(k)
        cb.append(cum)
        if wv > 0.0:
            while (k + 0.5) * hs < cum + wv:
                k += 1
            cum += wv
    kf.append(k)
    cb.append(cum)
    return kf, cb


def _smallest_k(x, hs):
    if not (0.5 * hs < x):
        return 0
    k = max(int(math.ceil(x / hs - 0.5)), 0)
    while k > 0 and (k - 1 + 0.5) * hs >= x:
        k -= 1
    while (k + 0.5) * hs < x:
        k += 1
    return k


def test_parallel_seed_index_equals_the_serial_walk():
    rng = random.Random(20241118)
    for _ in range(2000):
        n = rng.randint(0, 200)
        hs = rng.choice([1 / 2047, 1 / 1023, 0.1, 1 / 3, 2.0 ** -10, rng.uniform(1e-4, 1.0)])
        w = []
        for _ in range(n):
            r = rng.random()
            if r < 0.3:
                w.append(0.0)
            elif r < 0.4:
                w.append(-rng.random() * hs)
            elif r < 0.6:
                w.append(hs * rng.choice([0.5, 1.0, 2.0, 0.25]))  # levels met exactly
            else:
                w.append(rng.random() * hs * rng.choice([0.1, 1.0, 3.0]))
        kf, cb = _serial(w, hs)
        assert [_smallest_k(x, hs) for x in cb] == kf
