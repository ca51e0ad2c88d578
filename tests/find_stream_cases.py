"""Finds the stream cases that some tests use, with the oracle only.

    python tests/find_stream_cases.py

- Rejection seeds (tests/test_gpu_fills.py, REJECT_SEEDS): seeds whose
  first 100003 bounded words with m = 2^43 + 1 hold exactly one rejection,
  per engine.
- Long normal tails (tests/test_merge_points.py, LONG_TAILS): positions in
  the xoshiro256++ seed-2024 stream where a ziggurat tail candidate takes 11
  or more words.  The 2^30-variate scan takes about half a minute.
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), ".."))
import oracle  # noqa: E402


def reject_seeds(engine, want=2, m=2 ** 43 + 1, n=100003):
    found = []
    for seed in range(1, 1000):
        g = oracle.gen(engine, seed)
        oracle.fill(g, "bounded", n, m)
        if int(g.pos) == n + 1:
            found.append(seed)
            if len(found) == want:
                break
    return found


def long_tails(total=1 << 30, block=1 << 24, min_words=11):
    R = oracle.zig_table(0)[3]
    g = oracle.gen("xoshiro256pp", 2024)
    found, done = [], 0
    while done < total:
        x, st = oracle.fill(g, "normal", block, with_start=True)
        st = st.astype(np.int64)
        for j in np.nonzero(np.abs(x) > R)[0]:
            nxt = st[j + 1] if j + 1 < len(st) else int(g.pos)
            if nxt - st[j] >= min_words:   # the tail and anything rejected after it
                found.append(int(st[j]))
        done += block
    return found


if __name__ == "__main__":
    for eng in oracle.ENGINES:
        print("REJECT_SEEDS", eng, reject_seeds(eng))
    print("LONG_TAILS candidates", long_tails())
