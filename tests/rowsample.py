"""Row samples for the full-size parity tests (helper module, not a test file).

A far-field launch maps targets to blocks of 256 (32 threads x 8 targets, target
first + thread + k * 32 for k = 0..7 in the default shape and in the batched kernel): the sample
takes, in every block, its first row, the last row of thread 0's first stride, the first row of
its second stride and its last row (so the ragged last block is always covered), plus seeded
random rows. Every sampled row runs over all source tiles and chunks of the launch."""
import numpy as np


def boundary_rows(n: int, n_random: int, seed: int, block: int = 256) -> np.ndarray:
    starts = np.arange(0, n, block)
    cand = np.concatenate([starts, starts + 31, starts + 32, np.minimum(starts + block, n) - 1, [n - 1]])
    rng = np.random.default_rng(seed)
    rand = rng.choice(n, size=min(n_random, n), replace=False)
    rows = np.unique(np.concatenate([cand[cand < n], rand]))
    return rows.astype(np.int64)
