"""Position pairs (a, b) of the stored pairing derivatives of one sample, in
the block order the C ABI documents for vmc_get_samples: the up-up triangle
row-major, the down-down triangle, then the up-down rectangle row-major over
ascending positions (positions 0 .. n_up-1 are the up electrons)."""
import numpy as np


def block_pairs(n_up: int, n_dn: int) -> np.ndarray:
    N = n_up + n_dn
    pl = [(a, b) for a in range(n_up) for b in range(a + 1, n_up)]
    pl += [(a, b) for a in range(n_up, N) for b in range(a + 1, N)]
    pl += [(a, b) for a in range(n_up) for b in range(n_up, N)]
    return np.array(pl, dtype=np.int32).reshape(-1, 2)
