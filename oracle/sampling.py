"""Perfect samples from correlated batches (test infrastructure only).

A batch of correlated amplitudes (SM Sec. II: output indices left open)
yields one exact sample (main text on Fig. 3(b)): draw the completion x of
a batch with probability |amp_x|^2 / sum_x' |amp_x'|^2.  With a uniform u in
[0, 1): the smallest x whose running sum of |amp|^2 exceeds u times the
batch total (the last completion if none does).  Plain float64: |amp|^2 as
re*re + im*im, the running sum added in x order (numpy's cumulative sum),
the threshold u * total.
"""

import numpy as np


def sample_completions(amps: np.ndarray, n_open: int, uniform: np.ndarray) -> np.ndarray:
    a = np.asarray(amps, np.complex128).reshape(-1, 1 << n_open)
    p = a.real * a.real + a.imag * a.imag
    c = np.cumsum(p, axis=1)
    thr = np.asarray(uniform, np.float64) * c[:, -1]
    picks = np.array([np.searchsorted(c[i], thr[i], side="right") for i in range(a.shape[0])], np.int64)
    return np.minimum(picks, (1 << n_open) - 1)
