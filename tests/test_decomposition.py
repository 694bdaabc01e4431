"""The max-plus split the exhaustive kernels rely on, checked on the CPU
against the oracle's event simulation: for an order made of a prefix pi and
an order sigma of the remaining 4-task set S,

    makespan = max(d_pi + alpha_S, k_pi + beta_sigma, gamma_sigma)

where (h_pi, k_pi, d_pi) are the engine times after pi, alpha_S is the DtH
sum of S, beta_sigma the makespan of sigma alone when only the kernel engine
starts (free at 0, transfers unconstrained) and gamma_sigma the same when
only the HtD engine starts, free at the HtD sum of pi.  The recurrence is
written out here from the model's definition (Sec. 4.1), independently of
the CUDA code."""
import itertools

import numpy as np

import oracle

NEG = -(1 << 60)


def run(tasks, order, h, k, d):
    for j in order:
        H, K, D = (int(x) for x in tasks[j])
        h = h + H
        k = max(k, h) + K
        d = max(d, k) + D
    return h, k, d


def test_split_equals_the_event_simulation():
    rng = np.random.default_rng(5)
    for trial in range(60):
        n = int(rng.integers(4, 8))
        hi = int(rng.choice([6, 1000, 3_000_000]))
        t = rng.integers(0, hi, size=(n, 3)).astype(np.int64)
        dma = 1 + trial % 2
        d0 = int(t[:, 0].sum()) if dma == 1 else 0
        for order in itertools.islice(itertools.permutations(range(n)), 0, None, 7):
            prefix, sigma = order[:n - 4], order[n - 4:]
            h, k, d = run(t, prefix, 0, 0, d0)
            alpha = int(t[list(sigma), 2].sum())
            _, _, beta = run(t, sigma, NEG, 0, NEG)
            _, _, gamma = run(t, sigma, h, NEG, NEG)
            split = max(d + alpha, k + beta, gamma)
            assert split == oracle.predict(t.astype(np.int32), list(order), dma), (trial, order)
