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


def test_closed_forms_where_one_engine_ends_every_completion():
    """The three closed forms of the enumeration's walk modes 5 to 8, on the
    24 makespans of S's orders after a prefix (all from the event
    simulation): with c0 = d + alpha, (i) c0 >= max(k + max beta, max gamma):
    every makespan is c0; (ii) k >= max(gamma - beta) and c0 <= k + min beta:
    makespan sigma is k + beta_sigma; (iii) k <= min(gamma - beta) and
    c0 <= min gamma: makespan sigma is gamma_sigma.  Under any of them the
    minimum is max(c0, k + min beta, min gamma); the maximum is always
    max(c0, k + max beta, max gamma).  Each case is met on these inputs."""
    rng = np.random.default_rng(11)
    hits = [0, 0, 0]
    for trial in range(240):
        n = int(rng.integers(4, 8))
        dma = 1 + trial % 2
        scale = int(rng.choice([4, 1000, 2_000_000]))
        rows = []
        for _ in range(n):
            kind = rng.integers(0, 3)   # dominant kernel, dominant transfer, or even
            big, small = scale * int(rng.integers(5, 20)), int(rng.integers(0, scale + 1))
            rows.append([small, big, small] if kind == 0 else
                        [big, small, big] if kind == 1 else
                        [int(rng.integers(0, scale + 1)) for _ in range(3)])
        t = np.array(rows, dtype=np.int64)
        d0 = int(t[:, 0].sum()) if dma == 1 else 0
        perm = rng.permutation(n)
        S = sorted(int(x) for x in perm[:4])
        prefix = [int(x) for x in perm[4:]]
        h, k, d = run(t, prefix, 0, 0, d0)
        sigmas = list(itertools.permutations(S))
        alpha = int(t[S, 2].sum())
        beta = [run(t, s, NEG, 0, NEG)[2] for s in sigmas]
        gamma = [run(t, s, h, NEG, NEG)[2] for s in sigmas]
        ms = [oracle.predict(t.astype(np.int32), prefix + list(s), dma) for s in sigmas]
        c0 = d + alpha
        assert max(ms) == max(c0, k + max(beta), max(gamma)), trial
        case_d = c0 >= max(k + max(beta), max(gamma))
        case_k = k >= max(g - b for g, b in zip(gamma, beta)) and c0 <= k + min(beta)
        case_c = k <= min(g - b for g, b in zip(gamma, beta)) and c0 <= min(gamma)
        if case_d:
            hits[0] += 1
            assert ms == [c0] * 24, trial
        if case_k:
            hits[1] += 1
            assert ms == [k + b for b in beta], trial
            assert sum(ms) == 24 * k + sum(beta), trial
        if case_c:
            hits[2] += 1
            assert ms == gamma, trial
        if case_d or case_k or case_c:
            assert min(ms) == max(c0, k + min(beta), min(gamma)), trial
    assert all(c > 0 for c in hits), hits
