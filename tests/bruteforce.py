"""Unit-time brute-force simulation of the command queues (test helper).

A second, independent way to compute a group's total time: time advances one
unit at a time; every engine works on the command at the head of its queue
once the previous command of the same task has finished.  It shares nothing
with the oracle's event-driven simulator (which jumps from end time to end
time) nor with the CUDA recurrences, so it can only be used on small integer
durations.  Queue layout follows Sec. 3.2 / Fig. 4 of the paper: with two DMA
engines one queue per command type; with one DMA engine a single transfer
queue holding every HtD and then every DtH.
"""
import itertools

HTD, KER, DTH = 0, 1, 2


def stepped_total_time(tasks, order, dma_engines, workers=None):
    """Total time of `order` (positions -> task indices).  With `workers` set,
    the group is chained (the paper's experiment setup, Sec. 6.1): task index
    r * workers + w is worker w's round-r task, the order runs round by
    round, and a worker's round-r HtD waits until its round-(r - 1) DtH has
    finished; with one DMA engine each round's HtDs and then its DtHs take
    their turn in the single transfer queue."""
    n = len(order)
    chain = workers is not None
    rounds = n // workers if chain else 1
    blk = workers if chain else n
    if dma_engines == 2:
        queues = [[(i, HTD) for i in range(n)], [(i, KER) for i in range(n)],
                  [(i, DTH) for i in range(n)]]
    else:
        queues = [sum(([(i, HTD) for i in range(r * blk, (r + 1) * blk)] +
                       [(i, DTH) for i in range(r * blk, (r + 1) * blk)]
                       for r in range(rounds)), []),
                  [(i, KER) for i in range(n)]]
    pos_of = {int(t): i for i, t in enumerate(order)}

    def released(i):
        """A chained task's HtD waits for the previous task of its worker."""
        t = int(order[i])
        return not chain or t < workers or (pos_of[t - workers], DTH) in finished

    finished = set()
    running = [None] * len(queues)
    t = 0
    last = 0
    while True:
        changed = True
        while changed:                      # start every ready head at time t
            changed = False
            for qi, q in enumerate(queues):
                if running[qi] is None and q:
                    i, s = q[0]
                    if (s == HTD and released(i)) or (s != HTD and (i, s - 1) in finished):
                        q.pop(0)
                        d = int(tasks[order[i]][s])
                        if d == 0:
                            finished.add((i, s))
                            last = max(last, t)
                            changed = True
                        else:
                            running[qi] = [(i, s), d]
        if all(r is None for r in running):
            assert not any(queues), "queues cannot drain"
            return last
        t += 1                              # every busy engine works one unit
        for qi in range(len(queues)):
            r = running[qi]
            if r is not None:
                r[1] -= 1
                if r[1] == 0:
                    finished.add(r[0])
                    running[qi] = None
                    last = t


def all_orders(n):
    """All orders in lexicographic order (index == lexicographic rank)."""
    return list(itertools.permutations(range(n)))


def all_chain_orders(workers, rounds):
    """Every chained order, in lexicographic order: the rounds' permutations
    as the digits of a counter, round 0 most significant."""
    per_round = [[tuple(r * workers + w for w in p) for p in itertools.permutations(range(workers))]
                 for r in range(rounds)]
    return [sum(combo, ()) for combo in itertools.product(*per_round)]
