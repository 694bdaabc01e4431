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


def stepped_total_time(tasks, order, dma_engines):
    n = len(order)
    if dma_engines == 2:
        queues = [[(i, HTD) for i in range(n)], [(i, KER) for i in range(n)],
                  [(i, DTH) for i in range(n)]]
    else:
        queues = [[(i, HTD) for i in range(n)] + [(i, DTH) for i in range(n)],
                  [(i, KER) for i in range(n)]]
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
                    if s == HTD or (i, s - 1) in finished:
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
