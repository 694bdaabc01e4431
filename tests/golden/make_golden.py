"""Write the stored expected values under tests/golden/ from the oracle only.

    python tests/golden/make_golden.py

bk_table3_orders.txt: total time of every order of the paper's five synthetic
benchmarks (Table 3, built from the Table 2 tasks with a 10 ms time unit,
here in ms) under both device models.  The values come from ``oracle`` alone;
the test suite cross-checks them against an independent unit-time simulation.
"""
import itertools
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1806_10113_gb300 import inputs  # noqa: E402


def main():
    lines = [
        "# Total time (ms) of every order of the synthetic benchmarks of the paper",
        "# (Sec. 4.3, Table 3; tasks from Table 2 with a 10 ms time unit).",
        "# Written by tests/golden/make_golden.py from the CPU oracle only.",
        "# <benchmark> <dma_engines> <order> <total_ms>   (orders in lexicographic rank order)",
    ]
    for bk, names in inputs.TABLE3.items():
        tasks = inputs.table2_tasks(names, unit_ns=1)
        for dma in (2, 1):
            for order in itertools.permutations(range(len(names))):
                ms = oracle.predict(tasks, order, dma)
                lines.append(f"{bk} {dma} {','.join(map(str, order))} {ms}")
    with open(os.path.join(HERE, "bk_table3_orders.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
