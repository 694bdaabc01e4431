"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a temporary copy of the oracle source (a
dropped dependency, a wrong queue layout, transposed stages, a wrong clock
step, a wrong tie rule, a wrong divisor, a misread term, sign, start time or
tie rule in the heuristic's cost, a wrong link between chained tasks), builds
it, and runs the pin suites against it in a child process.  They must fail
for every mutant.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "tm_oracle.cpp")

MUTANTS = {
    "dth_ignores_kernel": (
        "bool ready = (c.type == HTD) || done[3 * c.pos + (c.type - 1)];",
        "bool ready = (c.type != KER) || done[3 * c.pos + (c.type - 1)];"),
    "kernel_ignores_htd": (
        "bool ready = (c.type == HTD) || done[3 * c.pos + (c.type - 1)];",
        "bool ready = (c.type != DTH) || done[3 * c.pos + (c.type - 1)];"),
    "one_dma_interleaved_queue": (
        "fifo[0].items.push_back({i, HTD, stage(tasks[order[i]], HTD)});\n"
        "        for (int i = 0; i < n; ++i)\n"
        "            fifo[0].items.push_back({i, DTH, stage(tasks[order[i]], DTH)});",
        "{ fifo[0].items.push_back({i, HTD, stage(tasks[order[i]], HTD)});\n"
        "          fifo[0].items.push_back({i, DTH, stage(tasks[order[i]], DTH)}); }\n"
        "        for (int i = 0; i < 0; ++i) {}"),
    "htd_dth_transposed": (
        "return type == HTD ? t.htd : (type == KER ? t.k : t.dth);",
        "return type == HTD ? t.dth : (type == KER ? t.k : t.htd);"),
    "clock_to_latest_end": (
        "next = std::min(next, f.end);", "next = std::max(next == INT64_MAX ? 0 : next, f.end);"),
    "end_drops_start_time": ("f.end = T_sim + c.dur;", "f.end = c.dur;"),
    "best_tie_goes_last": (
        "if (ms < r.best) {", "if (ms <= r.best) {"),
    "mean_wrong_divisor": (
        "out->mean = (double)r.sum / (double)factorial(n);",
        "out->mean = (double)r.sum / (double)factorial(n - 1);"),
    "first_task_min_gain": ("if (gj > gb ||", "if (gj < gb ||"),
    "last_two_not_compared": ("if (m_ab != m_ba) take_ba = m_ba < m_ab;",
                              "if (m_ab != m_ba) take_ba = false;"),
    # select_next_task (H3): each term of the cost, its sign, the kernel start
    # s_j and the tie rule
    "h3_drops_kernel_fit": ("std::llabs((e.t_dth - s) - k);", "0 * std::llabs((e.t_dth - s) - k);"),
    "h3_drops_htd_fit": ("int64_t cost = std::llabs((e.t_k - e.t_htd) - h) +",
                         "int64_t cost = 0 * std::llabs((e.t_k - e.t_htd) - h) +"),
    "h3_signed_cost": ("int64_t cost = std::llabs((e.t_k - e.t_htd) - h) +\n"
                       "                       std::llabs((e.t_dth - s) - k);",
                       "int64_t cost = ((e.t_k - e.t_htd) - h) +\n"
                       "                       ((e.t_dth - s) - k);"),
    "h3_kernel_starts_at_t_k": ("int64_t s = std::max(e.t_k, e.t_htd + h);",
                                "int64_t s = e.t_k;"),
    "h3_kernel_starts_after_htd": ("int64_t s = std::max(e.t_k, e.t_htd + h);",
                                   "int64_t s = e.t_htd + h;"),
    "h3_tie_prefers_shorter_k": ("(cost == best_cost && tasks[j].k > tasks[best].k)",
                                 "(cost == best_cost && tasks[j].k < tasks[best].k)"),
    "h3_tie_lower_index": ("(cost == best_cost && tasks[j].k > tasks[best].k)",
                           "(cost == best_cost && false)"),
    # chained tasks: the link between a worker's tasks, the rank order, the mean
    "chain_link_dropped": ("ready = t < workers || done[3 * pos_of[t - workers] + DTH];",
                           "ready = true;"),
    "chain_link_waits_for_kernel": ("ready = t < workers || done[3 * pos_of[t - workers] + DTH];",
                                    "ready = t < workers || done[3 * pos_of[t - workers] + KER];"),
    "chain_link_by_position": ("ready = t < workers || done[3 * pos_of[t - workers] + DTH];",
                               "ready = t < workers || done[3 * (c.pos - workers) + DTH];"),
    "chain_last_round_most_significant": ("for (int r = rounds - 1; r >= first_round; --r)",
                                          "for (int r = first_round; r < rounds; ++r)"),
    "chain_mean_over_n_factorial": ("out[g].mean = (double)acc.sum / (double)count;",
                                    "(void)count;"),
}
PIN_FILES = ("test_oracle_pins.py", "test_chain_oracle.py")


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    # every copy of the anchor is mutated (the full search and the prefix
    # samples share the reduction rule)
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mut = tmp_path / "tm_oracle.cpp"
    mut.write_text(src.replace(old, new))
    hdr = os.path.join(ROOT, "oracle", "tm_oracle.h")
    (tmp_path / "tm_oracle.h").write_text(open(hdr).read())
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-pthread", "-o", str(lib),
                    str(mut)], check=True)
    env = dict(os.environ, TM_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        *[os.path.join(ROOT, "tests", f) for f in PIN_FILES]],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
