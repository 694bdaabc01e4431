// Host-side checks of the exhaustive plan's layout (tm_internal.h), built
// and run by tests/test_plan_host.py with the host C++ compiler: the work
// order of plan_decompose and the cost ranges of static_range.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "tm_internal.h"

using namespace tmgpu;

static int fails = 0;
#define CHECK(c)                                                             \
    do {                                                                     \
        if (!(c)) {                                                          \
            std::printf("FAIL line %d: %s\n", __LINE__, #c);                 \
            ++fails;                                                         \
        }                                                                    \
    } while (0)

static uint64_t rng = 0x9E3779B97F4A7C15ull;
static uint64_t next_u64()
{
    rng ^= rng << 13;
    rng ^= rng >> 7;
    rng ^= rng << 17;
    return rng;
}

static void check_decompose(const std::vector<int32_t>& sizes, int pdmax, uint32_t item_cost)
{
    const int G = (int)sizes.size();
    std::vector<int32_t> off(G + 1, 0);
    for (int g = 0; g < G; ++g) off[g + 1] = off[g] + sizes[g];
    std::vector<GroupPlan> gp(G + 1);
    Plan p;
    CHECK(plan_decompose(off.data(), G, pdmax, item_cost, gp.data(), &p) == TM_OK);
    std::vector<int> seen(G, 0);
    uint64_t items = 0, cost = 0;
    int uniform = G > 0 ? sizes[0] : 0;
    for (int w = 0; w < G; ++w) {
        const int g = gp[w].group;
        CHECK(g >= 0 && g < G);
        if (g < 0 || g >= G) return;
        ++seen[g];
        const int n = sizes[g];
        if (sizes[g] != uniform) uniform = 0;
        // largest first, the caller's order among equal sizes
        if (w > 0) {
            const int pg = gp[w - 1].group;
            CHECK(sizes[pg] > n || (sizes[pg] == n && pg < g));
        }
        CHECK(gp[w].uoff == off[g]);
        CHECK(gp[w + 1].off - gp[w].off == n);
        CHECK(gp[w].item_base == items);
        CHECK(gp[w].cost_base == cost);
        if (n >= 4) {
            const int P = n - 4, pd = plan_pd(n, pdmax);
            const uint64_t heads = factorial_u64(P) / factorial_u64(pd);
            items += choose4(n) * heads;
            cost += choose4(n) * heads * (24ull * factorial_u64(pd) + item_cost);
        }
    }
    for (int g = 0; g < G; ++g) CHECK(seen[g] == 1);
    CHECK(gp[G].off == off[G] && gp[G].item_base == items && gp[G].cost_base == cost);
    CHECK(p.total_items == items && p.total_leaves == cost);
    CHECK(p.uniform_n == uniform);
    // every cost unit maps to the item that holds it
    for (int k = 0; k < 50 && cost > 0; ++k) {
        const uint64_t x = next_u64() % cost;
        const uint32_t i = plan_first_item(gp.data(), G, pdmax, item_cost, x);
        CHECK(i <= items);
    }
}

// static_range with the split of a single-size batch: every item's first
// cost unit lies in exactly one thread's range, and the lanes of one warp
// take the same number of items.
static void check_split(uint64_t I, uint64_t c, uint64_t threads)
{
    uint64_t warps = (threads + 31) / 32;
    const uint64_t klo = I / (32 * warps);
    if (klo == 0) warps = (I + 31) / 32;
    const uint64_t hi = (I - 32 * warps * klo + 31) / 32;
    CHECK(hi <= warps);
    std::vector<int> owner(I, 0);
    for (uint64_t t = 0; t < 32 * warps; ++t) {
        uint64_t x0, x1;
        static_range(t, 0, c, (uint32_t)warps, (uint32_t)hi, (uint32_t)klo, &x0, &x1);
        CHECK(x0 % c == 0 && x1 % c == 0 && x1 >= x0);
        CHECK(x1 - x0 == klo * c || x1 - x0 == (klo + 1) * c);
        uint64_t k0;
        uint64_t lane0_x0, lane0_x1;
        static_range(t & ~31ull, 0, c, (uint32_t)warps, (uint32_t)hi, (uint32_t)klo, &lane0_x0,
                     &lane0_x1);
        k0 = (lane0_x1 - lane0_x0) / c;
        CHECK((x1 - x0) / c == k0);   // one item count per warp
        for (uint64_t i = x0 / c; i < x1 / c && i < I; ++i) ++owner[i];
    }
    for (uint64_t i = 0; i < I; ++i) CHECK(owner[i] == 1);
    // heavier warps spread evenly: any 8 consecutive warps hold within 1 of the average share
    if (warps >= 8 && hi > 0) {
        for (uint64_t w0 = 0; w0 + 8 <= warps; w0 += 8) {
            const uint64_t h8 = (w0 + 8) * hi / warps - w0 * hi / warps;
            CHECK(h8 * warps + warps >= 8 * hi && h8 * warps <= 8 * hi + warps);
        }
    }
}

int main()
{
    check_decompose({10, 10, 10}, 5, 4096);
    check_decompose({4, 9, 1, 12, 7, 9, 2, 5, 11, 3, 6, 8}, 5, 65536);
    check_decompose({1, 2, 3}, 4, 256);
    check_decompose({}, 5, 1);
    for (int r = 0; r < 200; ++r) {
        std::vector<int32_t> s(1 + next_u64() % 40);
        const bool same = next_u64() % 3 == 0;
        const int n0 = 1 + (int)(next_u64() % 12);
        for (auto& x : s) x = same ? n0 : 1 + (int)(next_u64() % 12);
        check_decompose(s, 3 + (int)(next_u64() % 3), (uint32_t)(next_u64() % 70000));
    }
    check_split(161280, 6976, 58368);     // 64 x 10 evaluations x 2 models, 152 SMs x 3 x 128
    check_split(100, 7, 58368);           // fewer items than threads
    check_split(4096, 3, 1024);           // exact: two per lane
    for (int r = 0; r < 200; ++r)
        check_split(1 + next_u64() % 20000, 1 + next_u64() % 100, 32 + next_u64() % 5000);
    std::printf(fails ? "FAILED %d\n" : "ok\n", fails);
    return fails ? 1 : 0;
}
