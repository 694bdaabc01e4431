// rank_features.cuh -- the 32 features the learned ranker sees for "append
// task j next" (shared by training-row generation and the beam search).
// Times are scaled by s = n / (sum of all durations of the group).
#pragma once

#include <stdint.h>

#include "tm.h"

namespace tmgpu {

constexpr int kFeat = 32;

// tasks: the group's n tasks; used: bit e set for tasks already placed;
// (h, k, d): engine times after the placed prefix; dma: 1 or 2.
__device__ __forceinline__ void rank_features(const tm_task* __restrict__ tasks, int n,
                                              uint32_t used, int32_t h, int32_t k, int32_t d,
                                              int dma, float scale, int j, float* f)
{
    const tm_task tj = tasks[j];
    const int32_t h1 = h + tj.htd;
    const int32_t k1 = max(k, h1) + tj.k;
    const int32_t d1 = max(d, k1) + tj.dth;
    float sh = 0.f, sk = 0.f, sd = 0.f, mh = 0.f, mk = 0.f, md = 0.f;
    int rem = 0;
    for (int i = 0; i < n; ++i) {
        if (i == j || ((used >> i) & 1u)) continue;
        const tm_task t = tasks[i];
        sh += (float)t.htd; sk += (float)t.k; sd += (float)t.dth;
        mh = fmaxf(mh, (float)t.htd); mk = fmaxf(mk, (float)t.k); md = fmaxf(md, (float)t.dth);
        ++rem;
    }
    f[0] = tj.htd * scale;
    f[1] = tj.k * scale;
    f[2] = tj.dth * scale;
    f[3] = (float)(k - h) * scale;
    f[4] = (float)(d - k) * scale;
    f[5] = (float)(k1 - h1) * scale;
    f[6] = (float)(d1 - k1) * scale;
    f[7] = (float)(d1 - d) * scale;
    f[8] = sh * scale;
    f[9] = sk * scale;
    f[10] = sd * scale;
    f[11] = mh * scale;
    f[12] = mk * scale;
    f[13] = md * scale;
    f[14] = (float)rem / (float)n;
    f[15] = dma == 1 ? 1.f : 0.f;
    f[16] = (float)max(0, h1 - k) * scale;
    f[17] = (float)max(0, k1 - d) * scale;
    f[18] = (float)(tj.k - tj.htd) * scale;
    f[19] = (float)min(tj.htd, tj.dth) * scale;
    for (int i = 20; i < kFeat; ++i) f[i] = 0.f;
}

}  // namespace tmgpu
