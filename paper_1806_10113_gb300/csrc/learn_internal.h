// learn_internal.h -- the ranker handle and the beam-search driver shared by
// the C ABI of the learned ranker (learn_api.cu) and the serving loop
// (server.cu).  Nothing here is visible through tm.h.
#pragma once

#include <algorithm>
#include <cstdint>

#include "ranker.h"
#include "tm_internal.h"

namespace tmgpu {

// A device buffer that grows on demand (contents are not kept).
struct Grow {
    void* p = nullptr;
    size_t cap = 0;
    bool ensure(size_t bytes)
    {
        if (bytes <= cap) return true;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        const size_t want = std::max<size_t>(bytes, 256);
        if (cudaMalloc(&p, want) != cudaSuccess) { p = nullptr; return false; }
        cap = want;
        return true;
    }
    template <class T> T* as() const { return static_cast<T*>(p); }
    void release() { if (p) cudaFree(p); p = nullptr; cap = 0; }
};

// Working memory of one beam search in flight.
struct BeamScratch {
    Grow st[2], scale, bx, blog, hms, bstatus;
    // Sizes every buffer for G groups of up to nmax tasks at beam width B.
    bool reserve(int G, int nmax, int B);
    void release()
    {
        for (Grow* b : {&st[0], &st[1], &scale, &bx, &blog, &hms, &bstatus}) b->release();
    }
};

// Rows of one beam step are processed in chunks of groups so that the
// feature matrix stays below this many rows.
constexpr int64_t kBeamRowsPerChunk = int64_t(1) << 22;
// Batches with at most this many first-position rows let the selection
// kernel write the next position's rows (fewer launches); larger ones use a
// separate row kernel (more parallel).  At widths up to kBeamWarpSelectMaxB
// a warp per group selects and writes the next rows, at any batch size.
constexpr int64_t kBeamFusedRows = int64_t(1) << 19;
constexpr int kBeamWarpSelectMaxB = 16;

// Beam search of G groups (see tm_beam_batch_dev).  d_offsets / h_offsets
// hold G + 1 task offsets (h_offsets need not start at 0; only differences
// are used on the host).  Group sizes must be 1..16, B 1..64 and K (refine
// starts) 0..8 (checked by the callers).  Uses `sc` (grown if needed) and reads the ranker's weights.
int beam_batch(const tm_ranker* r, BeamScratch& sc, const tm_task* d_tasks,
               const int32_t* d_offsets, const int32_t* h_offsets, int G, const tm_device* d_devs,
               int B, int K, int32_t* d_orders_out, int32_t* d_makespans_out, int32_t* d_status,
               int32_t* d_beam_won, cudaStream_t s);

}  // namespace tmgpu

struct tm_ranker {
    int device = -1;
    int sms = 0;
    float* P = nullptr;              // float32 master parameters
    tmgpu::bf16_raw* Wb = nullptr;   // bfloat16 weight copies
    float* Mom = nullptr;
    float* Vel = nullptr;
    float* G = nullptr;              // gradient of the last tm_ranker_grad_dev
    float* loss = nullptr;
    unsigned char* Wimg = nullptr;   // weight image of the tensor-core forward pass
    int* d_err = nullptr;            // set by a forward pass whose bounded wait expired
    int adam_step = 0;
    tmgpu::Grow scan_rows, scan_states, logits, dlogit, act;   // training
    tmgpu::BeamScratch beam;                                    // tm_beam_batch_dev
    void release()
    {
        for (void* q : {(void*)P, (void*)Wb, (void*)Mom, (void*)Vel, (void*)G, (void*)loss,
                        (void*)Wimg, (void*)d_err})
            if (q) cudaFree(q);
        for (tmgpu::Grow* b : {&scan_rows, &scan_states, &logits, &dlogit, &act}) b->release();
        beam.release();
    }
};
