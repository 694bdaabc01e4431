// learn_api.cu -- the extern "C" entry points of the learned order ranker
// and of the beam search that uses it (declared in include/tm.h).  The
// paper has no learned component; these schedule groups beyond exhaustive
// reach, every returned order being judged by the exact model.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "learn_internal.h"

namespace tmgpu {
// beam.cu
size_t beam_state_bytes(int G, int B);
cudaError_t beam_init(const int32_t* offsets, const int32_t* status, const tm_task* tasks,
                      const tm_device* devs, int G, int B, int R, void* st, float* scale,
                      bf16_raw* X, cudaStream_t s);
cudaError_t beam_features(const int32_t* offsets, const tm_task* tasks, const tm_device* devs,
                          const float* scale, const void* st, int G, int B, int R, int pos,
                          bf16_raw* X, cudaStream_t s);
cudaError_t beam_select(const int32_t* offsets, const tm_task* tasks, const tm_device* devs,
                        const float* scale, const float* logits, const void* cur, void* nxt, int G,
                        int B, int R, int pos, bf16_raw* X, cudaStream_t s, bool pdl);
cudaError_t beam_finish(const int32_t* offsets, const int32_t* status, const void* st, int G,
                        int B, const int32_t* heur_ms, int32_t* orders, int32_t* ms,
                        int32_t* beam_won, cudaStream_t s);
cudaError_t beam_refine(const tm_task* tasks, const int32_t* offsets, const tm_device* devs,
                        const int32_t* status, const void* st, int G, int B, int K,
                        const int32_t* heur_ms, int32_t* orders, int32_t* ms, int32_t* beam_won,
                        cudaStream_t s);
cudaError_t rank_rows(const tm_task* tasks, const int32_t* offsets, int G, const tm_device* devs,
                      const int32_t* orders, const tm_stats* stats, int64_t* row_base,
                      int32_t* state_base, int64_t M, int S, bf16_raw* X, int32_t* state_off,
                      int32_t* target, int32_t* status, cudaStream_t s);
}  // namespace tmgpu

namespace {

// Rows a group of n tasks contributes to the training rows (states p = 0 ..
// n - 2 with n - p candidates each) and its number of states.
inline int64_t group_rows(int n) { return n < 2 ? 0 : (int64_t)n * (n + 1) / 2 - 1; }
inline int32_t group_states(int n) { return n < 2 ? 0 : n - 1; }

}  // namespace

namespace {

// Blocks of the tensor-core forward pass: one per SM (four 128-row tiles in
// flight each).
int forward_blocks(const tm_ranker* r, int64_t M)
{
    const int64_t tiles = (M + 127) / 128;
    return (int)std::max<int64_t>(1, std::min<int64_t>((tiles + 3) / 4, r->sms));
}

int on_device(const tm_ranker* r)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return TM_ECUDA;
    return dev == r->device ? TM_OK : TM_EINVAL;
}

}  // namespace

namespace tmgpu {

bool BeamScratch::reserve(int G, int nmax, int B)
{
    const int64_t per_group = (int64_t)B * nmax;
    const int Gc = (int)std::max<int64_t>(1, std::min<int64_t>(G, kBeamRowsPerChunk / per_group));
    return st[0].ensure(beam_state_bytes(Gc, B)) && st[1].ensure(beam_state_bytes(Gc, B)) &&
           scale.ensure((size_t)Gc * sizeof(float)) &&
           bx.ensure((size_t)Gc * per_group * kRankF * sizeof(bf16_raw)) &&
           blog.ensure((size_t)Gc * per_group * sizeof(float)) &&
           hms.ensure((size_t)G * sizeof(int32_t)) && bstatus.ensure((size_t)G * sizeof(int32_t));
}

int beam_batch(const tm_ranker* r, BeamScratch& sc, const tm_task* d_tasks,
               const int32_t* d_offsets, const int32_t* h_offsets, int G, const tm_device* d_devs,
               int B, int K, int32_t* d_orders_out, int32_t* d_makespans_out, int32_t* d_status,
               int32_t* d_beam_won, cudaStream_t s)
{
    if (G == 0) return TM_OK;
    int nmax = 0;
    for (int g = 0; g < G; ++g) nmax = std::max(nmax, h_offsets[g + 1] - h_offsets[g]);
    // groups per chunk: G_c * B * nmax rows at the first step
    const int64_t per_group = (int64_t)B * nmax;
    const int Gc = (int)std::max<int64_t>(1, std::min<int64_t>(G, kBeamRowsPerChunk / per_group));
    if (!sc.reserve(G, nmax, B)) return TM_ENOMEM;
    int32_t* status = d_status ? d_status : sc.bstatus.as<int32_t>();
    int32_t* hms = sc.hms.as<int32_t>();
    // the paper's heuristic first: its order is the fallback (Algorithm 1)
    cudaError_t e = launch_heuristic(d_tasks, d_offsets, G, d_devs, d_orders_out, hms, status, s);
    for (int g0 = 0; g0 < G && e == cudaSuccess; g0 += Gc) {
        const int gc = std::min(Gc, G - g0);
        int nm = 0;
        for (int g = g0; g < g0 + gc; ++g) nm = std::max(nm, h_offsets[g + 1] - h_offsets[g]);
        const int32_t* off = d_offsets + g0;
        void* cur = sc.st[0].p;
        void* nxt = sc.st[1].p;
        e = beam_init(off, status + g0, d_tasks, d_devs + g0, gc, B, nm, cur, sc.scale.as<float>(),
                      sc.bx.as<bf16_raw>(), s);
        // small batches: the selection writes the next rows (two launches per
        // position); large ones: a separate row kernel spreads them over the GPU
        const bool fused = B <= kBeamWarpSelectMaxB || (int64_t)gc * B * nm <= kBeamFusedRows;
        for (int pos = 0; pos < nm && e == cudaSuccess; ++pos) {
            const int R = nm - pos;
            // position 0: beam 0's rows alone (the other beams start dead)
            const int64_t rows = (int64_t)gc * (pos == 0 ? 1 : B) * R;
            if (!fused && pos > 0)
                e = beam_features(off, d_tasks, d_devs + g0, sc.scale.as<float>(), cur, gc, B, R,
                                  pos, sc.bx.as<bf16_raw>(), s);
            if (e == cudaSuccess)
                // programmatic dependent launches: each position's scores
                // and selection may start while the kernel before finishes
                e = ranker_forward_tc(sc.bx.as<bf16_raw>(), rows, r->Wimg, sc.blog.as<float>(),
                                      r->d_err, forward_blocks(r, rows), s, nullptr, true);
            if (e == cudaSuccess)
                e = beam_select(off, d_tasks, d_devs + g0, sc.scale.as<float>(), sc.blog.as<float>(),
                                cur, nxt, gc, B, R, pos, fused ? sc.bx.as<bf16_raw>() : nullptr, s,
                                true);
            std::swap(cur, nxt);
        }
        if (e == cudaSuccess && K == 0)
            e = beam_finish(off, status + g0, cur, gc, B, hms + g0, d_orders_out,
                            d_makespans_out ? d_makespans_out + g0 : nullptr,
                            d_beam_won ? d_beam_won + g0 : nullptr, s);
        else if (e == cudaSuccess)
            e = beam_refine(d_tasks, off, d_devs + g0, status + g0, cur, gc, B, std::min(K, B),
                            hms + g0, d_orders_out, d_makespans_out ? d_makespans_out + g0 : nullptr,
                            d_beam_won ? d_beam_won + g0 : nullptr, s);
    }
    return e == cudaSuccess ? TM_OK : TM_ECUDA;
}

}  // namespace tmgpu

extern "C" {

int tm_ranker_create(uint64_t seed, tm_ranker** out)
{
    if (!out) return TM_EINVAL;
    *out = nullptr;
    tm_ranker* r = new (std::nothrow) tm_ranker;
    if (!r) return TM_ENOMEM;
    if (cudaGetDevice(&r->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&r->sms, cudaDevAttrMultiProcessorCount, r->device) != cudaSuccess ||
        tmgpu::ranker_configure() != cudaSuccess || tmgpu::ranker_tc_configure() != cudaSuccess) {
        delete r;
        return TM_ECUDA;
    }
    const size_t pb = tmgpu::kRankParams * sizeof(float);
    if (cudaMalloc(&r->P, pb) != cudaSuccess || cudaMalloc(&r->Mom, pb) != cudaSuccess ||
        cudaMalloc(&r->Vel, pb) != cudaSuccess || cudaMalloc(&r->G, pb) != cudaSuccess ||
        cudaMalloc(&r->loss, sizeof(float)) != cudaSuccess ||
        cudaMalloc(&r->Wimg, tmgpu::ranker_image_bytes()) != cudaSuccess ||
        cudaMalloc(&r->d_err, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&r->Wb, tmgpu::kRankBf16 * sizeof(tmgpu::bf16_raw)) != cudaSuccess) {
        r->release();
        delete r;
        return TM_ENOMEM;
    }
    cudaError_t e = cudaMemset(r->Mom, 0, pb);
    if (e == cudaSuccess) e = cudaMemset(r->Vel, 0, pb);
    if (e == cudaSuccess) e = cudaMemset(r->G, 0, pb);
    if (e == cudaSuccess) e = cudaMemset(r->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = tmgpu::ranker_init(r->P, r->Wb, seed, nullptr);
    if (e == cudaSuccess) e = tmgpu::ranker_image(r->P, r->Wb, r->Wimg, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        r->release();
        delete r;
        return TM_ECUDA;
    }
    *out = r;
    return TM_OK;
}

void tm_ranker_destroy(tm_ranker* r)
{
    if (!r) return;
    cudaDeviceSynchronize();
    r->release();
    delete r;
}

int tm_ranker_get_params(const tm_ranker* r, float* h_params)
{
    if (!r || !h_params) return TM_EINVAL;
    if (int rc = on_device(r)) return rc;
    if (cudaDeviceSynchronize() != cudaSuccess) return TM_ECUDA;
    return cudaMemcpy(h_params, r->P, tmgpu::kRankParams * sizeof(float),
                      cudaMemcpyDeviceToHost) == cudaSuccess ? TM_OK : TM_ECUDA;
}

int tm_ranker_set_params(tm_ranker* r, const float* h_params)
{
    if (!r || !h_params) return TM_EINVAL;
    if (int rc = on_device(r)) return rc;
    const size_t pb = tmgpu::kRankParams * sizeof(float);
    if (cudaDeviceSynchronize() != cudaSuccess) return TM_ECUDA;
    cudaError_t e = cudaMemcpy(r->P, h_params, pb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(r->Mom, 0, pb);
    if (e == cudaSuccess) e = cudaMemset(r->Vel, 0, pb);
    if (e == cudaSuccess) e = tmgpu::ranker_refresh(r->P, r->Wb, nullptr);
    if (e == cudaSuccess) e = tmgpu::ranker_image(r->P, r->Wb, r->Wimg, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    r->adam_step = 0;
    return e == cudaSuccess ? TM_OK : TM_ECUDA;
}

int tm_ranker_errors(const tm_ranker* r, int32_t* count)
{
    if (!r || !count) return TM_EINVAL;
    if (int rc = on_device(r)) return rc;
    int v = 0;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(&v, r->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return TM_ECUDA;
    *count = v;
    return TM_OK;
}

int tm_ranker_rows_count(const int32_t* h_offsets, int G, int64_t* rows, int32_t* states)
{
    if (G < 0 || !rows || !states || (G > 0 && !h_offsets)) return TM_EINVAL;
    if (G > 0 && h_offsets[0] != 0) return TM_EINVAL;
    int64_t m = 0, s = 0;
    for (int g = 0; g < G; ++g) {
        const int n = h_offsets[g + 1] - h_offsets[g];
        if (n < 1 || n > TM_MAX_TASKS) return TM_EINVAL;
        m += group_rows(n);
        s += group_states(n);
    }
    if (m > INT32_MAX - 16 || s > INT32_MAX - 1) return TM_ECAPACITY;
    *rows = m;
    *states = (int32_t)s;
    return TM_OK;
}

int tm_ranker_rows_dev(tm_ranker* r, const tm_task* d_tasks, const int32_t* d_offsets, int G,
                       const tm_device* d_devs, const int32_t* d_orders, const tm_stats* d_stats,
                       int64_t rows, int32_t states, uint16_t* d_X, int32_t* d_state_off,
                       int32_t* d_target, int32_t* d_status, void* stream)
{
    if (!r || G < 0 || rows < 0 || states < 0 || rows > INT32_MAX - 16) return TM_EINVAL;
    if (!d_X || !d_state_off || (states > 0 && !d_target)) return TM_EINVAL;
    if (G > 0 && (!d_tasks || !d_offsets || !d_devs || (!d_orders && !d_stats))) return TM_EINVAL;
    if (int rc = on_device(r)) return rc;
    if (!r->scan_rows.ensure((size_t)(G + 1) * sizeof(int64_t)) ||
        !r->scan_states.ensure((size_t)(G + 1) * sizeof(int32_t)))
        return TM_ENOMEM;
    cudaError_t e = tmgpu::rank_rows(d_tasks, d_offsets, G, d_devs, d_orders, d_stats,
                                     r->scan_rows.as<int64_t>(), r->scan_states.as<int32_t>(),
                                     rows, states, d_X, d_state_off, d_target, d_status,
                                     (cudaStream_t)stream);
    return e == cudaSuccess ? TM_OK : TM_ECUDA;
}

int tm_ranker_forward_dev(tm_ranker* r, const uint16_t* d_X, int64_t rows, float* d_logits,
                          void* stream)
{
    if (!r || rows < 0 || (rows > 0 && (!d_X || !d_logits))) return TM_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_X) % 16) return TM_EINVAL;   // rows are read 16 bytes at a time
    if (int rc = on_device(r)) return rc;
    if (rows == 0) return TM_OK;
    cudaError_t e = tmgpu::ranker_forward_tc(d_X, rows, r->Wimg, d_logits, r->d_err,
                                             forward_blocks(r, rows), (cudaStream_t)stream);
    return e == cudaSuccess ? TM_OK : TM_ECUDA;
}

int tm_ranker_forward_keep_dev(tm_ranker* r, const uint16_t* d_X, int64_t rows, float* d_logits,
                               uint16_t* d_acts, int path, void* stream)
{
    if (!r || rows < 0 || (rows > 0 && (!d_X || !d_logits || !d_acts))) return TM_EINVAL;
    if (path != 0 && path != 1) return TM_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_X) % 16 || reinterpret_cast<uintptr_t>(d_acts) % 16)
        return TM_EINVAL;
    if (rows > INT32_MAX - 16) return TM_EINVAL;
    if (int rc = on_device(r)) return rc;
    if (rows == 0) return TM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    tmgpu::bf16_raw* keep = reinterpret_cast<tmgpu::bf16_raw*>(d_acts);
    cudaError_t e = path == 0
        ? tmgpu::ranker_forward_tc(d_X, rows, r->Wimg, d_logits, r->d_err, forward_blocks(r, rows),
                                   s, keep)
        : tmgpu::ranker_forward(d_X, rows, r->Wb, r->P, d_logits, keep, rows, 2 * r->sms, s);
    return e == cudaSuccess ? TM_OK : TM_ECUDA;
}

int tm_ranker_grad_dev(tm_ranker* r, const uint16_t* d_X, int64_t rows,
                       const int32_t* d_state_off, const int32_t* d_target, int32_t states,
                       float* d_grad, float* d_loss, void* stream)
{
    if (!r || rows <= 0 || states <= 0 || !d_X || !d_state_off || !d_target) return TM_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_X) % 16) return TM_EINVAL;
    if (rows > INT32_MAX - 16) return TM_EINVAL;
    if (int rc = on_device(r)) return rc;
    const int64_t M_pad = (rows + 15) / 16 * 16;
    const size_t slab = (size_t)M_pad * tmgpu::kRankH * sizeof(tmgpu::bf16_raw);
    if (!r->logits.ensure((size_t)M_pad * sizeof(float)) ||
        !r->dlogit.ensure((size_t)M_pad * sizeof(float)) || !r->act.ensure(5 * slab))
        return TM_ENOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    // a1, a2, a3, dzA, dzB: rows past `rows` must read as zero
    const size_t tail = (size_t)(M_pad - rows) * tmgpu::kRankH * sizeof(tmgpu::bf16_raw);
    cudaError_t e = cudaSuccess;
    if (tail)
        e = cudaMemset2DAsync(static_cast<char*>(r->act.p) + (slab - tail), slab, 0, tail, 5, s);
    tmgpu::bf16_raw* act = r->act.as<tmgpu::bf16_raw>();
    if (e == cudaSuccess)
        e = tmgpu::ranker_backward(d_X, rows, d_state_off, d_target, states, r->Wb, r->P,
                                   r->logits.as<float>(), r->dlogit.as<float>(), act,
                                   act + 3 * slab / sizeof(tmgpu::bf16_raw), r->G, r->loss,
                                   2 * r->sms, s);
    if (e == cudaSuccess && d_grad)
        e = cudaMemcpyAsync(d_grad, r->G, tmgpu::kRankParams * sizeof(float),
                            cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && d_loss)
        e = cudaMemcpyAsync(d_loss, r->loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? TM_OK : TM_ECUDA;
}

int tm_ranker_adam_dev(tm_ranker* r, float lr, void* stream)
{
    if (!r || !(lr > 0.0f)) return TM_EINVAL;
    if (int rc = on_device(r)) return rc;
    r->adam_step += 1;
    cudaError_t e = tmgpu::ranker_adam(r->P, r->Mom, r->Vel, r->G, r->Wb, lr, r->adam_step,
                                       (cudaStream_t)stream);
    if (e == cudaSuccess) e = tmgpu::ranker_image(r->P, r->Wb, r->Wimg, (cudaStream_t)stream);
    return e == cudaSuccess ? TM_OK : TM_ECUDA;
}

int tm_beam_batch_dev(tm_ranker* r, const tm_task* d_tasks, const int32_t* d_offsets,
                      const int32_t* h_offsets, int G, const tm_device* d_devs, int beam_width,
                      int refine_starts, int32_t* d_orders_out, int32_t* d_makespans_out,
                      int32_t* d_status, int32_t* d_beam_won, void* stream)
{
    if (!r || G < 0 || beam_width < 1 || beam_width > TM_BEAM_MAX_WIDTH) return TM_EINVAL;
    if (refine_starts < 0 || refine_starts > TM_BEAM_MAX_REFINE_STARTS) return TM_EINVAL;
    if (G == 0) return TM_OK;
    if (!d_tasks || !d_offsets || !h_offsets || !d_devs || !d_orders_out) return TM_EINVAL;
    if (h_offsets[0] != 0) return TM_EINVAL;
    for (int g = 0; g < G; ++g) {
        const int n = h_offsets[g + 1] - h_offsets[g];
        if (n < 1 || n > TM_MAX_TASKS) return TM_EINVAL;
    }
    if (int rc = on_device(r)) return rc;
    return tmgpu::beam_batch(r, r->beam, d_tasks, d_offsets, h_offsets, G, d_devs, beam_width,
                             refine_starts, d_orders_out, d_makespans_out, d_status, d_beam_won,
                             (cudaStream_t)stream);
}

}  // extern "C"
