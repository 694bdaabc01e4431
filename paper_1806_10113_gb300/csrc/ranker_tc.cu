// ranker_tc.cu -- the learned ranker's forward pass on the fifth-generation
// tensor cores (tcgen05): the scores of the beam search's candidate rows.
// The paper has no learned component; see ranker.cu for the model.
//
// One CTA per SM with four warpgroups; each warpgroup (4 warps, 128 threads)
// takes 128-row tiles in turn, so four tiles are in flight per SM and one
// warpgroup's epilogue overlaps the others' tensor-core work.  Shared memory
// holds the three weight matrices once (transposed, bfloat16, in the tensor
// cores' canonical K-major layout without swizzle: 8 x 16-byte core
// matrices) and the biases, plus one 128-row activation tile per warpgroup
// in the same layout; tensor memory holds one 128 x 128 f32 accumulator per
// warpgroup (512 columns).
// The weight image is prepared in global memory by image_kernel whenever the
// parameters change and copied once per CTA by a single bulk asynchronous
// copy (cp.async.bulk, completion on an mbarrier).  Per tile and layer:
//   1. the activation tile (the features for layer 1) is in shared memory;
//   2. one thread issues the layer's tcgen05.mma instructions (M = 128,
//      N = 128, K = 16 each; bf16 inputs, f32 accumulator in tensor memory,
//      128 columns allocated per CTA) and commits them to an mbarrier;
//   3. after the mbarrier completes, each warp reads its 32 rows of the
//      accumulator (tcgen05.ld), adds the bias, applies ReLU and rounds to
//      bfloat16 -- into the activation tile for the next layer, or, after
//      layer 3, straight into the dot product with w4 that gives the logit.
// Every wait on an mbarrier is bounded; on expiry the kernel records an
// error, writes NaN scores for its tile, waits (bounded) for its own
// tensor-core work, releases its tensor memory and returns.
#include <cuda_bf16.h>
#include <math.h>

#include "ranker.h"

namespace tmgpu {
namespace {

using bf16 = __nv_bfloat16;
constexpr int kF = kRankF, kH = kRankH;
constexpr int kTile = 128;                 // rows per tile = TMEM lanes
constexpr int kGroups = 4;                 // warpgroups per CTA
constexpr int kThreads = 128 * kGroups;

// Global weight image == the first kImgBytes of the CTA's shared memory.
// Each layer's bias enters the accumulator through one extra MMA of K = 16
// issued first (accumulate off): A = a constant tile whose first three
// columns are 1, B = a block holding the float32 bias split exactly into
// three bfloat16 parts (hi + mid + lo carry all 24 significand bits), so the
// accumulator starts at the bias and the epilogue adds nothing.
constexpr int kImgW1 = 0;                            // [128 n x 32 k] core layout
constexpr int kImgW2 = kImgW1 + kH * kF * 2;         // [128 x 128]
constexpr int kImgW3 = kImgW2 + kH * kH * 2;
constexpr int kBiasK = 16;
constexpr int kImgOnes = kImgW3 + kH * kH * 2;       // [128 rows x 16 k]: 1, 1, 1, 0, ...
constexpr int kImgB1 = kImgOnes + kTile * kBiasK * 2;   // [128 n x 16 k]: hi, mid, lo, 0, ...
constexpr int kImgB2 = kImgB1 + kH * kBiasK * 2;
constexpr int kImgB3 = kImgB2 + kH * kBiasK * 2;
// The head (logit = a3 . w4 + b4) is one more layer on the tensor cores with
// N = 16: B holds w4 (bfloat16) in its row 0 and zeros below; its bias block
// holds b4's three parts in row 0; the logit is accumulator column 0.
constexpr int kHeadN = 16;
constexpr int kImgW4 = kImgB3 + kH * kBiasK * 2;     // [16 n x 128 k]
constexpr int kImgB4 = kImgW4 + kHeadN * kH * 2;     // [16 n x 16 k]
constexpr int kImgBytes = kImgB4 + kHeadN * kBiasK * 2;
constexpr int kActOff = (kImgBytes + 127) / 128 * 128;
constexpr int kActBytes = kTile * kH * 2;            // per warpgroup
constexpr int kBarOff = kActOff + kGroups * kActBytes;
// mbarriers: [0] weights, [1 + g] warpgroup g's MMAs; then the TMEM address
constexpr int kSmemBytes = kBarOff + 8 * (1 + kGroups) + 16;
static_assert(kImgBytes % 16 == 0, "bulk copy size");

// Byte offset of element (r, k) of an R x K bf16 operand in the canonical
// K-major layout: 8-row x 8-element core matrices of 128 contiguous bytes,
// core matrix (r / 8, k / 8) at ((r / 8) * (K / 8) + k / 8) * 128.
__host__ __device__ constexpr int core_off(int r, int k, int K)
{
    return ((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// Shared-memory matrix descriptor (tcgen05): start address, leading-
// dimension byte offset (between the two core matrices along K of one
// K = 16 step), stride byte offset (between 8-row groups), descriptor
// version 1 (bits 46-47), no swizzle.
__device__ __forceinline__ uint64_t mat_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: f32 accumulator (bits 4-5 = 1), bf16 A
// and B (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at
// bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kH >> 3) << 17) |
                            ((uint32_t)(kTile >> 4) << 24);
constexpr uint32_t kIdescHead = (1u << 4) | (1u << 7) | (1u << 10) |
                                ((uint32_t)(kHeadN >> 3) << 17) | ((uint32_t)(kTile >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: about a second of clock cycles at most.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > (1ll << 31)) return false;
    return true;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_alloc(uint32_t dst, uint32_t cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst),
                 "r"(cols)
                 : "memory");
}
__device__ __forceinline__ void tc_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols)
                 : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     bar)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Barrier of one warpgroup (named barrier 1 + g, 128 threads), with a vote.
__device__ __forceinline__ void wg_sync(int g)
{
    asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory");
}
__device__ __forceinline__ bool wg_sync_and(int g, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n"
        ".reg .pred p, q;\n"
        "setp.ne.u32 p, %1, 0;\n"
        "bar.red.and.pred q, %2, 128, p;\n"
        "selp.u32 %0, 1, 0, q;\n"
        "}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(1 + g)
        : "memory");
    return r != 0;
}

// 32 consecutive f32 columns of this thread's accumulator row (warp w reads
// TMEM lanes 32 w .. 32 w + 31).
// Two float32 values rounded to bfloat16 and clamped at zero (relu after the
// rounding: the same value as rounding after relu, up to the sign of zero),
// packed with `lo` in the low half.
__device__ __forceinline__ uint32_t relu_bf16x2(float lo, float hi)
{
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// tcgen05.wait::ld tied to the registers of the loads it waits for, so that
// no use of them is scheduled before it.
__device__ __forceinline__ void tc_wait_ld32(uint32_t (&r)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr)
                 : "memory");
}

// Issues one layer: D (TMEM) = ones x bias-block^T (the bias, accumulate
// off), then D += A (activation tile, K columns) x W^T.
__device__ __forceinline__ void issue_layer(uint32_t tmem, uint32_t a_base, uint32_t w_base, int K,
                                            uint32_t ones, uint32_t bias_blk, uint32_t idesc)
{
    constexpr uint32_t sbo_b = (uint32_t)(kBiasK / 8) * 128u;
    tc_mma(tmem, mat_desc(ones, 128u, sbo_b), mat_desc(bias_blk, 128u, sbo_b), idesc, 0u);
    const uint32_t sbo = (uint32_t)(K / 8) * 128u;
    for (int s = 0; s < K / 16; ++s) {
        const uint64_t a = mat_desc(a_base + (uint32_t)s * 256u, 128u, sbo);
        const uint64_t b = mat_desc(w_base + (uint32_t)s * 256u, 128u, sbo);
        tc_mma(tmem, a, b, idesc, 1u);
    }
}

__device__ __forceinline__ void tc_ld1(uint32_t taddr, uint32_t& r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr) : "memory");
}

__device__ __forceinline__ void tc_wait_ld1(uint32_t& r)
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r) : : "memory");
}

// The three bfloat16 parts of a float32 value (hi + mid + lo == v exactly).
__device__ __forceinline__ void split3(float v, bf16& hi, bf16& mid, bf16& lo)
{
    hi = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(hi);
    mid = __float2bfloat16_rn(r1);
    lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
}

__global__ void image_kernel(const float* __restrict__ P, const bf16* __restrict__ Wb,
                             unsigned char* __restrict__ img)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    // weights: element (n, k) of W^T = W[k][n]
    if (i < kF * kH) {
        const int k = i / kH, n = i - k * kH;
        *reinterpret_cast<bf16*>(img + kImgW1 + core_off(n, k, kF)) = Wb[kBfW1 + i];
    }
    if (i < kH * kH) {
        const int k = i / kH, n = i - k * kH;
        *reinterpret_cast<bf16*>(img + kImgW2 + core_off(n, k, kH)) = Wb[kBfW2 + i];
        *reinterpret_cast<bf16*>(img + kImgW3 + core_off(n, k, kH)) = Wb[kBfW3 + i];
    }
    if (i < kTile * kBiasK) {
        const int r = i / kBiasK, k = i - r * kBiasK;
        *reinterpret_cast<bf16*>(img + kImgOnes + core_off(r, k, kBiasK)) =
            __float2bfloat16_rn(k < 3 ? 1.0f : 0.0f);
        const int offs[3] = {kImgB1, kImgB2, kImgB3};
        const int src[3] = {kOffB1, kOffB2, kOffB3};
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            bf16 parts[3];
            split3(P[src[l] + r], parts[0], parts[1], parts[2]);
            *reinterpret_cast<bf16*>(img + offs[l] + core_off(r, k, kBiasK)) =
                k < 3 ? parts[k] : __float2bfloat16_rn(0.0f);
        }
    }
    if (i < kHeadN * kH) {
        const int n = i / kH, k = i - n * kH;
        *reinterpret_cast<bf16*>(img + kImgW4 + core_off(n, k, kH)) =
            n == 0 ? Wb[kBfW4 + k] : __float2bfloat16_rn(0.0f);
    }
    if (i < kHeadN * kBiasK) {
        const int n = i / kBiasK, k = i - n * kBiasK;
        bf16 parts[3];
        split3(P[kOffB4], parts[0], parts[1], parts[2]);
        *reinterpret_cast<bf16*>(img + kImgB4 + core_off(n, k, kBiasK)) =
            (n == 0 && k < 3) ? parts[k] : __float2bfloat16_rn(0.0f);
    }
}

// KEEP: also store the three hidden layers' bfloat16 activations, row-major,
// layer l of row r at keep[(l * M + r) * 128] (for tests and inspection).
template <bool KEEP>
__global__ void __launch_bounds__(kThreads, 1)
forward_tc_kernel(const bf16* __restrict__ X, int64_t M, const unsigned char* __restrict__ img,
                  float* __restrict__ logits, int* __restrict__ err, bf16* __restrict__ keep)
{
    extern __shared__ __align__(128) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int grp = warp >> 2;                             // this thread's warpgroup
    const int row = tid & (kTile - 1);                     // its row of the group's tile
    const uint32_t s_base = smem_u32(sm);
    const uint32_t bar_w = s_base + kBarOff, bar_mma = s_base + kBarOff + 8 * (1 + grp);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + kBarOff + 8 * (1 + kGroups));

    if (warp == 0) {
        tc_alloc(smem_u32(s_tmem), kGroups * kH);   // one 128-column accumulator per warpgroup
        tc_relinquish();
    }
    if (tid == 0) {
        mbar_init(bar_w, 1);
        for (int g = 0; g < kGroups; ++g) mbar_init(s_base + kBarOff + 8 * (1 + g), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem + (uint32_t)(grp * kH);    // this warpgroup's columns
    if (tid == 0) {
        mbar_expect_tx(bar_w, kImgBytes);
        bulk_g2s(s_base, img, kImgBytes, bar_w);
    }
    // every decision to go on is taken by the whole warpgroup (a barrier vote)
    bool ok = __syncthreads_and(mbar_wait(bar_w, 0)) != 0;

    const int64_t tiles = (M + kTile - 1) / kTile;
    uint32_t phase = 0;
    const uint32_t act = s_base + kActOff + (uint32_t)(grp * kActBytes);
    unsigned char* act_p = sm + kActOff + grp * kActBytes;
    const uint32_t t_row = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const bool leader = row == 0;                           // issues the group's MMAs
    int64_t tile = (int64_t)blockIdx.x * kGroups + grp;
    const int64_t step = (int64_t)gridDim.x * kGroups;
    // this thread's row of features: loaded one tile ahead, so that the
    // global-memory latency hides behind the current tile's layers
    auto load_row = [&](int64_t t, uint4 (&v)[4]) {
        const int64_t r = t * kTile + row;
        if (t < tiles && r < M) {
            const uint4* src = reinterpret_cast<const uint4*>(X + (size_t)r * kF);
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = src[q];
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = make_uint4(0, 0, 0, 0);
        }
    };
    uint4 v[4];
    // launched as a programmatic dependent launch (the beam search), the
    // prologue above overlaps the kernel before; its rows are read only now
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    load_row(tile, v);
    for (; ok && tile < tiles; tile += step) {
        const int64_t r0 = tile * kTile;
        // features -> activation tile (K = 32 layout)
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<uint4*>(act_p + core_off(row, 8 * q, kF)) = v[q];
        load_row(tile + step, v);
        fence_async_smem();
        tc_fence_before();
        wg_sync(grp);
        tc_fence_after();
#pragma unroll 1
        for (int layer = 0; layer < 3 && ok; ++layer) {
            const int K = layer == 0 ? kF : kH;
            const uint32_t w = s_base + (layer == 0 ? kImgW1 : layer == 1 ? kImgW2 : kImgW3);
            if (leader) {
                const uint32_t bias_blk =
                    s_base + (layer == 0 ? kImgB1 : layer == 1 ? kImgB2 : kImgB3);
                issue_layer(tmem, act, w, K, s_base + kImgOnes, bias_blk, kIdesc);
                tc_commit(bar_mma);
            }
            ok = wg_sync_and(grp, mbar_wait(bar_mma, phase));
            phase ^= 1u;
            if (!ok) break;
            tc_fence_after();
            // 32 columns at a time, the next chunk's TMEM load in flight
            // while this one is converted and stored
            uint32_t rb[2][32];
            tc_ld32(t_row, rb[0]);
            tc_wait_ld32(rb[0]);
#pragma unroll
            for (int c = 0; c < kH / 32; ++c) {
                uint32_t (&r)[32] = rb[c & 1];
                if (c + 1 < kH / 32) tc_ld32(t_row + (uint32_t)(32 * (c + 1)), rb[(c + 1) & 1]);
                {
                    uint32_t packed[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        packed[j] = relu_bf16x2(__uint_as_float(r[2 * j]),
                                                __uint_as_float(r[2 * j + 1]));
                    // 32 columns = 4 core matrices along K of this row
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        *reinterpret_cast<uint4*>(act_p + core_off(row, 32 * c + 8 * q, kH)) =
                            make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2],
                                       packed[4 * q + 3]);
                    if (KEEP && r0 + row < M) {
                        uint4* dst = reinterpret_cast<uint4*>(
                            keep + ((size_t)layer * M + r0 + row) * kH + 32 * c);
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            dst[q] = make_uint4(packed[4 * q], packed[4 * q + 1],
                                                packed[4 * q + 2], packed[4 * q + 3]);
                    }
                }
                if (c + 1 < kH / 32) tc_wait_ld32(rb[(c + 1) & 1]);
            }
            // the next layer's MMAs read the tile this layer just wrote, and
            // overwrite the accumulator this layer just read
            fence_async_smem();
            tc_fence_before();
            wg_sync(grp);
            tc_fence_after();
        }
        if (!ok) break;
        // the head: a3 (now in the activation tile) x w4 + b4, column 0
        if (leader) {
            issue_layer(tmem, act, s_base + kImgW4, kH, s_base + kImgOnes, s_base + kImgB4,
                        kIdescHead);
            tc_commit(bar_mma);
        }
        ok = wg_sync_and(grp, mbar_wait(bar_mma, phase));
        phase ^= 1u;
        if (!ok) break;
        tc_fence_after();
        uint32_t lv;
        tc_ld1(t_row, lv);
        tc_wait_ld1(lv);
        if (r0 + row < M) logits[r0 + row] = __uint_as_float(lv);
    }
    if (!ok) {
        // a wait expired: report, mark this tile's scores, let in-flight
        // tensor-core work finish (bounded), then release tensor memory
        if (row == 0) atomicExch(err, 1);
        if (tile < tiles && tile * kTile + row < M) logits[tile * kTile + row] = nanf("");
        mbar_wait(bar_mma, phase ^ 1u);   // the phase that expired, once more
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tc_dealloc(*s_tmem, kGroups * kH);
}

}  // namespace

size_t ranker_image_bytes() { return (size_t)kImgBytes; }

cudaError_t ranker_image(const float* P, const bf16_raw* Wb, unsigned char* img, cudaStream_t s)
{
    image_kernel<<<(kH * kH + 255) / 256, 256, 0, s>>>(P, reinterpret_cast<const bf16*>(Wb), img);
    return cudaGetLastError();
}

cudaError_t ranker_tc_configure()
{
    cudaError_t e = cudaFuncSetAttribute(forward_tc_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(forward_tc_kernel<true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
}

cudaError_t ranker_forward_tc(const bf16_raw* X, int64_t M, const unsigned char* img,
                              float* logits, int* err, int blocks, cudaStream_t s, bf16_raw* keep,
                              bool pdl)
{
    if (M <= 0) return cudaSuccess;
    const int64_t groups = (M + (int64_t)kTile * kGroups - 1) / ((int64_t)kTile * kGroups);
    const int grid = (int)(groups < blocks ? groups : blocks);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kSmemBytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? attr : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    if (keep)
        return cudaLaunchKernelEx(&cfg, forward_tc_kernel<true>, reinterpret_cast<const bf16*>(X),
                                  M, img, logits, err, reinterpret_cast<bf16*>(keep));
    return cudaLaunchKernelEx(&cfg, forward_tc_kernel<false>, reinterpret_cast<const bf16*>(X), M,
                              img, logits, err, (bf16*)nullptr);
}

}  // namespace tmgpu
