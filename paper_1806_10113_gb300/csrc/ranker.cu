// ranker.cu -- the learned order ranker: a 4-layer MLP (32 -> 128 -> 128 ->
// 128 -> 1, ReLU) that scores "append task j next" from 32 features of the
// candidate and the engine state.  The paper has no learned component: the
// ranker only proposes orders to a beam search (beam.cu) for groups beyond
// exhaustive reach; the exact model judges every order it returns.
//
// Arithmetic: bfloat16 weights and activations, float32 accumulation
// (tensor cores through WMMA 16x16x16), float32 master weights, Adam.
// Layout of the float32 parameter vector (kOff*): W1 [32 x 128] (in x out,
// row-major), b1, W2 [128 x 128], b2, W3 [128 x 128], b3, w4 [128], b4.
#include <cuda_bf16.h>
#include <mma.h>

#include "ranker.h"

namespace tmgpu {
namespace {

using namespace nvcuda;
using bf16 = __nv_bfloat16;
constexpr int kF = kRankF, kH = kRankH;
constexpr int kWarps = 8;         // warps per block of the row kernels
constexpr int kSlab = 16;         // rows per warp

// ---- forward ----------------------------------------------------------------

// One warp's 16-row slab through a [16 x K] x [K x 128] layer: the
// accumulators land in `stage` (row-major float, ld 128).
template <int K>
__device__ __forceinline__ void slab_layer(const bf16* __restrict__ act, const bf16* __restrict__ W,
                                           float* __restrict__ stage)
{
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) wmma::fill_fragment(acc[t], 0.0f);
#pragma unroll
    for (int kk = 0; kk < K; kk += 16) {
        wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::row_major> a;
        wmma::load_matrix_sync(a, act + kk, K);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> b;
            wmma::load_matrix_sync(b, W + kk * kH + 16 * t, kH);
            wmma::mma_sync(acc[t], a, b, acc[t]);
        }
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) wmma::store_matrix_sync(stage + 16 * t, acc[t], kH, wmma::mem_row_major);
    __syncwarp();
}

// stage + bias, ReLU, rounded to bfloat16 into `out` (and `keep` if given).
__device__ __forceinline__ void slab_epilogue(const float* __restrict__ stage,
                                              const float* __restrict__ bias, bf16* __restrict__ out,
                                              bf16* __restrict__ keep, int rows_valid)
{
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < kSlab * kH; i += 32) {
        const int r = i / kH, c = i - r * kH;
        const bf16 v = __float2bfloat16_rn(fmaxf(stage[i] + bias[c], 0.0f));
        out[i] = v;
        if (keep && r < rows_valid) keep[(size_t)r * kH + c] = v;
    }
    __syncwarp();
}

struct __align__(128) FwdShared {
    bf16 W1[kF * kH];
    bf16 W2[kH * kH];
    bf16 W3[kH * kH];
    float w4[kH];
    float b1[kH], b2[kH], b3[kH];
    float b4;
    struct __align__(128) Slab {
        bf16 x[kSlab * kF];
        bf16 a[kSlab * kH];
        bf16 b[kSlab * kH];
        float stage[kSlab * kH];
    } slab[kWarps];
};

__device__ __forceinline__ float bf(const bf16 v) { return __bfloat162float(v); }
__host__ __device__ __forceinline__ int64_t lmin(int64_t a, int64_t b) { return a < b ? a : b; }

// logits[r] for rows r < M of X; with keep != null also stores a1, a2, a3
// ([stride x 128] each, at keep + l * stride * 128).  Persistent: each warp
// takes 16-row slabs in turn.
__global__ void __launch_bounds__(kWarps * 32)
forward_kernel(const bf16* __restrict__ X, int64_t M, const bf16* __restrict__ Wb,
               const float* __restrict__ P, float* __restrict__ logits, bf16* __restrict__ keep,
               int64_t stride)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    FwdShared& s = *reinterpret_cast<FwdShared*>(smem_raw);
    for (int i = threadIdx.x; i < kF * kH; i += blockDim.x) s.W1[i] = Wb[kBfW1 + i];
    for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) {
        s.W2[i] = Wb[kBfW2 + i];
        s.W3[i] = Wb[kBfW3 + i];
    }
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        s.w4[i] = bf(Wb[kBfW4 + i]);
        s.b1[i] = P[kOffB1 + i];
        s.b2[i] = P[kOffB2 + i];
        s.b3[i] = P[kOffB3 + i];
    }
    if (threadIdx.x == 0) s.b4 = P[kOffB4];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    FwdShared::Slab& w = s.slab[warp];
    const int64_t slabs = (M + kSlab - 1) / kSlab;
    for (int64_t sl = (int64_t)blockIdx.x * kWarps + warp; sl < slabs;
         sl += (int64_t)gridDim.x * kWarps) {
        const int64_t r0 = sl * kSlab;
        const int rows = (int)lmin(kSlab, M - r0);
        for (int i = lane; i < kSlab * kF; i += 32) {
            const int r = i / kF;
            w.x[i] = r < rows ? X[(size_t)r0 * kF + i] : __float2bfloat16_rn(0.0f);
        }
        __syncwarp();
        bf16* k1 = keep ? keep + (size_t)r0 * kH : nullptr;
        bf16* k2 = keep ? keep + (size_t)stride * kH + (size_t)r0 * kH : nullptr;
        bf16* k3 = keep ? keep + 2 * (size_t)stride * kH + (size_t)r0 * kH : nullptr;
        slab_layer<kF>(w.x, s.W1, w.stage);
        slab_epilogue(w.stage, s.b1, w.a, k1, rows);
        slab_layer<kH>(w.a, s.W2, w.stage);
        slab_epilogue(w.stage, s.b2, w.b, k2, rows);
        slab_layer<kH>(w.b, s.W3, w.stage);
        slab_epilogue(w.stage, s.b3, w.a, k3, rows);
        // head: one row per half-warp pass, lanes over the 128 inputs
        for (int r = 0; r < rows; ++r) {
            float acc = 0.0f;
            for (int c = lane; c < kH; c += 32) acc += bf(w.a[r * kH + c]) * s.w4[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
            if (lane == 0) logits[r0 + r] = acc + s.b4;
        }
        __syncwarp();
    }
}

// ---- loss ---------------------------------------------------------------------

// Softmax cross-entropy per state (rows off[s] .. off[s+1]) against its
// target row; dlogit = (softmax - onehot) / S (rows outside every state keep
// the zero the caller set); loss summed into *loss.  Offsets are clamped to
// [0, M]; a state whose target lies outside its rows contributes nothing.
__global__ void loss_kernel(const float* __restrict__ logits, int64_t M,
                            const int32_t* __restrict__ off, const int32_t* __restrict__ target,
                            int S, float* __restrict__ dlogit, float* __restrict__ loss)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int64_t lo = lmin(max((int64_t)off[s], (int64_t)0), M);
    const int64_t hi = lmin(max((int64_t)off[s + 1], lo), M);
    const int64_t t = target[s];
    if (t < lo || t >= hi) return;
    float mx = -INFINITY;
    for (int64_t r = lo; r < hi; ++r) mx = fmaxf(mx, logits[r]);
    float z = 0.0f;
    for (int64_t r = lo; r < hi; ++r) z += expf(logits[r] - mx);
    const float inv = 1.0f / (z * (float)S);
    for (int64_t r = lo; r < hi; ++r) dlogit[r] = expf(logits[r] - mx) * inv;
    dlogit[t] -= 1.0f / (float)S;
    atomicAdd(loss, (logf(z) + mx - logits[t]) / (float)S);
}

// ---- backward -------------------------------------------------------------------

// dz3 = dlogit (x) w4, masked by a3 > 0 (bfloat16); dw4 += a3^T dlogit;
// db4 += sum dlogit.  One block per 256-row chunk.
__global__ void head_backward_kernel(const float* __restrict__ dlogit, const bf16* __restrict__ a3,
                                     int64_t M, const bf16* __restrict__ Wb,
                                     bf16* __restrict__ dz3, float* __restrict__ G)
{
    __shared__ float part[kH];
    __shared__ float bpart;
    for (int c = threadIdx.x; c < kH; c += blockDim.x) part[c] = 0.0f;
    if (threadIdx.x == 0) bpart = 0.0f;
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * 256;
    const int64_t r1 = lmin(r0 + 256, M);
    const int c = threadIdx.x & (kH - 1);
    const float w4c = bf(Wb[kBfW4 + c]);
    float acc = 0.0f, bacc = 0.0f;
    for (int64_t r = r0 + threadIdx.x / kH; r < r1; r += blockDim.x / kH) {
        const float g = dlogit[r];
        const bf16 av = a3[(size_t)r * kH + c];
        acc += g * bf(av);
        dz3[(size_t)r * kH + c] = __float2bfloat16_rn(bf(av) > 0.0f ? g * w4c : 0.0f);
        if (c == 0) bacc += g;
    }
    atomicAdd(&part[c], acc);
    if (c == 0) atomicAdd(&bpart, bacc);
    __syncthreads();
    for (int i = threadIdx.x; i < kH; i += blockDim.x) atomicAdd(&G[kOffW4 + i], part[i]);
    if (threadIdx.x == 0) atomicAdd(&G[kOffB4], bpart);
}

// dz_prev = (dz W^T) masked by a_prev > 0, for a 128 x 128 layer W.
__global__ void __launch_bounds__(kWarps * 32)
dgrad_kernel(const bf16* __restrict__ dz, const bf16* __restrict__ a_prev, int64_t M,
             const bf16* __restrict__ W, bf16* __restrict__ dz_prev)
{
    extern __shared__ __align__(128) unsigned char dg_raw[];
    bf16* sW = reinterpret_cast<bf16*>(dg_raw);                                   // [128 x 128]
    float (*stage)[kSlab * kH] = reinterpret_cast<float (*)[kSlab * kH]>(dg_raw + kH * kH * 2);
    for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) sW[i] = W[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t slabs = (M + kSlab - 1) / kSlab;
    for (int64_t sl = (int64_t)blockIdx.x * kWarps + warp; sl < slabs;
         sl += (int64_t)gridDim.x * kWarps) {
        const int64_t r0 = sl * kSlab;
        const int rows = (int)lmin(kSlab, M - r0);
        wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) wmma::fill_fragment(acc[t], 0.0f);
        // rows past M read the zero padding the caller keeps after dz
#pragma unroll
        for (int kk = 0; kk < kH; kk += 16) {
            wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::row_major> a;
            wmma::load_matrix_sync(a, dz + (size_t)r0 * kH + kk, kH);
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                // (W^T)[kk.., 16 t..] = W[16 t.., kk..]^T: W read column-major
                wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::col_major> b;
                wmma::load_matrix_sync(b, sW + (16 * t) * kH + kk, kH);
                wmma::mma_sync(acc[t], a, b, acc[t]);
            }
        }
        float* st = stage[warp];
#pragma unroll
        for (int t = 0; t < 8; ++t) wmma::store_matrix_sync(st + 16 * t, acc[t], kH, wmma::mem_row_major);
        __syncwarp();
        for (int i = lane; i < rows * kH; i += 32) {
            const size_t gi = (size_t)r0 * kH + i;
            dz_prev[gi] = __float2bfloat16_rn(bf(a_prev[gi]) > 0.0f ? st[i] : 0.0f);
        }
        __syncwarp();
    }
}

// G_W += a^T dz over a chunk of rows (split-K), G_b += column sums of dz.
// a: [M x K] bf16, dz: [M x 128] bf16, both zero-padded to a multiple of 16
// rows.  Warp w owns output rows 16 w' for w' = w, w + 8, ... (< K / 16).
template <int K>
__global__ void __launch_bounds__(kWarps * 32)
wgrad_kernel(const bf16* __restrict__ a, const bf16* __restrict__ dz, int64_t M_pad,
             int64_t chunk, float* __restrict__ GW, float* __restrict__ Gb)
{
    __shared__ __align__(128) float stage[kWarps][16 * 16];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = (int64_t)blockIdx.x * chunk;
    const int64_t r1 = lmin(r0 + chunk, M_pad);
    for (int ot = warp; ot < K / 16; ot += kWarps) {
        wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) wmma::fill_fragment(acc[t], 0.0f);
        for (int64_t r = r0; r < r1; r += 16) {
            // (a^T)[16 ot.., r..] : a read column-major with ld K
            wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::col_major> fa;
            wmma::load_matrix_sync(fa, a + (size_t)r * K + 16 * ot, K);
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> fb;
                wmma::load_matrix_sync(fb, dz + (size_t)r * kH + 16 * t, kH);
                wmma::mma_sync(acc[t], fa, fb, acc[t]);
            }
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            wmma::store_matrix_sync(stage[warp], acc[t], 16, wmma::mem_row_major);
            __syncwarp();
            for (int i = lane; i < 256; i += 32)
                atomicAdd(&GW[(16 * ot + i / 16) * kH + 16 * t + (i % 16)], stage[warp][i]);
            __syncwarp();
        }
    }
    // bias: column sums of dz over the chunk
    for (int c = threadIdx.x; c < kH; c += blockDim.x) {
        float s = 0.0f;
        for (int64_t r = r0; r < r1; ++r) s += bf(dz[(size_t)r * kH + c]);
        atomicAdd(&Gb[c], s);
    }
}

// ---- optimiser and init ------------------------------------------------------------

// Adam (Kingma and Ba, 2015) on the float32 master parameters; refreshes
// the bfloat16 copies of the weights.
__global__ void adam_kernel(float* __restrict__ P, float* __restrict__ Mom, float* __restrict__ Vel,
                            const float* __restrict__ G, bf16* __restrict__ Wb, float lr,
                            float beta1, float beta2, float eps, float bc1, float bc2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kRankParams) return;
    const float g = G[i];
    const float m = beta1 * Mom[i] + (1.0f - beta1) * g;
    const float v = beta2 * Vel[i] + (1.0f - beta2) * g * g;
    Mom[i] = m;
    Vel[i] = v;
    const float p = P[i] - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
    P[i] = p;
    const int b = rank_bf16_index(i);
    if (b >= 0) Wb[b] = __float2bfloat16_rn(p);
}

__global__ void refresh_bf16_kernel(const float* __restrict__ P, bf16* __restrict__ Wb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kRankParams) return;
    const int b = rank_bf16_index(i);
    if (b >= 0) Wb[b] = __float2bfloat16_rn(P[i]);
}

// He-uniform weights from SplitMix64 (Steele, Lea and Flood 2014) of
// seed ^ index; zero biases.
__global__ void init_kernel(float* __restrict__ P, unsigned long long seed)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kRankParams) return;
    unsigned long long z = seed ^ ((unsigned long long)i * 0x9E3779B97F4A7C15ull);
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const float u = (float)(z >> 40) * (1.0f / 16777216.0f) * 2.0f - 1.0f;   // [-1, 1)
    float fan_in = 0.0f;
    if (i < kOffB1) fan_in = kF;
    else if ((i >= kOffW2 && i < kOffB2) || (i >= kOffW3 && i < kOffB3) ||
             (i >= kOffW4 && i < kOffB4))
        fan_in = kH;
    P[i] = fan_in > 0.0f ? u * sqrtf(6.0f / fan_in) : 0.0f;
}

}  // namespace

size_t ranker_forward_smem() { return sizeof(FwdShared); }

constexpr size_t kDgradSmem = (size_t)kH * kH * 2 + (size_t)kWarps * kSlab * kH * 4;

cudaError_t ranker_configure()
{
    cudaError_t e = cudaFuncSetAttribute(forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(FwdShared));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(dgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kDgradSmem);
}

cudaError_t ranker_init(float* P, bf16_raw* Wb, unsigned long long seed, cudaStream_t s)
{
    init_kernel<<<(kRankParams + 255) / 256, 256, 0, s>>>(P, seed);
    refresh_bf16_kernel<<<(kRankParams + 255) / 256, 256, 0, s>>>(P, reinterpret_cast<bf16*>(Wb));
    return cudaGetLastError();
}

cudaError_t ranker_refresh(const float* P, bf16_raw* Wb, cudaStream_t s)
{
    refresh_bf16_kernel<<<(kRankParams + 255) / 256, 256, 0, s>>>(P, reinterpret_cast<bf16*>(Wb));
    return cudaGetLastError();
}

cudaError_t ranker_forward(const bf16_raw* X, int64_t M, const bf16_raw* Wb, const float* P,
                           float* logits, bf16_raw* keep, int64_t keep_stride, int blocks,
                           cudaStream_t s)
{
    if (M <= 0) return cudaSuccess;
    forward_kernel<<<blocks, kWarps * 32, sizeof(FwdShared), s>>>(
        reinterpret_cast<const bf16*>(X), M, reinterpret_cast<const bf16*>(Wb), P, logits,
        reinterpret_cast<bf16*>(keep), keep_stride);
    return cudaGetLastError();
}

cudaError_t ranker_backward(const bf16_raw* X, int64_t M, const int32_t* off, const int32_t* target,
                            int S, const bf16_raw* Wb, const float* P, float* logits,
                            float* dlogit, bf16_raw* act, bf16_raw* dz, float* G, float* loss,
                            int blocks, cudaStream_t s)
{
    if (M <= 0 || S <= 0) return cudaErrorInvalidValue;
    const int64_t M_pad = (M + 15) / 16 * 16;
    bf16* a1 = reinterpret_cast<bf16*>(act);
    bf16* a2 = a1 + (size_t)M_pad * kH;
    bf16* a3 = a2 + (size_t)M_pad * kH;
    bf16* dzA = reinterpret_cast<bf16*>(dz);
    bf16* dzB = dzA + (size_t)M_pad * kH;
    const bf16* W = reinterpret_cast<const bf16*>(Wb);
    const bf16* x = reinterpret_cast<const bf16*>(X);
    cudaError_t e;
    if ((e = ranker_forward(X, M, Wb, P, logits, act, M_pad, blocks, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(loss, 0, sizeof(float), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(G, 0, kRankParams * sizeof(float), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(dlogit, 0, M * sizeof(float), s)) != cudaSuccess) return e;
    loss_kernel<<<(S + 127) / 128, 128, 0, s>>>(logits, M, off, target, S, dlogit, loss);
    head_backward_kernel<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(dlogit, a3, M, W, dzA, G);
    const int64_t chunk = 4096;
    const unsigned wblocks = (unsigned)((M_pad + chunk - 1) / chunk);
    wgrad_kernel<kH><<<wblocks, kWarps * 32, 0, s>>>(a2, dzA, M_pad, chunk, G + kOffW3, G + kOffB3);
    dgrad_kernel<<<blocks, kWarps * 32, kDgradSmem, s>>>(dzA, a2, M, W + kBfW3, dzB);
    wgrad_kernel<kH><<<wblocks, kWarps * 32, 0, s>>>(a1, dzB, M_pad, chunk, G + kOffW2, G + kOffB2);
    dgrad_kernel<<<blocks, kWarps * 32, kDgradSmem, s>>>(dzB, a1, M, W + kBfW2, dzA);
    wgrad_kernel<kF><<<wblocks, kWarps * 32, 0, s>>>(x, dzA, M_pad, chunk, G + kOffW1, G + kOffB1);
    return cudaGetLastError();
}

cudaError_t ranker_adam(float* P, float* Mom, float* Vel, const float* G, bf16_raw* Wb, float lr,
                        int step, cudaStream_t s)
{
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.0f - powf(b1, (float)step), bc2 = 1.0f - powf(b2, (float)step);
    adam_kernel<<<(kRankParams + 255) / 256, 256, 0, s>>>(P, Mom, Vel, G,
                                                          reinterpret_cast<bf16*>(Wb), lr, b1, b2,
                                                          1e-8f, bc1, bc2);
    return cudaGetLastError();
}

}  // namespace tmgpu
