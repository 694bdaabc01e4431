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

// The forward pass keeps each warp's 16 rows in registers from the input to
// the logit: mma.sync m16n8k16 (bf16 in, f32 accumulate).  The f32
// accumulator fragment of an output n-tile pair has exactly the register
// layout of the bf16 A fragment of the next layer's k-tile (PTX ISA,
// "Matrix fragments for mma.m16n8k16"), so bias, ReLU and the bfloat16
// rounding happen in registers and no activation goes through shared
// memory.  Weights sit in shared memory transposed (n-major, rows padded by
// 16 bytes so that ldmatrix is free of bank conflicts); one ldmatrix.x4
// gives the B fragments of two n-tiles.
//
// Fragment coordinates, with g = lane / 4 and t = lane % 4:
//   A (16 x 16): reg0 = (g, 2t..2t+1), reg1 = (g+8, 2t..), reg2 = (g, 8+2t..),
//                reg3 = (g+8, 8+2t..)
//   C (16 x 8):  c0, c1 = (g, 2t..2t+1), c2, c3 = (g+8, 2t..2t+1)
// The first layer reads each row's 32 features with one 16-byte load per
// thread: thread t takes features 8t .. 8t+7, which it feeds to the mma as
// k = 16 kt + 8 h + 2t + j  <->  feature 8t + 4 kt + 2 h + j  (j, h in {0, 1});
// the rows of W1 are stored in that order.

constexpr int kW1Ld = kF + 8;     // padded row length (elements) of W1^T in shared memory
constexpr int kWLd = kH + 8;      // ... of W2^T and W3^T

struct __align__(16) FwdShared {
    bf16 W1t[kH * kW1Ld];
    bf16 W2t[kH * kWLd];
    bf16 W3t[kH * kWLd];
    float b1[kH], b2[kH], b3[kH], w4[kH];
    float b4;
};

__device__ __forceinline__ float bf(const bf16 v) { return __bfloat162float(v); }
__host__ __device__ __forceinline__ int64_t lmin(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                        uint32_t& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// acc[16 n-tiles][4] += A (16 x 16 KT) x W^T-tile, W^T in shared memory at
// `wt` with row length ld (elements).
template <int KT>
__device__ __forceinline__ void layer_mma(float (&acc)[16][4], const uint32_t (&A)[KT][4],
                                          uint32_t wt, int ld, int lane)
{
    // lanes 0-7 / 8-15 / 16-23 / 24-31 address the rows of the four 8x8
    // matrices: (n-tile 2p, k 0-7), (2p, k 8-15), (2p+1, k 0-7), (2p+1, k 8-15)
    const int n_in = (lane & 7) + ((lane >> 4) << 3);
    const int k_in = ((lane >> 3) & 1) * 8;
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            uint32_t b0, b1, b2, b3;
            ldsm_x4(wt + (uint32_t)(((16 * p + n_in) * ld + 16 * kt + k_in) * 2), b0, b1, b2, b3);
            mma_bf16(acc[2 * p], A[kt], b0, b1);
            mma_bf16(acc[2 * p + 1], A[kt], b2, b3);
        }
    }
}

// Bias + ReLU + bfloat16 rounding of a 16 x 128 accumulator into the A
// fragments of the next layer (and the kept activations, row-major, when
// `keep` is set).
__device__ __forceinline__ void layer_epilogue(float (&acc)[16][4], const float* __restrict__ bias,
                                               uint32_t (&A)[8][4], bf16* __restrict__ keep,
                                               int rows, int lane)
{
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const float bl = bias[8 * j + 2 * t], bh = bias[8 * j + 2 * t + 1];
        const uint32_t top = pack_bf16(fmaxf(acc[j][0] + bl, 0.f), fmaxf(acc[j][1] + bh, 0.f));
        const uint32_t bot = pack_bf16(fmaxf(acc[j][2] + bl, 0.f), fmaxf(acc[j][3] + bh, 0.f));
        A[j >> 1][(j & 1) * 2] = top;
        A[j >> 1][(j & 1) * 2 + 1] = bot;
        if (keep) {
            if (g < rows) *reinterpret_cast<uint32_t*>(keep + (size_t)g * kH + 8 * j + 2 * t) = top;
            if (g + 8 < rows)
                *reinterpret_cast<uint32_t*>(keep + (size_t)(g + 8) * kH + 8 * j + 2 * t) = bot;
        }
    }
}

// logits[r] for rows r < M of X; with keep != null also stores a1, a2, a3
// ([stride x 128] each, at keep + l * stride * 128).  Persistent: each warp
// takes 16-row slabs in turn.
__global__ void __launch_bounds__(kWarps * 32, 2)
forward_kernel(const bf16* __restrict__ X, int64_t M, const bf16* __restrict__ Wb,
               const float* __restrict__ P, float* __restrict__ logits, bf16* __restrict__ keep,
               int64_t stride)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FwdShared& s = *reinterpret_cast<FwdShared*>(smem_raw);
    // W1 (in x out) -> W1^T with the input features permuted (see above)
    for (int i = threadIdx.x; i < kF * kH; i += blockDim.x) {
        const int k = i / kH, n = i - k * kH;          // W1[k][n], k a feature
        const int tt = k >> 3, r = k & 7;               // feature 8 tt + r
        const int kt = r >> 2, h = (r >> 1) & 1, j = r & 1;
        s.W1t[n * kW1Ld + 16 * kt + 8 * h + 2 * tt + j] = Wb[kBfW1 + i];
    }
    for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) {
        const int k = i / kH, n = i - k * kH;
        s.W2t[n * kWLd + k] = Wb[kBfW2 + i];
        s.W3t[n * kWLd + k] = Wb[kBfW3 + i];
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
    const int g = lane >> 2, t = lane & 3;
    const uint32_t w1 = (uint32_t)__cvta_generic_to_shared(s.W1t);
    const uint32_t w2 = (uint32_t)__cvta_generic_to_shared(s.W2t);
    const uint32_t w3 = (uint32_t)__cvta_generic_to_shared(s.W3t);
    const int64_t slabs = (M + kSlab - 1) / kSlab;
    for (int64_t sl = (int64_t)blockIdx.x * kWarps + warp; sl < slabs;
         sl += (int64_t)gridDim.x * kWarps) {
        const int64_t r0 = sl * kSlab;
        const int rows = (int)lmin(kSlab, M - r0);
        // layer 1 A fragments straight from global memory
        uint4 top = make_uint4(0, 0, 0, 0), bot = make_uint4(0, 0, 0, 0);
        if (g < rows) top = *reinterpret_cast<const uint4*>(X + (size_t)(r0 + g) * kF + 8 * t);
        if (g + 8 < rows) bot = *reinterpret_cast<const uint4*>(X + (size_t)(r0 + g + 8) * kF + 8 * t);
        uint32_t A1[2][4] = {{top.x, bot.x, top.y, bot.y}, {top.z, bot.z, top.w, bot.w}};
        float acc[16][4];
        uint32_t A[8][4];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
        layer_mma<2>(acc, A1, w1, kW1Ld, lane);
        layer_epilogue(acc, s.b1, A, keep ? keep + (size_t)r0 * kH : nullptr, rows, lane);
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
        layer_mma<8>(acc, A, w2, kWLd, lane);
        layer_epilogue(acc, s.b2, A, keep ? keep + ((size_t)stride + r0) * kH : nullptr, rows, lane);
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
        layer_mma<8>(acc, A, w3, kWLd, lane);
        layer_epilogue(acc, s.b3, A, keep ? keep + (2 * (size_t)stride + r0) * kH : nullptr, rows,
                       lane);
        // head: a3 . w4 over this thread's columns, then over the 4 threads of a row
        float lo = 0.f, hi = 0.f;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const __nv_bfloat162 vt = *reinterpret_cast<const __nv_bfloat162*>(&A[j >> 1][(j & 1) * 2]);
            const __nv_bfloat162 vb =
                *reinterpret_cast<const __nv_bfloat162*>(&A[j >> 1][(j & 1) * 2 + 1]);
            const float wl = s.w4[8 * j + 2 * t], wh = s.w4[8 * j + 2 * t + 1];
            lo += __low2float(vt) * wl + __high2float(vt) * wh;
            hi += __low2float(vb) * wl + __high2float(vb) * wh;
        }
        lo += __shfl_xor_sync(0xFFFFFFFFu, lo, 1);
        lo += __shfl_xor_sync(0xFFFFFFFFu, lo, 2);
        hi += __shfl_xor_sync(0xFFFFFFFFu, hi, 1);
        hi += __shfl_xor_sync(0xFFFFFFFFu, hi, 2);
        if (t == 0) {
            if (g < rows) logits[r0 + g] = lo + s.b4;
            if (g + 8 < rows) logits[r0 + g + 8] = hi + s.b4;
        }
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
