// ranker.h -- layout constants and launchers of the learned order ranker
// (ranker.cu) and the beam search that uses it (beam.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace tmgpu {

typedef uint16_t bf16_raw;   // bfloat16 bits, as seen from host code

constexpr int kRankF = 32;    // features per candidate
constexpr int kRankH = 128;   // hidden width
// float32 parameter vector
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kRankF * kRankH;
constexpr int kOffW2 = kOffB1 + kRankH;
constexpr int kOffB2 = kOffW2 + kRankH * kRankH;
constexpr int kOffW3 = kOffB2 + kRankH;
constexpr int kOffB3 = kOffW3 + kRankH * kRankH;
constexpr int kOffW4 = kOffB3 + kRankH;
constexpr int kOffB4 = kOffW4 + kRankH;
constexpr int kRankParams = kOffB4 + 1;
// bfloat16 copies of the weights (biases stay float32)
constexpr int kBfW1 = 0;
constexpr int kBfW2 = kBfW1 + kRankF * kRankH;
constexpr int kBfW3 = kBfW2 + kRankH * kRankH;
constexpr int kBfW4 = kBfW3 + kRankH * kRankH;
constexpr int kRankBf16 = kBfW4 + kRankH;

// Index of parameter i in the bfloat16 copy, or -1 for a bias.
__host__ __device__ inline int rank_bf16_index(int i)
{
    if (i < kOffB1) return kBfW1 + (i - kOffW1);
    if (i >= kOffW2 && i < kOffB2) return kBfW2 + (i - kOffW2);
    if (i >= kOffW3 && i < kOffB3) return kBfW3 + (i - kOffW3);
    if (i >= kOffW4 && i < kOffB4) return kBfW4 + (i - kOffW4);
    return -1;
}

size_t ranker_forward_smem();
cudaError_t ranker_configure();
cudaError_t ranker_init(float* P, bf16_raw* Wb, unsigned long long seed, cudaStream_t s);
cudaError_t ranker_refresh(const float* P, bf16_raw* Wb, cudaStream_t s);
// logits[M] from X [M x 32]; with keep != nullptr also a1..a3 at keep +
// l * keep_stride * 128 (l = 0, 1, 2).
cudaError_t ranker_forward(const bf16_raw* X, int64_t M, const bf16_raw* Wb, const float* P,
                           float* logits, bf16_raw* keep, int64_t keep_stride, int blocks,
                           cudaStream_t s);
// Forward, softmax cross-entropy per state and backward into G (float32,
// kRankParams).  X, act (3 buffers) and dz (2 buffers) have M_pad =
// ceil16(M) rows whose tails beyond M the caller has zeroed.
cudaError_t ranker_backward(const bf16_raw* X, int64_t M, const int32_t* off,
                            const int32_t* target, int S, const bf16_raw* Wb, const float* P,
                            float* logits, float* dlogit, bf16_raw* act, bf16_raw* dz, float* G,
                            float* loss, int blocks, cudaStream_t s);
cudaError_t ranker_adam(float* P, float* Mom, float* Vel, const float* G, bf16_raw* Wb, float lr,
                        int step, cudaStream_t s);

// ranker_tc.cu: the inference forward pass on tcgen05 tensor cores.  It
// reads a weight image (ranker_image_bytes()) that ranker_image builds from
// the parameters; rebuild it after every parameter change.  *err is set to 1
// if a bounded wait of the kernel expired (its scores are then NaN).
size_t ranker_image_bytes();
cudaError_t ranker_image(const float* P, const bf16_raw* Wb, unsigned char* img, cudaStream_t s);
cudaError_t ranker_tc_configure();
// keep (may be null): also the hidden layers' bfloat16 activations, [3][M][128].
// pdl: launched as a programmatic dependent launch (its prologue, which
// reads only the weight image, overlaps the end of the kernel before).
cudaError_t ranker_forward_tc(const bf16_raw* X, int64_t M, const unsigned char* img,
                              float* logits, int* err, int blocks, cudaStream_t s,
                              bf16_raw* keep = nullptr, bool pdl = false);

}  // namespace tmgpu
