// mlp_internal.h -- learned early-stop network: sizes and launchers (k_mlp.cu).
#pragma once

#include <stdint.h>

#include <cuda_runtime.h>

namespace cng {

constexpr int MLP_NPARAMS = 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1;  // 5313
constexpr int MLP_NPARAMS_PAD = 5316;

size_t mlp_fwd_bwd_smem();
int mlp_parts(int B);
// Gradient of the mean loss over B rows (rows drawn by hash of (seed, step) when seed != 0,
// else rows 0..B-1).  part: mlp_parts(B) * MLP_NPARAMS floats; part_loss: mlp_parts(B).
cudaError_t launch_mlp_grad(const float* P, const float* X, const float* Y, int64_t N, int B,
                            uint64_t seed, int64_t step, float* part, float* part_loss, float* grad,
                            float* loss, cudaStream_t s);
cudaError_t launch_adam(float* P, float* m, float* v, const float* g, int64_t t, float lr,
                        cudaStream_t s);
cudaError_t launch_mlp_init(float* P, uint64_t seed, cudaStream_t s);
cudaError_t launch_pack_model(const float* P, const float* mu, const float* sg, void* blk,
                              cudaStream_t s);
cudaError_t launch_offsets(const int32_t* hops, int64_t nq, int T, int64_t* off, cudaStream_t s);
cudaError_t launch_samples(const float* feats, const int32_t* hops, const int32_t* tlc, int64_t nq,
                           int T, int64_t* off, float* X, float* y, cudaStream_t s);
// part: 64 * 32 doubles
cudaError_t launch_standardise(float* X, int64_t N, double* part, float* mu, float* sg,
                               cudaStream_t s);

}  // namespace cng
