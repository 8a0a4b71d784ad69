// Learned MDF initializer: sizes and launchers (internal to libibmlbm.so).
#pragma once

#include <cuda_fp16.h>

#include "common.cuh"

namespace ibmlbm {

constexpr int kMlpIn = 27, kMlpH = 64, kMlpOut = 3;
constexpr int kMlpParams = kMlpIn * kMlpH + kMlpH + kMlpH * kMlpH + kMlpH + kMlpH * kMlpOut + kMlpOut + 2;

size_t mlp_scratch_floats(int batch);
cudaError_t launch_mlp_samples(const IbmArgs& A, float* X, float* Y, cudaStream_t s);
cudaError_t launch_mlp_step(const IbmArgs& A, const float* P, const void* img, cudaStream_t s);
size_t mlp_image_bytes();  // shared-memory image of the weights
cudaError_t launch_mlp_image(const float* P, void* img, cudaStream_t s);
int mlp_max_points();  // points per particle the step kernel supports
cudaError_t launch_mlp_infer(const float* P, const float* X, long long n, float* Y, cudaStream_t s);
cudaError_t launch_mlp_grad(const float* P, const float* X, const float* T, int batch, float* G,
                            double* d_loss, float* scratch, cudaStream_t s);
cudaError_t launch_mlp_adam(float* P, const float* G, float* M, float* V, long long t, float lr,
                            cudaStream_t s);

}  // namespace ibmlbm
