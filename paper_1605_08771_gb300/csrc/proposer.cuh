// Learned m0 / node proposer: spectral-density moments and the MLP kernels.
#pragma once

#include "common.cuh"

namespace feast {

constexpr int kMlpLayers = 4;
constexpr int kMlpDims[kMlpLayers + 1] = {64, 256, 256, 256, 9};
constexpr int kMomentBlocks = 256;   // partial sums per moment (fixed order)

// FP32 parameters of the MLP (weights and biases of every layer).
size_t mlp_param_count();
// FP32 activations of a batch of B samples (input and every layer's output).
size_t mlp_act_floats(int64_t B);

// Chebyshev moments by the three-term recurrence on the probe block V
// (n x nv, ld n).  T0, T1, AT: n x nv scratch; partial: M x kMomentBlocks
// doubles receiving the partial sums of Re(v^H T_k v) (the caller adds each
// row in order and divides by n nv).
template <typename S>
void chebyshev_moments(const S* A, int64_t n, int64_t lda, double c, double r, const S* V, int64_t nv, int M,
                       S* T0, S* T1, S* AT, double* partial, double* mu, cudaStream_t s);

// acts: mlp_act_floats(B) floats; X (B x 64) is copied to its front and
// every layer's output follows; the network's output is the last B x 9.
void mlp_forward(const float* params, const float* X, int64_t B, float* acts, cudaStream_t s);
// Gradient of the mean squared error against T (B x 9) after mlp_forward:
// grad (mlp_param_count floats), dbuf0/dbuf1 (B x 256 scratch), sq (B x 9
// squared errors).
void mlp_backward(const float* params, const float* acts, const float* T, int64_t B, float* grad, float* dbuf0,
                  float* dbuf1, float* sq, cudaStream_t s);
// One Adam step (b1 = 0.9, b2 = 0.999, eps = 1e-8), step counted from 1.
void adam_update(float* params, const float* grad, float* m, float* v, int64_t count, int step, float lr,
                 cudaStream_t s);

}  // namespace feast
