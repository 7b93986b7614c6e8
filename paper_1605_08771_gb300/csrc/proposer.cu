// Kernels of the learned m0 / node proposer (spectrum estimation ahead of the
// solve, which the paper names as future work in Sect. IV):
//
//  * stochastic-trace Chebyshev moments of the spectral density:
//    mu_k = (1/(n nv)) sum_v Re(v^H T_k(B) v), B = (A - c I)/r, by the
//    three-term recurrence t_{k+1} = 2 B t_k - t_{k-1} on a block of nv probe
//    vectors (the products A t_k by the library's FP64 GEMM, the recurrence
//    update and the probe dot products fused in one kernel);
//  * a 64 -> 256 -> 256 -> 256 -> 9 ReLU multilayer perceptron in FP32:
//    forward, backward (mean squared error) and the Adam update, one kernel
//    per layer and direction.
//
// Parameter layout (one contiguous FP32 array): for each layer l in order,
// W_l (d_out x d_in, row major: W_l[o * d_in + i]) followed by b_l (d_out).
// Activations are row major, one row per sample.
#include <cmath>
#include <vector>

#include "gemm.cuh"
#include "proposer.cuh"

namespace feast {

namespace {

template <typename S>
__global__ void cheb_step_kernel(S* Tprev, const S* T, const S* AT, const S* V, int64_t n, int64_t nv, double c,
                                 double r, int first, double* partial) {
  // first: T_1 = (A - c) T_0 / r (Tprev unused on input); else
  // T_{k+1} = 2 (A T_k - c T_k)/r - T_{k-1}, written over T_{k-1}
  __shared__ double red[8];
  const int64_t total = n * nv;
  double acc = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    S x = (AT[t] - c * T[t]) * (1.0 / r);
    if (!first) x = 2.0 * x - Tprev[t];
    Tprev[t] = x;
    acc += real_part(conj(V[t]) * x);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    partial[blockIdx.x] = s;
  }
}

template <typename S>
__global__ void dot_re_kernel(const S* V, const S* T, int64_t total, double* partial) {
  __shared__ double red[8];
  double acc = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
    acc += real_part(conj(V[t]) * T[t]);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    partial[blockIdx.x] = s;
  }
}

constexpr int kDotBlocks = kMomentBlocks;

// ---- MLP ----
// Y[b, o] = act(sum_i X[b, i] W[o, i] + bias[o]); one thread per output
__global__ void dense_fwd_kernel(const float* __restrict__ X, const float* __restrict__ W,
                                 const float* __restrict__ bias, float* __restrict__ Y, int64_t B, int din, int dout,
                                 int relu) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * dout) return;
  const int64_t b = t / dout;
  const int o = (int)(t % dout);
  const float* x = X + b * din;
  const float* w = W + (int64_t)o * din;
  float acc = bias[o];
  for (int i = 0; i < din; ++i) acc = fmaf(x[i], w[i], acc);
  Y[t] = relu ? fmaxf(acc, 0.f) : acc;
}

// delta of the output layer of the mean squared error: 2 (Y - T) / (B d),
// and the per-sample squared errors for the loss
__global__ void mse_delta_kernel(const float* Y, const float* T, float* D, float* sq, int64_t total, float scale) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const float e = Y[t] - T[t];
  D[t] = scale * e;
  sq[t] = e * e;
}

// dW[o, i] = sum_b D[b, o] X[b, i]; db[o] = sum_b D[b, o]; one thread per
// weight (and the bias with i == din)
__global__ void dense_wgrad_kernel(const float* __restrict__ D, const float* __restrict__ X, float* __restrict__ dW,
                                   float* __restrict__ db, int64_t B, int din, int dout) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)dout * (din + 1)) return;
  const int o = (int)(t / (din + 1));
  const int i = (int)(t % (din + 1));
  float acc = 0.f;
  if (i < din) {
    for (int64_t b = 0; b < B; ++b) acc = fmaf(D[b * dout + o], X[b * din + i], acc);
    dW[(int64_t)o * din + i] = acc;
  } else {
    for (int64_t b = 0; b < B; ++b) acc += D[b * dout + o];
    db[o] = acc;
  }
}

// Dprev[b, i] = (sum_o D[b, o] W[o, i]) * (H[b, i] > 0), H the layer's input
// (the previous layer's ReLU output)
__global__ void dense_bgrad_kernel(const float* __restrict__ D, const float* __restrict__ W,
                                   const float* __restrict__ H, float* __restrict__ Dprev, int64_t B, int din,
                                   int dout) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * din) return;
  const int64_t b = t / din;
  const int i = (int)(t % din);
  float acc = 0.f;
  for (int o = 0; o < dout; ++o) acc = fmaf(D[b * dout + o], W[(int64_t)o * din + i], acc);
  Dprev[t] = H[t] > 0.f ? acc : 0.f;
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int64_t count, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const float gt = g[t];
  const float mt = b1 * m[t] + (1.f - b1) * gt;
  const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
  m[t] = mt;
  v[t] = vt;
  p[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

unsigned blocks_for(int64_t total, int threads = 256) {
  return (unsigned)std::max<int64_t>(1, cdiv(total, threads));
}

}  // namespace

size_t mlp_param_count() {
  size_t c = 0;
  for (int l = 0; l < kMlpLayers; ++l) c += (size_t)kMlpDims[l + 1] * (kMlpDims[l] + 1);
  return c;
}

size_t mlp_act_floats(int64_t B) {
  size_t c = 0;
  for (int l = 0; l <= kMlpLayers; ++l) c += (size_t)B * kMlpDims[l];
  return c;
}

template <typename S>
void chebyshev_moments(const S* A, int64_t n, int64_t lda, double c, double r, const S* V, int64_t nv, int M,
                       S* T0, S* T1, S* AT, double* partial, double* mu, cudaStream_t s) {
  // mu[k] = partial sums of block k; the host adds them in order
  const int64_t total = n * nv;
  const unsigned blocks = (unsigned)std::min<int64_t>(kDotBlocks, std::max<int64_t>(1, cdiv(total, 256)));
  FEAST_CUDA_TRY(cudaMemsetAsync(partial, 0, sizeof(double) * kDotBlocks * M, s));
  FEAST_CUDA_TRY(cudaMemcpyAsync(T0, V, sizeof(S) * total, cudaMemcpyDeviceToDevice, s));
  dot_re_kernel<S><<<blocks, 256, 0, s>>>(V, T0, total, partial);
  FEAST_LAUNCH_CHECK();
  S* Tk = T0;     // T_k
  S* Tkm = T1;    // T_{k-1}, overwritten by T_{k+1}
  for (int k = 1; k < M; ++k) {
    gemm_simple<S, S, S>(n, nv, n, C1(1.0), A, lda, OP_N, Tk, n, OP_N, C1(0.0), AT, n, s);
    cheb_step_kernel<S><<<blocks, 256, 0, s>>>(Tkm, Tk, AT, V, n, nv, c, r, k == 1 ? 1 : 0,
                                               partial + (int64_t)k * kDotBlocks);
    FEAST_LAUNCH_CHECK();
    std::swap(Tk, Tkm);
  }
  (void)mu;
}

void mlp_forward(const float* params, const float* X, int64_t B, float* acts, cudaStream_t s) {
  // acts: X copied in front, then every layer's output
  FEAST_CUDA_TRY(cudaMemcpyAsync(acts, X, sizeof(float) * B * kMlpDims[0], cudaMemcpyDeviceToDevice, s));
  const float* p = params;
  float* in = acts;
  for (int l = 0; l < kMlpLayers; ++l) {
    const int din = kMlpDims[l], dout = kMlpDims[l + 1];
    float* out = in + B * din;
    dense_fwd_kernel<<<blocks_for(B * dout), 256, 0, s>>>(in, p, p + (int64_t)dout * din, out, B, din, dout,
                                                          l + 1 < kMlpLayers ? 1 : 0);
    FEAST_LAUNCH_CHECK();
    p += (int64_t)dout * (din + 1);
    in = out;
  }
}

void mlp_backward(const float* params, const float* acts, const float* T, int64_t B, float* grad, float* dbuf0,
                  float* dbuf1, float* sq, cudaStream_t s) {
  // parameter offsets of each layer
  int64_t off[kMlpLayers + 1];
  off[0] = 0;
  for (int l = 0; l < kMlpLayers; ++l) off[l + 1] = off[l] + (int64_t)kMlpDims[l + 1] * (kMlpDims[l] + 1);
  int64_t aoff[kMlpLayers + 1];
  aoff[0] = 0;
  for (int l = 0; l < kMlpLayers; ++l) aoff[l + 1] = aoff[l] + B * kMlpDims[l];
  const int dlast = kMlpDims[kMlpLayers];
  const float* Y = acts + aoff[kMlpLayers];
  mse_delta_kernel<<<blocks_for(B * dlast), 256, 0, s>>>(Y, T, dbuf0, sq, B * dlast, 2.f / (float)(B * dlast));
  FEAST_LAUNCH_CHECK();
  float* D = dbuf0;
  float* Dn = dbuf1;
  for (int l = kMlpLayers - 1; l >= 0; --l) {
    const int din = kMlpDims[l], dout = kMlpDims[l + 1];
    const float* X = acts + aoff[l];
    float* dW = grad + off[l];
    dense_wgrad_kernel<<<blocks_for((int64_t)dout * (din + 1)), 256, 0, s>>>(D, X, dW, dW + (int64_t)dout * din, B,
                                                                             din, dout);
    FEAST_LAUNCH_CHECK();
    if (l > 0) {
      dense_bgrad_kernel<<<blocks_for(B * din), 256, 0, s>>>(D, params + off[l], X, Dn, B, din, dout);
      FEAST_LAUNCH_CHECK();
      std::swap(D, Dn);
    }
  }
}

void adam_update(float* params, const float* grad, float* m, float* v, int64_t count, int step, float lr,
                 cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<blocks_for(count), 256, 0, s>>>(params, grad, m, v, count, lr, b1, b2, eps, c1, c2);
  FEAST_LAUNCH_CHECK();
}

template void chebyshev_moments<double>(const double*, int64_t, int64_t, double, double, const double*, int64_t, int,
                                        double*, double*, double*, double*, double*, cudaStream_t);
template void chebyshev_moments<c128>(const c128*, int64_t, int64_t, double, double, const c128*, int64_t, int,
                                      c128*, c128*, c128*, double*, double*, cudaStream_t);

}  // namespace feast
