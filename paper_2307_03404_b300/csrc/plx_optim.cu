// The paper's optimisers (Sec. 5.4): RMSProp on the grid values for mapping,
// Adam on the pose for tracking with rays sampled at random from the frame.
//
// RMSProp is one elementwise pass over the allocated vertices (it cannot ride
// on the adjoint's scatter: a gradient is final only once every ray is done):
// per value v <- alpha v + (1 - alpha) g^2, x <- x - lr g / (sqrt(v) + eps),
// reading and writing the record in its storage format and, on request,
// zeroing the gradient for the next step in the same pass.
//
// Adam tracking samples its rays with SplitMix64 (Steele, Lea and Flood, 2014)
// on a device-side iteration counter, so a whole tracking loop can be captured
// in one CUDA graph; the gradient is d loss / d xi = 2 J^T W r from the pose
// kernel, and the step exp(-lr m_hat / (sqrt(v_hat) + eps))^ is applied on the
// left of the pose.
#include "plx_internal.cuh"

namespace plx {

__device__ __forceinline__ float rms_update(float x, float g, float& v, float lr, float alpha,
                                            float eps) {
  v = fmaf(alpha, v, (1.f - alpha) * g * g);
  return x - lr * g / (sqrtf(v) + eps);
}

template <int STORE>
__global__ void k_rmsprop(void* __restrict__ rec, float* __restrict__ grad,
                          float* __restrict__ state, int64_t n, float lr_density, float lr_sh,
                          float alpha, float eps, int zero_grad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float4* g4 = reinterpret_cast<float4*>(grad + i * PLX_GRAD_STRIDE);
    float4* s4 = reinterpret_cast<float4*>(state + i * PLX_GRAD_STRIDE);
    float g[28], v[28], x[28];
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      const float4 a = g4[j], b = s4[j];
      g[4 * j] = a.x; g[4 * j + 1] = a.y; g[4 * j + 2] = a.z; g[4 * j + 3] = a.w;
      v[4 * j] = b.x; v[4 * j + 1] = b.y; v[4 * j + 2] = b.z; v[4 * j + 3] = b.w;
    }
    load_record<STORE>(rec, (int32_t)i, x);
#pragma unroll
    for (int j = 0; j < 28; ++j)
      x[j] = rms_update(x[j], g[j], v[j], j == 0 ? lr_density : lr_sh, alpha, eps);
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      s4[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
      if (zero_grad) g4[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if constexpr (STORE == PLX_STORE_F32) {
      float4* r4 = reinterpret_cast<float4*>(rec) + i * 8;
#pragma unroll
      for (int j = 0; j < 7; ++j) r4[j] = make_float4(x[4 * j], x[4 * j + 1], x[4 * j + 2], x[4 * j + 3]);
    } else {
      uint32_t w[14];
      if constexpr (STORE == PLX_STORE_F32_BF16) {
        w[0] = __float_as_uint(x[0]);
#pragma unroll
        for (int j = 0; j < 13; ++j)
          w[j + 1] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x[1 + 2 * j])) |
                     ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x[2 + 2 * j])) << 16);
        // slot 28 of the 16-bit record holds SH 26 alone; keep the pad half zero
        const uint32_t last = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x[27]));
        uint32_t* r = reinterpret_cast<uint32_t*>(rec) + i * 16;
#pragma unroll
        for (int j = 0; j < 14; ++j) r[j] = w[j];
        r[14] = last;
      } else {
#pragma unroll
        for (int j = 0; j < 14; ++j) {
          if constexpr (STORE == PLX_STORE_BF16)
            w[j] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x[2 * j])) |
                   ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x[2 * j + 1])) << 16);
          else
            w[j] = (uint32_t)__half_as_ushort(__float2half_rn(x[2 * j])) |
                   ((uint32_t)__half_as_ushort(__float2half_rn(x[2 * j + 1])) << 16);
        }
        uint32_t* r = reinterpret_cast<uint32_t*>(rec) + i * 16;
#pragma unroll
        for (int j = 0; j < 14; ++j) r[j] = w[j];
      }
    }
  }
}

void launch_rmsprop(int store, void* rec, float* grad, float* state, int64_t n, float lr_density,
                    float lr_sh, float alpha, float eps, int zero_grad, int num_sms,
                    cudaStream_t s) {
  if (n <= 0) return;
  const int64_t want = (n + 255) / 256;
  const unsigned blocks = (unsigned)(want < 16 * num_sms ? want : 16 * num_sms);
  switch (store) {
    case PLX_STORE_F32:
      k_rmsprop<PLX_STORE_F32><<<blocks, 256, 0, s>>>(rec, grad, state, n, lr_density, lr_sh, alpha, eps, zero_grad);
      break;
    case PLX_STORE_BF16:
      k_rmsprop<PLX_STORE_BF16><<<blocks, 256, 0, s>>>(rec, grad, state, n, lr_density, lr_sh, alpha, eps, zero_grad);
      break;
    case PLX_STORE_F16:
      k_rmsprop<PLX_STORE_F16><<<blocks, 256, 0, s>>>(rec, grad, state, n, lr_density, lr_sh, alpha, eps, zero_grad);
      break;
    default:
      k_rmsprop<PLX_STORE_F32_BF16><<<blocks, 256, 0, s>>>(rec, grad, state, n, lr_density, lr_sh,
                                                           alpha, eps, zero_grad);
      break;
  }
}

// ---------------------------------------------------------------- Adam
// state: m[0..5], v[6..11], t at [12] (iterations done), last step xi at
// [13..18]. g = 2 JtWr is the loss gradient with respect to a left
// perturbation of the pose.
__global__ void k_adam_pose(const double* __restrict__ JtWr, double* __restrict__ state,
                            double* __restrict__ pose, double lr, double b1, double b2,
                            double eps) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double t = state[12] + 1.0;
  double xi[6];
  for (int j = 0; j < 6; ++j) {
    const double g = 2.0 * JtWr[j];
    const double m = b1 * state[j] + (1.0 - b1) * g;
    const double v = b2 * state[6 + j] + (1.0 - b2) * g * g;
    state[j] = m;
    state[6 + j] = v;
    const double mh = m / (1.0 - pow(b1, t));
    const double vh = v / (1.0 - pow(b2, t));
    xi[j] = -lr * mh / (sqrt(vh) + eps);
  }
  state[12] = t;
  for (int j = 0; j < 6; ++j) state[13 + j] = xi[j];
  se3_exp_left(xi, pose);
}

void launch_adam_pose(const double* JtWr, double* state, double* pose, double lr, double b1,
                      double b2, double eps, cudaStream_t s) {
  k_adam_pose<<<1, 32, 0, s>>>(JtWr, state, pose, lr, b1, b2, eps);
}

}  // namespace plx
