// The paper's optimisers (Sec. 5.4): RMSProp on the grid values for mapping,
// Adam on the pose for tracking with rays sampled at random from the frame.
//
// RMSProp is one elementwise pass over the allocated vertices (it cannot ride
// on the adjoint's scatter: a gradient is final only once every ray is done),
// streamed so that consecutive threads touch consecutive 16-byte chunks:
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

// Streaming forms: the same update with consecutive threads on consecutive
// 16-byte chunks of the rows, so every warp load and store is contiguous.
// FP32 records: thread j takes chunk q = j mod 7 of vertex j / 7 (4 values of
// the record, the gradient and the state; the padding chunk 7 is skipped).
__global__ void k_rmsprop_f32(float4* __restrict__ rec, float4* __restrict__ grad,
                              float4* __restrict__ state, int64_t n, float lr_density, float lr_sh,
                              float alpha, float eps, int zero_grad) {
  const int64_t total = n * 7;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < total;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = j / 7;
    const int q = (int)(j - v * 7);
    const int64_t at = v * 8 + q;
    const float4 g = grad[at];
    float4 m = state[at];
    float4 x = rec[at];
    const float l0 = q == 0 ? lr_density : lr_sh;
    x.x = rms_update(x.x, g.x, m.x, l0, alpha, eps);
    x.y = rms_update(x.y, g.y, m.y, lr_sh, alpha, eps);
    x.z = rms_update(x.z, g.z, m.z, lr_sh, alpha, eps);
    x.w = rms_update(x.w, g.w, m.w, lr_sh, alpha, eps);
    state[at] = m;
    rec[at] = x;
    if (zero_grad) grad[at] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// 16-bit records (BF16 or FP16, 2 values per word): thread j takes the
// 16-byte record chunk q = j mod 4 of vertex j / 4 (values 8q .. 8q+7; for
// q = 3 only 24..27 are values, 28..31 padding kept at zero) and the matching
// two 16-byte chunks of the gradient and state rows.
template <int STORE>
__global__ void k_rmsprop_16(uint4* __restrict__ rec, float4* __restrict__ grad,
                             float4* __restrict__ state, int64_t n, float lr_density, float lr_sh,
                             float alpha, float eps, int zero_grad) {
  const int64_t total = n * 4;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < total;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = j >> 2;
    const int q = (int)(j & 3);
    const int64_t ga = v * 8 + 2 * q;  // first of the two gradient / state chunks
    const int nc = q < 3 ? 2 : 1;       // chunks holding values
    uint4 w = rec[j];
    uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h >= nc) break;
      const float4 g = grad[ga + h];
      float4 m = state[ga + h];
      float x[4], gg[4] = {g.x, g.y, g.z, g.w}, mm[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const uint32_t word = ww[2 * h + e];
        x[2 * e] = STORE == PLX_STORE_BF16 ? bf16_lo(word) : f16_lo(word);
        x[2 * e + 1] = STORE == PLX_STORE_BF16 ? bf16_hi(word) : f16_hi(word);
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float lr = (q == 0 && h == 0 && e == 0) ? lr_density : lr_sh;
        x[e] = rms_update(x[e], gg[e], mm[e], lr, alpha, eps);
      }
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        if constexpr (STORE == PLX_STORE_BF16)
          ww[2 * h + e] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x[2 * e])) |
                          ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x[2 * e + 1])) << 16);
        else
          ww[2 * h + e] = (uint32_t)__half_as_ushort(__float2half_rn(x[2 * e])) |
                          ((uint32_t)__half_as_ushort(__float2half_rn(x[2 * e + 1])) << 16);
      }
      state[ga + h] = make_float4(mm[0], mm[1], mm[2], mm[3]);
      if (zero_grad) grad[ga + h] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    rec[j] = make_uint4(ww[0], ww[1], ww[2], ww[3]);
  }
}

void launch_rmsprop(int store, void* rec, float* grad, float* state, int64_t n, float lr_density,
                    float lr_sh, float alpha, float eps, int zero_grad, int num_sms,
                    cudaStream_t s) {
  if (n <= 0) return;
  const int64_t want = (n + 255) / 256;
  const unsigned blocks = (unsigned)(want < 16 * num_sms ? want : 16 * num_sms);
  const int64_t chunks = store == PLX_STORE_F32 ? n * 7 : n * 4;
  const int64_t want_s = (chunks + 255) / 256;
  const unsigned sblocks = (unsigned)(want_s < 16 * num_sms ? want_s : 16 * num_sms);
  switch (store) {
    case PLX_STORE_F32:
      k_rmsprop_f32<<<sblocks, 256, 0, s>>>(reinterpret_cast<float4*>(rec),
                                            reinterpret_cast<float4*>(grad),
                                            reinterpret_cast<float4*>(state), n, lr_density, lr_sh,
                                            alpha, eps, zero_grad);
      break;
    case PLX_STORE_BF16:
      k_rmsprop_16<PLX_STORE_BF16><<<sblocks, 256, 0, s>>>(
          reinterpret_cast<uint4*>(rec), reinterpret_cast<float4*>(grad),
          reinterpret_cast<float4*>(state), n, lr_density, lr_sh, alpha, eps, zero_grad);
      break;
    case PLX_STORE_F16:
      k_rmsprop_16<PLX_STORE_F16><<<sblocks, 256, 0, s>>>(
          reinterpret_cast<uint4*>(rec), reinterpret_cast<float4*>(grad),
          reinterpret_cast<float4*>(state), n, lr_density, lr_sh, alpha, eps, zero_grad);
      break;
    default:  // FP32 density + BF16 SH: values straddle the chunks, one vertex per thread
      k_rmsprop<PLX_STORE_F32_BF16><<<blocks, 256, 0, s>>>(rec, grad, state, n, lr_density, lr_sh,
                                                           alpha, eps, zero_grad);
      break;
  }
}

// ------------------------------------------------ random rays, image order
// The n pixels of Adam iteration t (pixel splitmix64(seed, t n + i) mod W H,
// the same set as drawn inline) put in the Z-order of (u, v) by a bitonic sort
// in shared memory, so that a warp's rays are image neighbours: they share grid
// lines and take similar paths. One block; n <= kMaxSortedRays.
__device__ __forceinline__ uint32_t spread_bits16(uint32_t a) {
  a &= 0xFFFFu;
  a = (a | (a << 8)) & 0x00FF00FFu;
  a = (a | (a << 4)) & 0x0F0F0F0Fu;
  a = (a | (a << 2)) & 0x33333333u;
  a = (a | (a << 1)) & 0x55555555u;
  return a;
}

__device__ __forceinline__ uint32_t compact_bits16(uint32_t a) {
  a &= 0x55555555u;
  a = (a | (a >> 1)) & 0x33333333u;
  a = (a | (a >> 2)) & 0x0F0F0F0Fu;
  a = (a | (a >> 4)) & 0x00FF00FFu;
  a = (a | (a >> 8)) & 0x0000FFFFu;
  return a;
}

__global__ void k_random_pixels_sorted(uint64_t seed, const double* __restrict__ iter, int n,
                                       int width, int height, int32_t* __restrict__ out) {
  __shared__ uint32_t keys[kMaxSortedRays];
  const uint64_t t = (uint64_t)*iter;
  const uint64_t npx = (uint64_t)width * height;
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    uint32_t key = 0xFFFFFFFFu;  // padding sorts last
    if (i < n) {
      const uint32_t pix = (uint32_t)(splitmix64(seed, t * (uint64_t)n + (uint64_t)i) % npx);
      const uint32_t u = pix % (uint32_t)width, v = pix / (uint32_t)width;
      key = spread_bits16(u) | (spread_bits16(v) << 1);
    }
    keys[i] = key;
  }
  __syncthreads();
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const uint32_t a = keys[i], b = keys[ixj];
          if ((a > b) == ((i & k) == 0)) {
            keys[i] = b;
            keys[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const uint32_t key = keys[i];
    out[i] = (int32_t)(compact_bits16(key >> 1) * (uint32_t)width + compact_bits16(key));
  }
}

void launch_random_pixels_sorted(uint64_t seed, const double* iter, int n, int width, int height,
                                 int32_t* out, cudaStream_t s) {
  k_random_pixels_sorted<<<1, 1024, 0, s>>>(seed, iter, n, width, height, out);
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
  // bias corrections 1 - b^t; t is an integer, so b^t by repeated squaring
  // (a few multiplications instead of a transcendental pow per component)
  double p1 = 1.0, p2 = 1.0, s1 = b1, s2 = b2;
  for (uint64_t e = (uint64_t)t; e; e >>= 1) {
    if (e & 1) {
      p1 *= s1;
      p2 *= s2;
    }
    s1 *= s1;
    s2 *= s2;
  }
  const double c1 = 1.0 / (1.0 - p1), c2 = 1.0 / (1.0 - p2);
  double xi[6];
  for (int j = 0; j < 6; ++j) {
    const double g = 2.0 * JtWr[j];
    const double m = b1 * state[j] + (1.0 - b1) * g;
    const double v = b2 * state[6 + j] + (1.0 - b2) * g * g;
    state[j] = m;
    state[6 + j] = v;
    xi[j] = -lr * (m * c1) / (sqrt(v * c2) + eps);
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
