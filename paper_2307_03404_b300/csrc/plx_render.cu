// Forward render (Sec. 4, Eq. 1-3) and mapping adjoint (Sec. 5.2, Eq. 4-11).
//
// Forward: one thread per ray, samples marched front to back with the
// transmittance carried multiplicatively; the 8 corners of the current cell
// live in registers (density + view-projected colour), reloaded only when the
// sample leaves the cell.
//
// Adjoint: the ray is marched again with the forward's C and D, recomputing
// T_i, T_{i+1}, w_i and the inclusive prefix sums S_i = sum_{j<=i} w_j c_j,
// SD_i = sum_{j<=i} w_j t_j (nothing per sample is stored between the two
// passes). Per sample, Eq. 8 gives dL/dc_i = g_C w_i and Eq. 9-10 give
//   dL/dsigma_i = g_C . delta (c_i T_{i+1} - C + S_i) + g_D delta (t_i T_{i+1} - D + SD_i).
// The gradients are accumulated per corner in registers while the ray stays in
// one cell, as (d density, d projected colour per channel); SH gradients are
// recovered at flush time as d colour_ch * Y_k(d), because the SH basis
// depends on the ray only. A flush is 7 vector atomics (float4) per allocated
// corner into the 128-byte gradient row of the vertex; when the ray steps into
// a face-adjacent cell the 4 shared corners are carried instead of flushed.
#include "plx_internal.cuh"

namespace plx {

template <int STORE, bool COUNT>
__device__ __forceinline__ void march_forward(const Common& P, const RayF& r, const float Y[9],
                                              float C[3], float& D, float& T, int& n_all,
                                              int& n_occ) {
  const int rm2x = P.g.rx - 2, rm2y = P.g.ry - 2, rm2z = P.g.rz - 2;
  int cx = -1, cy = -1, cz = -1;
  bool empty = true;
  int32_t l[8];
  float cs[8], cc[8][3];
  C[0] = C[1] = C[2] = 0.f;
  D = 0.f;
  T = 1.f;
  n_all = r.n;
  for (int k = 0; k < r.n; ++k) {
    const float kf = (float)k;
    int ix, iy, iz;
    float fx, fy, fz;
    sample_axis(r.bh[0], r.bl[0], r.sh[0], r.sl[0], kf, rm2x, ix, fx);
    sample_axis(r.bh[1], r.bl[1], r.sh[1], r.sl[1], kf, rm2y, iy, fy);
    sample_axis(r.bh[2], r.bl[2], r.sh[2], r.sl[2], kf, rm2z, iz, fz);
    if (ix != cx || iy != cy || iz != cz) {
      cx = ix; cy = iy; cz = iz;
      if (block_empty(P.g, ix, iy, iz)) {
        empty = true;
        k = block_exit(r, ix, iy, iz, k) - 1;
        continue;
      }
      empty = load_cell<STORE>(P.g, ix, iy, iz, Y, l, cs, cc);
    }
    if (COUNT) n_occ += empty ? 0 : 1;
    if (empty) continue;
    float w[8];
    corner_weights(fx, fy, fz, w);
    float sig = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) sig = fmaf(w[c], cs[c], sig);
    if (!(sig > 0.f)) continue;
    float col[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      float a = 0.f;
#pragma unroll
      for (int c = 0; c < 8; ++c) a = fmaf(w[c], cc[c][ch], a);
      float dact;
      col[ch] = activate(a, P.o.color_act, dact);
    }
    float alpha, keep;
    alpha_of(sig * r.dt, alpha, keep);
    const float wgt = T * alpha;
    const float t = fmaf(kf, r.dt, r.t0);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) C[ch] = fmaf(wgt, col[ch], C[ch]);
    D = fmaf(wgt, t, D);
    T *= keep;
    if (T < P.o.stop_T) {
      n_all = k + 1;
      break;
    }
  }
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) C[ch] = fmaf(T, P.o.bg[ch], C[ch]);
}

template <int STORE, bool COUNT>
__global__ void __launch_bounds__(kBlock, PLX_FWD_MIN_BLOCKS)
k_forward(const __grid_constant__ Common P, float* __restrict__ rgb, float* __restrict__ depth,
          float* __restrict__ state, int32_t* __restrict__ counts) {
  const int lane = threadIdx.x & 31;
  const int64_t tile = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (tile >= P.ct.n_tiles) return;  // whole warps only
  const RayId id = ray_of(P, tile, lane);
  RayF r;
  setup_ray(P, id, r, lane);
  if (!id.valid) {
    if (!P.ct.dense && id.out < P.ct.n_rays) {  // bad list entry: loud NaN output
      const float nan = __int_as_float(0x7fc00000);
      rgb[3 * id.out] = rgb[3 * id.out + 1] = rgb[3 * id.out + 2] = nan;
      depth[id.out] = nan;
    }
    return;
  }
  float Y[9];
  sh_basis(r.dir, Y);
  float C[3], D, T;
  int n_all = 0, n_occ = 0;
  march_forward<STORE, COUNT>(P, r, Y, C, D, T, n_all, n_occ);
  rgb[3 * id.out] = C[0];
  rgb[3 * id.out + 1] = C[1];
  rgb[3 * id.out + 2] = C[2];
  depth[id.out] = D;
  if (state) state[id.out] = T;
  if (COUNT) {
    counts[2 * id.out] = n_all;
    counts[2 * id.out + 1] = n_occ;
  }
}

// ------------------------------------------------------------------ adjoint
__device__ __forceinline__ void flush_corner(float* __restrict__ grad, int32_t link, float gs,
                                             const float gc[3], const float Y[9]) {
  if (link < 0) return;
  float v[28];
  v[0] = gs;
#pragma unroll
  for (int ch = 0; ch < 3; ++ch)
#pragma unroll
    for (int k = 0; k < 9; ++k) v[1 + 9 * ch + k] = gc[ch] * Y[k];
  float4* dst = reinterpret_cast<float4*>(grad + (int64_t)link * PLX_GRAD_STRIDE);
#pragma unroll
  for (int j = 0; j < 7; ++j)
    atomicAdd(dst + j, make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]));
}

__device__ __forceinline__ void clear_corner(float& gs, float gc[3]) {
  gs = 0.f;
  gc[0] = gc[1] = gc[2] = 0.f;
}

__device__ __forceinline__ void flush_cell(float* __restrict__ grad, const int32_t l[8],
                                           float gs[8], float gc[8][3], const float Y[9]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    flush_corner(grad, l[c], gs[c], gc[c], Y);
    clear_corner(gs[c], gc[c]);
  }
}

// The ray steps into the face-adjacent cell along corner bit B (1 = x, 2 = y,
// 4 = z), forward if POS. The 4 corners on the shared face are the same
// vertices in both cells: their sums stay in registers and move to their slot
// in the new cell; only the 4 corners left behind are flushed. This cuts the
// adjoint's atomics by up to half.
template <int B, bool POS>
__device__ __forceinline__ void carry_cell(float* __restrict__ grad, const int32_t l[8],
                                           float gs[8], float gc[8][3], const float Y[9]) {
#pragma unroll
  for (int c = 0; c < 8; ++c)
    if (POS == ((c & B) == 0)) flush_corner(grad, l[c], gs[c], gc[c], Y);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (POS == ((c & B) == 0)) {  // new corner c takes old corner c ^ B
      gs[c] = gs[c ^ B];
      gc[c][0] = gc[c ^ B][0];
      gc[c][1] = gc[c ^ B][1];
      gc[c][2] = gc[c ^ B][2];
      clear_corner(gs[c ^ B], gc[c ^ B]);
    }
  }
}

template <int STORE>
__device__ __forceinline__ void march_backward(const Common& P, const RayF& r, const float Y[9],
                                               const float Cf[3], float Df, const float gC[3],
                                               float gD, float* __restrict__ grad) {
  const int rm2x = P.g.rx - 2, rm2y = P.g.ry - 2, rm2z = P.g.rz - 2;
  int cx = -1, cy = -1, cz = -1;
  bool empty = true, dirty = false;
  int32_t l[8];
  __shared__ float cache[32 * kBlock];  // corner cache in shared memory: frees 32 registers
  float* sc = cache + threadIdx.x;
  float gs[8], gc[8][3];
#pragma unroll
  for (int c = 0; c < 8; ++c) clear_corner(gs[c], gc[c]);
  float S[3] = {0.f, 0.f, 0.f}, SD = 0.f, T = 1.f;
  const float dt = r.dt;
  for (int k = 0; k < r.n; ++k) {
    const float kf = (float)k;
    int ix, iy, iz;
    float fx, fy, fz;
    sample_axis(r.bh[0], r.bl[0], r.sh[0], r.sl[0], kf, rm2x, ix, fx);
    sample_axis(r.bh[1], r.bl[1], r.sh[1], r.sl[1], kf, rm2y, iy, fy);
    sample_axis(r.bh[2], r.bl[2], r.sh[2], r.sl[2], kf, rm2z, iz, fz);
    if (ix != cx || iy != cy || iz != cz) {
      const bool skip = block_empty(P.g, ix, iy, iz);
      if (dirty) {
        const int dx = ix - cx, dy = iy - cy, dz = iz - cz;
        int step = -1;  // face-adjacent step: 0/1 = +x/-x, 2/3 = +y/-y, 4/5 = +z/-z
        if (!skip) {
          if (dy == 0 && dz == 0) step = dx == 1 ? 0 : (dx == -1 ? 1 : -1);
          else if (dx == 0 && dz == 0) step = dy == 1 ? 2 : (dy == -1 ? 3 : -1);
          else if (dx == 0 && dy == 0) step = dz == 1 ? 4 : (dz == -1 ? 5 : -1);
        }
        switch (step) {
          case 0: carry_cell<1, true>(grad, l, gs, gc, Y); break;
          case 1: carry_cell<1, false>(grad, l, gs, gc, Y); break;
          case 2: carry_cell<2, true>(grad, l, gs, gc, Y); break;
          case 3: carry_cell<2, false>(grad, l, gs, gc, Y); break;
          case 4: carry_cell<4, true>(grad, l, gs, gc, Y); break;
          case 5: carry_cell<4, false>(grad, l, gs, gc, Y); break;
          default: flush_cell(grad, l, gs, gc, Y); break;
        }
        dirty = step >= 0;  // carried sums still have to reach memory
      }
      cx = ix; cy = iy; cz = iz;
      if (skip) {
        empty = true;
        k = block_exit(r, ix, iy, iz, k) - 1;
        continue;
      }
      empty = load_cell_smem<STORE>(P.g, ix, iy, iz, Y, l, sc);
    }
    if (empty) continue;
    float w[8];
    corner_weights(fx, fy, fz, w);
    float sig = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) sig = fmaf(w[c], sc[(4 * c) * kBlock], sig);
    if (!(sig > 0.f)) continue;
    float col[3], dact[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      float a = 0.f;
#pragma unroll
      for (int c = 0; c < 8; ++c) a = fmaf(w[c], sc[(4 * c + 1 + ch) * kBlock], a);
      col[ch] = activate(a, P.o.color_act, dact[ch]);
    }
    float alpha, keep;
    alpha_of(sig * dt, alpha, keep);
    const float wgt = T * alpha;
    const float Tn = T * keep;
    const float t = fmaf(kf, dt, r.t0);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) S[ch] = fmaf(wgt, col[ch], S[ch]);
    SD = fmaf(wgt, t, SD);
    // Eq. 9 and Eq. 10
    float dsig = gD * dt * (t * Tn - Df + SD);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) dsig = fmaf(gC[ch] * dt, col[ch] * Tn - Cf[ch] + S[ch], dsig);
    // Eq. 8 through the colour activation
    float dch[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) dch[ch] = gC[ch] * wgt * dact[ch];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      gs[c] = fmaf(w[c], dsig, gs[c]);
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) gc[c][ch] = fmaf(w[c], dch[ch], gc[c][ch]);
    }
    dirty = true;
    T = Tn;
    if (T < P.o.stop_T) break;
  }
  if (dirty) flush_cell(grad, l, gs, gc, Y);
}

__global__ void k_count_valid(const float* __restrict__ depth_t, int64_t n,
                              unsigned long long* __restrict__ M) {
  unsigned long long local = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    local += depth_valid(__ldg(depth_t + i)) ? 1 : 0;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(M, local);
}

template <int STORE>
__global__ void __launch_bounds__(kBlock, PLX_BWD_MIN_BLOCKS)
k_backward_grid(const __grid_constant__ Common P, const float* __restrict__ rgb_t,
                const float* __restrict__ depth_t, const float* __restrict__ rgb,
                const float* __restrict__ depth, float* __restrict__ grad,
                double* __restrict__ loss_out, const unsigned long long* __restrict__ Mc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tile = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
  float loss = 0.f;
  if (tile < P.ct.n_tiles) {
    const RayId id = ray_of(P, tile, lane);
    RayF r;
    setup_ray(P, id, r, lane);
    const unsigned long long M = *Mc;
    if (id.valid && M > 0) {
      const float dz = __ldg(depth_t + id.out);
      if (depth_valid(dz)) {
        float Y[9];
        sh_basis(r.dir, Y);
        const float invM = (float)(1.0 / (double)M);
        const float Dt = P.o.depth_is_z ? dz * r.dc_norm : dz;
        float Cf[3], gC[3];
        float e2 = 0.f;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
          Cf[ch] = __ldg(rgb + 3 * id.out + ch);
          const float e = Cf[ch] - __ldg(rgb_t + 3 * id.out + ch);
          e2 = fmaf(e, e, e2);
          gC[ch] = 2.f * e * invM;
        }
        const float Df = __ldg(depth + id.out);
        const float eD = Df - Dt;
        loss = fmaf(P.o.lambda_d * eD, eD, e2);
        const float gD = 2.f * P.o.lambda_d * eD * invM;
        march_backward<STORE>(P, r, Y, Cf, Df, gC, gD, grad);
      }
    }
  }
  if (loss_out) {
    // per warp: FP64 sum of the rays' squared residuals, one atomic per warp
    double s = (double)loss;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    const unsigned long long M = *Mc;
    if (lane == 0 && s != 0.0) atomicAdd(loss_out, s / (double)M);
    if (blockIdx.x == 0 && threadIdx.x == 0) loss_out[1] = (double)M;
  }
}

// ------------------------------------------------------------ host launch
#define PLX_DISPATCH_STORE(store, F, ...)                                  \
  switch (store) {                                                        \
    case PLX_STORE_F32: F<PLX_STORE_F32>(__VA_ARGS__); break;             \
    case PLX_STORE_BF16: F<PLX_STORE_BF16>(__VA_ARGS__); break;           \
    case PLX_STORE_F16: F<PLX_STORE_F16>(__VA_ARGS__); break;             \
    default: F<PLX_STORE_F32_BF16>(__VA_ARGS__); break;                   \
  }

template <int STORE>
static void launch_forward_t(const Common& P, float* rgb, float* depth, float* state,
                             int32_t* counts, cudaStream_t s) {
  const unsigned blocks = (unsigned)((P.ct.n_tiles + kWarpsPerBlock - 1) / kWarpsPerBlock);
  if (counts)
    k_forward<STORE, true><<<blocks, kBlock, 0, s>>>(P, rgb, depth, state, counts);
  else
    k_forward<STORE, false><<<blocks, kBlock, 0, s>>>(P, rgb, depth, state, counts);
}

void launch_forward(int store, const Common& P, float* rgb, float* depth, float* state,
                    int32_t* counts, cudaStream_t s) {
  if (P.ct.n_tiles == 0) return;
  PLX_DISPATCH_STORE(store, launch_forward_t, P, rgb, depth, state, counts, s);
}

template <int STORE>
static void launch_backward_t(const Common& P, const float* rgb_t, const float* depth_t,
                              const float* rgb, const float* depth, float* grad,
                              double* loss_out, const unsigned long long* M, cudaStream_t s) {
  const unsigned blocks = (unsigned)((P.ct.n_tiles + kWarpsPerBlock - 1) / kWarpsPerBlock);
  k_backward_grid<STORE><<<blocks, kBlock, 0, s>>>(P, rgb_t, depth_t, rgb, depth, grad,
                                                   loss_out, M);
}

void launch_backward_grid(int store, const Common& P, const float* rgb_t, const float* depth_t,
                          const float* rgb, const float* depth, float* grad, double* loss_out,
                          unsigned long long* M, int num_sms, cudaStream_t s) {
  cudaMemsetAsync(M, 0, sizeof(unsigned long long), s);
  if (loss_out) cudaMemsetAsync(loss_out, 0, 2 * sizeof(double), s);
  if (P.ct.n_rays > 0) {
    const int64_t want = (P.ct.n_rays + kBlock - 1) / kBlock;
    const unsigned blocks = (unsigned)(want < 4 * num_sms ? want : 4 * num_sms);
    k_count_valid<<<blocks, kBlock, 0, s>>>(depth_t, P.ct.n_rays, M);
  }
  if (P.ct.n_tiles == 0) return;
  PLX_DISPATCH_STORE(store, launch_backward_t, P, rgb_t, depth_t, rgb, depth, grad, loss_out,
                     M, s);
}

}  // namespace plx
