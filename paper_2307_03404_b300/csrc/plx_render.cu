// Forward render (Sec. 4, Eq. 1-3) and mapping adjoint (Sec. 5.2, Eq. 4-11).
//
// Forward: one thread per ray, samples marched front to back with the
// transmittance carried multiplicatively; the 8 corners of the current cell
// live in registers (density + view-projected colour), reloaded only when the
// sample leaves the cell.
//
// Adjoint: the ray is marched again with the forward's C and D, recomputing
// T_i, T_{i+1}, w_i and the inclusive prefix sums S_i = sum_{j<=i} w_j c_j,
// SD_i = sum_{j<=i} w_j t_j. With a sample cache the forward keeps the index,
// density and colour of each compositing sample (up to K per ray) and the
// adjoint visits just those; rays with more re-march in full. Per sample, Eq. 8 gives dL/dc_i = g_C w_i and Eq. 9-10 give
//   dL/dsigma_i = g_C . delta (c_i T_{i+1} - C + S_i) + g_D delta (t_i T_{i+1} - D + SD_i).
// The gradients are accumulated per corner in registers while the ray stays in
// one cell, as (d density, d projected colour per channel); SH gradients are
// recovered at flush time as d colour_ch * Y_k(d), because the SH basis
// depends on the ray only. A flush is 7 vector atomics (float4) per allocated
// corner into the 128-byte gradient row of the vertex; when the ray steps into
// a face-adjacent cell the 4 shared corners are carried instead of flushed.
#include "plx_march.cuh"

namespace plx {

template <int STORE, bool COUNT, int MINB, bool RANGE = false>
__global__ void __launch_bounds__(kBlock, MINB)
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
  march_forward<STORE, COUNT, false, false, RANGE>(P, r, Y, C, D, T, n_all, n_occ, id.out,
                                                   P.o.ccap);
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

// Warp-per-ray forward for few rays (a frame of a few thousand pixels leaves
// most of the GPU idle one ray per thread, and each warp waits on its slowest
// ray): the 32 lanes march consecutive segments of one ray and seg_scan
// composites them. Needs stop_T = 0 and no sample cache (the caller checks).
template <int STORE, bool COUNT, int MINB>
__global__ void __launch_bounds__(kBlock, MINB)
k_forward_seg(const __grid_constant__ Common P, float* __restrict__ rgb,
              float* __restrict__ depth, float* __restrict__ state, int32_t* __restrict__ counts) {
  const int lane = threadIdx.x & 31;
  const int64_t n_slots = P.ct.n_tiles * 32;
  const int64_t warps = (int64_t)gridDim.x * kWarpsPerBlock;
  for (int64_t ray = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); ray < n_slots;
       ray += warps) {
    const RayId id = ray_of(P, ray >> 5, (int)(ray & 31));
    RayF r;
    setup_ray(P, id, r, lane);
    if (!id.valid) {  // warp-uniform: every lane has the same ray
      if (lane == 0 && !P.ct.dense && id.out < P.ct.n_rays) {  // bad list entry: loud NaN
        const float nan = __int_as_float(0x7fc00000);
        rgb[3 * id.out] = rgb[3 * id.out + 1] = rgb[3 * id.out + 2] = nan;
        depth[id.out] = nan;
      }
      continue;
    }
    float Y[9];
    sh_basis(r.dir, Y);
    const int k0 = (int)(((int64_t)r.n * lane) >> 5), k1 = (int)(((int64_t)r.n * (lane + 1)) >> 5);
    float S[3], SD, T;
    int n_all = 0, n_occ = 0;
    march_forward<STORE, COUNT, true>(P, r, Y, S, SD, T, n_all, n_occ, id.out, 0, k0, k1);
    float T0, S0[3], SD0, Tn, C[3], D;
    seg_scan(T, S, SD, lane, T0, S0, SD0, Tn, C, D);
    if (COUNT) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) n_occ += __shfl_xor_sync(0xffffffffu, n_occ, off);
    }
    if (lane == 0) {
      rgb[3 * id.out] = fmaf(Tn, P.o.bg[0], C[0]);
      rgb[3 * id.out + 1] = fmaf(Tn, P.o.bg[1], C[1]);
      rgb[3 * id.out + 2] = fmaf(Tn, P.o.bg[2], C[2]);
      depth[id.out] = D;
      if (state) state[id.out] = Tn;
      if (COUNT) {
        counts[2 * id.out] = r.n;
        counts[2 * id.out + 1] = n_occ;
      }
    }
  }
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

// A valid ray's RGB-D residual terms (Eq. 4, 5, 11): returns its squared
// residual (loss before 1/M) and fills the forward's C, D and the loss
// gradients dL/dC = 2 (C - C_t) / M, dL/dD = 2 lambda_d (D - D_t) / M.
__device__ __forceinline__ float ray_residual(const Common& P, const RayF& r, int64_t out,
                                              float dz, float invM,
                                              const float* __restrict__ rgb_t,
                                              const float* __restrict__ rgb,
                                              const float* __restrict__ depth, float Cf[3],
                                              float gC[3], float& Df, float& gD) {
  const float Dt = P.o.depth_is_z ? dz * r.dc_norm : dz;
  float e2 = 0.f;
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    Cf[ch] = __ldg(rgb + 3 * out + ch);
    const float e = Cf[ch] - __ldg(rgb_t + 3 * out + ch);
    e2 = fmaf(e, e, e2);
    gC[ch] = 2.f * e * invM;
  }
  Df = __ldg(depth + out);
  const float eD = Df - Dt;
  gD = 2.f * P.o.lambda_d * eD * invM;
  return fmaf(P.o.lambda_d * eD, eD, e2);
}

// Per warp: the FP64 sum of the lanes' squared residuals / M, one atomic per
// warp; (L, M) in loss_out. All 32 lanes call it.
__device__ __forceinline__ void add_warp_loss(float loss, double* __restrict__ loss_out,
                                              const unsigned long long* __restrict__ Mc,
                                              int lane) {
  double s = (double)loss;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  const unsigned long long M = *Mc;
  if (lane == 0 && s != 0.0) atomicAdd(loss_out, s / (double)M);
  if (blockIdx.x == 0 && threadIdx.x == 0) loss_out[1] = (double)M;
}

template <int STORE, int MINB>
__global__ void __launch_bounds__(kBlock, MINB)
k_backward_grid(const __grid_constant__ Common P, const float* __restrict__ rgb_t,
                const float* __restrict__ depth_t, const float* __restrict__ rgb,
                const float* __restrict__ depth, float* __restrict__ grad,
                double* __restrict__ loss_out, const unsigned long long* __restrict__ Mc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tile = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
  float loss = 0.f;
  // with a sample cache this launch re-marches only the rays it could not
  // hold, and a warp without such a ray leaves at once (the loss is then
  // summed by the cached launch, loss_out is null here)
  const RayId id = ray_of(P, tile < P.ct.n_tiles ? tile : 0, lane);
  // grad null: the loss of every valid ray and nothing else
  const bool loss_only = grad == nullptr;
  const bool todo = loss_only || P.o.ccap == 0 ||
                    (id.valid && __ldg(P.o.ccount + id.out) > P.o.ccap);
  if (tile < P.ct.n_tiles && __any_sync(0xffffffffu, todo)) {
    RayF r;
    setup_ray(P, id, r, lane);
    const unsigned long long M = *Mc;
    if (id.valid && M > 0 && todo) {
      const float dz = __ldg(depth_t + id.out);
      if (depth_valid(dz)) {
        float Y[9];
        sh_basis(r.dir, Y);
        float Cf[3], gC[3], Df, gD;
        loss = ray_residual(P, r, id.out, dz, (float)(1.0 / (double)M), rgb_t, rgb, depth, Cf,
                            gC, Df, gD);
        if (!loss_only) {
          const int2 range = P.o.range ? __ldg(P.o.range + id.out) : make_int2(0, 0x7fffffff);
          march_backward<STORE>(P, r, Y, Cf, Df, gC, gD, grad, 0, 0, 1.f, nullptr, 0.f, range);
        }
      }
    }
  }
  if (loss_out) add_warp_loss(loss, loss_out, Mc, lane);
}

// Warp-per-ray grid adjoint for few rays, without a sample cache: each lane
// marches its segment of the ray once for the local (T, S, SD), seg_scan
// gives the segment's entry transmittance and prefix sums, and the lane
// re-marches the segment from them with the per-sample adjoint of Eq. 8-10
// (the same arithmetic as march_backward), flushing its own corners. Needs
// stop_T = 0.
template <int STORE, int MINB>
__global__ void __launch_bounds__(kBlock, MINB)
k_backward_grid_seg(const __grid_constant__ Common P, const float* __restrict__ rgb_t,
                    const float* __restrict__ depth_t, const float* __restrict__ rgb,
                    const float* __restrict__ depth, float* __restrict__ grad,
                    double* __restrict__ loss_out, const unsigned long long* __restrict__ Mc) {
  const int lane = threadIdx.x & 31;
  const int64_t n_slots = P.ct.n_tiles * 32;
  const int64_t warps = (int64_t)gridDim.x * kWarpsPerBlock;
  const bool loss_only = grad == nullptr;
  const unsigned long long M = *Mc;
  float loss = 0.f;
  for (int64_t ray = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); ray < n_slots;
       ray += warps) {
    const RayId id = ray_of(P, ray >> 5, (int)(ray & 31));
    RayF r;
    setup_ray(P, id, r, lane);
    if (!id.valid || M == 0) continue;  // warp-uniform
    const float dz = __ldg(depth_t + id.out);
    if (!depth_valid(dz)) continue;
    float Cf[3], gC[3], Df, gD;
    const float e = ray_residual(P, r, id.out, dz, (float)(1.0 / (double)M), rgb_t, rgb, depth,
                                 Cf, gC, Df, gD);
    if (lane == 0) loss += e;
    if (loss_only) continue;
    float Y[9];
    sh_basis(r.dir, Y);
    const int k0 = (int)(((int64_t)r.n * lane) >> 5), k1 = (int)(((int64_t)r.n * (lane + 1)) >> 5);
    float S[3], SD, T;
    int n_all = 0, n_occ = 0;
    // the segment's corners in the shared corner cache, which its adjoint
    // march below uses too (fewer registers: 332 -> 124 bytes of spills)
    march_forward<STORE, false, true, true>(P, r, Y, S, SD, T, n_all, n_occ, id.out, 0, k0, k1);
    float T0, S0[3], SD0, Tn, C[3], D;
    seg_scan(T, S, SD, lane, T0, S0, SD0, Tn, C, D);
    march_backward<STORE, true>(P, r, Y, Cf, Df, gC, gD, grad, k0, k1, T0, S0, SD0);
  }
  if (loss_out) add_warp_loss(loss, loss_out, Mc, lane);
}

// The grid adjoint from the sample cache: every valid ray's loss term, and the
// gradients of the rays whose compositing samples all fit in it.
template <int MINB>
__global__ void __launch_bounds__(kBlock, MINB)
k_backward_grid_cached(const __grid_constant__ Common P, const float* __restrict__ rgb_t,
                       const float* __restrict__ depth_t, const float* __restrict__ rgb,
                       const float* __restrict__ depth, float* __restrict__ grad,
                       double* __restrict__ loss_out, const unsigned long long* __restrict__ Mc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tile = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
  __shared__ __align__(16) float stage[kWarpsPerBlock * stage_floats(32)];
  float loss = 0.f;
  if (tile < P.ct.n_tiles) {  // the whole warp: the scatter is cooperative
    const RayId id = ray_of(P, tile, lane);
    RayF r;
    setup_ray(P, id, r, lane);
    const unsigned long long M = *Mc;
    float Cf[3] = {0.f, 0.f, 0.f}, gC[3] = {0.f, 0.f, 0.f}, Df = 0.f, gD = 0.f, Y[9];
    int n_kept = 0;
    if (id.valid && M > 0) {
      const float dz = __ldg(depth_t + id.out);
      if (depth_valid(dz)) {
        loss = ray_residual(P, r, id.out, dz, (float)(1.0 / (double)M), rgb_t, rgb, depth, Cf,
                            gC, Df, gD);
        const int nk = __ldg(P.o.ccount + id.out);
        if (nk <= P.o.ccap) n_kept = nk;  // else the re-marching kernel takes the ray
      }
    }
    sh_basis(r.dir, Y);
    march_backward_cached_warp<32>(P, r, Y, Cf, Df, gC, gD, grad, id.out, n_kept,
                                   stage + warp * stage_floats(32), lane);
  }
  if (loss_out) add_warp_loss(loss, loss_out, Mc, lane);
}

// ------------------------------------------------------------ host launch
// Few rays, no early stop, no sample cache and the sigmoid colour: a warp per
// ray. (With identity colours, kept for closed-form tests, terms of both signs
// can cancel to a colour near zero, where summing in the scan's order instead
// of front to back costs about 1e-8 absolute, over 1e-5 of a 1e-3 floor.)
static bool use_seg(const Common& P) {
  return P.ct.n_tiles * 32 <= (int64_t)P.g.seg_rays && !(P.o.stop_T > 0.f) && P.o.ccap == 0 &&
         !P.o.range &&
         P.o.color_act == PLX_ACT_SIGMOID;
}

static unsigned seg_blocks(const Common& P, int num_sms) {
  const int64_t want = (P.ct.n_tiles * 32 + kWarpsPerBlock - 1) / kWarpsPerBlock;
  const int64_t cap = (int64_t)num_sms * 2;
  return (unsigned)(want < cap ? want : cap);
}

void launch_forward(int store, int minb, const Common& P, float* rgb, float* depth, float* state,
                    int32_t* counts, int num_sms, cudaStream_t s) {
  if (P.ct.n_tiles == 0) return;
  if (use_seg(P)) {
    const unsigned sb = seg_blocks(P, num_sms);
#define PLX_FWD_SEG(S, M)                                                               \
  if (counts)                                                                           \
    k_forward_seg<S, true, M><<<sb, kBlock, 0, s>>>(P, rgb, depth, state, counts);      \
  else                                                                                  \
    k_forward_seg<S, false, M><<<sb, kBlock, 0, s>>>(P, rgb, depth, state, counts)
    PLX_DISPATCH_SM(store, minb, PLX_FWD_SEG);
#undef PLX_FWD_SEG
    return;
  }
  const unsigned blocks = (unsigned)((P.ct.n_tiles + kWarpsPerBlock - 1) / kWarpsPerBlock);
#define PLX_FWD(S, M)                                                                     \
  if (counts && P.o.range)                                                                \
    k_forward<S, true, M, true><<<blocks, kBlock, 0, s>>>(P, rgb, depth, state, counts);  \
  else if (counts)                                                                        \
    k_forward<S, true, M><<<blocks, kBlock, 0, s>>>(P, rgb, depth, state, counts);        \
  else if (P.o.range)                                                                     \
    k_forward<S, false, M, true><<<blocks, kBlock, 0, s>>>(P, rgb, depth, state, counts); \
  else                                                                                    \
    k_forward<S, false, M><<<blocks, kBlock, 0, s>>>(P, rgb, depth, state, counts)
  PLX_DISPATCH_SM3(store, minb, PLX_FWD);
#undef PLX_FWD
}

void launch_backward_grid(int store, int minb, const Common& P, const float* rgb_t,
                          const float* depth_t, const float* rgb, const float* depth, float* grad,
                          double* loss_out, unsigned long long* M, int num_sms, cudaStream_t s) {
  cudaMemsetAsync(M, 0, sizeof(unsigned long long), s);
  if (loss_out) cudaMemsetAsync(loss_out, 0, 2 * sizeof(double), s);
  if (P.ct.n_rays > 0) {
    const int64_t want = (P.ct.n_rays + kBlock - 1) / kBlock;
    const unsigned cb = (unsigned)(want < 4 * num_sms ? want : 4 * num_sms);
    k_count_valid<<<cb, kBlock, 0, s>>>(depth_t, P.ct.n_rays, M);
  }
  if (P.ct.n_tiles == 0) return;
  const unsigned blocks = (unsigned)((P.ct.n_tiles + kWarpsPerBlock - 1) / kWarpsPerBlock);
  double* loss_full = loss_out;
  if (P.o.ccap > 0 && grad) {  // the cache's rays (and every loss term), then the overflow
    if (minb == 1)
      k_backward_grid_cached<1><<<blocks, kBlock, 0, s>>>(P, rgb_t, depth_t, rgb, depth, grad,
                                                          loss_out, M);
    else
      k_backward_grid_cached<2><<<blocks, kBlock, 0, s>>>(P, rgb_t, depth_t, rgb, depth, grad,
                                                          loss_out, M);
    loss_full = nullptr;
  }
  if (use_seg(P)) {
    const unsigned sb = seg_blocks(P, num_sms);
#define PLX_BWD_SEG(S, M_)                                                                   \
  k_backward_grid_seg<S, M_><<<sb, kBlock, 0, s>>>(P, rgb_t, depth_t, rgb, depth, grad,     \
                                                   loss_full, M)
    PLX_DISPATCH_SM(store, minb, PLX_BWD_SEG);
#undef PLX_BWD_SEG
    return;
  }
#define PLX_BWD(S, M_)                                                                   \
  k_backward_grid<S, M_><<<blocks, kBlock, 0, s>>>(P, rgb_t, depth_t, rgb, depth, grad, \
                                                  loss_full, M)
  PLX_DISPATCH_SM(store, minb, PLX_BWD);
#undef PLX_BWD
}

}  // namespace plx
