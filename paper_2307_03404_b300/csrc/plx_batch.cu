// Batched work in one persistent launch: keyframes to map (forward + adjoint
// to the grid, Sec. 5.2) and frames to track (pose Jacobian, Sec. 5.3), of any
// image sizes, in the same kernel.
//
// The work items form one tile space: mapping items first (a mapping ray
// costs two marches and the gradient atomics), then tracking items, each item
// numbered by 16x16-pixel supertiles of 8x4-pixel warp tiles. Resident blocks
// pull supertiles from a global counter until none are left, so uneven frame
// sizes and the two kinds of work balance across the GPU without host
// involvement.
//
// Mapping tile: each lane marches its ray forward (C, D), forms the loss
// gradient and marches again for the adjoint (as the separate kernels do);
// with a sample cache the lane keeps its ray's compositing samples in its
// own slot of it and the adjoint reads them back instead of re-marching.
// Tracking tile: the per-ray Gauss-Newton contributions go through the warp
// reduce-scatter; each lane keeps the FP64 sum of its value for the item it is
// on and adds it into that item's FP64 accumulator when the warp moves to
// another item (one atomic per lane and item change: the order of those
// additions, not their precision, varies from run to run).
#include "plx_march.cuh"
#include "plx_pose_march.cuh"

namespace plx {

// Valid rays of the mapping items (their loss normaliser M), walking the same
// tile space as the main kernel.
__global__ void k_count_batch(const __grid_constant__ Common P, const float* __restrict__ depth_t,
                              unsigned long long* __restrict__ M) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned long long local = 0;
  for (int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile < P.ct.n_tiles;
       tile += warps) {
    const RayId id = ray_of(P, tile, lane);
    if (id.valid && P.ct.cam[id.cam].mode == PLX_WORK_MAP && depth_valid(__ldg(depth_t + id.out)))
      ++local;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
  if (lane == 0 && local) atomicAdd(M, local);
}

template <int STORE, int MINB, bool DIRT = false>
__global__ void __launch_bounds__(kBlock, MINB)
k_batch(const __grid_constant__ Common P, const float* __restrict__ rgb_t,
        const float* __restrict__ depth_t, float* __restrict__ grad, double* __restrict__ map_loss,
        const unsigned long long* __restrict__ Mmap, double* __restrict__ track_acc,
        unsigned long long* __restrict__ counter) {
  __shared__ unsigned long long s_super;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long M = *Mmap;
  const float invM = M > 0 ? (float)(1.0 / (double)M) : 0.f;
  int slot = -1;
  double acc = 0.0, mloss = 0.0;
  for (;;) {
    // a block takes a whole 16x16 supertile (its 8 warp tiles) at a time, so
    // its warps march neighbouring rays and share L1 lines
    if (threadIdx.x == 0) s_super = atomicAdd(counter, 1ull);
    __syncthreads();
    const int64_t tile = (int64_t)s_super * kWarpsPerBlock + warp;
    __syncthreads();
    if (tile - warp >= P.ct.n_tiles) break;  // block-uniform
    if (tile >= P.ct.n_tiles) continue;      // (item tile counts are multiples of 8)
    const RayId id = ray_of(P, tile, lane);
    RayF r;
    setup_ray(P, id, r, lane);
    const CamParam& it = P.ct.cam[id.cam];
    const float dz = id.valid ? __ldg(depth_t + id.out) : 0.f;
    if (it.mode == PLX_WORK_TRACK) {  // warp-uniform: a tile lies in one item
      if (it.slot != slot) {
        if (slot >= 0) atomicAdd(track_acc + 32 * slot + lane, acc);
        acc = 0.0;
        slot = it.slot;
      }
      float v[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = 0.f;
      if (id.valid && depth_valid(dz))
        pose_ray_values<STORE, DIRT, true>(P, r, rgb_t + 3 * id.out, dz, v);
      acc += warp_reduce_scatter(v, lane);
    } else if (id.valid && M > 0 && depth_valid(dz)) {
      float Y[9];
      sh_basis(r.dir, Y);
      float C[3], D, T;
      int n_all = 0, n_occ = 0;
      // with a sample cache, thread slot `cslot` keeps this ray's compositing
      // samples between its two marches (slots past the cache re-march)
      const int64_t cslot = (int64_t)blockIdx.x * kBlock + threadIdx.x;
      const int cap = cslot < P.o.cn ? P.o.ccap : 0;
      const int kept =
          march_forward<STORE, false, false, true>(P, r, Y, C, D, T, n_all, n_occ, cslot, cap);
      const float Dt = P.o.depth_is_z ? dz * r.dc_norm : dz;
      float gC[3], e2 = 0.f;
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const float e = C[ch] - __ldg(rgb_t + 3 * id.out + ch);
        e2 = fmaf(e, e, e2);
        gC[ch] = 2.f * e * invM;
      }
      const float eD = D - Dt;
      mloss += (double)fmaf(P.o.lambda_d * eD, eD, e2);
      if (cap > 0 && kept <= cap)
        march_backward_cached(P, r, Y, C, D, gC, 2.f * P.o.lambda_d * eD * invM, grad,
                                     cslot, kept);
      else
        march_backward<STORE, false, false>(P, r, Y, C, D, gC, 2.f * P.o.lambda_d * eD * invM,
                                            grad);
    }
  }
  if (slot >= 0) atomicAdd(track_acc + 32 * slot + lane, acc);
  if (map_loss) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mloss += __shfl_xor_sync(0xffffffffu, mloss, off);
    if (lane == 0 && mloss != 0.0) atomicAdd(map_loss, mloss / (double)M);
  }
}

// Per tracking item: JtWJ, JtWr and (loss, M) from the FP64 accumulators.
__global__ void k_batch_finalize(const double* __restrict__ track_acc, int n_track,
                                 double* __restrict__ JtWJ, double* __restrict__ JtWr,
                                 double* __restrict__ track_loss, double* __restrict__ map_loss,
                                 const unsigned long long* __restrict__ Mmap) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f == 0 && map_loss) map_loss[1] = (double)*Mmap;
  if (f >= n_track) return;
  const double* a = track_acc + 32 * f;
  const double M = a[28];
  const double inv = M > 0.0 ? 1.0 / M : 0.0;
  for (int i = 0; i < 6; ++i) {
    for (int j = i; j < 6; ++j) {
      const double h = a[hidx(i, j)] * inv;
      JtWJ[36 * f + 6 * i + j] = h;
      JtWJ[36 * f + 6 * j + i] = h;
    }
    JtWr[6 * f + i] = a[21 + i] * inv;
  }
  track_loss[2 * f] = a[27] * inv;
  track_loss[2 * f + 1] = M;
}

void launch_batch(int store, int minb, const Common& P, int n_track, const float* rgb_t,
                  const float* depth_t, float* grad, double* map_loss, double* JtWJ, double* JtWr,
                  double* track_loss, unsigned long long* Mmap, double* track_acc,
                  unsigned long long* counter, int blocks, int num_sms, cudaStream_t s) {
  cudaMemsetAsync(Mmap, 0, sizeof(unsigned long long), s);
  cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
  cudaMemsetAsync(track_acc, 0, (size_t)(n_track > 0 ? n_track : 1) * 32 * sizeof(double), s);
  if (map_loss) cudaMemsetAsync(map_loss, 0, 2 * sizeof(double), s);
  if (P.ct.n_tiles > 0) {
    const int64_t want = (P.ct.n_tiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const unsigned cb = (unsigned)(want < 8 * num_sms ? want : 8 * num_sms);
    k_count_batch<<<cb, kBlock, 0, s>>>(P, depth_t, Mmap);
  }
  if (P.ct.n_tiles > 0) {
#define PLX_BATCH(S, M_)                                                                      \
  k_batch<S, M_><<<blocks, kBlock, 0, s>>>(P, rgb_t, depth_t, grad, map_loss, Mmap, track_acc, \
                                           counter)
#define PLX_BATCH_DIR(S, M_)                                                                  \
  k_batch<S, M_, true><<<blocks, kBlock, 0, s>>>(P, rgb_t, depth_t, grad, map_loss, Mmap,     \
                                                 track_acc, counter)
    if (P.o.dir_term)
      PLX_DISPATCH_SM(store, minb, PLX_BATCH_DIR);
    else
      PLX_DISPATCH_SM(store, minb, PLX_BATCH);
#undef PLX_BATCH_DIR
#undef PLX_BATCH
  }
  const int fb = n_track > 0 ? (n_track + 127) / 128 : 1;
  k_batch_finalize<<<fb, 128, 0, s>>>(track_acc, n_track, JtWJ, JtWr, track_loss, map_loss, Mmap);
}

int batch_kernel_blocks_per_sm(int store, int minb) {
  int n = 0;
#define PLX_OCC(S, M) \
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<S, M>, kBlock, 0)
  PLX_DISPATCH_SM(store, minb, PLX_OCC);
#undef PLX_OCC
  return n > 0 ? n : 1;
}

}  // namespace plx
