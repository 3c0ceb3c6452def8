// The dynamic grid (Sec. 6.1 maps with "a dynamic voxel grid" and does not say
// how it grows). Growth from observed depth: every valid depth pixel is lifted
// to its surface point X = o + s R d_c (s = z for a z-depth, z / |d_c| for a
// ray distance) and every vertex whose grid coordinates lie within `band` of
// X's on each axis is allocated. New vertices are numbered after the existing
// ones in link order (x fastest), so the result does not depend on the order
// in which pixels run.
//
// Four passes over the link array: (1) one thread per pixel marks the
// unallocated vertices of its box with -2 (concurrent marks write the same
// value); (2) one block per 4096-vertex chunk counts its marks; (3) a single
// block scans the chunk counts; (4) one block per chunk numbers its marks in
// order with a block-wide prefix count. The per-pixel arithmetic is FP64 with
// every operation rounded separately (no contraction), so the integer box of
// each pixel is reproducible on any IEEE machine that follows the same steps.
#include <cuda_runtime.h>
#include <stdint.h>

#include "plx.h"

namespace plx {

constexpr int kGrowChunk = 4096;   // vertices per numbering block
constexpr int kGrowThreads = 256;

struct GrowCams {
  double fx[PLX_MAX_CAMERAS], fy[PLX_MAX_CAMERAS], cx[PLX_MAX_CAMERAS], cy[PLX_MAX_CAMERAS];
  int32_t width[PLX_MAX_CAMERAS];
  int64_t row0[PLX_MAX_CAMERAS + 1];  // first depth row of each camera; row0[n] = total
  int32_t n;
};

struct GrowGeom {
  int32_t res[3];
  double lo[3], h[3];
  double band;
  int32_t depth_is_z;
};

__global__ void k_grow_mark(int32_t* __restrict__ links, const __grid_constant__ GrowGeom G,
                            const __grid_constant__ GrowCams C, const double* __restrict__ poses,
                            const float* __restrict__ depth) {
  const int64_t n = C.row0[C.n];
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n;
       row += (int64_t)gridDim.x * blockDim.x) {
    const double z = (double)depth[row];
    if (!(isfinite(z) && z > 0.0)) continue;
    int c = 0;
    while (row >= C.row0[c + 1]) ++c;
    const int64_t pix = row - C.row0[c];
    const int32_t u = (int32_t)(pix % C.width[c]), v = (int32_t)(pix / C.width[c]);
    const double dc0 = __ddiv_rn(__dsub_rn(__dadd_rn((double)u, 0.5), C.cx[c]), C.fx[c]);
    const double dc1 = __ddiv_rn(__dsub_rn(__dadd_rn((double)v, 0.5), C.cy[c]), C.fy[c]);
    const double dc2 = 1.0;
    double s = z;
    if (!G.depth_is_z) {
      const double nn = __dadd_rn(__dadd_rn(__dmul_rn(dc0, dc0), __dmul_rn(dc1, dc1)),
                                  __dmul_rn(dc2, dc2));
      s = __ddiv_rn(z, __dsqrt_rn(nn));
    }
    const double* T = poses + 12 * c;
    int32_t i0[3], i1[3];
    bool empty = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double w = __dadd_rn(__dadd_rn(__dmul_rn(T[4 * a], dc0), __dmul_rn(T[4 * a + 1], dc1)),
                                 __dmul_rn(T[4 * a + 2], dc2));
      const double X = __dadd_rn(T[4 * a + 3], __dmul_rn(s, w));
      const double gc = __ddiv_rn(__dsub_rn(X, G.lo[a]), G.h[a]);
      double first = ceil(__dsub_rn(gc, G.band)), last = floor(__dadd_rn(gc, G.band));
      first = first < 0.0 ? 0.0 : first;
      last = last > (double)(G.res[a] - 1) ? (double)(G.res[a] - 1) : last;
      if (!(first <= last)) empty = true;
      i0[a] = empty ? 0 : (int32_t)first;
      i1[a] = empty ? -1 : (int32_t)last;
    }
    if (empty) continue;
    for (int32_t iz = i0[2]; iz <= i1[2]; ++iz)
      for (int32_t iy = i0[1]; iy <= i1[1]; ++iy) {
        int32_t* line = links + ((int64_t)iz * G.res[1] + iy) * G.res[0];
        for (int32_t ix = i0[0]; ix <= i1[0]; ++ix)
          if (line[ix] == -1) line[ix] = -2;
      }
  }
}

__global__ void k_grow_count(const int32_t* __restrict__ links, int64_t n_links,
                             unsigned long long* __restrict__ counts) {
  __shared__ unsigned warp_sum[kGrowThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kGrowChunk;
  unsigned local = 0;
  for (int i = threadIdx.x; i < kGrowChunk; i += kGrowThreads) {
    const int64_t k = base + i;
    if (k < n_links && links[k] == -2) ++local;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = 0;
    for (int w = 0; w < kGrowThreads / 32; ++w) t += warp_sum[w];
    counts[blockIdx.x] = t;
  }
}

// Exclusive scan of the chunk counts in place (one block); total to *n_new.
__global__ void k_grow_scan(unsigned long long* __restrict__ counts, int64_t n_chunks,
                            int64_t* __restrict__ n_new) {
  __shared__ unsigned long long warp_sum[32];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t base = 0; base < n_chunks; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const unsigned long long x = i < n_chunks ? counts[i] : 0ull;
    unsigned long long incl = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += y;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      unsigned long long ws = lane < nw ? warp_sum[lane] : 0ull;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, ws, off);
        if (lane >= off) ws += y;
      }
      if (lane < nw) warp_sum[lane] = ws;  // inclusive over warps
    }
    __syncthreads();
    const unsigned long long before = carry + (warp > 0 ? warp_sum[warp - 1] : 0ull);
    if (i < n_chunks) counts[i] = before + incl - x;
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_sum[nw - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_new = (int64_t)carry;
}

// Numbers the marks of one chunk in link order; if the numbers would not fit
// int32 the marks are cleared instead and *n_new is set to -1.
__global__ void k_grow_assign(int32_t* __restrict__ links, int64_t n_links,
                              const unsigned long long* __restrict__ offs, int64_t n_alloc,
                              int64_t* __restrict__ n_new) {
  __shared__ unsigned warp_cnt[kGrowThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t total = *n_new;
  const bool fits = total >= 0 && n_alloc + total <= (int64_t)INT32_MAX;
  int64_t next = n_alloc + (int64_t)offs[blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kGrowChunk;
  for (int t = 0; t < kGrowChunk; t += kGrowThreads) {
    const int64_t k = base + t + threadIdx.x;
    const bool m = k < n_links && links[k] == -2;
    const unsigned bal = __ballot_sync(0xffffffffu, m);
    if (lane == 0) warp_cnt[warp] = __popc(bal);
    __syncthreads();
    unsigned before = 0, all = 0;
    for (int w = 0; w < kGrowThreads / 32; ++w) {
      before += w < warp ? warp_cnt[w] : 0u;
      all += warp_cnt[w];
    }
    if (m) {
      const unsigned rank = before + __popc(bal & ((1u << lane) - 1u));
      links[k] = fits ? (int32_t)(next + rank) : -1;
    }
    next += all;
    __syncthreads();
  }
  if (!fits && blockIdx.x == 0 && threadIdx.x == 0) *n_new = -1;
}

plx_status grow_impl(const plx_grid_desc* d, int32_t* links, const plx_cameras* cams,
                     const float* depth, int32_t depth_is_z, double band, int64_t* n_new,
                     cudaStream_t s, const char** why) {
  GrowGeom G;
  for (int a = 0; a < 3; ++a) {
    G.res[a] = d->res[a];
    G.lo[a] = d->lo[a];
    G.h[a] = (d->hi[a] - d->lo[a]) / (double)(d->res[a] - 1);
  }
  G.band = band;
  G.depth_is_z = depth_is_z ? 1 : 0;
  GrowCams C;
  C.n = cams->n_cams;
  C.row0[0] = 0;
  for (int c = 0; c < cams->n_cams; ++c) {
    const plx_intrinsics& in = cams->intr[c];
    C.fx[c] = in.fx;
    C.fy[c] = in.fy;
    C.cx[c] = in.cx;
    C.cy[c] = in.cy;
    C.width[c] = in.width;
    C.row0[c + 1] = C.row0[c] + (int64_t)in.width * in.height;
  }
  const int64_t n_links = (int64_t)d->res[0] * d->res[1] * d->res[2];
  const int64_t n_chunks = (n_links + kGrowChunk - 1) / kGrowChunk;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  unsigned long long* counts = nullptr;
  cudaError_t e = cudaMallocAsync(&counts, (size_t)n_chunks * sizeof(unsigned long long), s);
  if (e != cudaSuccess) {
    *why = cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PLX_ENOMEM : PLX_ECUDA;
  }
  const int64_t rows = C.row0[C.n];
  if (rows > 0) {
    const int64_t want = (rows + kGrowThreads - 1) / kGrowThreads;
    const unsigned blocks = (unsigned)(want < 16LL * sms ? want : 16LL * sms);
    k_grow_mark<<<blocks, kGrowThreads, 0, s>>>(links, G, C, cams->poses, depth);
  }
  k_grow_count<<<(unsigned)n_chunks, kGrowThreads, 0, s>>>(links, n_links, counts);
  k_grow_scan<<<1, 1024, 0, s>>>(counts, n_chunks, n_new);
  k_grow_assign<<<(unsigned)n_chunks, kGrowThreads, 0, s>>>(links, n_links, counts, d->n_alloc,
                                                            n_new);
  e = cudaGetLastError();
  cudaFreeAsync(counts, s);
  if (e != cudaSuccess) {
    *why = cudaGetErrorString(e);
    return PLX_ECUDA;
  }
  return PLX_OK;
}
}  // namespace plx
