// Device-side building blocks of the sm_103a Plenoxel renderer.
//
// One thread marches one ray; a warp owns an 8x4 pixel tile in dense mode so
// that its rays stay close in space and share cached grid lines. Per ray the
// geometry is set up once in FP64 (ray direction, box clip, grid-space origin)
// and handed to the sample loop as float-float pairs, so that sample positions
// keep ~1e-7 voxel accuracy on 1024^3 grids while the loop itself runs in
// FP32 only. The 8 corner records of the current cell are cached in registers
// as (density, SH projected on the ray's direction per channel): the SH basis
// of Sec. 5.2 depends on the ray only, so sum_k Y_k trilerp(SH_k) equals
// trilerp(sum_k Y_k SH_k) and a cell visit costs 8 record loads while each
// sample costs 32 FMAs.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "plx.h"

namespace plx {

constexpr int kTileW = 8;             // dense-mode warp tile: 8 x 4 pixels
constexpr int kTileH = 4;
constexpr int kSuperW = 2;            // a block's 8 warp tiles form a 16 x 16 supertile
constexpr int kSuperH = 4;
constexpr int kBlock = 256;           // threads per block of the ray kernels
constexpr int kWarpsPerBlock = kBlock / 32;
constexpr int kRecordSlots = 32;      // record = 32 slots (28 used)

// Calls CALL(S, M) with S the storage mode and M (1 or 2) the blocks per SM.
#define PLX_DISPATCH_SM(store, minb, CALL)                         \
  do {                                                            \
    const int key_ = (store) * 2 + ((minb) >= 2 ? 1 : 0);         \
    switch (key_) {                                               \
      case 0: CALL(PLX_STORE_F32, 1); break;                      \
      case 1: CALL(PLX_STORE_F32, 2); break;                      \
      case 2: CALL(PLX_STORE_BF16, 1); break;                     \
      case 3: CALL(PLX_STORE_BF16, 2); break;                     \
      case 4: CALL(PLX_STORE_F16, 1); break;                      \
      case 5: CALL(PLX_STORE_F16, 2); break;                      \
      case 6: CALL(PLX_STORE_F32_BF16, 1); break;                 \
      default: CALL(PLX_STORE_F32_BF16, 2); break;                \
    }                                                             \
  } while (0)

// The same with a third choice, 3 blocks per SM (a register budget of 80):
// the forward, whose 16-bit storage modes spill little there.
#define PLX_DISPATCH_SM3(store, minb, CALL)                        \
  do {                                                            \
    if ((minb) >= 3) {                                            \
      switch (store) {                                            \
        case PLX_STORE_F32: CALL(PLX_STORE_F32, 3); break;        \
        case PLX_STORE_BF16: CALL(PLX_STORE_BF16, 3); break;      \
        case PLX_STORE_F16: CALL(PLX_STORE_F16, 3); break;        \
        default: CALL(PLX_STORE_F32_BF16, 3); break;              \
      }                                                           \
    } else {                                                      \
      PLX_DISPATCH_SM(store, minb, CALL);                         \
    }                                                             \
  } while (0)

// ---------------------------------------------------------------- params
struct CamParam {
  float2 inv_fx, inv_fy, cx, cy;  // 1/fx, 1/fy, principal point as (hi, lo) float pairs
  int32_t width, height;
  int64_t ray_off;                // dense mode: index of the camera's ray 0
  int64_t tile_off;               // dense mode: index of the camera's tile 0
  int32_t supers_x;               // 16x16 supertiles per row
  int32_t pose_idx;               // row of the poses array (a batch may name a camera twice)
  int32_t mode;                   // batch work: PLX_WORK_MAP or PLX_WORK_TRACK
  int32_t slot;                   // batch work: index among the tracking items
};

struct CamTable {
  int32_t n_cams;
  int32_t dense;                  // 1: every pixel of every camera
  int64_t n_rays;
  int64_t n_tiles;                // dense: 8x4 tiles; list: ceil(n_rays / 32)
  CamParam cam[PLX_MAX_CAMERAS];
};

struct RayList {
  const int32_t* cam_id;          // list mode, may be null (single camera)
  const int32_t* pixel;           // list mode
  int32_t fixed_cam;              // >= 0: every ray belongs to this camera
  int32_t random;                 // 1: rays are random pixels of fixed_cam (see below;
                                  // pixel, if set, holds them already drawn)
  uint64_t seed;                  // random mode: generator seed
  const double* iter;             // random mode: device iteration counter (an integer)
};

// SplitMix64 output function (Steele, Lea and Flood, 2014) used as a
// counter-based generator: value k of stream `seed` is
// mix(seed + (k + 1) * 0x9E3779B97F4A7C15).
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Launch choices the autotuner can change (plx_grid_set_config). Each ray
// kernel is compiled for 1 and 2 resident blocks per SM (register budget 255 or
// 128 per thread); the empty-space map uses blocks of 2^shift cells per axis.
// Defaults: the best measured on B300 for the room workloads.
constexpr int kDefaultBlkShift = 3;
constexpr int kDefaultFwdBlocks = 1;
constexpr int kDefaultBwdBlocks = 2;
constexpr int kDefaultPoseBlocks = 2;
constexpr int kDefaultBatchBlocks = 1;
constexpr int kDefaultFineSkip = PLX_FINE_ADJOINT | PLX_FINE_POSE | PLX_FINE_BATCH;
constexpr int kFineShift = 1;         // second-level empty-space blocks: 2^1 cells per axis
constexpr int kMaxSortedRays = 8192;  // Adam tracking: random rays put in image order up to this
constexpr int32_t kSegRays = 16384;   // default seg_rays: a warp per ray up to this many rays
                                      // (forward, grid adjoint without a sample cache, pose
                                      // Jacobian)

struct GridView {
  const int32_t* links;           // [rz][ry][rx]
  const void* rec;                // [n_alloc] records
  const uint8_t* blk;             // [nbz][nby][nbx] 1 = some cell has an allocated corner;
                                  // null = no block may be skipped
  int32_t rx, ry, rz;
  int32_t n_alloc;
  int32_t nbx, nby;
  int32_t blk_shift;              // blocks of 2^blk_shift cells per axis
  int32_t seg_rays;               // a warp per ray for calls of at most this many ray slots
  const uint8_t* fblk;            // second level: blocks of 2^3 cells (null: none)
  int32_t fnbx, fnby;
  double lo[3];                   // box of the vertices
  double hi[3];
  double inv_h[3];                // 1 / spacing
  float2 lo_ff[3];                // lo as (hi, lo) float pairs
  float2 inv_h_ff[3];             // 1 / spacing as (hi, lo) float pairs
  float ext[3];                   // res - 1: the box in grid coordinates is [0, ext]
};

struct Opts {
  double step, near_t;
  float2 step_ff, half_step_ff, inv_step_ff, near_ff;  // (hi, lo) float pairs
  float stop_T;
  float step_f;
  float bg[3];
  float lambda_d;
  int32_t max_samples;
  int32_t color_act;
  int32_t depth_is_z;
  int32_t dir_term;               // pose Jacobian: add the SH view-direction term
  // sample cache (forward writes, grid adjoint reads; all null / 0 when off):
  // kept sample j of ray row r at [j * cn + r]
  float4* cval;                   // (sigma, c_r, c_g, c_b)
  int32_t* ck;                    // sample index k
  int32_t* ccount;                // [cn] samples with sigma > 0 per ray
  int64_t cn;                     // rays of the call
  int32_t ccap;                   // K
  int2* range;                    // [n_rays] first and one past the last compositing
                                  // sample of each ray (null: off)
};

struct Common {
  GridView g;
  Opts o;
  RayList rl;
  const double* poses;            // [n_cams][12]
  int32_t* err;                   // device error word
  CamTable ct;                    // last: large
};

// ----------------------------------------------------------- ray identity
// Where the thread's ray comes from and where its outputs go.
struct RayId {
  int32_t cam;
  int32_t u, v;
  int64_t out;                    // output row
  bool valid;
};

__device__ __forceinline__ int find_cam(const CamTable& ct, int64_t tile) {
  int lo = 0, hi = ct.n_cams - 1;
  while (lo < hi) {                       // last camera with tile_off <= tile
    const int mid = (lo + hi + 1) >> 1;
    if (ct.cam[mid].tile_off <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Ray of lane `lane` in warp-tile `tile`.
__device__ __forceinline__ RayId ray_of(const Common& P, int64_t tile, int lane) {
  RayId r;
  if (P.ct.dense) {
    const int c = P.rl.fixed_cam >= 0 ? P.rl.fixed_cam : find_cam(P.ct, tile);
    const CamParam& cp = P.ct.cam[c];
    // tiles are numbered supertile by supertile (8 per 16x16 pixels), so the
    // 8 warps of a block march neighbouring rays and share grid vertices
    const int64_t lt = tile - cp.tile_off;
    const int64_t st = lt >> 3;
    const int sub = (int)(lt & 7);
    const int sty = (int)(st / cp.supers_x), stx = (int)(st - (int64_t)sty * cp.supers_x);
    const int tx = stx * kSuperW + (sub % kSuperW), ty = sty * kSuperH + (sub / kSuperW);
    r.cam = c;
    r.u = tx * kTileW + (lane & (kTileW - 1));
    r.v = ty * kTileH + (lane / kTileW);
    r.valid = r.u < cp.width && r.v < cp.height;
    r.out = cp.ray_off + (int64_t)r.v * cp.width + r.u;
  } else {
    const int64_t i = tile * 32 + lane;
    r.valid = i < P.ct.n_rays;
    r.out = i;
    r.cam = 0;
    r.u = r.v = 0;
    if (r.valid && P.rl.random) {
      // random mode: ray i of iteration t is pixel splitmix64(seed, t n + i) mod (W H)
      // of the fixed camera; its targets are the full frame's row of that pixel
      const int c = P.rl.fixed_cam;
      const uint64_t t = (uint64_t)__ldg(P.rl.iter);
      const uint64_t npx = (uint64_t)P.ct.cam[c].width * P.ct.cam[c].height;
      // the iteration's pixels, when already drawn and put in image order by
      // k_random_pixels_sorted, else drawn here
      const int pix = P.rl.pixel ? __ldg(P.rl.pixel + i)
                                 : (int)(splitmix64(P.rl.seed, t * (uint64_t)P.ct.n_rays +
                                                                   (uint64_t)i) % npx);
      r.cam = c;
      r.u = pix % P.ct.cam[c].width;
      r.v = pix / P.ct.cam[c].width;
      r.out = pix;
    } else if (r.valid) {
      const int c = P.rl.fixed_cam >= 0 ? P.rl.fixed_cam
                    : (P.rl.cam_id ? __ldg(P.rl.cam_id + i) : 0);
      const int pix = __ldg(P.rl.pixel + i);
      bool ok = c >= 0 && c < P.ct.n_cams;
      if (ok) ok = pix >= 0 && pix < P.ct.cam[c].width * P.ct.cam[c].height;
      if (!ok) {
        r.valid = false;
        atomicOr(P.err, 1);
      } else {
        r.cam = c;
        r.u = pix % P.ct.cam[c].width;
        r.v = pix / P.ct.cam[c].width;
      }
    }
  }
  return r;
}

// ------------------------------------------------------------ ray setup
// Float-float arithmetic: a value is an unevaluated sum hi + lo of two floats
// (about 44 significant bits). Built from error-free transformations (Knuth's
// two-sum, the FMA product error), it gives the per-ray set-up the accuracy
// it needs on the FP32 pipes; FP64 is slow on this part.
struct ff {
  float h, l;
};
__device__ __forceinline__ ff ffv(float h, float l = 0.f) { ff r; r.h = h; r.l = l; return r; }
__device__ __forceinline__ ff ffv(float2 v) { return ffv(v.x, v.y); }
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return ffv(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ ff quick_two_sum(float a, float b) {  // needs |a| >= |b| or a == 0
  const float s = a + b;
  return ffv(s, b - (s - a));
}
__device__ __forceinline__ ff two_prod(float a, float b) {
  const float p = a * b;
  return ffv(p, fmaf(a, b, -p));
}
__device__ __forceinline__ ff ff_neg(ff a) { return ffv(-a.h, -a.l); }
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.h, b.h);
  s.l += a.l + b.l;
  return quick_two_sum(s.h, s.l);
}
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  ff p = two_prod(a.h, b.h);
  p.l = fmaf(a.h, b.l, fmaf(a.l, b.h, p.l));
  return quick_two_sum(p.h, p.l);
}
__device__ __forceinline__ ff ff_div(ff a, ff b) {
  const float q = __fdividef(a.h, b.h);
  const ff r = ff_sub(a, ff_mul(ffv(q), b));
  return quick_two_sum(q, __fdividef(r.h, b.h));
}
__device__ __forceinline__ bool ff_gt(ff a, ff b) { return a.h > b.h || (a.h == b.h && a.l > b.l); }

// Per ray: direction, box clip, sample count, and the grid-space position of
// sample k as b + k*s, handed to the sample loop as float pairs.
struct RayF {
  uint64_t B[3];        // grid coords of sample 0: signed fixed point, 32 fraction bits
  uint64_t S[3];        // grid-coord increment per sample, same format
  float inv_s[3];       // 1 / S as a float (for block exits), 0 where S = 0
  float t0, dt;         // t of sample 0, step
  float dir[3];         // unit direction
  float org[3];         // camera centre
  float dc_norm;        // |d_c|
  int n;                // samples to march
};

// Must be called by all 32 lanes of the warp (id.cam valid on every lane).
__device__ __forceinline__ void setup_ray(const Common& P, const RayId& id, RayF& r, int lane) {
  // the pose [R | o] as float pairs: converted once per warp when the warp
  // shares a camera (always in dense mode), else by each lane
  float Ph[12], Pl[12];
  const int pidx = P.ct.cam[id.cam].pose_idx;
  const int p0 = __shfl_sync(0xffffffffu, pidx, 0);
  if (__all_sync(0xffffffffu, pidx == p0)) {
    const double v = __ldg(P.poses + 12 * p0 + (lane < 12 ? lane : 0));
    const float vh = (float)v, vl = (float)(v - (double)vh);
#pragma unroll
    for (int j = 0; j < 12; ++j) {
      Ph[j] = __shfl_sync(0xffffffffu, vh, j);
      Pl[j] = __shfl_sync(0xffffffffu, vl, j);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 12; ++j) {
      const double v = __ldg(P.poses + 12 * pidx + j);
      Ph[j] = (float)v;
      Pl[j] = (float)(v - (double)Ph[j]);
    }
  }
  const CamParam& cp = P.ct.cam[id.cam];
  // d_c = ((u + 1/2 - cx) / fx, (v + 1/2 - cy) / fy, 1), normalised
  const ff x = ff_mul(ff_sub(ffv((float)id.u + 0.5f), ffv(cp.cx)), ffv(cp.inv_fx));
  const ff y = ff_mul(ff_sub(ffv((float)id.v + 0.5f), ffv(cp.cy)), ffv(cp.inv_fy));
  const ff n2 = ff_add(ff_add(ff_mul(x, x), ff_mul(y, y)), ffv(1.f));
  const float y0 = rsqrtf(n2.h);
  const ff e = ff_sub(ffv(1.f), ff_mul(n2, two_prod(y0, y0)));  // 1 - n2 y0^2
  const ff inv_n = quick_two_sum(y0, 0.5f * y0 * e.h);           // one Newton step
  const ff dcn[3] = {ff_mul(x, inv_n), ff_mul(y, inv_n), inv_n};
  ff og[3], dg[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const ff d = ff_add(ff_add(ff_mul(ffv(Ph[4 * a], Pl[4 * a]), dcn[0]),
                               ff_mul(ffv(Ph[4 * a + 1], Pl[4 * a + 1]), dcn[1])),
                        ff_mul(ffv(Ph[4 * a + 2], Pl[4 * a + 2]), dcn[2]));
    const ff o = ffv(Ph[4 * a + 3], Pl[4 * a + 3]);
    og[a] = ff_mul(ff_sub(o, ffv(P.g.lo_ff[a])), ffv(P.g.inv_h_ff[a]));
    dg[a] = ff_mul(d, ffv(P.g.inv_h_ff[a]));
    r.dir[a] = d.h;
    r.org[a] = o.h;
  }
  // slab clip against [0, ext] in grid coordinates (t is still the world
  // distance along the unit direction); the binding planes are found in FP32
  // and their crossing parameters recomputed in float-float
  float tn = -3.0e38f, tf = 3.0e38f;
  int ina = -1, outa = -1;
  float inb = 0.f, outb = 0.f;
  bool hit = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (fabsf(dg[a].h) > 1e-30f) {
      const float inv = 1.f / dg[a].h;
      float b0 = 0.f, b1 = P.g.ext[a];
      if (inv < 0.f) { b0 = P.g.ext[a]; b1 = 0.f; }
      const float t0 = (b0 - og[a].h) * inv, t1 = (b1 - og[a].h) * inv;
      if (t0 > tn) { tn = t0; ina = a; inb = b0; }
      if (t1 < tf) { tf = t1; outa = a; outb = b1; }
    } else if (og[a].h < 0.f || og[a].h > P.g.ext[a]) {
      hit = false;
    }
  }
  ff t_enter = ffv(-3.0e38f), t_exit = ffv(3.0e38f);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a == ina) t_enter = ff_div(ff_sub(ffv(inb), og[a]), dg[a]);
    if (a == outa) t_exit = ff_div(ff_sub(ffv(outb), og[a]), dg[a]);
  }
  const ff near_t = ffv(P.o.near_ff);
  const ff t_min = ff_gt(near_t, t_enter) ? near_t : t_enter;
  int n = 0;
  if (hit && ff_gt(t_exit, t_min)) {
    const ff cnt = ff_mul(ff_sub(t_exit, t_min), ffv(P.o.inv_step_ff));
    float fl = floorf(cnt.h);
    if (fl == cnt.h && cnt.l < 0.f) fl -= 1.f;
    n = (int)fminf(fl, (float)P.o.max_samples);
  }
  r.n = n;
  const ff t0 = ff_add(t_min, ffv(P.o.half_step_ff));
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const ff b = ff_add(og[a], ff_mul(t0, dg[a]));
    const ff st = ff_mul(ffv(P.o.step_ff), dg[a]);
    // x 2^32 is exact on the high parts; the low parts round to 2^-33 cells
    // (conversion saturates for rays that miss the grid, which march nothing)
    r.B[a] = (uint64_t)__float2ll_rn(b.h * 4294967296.f) + (uint64_t)__float2ll_rn(b.l * 4294967296.f);
    r.S[a] = (uint64_t)__float2ll_rn(st.h * 4294967296.f) + (uint64_t)__float2ll_rn(st.l * 4294967296.f);
    r.inv_s[a] = r.S[a] != 0 ? 1.f / (float)(int64_t)r.S[a] : 0.f;
  }
  r.t0 = n > 0 ? t0.h : 0.f;
  r.dt = P.o.step_f;
  r.dc_norm = n2.h * inv_n.h;
}

// Real SH of degree 0..2 (orthonormal; order 1; y, z, x; xy, yz, 3z^2-1,
// xz, x^2-y^2).
__device__ __forceinline__ void sh_basis(const float d[3], float Y[9]) {
  const float x = d[0], y = d[1], z = d[2];
  Y[0] = 0.28209479177387814f;
  Y[1] = 0.48860251190291992f * y;
  Y[2] = 0.48860251190291992f * z;
  Y[3] = 0.48860251190291992f * x;
  Y[4] = 1.09254843059207907f * x * y;
  Y[5] = 1.09254843059207907f * y * z;
  Y[6] = 0.31539156525252005f * (3.f * z * z - 1.f);
  Y[7] = 1.09254843059207907f * x * z;
  Y[8] = 0.54627421529603959f * (x * x - y * y);
}

// Cell index and in-cell fraction of sample k along one axis from the
// fixed-point position B + k*S (32.32, two's complement; exact modulo 2^64):
// one wide multiply-add for the low word, one multiply-add for the high word.
// The high word is the cell (floor), the fraction is the low word rounded to
// a float (relative error 2^-24, as a float-float sum rounded once; it may
// round up to 1.0, which is the same point as 0 in the next cell: the
// trilinear value is continuous and both cells share that face's corners).
// Against the real position the error adds the rounding of B and S, below
// (k + 1) 2^-33 cells: 2e-7 cells at k = 1800.
__device__ __forceinline__ void sample_axis(uint64_t B, uint64_t S, int k, int rm2, int& cell,
                                            float& frac) {
  const uint32_t ku = (uint32_t)k;
  const uint64_t p = (uint64_t)ku * (uint32_t)S + B;
  const uint32_t hi = (uint32_t)(p >> 32) + ku * (uint32_t)(S >> 32);
  float f = __uint2float_rn((uint32_t)p) * 2.3283064365386963e-10f;  // x 2^-32
  int ci = (int)hi;
  if (ci < 0) { f += (float)ci; ci = 0; }
  else if (ci > rm2) { f += (float)(ci - rm2); ci = rm2; }
  cell = ci;
  frac = f;
}

// --------------------------------------------------------- record gathers
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ float f16_lo(uint32_t w) {
  return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu)));
}
__device__ __forceinline__ float f16_hi(uint32_t w) {
  return __half2float(__ushort_as_half((unsigned short)(w >> 16)));
}

// 32 bytes from global memory through the read-only path in one 256-bit
// load (sm_100 and later); p must be 32-byte aligned.
__device__ __forceinline__ void ld_v8(const void* p, uint32_t w[8]) {
  asm("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]),
        "=r"(w[7])
      : "l"(p));
}

// Loads the 28 values of record `link` into v[0..27] (density, then SH): a
// 128-byte FP32 record in four 256-bit loads (the padding slots 28..31
// included; against seven 128-bit loads of slots 0..27 this took the FP32
// forward from 4.15 to 3.83 ms on room256 and the pose kernel from 1.36 to
// 1.24 ms), a 64-byte 16-bit record in two. Records start 32-byte aligned.
template <int STORE>
__device__ __forceinline__ void load_record(const void* rec, int32_t link, float v[28]) {
  if constexpr (STORE == PLX_STORE_F32) {
    const char* p = reinterpret_cast<const char*>(rec) + (int64_t)link * 128;
    uint32_t w[32];
#pragma unroll
    for (int j = 0; j < 4; ++j) ld_v8(p + 32 * j, w + 8 * j);
#pragma unroll
    for (int j = 0; j < 28; ++j) v[j] = __uint_as_float(w[j]);
  } else {
    const char* p = reinterpret_cast<const char*>(rec) + (int64_t)link * 64;
    uint32_t w[16];
    ld_v8(p, w);
    ld_v8(p + 32, w + 8);
    if constexpr (STORE == PLX_STORE_BF16) {
#pragma unroll
      for (int j = 0; j < 14; ++j) { v[2 * j] = bf16_lo(w[j]); v[2 * j + 1] = bf16_hi(w[j]); }
    } else if constexpr (STORE == PLX_STORE_F16) {
#pragma unroll
      for (int j = 0; j < 14; ++j) { v[2 * j] = f16_lo(w[j]); v[2 * j + 1] = f16_hi(w[j]); }
    } else {  // F32 density in slots 0-1, 27 BF16 SH in slots 2..28
      v[0] = __uint_as_float(w[0]);
#pragma unroll
      for (int j = 0; j < 14; ++j) {
        if (2 * j + 1 <= 27) v[2 * j + 1] = bf16_lo(w[j + 1]);
        if (2 * j + 2 <= 27) v[2 * j + 2] = bf16_hi(w[j + 1]);
      }
    }
  }
}

// Density and view-projected colour (per channel sum_k Y_k SH_k) of a corner.
template <int STORE>
__device__ __forceinline__ void load_corner(const void* rec, int32_t link, const float Y[9],
                                            float& sig, float col[3]) {
  float v[28];
  load_record<STORE>(rec, link, v);
  sig = v[0];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float a = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) a = fmaf(Y[k], v[1 + 9 * ch + k], a);
    col[ch] = a;
  }
}

// The 8 links of cell (ix, iy, iz); corner c = dx + 2 dy + 4 dz.
__device__ __forceinline__ void load_links(const GridView& g, int ix, int iy, int iz,
                                           int32_t l[8]) {
  const int64_t sx = 1, sy = g.rx, sz = (int64_t)g.rx * g.ry;
  const int32_t* p = g.links + (int64_t)iz * sz + (int64_t)iy * sy + ix;
  l[0] = __ldg(p);
  l[1] = __ldg(p + sx);
  l[2] = __ldg(p + sy);
  l[3] = __ldg(p + sy + sx);
  l[4] = __ldg(p + sz);
  l[5] = __ldg(p + sz + sx);
  l[6] = __ldg(p + sz + sy);
  l[7] = __ldg(p + sz + sy + sx);
}

// Loads the cell's corner cache; returns true if no corner is allocated.
template <int STORE>
__device__ __forceinline__ bool load_cell(const GridView& g, int ix, int iy, int iz,
                                          const float Y[9], int32_t l[8], float cs[8],
                                          float cc[8][3]) {
  load_links(g, ix, iy, iz, l);
  bool any = false;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (l[c] >= 0) {
      any = true;
      load_corner<STORE>(g.rec, l[c], Y, cs[c], cc[c]);
    } else {
      cs[c] = 0.f;
      cc[c][0] = cc[c][1] = cc[c][2] = 0.f;
    }
  }
  return !any;
}

// Empty-space skipping. Samples whose cell lies in a block without any
// allocated vertex contribute exactly nothing (sigma = 0 there), so the march
// may jump over them; later samples keep their own index k, so nothing else
// changes. Two levels: blocks of 2^blk_shift cells, and inside a non-empty one
// blocks of 2 cells per axis. Returns the shift (log2 of the block size) of
// an empty block holding cell (ix, iy, iz), or -1 if there is none.
__device__ __forceinline__ int empty_block_shift(const GridView& g, int ix, int iy, int iz) {
  if (!g.blk) return -1;
  const int sh = g.blk_shift;
  if (__ldg(g.blk + ((int64_t)(iz >> sh) * g.nby + (iy >> sh)) * g.nbx + (ix >> sh)) == 0)
    return sh;
  if (g.fblk && __ldg(g.fblk + ((int64_t)(iz >> kFineShift) * g.fnby + (iy >> kFineShift)) * g.fnbx +
                      (ix >> kFineShift)) == 0)
    return kFineShift;
  return -1;
}

// Index of the first sample that may lie outside the empty block of 2^sh
// cells per axis holding cell (ix, iy, iz) (conservative: never past the
// first sample outside). Per axis the ray leaves the block at grid
// coordinate (block face) - B = k S, solved for k in FP32 from the exact
// fixed-point difference: the relative error is a few 2^-24, below 3e-4
// samples at k = 2000, and 0.01 samples of margin keep the jump on the safe
// side. Always > k.
__device__ __forceinline__ int block_exit(const RayF& r, int ix, int iy, int iz, int k, int sh) {
  const int c[3] = {ix, iy, iz};
  float kmin = 3.0e38f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int b = c[a] >> sh;
    const int64_t s = (int64_t)r.S[a];
    if (s != 0) {
      const uint32_t face = (uint32_t)((s > 0 ? b + 1 : b) << sh);
      const int64_t d = (int64_t)(((uint64_t)face << 32) - r.B[a]);
      kmin = fminf(kmin, (float)d * r.inv_s[a]);
    }
  }
  const float kn = ceilf(kmin - 0.01f);
  return kn > (float)k ? (kn < 2.0e9f ? (int)kn : 2000000000) : k + 1;
}

// The block's per-thread corner caches in shared memory (32 floats per thread):
// one array per kernel, shared by every march that keeps its corners there
// (the batched kernel's re-marching adjoint and pose Jacobian use the same
// 32 KB; a thread runs one of them at a time and uses only its own column).
__device__ __forceinline__ float* corner_cache_smem() {
  __shared__ float cache[32 * kBlock];
  return cache;
}

// Same as load_cell, with the corner cache in shared memory: slot s of the
// calling thread is sc[s * kBlock] (s = 4c: density of corner c, 4c+1+ch: its
// projected colour), so the lanes of a warp hit distinct banks.
template <int STORE>
__device__ __forceinline__ bool load_cell_smem(const GridView& g, int ix, int iy, int iz,
                                               const float Y[9], int32_t l[8], float* sc) {
  load_links(g, ix, iy, iz, l);
  bool any = false;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    float sig = 0.f, col[3] = {0.f, 0.f, 0.f};
    if (l[c] >= 0) {
      any = true;
      load_corner<STORE>(g.rec, l[c], Y, sig, col);
    }
    sc[(4 * c) * kBlock] = sig;
    sc[(4 * c + 1) * kBlock] = col[0];
    sc[(4 * c + 2) * kBlock] = col[1];
    sc[(4 * c + 3) * kBlock] = col[2];
  }
  return !any;
}

__device__ __forceinline__ void corner_weights(float fx, float fy, float fz, float w[8]) {
  const float gx = 1.f - fx, gy = 1.f - fy, gz = 1.f - fz;
  const float a0 = gy * gz, a1 = fy * gz, a2 = gy * fz, a3 = fy * fz;
  w[0] = gx * a0; w[1] = fx * a0;
  w[2] = gx * a1; w[3] = fx * a1;
  w[4] = gx * a2; w[5] = fx * a2;
  w[6] = gx * a3; w[7] = fx * a3;
}

__device__ __forceinline__ float activate(float chat, int act, float& dact) {
  if (act == PLX_ACT_IDENTITY) { dact = 1.f; return chat; }
  const float c = __fdividef(1.f, 1.f + __expf(-chat));
  dact = c * (1.f - c);
  return c;
}

// 1 - exp(-x) for x >= 0 without cancellation, and exp(-x). Below x = 1/4 the
// Taylor polynomial of 1 - e^-x through x^6 (relative truncation error below
// x^6 / 5040 = 5e-8); above, 1 - e^-x >= 0.22 and the rounding error of the
// fast exponential stays near 1e-6 relative.
__device__ __forceinline__ void alpha_of(float x, float& alpha, float& keep) {
  keep = __expf(-x);
  if (x < 0.25f) {
    const float p = fmaf(x, fmaf(x, fmaf(x, fmaf(x, fmaf(x, -1.f / 720.f, 1.f / 120.f),
                                                 -1.f / 24.f), 1.f / 6.f), -0.5f), 1.f);
    alpha = x * p;
  } else {
    alpha = 1.f - keep;
  }
}

__device__ __forceinline__ bool depth_valid(float d) { return isfinite(d) && d > 0.f; }

// Warp-per-ray compositing: lane L holds the local (T, S[3], SD) of its
// segment of the ray's samples (marched from transmittance 1 and zero sums).
// Front-to-back compositing composes segments as
//   (T_a, S_a) o (T_b, S_b) = (T_a T_b, S_a + T_a S_b),
// so an exclusive scan over the lanes gives each segment's entry state
// (T0, S0, SD0: the transmittance and colour / depth sums of all samples
// before it) and the full composition gives the ray's (Tn, C, D). The sums
// are carried as float-float pairs through the scan, so that its five levels
// of additions do not add to the rounding of the terms themselves (colours
// that cancel, as identity-activated ones can, would otherwise lose about
// 1e-8 absolute). All 32 lanes call it.
__device__ __forceinline__ void seg_scan(float T, const float S[3], float SD, int lane,
                                         float& T0, float S0[3], float& SD0, float& Tn,
                                         float C[3], float& D) {
  float iT = T;
  ff acc[4] = {ffv(S[0]), ffv(S[1]), ffv(S[2]), ffv(SD)};
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float pT = __shfl_up_sync(0xffffffffu, iT, off);
    ff prev[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      prev[q] = ffv(__shfl_up_sync(0xffffffffu, acc[q].h, off),
                    __shfl_up_sync(0xffffffffu, acc[q].l, off));
    if (lane >= off) {  // (earlier prefix) o (this lane's inclusive part)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        ff prod = two_prod(pT, acc[q].h);
        prod.l = fmaf(pT, acc[q].l, prod.l);
        acc[q] = ff_add(prev[q], prod);
      }
      iT *= pT;
    }
  }
  float e[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) e[q] = __shfl_up_sync(0xffffffffu, acc[q].h + acc[q].l, 1);
  T0 = __shfl_up_sync(0xffffffffu, iT, 1);
  if (lane == 0) {
    T0 = 1.f;
    e[0] = e[1] = e[2] = e[3] = 0.f;
  }
  S0[0] = e[0]; S0[1] = e[1]; S0[2] = e[2]; SD0 = e[3];
  Tn = __shfl_sync(0xffffffffu, iT, 31);
  C[0] = __shfl_sync(0xffffffffu, acc[0].h + acc[0].l, 31);
  C[1] = __shfl_sync(0xffffffffu, acc[1].h + acc[1].l, 31);
  C[2] = __shfl_sync(0xffffffffu, acc[2].h + acc[2].l, 31);
  D = __shfl_sync(0xffffffffu, acc[3].h + acc[3].l, 31);
}

// pose <- exp(xi^) pose for the twist xi = (rho, phi) (Sec. 5.3: the pose is
// optimised directly): Rodrigues' rotation, translation V rho, composed on the
// left of the row-major 3x4 camera-to-world pose. FP64.
__device__ __forceinline__ void se3_exp_left(const double xi[6], double* pose) {
  const double px = xi[3], py = xi[4], pz = xi[5];
  const double th2 = px * px + py * py + pz * pz;
  double A, B, Cc;
  if (th2 < 1e-12) {
    A = 1.0 - th2 / 6.0;
    B = 0.5 - th2 / 24.0;
    Cc = 1.0 / 6.0 - th2 / 120.0;
  } else {
    const double th = sqrt(th2);
    double sn, cs;
    sincos(th, &sn, &cs);
    A = sn / th;
    B = (1.0 - cs) / th2;
    Cc = (th - sn) / (th2 * th);
  }
  const double K[3][3] = {{0.0, -pz, py}, {pz, 0.0, -px}, {-py, px, 0.0}};
  double R[3][3], t[3];
  for (int i = 0; i < 3; ++i) {
    t[i] = 0.0;
    for (int j = 0; j < 3; ++j) {
      double k2 = 0.0;
      for (int m = 0; m < 3; ++m) k2 += K[i][m] * K[m][j];
      const double I = i == j ? 1.0 : 0.0;
      R[i][j] = I + A * K[i][j] + B * k2;
      t[i] += (I + B * K[i][j] + Cc * k2) * xi[j];
    }
  }
  double out[12];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = j == 3 ? t[i] : 0.0;
      for (int m = 0; m < 3; ++m) s += R[i][m] * pose[4 * m + j];
      out[4 * i + j] = s;
    }
  for (int q = 0; q < 12; ++q) pose[q] = out[q];
}

}  // namespace plx
