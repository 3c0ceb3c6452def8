// C ABI of the renderer: argument checks, grid ownership and layout, launch
// parameter set-up. Every compute step runs in the kernels of plx_render.cu
// and plx_pose.cu; this file only validates, allocates (grid create/destroy)
// and launches.
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "plx_internal.cuh"

namespace plx {
void launch_forward(int store, int minb, const Common& P, float* rgb, float* depth, float* state,
                    int32_t* counts, int num_sms, cudaStream_t s);
void launch_backward_grid(int store, int minb, const Common& P, const float* rgb_t,
                          const float* depth_t, const float* rgb, const float* depth, float* grad,
                          double* loss_out, unsigned long long* M, int num_sms, cudaStream_t s);
void launch_backward_pose(int store, int minb, const Common& P, const float* rgb_t,
                          const float* depth_t, double* partials, unsigned* retire, double* JtWJ,
                          double* JtWr, double* loss, int max_blocks, cudaStream_t s);
void launch_pose_step(const double* H, const double* b, double damping, double* pose,
                      double* xi_out, int32_t* status, cudaStream_t s);
int pose_kernel_blocks_per_sm(int store, int minb);
int batch_kernel_blocks_per_sm(int store, int minb);
void launch_rmsprop(int store, void* rec, float* grad, float* state, int64_t n, float lr_density,
                    float lr_sh, float alpha, float eps, int zero_grad, int num_sms,
                    cudaStream_t s);
void launch_pose_step_lm(const double* H, const double* b, const double* loss, double* state,
                         double lambda_init, double factor, double* pose, double* xi_out,
                         int32_t* status, cudaStream_t s);
void launch_random_pixels_sorted(uint64_t seed, const double* iter, int n, int width, int height,
                                 int32_t* out, cudaStream_t s);
void launch_adam_pose(const double* JtWr, double* state, double* pose, double lr, double b1,
                      double b2, double eps, cudaStream_t s);
void launch_batch(int store, int minb, const Common& P, int n_track, const float* rgb_t,
                  const float* depth_t, float* grad, double* map_loss, double* JtWJ, double* JtWr,
                  double* track_loss, unsigned long long* Mmap, double* track_acc,
                  unsigned long long* counter, int blocks, int num_sms, cudaStream_t s);
void launch_probe(int kind, float* buf, uint32_t n_rows, int group, int ops, int blocks,
                  cudaStream_t s);
}  // namespace plx

using namespace plx;

// Scratch owned by a grid handle (device memory).
struct Workspace {
  int32_t err;                    // device error word
  unsigned int retire;            // pose-reduction retirement counter
  unsigned long long M;           // valid-ray count of the last backward call
  unsigned long long tile_counter; // batch: next tile to hand out
  unsigned long long M_map;       // batch: valid rays of the mapping items
  unsigned long long pad[3];
  // followed by double partials[max_blocks][32], then the batch's per-item
  // tracking accumulators double[PLX_MAX_CAMERAS][32]
};

struct plx_grid {
  plx_grid_desc desc;
  int32_t* links = nullptr;
  void* rec = nullptr;
  uint8_t* blk = nullptr;         // empty-space blocks (null: none)
  int nb[3] = {0, 0, 0};
  uint8_t* fblk = nullptr;        // second level, blocks of 2^kFineShift cells
  int32_t* rand_pix = nullptr;    // Adam tracking: one iteration's pixels in image order
  int fnb[3] = {0, 0, 0};
  int rec_bytes = 0;
  char* ws = nullptr;
  int max_pose_blocks = 0;        // partials the workspace holds (max over variants)
  plx_launch_config cfg;          // launch choices (autotuner)
  int pose_blocks = 0;            // resident blocks of the chosen pose variant
  int batch_blocks = 0;           // resident blocks of the chosen batch variant
  int num_sms = 0;
  int device = 0;
  double inv_h[3];
};

static thread_local std::string g_err;

static plx_status fail(plx_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define CUDA_TRY(call)                                                               \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail(e_ == cudaErrorMemoryAllocation ? PLX_ENOMEM : PLX_ECUDA, "%s: %s", \
                  #call, cudaGetErrorString(e_));                                    \
  } while (0)

static plx_status launch_check(const char* what) {
  const cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(PLX_ECUDA, "%s: launch failed: %s", what, cudaGetErrorString(e));
  }
  return PLX_OK;
}

static int record_bytes(int storage) { return storage == PLX_STORE_F32 ? 128 : 64; }

// A double as an unevaluated (hi, lo) sum of two floats.
static float2 split_ff(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

// ----------------------------------------------------------- repack kernels
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(a));
  const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(b));
  return lo | (hi << 16);
}
__device__ __forceinline__ uint32_t pack_f16(float a, float b) {
  const uint32_t lo = __half_as_ushort(__float2half_rn(a));
  const uint32_t hi = __half_as_ushort(__float2half_rn(b));
  return lo | (hi << 16);
}

__global__ void k_repack(const float* __restrict__ density, const float* __restrict__ sh,
                         int64_t n, int storage, void* __restrict__ rec) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float v[32];
    v[0] = density[i];
    for (int j = 0; j < 27; ++j) v[1 + j] = sh[i * 27 + j];
    for (int j = 28; j < 32; ++j) v[j] = 0.f;
    if (storage == PLX_STORE_F32) {
      float4* d = reinterpret_cast<float4*>(rec) + i * 8;
      for (int j = 0; j < 8; ++j) d[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    } else {
      uint32_t w[16];
      if (storage == PLX_STORE_BF16) {
        for (int j = 0; j < 16; ++j) w[j] = pack_bf16(v[2 * j], v[2 * j + 1]);
      } else if (storage == PLX_STORE_F16) {
        for (int j = 0; j < 16; ++j) w[j] = pack_f16(v[2 * j], v[2 * j + 1]);
      } else {
        w[0] = __float_as_uint(v[0]);
        for (int j = 0; j < 15; ++j) w[j + 1] = pack_bf16(v[1 + 2 * j], v[2 + 2 * j]);
      }
      uint4* d = reinterpret_cast<uint4*>(rec) + i * 4;
      for (int j = 0; j < 4; ++j) d[j] = make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
    }
  }
}

__global__ void k_unpack(const void* __restrict__ rec, int64_t n, int storage,
                         float* __restrict__ density, float* __restrict__ sh) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float v[28];
    switch (storage) {
      case PLX_STORE_F32: load_record<PLX_STORE_F32>(rec, (int32_t)i, v); break;
      case PLX_STORE_BF16: load_record<PLX_STORE_BF16>(rec, (int32_t)i, v); break;
      case PLX_STORE_F16: load_record<PLX_STORE_F16>(rec, (int32_t)i, v); break;
      default: load_record<PLX_STORE_F32_BF16>(rec, (int32_t)i, v); break;
    }
    density[i] = v[0];
    for (int j = 0; j < 27; ++j) sh[i * 27 + j] = v[1 + j];
  }
}

__global__ void k_check_links(const int32_t* __restrict__ links, int64_t n, int64_t n_alloc,
                              int32_t* __restrict__ err) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t l = links[i];
    bad |= l < -1 || (int64_t)l >= n_alloc;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, 2);
}

// Marks every 8^3-cell block that has a cell with an allocated corner: vertex
// x is a corner of cells x-1 and x (those that exist), on each axis.
__global__ void k_build_blocks(const int32_t* __restrict__ links, int rx, int ry, int rz,
                               uint8_t* __restrict__ blk, int nbx, int nby, int sh) {
  const int64_t n = (int64_t)rx * ry * rz;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (links[i] < 0) continue;
    const int x = (int)(i % rx), y = (int)((i / rx) % ry), z = (int)(i / ((int64_t)rx * ry));
    const int x0 = x > 0 ? x - 1 : x, x1 = x < rx - 1 ? x : x - 1;
    const int y0 = y > 0 ? y - 1 : y, y1 = y < ry - 1 ? y : y - 1;
    const int z0 = z > 0 ? z - 1 : z, z1 = z < rz - 1 ? z : z - 1;
    for (int cz = z0; cz <= z1; ++cz)
      for (int cy = y0; cy <= y1; ++cy)
        for (int cx = x0; cx <= x1; ++cx)
          blk[((int64_t)(cz >> sh) * nby + (cy >> sh)) * nbx + (cx >> sh)] = 1;
  }
}

static unsigned grid_stride_blocks(int64_t n, int num_sms) {
  const int64_t want = (n + 255) / 256;
  const int64_t cap = (int64_t)num_sms * 8;
  return (unsigned)(want < 1 ? 1 : (want < cap ? want : cap));
}

// Builds a map of blocks of 2^shift cells (1 = some cell has an allocated
// corner) into freshly allocated memory.
static cudaError_t make_block_map(const plx_grid* g, int shift, cudaStream_t s, uint8_t** out,
                                  int nb[3]) {
  for (int a = 0; a < 3; ++a) nb[a] = ((g->desc.res[a] - 1) + (1 << shift) - 1) >> shift;
  const size_t bytes = (size_t)nb[0] * nb[1] * nb[2];
  uint8_t* blk = nullptr;
  cudaError_t e = cudaMalloc(&blk, bytes);
  if (e == cudaSuccess) e = cudaMemsetAsync(blk, 0, bytes, s);
  if (e != cudaSuccess) {
    cudaFree(blk);
    return e;
  }
  const int64_t n_links = (int64_t)g->desc.res[0] * g->desc.res[1] * g->desc.res[2];
  k_build_blocks<<<grid_stride_blocks(n_links, g->num_sms), 256, 0, s>>>(
      g->links, g->desc.res[0], g->desc.res[1], g->desc.res[2], blk, nb[0], nb[1], shift);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(blk);
    return e;
  }
  *out = blk;
  return cudaSuccess;
}

// (Re)builds the empty-space maps of `g`: blocks of 2^shift cells, and the
// second level of 2^kFineShift cells when `fine` is set.
static cudaError_t build_block_map(plx_grid* g, int shift, int fine, cudaStream_t s) {
  int nb[3], fnb[3] = {0, 0, 0};
  uint8_t *blk = nullptr, *fblk = nullptr;
  cudaError_t e = make_block_map(g, shift, s, &blk, nb);
  if (e == cudaSuccess && fine) e = make_block_map(g, kFineShift, s, &fblk, fnb);
  if (e != cudaSuccess) {
    cudaFree(blk);
    return e;
  }
  cudaFree(g->blk);
  cudaFree(g->fblk);
  g->blk = blk;
  g->fblk = fblk;
  for (int a = 0; a < 3; ++a) {
    g->nb[a] = nb[a];
    g->fnb[a] = fnb[a];
  }
  g->cfg.block_shift = shift;
  return cudaSuccess;
}

// Resident blocks of the chosen pose and batch variants.
static void apply_config(plx_grid* g) {
  g->pose_blocks = g->num_sms * pose_kernel_blocks_per_sm(g->desc.storage, g->cfg.pose_blocks);
  g->batch_blocks = g->num_sms * batch_kernel_blocks_per_sm(g->desc.storage, g->cfg.batch_blocks);
  if (g->pose_blocks > g->max_pose_blocks) g->pose_blocks = g->max_pose_blocks;
}

// ------------------------------------------------------------------- ABI
extern "C" {

const char* plx_last_error(void) { return g_err.c_str(); }

const char* plx_version(void) { return "plx 0.1 sm_103a"; }

plx_status plx_grid_create(const plx_grid_desc* desc, const int32_t* links, const float* density,
                           const float* sh, void* stream, plx_grid** out) {
  if (!desc || !out) return fail(PLX_EINVAL, "grid_create: null desc or out");
  *out = nullptr;
  for (int a = 0; a < 3; ++a) {
    if (desc->res[a] < 2 || desc->res[a] > 65536)
      return fail(PLX_EINVAL, "grid_create: res[%d] = %d out of [2, 65536]", a, desc->res[a]);
    if (!(desc->hi[a] > desc->lo[a]) || !std::isfinite(desc->lo[a]) || !std::isfinite(desc->hi[a]))
      return fail(PLX_EINVAL, "grid_create: need lo < hi on axis %d", a);
  }
  if (desc->n_alloc < 0 || desc->n_alloc > INT32_MAX)
    return fail(PLX_EINVAL, "grid_create: n_alloc %lld out of range", (long long)desc->n_alloc);
  if (desc->storage < PLX_STORE_F32 || desc->storage > PLX_STORE_F32_BF16)
    return fail(PLX_EINVAL, "grid_create: unknown storage %d", desc->storage);
  if (!links) return fail(PLX_EINVAL, "grid_create: null links");
  if (desc->n_alloc > 0 && (!density || !sh))
    return fail(PLX_EINVAL, "grid_create: null density or sh");
  const int64_t n_links = (int64_t)desc->res[0] * desc->res[1] * desc->res[2];
  cudaStream_t s = (cudaStream_t)stream;
  // optional cap on the device memory one grid may take (PLX_ALLOC_CAP_BYTES),
  // checked before anything is allocated: a way to meet the out-of-memory path
  // on purpose without exhausting a shared device
  if (const char* cap_s = std::getenv("PLX_ALLOC_CAP_BYTES")) {
    const double cap = std::atof(cap_s);
    const double need = (double)n_links * 4.0 * 1.15 +
                        (double)(desc->n_alloc > 0 ? desc->n_alloc : 1) * record_bytes(desc->storage);
    if (cap > 0.0 && need > cap)
      return fail(PLX_ENOMEM, "grid_create: needs %.0f bytes, over PLX_ALLOC_CAP_BYTES = %.0f",
                  need, cap);
  }

  plx_grid* g = new plx_grid();
  g->desc = *desc;
  g->rec_bytes = record_bytes(desc->storage);
  for (int a = 0; a < 3; ++a) g->inv_h[a] = (double)(desc->res[a] - 1) / (desc->hi[a] - desc->lo[a]);
  auto cleanup = [&](plx_status st) {
    cudaFree(g->links);
    cudaFree(g->rec);
    cudaFree(g->blk);
    cudaFree(g->fblk);
    cudaFree(g->ws);
    cudaFree(g->rand_pix);
    delete g;
    return st;
  };
  cudaError_t e = cudaGetDevice(&g->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
  if (e != cudaSuccess) return cleanup(fail(PLX_ECUDA, "grid_create: %s", cudaGetErrorString(e)));
  int bps = 1;
  for (int m = 1; m <= 2; ++m) {
    const int b = pose_kernel_blocks_per_sm(desc->storage, m);
    bps = b > bps ? b : bps;
  }
  g->max_pose_blocks = g->num_sms * bps;
  g->cfg.block_shift = kDefaultBlkShift;
  g->cfg.forward_blocks = kDefaultFwdBlocks;
  g->cfg.adjoint_blocks = kDefaultBwdBlocks;
  g->cfg.pose_blocks = kDefaultPoseBlocks;
  g->cfg.batch_blocks = kDefaultBatchBlocks;
  g->cfg.fine_skip = kDefaultFineSkip;
  g->cfg.seg_rays = kSegRays;
  apply_config(g);
  const size_t ws_bytes = sizeof(Workspace) +
                          ((size_t)g->max_pose_blocks + PLX_MAX_CAMERAS) * 32 * sizeof(double);
  e = cudaMalloc(&g->links, (size_t)n_links * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&g->rec, (size_t)(desc->n_alloc > 0 ? desc->n_alloc : 1) * g->rec_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&g->ws, ws_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&g->rand_pix, kMaxSortedRays * sizeof(int32_t));
  if (e != cudaSuccess)
    return cleanup(fail(e == cudaErrorMemoryAllocation ? PLX_ENOMEM : PLX_ECUDA,
                        "grid_create: allocation failed: %s", cudaGetErrorString(e)));
  e = cudaMemsetAsync(g->ws, 0, ws_bytes, s);

  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->links, links, (size_t)n_links * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cleanup(fail(PLX_ECUDA, "grid_create: %s", cudaGetErrorString(e)));
  Workspace* ws = reinterpret_cast<Workspace*>(g->ws);
  k_check_links<<<grid_stride_blocks(n_links, g->num_sms), 256, 0, s>>>(g->links, n_links,
                                                                      desc->n_alloc, &ws->err);
  if (desc->n_alloc > 0)
    k_repack<<<grid_stride_blocks(desc->n_alloc, g->num_sms), 256, 0, s>>>(
        density, sh, desc->n_alloc, desc->storage, g->rec);
  if (launch_check("grid_create") != PLX_OK) return cleanup(PLX_ECUDA);
  int32_t err = 0;
  e = cudaMemcpyAsync(&err, &ws->err, sizeof(err), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cleanup(fail(PLX_ECUDA, "grid_create: %s", cudaGetErrorString(e)));
  if (err) return cleanup(fail(PLX_EINVAL, "grid_create: a link is outside [-1, n_alloc)"));
  e = build_block_map(g, kDefaultBlkShift, kDefaultFineSkip != 0, s);
  if (e != cudaSuccess)
    return cleanup(fail(e == cudaErrorMemoryAllocation ? PLX_ENOMEM : PLX_ECUDA,
                        "grid_create: empty-space map: %s", cudaGetErrorString(e)));
  *out = g;
  return PLX_OK;
}

plx_status plx_grid_upload(plx_grid* g, const float* density, const float* sh, void* stream) {
  if (!g) return fail(PLX_EINVAL, "grid_upload: null grid");
  if (g->desc.n_alloc == 0) return PLX_OK;
  if (!density || !sh) return fail(PLX_EINVAL, "grid_upload: null density or sh");
  k_repack<<<grid_stride_blocks(g->desc.n_alloc, g->num_sms), 256, 0, (cudaStream_t)stream>>>(
      density, sh, g->desc.n_alloc, g->desc.storage, g->rec);
  return launch_check("grid_upload");
}

plx_status plx_grid_download(const plx_grid* g, float* density, float* sh, void* stream) {
  if (!g) return fail(PLX_EINVAL, "grid_download: null grid");
  if (g->desc.n_alloc == 0) return PLX_OK;
  if (!density || !sh) return fail(PLX_EINVAL, "grid_download: null density or sh");
  k_unpack<<<grid_stride_blocks(g->desc.n_alloc, g->num_sms), 256, 0, (cudaStream_t)stream>>>(
      g->rec, g->desc.n_alloc, g->desc.storage, density, sh);
  return launch_check("grid_download");
}

plx_status plx_grid_info(const plx_grid* g, plx_grid_desc* out) {
  if (!g || !out) return fail(PLX_EINVAL, "grid_info: null argument");
  *out = g->desc;
  return PLX_OK;
}

plx_status plx_grid_destroy(plx_grid* g) {
  if (!g) return PLX_OK;
  cudaError_t e = cudaDeviceSynchronize();
  cudaFree(g->links);
  cudaFree(g->rec);
  cudaFree(g->blk);
  cudaFree(g->fblk);
  cudaFree(g->ws);
  cudaFree(g->rand_pix);
  delete g;
  if (e != cudaSuccess) return fail(PLX_ECUDA, "grid_destroy: %s", cudaGetErrorString(e));
  return PLX_OK;
}

plx_status plx_grid_check(const plx_grid* g, void* stream) {
  if (!g) return fail(PLX_EINVAL, "grid_check: null grid");
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* ws = reinterpret_cast<Workspace*>(g->ws);
  int32_t err = 0;
  CUDA_TRY(cudaMemcpyAsync(&err, &ws->err, sizeof(err), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemsetAsync(&ws->err, 0, sizeof(int32_t), s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (err & 1) return fail(PLX_EDEVICE_CHECK, "a ray list held a camera or pixel out of range");
  if (err) return fail(PLX_EDEVICE_CHECK, "device check failed (code %d)", err);
  return PLX_OK;
}

}  // extern "C"

// ------------------------------------------------------------ call set-up
// fine_bit: the PLX_FINE_* bit of the kernel about to run (its second-level
// empty-space map is used if that bit is set in the grid's fine_skip).
static plx_status build_common(const char* what, const plx_grid* g, const plx_cameras* cams,
                               const plx_rays* rays, const plx_render_opts* o, int32_t fixed_cam,
                               int fine_bit, Common& P) {
  if (!g || !cams || !rays || !o) return fail(PLX_EINVAL, "%s: null argument", what);
  if (cams->n_cams < 1 || cams->n_cams > PLX_MAX_CAMERAS)
    return fail(PLX_EINVAL, "%s: n_cams %d out of [1, %d]", what, cams->n_cams, PLX_MAX_CAMERAS);
  if (!cams->intr || !cams->poses) return fail(PLX_EINVAL, "%s: null intrinsics or poses", what);
  if (!(o->step > 0.0) || !std::isfinite(o->step))
    return fail(PLX_EINVAL, "%s: step must be > 0", what);
  if (!(o->near_t >= 0.0) || !(o->stop_T >= 0.0) || o->max_samples < 0 || !(o->lambda_d >= 0.f))
    return fail(PLX_EINVAL, "%s: near_t, stop_T, max_samples, lambda_d must be >= 0", what);
  if (o->color_act != PLX_ACT_SIGMOID && o->color_act != PLX_ACT_IDENTITY)
    return fail(PLX_EINVAL, "%s: unknown color_act %d", what, o->color_act);
  if (fixed_cam >= cams->n_cams) return fail(PLX_EINVAL, "%s: cam %d out of range", what, fixed_cam);
  if (o->pose_flags & ~PLX_POSE_VIEW_DIR)
    return fail(PLX_EINVAL, "%s: unknown pose_flags 0x%x", what, o->pose_flags);
  std::memset(&P, 0, sizeof(P));
  P.g.links = g->links;
  P.g.rec = g->rec;
  P.g.blk = g->blk;
  P.g.nbx = g->nb[0];
  P.g.nby = g->nb[1];
  P.g.blk_shift = g->cfg.block_shift;
  P.g.seg_rays = g->cfg.seg_rays;
  P.g.fblk = (g->cfg.fine_skip & fine_bit) ? g->fblk : nullptr;
  P.g.fnbx = g->fnb[0];
  P.g.fnby = g->fnb[1];
  P.g.rx = g->desc.res[0];
  P.g.ry = g->desc.res[1];
  P.g.rz = g->desc.res[2];
  P.g.n_alloc = (int32_t)g->desc.n_alloc;
  for (int a = 0; a < 3; ++a) {
    P.g.lo[a] = g->desc.lo[a];
    P.g.hi[a] = g->desc.hi[a];
    P.g.inv_h[a] = g->inv_h[a];
    P.g.lo_ff[a] = split_ff(g->desc.lo[a]);
    P.g.inv_h_ff[a] = split_ff(g->inv_h[a]);
    P.g.ext[a] = (float)(g->desc.res[a] - 1);
  }
  P.o.step = o->step;
  P.o.near_t = o->near_t;
  P.o.step_ff = split_ff(o->step);
  P.o.half_step_ff = split_ff(0.5 * o->step);
  P.o.inv_step_ff = split_ff(1.0 / o->step);
  P.o.near_ff = split_ff(o->near_t);
  P.o.stop_T = (float)o->stop_T;
  P.o.step_f = (float)o->step;
  for (int c = 0; c < 3; ++c) P.o.bg[c] = o->bg[c];
  P.o.lambda_d = o->lambda_d;
  P.o.max_samples = o->max_samples;
  P.o.color_act = o->color_act;
  P.o.depth_is_z = o->depth_is_z;
  P.o.dir_term = (o->pose_flags & PLX_POSE_VIEW_DIR) ? 1 : 0;
  P.poses = cams->poses;
  P.err = &reinterpret_cast<Workspace*>(g->ws)->err;
  P.ct.n_cams = cams->n_cams;
  int64_t ray_off = 0, tile_off = 0;
  for (int c = 0; c < cams->n_cams; ++c) {
    const plx_intrinsics& in = cams->intr[c];
    if (in.width < 1 || in.height < 1 || (int64_t)in.width * in.height >= (1ll << 31))
      return fail(PLX_EINVAL, "%s: camera %d size %dx%d", what, c, in.width, in.height);
    if (!(in.fx != 0.0) || !(in.fy != 0.0) || !std::isfinite(in.fx) || !std::isfinite(in.fy))
      return fail(PLX_EINVAL, "%s: camera %d focal length", what, c);
    CamParam& cp = P.ct.cam[c];
    cp.inv_fx = split_ff(1.0 / in.fx);
    cp.inv_fy = split_ff(1.0 / in.fy);
    cp.cx = split_ff(in.cx);
    cp.cy = split_ff(in.cy);
    cp.width = in.width;
    cp.height = in.height;
    cp.pose_idx = c;
    cp.supers_x = (in.width + kTileW * kSuperW - 1) / (kTileW * kSuperW);
    const int supers_y = (in.height + kTileH * kSuperH - 1) / (kTileH * kSuperH);
    const bool use = fixed_cam < 0 || fixed_cam == c;
    cp.ray_off = ray_off;
    cp.tile_off = tile_off;
    if (use) {
      ray_off += (int64_t)in.width * in.height;
      tile_off += (int64_t)cp.supers_x * supers_y * kSuperW * kSuperH;
    }
  }
  const bool dense = rays->pixel == nullptr;
  if (dense && rays->cam_id)
    return fail(PLX_EINVAL, "%s: cam_id given without pixel", what);
  P.rl.cam_id = rays->cam_id;
  P.rl.pixel = rays->pixel;
  P.rl.fixed_cam = fixed_cam;
  P.ct.dense = dense ? 1 : 0;
  if (dense) {
    if (fixed_cam >= 0) {  // only camera `fixed_cam` is marched; its rays start at 0
      P.ct.cam[fixed_cam].tile_off = 0;
      P.ct.cam[fixed_cam].ray_off = 0;
    }
    if (rays->n_rays != 0 && rays->n_rays != ray_off)
      return fail(PLX_EINVAL, "%s: dense mode covers %lld rays, n_rays = %lld", what,
                  (long long)ray_off, (long long)rays->n_rays);
    P.ct.n_rays = ray_off;
    P.ct.n_tiles = tile_off;
  } else {
    if (rays->n_rays < 0) return fail(PLX_EINVAL, "%s: n_rays < 0", what);
    if (!rays->cam_id && cams->n_cams > 1 && fixed_cam < 0)
      return fail(PLX_EINVAL, "%s: cam_id needed with several cameras", what);
    P.ct.n_rays = rays->n_rays;
    P.ct.n_tiles = (rays->n_rays + 31) / 32;
  }
  return PLX_OK;
}

// The sample cache of opts, laid out for n = sample_rays rows: float4 [K][n],
// int32 [K][n], int32 [n]. Rows are rays (forward and grid adjoint: n must
// cover the call's rays) or, with per_ray false, thread slots (batched launch).
// The compositing range of plx_render_forward / plx_render_backward_grid
// (every other call leaves P.o.range null).
static plx_status set_ray_range(const char* what, const plx_render_opts* o, Common& P) {
  if (!o->ray_range) return PLX_OK;
  if (reinterpret_cast<uintptr_t>(o->ray_range) % 8 != 0)
    return fail(PLX_EINVAL, "%s: ray_range must be 8-byte aligned", what);
  P.o.range = reinterpret_cast<int2*>(o->ray_range);
  return PLX_OK;
}

static plx_status set_sample_cache(const char* what, const plx_render_opts* o, Common& P,
                                   bool per_ray = true) {
  if (!o->sample_cache || o->sample_cap == 0) return PLX_OK;
  if (o->sample_cap < 0) return fail(PLX_EINVAL, "%s: sample_cap < 0", what);
  if (reinterpret_cast<uintptr_t>(o->sample_cache) % 16 != 0)
    return fail(PLX_EINVAL, "%s: sample_cache must be 16-byte aligned", what);
  if (o->sample_rays < 0) return fail(PLX_EINVAL, "%s: sample_rays < 0", what);
  if (per_ray && o->sample_rays < P.ct.n_rays)
    return fail(PLX_EINVAL, "%s: sample cache sized for %lld rays, call has %lld", what,
                (long long)o->sample_rays, (long long)P.ct.n_rays);
  const int64_t n = o->sample_rays, K = o->sample_cap;
  char* base = static_cast<char*>(o->sample_cache);
  P.o.cval = reinterpret_cast<float4*>(base);
  P.o.ck = reinterpret_cast<int32_t*>(base + 16 * K * n);
  P.o.ccount = reinterpret_cast<int32_t*>(base + 20 * K * n);
  P.o.cn = n;
  P.o.ccap = (int32_t)K;
  return PLX_OK;
}

extern "C" {

int64_t plx_sample_cache_bytes(int64_t n_rays, int32_t cap) {
  if (n_rays < 0 || cap < 0) return -1;
  return n_rays * (20 * (int64_t)cap + 4);
}

plx_status plx_render_forward(const plx_grid* g, const plx_cameras* cams, const plx_rays* rays,
                              const plx_render_opts* opts, float* rgb_out, float* depth_out,
                              float* state_out, int32_t* counts_out, void* stream) {
  Common P;
  plx_status st = build_common("render_forward", g, cams, rays, opts, -1, PLX_FINE_FORWARD, P);
  if (st == PLX_OK) st = set_sample_cache("render_forward", opts, P);
  if (st == PLX_OK) st = set_ray_range("render_forward", opts, P);
  if (st != PLX_OK) return st;
  if (P.ct.n_rays > 0 && (!rgb_out || !depth_out))
    return fail(PLX_EINVAL, "render_forward: null rgb_out or depth_out");
  launch_forward(g->desc.storage, g->cfg.forward_blocks, P, rgb_out, depth_out, state_out, counts_out,
                 g->num_sms, (cudaStream_t)stream);
  return launch_check("render_forward");
}

plx_status plx_render_backward_grid(const plx_grid* g, const plx_cameras* cams,
                                    const plx_rays* rays, const plx_render_opts* opts,
                                    const float* rgb_target, const float* depth_target,
                                    const float* rgb, const float* depth, float* grad,
                                    double* loss_out, void* stream) {
  Common P;
  plx_status st = build_common("render_backward_grid", g, cams, rays, opts, -1, PLX_FINE_ADJOINT, P);
  if (st == PLX_OK) st = set_sample_cache("render_backward_grid", opts, P);
  if (st == PLX_OK) st = set_ray_range("render_backward_grid", opts, P);
  if (st != PLX_OK) return st;
  if (P.ct.n_rays > 0 && (!rgb_target || !depth_target || !rgb || !depth))
    return fail(PLX_EINVAL, "render_backward_grid: null array argument");
  if (!grad && !loss_out)
    return fail(PLX_EINVAL, "render_backward_grid: grad and loss_out both null");
  if (reinterpret_cast<uintptr_t>(grad) % 16 != 0)
    return fail(PLX_EINVAL, "render_backward_grid: grad must be 16-byte aligned");
  Workspace* ws = reinterpret_cast<Workspace*>(g->ws);
  launch_backward_grid(g->desc.storage, g->cfg.adjoint_blocks, P, rgb_target, depth_target, rgb, depth, grad, loss_out,
                       &ws->M, g->num_sms, (cudaStream_t)stream);
  return launch_check("render_backward_grid");
}

plx_status plx_render_backward_pose(const plx_grid* g, const plx_cameras* cams, int32_t cam,
                                    const plx_rays* rays, const plx_render_opts* opts,
                                    const float* rgb_target, const float* depth_target,
                                    double* JtWJ, double* JtWr, double* loss, void* stream) {
  if (cam < 0) return fail(PLX_EINVAL, "render_backward_pose: cam < 0");
  Common P;
  plx_status st = build_common("render_backward_pose", g, cams, rays, opts, cam, PLX_FINE_POSE, P);
  if (st != PLX_OK) return st;
  if (!JtWJ || !JtWr || !loss) return fail(PLX_EINVAL, "render_backward_pose: null output");
  if (P.ct.n_rays > 0 && (!rgb_target || !depth_target))
    return fail(PLX_EINVAL, "render_backward_pose: null target");
  Workspace* ws = reinterpret_cast<Workspace*>(g->ws);
  double* partials = reinterpret_cast<double*>(g->ws + sizeof(Workspace));
  launch_backward_pose(g->desc.storage, g->cfg.pose_blocks, P, rgb_target, depth_target, partials,
                       &ws->retire, JtWJ, JtWr, loss, g->pose_blocks, (cudaStream_t)stream);
  return launch_check("render_backward_pose");
}

plx_status plx_pose_step(const double* JtWJ, const double* JtWr, double damping, double* pose,
                         double* xi_out, int32_t* status, void* stream) {
  if (!JtWJ || !JtWr || !pose) return fail(PLX_EINVAL, "pose_step: null argument");
  if (!(damping >= 0.0) || !std::isfinite(damping))
    return fail(PLX_EINVAL, "pose_step: damping must be finite and >= 0");
  launch_pose_step(JtWJ, JtWr, damping, pose, xi_out, status, (cudaStream_t)stream);
  return launch_check("pose_step");
}

}  // extern "C"

// ------------------------------------------------------------ launch config
extern "C" plx_status plx_pose_step_lm(const double* JtWJ, const double* JtWr, const double* loss,
                                       double* state, double lambda_init, double factor,
                                       double* pose, double* xi_out, int32_t* status,
                                       void* stream) {
  if (!JtWJ || !JtWr || !loss || !state || !pose)
    return fail(PLX_EINVAL, "pose_step_lm: null argument");
  if (!(lambda_init >= 0.0) || !std::isfinite(lambda_init) || !(factor > 1.0) ||
      !std::isfinite(factor))
    return fail(PLX_EINVAL, "pose_step_lm: need lambda_init >= 0 and factor > 1");
  launch_pose_step_lm(JtWJ, JtWr, loss, state, lambda_init, factor, pose, xi_out, status,
                      (cudaStream_t)stream);
  return launch_check("pose_step_lm");
}

extern "C" plx_status plx_grid_get_config(const plx_grid* g, plx_launch_config* out) {
  if (!g || !out) return fail(PLX_EINVAL, "grid_get_config: null argument");
  *out = g->cfg;
  return PLX_OK;
}

extern "C" plx_status plx_grid_set_config(plx_grid* g, const plx_launch_config* c, void* stream) {
  const char* what = "grid_set_config";
  if (!g || !c) return fail(PLX_EINVAL, "%s: null argument", what);
  if (c->block_shift < 1 || c->block_shift > 6)
    return fail(PLX_EINVAL, "%s: block_shift %d out of [1, 6]", what, c->block_shift);
  if (c->forward_blocks < 1 || c->forward_blocks > 3)
    return fail(PLX_EINVAL, "%s: forward blocks per SM must be 1, 2 or 3", what);
  const int v[3] = {c->adjoint_blocks, c->pose_blocks, c->batch_blocks};
  for (int i = 0; i < 3; ++i)
    if (v[i] != 1 && v[i] != 2)
      return fail(PLX_EINVAL, "%s: blocks per SM must be 1 or 2", what);
  if (c->fine_skip < 0 || c->fine_skip > 15)
    return fail(PLX_EINVAL, "%s: fine_skip must be a mask of PLX_FINE_* bits", what);
  if (c->seg_rays < 0 || c->seg_rays > (1 << 24))
    return fail(PLX_EINVAL, "%s: seg_rays %d out of [0, 2^24]", what, c->seg_rays);
  if (c->block_shift != g->cfg.block_shift || (c->fine_skip != 0) != (g->cfg.fine_skip != 0)) {
    const cudaError_t e =
        build_block_map(g, c->block_shift, c->fine_skip != 0, (cudaStream_t)stream);
    if (e != cudaSuccess)
      return fail(e == cudaErrorMemoryAllocation ? PLX_ENOMEM : PLX_ECUDA, "%s: %s", what,
                  cudaGetErrorString(e));
  }
  g->cfg = *c;
  apply_config(g);
  return PLX_OK;
}

// ------------------------------------------------------------ batched work
extern "C" plx_status plx_render_batch(const plx_grid* g, const plx_cameras* cams,
                                       const plx_work* work, int32_t n_work,
                                       const plx_render_opts* opts, const float* rgb_target,
                                       const float* depth_target, float* grad, double* map_loss,
                                       double* JtWJ, double* JtWr, double* track_loss,
                                       void* stream) {
  const char* what = "render_batch";
  if (!work || n_work < 1 || n_work > PLX_MAX_CAMERAS)
    return fail(PLX_EINVAL, "%s: n_work %d out of [1, %d]", what, n_work, PLX_MAX_CAMERAS);
  plx_rays dense;
  dense.n_rays = 0;
  dense.cam_id = nullptr;
  dense.pixel = nullptr;
  Common P;
  plx_status st = build_common(what, g, cams, &dense, opts, -1, PLX_FINE_BATCH, P);
  if (st != PLX_OK) return st;
  const CamTable base = P.ct;
  int n_map = 0, n_track = 0;
  int64_t rows = 0;
  int64_t row_of[PLX_MAX_CAMERAS];
  for (int i = 0; i < n_work; ++i) {
    if (work[i].cam < 0 || work[i].cam >= cams->n_cams)
      return fail(PLX_EINVAL, "%s: work[%d].cam = %d out of range", what, i, work[i].cam);
    if (work[i].mode != PLX_WORK_MAP && work[i].mode != PLX_WORK_TRACK)
      return fail(PLX_EINVAL, "%s: work[%d].mode = %d", what, i, work[i].mode);
    row_of[i] = rows;
    rows += (int64_t)base.cam[work[i].cam].width * base.cam[work[i].cam].height;
    (work[i].mode == PLX_WORK_MAP ? n_map : n_track) += 1;
  }
  if (n_map > 0 && (!grad || reinterpret_cast<uintptr_t>(grad) % 16 != 0))
    return fail(PLX_EINVAL, "%s: mapping work needs a 16-byte aligned grad", what);
  if (n_track > 0 && (!JtWJ || !JtWr || !track_loss))
    return fail(PLX_EINVAL, "%s: tracking work needs JtWJ, JtWr and track_loss", what);
  if (rows > 0 && (!rgb_target || !depth_target))
    return fail(PLX_EINVAL, "%s: null target", what);
  // the tile space: mapping items first, then tracking items, each in work order
  int e = 0, slot = 0;
  int64_t tiles = 0;
  for (int pass = 0; pass < 2; ++pass) {
    for (int i = 0; i < n_work; ++i) {
      if ((work[i].mode == PLX_WORK_TRACK) != (pass == 1)) continue;
      CamParam cp = base.cam[work[i].cam];
      const int supers_y = (cp.height + kTileH * kSuperH - 1) / (kTileH * kSuperH);
      cp.pose_idx = work[i].cam;
      cp.mode = work[i].mode;
      cp.slot = pass == 1 ? slot++ : -1;
      cp.ray_off = row_of[i];
      cp.tile_off = tiles;
      tiles += (int64_t)cp.supers_x * supers_y * kSuperW * kSuperH;
      P.ct.cam[e++] = cp;
    }
  }
  P.ct.n_cams = n_work;
  P.ct.dense = 1;
  P.ct.n_rays = rows;
  P.ct.n_tiles = tiles;
  st = set_sample_cache(what, opts, P, false);
  if (st != PLX_OK) return st;
  Workspace* ws = reinterpret_cast<Workspace*>(g->ws);
  double* track_acc =
      reinterpret_cast<double*>(g->ws + sizeof(Workspace)) + (size_t)g->max_pose_blocks * 32;
  launch_batch(g->desc.storage, g->cfg.batch_blocks, P, n_track, rgb_target, depth_target, grad, map_loss, JtWJ, JtWr,
               track_loss, &ws->M_map, track_acc, &ws->tile_counter, g->batch_blocks,
               g->num_sms, (cudaStream_t)stream);
  return launch_check(what);
}

// ------------------------------------------------------------ optimisers
namespace plx {
plx_status grow_impl(const plx_grid_desc* d, int32_t* links, const plx_cameras* cams,
                     const float* depth, int32_t depth_is_z, double band, int64_t* n_new,
                     cudaStream_t s, const char** why);
}

extern "C" plx_status plx_grid_grow(const plx_grid_desc* d, int32_t* links,
                                    const plx_cameras* cams, const float* depth,
                                    int32_t depth_is_z, double band, int64_t* n_new,
                                    void* stream) {
  if (!d || !links || !cams || !n_new) return fail(PLX_EINVAL, "grid_grow: null argument");
  for (int a = 0; a < 3; ++a) {
    if (d->res[a] < 2 || d->res[a] > 65536)
      return fail(PLX_EINVAL, "grid_grow: res[%d] = %d out of [2, 65536]", a, d->res[a]);
    if (!(d->hi[a] > d->lo[a]) || !std::isfinite(d->lo[a]) || !std::isfinite(d->hi[a]))
      return fail(PLX_EINVAL, "grid_grow: need lo < hi on axis %d", a);
  }
  if (d->n_alloc < 0 || d->n_alloc > INT32_MAX)
    return fail(PLX_EINVAL, "grid_grow: n_alloc %lld out of range", (long long)d->n_alloc);
  if (!(band >= 0.0 && band <= 16.0)) return fail(PLX_EINVAL, "grid_grow: band outside [0, 16]");
  if (cams->n_cams < 1 || cams->n_cams > PLX_MAX_CAMERAS)
    return fail(PLX_EINVAL, "grid_grow: n_cams %d out of [1, %d]", cams->n_cams, PLX_MAX_CAMERAS);
  if (!cams->intr || !cams->poses) return fail(PLX_EINVAL, "grid_grow: null intrinsics or poses");
  int64_t rows = 0;
  for (int c = 0; c < cams->n_cams; ++c) {
    const plx_intrinsics& in = cams->intr[c];
    if (in.width < 1 || in.height < 1 || (int64_t)in.width * in.height > INT32_MAX)
      return fail(PLX_EINVAL, "grid_grow: camera %d has a bad image size", c);
    if (!(std::isfinite(in.fx) && std::isfinite(in.fy) && in.fx != 0.0 && in.fy != 0.0 &&
          std::isfinite(in.cx) && std::isfinite(in.cy)))
      return fail(PLX_EINVAL, "grid_grow: camera %d has bad intrinsics", c);
    rows += (int64_t)in.width * in.height;
  }
  if (!depth) return fail(PLX_EINVAL, "grid_grow: null depth");
  const char* why = "";
  const plx_status st = grow_impl(d, links, cams, depth, depth_is_z, band, n_new,
                                  (cudaStream_t)stream, &why);
  if (st != PLX_OK) return fail(st, "grid_grow: %s", why);
  return PLX_OK;
}

extern "C" plx_status plx_grid_rmsprop(plx_grid* g, float* grad, float* state, float lr_density,
                                       float lr_sh, float alpha, float eps, int32_t zero_grad,
                                       void* stream) {
  const char* what = "grid_rmsprop";
  if (!g) return fail(PLX_EINVAL, "%s: null grid", what);
  if (g->desc.n_alloc == 0) return PLX_OK;
  if (!grad || !state || reinterpret_cast<uintptr_t>(grad) % 16 != 0 ||
      reinterpret_cast<uintptr_t>(state) % 16 != 0)
    return fail(PLX_EINVAL, "%s: grad and state must be non-null and 16-byte aligned", what);
  if (!(lr_density >= 0.f) || !(lr_sh >= 0.f) || !(alpha >= 0.f && alpha <= 1.f) || !(eps > 0.f))
    return fail(PLX_EINVAL, "%s: need lr_density, lr_sh >= 0, 0 <= alpha <= 1, eps > 0", what);
  launch_rmsprop(g->desc.storage, g->rec, grad, state, g->desc.n_alloc, lr_density, lr_sh, alpha,
                 eps, zero_grad ? 1 : 0, g->num_sms, (cudaStream_t)stream);
  return launch_check(what);
}

extern "C" plx_status plx_track_adam_step(const plx_grid* g, const plx_cameras* cams, int32_t cam,
                                          const plx_render_opts* opts, int32_t n_rays,
                                          uint64_t seed, const float* rgb_target,
                                          const float* depth_target, double* state, double lr,
                                          double beta1, double beta2, double eps, double* JtWJ,
                                          double* JtWr, double* loss, void* stream) {
  const char* what = "track_adam_step";
  if (cam < 0) return fail(PLX_EINVAL, "%s: cam < 0", what);
  if (n_rays < 1) return fail(PLX_EINVAL, "%s: n_rays must be >= 1", what);
  if (!state || !JtWJ || !JtWr || !loss || !rgb_target || !depth_target)
    return fail(PLX_EINVAL, "%s: null argument", what);
  if (!(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) ||
      !(eps > 0.0))
    return fail(PLX_EINVAL, "%s: need lr >= 0, 0 <= beta < 1, eps > 0", what);
  plx_rays dense;
  dense.n_rays = 0;
  dense.cam_id = nullptr;
  dense.pixel = nullptr;
  Common P;
  plx_status st = build_common(what, g, cams, &dense, opts, cam, PLX_FINE_POSE, P);
  if (st != PLX_OK) return st;
  P.ct.dense = 0;
  P.ct.n_rays = n_rays;
  P.ct.n_tiles = ((int64_t)n_rays + 31) / 32;
  P.rl.random = 1;
  P.rl.seed = seed;
  P.rl.iter = state + 12;
  Workspace* ws = reinterpret_cast<Workspace*>(g->ws);
  double* partials = reinterpret_cast<double*>(g->ws + sizeof(Workspace));
  cudaStream_t s = (cudaStream_t)stream;
  const plx_intrinsics& in = cams->intr[cam];
  if (n_rays <= kMaxSortedRays && in.width <= 65535 && in.height <= 65535) {
    launch_random_pixels_sorted(seed, state + 12, n_rays, in.width, in.height, g->rand_pix, s);
    P.rl.pixel = g->rand_pix;
  }
  launch_backward_pose(g->desc.storage, g->cfg.pose_blocks, P, rgb_target, depth_target, partials,
                       &ws->retire, JtWJ, JtWr, loss, g->pose_blocks, s);
  launch_adam_pose(JtWr, state, const_cast<double*>(cams->poses) + 12 * cam, lr, beta1, beta2, eps,
                   s);
  return launch_check(what);
}

// -------------------------------------------------- allocation-free variant
// plx_render_backward_pose_noalloc keeps its scratch (error word, retirement
// counter and the FP64 per-block partial sums) in this file-scope array
// instead of memory that plx_grid_create allocated. Every GPU that loads the
// library holds the array until the process exits. Host code must not pass
// the array's name to a kernel: its device address comes from
// cudaGetSymbolAddress, taken once per device.
#define PLX_NOALLOC_MAX_BLOCKS 1024
#define PLX_NOALLOC_MAX_DEVICES 64
static __device__ __align__(256) unsigned char
    g_noalloc_scratch[sizeof(Workspace) + PLX_NOALLOC_MAX_BLOCKS * 32 * sizeof(double)];

static std::mutex g_noalloc_mu;
static char* g_noalloc_ptr[PLX_NOALLOC_MAX_DEVICES];
static int g_noalloc_blocks[PLX_NOALLOC_MAX_DEVICES][4];

// Device address of the scratch and the block cap per storage mode, set up on
// the first call on each device (with that device current).
static plx_status noalloc_setup(int dev, int storage, char** ptr, int* max_blocks) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(PLX_ECUDA, "render_backward_pose_noalloc: cudaGetSymbolAddress: %s",
                  cudaGetErrorString(e));
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
      return fail(PLX_ECUDA, "render_backward_pose_noalloc: %s", cudaGetErrorString(e));
    for (int st = 0; st < 4; ++st) {
      const int b = sms * pose_kernel_blocks_per_sm(st, kDefaultPoseBlocks);
      g_noalloc_blocks[dev][st] = b < PLX_NOALLOC_MAX_BLOCKS ? b : PLX_NOALLOC_MAX_BLOCKS;
    }
    g_noalloc_ptr[dev] = static_cast<char*>(p);
  }
  *ptr = g_noalloc_ptr[dev];
  *max_blocks = g_noalloc_blocks[dev][storage];
  return PLX_OK;
}

extern "C" plx_status plx_render_backward_pose_noalloc(
    const plx_grid_desc* desc, const int32_t* links, const void* records,
    const plx_cameras* cams, int32_t cam, const plx_rays* rays, const plx_render_opts* opts,
    const float* rgb_target, const float* depth_target, double* JtWJ, double* JtWr,
    double* loss, void* stream) {
  const char* what = "render_backward_pose_noalloc";
  if (!desc) return fail(PLX_EINVAL, "%s: null desc", what);
  for (int a = 0; a < 3; ++a) {
    if (desc->res[a] < 2 || desc->res[a] > 65536)
      return fail(PLX_EINVAL, "%s: res[%d] = %d out of [2, 65536]", what, a, desc->res[a]);
    if (!(desc->hi[a] > desc->lo[a]) || !std::isfinite(desc->lo[a]) || !std::isfinite(desc->hi[a]))
      return fail(PLX_EINVAL, "%s: need lo < hi on axis %d", what, a);
  }
  if (desc->n_alloc < 0 || desc->n_alloc > INT32_MAX)
    return fail(PLX_EINVAL, "%s: n_alloc %lld out of range", what, (long long)desc->n_alloc);
  if (desc->storage < PLX_STORE_F32 || desc->storage > PLX_STORE_F32_BF16)
    return fail(PLX_EINVAL, "%s: unknown storage %d", what, desc->storage);
  if (!links || (desc->n_alloc > 0 && !records))
    return fail(PLX_EINVAL, "%s: null links or records", what);
  if (reinterpret_cast<uintptr_t>(records) % 32 != 0)  // read with 256-bit loads
    return fail(PLX_EINVAL, "%s: records must be 32-byte aligned", what);
  if (cam < 0) return fail(PLX_EINVAL, "%s: cam < 0", what);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(PLX_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  if (dev < 0 || dev >= PLX_NOALLOC_MAX_DEVICES)
    return fail(PLX_EUNSUPPORTED, "%s: device %d beyond %d", what, dev, PLX_NOALLOC_MAX_DEVICES);
  char* scratch = nullptr;
  int max_blocks = 0;
  plx_status st = noalloc_setup(dev, desc->storage, &scratch, &max_blocks);
  if (st != PLX_OK) return st;
  // a grid view on the caller's arrays; nothing is allocated or copied
  plx_grid view;
  view.desc = *desc;
  view.links = const_cast<int32_t*>(links);
  view.rec = const_cast<void*>(records);
  view.rec_bytes = record_bytes(desc->storage);
  view.ws = scratch;
  view.cfg.block_shift = kDefaultBlkShift;  // unused: the view has no empty-space map
  view.cfg.fine_skip = 0;
  view.cfg.seg_rays = kSegRays;
  for (int a = 0; a < 3; ++a) view.inv_h[a] = (double)(desc->res[a] - 1) / (desc->hi[a] - desc->lo[a]);
  Common P;
  st = build_common(what, &view, cams, rays, opts, cam, PLX_FINE_POSE, P);
  if (st != PLX_OK) return st;
  if (!JtWJ || !JtWr || !loss) return fail(PLX_EINVAL, "%s: null output", what);
  if (P.ct.n_rays > 0 && (!rgb_target || !depth_target))
    return fail(PLX_EINVAL, "%s: null target", what);
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* ws = reinterpret_cast<Workspace*>(scratch);
  e = cudaMemsetAsync(ws, 0, sizeof(Workspace), s);  // error word and retirement counter
  if (e != cudaSuccess) return fail(PLX_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  launch_backward_pose(desc->storage, kDefaultPoseBlocks, P, rgb_target, depth_target,
                       reinterpret_cast<double*>(scratch + sizeof(Workspace)), &ws->retire, JtWJ,
                       JtWr, loss, max_blocks, s);
  return launch_check(what);
}

extern "C" plx_status plx_noalloc_error(int32_t* err_out, void* stream) {
  const char* what = "noalloc_error";
  if (!err_out) return fail(PLX_EINVAL, "%s: null err_out", what);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(PLX_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  if (dev < 0 || dev >= PLX_NOALLOC_MAX_DEVICES)
    return fail(PLX_EUNSUPPORTED, "%s: device %d beyond %d", what, dev, PLX_NOALLOC_MAX_DEVICES);
  char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    scratch = g_noalloc_ptr[dev];
  }
  if (!scratch)
    return fail(PLX_EINVAL, "%s: no render_backward_pose_noalloc call on device %d yet", what,
                dev);
  Workspace* ws = reinterpret_cast<Workspace*>(scratch);
  e = cudaMemcpyAsync(err_out, &ws->err, sizeof(int32_t), cudaMemcpyDefault, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(PLX_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  return PLX_OK;
}

// ------------------------------------------------------------ ceilings probe
extern "C" plx_status plx_probe(int32_t kind, float* buf, int64_t n_rows, int32_t group,
                                int32_t ops, int32_t blocks, void* stream) {
  const char* what = "plx_probe";
  if (kind != PLX_PROBE_RED && kind != PLX_PROBE_GATHER && kind != PLX_PROBE_STREAM &&
      kind != PLX_PROBE_RED_ROWS && kind != PLX_PROBE_ISSUE)
    return fail(PLX_EINVAL, "%s: unknown kind %d", what, kind);
  if (!buf || (reinterpret_cast<uintptr_t>(buf) & 15) != 0)
    return fail(PLX_EINVAL, "%s: buffer null or not 16-byte aligned", what);
  if (n_rows < 1 || n_rows > 0xffffffffll)
    return fail(PLX_EINVAL, "%s: n_rows %lld out of [1, 2^32)", what, (long long)n_rows);
  if (ops < 1 || ops > 1024 || blocks < 1 || blocks > (1 << 20))
    return fail(PLX_EINVAL, "%s: ops %d or blocks %d out of range", what, ops, blocks);
  if ((kind == PLX_PROBE_RED || kind == PLX_PROBE_GATHER) && (group < 1 || group > 32))
    return fail(PLX_EINVAL, "%s: group %d out of [1, 32]", what, group);
  launch_probe(kind, buf, (uint32_t)n_rows, group, ops, blocks, (cudaStream_t)stream);
  return launch_check(what);
}
