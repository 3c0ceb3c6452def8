// Tracking: pose Jacobian (Sec. 5.3, Eq. 12-14, Appendix A) reduced to a
// Gauss-Newton system, and the GN step on SE(3).
//
// The Jacobian needs C and D (Eq. 9-10 hold C - S_i), which are only known at
// the end of the ray. Written as
//   dC/dp_i = delta (c_i T_{i+1} + S_i) grad sigma_i + w_i grad c_i  -  C delta grad sigma_i
// every term except the last is known at sample i, and the last is C times a
// running sum, so one pass suffices: per ray the kernel carries
//   P_X = sum_i (coefficient of grad sigma_i for output X) grad sigma_i [+ w_i grad c_i]
//   Q   = sum_i delta grad sigma_i
// each with its [1, t_i] companion (Eq. 14: dp/do = I, dp/dd = t_i I), and
// forms dX/do = P_X - X Q, dX/dd = P^t_X - X Q^t once X is known. The chain to
// the left perturbation xi = (rho, phi) of the pose is
//   dX/drho = dX/do,  dX/dphi = o x dX/do + d x dX/dd.
// The view-direction variant (not in the paper) adds to the colour rows'
// dX/dd the derivative of the SH colour through Y(d), gathered per cell
// (plx_pose_march.cuh: dir_flush).
//
// Reduction: per ray 29 values (21 of J^T W J, 6 of J^T W r, r^T W r, valid
// count) are formed in FP32 from the FP32 Jacobian. A warp reduce-scatter in
// compensated float-float arithmetic leaves lane L with the warp's sum of
// value L; from there everything is FP64: each lane keeps one FP64
// accumulator across the rays it visits, and blocks write FP64 partials that
// the last block to finish sums in a fixed order. The result is deterministic.
#include "plx_pose_march.cuh"

namespace plx {

// SEGK: one ray per warp, its samples split over the lanes
// (pose_ray_values_seg), for ray counts too small to fill the GPU one ray per
// thread; otherwise one ray per thread, a warp per 32 rays.
template <int STORE, int MINB, bool DIRT = false, bool SEGK = false>
__global__ void __launch_bounds__(kBlock, MINB)
k_backward_pose(const __grid_constant__ Common P, const float* __restrict__ rgb_t,
                const float* __restrict__ depth_t, double* __restrict__ partials,
                unsigned int* __restrict__ retire, double* __restrict__ JtWJ,
                double* __restrict__ JtWr, double* __restrict__ loss_out) {
  __shared__ double red[kWarpsPerBlock][32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc = 0.0;
  const int64_t warps_total = (int64_t)gridDim.x * kWarpsPerBlock;
  if constexpr (SEGK) {
    const int64_t n_slots = P.ct.n_tiles * 32;  // ray slots (some invalid in dense mode)
    for (int64_t ray = (int64_t)blockIdx.x * kWarpsPerBlock + warp; ray < n_slots;
         ray += warps_total) {
      const RayId id = ray_of(P, ray >> 5, (int)(ray & 31));
      RayF r;
      setup_ray(P, id, r, lane);
      const float dz = id.valid ? __ldg(depth_t + id.out) : 0.f;
      if (id.valid && depth_valid(dz)) {  // warp-uniform: every lane has the same ray
        float v[32];
        pose_ray_values_seg<STORE>(P, r, rgb_t + 3 * id.out, dz, lane, v);
        float mine = 0.f;
#pragma unroll
        for (int i = 0; i < 29; ++i) mine = i == lane ? v[i] : mine;
        acc += (double)mine;
      }
    }
  }
  for (int64_t tile = (int64_t)blockIdx.x * kWarpsPerBlock + warp; !SEGK && tile < P.ct.n_tiles;
       tile += warps_total) {
    float v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = 0.f;
    const RayId id = ray_of(P, tile, lane);
    RayF r;
    setup_ray(P, id, r, lane);
    float dz = 0.f;
    if (id.valid) dz = __ldg(depth_t + id.out);
    if (id.valid && depth_valid(dz))
      pose_ray_values<STORE, DIRT, true>(P, r, rgb_t + 3 * id.out, dz, v);
    acc += warp_reduce_scatter(v, lane);
  }
  red[warp][lane] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kWarpsPerBlock; ++w) s += red[w][threadIdx.x];
    partials[(int64_t)blockIdx.x * 32 + threadIdx.x] = s;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned ticket = atomicAdd(retire, 1u);
    last = ticket == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // last block: fixed-order sum of the partials
  double s = 0.0;
  for (int b = warp; b < (int)gridDim.x; b += kWarpsPerBlock)
    s += __ldcg(partials + (int64_t)b * 32 + lane);
  red[warp][lane] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kWarpsPerBlock; ++w) t += red[w][threadIdx.x];
    red[0][threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double M = red[0][28];
    const double inv = M > 0.0 ? 1.0 / M : 0.0;
    for (int i = 0; i < 6; ++i) {
      for (int j = i; j < 6; ++j) {
        const double h = red[0][hidx(i, j)] * inv;
        JtWJ[6 * i + j] = h;
        JtWJ[6 * j + i] = h;
      }
      JtWr[i] = red[0][21 + i] * inv;
    }
    loss_out[0] = red[0][27] * inv;
    loss_out[1] = M;
    *retire = 0u;
  }
}

// ------------------------------------------------------------- GN step
// Solve (H + damping I) xi = -b by Cholesky, pose <- exp(xi^) pose.
__global__ void k_pose_step(const double* __restrict__ H, const double* __restrict__ b,
                            double damping, double* __restrict__ pose,
                            double* __restrict__ xi_out, int32_t* __restrict__ status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double L[6][6], y[6], xi[6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) L[i][j] = 0.0;
  for (int i = 0; i < 6; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = H[6 * i + j] + (i == j ? damping : 0.0);
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      if (i == j) {
        if (!(s > 0.0)) {
          if (status) *status = 1;
          if (xi_out)
            for (int q = 0; q < 6; ++q) xi_out[q] = 0.0;
          return;
        }
        L[i][i] = sqrt(s);
      } else {
        L[i][j] = s / L[j][j];
      }
    }
  }
  for (int i = 0; i < 6; ++i) {
    double s = -b[i];
    for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
    y[i] = s / L[i][i];
  }
  for (int i = 5; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < 6; ++k) s -= L[k][i] * xi[k];
    xi[i] = s / L[i][i];
  }
  se3_exp_left(xi, pose);
  if (xi_out)
    for (int q = 0; q < 6; ++q) xi_out[q] = xi[q];
  if (status) *status = 0;
}

// ---------------------------------------------------- Levenberg-Marquardt
// Solves (H + lam (diag H + 1e-12 max diag H)) xi = -b by Cholesky; false if
// that matrix is not positive definite.
__device__ bool solve_marquardt(const double* H, const double* b, double lam, double xi[6]) {
  double L[6][6], y[6], dmax = 0.0;
  for (int i = 0; i < 6; ++i) dmax = fmax(dmax, H[7 * i]);
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) L[i][j] = 0.0;
  for (int i = 0; i < 6; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = H[6 * i + j] + (i == j ? lam * (H[7 * i] + 1e-12 * dmax) : 0.0);
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      if (i == j) {
        if (!(s > 0.0)) return false;
        L[i][i] = sqrt(s);
      } else {
        L[i][j] = s / L[j][j];
      }
    }
  }
  for (int i = 0; i < 6; ++i) {
    double s = -b[i];
    for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
    y[i] = s / L[i][i];
  }
  for (int i = 5; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < 6; ++k) s -= L[k][i] * xi[k];
    xi[i] = s / L[i][i];
  }
  return true;
}

// One damped step per Jacobian evaluation; state layout in plx.h.
__global__ void k_pose_step_lm(const double* __restrict__ H, const double* __restrict__ b,
                               const double* __restrict__ loss, double* __restrict__ st,
                               double lambda_init, double factor, double* __restrict__ pose,
                               double* __restrict__ xi_out, int32_t* __restrict__ status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const bool first = st[2] == 0.0;
  const double L = loss[0];
  const bool accept = first || !(L > st[1]);
  double lam = first ? lambda_init : st[0];
  if (accept) {
    if (!first) lam = fmax(lam / factor, 1e-12);
    for (int i = 0; i < 12; ++i) st[4 + i] = pose[i];
    st[1] = L;
    for (int i = 0; i < 36; ++i) st[16 + i] = H[i];
    for (int i = 0; i < 6; ++i) st[52 + i] = b[i];
  } else {
    lam = fmin(lam * factor, 1e12);
    for (int i = 0; i < 12; ++i) pose[i] = st[4 + i];
  }
  double xi[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  bool ok = false;
  for (int tries = 0; tries <= 8 && !ok; ++tries) {
    ok = solve_marquardt(st + 16, st + 52, lam, xi);
    if (!ok) lam *= factor;
  }
  st[0] = lam;
  st[2] += 1.0;
  st[3] = accept ? 1.0 : 0.0;
  if (!ok)
    for (int q = 0; q < 6; ++q) xi[q] = 0.0;
  else
    se3_exp_left(xi, pose);
  if (xi_out)
    for (int q = 0; q < 6; ++q) xi_out[q] = xi[q];
  if (status) *status = !ok ? 1 : (accept ? 0 : 2);
}

// ------------------------------------------------------------ host launch
void launch_backward_pose(int store, int minb, const Common& P, const float* rgb_t,
                          const float* depth_t, double* partials, unsigned* retire, double* JtWJ,
                          double* JtWr, double* loss, int max_blocks, cudaStream_t s) {
  int64_t want = (P.ct.n_tiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (want < 1) want = 1;
  const unsigned blocks = (unsigned)(want < max_blocks ? want : max_blocks);
#define PLX_POSE(S, M)                                                                 \
  k_backward_pose<S, M><<<blocks, kBlock, 0, s>>>(P, rgb_t, depth_t, partials, retire, \
                                                  JtWJ, JtWr, loss)
#define PLX_POSE_DIR(S, M)                                                             \
  k_backward_pose<S, M, true><<<blocks, kBlock, 0, s>>>(P, rgb_t, depth_t, partials,   \
                                                        retire, JtWJ, JtWr, loss)
#define PLX_POSE_SEG(S, M)                                                                    \
  k_backward_pose<S, M, false, true><<<seg_blocks, kBlock, 0, s>>>(P, rgb_t, depth_t, partials, \
                                                                   retire, JtWJ, JtWr, loss)
  // few rays: a warp per ray (needs stop_T = 0; the paper's Jacobian only)
  const bool seg =
      P.ct.n_tiles * 32 <= (int64_t)P.g.seg_rays && !(P.o.stop_T > 0.f) && !P.o.dir_term;
  int64_t seg_want = (P.ct.n_tiles * 32 + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (seg_want < 1) seg_want = 1;
  const unsigned seg_blocks = (unsigned)(seg_want < max_blocks ? seg_want : max_blocks);
  if (seg)
    PLX_DISPATCH_SM(store, minb, PLX_POSE_SEG);
  else if (P.o.dir_term)
    PLX_DISPATCH_SM(store, minb, PLX_POSE_DIR);
  else
    PLX_DISPATCH_SM(store, minb, PLX_POSE);
#undef PLX_POSE_SEG
#undef PLX_POSE_DIR
#undef PLX_POSE
}

void launch_pose_step(const double* H, const double* b, double damping, double* pose,
                      double* xi_out, int32_t* status, cudaStream_t s) {
  k_pose_step<<<1, 32, 0, s>>>(H, b, damping, pose, xi_out, status);
}

void launch_pose_step_lm(const double* H, const double* b, const double* loss, double* state,
                         double lambda_init, double factor, double* pose, double* xi_out,
                         int32_t* status, cudaStream_t s) {
  k_pose_step_lm<<<1, 32, 0, s>>>(H, b, loss, state, lambda_init, factor, pose, xi_out, status);
}

int pose_kernel_blocks_per_sm(int store, int minb) {
  int n = 0;
#define PLX_OCC(S, M) \
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_backward_pose<S, M>, kBlock, 0)
  PLX_DISPATCH_SM(store, minb, PLX_OCC);
#undef PLX_OCC
  return n > 0 ? n : 1;
}

}  // namespace plx
