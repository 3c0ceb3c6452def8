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
//
// Reduction: per ray 29 values (21 of J^T W J, 6 of J^T W r, r^T W r, valid
// count) are formed in FP32 from the FP32 Jacobian. A warp reduce-scatter in
// compensated float-float arithmetic leaves lane L with the warp's sum of
// value L; from there everything is FP64: each lane keeps one FP64
// accumulator across the rays it visits, and blocks write FP64 partials that
// the last block to finish sums in a fixed order. The result is deterministic.
#include "plx_internal.cuh"

namespace plx {

// local gradient of the trilinear interpolant of corner values V (unit cell)
__device__ __forceinline__ void grad_local(const float V[8], float x, float y, float z,
                                           float g[3]) {
  const float gx = 1.f - x, gy = 1.f - y, gz = 1.f - z;
  g[0] = gy * gz * (V[1] - V[0]) + y * gz * (V[3] - V[2]) + gy * z * (V[5] - V[4]) +
         y * z * (V[7] - V[6]);
  g[1] = gx * gz * (V[2] - V[0]) + x * gz * (V[3] - V[1]) + gx * z * (V[6] - V[4]) +
         x * z * (V[7] - V[5]);
  g[2] = gx * gy * (V[4] - V[0]) + x * gy * (V[5] - V[1]) + gx * y * (V[6] - V[2]) +
         x * y * (V[7] - V[3]);
}

struct PoseAcc {
  float Po[4][3], Pd[4][3];  // per output X in (R, G, B, D)
  float Qo[3], Qd[3];
};

template <int STORE>
__device__ __forceinline__ void march_pose(const Common& P, const RayF& r, const float Y[9],
                                           float C[3], float& D, float& T, PoseAcc& A) {
  const int rm2x = P.g.rx - 2, rm2y = P.g.ry - 2, rm2z = P.g.rz - 2;
  const float ihx = (float)P.g.inv_h[0], ihy = (float)P.g.inv_h[1], ihz = (float)P.g.inv_h[2];
  int cx = -1, cy = -1, cz = -1;
  bool empty = true;
  int32_t l[8];
  float cs[8], cc[8][3];
  float S[3] = {0.f, 0.f, 0.f}, SD = 0.f;
  T = 1.f;
  const float dt = r.dt;
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
    if (empty) continue;
    float w[8];
    corner_weights(fx, fy, fz, w);
    float sig = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) sig = fmaf(w[c], cs[c], sig);
    if (!(sig > 0.f)) continue;
    float gsig[3];
    grad_local(cs, fx, fy, fz, gsig);
    gsig[0] *= ihx; gsig[1] *= ihy; gsig[2] *= ihz;
    float alpha, keep;
    alpha_of(sig * dt, alpha, keep);
    const float wgt = T * alpha;
    const float Tn = T * keep;
    const float t = fmaf(kf, dt, r.t0);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      float V[8];
      float a = 0.f;
#pragma unroll
      for (int c = 0; c < 8; ++c) { V[c] = cc[c][ch]; a = fmaf(w[c], V[c], a); }
      float dact;
      const float col = activate(a, P.o.color_act, dact);
      float gch[3];
      grad_local(V, fx, fy, fz, gch);
      S[ch] = fmaf(wgt, col, S[ch]);
      const float cs_coef = dt * (col * Tn + S[ch]);
      const float cc_coef = wgt * dact;
      const float u0 = cs_coef * gsig[0] + cc_coef * gch[0] * ihx;
      const float u1 = cs_coef * gsig[1] + cc_coef * gch[1] * ihy;
      const float u2 = cs_coef * gsig[2] + cc_coef * gch[2] * ihz;
      A.Po[ch][0] += u0; A.Po[ch][1] += u1; A.Po[ch][2] += u2;
      A.Pd[ch][0] = fmaf(t, u0, A.Pd[ch][0]);
      A.Pd[ch][1] = fmaf(t, u1, A.Pd[ch][1]);
      A.Pd[ch][2] = fmaf(t, u2, A.Pd[ch][2]);
    }
    SD = fmaf(wgt, t, SD);
    const float dcoef = dt * (t * Tn + SD);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float ud = dcoef * gsig[a];
      A.Po[3][a] += ud;
      A.Pd[3][a] = fmaf(t, ud, A.Pd[3][a]);
      const float q = dt * gsig[a];
      A.Qo[a] += q;
      A.Qd[a] = fmaf(t, q, A.Qd[a]);
    }
    T = Tn;
    if (T < P.o.stop_T) break;
  }
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) C[ch] = fmaf(T, P.o.bg[ch], S[ch]);
  D = SD;
}

// Per-ray values reduced: 21 of H (index below), 6 of b at 21..26, the loss at
// 27 and the valid-ray count at 28. Value index of H_ij (i <= j):
__host__ __device__ constexpr int hidx(int i, int j) { return i * 6 - i * (i - 1) / 2 + (j - i); }

// Warp reduce-scatter of v[0..31]: lane L returns the sum over the warp of
// v[L]. Sums are carried as float-float pairs (about 44 significant bits), so
// the FP32 pipes do the work and the FP64 pipe, slow on this part, is used
// once per lane at the end.
__device__ __forceinline__ double warp_reduce_scatter(const float v[32], int lane) {
  ff a[16];
  {
    const bool up = lane & 16;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float send = up ? v[i] : v[i + 16];
      const float keep = up ? v[i + 16] : v[i];
      a[i] = two_sum(keep, __shfl_xor_sync(0xffffffffu, send, 16));
    }
  }
#pragma unroll
  for (int off = 8; off >= 1; off >>= 1) {
    const bool up = lane & off;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      const ff send = up ? a[i] : a[i + off];
      const ff keep = up ? a[i + off] : a[i];
      const ff recv = ffv(__shfl_xor_sync(0xffffffffu, send.h, off),
                          __shfl_xor_sync(0xffffffffu, send.l, off));
      a[i] = ff_add(keep, recv);
    }
  }
  return (double)a[0].h + (double)a[0].l;
}

template <int STORE>
__global__ void __launch_bounds__(kBlock, PLX_POSE_MIN_BLOCKS)
k_backward_pose(const __grid_constant__ Common P, const float* __restrict__ rgb_t,
                const float* __restrict__ depth_t, double* __restrict__ partials,
                unsigned int* __restrict__ retire, double* __restrict__ JtWJ,
                double* __restrict__ JtWr, double* __restrict__ loss_out) {
  __shared__ double red[kWarpsPerBlock][32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float lam = P.o.lambda_d;
  double acc = 0.0;
  const int64_t warps_total = (int64_t)gridDim.x * kWarpsPerBlock;
  for (int64_t tile = (int64_t)blockIdx.x * kWarpsPerBlock + warp; tile < P.ct.n_tiles;
       tile += warps_total) {
    float v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = 0.f;
    const RayId id = ray_of(P, tile, lane);
    RayF r;
    setup_ray(P, id, r, lane);
    float dz = 0.f;
    if (id.valid) dz = __ldg(depth_t + id.out);
    if (id.valid && depth_valid(dz)) {
      float Y[9];
      sh_basis(r.dir, Y);
      PoseAcc A;
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int a = 0; a < 3; ++a) A.Po[x][a] = A.Pd[x][a] = 0.f;
#pragma unroll
      for (int a = 0; a < 3; ++a) A.Qo[a] = A.Qd[a] = 0.f;
      float C[3], D, T;
      march_pose<STORE>(P, r, Y, C, D, T, A);
      const float Dt = P.o.depth_is_z ? dz * r.dc_norm : dz;
      float res[4], J[4][6];
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        const float X = x < 3 ? C[x] : D;
        res[x] = X - (x < 3 ? __ldg(rgb_t + 3 * id.out + x) : Dt);
        float jo[3], jd[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          jo[a] = A.Po[x][a] - X * A.Qo[a];
          jd[a] = A.Pd[x][a] - X * A.Qd[a];
        }
        const float* o = r.org;
        const float* d = r.dir;
        J[x][0] = jo[0]; J[x][1] = jo[1]; J[x][2] = jo[2];
        J[x][3] = (o[1] * jo[2] - o[2] * jo[1]) + (d[1] * jd[2] - d[2] * jd[1]);
        J[x][4] = (o[2] * jo[0] - o[0] * jo[2]) + (d[2] * jd[0] - d[0] * jd[2]);
        J[x][5] = (o[0] * jo[1] - o[1] * jo[0]) + (d[0] * jd[1] - d[1] * jd[0]);
      }
#pragma unroll
      for (int i = 0; i < 6; ++i) {
#pragma unroll
        for (int j = i; j < 6; ++j) {
          float h = J[3][i] * J[3][j] * lam;
#pragma unroll
          for (int x = 0; x < 3; ++x) h = fmaf(J[x][i], J[x][j], h);
          v[hidx(i, j)] = h;
        }
        float bb = J[3][i] * res[3] * lam;
#pragma unroll
        for (int x = 0; x < 3; ++x) bb = fmaf(J[x][i], res[x], bb);
        v[21 + i] = bb;
      }
      v[27] = res[0] * res[0] + res[1] * res[1] + res[2] * res[2] + lam * res[3] * res[3];
      v[28] = 1.f;
    }
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
  // SE(3) exponential of (rho, phi)
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
  if (xi_out)
    for (int q = 0; q < 6; ++q) xi_out[q] = xi[q];
  if (status) *status = 0;
}

// ------------------------------------------------------------ host launch
template <int STORE>
static void launch_pose_t(const Common& P, const float* rgb_t, const float* depth_t,
                          double* partials, unsigned* retire, double* JtWJ, double* JtWr,
                          double* loss, int max_blocks, cudaStream_t s) {
  int64_t want = (P.ct.n_tiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (want < 1) want = 1;
  const unsigned blocks = (unsigned)(want < max_blocks ? want : max_blocks);
  k_backward_pose<STORE><<<blocks, kBlock, 0, s>>>(P, rgb_t, depth_t, partials, retire, JtWJ,
                                                   JtWr, loss);
}

void launch_backward_pose(int store, const Common& P, const float* rgb_t, const float* depth_t,
                          double* partials, unsigned* retire, double* JtWJ, double* JtWr,
                          double* loss, int max_blocks, cudaStream_t s) {
  switch (store) {
    case PLX_STORE_F32:
      launch_pose_t<PLX_STORE_F32>(P, rgb_t, depth_t, partials, retire, JtWJ, JtWr, loss,
                                   max_blocks, s);
      break;
    case PLX_STORE_BF16:
      launch_pose_t<PLX_STORE_BF16>(P, rgb_t, depth_t, partials, retire, JtWJ, JtWr, loss,
                                    max_blocks, s);
      break;
    case PLX_STORE_F16:
      launch_pose_t<PLX_STORE_F16>(P, rgb_t, depth_t, partials, retire, JtWJ, JtWr, loss,
                                   max_blocks, s);
      break;
    default:
      launch_pose_t<PLX_STORE_F32_BF16>(P, rgb_t, depth_t, partials, retire, JtWJ, JtWr, loss,
                                        max_blocks, s);
      break;
  }
}

void launch_pose_step(const double* H, const double* b, double damping, double* pose,
                      double* xi_out, int32_t* status, cudaStream_t s) {
  k_pose_step<<<1, 32, 0, s>>>(H, b, damping, pose, xi_out, status);
}

int pose_kernel_blocks_per_sm(int store) {
  int n = 0;
  switch (store) {
    case PLX_STORE_F32:
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_backward_pose<PLX_STORE_F32>, kBlock, 0);
      break;
    case PLX_STORE_BF16:
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_backward_pose<PLX_STORE_BF16>, kBlock, 0);
      break;
    case PLX_STORE_F16:
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_backward_pose<PLX_STORE_F16>, kBlock, 0);
      break;
    default:
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_backward_pose<PLX_STORE_F32_BF16>,
                                                    kBlock, 0);
      break;
  }
  return n > 0 ? n : 1;
}

}  // namespace plx
