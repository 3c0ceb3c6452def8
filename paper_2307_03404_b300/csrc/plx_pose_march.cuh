// Pose-Jacobian march and the warp reduction shared by the tracking and
// batched kernels (see plx_pose.cu for the derivation).
#pragma once

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
  float G[3][3];             // view-direction variant: d C_ch / d d through Y(d)
};

// sum_k k9[k] grad Y_k(d): the gradient of the SH sum with respect to the
// direction, from the polynomials of sh_basis.
__device__ __forceinline__ void sh_dir_grad(const float d[3], const float* k9, float q[3]) {
  const float c1 = 0.48860251190291992f, c2 = 1.09254843059207907f;
  const float c20 = 0.31539156525252005f, c22 = 0.54627421529603959f;
  const float x = d[0], y = d[1], z = d[2];
  q[0] = c1 * k9[3] + c2 * (y * k9[4] + z * k9[7]) + 2.f * c22 * x * k9[8];
  q[1] = c1 * k9[1] + c2 * (x * k9[4] + z * k9[5]) - 2.f * c22 * y * k9[8];
  q[2] = c1 * k9[2] + c2 * (y * k9[5] + x * k9[7]) + 6.f * c20 * z * k9[6];
}

// View-direction variant: the per-corner weights sum_i w_i dc_i/dchat w_c(p_i)
// gathered over the samples a ray took in one cell are applied when it leaves
// the cell, to the corner's SH sum differentiated in the direction (the
// records are re-read; they were loaded for this cell moments before).
template <int STORE>
__device__ __forceinline__ void dir_flush(const GridView& g, const int32_t l[8], float Ac[8][3],
                                          const float d[3], float G[3][3]) {
#pragma unroll 1
  for (int c = 0; c < 8; ++c) {
    if (l[c] >= 0 && (Ac[c][0] != 0.f || Ac[c][1] != 0.f || Ac[c][2] != 0.f)) {
      float v[28];
      load_record<STORE>(g.rec, l[c], v);
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        float q[3];
        sh_dir_grad(d, v + 1 + 9 * ch, q);
        G[ch][0] = fmaf(Ac[c][ch], q[0], G[ch][0]);
        G[ch][1] = fmaf(Ac[c][ch], q[1], G[ch][1]);
        G[ch][2] = fmaf(Ac[c][ch], q[2], G[ch][2]);
      }
    }
    Ac[c][0] = Ac[c][1] = Ac[c][2] = 0.f;
  }
}

// SMEM: the cell's corner cache lives in shared memory (slot s of this
// thread at sc[s * kBlock], as in the adjoint), so registers hold the corner
// values only while a sample uses them.
// SEG: march only samples [k0, k1) of the ray as if they were the whole ray
// (transmittance from 1, colour and depth sums from 0, no background, no early
// stop): the segment's local quantities, combined across segments by
// pose_ray_values_seg.
template <int STORE, bool DIRT = false, bool SMEM = false, bool SEG = false>
__device__ __forceinline__ void march_pose(const Common& P, const RayF& r, const float Y[9],
                                           float C[3], float& D, float& T, PoseAcc& A,
                                           int k0 = 0, int k1 = 0) {
  const int rm2x = P.g.rx - 2, rm2y = P.g.ry - 2, rm2z = P.g.rz - 2;
  const float ihx = (float)P.g.inv_h[0], ihy = (float)P.g.inv_h[1], ihz = (float)P.g.inv_h[2];
  int cx = -1, cy = -1, cz = -1;
  bool empty = true;
  int32_t l[8];
  float cs_r[SMEM ? 1 : 8], cc_r[SMEM ? 1 : 8][3];
  float* sc = nullptr;
  if constexpr (SMEM) {
    sc = corner_cache_smem() + threadIdx.x;
  }
  float S[3] = {0.f, 0.f, 0.f}, SD = 0.f;
  float Ac[DIRT ? 8 : 1][3];
  if constexpr (DIRT) {
#pragma unroll
    for (int c = 0; c < 8; ++c) Ac[c][0] = Ac[c][1] = Ac[c][2] = 0.f;
  }
  T = 1.f;
  const float dt = r.dt;
  const int k_end = SEG ? k1 : r.n;
  for (int k = SEG ? k0 : 0; k < k_end; ++k) {
    const float kf = (float)k;
    int ix, iy, iz;
    float fx, fy, fz;
    sample_axis(r.B[0], r.S[0], k, rm2x, ix, fx);
    sample_axis(r.B[1], r.S[1], k, rm2y, iy, fy);
    sample_axis(r.B[2], r.S[2], k, rm2z, iz, fz);
    if (ix != cx || iy != cy || iz != cz) {
      if constexpr (DIRT) {
        if (!empty) dir_flush<STORE>(P.g, l, Ac, r.dir, A.G);
      }
      cx = ix; cy = iy; cz = iz;
      const int esh = empty_block_shift(P.g, ix, iy, iz);
      if (esh >= 0) {
        empty = true;
        k = block_exit(r, ix, iy, iz, k, esh) - 1;
        continue;
      }
      if constexpr (SMEM)
        empty = load_cell_smem<STORE>(P.g, ix, iy, iz, Y, l, sc);
      else
        empty = load_cell<STORE>(P.g, ix, iy, iz, Y, l, cs_r, cc_r);
    }
    if (empty) continue;
    float w[8], cs[8];
    corner_weights(fx, fy, fz, w);
#pragma unroll
    for (int c = 0; c < 8; ++c) cs[c] = SMEM ? sc[(4 * c) * kBlock] : cs_r[SMEM ? 0 : c];
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
      for (int c = 0; c < 8; ++c) {
        V[c] = SMEM ? sc[(4 * c + 1 + ch) * kBlock] : cc_r[SMEM ? 0 : c][ch];
        a = fmaf(w[c], V[c], a);
      }
      float dact;
      const float col = activate(a, P.o.color_act, dact);
      float gch[3];
      grad_local(V, fx, fy, fz, gch);
      S[ch] = fmaf(wgt, col, S[ch]);
      const float cs_coef = dt * (col * Tn + S[ch]);
      const float cc_coef = wgt * dact;
      if constexpr (DIRT) {
#pragma unroll
        for (int c = 0; c < 8; ++c) Ac[c][ch] = fmaf(cc_coef, w[c], Ac[c][ch]);
      }
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
    if (!SEG && T < P.o.stop_T) break;
  }
  if constexpr (DIRT) {
    if (!empty) dir_flush<STORE>(P.g, l, Ac, r.dir, A.G);
  }
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) C[ch] = SEG ? S[ch] : fmaf(T, P.o.bg[ch], S[ch]);
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

// The ray's 29 values from its colour C, depth D and accumulators (see
// pose_ray_values).
template <bool DIRT>
__device__ __forceinline__ void pose_values_from(const Common& P, const RayF& r,
                                                 const float* __restrict__ rgb_t, float dz,
                                                 const float C[3], float D, const PoseAcc& A,
                                                 float v[32]) {
  const float lam = P.o.lambda_d;
  const float Dt = P.o.depth_is_z ? dz * r.dc_norm : dz;
  float res[4], J[4][6];
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const float X = x < 3 ? C[x] : D;
    res[x] = X - (x < 3 ? __ldg(rgb_t + x) : Dt);
    float jo[3], jd[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      jo[a] = A.Po[x][a] - X * A.Qo[a];
      jd[a] = A.Pd[x][a] - X * A.Qd[a];
      if constexpr (DIRT) {
        if (x < 3) jd[a] += A.G[x][a];
      }
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

// One valid ray's contribution to the Gauss-Newton system: v[0..20] = the upper
// triangle of J^T W J (index hidx), v[21..26] = J^T W r, v[27] = r^T W r,
// v[28] = 1 (count), with W = diag(1, 1, 1, lambda_d) (1/M is applied after the
// reduction). rgb_t points at the ray's colour target, dz is its depth target.
template <int STORE, bool DIRT = false, bool SMEM = false>
__device__ __forceinline__ void pose_ray_values(const Common& P, const RayF& r,
                                                const float* __restrict__ rgb_t, float dz,
                                                float v[32]) {
  float Y[9];
  sh_basis(r.dir, Y);
  PoseAcc A;
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int a = 0; a < 3; ++a) A.Po[x][a] = A.Pd[x][a] = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) A.Qo[a] = A.Qd[a] = 0.f;
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) A.G[ch][0] = A.G[ch][1] = A.G[ch][2] = 0.f;
  float C[3], D, T;
  march_pose<STORE, DIRT, SMEM>(P, r, Y, C, D, T, A);
  pose_values_from<DIRT>(P, r, rgb_t, dz, C, D, A, v);
}

// Warp-per-ray form of pose_ray_values, for few rays (tracking on a random
// subset of a frame): the 32 lanes of the warp march consecutive segments of
// the same ray, each from transmittance 1 and zero sums. A segment's true
// transmittance at entry T0 and colour/depth sums S0, SD0 follow from an
// exclusive scan over the lanes of (T_seg, S_seg) under
// (T_a, S_a) o (T_b, S_b) = (T_a T_b, S_a + T_a S_b); every per-sample term of
// the single-pass Jacobian is then T0 times its local value plus S0 (SD0 for
// depth) times the local Q = sum delta grad sigma, so the ray's sums are
// sum_lanes (T0 P_loc + S0 Q_loc). The warp then holds the whole ray's values
// in every lane. Needs stop_T = 0 (a lane cannot stop on the global T).
// Must be called by all 32 lanes with the same ray.
template <int STORE>
__device__ __forceinline__ void pose_ray_values_seg(const Common& P, const RayF& r,
                                                    const float* __restrict__ rgb_t, float dz,
                                                    int lane, float v[32]) {
  float Y[9];
  sh_basis(r.dir, Y);
  PoseAcc A;
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int a = 0; a < 3; ++a) A.Po[x][a] = A.Pd[x][a] = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) A.Qo[a] = A.Qd[a] = 0.f;
  const int k0 = (int)(((int64_t)r.n * lane) >> 5), k1 = (int)(((int64_t)r.n * (lane + 1)) >> 5);
  float S[3], SD, T;
  march_pose<STORE, false, true, true>(P, r, Y, S, SD, T, A, k0, k1);
  // inclusive scan of (T, S[3], SD) over lanes, then shift to exclusive
  float iT = T, iS0 = S[0], iS1 = S[1], iS2 = S[2], iSD = SD;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float pT = __shfl_up_sync(0xffffffffu, iT, off);
    const float p0 = __shfl_up_sync(0xffffffffu, iS0, off);
    const float p1 = __shfl_up_sync(0xffffffffu, iS1, off);
    const float p2 = __shfl_up_sync(0xffffffffu, iS2, off);
    const float pD = __shfl_up_sync(0xffffffffu, iSD, off);
    if (lane >= off) {  // (earlier prefix) o (this lane's inclusive part)
      iS0 = fmaf(pT, iS0, p0);
      iS1 = fmaf(pT, iS1, p1);
      iS2 = fmaf(pT, iS2, p2);
      iSD = fmaf(pT, iSD, pD);
      iT *= pT;
    }
  }
  float T0 = __shfl_up_sync(0xffffffffu, iT, 1);
  float S00 = __shfl_up_sync(0xffffffffu, iS0, 1), S01 = __shfl_up_sync(0xffffffffu, iS1, 1);
  float S02 = __shfl_up_sync(0xffffffffu, iS2, 1), SD0 = __shfl_up_sync(0xffffffffu, iSD, 1);
  if (lane == 0) T0 = 1.f, S00 = S01 = S02 = SD0 = 0.f;
  const float Tn = __shfl_sync(0xffffffffu, iT, 31);
  float C[3] = {__shfl_sync(0xffffffffu, iS0, 31), __shfl_sync(0xffffffffu, iS1, 31),
                __shfl_sync(0xffffffffu, iS2, 31)};
  const float D = __shfl_sync(0xffffffffu, iSD, 31);
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) C[ch] = fmaf(Tn, P.o.bg[ch], C[ch]);
  // this lane's share of the ray's sums, then the warp sum in every lane
  const float S0[4] = {S00, S01, S02, SD0};
  PoseAcc R;
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      R.Po[x][a] = fmaf(T0, A.Po[x][a], S0[x] * A.Qo[a]);
      R.Pd[x][a] = fmaf(T0, A.Pd[x][a], S0[x] * A.Qd[a]);
    }
#pragma unroll
  for (int a = 0; a < 3; ++a) {  // Q = sum delta grad sigma does not depend on T
    R.Qo[a] = A.Qo[a];
    R.Qd[a] = A.Qd[a];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        R.Po[x][a] += __shfl_xor_sync(0xffffffffu, R.Po[x][a], off);
        R.Pd[x][a] += __shfl_xor_sync(0xffffffffu, R.Pd[x][a], off);
      }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      R.Qo[a] += __shfl_xor_sync(0xffffffffu, R.Qo[a], off);
      R.Qd[a] += __shfl_xor_sync(0xffffffffu, R.Qd[a], off);
    }
  }
  pose_values_from<false>(P, r, rgb_t, dz, C, D, R, v);
}

}  // namespace plx
