// Ray-march loops shared by the forward, adjoint and batched kernels.
#pragma once

#include "plx_internal.cuh"

namespace plx {

// With cap > 0 (the sample cache on) the samples that composite are kept for
// the grid adjoint: (sigma, colour) and k of the first cap of them, and their
// number, in row `out` of the cache; returns that number (0 when off).
// SEG: march only samples [k0, k1) as if they were the whole ray
// (transmittance from 1, sums from 0, no background, no early stop, no
// cache): the segment's local (T, C, D), combined across the lanes of a warp
// by seg_scan.
// SMEM: the cell's corners in the block's shared corner cache (this
// thread's column of corner_cache_smem) instead of 32 registers: slower in
// the forward kernel, but the batched kernel, whose paths compete for 128
// registers, spills less.
// RANGE: also write the ray's compositing range (first sample with
// sigma > 0, one past the last; 0, 0 when none) to P.o.range[out].
template <int STORE, bool COUNT, bool SEG = false, bool SMEM = false, bool RANGE = false>
__device__ __forceinline__ int march_forward(const Common& P, const RayF& r, const float Y[9],
                                             float C[3], float& D, float& T, int& n_all,
                                             int& n_occ, int64_t out, int cap, int k0 = 0,
                                             int k1 = 0) {
  const int rm2x = P.g.rx - 2, rm2y = P.g.ry - 2, rm2z = P.g.rz - 2;
  int cx = -1, cy = -1, cz = -1;
  bool empty = true;
  int32_t l[8];
  float cs_r[SMEM ? 1 : 8], cc_r[SMEM ? 1 : 8][3];
  float* sc = nullptr;
  if constexpr (SMEM) sc = corner_cache_smem() + threadIdx.x;
  C[0] = C[1] = C[2] = 0.f;
  D = 0.f;
  T = 1.f;
  n_all = r.n;
  int kept = 0;
  int rfirst = -1, rlast = -1;
  if constexpr (SEG) cap = 0;
  const int k_end = SEG ? k1 : r.n;
  for (int k = SEG ? k0 : 0; k < k_end; ++k) {
    const float kf = (float)k;
    int ix, iy, iz;
    float fx, fy, fz;
    sample_axis(r.B[0], r.S[0], k, rm2x, ix, fx);
    sample_axis(r.B[1], r.S[1], k, rm2y, iy, fy);
    sample_axis(r.B[2], r.S[2], k, rm2z, iz, fz);
    if (ix != cx || iy != cy || iz != cz) {
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
    if (COUNT) n_occ += empty ? 0 : 1;
    if (empty) continue;
    float w[8];
    corner_weights(fx, fy, fz, w);
    float sig = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c)
      sig = fmaf(w[c], SMEM ? sc[(4 * c) * kBlock] : cs_r[SMEM ? 0 : c], sig);
    if (!(sig > 0.f)) continue;
    float col[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      float a = 0.f;
#pragma unroll
      for (int c = 0; c < 8; ++c)
        a = fmaf(w[c], SMEM ? sc[(4 * c + 1 + ch) * kBlock] : cc_r[SMEM ? 0 : c][ch], a);
      float dact;
      col[ch] = activate(a, P.o.color_act, dact);
    }
    if constexpr (RANGE) {
      if (rfirst < 0) rfirst = k;
      rlast = k;
    }
    if (cap > 0) {
      if (kept < cap) {
        const int64_t at = (int64_t)kept * P.o.cn + out;
        // streaming stores: the cache is read once, by the next launch, and
        // should not push the grid's lines out of L2
        __stcs(P.o.cval + at, make_float4(sig, col[0], col[1], col[2]));
        __stcs(P.o.ck + at, k);
      }
      ++kept;
    }
    float alpha, keep;
    alpha_of(sig * r.dt, alpha, keep);
    const float wgt = T * alpha;
    const float t = fmaf(kf, r.dt, r.t0);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) C[ch] = fmaf(wgt, col[ch], C[ch]);
    D = fmaf(wgt, t, D);
    T *= keep;
    if (!SEG && T < P.o.stop_T) {
      n_all = k + 1;
      break;
    }
  }
  if (cap > 0) P.o.ccount[out] = kept;
  if constexpr (RANGE)
    P.o.range[out] = rfirst < 0 ? make_int2(0, 0) : make_int2(rfirst, rlast + 1);
  if constexpr (!SEG) {
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) C[ch] = fmaf(T, P.o.bg[ch], C[ch]);
  }
  return kept;
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

// Leaves the current cell for the one (dx, dy, dz) away: if `carry` and the
// step is to a face-adjacent cell, the shared face's sums move to their new
// slots and the rest are flushed; otherwise all are flushed. Returns whether
// carried sums remain in registers. The re-march of the batched kernel uses
// this form (its registers are the scarcest).
__device__ __forceinline__ bool leave_cell_face(float* __restrict__ grad, const int32_t l[8],
                                           float gs[8], float gc[8][3], const float Y[9], int dx,
                                           int dy, int dz, bool carry) {
  int step = -1;  // face-adjacent step: 0/1 = +x/-x, 2/3 = +y/-y, 4/5 = +z/-z
  if (carry) {
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
  return step >= 0;
}

// The register moves of a step by (DX, DY, DZ) (each -1, 0 or 1) into a
// neighbouring cell: corner n of the new cell is corner n + (DX, DY, DZ) of
// the old one when that lies in the old cell (a face step shares 4 corners,
// an edge step 2, a corner step 1) and keeps its sums; the other slots start
// from zero. Every index is a compile-time constant.
template <int DX, int DY, int DZ>
__device__ __forceinline__ void move_shared(float gs[8], float gc[8][3]) {
  float ts[8], tc[8][3];
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const int ox = (n & 1) + DX, oy = ((n >> 1) & 1) + DY, oz = ((n >> 2) & 1) + DZ;
    const bool from = ox >= 0 && ox <= 1 && oy >= 0 && oy <= 1 && oz >= 0 && oz <= 1;
    const int o = from ? ox + 2 * oy + 4 * oz : 0;
    ts[n] = from ? gs[o] : 0.f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) tc[n][ch] = from ? gc[o][ch] : 0.f;
  }
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    gs[n] = ts[n];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) gc[n][ch] = tc[n][ch];
  }
}

// The register moves of move_shared<dx, dy, dz> for a step known only at run
// time, as up to three one-axis moves: moving by dx along x, then dy along y,
// then dz along z leaves slot n holding old corner n + (dx, dy, dz) when that
// lies in the old cell on every axis and zero otherwise, which is the
// diagonal move. Six short bodies instead of 26 keep the adjoint's loop small
// enough for the instruction cache.
__device__ __forceinline__ void move_by(int dx, int dy, int dz, float gs[8], float gc[8][3]) {
  if (dx > 0) move_shared<1, 0, 0>(gs, gc);
  else if (dx < 0) move_shared<-1, 0, 0>(gs, gc);
  if (dy > 0) move_shared<0, 1, 0>(gs, gc);
  else if (dy < 0) move_shared<0, -1, 0>(gs, gc);
  if (dz > 0) move_shared<0, 0, 1>(gs, gc);
  else if (dz < 0) move_shared<0, 0, -1>(gs, gc);
}

// Leaves the current cell for the one (dx, dy, dz) away. If `carry` and the
// new cell touches the old one (every |d| <= 1), the corners the two cells
// share are the same vertices: their sums stay in registers and move to their
// new slots, and only the other corners are flushed (4 of 8 on a face step,
// 6 on an edge step, 7 on a corner step); otherwise all are flushed. Returns
// whether carried sums remain in registers. Against carrying on face steps
// only it cut the sample-cache adjoint's flushes from 2.26 to 2.06 per kept
// sample on room256. AXIS: the moves by move_by (the re-marching adjoint),
// else by one of 26 compile-time bodies (the batched kernel, where move_by
// measured slower).
template <bool AXIS>
__device__ __forceinline__ bool leave_cell(float* __restrict__ grad, const int32_t l[8],
                                           float gs[8], float gc[8][3], const float Y[9], int dx,
                                           int dy, int dz, bool carry) {
  const bool adj = carry && dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1;
  // old corner c = (bx, by, bz) is shared when, on every axis that moves, it
  // lies on the side the ray moves to
  unsigned keep = 0;
  if (adj) {
    const unsigned mx = dx == 0 ? 0xffu : (dx > 0 ? 0xaau : 0x55u);
    const unsigned my = dy == 0 ? 0xffu : (dy > 0 ? 0xccu : 0x33u);
    const unsigned mz = dz == 0 ? 0xffu : (dz > 0 ? 0xf0u : 0x0fu);
    keep = mx & my & mz;
  }
#pragma unroll
  for (int c = 0; c < 8; ++c)
    if (!((keep >> c) & 1u)) flush_corner(grad, l[c], gs[c], gc[c], Y);
  if (!adj) {
#pragma unroll
    for (int c = 0; c < 8; ++c) clear_corner(gs[c], gc[c]);
    return false;
  }
  if constexpr (AXIS) {
    move_by(dx, dy, dz, gs, gc);
  } else {
    switch ((dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)) {
#define PLX_MOVE(X, Y_, Z)                         \
  case ((X) + 1) + 3 * ((Y_) + 1) + 9 * ((Z) + 1): \
    move_shared<X, Y_, Z>(gs, gc);                 \
    break;
      PLX_MOVE(-1, -1, -1) PLX_MOVE(0, -1, -1) PLX_MOVE(1, -1, -1)
      PLX_MOVE(-1, 0, -1) PLX_MOVE(0, 0, -1) PLX_MOVE(1, 0, -1)
      PLX_MOVE(-1, 1, -1) PLX_MOVE(0, 1, -1) PLX_MOVE(1, 1, -1)
      PLX_MOVE(-1, -1, 0) PLX_MOVE(0, -1, 0) PLX_MOVE(1, -1, 0)
      PLX_MOVE(-1, 0, 0) PLX_MOVE(1, 0, 0)
      PLX_MOVE(-1, 1, 0) PLX_MOVE(0, 1, 0) PLX_MOVE(1, 1, 0)
      PLX_MOVE(-1, -1, 1) PLX_MOVE(0, -1, 1) PLX_MOVE(1, -1, 1)
      PLX_MOVE(-1, 0, 1) PLX_MOVE(0, 0, 1) PLX_MOVE(1, 0, 1)
      PLX_MOVE(-1, 1, 1) PLX_MOVE(0, 1, 1) PLX_MOVE(1, 1, 1)
#undef PLX_MOVE
      default: break;  // (0, 0, 0): the same cell, not a step
    }
  }
  return true;
}

// FULL: carry the corners shared on face, edge and corner steps
// (leave_cell<true>, the moves done axis by axis), else on face steps only.
// The full carry with one of 26 move bodies per step took 13.8 against 11.4
// ms on room256 (spills, code size); with the axis moves 10.7 against 10.9 ms
// in FP32 and 8.7 against 12.2 ms in BF16.
// SEG: samples [k0, k1) only, entered with transmittance T0 and prefix sums
// S0, SD0 of the samples before k0 (from seg_scan), no early stop.
template <int STORE, bool SEG = false, bool FULL = true>
__device__ __forceinline__ void march_backward(const Common& P, const RayF& r, const float Y[9],
                                               const float Cf[3], float Df, const float gC[3],
                                               float gD, float* __restrict__ grad, int k0 = 0,
                                               int k1 = 0, float T0 = 1.f,
                                               const float* S0 = nullptr, float SD0 = 0.f,
                                               int2 range = make_int2(0, 0x7fffffff)) {
  const int rm2x = P.g.rx - 2, rm2y = P.g.ry - 2, rm2z = P.g.rz - 2;
  int cx = -1, cy = -1, cz = -1;
  bool empty = true, dirty = false;
  int32_t l[8];
  float* sc = corner_cache_smem() + threadIdx.x;  // corner cache in shared memory: frees 32 registers
  float gs[8], gc[8][3];
#pragma unroll
  for (int c = 0; c < 8; ++c) clear_corner(gs[c], gc[c]);
  float S[3] = {0.f, 0.f, 0.f}, SD = 0.f, T = 1.f;
  if constexpr (SEG) {
    T = T0;
    S[0] = S0[0]; S[1] = S0[1]; S[2] = S0[2];
    SD = SD0;
  }
  const float dt = r.dt;
  // without SEG, `range` limits the march to the ray's compositing samples:
  // nothing before range.x composites (T = 1, sums 0 there), nothing after
  const int k_end = SEG ? k1 : (range.y < r.n ? range.y : r.n);
  for (int k = SEG ? k0 : range.x; k < k_end; ++k) {
    const float kf = (float)k;
    int ix, iy, iz;
    float fx, fy, fz;
    sample_axis(r.B[0], r.S[0], k, rm2x, ix, fx);
    sample_axis(r.B[1], r.S[1], k, rm2y, iy, fy);
    sample_axis(r.B[2], r.S[2], k, rm2z, iz, fz);
    if (ix != cx || iy != cy || iz != cz) {
      const int esh = empty_block_shift(P.g, ix, iy, iz);
      const bool skip = esh >= 0;
      if (dirty)  // carried sums still have to reach memory
        dirty = FULL ? leave_cell<true>(grad, l, gs, gc, Y, ix - cx, iy - cy, iz - cz, !skip)
                     : leave_cell_face(grad, l, gs, gc, Y, ix - cx, iy - cy, iz - cz, !skip);
      cx = ix; cy = iy; cz = iz;
      if (skip) {
        empty = true;
        k = block_exit(r, ix, iy, iz, k, esh) - 1;
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
    if (!SEG && T < P.o.stop_T) break;
  }
  if (dirty) flush_cell(grad, l, gs, gc, Y);
}

// The same adjoint over the n_kept samples the forward kept in the sample
// cache (row `out`): sigma and colour are read back instead of interpolated,
// so no cell record is gathered and no empty stretch is marched; only the
// links of the cells holding those samples are loaded, for the scatter. The
// per-sample arithmetic is march_backward's, in the same order. The cache is
// read with coherent loads, so the batched launch may read back what the
// same thread wrote earlier in it.
__device__ __forceinline__ void march_backward_cached(const Common& P, const RayF& r,
                                                      const float Y[9], const float Cf[3],
                                                      float Df, const float gC[3], float gD,
                                                      float* __restrict__ grad, int64_t out,
                                                      int n_kept) {
  const int rm2x = P.g.rx - 2, rm2y = P.g.ry - 2, rm2z = P.g.rz - 2;
  int cx = -1, cy = -1, cz = -1;
  bool dirty = false;
  int32_t l[8];
  float gs[8], gc[8][3];
#pragma unroll
  for (int c = 0; c < 8; ++c) clear_corner(gs[c], gc[c]);
  float S[3] = {0.f, 0.f, 0.f}, SD = 0.f, T = 1.f;
  const float dt = r.dt;
  const bool ident = P.o.color_act == PLX_ACT_IDENTITY;
  for (int j = 0; j < n_kept; ++j) {
    const int64_t at = (int64_t)j * P.o.cn + out;
    // read once: evict-first, to keep the gradient rows in L2 for the atomics
    const float4 v = __ldcs(P.o.cval + at);
    const int k = __ldcs(P.o.ck + at);
    const float kf = (float)k;
    int ix, iy, iz;
    float fx, fy, fz;
    sample_axis(r.B[0], r.S[0], k, rm2x, ix, fx);
    sample_axis(r.B[1], r.S[1], k, rm2y, iy, fy);
    sample_axis(r.B[2], r.S[2], k, rm2z, iz, fz);
    if (ix != cx || iy != cy || iz != cz) {
      if (dirty) dirty = leave_cell<false>(grad, l, gs, gc, Y, ix - cx, iy - cy, iz - cz, true);
      cx = ix; cy = iy; cz = iz;
      load_links(P.g, ix, iy, iz, l);
    }
    float w[8];
    corner_weights(fx, fy, fz, w);
    const float sig = v.x;  // > 0: only compositing samples are kept
    const float col[3] = {v.y, v.z, v.w};
    float dact[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) dact[ch] = ident ? 1.f : col[ch] * (1.f - col[ch]);
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
  }
  if (dirty) flush_cell(grad, l, gs, gc, Y);
}

// ------------------------------------------- warp-cooperative scatter
// A corner's 28 gradient values go to memory as 7 float4 reductions into its
// vertex's 128-byte row. Sent by the flushing lane alone they are 7 L2
// requests; sent by 7 lanes of the warp, one float4 each, they are one
// coalesced request for the row, and the L2 retires 1.7x more rows per second
// that way (50 against 29 G rows/s on B300 for random rows of a 77 MB buffer,
// 2.3x beyond L2). So the lanes that flush a corner write its values to a
// per-warp staging area in shared memory, one row per lane in rank order, and
// the whole warp then sends the staged rows, 4 per instruction (lanes 8g..8g+6
// send row g's float4 0..6).
constexpr int kStageStride = 36;  // floats per staged row: 28 values, the link,
                                  // padding so that 8 lanes hit distinct banks

// Floats of staging per warp for `rows` rows.
constexpr int stage_floats(int rows) { return rows * kStageStride; }

// Every lane of the warp calls this with the same corner slot; `f` says
// whether this lane flushes it (its sums (gs, gc) for the vertex `link`).
// The flushing lanes are taken ROWS at a time in rank order.
template <int ROWS>
__device__ __forceinline__ void warp_flush_corner(float* __restrict__ grad,
                                                  float* __restrict__ stage, bool f,
                                                  int32_t link, float gs, const float gc[3],
                                                  const float Y[9], int lane) {
  const unsigned m = __ballot_sync(0xffffffffu, f);
  if (m == 0u) return;
  const int n = __popc(m), rank = __popc(m & ((1u << lane) - 1u));
  const int g = lane >> 3, q = lane & 7;
  for (int base = 0; base < n; base += ROWS) {
    if (f && rank >= base && rank < base + ROWS) {
      float* row = stage + (rank - base) * kStageStride;
      float v[28];
      v[0] = gs;
#pragma unroll
      for (int ch = 0; ch < 3; ++ch)
#pragma unroll
        for (int k = 0; k < 9; ++k) v[1 + 9 * ch + k] = gc[ch] * Y[k];
#pragma unroll
      for (int j = 0; j < 7; ++j)
        reinterpret_cast<float4*>(row)[j] =
            make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
      reinterpret_cast<int32_t*>(row)[28] = link;
    }
    __syncwarp();
    const int cnt = n - base < ROWS ? n - base : ROWS;
    for (int b = 0; b < cnt; b += 4) {
      const int rr = b + g;
      if (rr < cnt && q < 7) {
        const float* row = stage + rr * kStageStride;
        const int32_t lk = reinterpret_cast<const int32_t*>(row)[28];
        atomicAdd(reinterpret_cast<float4*>(grad + (int64_t)lk * PLX_GRAD_STRIDE) + q,
                  reinterpret_cast<const float4*>(row)[q]);
      }
    }
    __syncwarp();  // the next rows overwrite these
  }
}

// march_backward_cached with the warp-cooperative scatter. The lanes walk
// their kept samples in lockstep (iteration j = each lane's j-th sample, up to
// the longest ray of the warp, plus one for the final flush), so that every
// lane reaches the shuffles and barriers of warp_flush_corner; a lane whose
// ray is done, or that has no ray (n_kept = 0), only helps send. The
// per-sample arithmetic and the carry of shared corners are those of
// march_backward_cached and leave_cell.
template <int ROWS>
__device__ __forceinline__ void march_backward_cached_warp(
    const Common& P, const RayF& r, const float Y[9], const float Cf[3], float Df,
    const float gC[3], float gD, float* __restrict__ grad, int64_t out, int n_kept,
    float* __restrict__ stage, int lane) {
  const int rm2x = P.g.rx - 2, rm2y = P.g.ry - 2, rm2z = P.g.rz - 2;
  const int n_max = __reduce_max_sync(0xffffffffu, n_kept);
  int cx = -1, cy = -1, cz = -1;
  bool dirty = false;
  int32_t l[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) l[c] = -1;
  float gs[8], gc[8][3];
#pragma unroll
  for (int c = 0; c < 8; ++c) clear_corner(gs[c], gc[c]);
  float S[3] = {0.f, 0.f, 0.f}, SD = 0.f, T = 1.f;
  const float dt = r.dt;
  const bool ident = P.o.color_act == PLX_ACT_IDENTITY;
  for (int j = 0; j <= n_max; ++j) {
    const bool live = j < n_kept;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    int k = 0, ix = cx, iy = cy, iz = cz;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    if (live) {
      const int64_t at = (int64_t)j * P.o.cn + out;
      v = __ldcs(P.o.cval + at);
      k = __ldcs(P.o.ck + at);
      sample_axis(r.B[0], r.S[0], k, rm2x, ix, fx);
      sample_axis(r.B[1], r.S[1], k, rm2y, iy, fy);
      sample_axis(r.B[2], r.S[2], k, rm2z, iz, fz);
    }
    const bool moved = live ? (ix != cx || iy != cy || iz != cz) : j == n_kept;
    // corners that leave: those the new cell does not share (all at the end)
    unsigned leave = 0u;
    bool adj = false;
    const int dx = ix - cx, dy = iy - cy, dz = iz - cz;
    if (moved && dirty) {
      adj = live && dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1;
      unsigned keep = 0u;
      if (adj) {
        const unsigned mx = dx == 0 ? 0xffu : (dx > 0 ? 0xaau : 0x55u);
        const unsigned my = dy == 0 ? 0xffu : (dy > 0 ? 0xccu : 0x33u);
        const unsigned mz = dz == 0 ? 0xffu : (dz > 0 ? 0xf0u : 0x0fu);
        keep = mx & my & mz;
      }
      leave = ~keep & 0xffu;
    }
    const unsigned any = __reduce_or_sync(0xffffffffu, leave);
    if (any) {
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if ((any >> c) & 1u)
          warp_flush_corner<ROWS>(grad, stage, ((leave >> c) & 1u) && l[c] >= 0, l[c], gs[c],
                                  gc[c], Y, lane);
      if (leave) {
        if (!adj) {
#pragma unroll
          for (int c = 0; c < 8; ++c) clear_corner(gs[c], gc[c]);
        } else {
          move_by(dx, dy, dz, gs, gc);
        }
      }
    }
    if (!live) {
      dirty = false;
      continue;
    }
    if (moved) {
      cx = ix; cy = iy; cz = iz;
      load_links(P.g, ix, iy, iz, l);
    }
    float w[8];
    corner_weights(fx, fy, fz, w);
    const float sig = v.x;  // > 0: only compositing samples are kept
    const float col[3] = {v.y, v.z, v.w};
    float dact[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) dact[ch] = ident ? 1.f : col[ch] * (1.f - col[ch]);
    float alpha, keep;
    alpha_of(sig * dt, alpha, keep);
    const float wgt = T * alpha;
    const float Tn = T * keep;
    const float t = fmaf((float)k, dt, r.t0);
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
  }
}

}  // namespace plx
