/*
 * FP64 CPU oracle for the Plenoxel RGB-D renderer, its grid adjoint and its
 * pose Jacobian ("RGB-D Mapping and Tracking in a Plenoxel Radiance Field",
 * arXiv 2307.03404).
 *
 * TEST INFRASTRUCTURE. This file is the slow, plain, double-precision
 * statement of what the GPU path computes. Only the test-suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it. It shares no code,
 * header, table or constant with the CUDA library: every formula here is
 * written out again from the paper.
 *
 * Readings of the paper that the oracle fixes (the paper is silent or garbled
 * on these points):
 *   - pixel centre at (u+1/2, v+1/2); ray direction d = R d_c / |d_c| is unit
 *     length and t is Euclidean distance from the camera centre (Sec. 4);
 *   - sample k of a ray sits at t_k = t_min + (k+1/2) * step, every delta_k is
 *     the step, and the sample count is floor((t_max - t_min)/step) capped by
 *     max_samples, where [t_min, t_max] is the ray's overlap with the grid box
 *     (t_min no smaller than the near distance);
 *   - density activation sigma = max(0, f_sigma); colour activation sigmoid of
 *     the SH sum (or identity, for closed-form tests);
 *   - real SH of degree 2 with orthonormal constants, order
 *     (1; y, z, x; xy, yz, 3z^2-1, xz, x^2-y^2), no Condon-Shortley phase;
 *   - the rendered colour includes the background term T_{N+1} * bg; Eq. 9's
 *     prefix sum includes sample i (sum over j = 1..i);
 *   - a ray whose sensor depth is not positive or not finite is left out of
 *     both losses and of the count M; the sensor depth is a z-depth that is
 *     turned into a ray distance by multiplying with |d_c|;
 *   - the loss gradient of Eq. 7 is d L_g / d D (the paper prints L_p);
 *   - the pose is camera-to-world, perturbed on the left in the world frame,
 *     T <- exp(xi^) T with xi = (rho, phi), translation first;
 *   - the dynamic grid grows by allocating every vertex within a band (in
 *     grid units, per axis) of each back-projected depth point, new vertices
 *     numbered after the existing ones in link order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int32_t res[3];          /* vertices per axis (x, y, z) */
  double lo[3], hi[3];     /* axis-aligned box spanned by the vertices */
  const int32_t *links;    /* [res_z][res_y][res_x], -1 = vertex not allocated */
  const double *density;   /* [n_alloc] */
  const double *sh;        /* [n_alloc][3][9]: channel-major, basis index fastest */
  int64_t n_alloc;
} orc_grid;

typedef struct {
  double fx, fy, cx, cy;
  int32_t width, height;
  double T_wc[12];         /* camera-to-world, row-major 3x4 [R | o] */
} orc_camera;

typedef struct {
  double step;             /* sample spacing delta, world units */
  double near_t;           /* smallest t marched */
  double stop_T;           /* stop once T_{i+1} < stop_T (0 = never) */
  double bg[3];            /* background colour */
  double lambda_d;         /* weight of the geometric loss, Eq. 11 */
  int32_t max_samples;
  int32_t color_act;       /* 0 = sigmoid, 1 = identity */
  int32_t depth_is_z;      /* 1 = depth targets are sensor z-depths */
  int32_t dir_term;        /* 1 = tracking Jacobian includes dc/dd (variant) */
} orc_opts;

static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n > 0 ? n : 1; }
int orc_get_threads(void) { return g_threads; }

/* ---------------------------------------------------------------- SH basis */
/* Real spherical harmonics of degree 0..2 evaluated on a unit direction
 * (Sec. 5.2: nine coefficients per colour channel). */
void orc_sh_basis(const double dir[3], double Y[9]) {
  const double pi = 3.14159265358979323846;
  const double x = dir[0], y = dir[1], z = dir[2];
  const double k0 = sqrt(1.0 / (4.0 * pi));
  const double k1 = sqrt(3.0 / (4.0 * pi));
  const double k2 = sqrt(15.0 / (4.0 * pi));
  const double k20 = sqrt(5.0 / (16.0 * pi));
  const double k22 = sqrt(15.0 / (16.0 * pi));
  Y[0] = k0;
  Y[1] = k1 * y;
  Y[2] = k1 * z;
  Y[3] = k1 * x;
  Y[4] = k2 * x * y;
  Y[5] = k2 * y * z;
  Y[6] = k20 * (3.0 * z * z - 1.0);
  Y[7] = k2 * x * z;
  Y[8] = k22 * (x * x - y * y);
}

/* Gradient of the same nine polynomials in (x, y, z), dY[k][a] = dY_k/dx_a
 * (the view-direction term of the tracking Jacobian variant; only its
 * component tangent to the sphere matters, and the rotation of a direction
 * is tangent). */
void orc_sh_basis_grad(const double dir[3], double dY[9][3]) {
  const double pi = 3.14159265358979323846;
  const double x = dir[0], y = dir[1], z = dir[2];
  const double k1 = sqrt(3.0 / (4.0 * pi));
  const double k2 = sqrt(15.0 / (4.0 * pi));
  const double k20 = sqrt(5.0 / (16.0 * pi));
  const double k22 = sqrt(15.0 / (16.0 * pi));
  for (int k = 0; k < 9; ++k) dY[k][0] = dY[k][1] = dY[k][2] = 0.0;
  dY[1][1] = k1;
  dY[2][2] = k1;
  dY[3][0] = k1;
  dY[4][0] = k2 * y;  dY[4][1] = k2 * x;
  dY[5][1] = k2 * z;  dY[5][2] = k2 * y;
  dY[6][2] = k20 * 6.0 * z;
  dY[7][0] = k2 * z;  dY[7][2] = k2 * x;
  dY[8][0] = k22 * 2.0 * x;  dY[8][1] = -k22 * 2.0 * y;
}

/* ----------------------------------------------------- trilinear, App. A */
/* Appendix A (Eq. 15-16): inside one voxel with its lower lattice point moved
 * to the origin and unit spacing, the interpolant is the polynomial
 *   f = a0 + a1 x + a2 y + a3 z + a4 xy + a5 xz + a6 yz + a7 xyz
 * whose coefficients solve the 8x8 system that makes f equal the corner
 * values. With x0=y0=z0=0 and x1=y1=z1=1 the system is triangular and its
 * solution is the inclusion-exclusion below. V is indexed by
 * c = dx + 2 dy + 4 dz (dx, dy, dz in {0,1}). */
static void appA_coeffs(const double V[8], double a[8]) {
  a[0] = V[0];
  a[1] = V[1] - V[0];
  a[2] = V[2] - V[0];
  a[3] = V[4] - V[0];
  a[4] = V[3] - V[1] - V[2] + V[0];
  a[5] = V[5] - V[1] - V[4] + V[0];
  a[6] = V[6] - V[2] - V[4] + V[0];
  a[7] = V[7] - V[3] - V[5] - V[6] + V[1] + V[2] + V[4] - V[0];
}

/* f(x,y,z) and its local gradient (Eq. 16) */
void orc_trilerp(const double V[8], double x, double y, double z, double *f,
                 double grad[3]) {
  double a[8];
  appA_coeffs(V, a);
  *f = a[0] + a[1] * x + a[2] * y + a[3] * z + a[4] * x * y + a[5] * x * z +
       a[6] * y * z + a[7] * x * y * z;
  if (grad) {
    grad[0] = a[1] + a[4] * y + a[5] * z + a[7] * y * z;
    grad[1] = a[2] + a[4] * x + a[6] * z + a[7] * x * z;
    grad[2] = a[3] + a[5] * x + a[6] * y + a[7] * x * y;
  }
}

/* ---------------------------------------------------------------- geometry */
static double grid_h(const orc_grid *g, int a) {
  return (g->hi[a] - g->lo[a]) / (double)(g->res[a] - 1);
}

/* Sec. 4: r = o + t d, o the camera centre, d towards the pixel. */
static void pixel_ray(const orc_camera *cam, int32_t pix, double o[3],
                      double d[3], double *dc_norm) {
  const int u = pix % cam->width, v = pix / cam->width;
  const double dc[3] = {(u + 0.5 - cam->cx) / cam->fx,
                        (v + 0.5 - cam->cy) / cam->fy, 1.0};
  const double n = sqrt(dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2]);
  const double *T = cam->T_wc;
  for (int a = 0; a < 3; ++a) {
    d[a] = (T[4 * a + 0] * dc[0] + T[4 * a + 1] * dc[1] + T[4 * a + 2] * dc[2]) / n;
    o[a] = T[4 * a + 3];
  }
  *dc_norm = n;
}

/* exported for tests: the ray of one pixel and its overlap with the grid box */
static int clip_ray(const orc_grid *g, const double o[3], const double d[3],
                    double near_t, double *t_min, double *t_max);
int orc_pixel_ray(const orc_grid *g, const orc_camera *cam, int32_t pix,
                  double near_t, double o[3], double d[3], double *dc_norm,
                  double t_range[2]) {
  pixel_ray(cam, pix, o, d, dc_norm);
  return clip_ray(g, o, d, near_t, &t_range[0], &t_range[1]);
}

/* Overlap of the ray with the grid box, from the three slabs. */
static int clip_ray(const orc_grid *g, const double o[3], const double d[3],
                    double near_t, double *t_min, double *t_max) {
  double tn = -INFINITY, tf = INFINITY;
  for (int a = 0; a < 3; ++a) {
    if (d[a] != 0.0) {
      double ta = (g->lo[a] - o[a]) / d[a];
      double tb = (g->hi[a] - o[a]) / d[a];
      if (ta > tb) { double s = ta; ta = tb; tb = s; }
      if (ta > tn) tn = ta;
      if (tb < tf) tf = tb;
    } else if (o[a] < g->lo[a] || o[a] > g->hi[a]) {
      return 0;
    }
  }
  if (near_t > tn) tn = near_t;
  *t_min = tn;
  *t_max = tf;
  return tf > tn;
}

static int64_t sample_count(const orc_opts *op, double t_min, double t_max) {
  double n = floor((t_max - t_min) / op->step);
  if (n < 0) n = 0;
  if (n > op->max_samples) n = op->max_samples;
  return (int64_t)n;
}

/* ---------------------------------------------------------- one sample */
typedef struct {
  int any_alloc;
  int32_t link[8];
  double wc[8];          /* d f / d V_c for each corner (trilinear weight) */
  double f_sigma;        /* interpolated raw density */
  double sigma;          /* max(0, f_sigma) */
  double chat[3];        /* sum_k Y_k f_{ch,k} */
  double c[3];           /* activated colour */
  double dc_dchat[3];    /* activation derivative */
  double gsig[3];        /* d f_sigma / d p (world) */
  double gchat[3][3];    /* d chat_ch / d p (world), [ch][axis] */
  double f_sh[3][9];     /* interpolated SH coefficients at p */
} orc_sample;

static void eval_sample(const orc_grid *g, const double p[3], const double Y[9],
                        int color_act, orc_sample *s) {
  double xl[3], h[3];
  int cell[3];
  for (int a = 0; a < 3; ++a) {
    h[a] = grid_h(g, a);
    const double xg = (p[a] - g->lo[a]) / h[a];
    int ci = (int)floor(xg);
    if (ci < 0) ci = 0;
    if (ci > g->res[a] - 2) ci = g->res[a] - 2;
    cell[a] = ci;
    xl[a] = xg - ci;
  }
  s->any_alloc = 0;
  for (int c = 0; c < 8; ++c) {
    const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
    const int64_t idx =
        ((int64_t)(cell[2] + dz) * g->res[1] + (cell[1] + dy)) * g->res[0] +
        (cell[0] + dx);
    s->link[c] = g->links[idx];
    if (s->link[c] >= 0) s->any_alloc = 1;
  }
  /* corner weight = value of the interpolant when corner c holds 1, others 0 */
  for (int c = 0; c < 8; ++c) {
    double e[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    e[c] = 1.0;
    orc_trilerp(e, xl[0], xl[1], xl[2], &s->wc[c], NULL);
  }
  double V[8], gl[3];
  for (int c = 0; c < 8; ++c) V[c] = s->link[c] >= 0 ? g->density[s->link[c]] : 0.0;
  orc_trilerp(V, xl[0], xl[1], xl[2], &s->f_sigma, gl);
  for (int a = 0; a < 3; ++a) s->gsig[a] = gl[a] / h[a];
  s->sigma = s->f_sigma > 0.0 ? s->f_sigma : 0.0;
  for (int ch = 0; ch < 3; ++ch) {
    s->chat[ch] = 0.0;
    for (int a = 0; a < 3; ++a) s->gchat[ch][a] = 0.0;
    for (int k = 0; k < 9; ++k) {
      double f;
      for (int c = 0; c < 8; ++c)
        V[c] = s->link[c] >= 0 ? g->sh[(int64_t)s->link[c] * 27 + ch * 9 + k] : 0.0;
      orc_trilerp(V, xl[0], xl[1], xl[2], &f, gl);
      s->f_sh[ch][k] = f;
      s->chat[ch] += Y[k] * f;
      for (int a = 0; a < 3; ++a) s->gchat[ch][a] += Y[k] * gl[a] / h[a];
    }
    if (color_act == 1) {
      s->c[ch] = s->chat[ch];
      s->dc_dchat[ch] = 1.0;
    } else {
      s->c[ch] = 1.0 / (1.0 + exp(-s->chat[ch]));
      s->dc_dchat[ch] = s->c[ch] * (1.0 - s->c[ch]);
    }
  }
}

/* ----------------------------------------------------- forward, Eq. 1-3 */
typedef struct {
  double o[3], d[3], dc_norm, Y[9];
  double t_min;
  int64_t n;             /* samples marched */
} orc_ray;

static void setup_ray(const orc_grid *g, const orc_camera *cam, int32_t pix,
                      const orc_opts *op, orc_ray *r) {
  double t_max;
  pixel_ray(cam, pix, r->o, r->d, &r->dc_norm);
  orc_sh_basis(r->d, r->Y);
  r->n = 0;
  r->t_min = 0.0;
  if (clip_ray(g, r->o, r->d, op->near_t, &r->t_min, &t_max))
    r->n = sample_count(op, r->t_min, t_max);
}

typedef struct {
  double C[3], D, T_final;
  int64_t n_marched, n_alloc;
} orc_fwd;

/* Colour (Eq. 1) with transmittance (Eq. 2) and expected depth (Eq. 3) of the
 * samples o + t_k d; the sample positions may be taken from another pose
 * (o_s, d_s) than the one that fixed t_k, and the SH basis Y_s from another
 * direction (the frozen-sample form used to difference the pose Jacobian). */
static void forward_ray(const orc_grid *g, const orc_ray *r, const double *o_s,
                        const double *d_s, const double *Y_s, const orc_opts *op,
                        orc_fwd *out) {
  double tau = 0.0; /* sum_{j<i} sigma_j delta_j */
  for (int ch = 0; ch < 3; ++ch) out->C[ch] = 0.0;
  out->D = 0.0;
  out->n_marched = 0;
  out->n_alloc = 0;
  for (int64_t k = 0; k < r->n; ++k) {
    const double t = r->t_min + (k + 0.5) * op->step;
    double p[3];
    orc_sample s;
    for (int a = 0; a < 3; ++a) p[a] = o_s[a] + t * d_s[a];
    eval_sample(g, p, Y_s, op->color_act, &s);
    out->n_marched++;
    out->n_alloc += s.any_alloc;
    const double T_i = exp(-tau);
    const double w = T_i * (1.0 - exp(-s.sigma * op->step));
    for (int ch = 0; ch < 3; ++ch) out->C[ch] += w * s.c[ch];
    out->D += w * t;
    tau += s.sigma * op->step;
    if (op->stop_T > 0.0 && exp(-tau) < op->stop_T) break;
  }
  out->T_final = exp(-tau);
  for (int ch = 0; ch < 3; ++ch) out->C[ch] += out->T_final * op->bg[ch];
}

static int depth_valid(double dz) { return isfinite(dz) && dz > 0.0; }

void orc_render(const orc_grid *g, const orc_camera *cams, int64_t n_rays,
                const int32_t *cam_id, const int32_t *pix, const orc_opts *op,
                double *rgb, double *depth, double *T_final, int64_t *n_marched,
                int64_t *n_alloc) {
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads)
  for (int64_t i = 0; i < n_rays; ++i) {
    orc_ray r;
    orc_fwd f;
    const orc_camera *cam = &cams[cam_id[i]];
    setup_ray(g, cam, pix[i], op, &r);
    forward_ray(g, &r, r.o, r.d, r.Y, op, &f);
    for (int ch = 0; ch < 3; ++ch) rgb[3 * i + ch] = f.C[ch];
    depth[i] = f.D;
    if (T_final) T_final[i] = f.T_final;
    if (n_marched) n_marched[i] = f.n_marched;
    if (n_alloc) n_alloc[i] = f.n_alloc;
  }
}

/* Frozen-sample forward: t_k, delta_k (and, unless op->dir_term, the SH
 * direction) come from the camera's own pose; the positions (and with
 * op->dir_term the SH direction) come from exp(xi^) T_wc. */
void orc_se3_exp(const double xi[6], double T[12]);

void orc_render_frozen(const orc_grid *g, const orc_camera *cams, int64_t n_rays,
                       const int32_t *cam_id, const int32_t *pix,
                       const orc_opts *op, const double xi[6], double *rgb,
                       double *depth) {
  double E[12];
  orc_se3_exp(xi, E);
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads)
  for (int64_t i = 0; i < n_rays; ++i) {
    orc_ray r;
    orc_fwd f;
    double o2[3], d2[3];
    setup_ray(g, &cams[cam_id[i]], pix[i], op, &r);
    for (int a = 0; a < 3; ++a) {
      o2[a] = E[4 * a + 0] * r.o[0] + E[4 * a + 1] * r.o[1] + E[4 * a + 2] * r.o[2] + E[4 * a + 3];
      d2[a] = E[4 * a + 0] * r.d[0] + E[4 * a + 1] * r.d[1] + E[4 * a + 2] * r.d[2];
    }
    double Y2[9];
    orc_sh_basis(d2, Y2);
    forward_ray(g, &r, o2, d2, op->dir_term ? Y2 : r.Y, op, &f);
    for (int ch = 0; ch < 3; ++ch) rgb[3 * i + ch] = f.C[ch];
    depth[i] = f.D;
  }
}

/* ---------------------------------------------------- losses, Eq. 4, 5, 11 */
static double target_ray_depth(const orc_opts *op, double dz, double dc_norm) {
  return op->depth_is_z ? dz * dc_norm : dz;
}

static int64_t count_valid(int64_t n_rays, const double *depth_t) {
  int64_t m = 0;
  for (int64_t i = 0; i < n_rays; ++i) m += depth_valid(depth_t[i]);
  return m;
}

/* ------------------------------------------- grid adjoint, Eq. 6-10 */
/* For every valid ray: a first pass gives C and D (Eq. 1, 3); a second pass
 * walks the same samples, recomputes T_i, T_{i+1}, w_i and the inclusive
 * prefix sums, applies Eq. 8, 9, 10, chains through the activations, the SH
 * basis and the trilinear weights, and adds into the corners' gradients.
 * Returns the loss L = L_p + lambda_d L_g and writes M. */
double orc_grad_grid(const orc_grid *g, const orc_camera *cams, int64_t n_rays,
                     const int32_t *cam_id, const int32_t *pix,
                     const orc_opts *op, const double *rgb_t,
                     const double *depth_t, double *grad_density,
                     double *grad_sh, int64_t *M_out) {
  const int64_t M = count_valid(n_rays, depth_t);
  if (M_out) *M_out = M;
  if (M == 0) return 0.0;
  double loss = 0.0;
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads) reduction(+ : loss)
  for (int64_t i = 0; i < n_rays; ++i) {
    if (!depth_valid(depth_t[i])) continue;
    orc_ray r;
    orc_fwd f;
    setup_ray(g, &cams[cam_id[i]], pix[i], op, &r);
    forward_ray(g, &r, r.o, r.d, r.Y, op, &f);
    const double Dt = target_ray_depth(op, depth_t[i], r.dc_norm);
    double dL_dC[3], e2 = 0.0;
    for (int ch = 0; ch < 3; ++ch) {
      const double e = f.C[ch] - rgb_t[3 * i + ch];
      e2 += e * e;
      dL_dC[ch] = 2.0 * e / (double)M;            /* d L_p / d C, Eq. 4 */
    }
    const double eD = f.D - Dt;
    const double dL_dD = 2.0 * op->lambda_d * eD / (double)M; /* Eq. 5, 11 */
    loss += (e2 + op->lambda_d * eD * eD) / (double)M;

    double tau = 0.0, S[3] = {0, 0, 0}, SD = 0.0;
    for (int64_t k = 0; k < r.n; ++k) {
      const double t = r.t_min + (k + 0.5) * op->step;
      const double delta = op->step;
      double p[3];
      orc_sample s;
      for (int a = 0; a < 3; ++a) p[a] = r.o[a] + t * r.d[a];
      eval_sample(g, p, r.Y, op->color_act, &s);
      const double T_i = exp(-tau);
      const double T_next = exp(-(tau + s.sigma * delta));
      const double w = T_i * (1.0 - exp(-s.sigma * delta)); /* Eq. 8 */
      for (int ch = 0; ch < 3; ++ch) S[ch] += w * s.c[ch];  /* sum_{j<=i} c_j w_j */
      SD += w * t;                                          /* sum_{j<=i} t_j w_j */
      double dL_dsigma = 0.0;
      for (int ch = 0; ch < 3; ++ch)                        /* Eq. 9 */
        dL_dsigma += dL_dC[ch] * delta * (s.c[ch] * T_next - f.C[ch] + S[ch]);
      dL_dsigma += dL_dD * delta * (t * T_next - f.D + SD); /* Eq. 10 */
      const double dL_dfsig = s.f_sigma > 0.0 ? dL_dsigma : 0.0;
      double dL_dchat[3];
      for (int ch = 0; ch < 3; ++ch) dL_dchat[ch] = dL_dC[ch] * w * s.dc_dchat[ch];
      for (int c = 0; c < 8; ++c) {
        const int32_t l = s.link[c];
        if (l < 0) continue;
#pragma omp atomic
        grad_density[l] += s.wc[c] * dL_dfsig;
        for (int ch = 0; ch < 3; ++ch)
          for (int kk = 0; kk < 9; ++kk) {
#pragma omp atomic
            grad_sh[(int64_t)l * 27 + ch * 9 + kk] += s.wc[c] * dL_dchat[ch] * r.Y[kk];
          }
      }
      tau += s.sigma * delta;
      if (op->stop_T > 0.0 && exp(-tau) < op->stop_T) break;
    }
  }
  return loss;
}

/* --------------------------------------------- pose Jacobian, Eq. 12-16 */
/* Per valid ray: the 4x6 Jacobian of the residual (C - C_target, D - D_target)
 * with respect to xi, from Eq. 12-13 with dp/dr = [I, t_i I] (Eq. 14) and the
 * trilinear spatial derivatives of Appendix A; t_i, delta_i, the clip and the
 * SH direction are held fixed, as in the paper (with op->dir_term, the variant,
 * the colour rows also get sum_i w_i dc_i/dchat sum_k f_k dY_k/dd through d).
 * Then
 *   H = sum J^T W J, b = sum J^T W r, loss = sum r^T W r
 * with W = diag(1,1,1,lambda_d)/M. J [n][4][6] and r [n][4] may be NULL;
 * invalid rays get zero rows. */
double orc_pose_jacobian(const orc_grid *g, const orc_camera *cams,
                         int64_t n_rays, const int32_t *cam_id,
                         const int32_t *pix, const orc_opts *op,
                         const double *rgb_t, const double *depth_t, double *J,
                         double *resid, double H[36], double b[6],
                         int64_t *M_out) {
  const int64_t M = count_valid(n_rays, depth_t);
  if (M_out) *M_out = M;
  double *Jall = (double *)calloc((size_t)n_rays * 24, sizeof(double));
  double *rall = (double *)calloc((size_t)n_rays * 4, sizeof(double));
  char *valid = (char *)calloc((size_t)n_rays, 1);
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads)
  for (int64_t i = 0; i < n_rays; ++i) {
    if (!depth_valid(depth_t[i])) continue;
    valid[i] = 1;
    orc_ray r;
    orc_fwd f;
    setup_ray(g, &cams[cam_id[i]], pix[i], op, &r);
    forward_ray(g, &r, r.o, r.d, r.Y, op, &f);
    const double Dt = target_ray_depth(op, depth_t[i], r.dc_norm);
    double *ri = rall + 4 * i;
    for (int ch = 0; ch < 3; ++ch) ri[ch] = f.C[ch] - rgb_t[3 * i + ch];
    ri[3] = f.D - Dt;
    /* dX/do and dX/dd for X in (R, G, B, D): Eq. 12, 13 with Eq. 14 */
    double dX_do[4][3] = {{0}}, dX_dd[4][3] = {{0}};
    double tau = 0.0, S[3] = {0, 0, 0}, SD = 0.0;
    double dY[9][3];
    orc_sh_basis_grad(r.d, dY);
    for (int64_t k = 0; k < r.n; ++k) {
      const double t = r.t_min + (k + 0.5) * op->step;
      const double delta = op->step;
      double p[3];
      orc_sample s;
      for (int a = 0; a < 3; ++a) p[a] = r.o[a] + t * r.d[a];
      eval_sample(g, p, r.Y, op->color_act, &s);
      const double T_i = exp(-tau);
      const double T_next = exp(-(tau + s.sigma * delta));
      const double w = T_i * (1.0 - exp(-s.sigma * delta));
      for (int ch = 0; ch < 3; ++ch) S[ch] += w * s.c[ch];
      SD += w * t;
      double dsig_dp[3];
      for (int a = 0; a < 3; ++a) dsig_dp[a] = s.f_sigma > 0.0 ? s.gsig[a] : 0.0;
      double dX_dp[4][3];
      for (int ch = 0; ch < 3; ++ch) {
        const double dC_dsig = delta * (s.c[ch] * T_next - f.C[ch] + S[ch]); /* Eq. 9 */
        for (int a = 0; a < 3; ++a)
          dX_dp[ch][a] = dC_dsig * dsig_dp[a] + w * s.dc_dchat[ch] * s.gchat[ch][a];
      }
      const double dD_dsig = delta * (t * T_next - f.D + SD); /* Eq. 10 */
      for (int a = 0; a < 3; ++a) dX_dp[3][a] = dD_dsig * dsig_dp[a];
      if (op->dir_term) /* variant: c_i also depends on d through Y(d) */
        for (int ch = 0; ch < 3; ++ch)
          for (int a = 0; a < 3; ++a) {
            double gy = 0.0;
            for (int k = 0; k < 9; ++k) gy += s.f_sh[ch][k] * dY[k][a];
            dX_dd[ch][a] += w * s.dc_dchat[ch] * gy;
          }
      for (int x = 0; x < 4; ++x)
        for (int a = 0; a < 3; ++a) {
          dX_do[x][a] += dX_dp[x][a];      /* dp/do = I   */
          dX_dd[x][a] += dX_dp[x][a] * t;  /* dp/dd = t I */
        }
      tau += s.sigma * delta;
      if (op->stop_T > 0.0 && exp(-tau) < op->stop_T) break;
    }
    /* do/dxi = [I, -[o]x], dd/dxi = [0, -[d]x] */
    double Do[3][6], Dd[3][6];
    const double *o = r.o, *d = r.d;
    const double ox[3][3] = {{0, -o[2], o[1]}, {o[2], 0, -o[0]}, {-o[1], o[0], 0}};
    const double dx[3][3] = {{0, -d[2], d[1]}, {d[2], 0, -d[0]}, {-d[1], d[0], 0}};
    for (int a = 0; a < 3; ++a)
      for (int j = 0; j < 3; ++j) {
        Do[a][j] = a == j ? 1.0 : 0.0;
        Do[a][3 + j] = -ox[a][j];
        Dd[a][j] = 0.0;
        Dd[a][3 + j] = -dx[a][j];
      }
    double *Ji = Jall + 24 * i;
    for (int x = 0; x < 4; ++x)
      for (int j = 0; j < 6; ++j) {
        double v = 0.0;
        for (int a = 0; a < 3; ++a) v += dX_do[x][a] * Do[a][j] + dX_dd[x][a] * Dd[a][j];
        Ji[6 * x + j] = v;
      }
  }
  /* reduction in ray order */
  double loss = 0.0;
  for (int j = 0; j < 36; ++j) H[j] = 0.0;
  for (int j = 0; j < 6; ++j) b[j] = 0.0;
  if (M > 0) {
    const double Wd[4] = {1.0 / M, 1.0 / M, 1.0 / M, op->lambda_d / M};
    for (int64_t i = 0; i < n_rays; ++i) {
      if (!valid[i]) continue;
      const double *Ji = Jall + 24 * i, *ri = rall + 4 * i;
      for (int x = 0; x < 4; ++x) {
        loss += Wd[x] * ri[x] * ri[x];
        for (int j = 0; j < 6; ++j) {
          b[j] += Ji[6 * x + j] * Wd[x] * ri[x];
          for (int l = 0; l < 6; ++l) H[6 * j + l] += Ji[6 * x + j] * Wd[x] * Ji[6 * x + l];
        }
      }
    }
  }
  if (J) memcpy(J, Jall, (size_t)n_rays * 24 * sizeof(double));
  if (resid) memcpy(resid, rall, (size_t)n_rays * 4 * sizeof(double));
  free(Jall);
  free(rall);
  free(valid);
  return loss;
}

/* ------------------------------------------------------ SE(3), pose step */
/* exp of the twist xi = (rho, phi): R by Rodrigues' formula, translation V rho,
 * returned as a row-major 3x4 [R | t]. */
void orc_se3_exp(const double xi[6], double T[12]) {
  const double *rho = xi, *phi = xi + 3;
  const double th2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
  const double th = sqrt(th2);
  double A, B, Cc;
  if (th < 1e-6) {
    A = 1.0 - th2 / 6.0;
    B = 0.5 - th2 / 24.0;
    Cc = 1.0 / 6.0 - th2 / 120.0;
  } else {
    A = sin(th) / th;
    B = (1.0 - cos(th)) / th2;
    Cc = (th - sin(th)) / (th2 * th);
  }
  const double K[3][3] = {{0, -phi[2], phi[1]}, {phi[2], 0, -phi[0]}, {-phi[1], phi[0], 0}};
  double K2[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      K2[i][j] = 0.0;
      for (int l = 0; l < 3; ++l) K2[i][j] += K[i][l] * K[l][j];
    }
  for (int i = 0; i < 3; ++i) {
    double t = 0.0;
    for (int j = 0; j < 3; ++j) {
      const double I = i == j ? 1.0 : 0.0;
      T[4 * i + j] = I + A * K[i][j] + B * K2[i][j];
      t += (I + B * K[i][j] + Cc * K2[i][j]) * rho[j];
    }
    T[4 * i + 3] = t;
  }
}

/* Gauss-Newton step on the pose: solve (H + damping I) xi = -b by Cholesky,
 * then T_wc <- exp(xi^) T_wc. Returns 0, or 1 (pose untouched) when the
 * damped H is not positive definite. */
int orc_pose_step(const double H[36], const double b[6], double damping,
                  double T_wc[12], double xi_out[6]) {
  double L[6][6] = {{0}}, y[6], xi[6];
  for (int i = 0; i < 6; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = H[6 * i + j] + (i == j ? damping : 0.0);
      for (int l = 0; l < j; ++l) s -= L[i][l] * L[j][l];
      if (i == j) {
        if (!(s > 0.0)) return 1;
        L[i][i] = sqrt(s);
      } else {
        L[i][j] = s / L[j][j];
      }
    }
  }
  for (int i = 0; i < 6; ++i) {
    double s = -b[i];
    for (int l = 0; l < i; ++l) s -= L[i][l] * y[l];
    y[i] = s / L[i][i];
  }
  for (int i = 5; i >= 0; --i) {
    double s = y[i];
    for (int l = i + 1; l < 6; ++l) s -= L[l][i] * xi[l];
    xi[i] = s / L[i][i];
  }
  double E[12], Tn[12];
  orc_se3_exp(xi, E);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = j == 3 ? E[4 * i + 3] : 0.0;
      for (int l = 0; l < 3; ++l) s += E[4 * i + l] * T_wc[4 * l + j];
      Tn[4 * i + j] = s;
    }
  memcpy(T_wc, Tn, sizeof(Tn));
  if (xi_out) memcpy(xi_out, xi, sizeof(xi));
  return 0;
}

/* ------------------------------------------------------- grid growth */
/* Sec. 6.1 ("a dynamic voxel grid"; how it grows is not given). Reading:
 * every valid depth pixel of the cameras is lifted to its surface point
 * X = o + s R d_c (s = z for a z-depth, z / |d_c| for a ray distance), and
 * every vertex whose grid coordinates lie within `band` of X's on each axis
 * (|i - (X - lo) / h| <= band) is allocated if it was not. Vertices that were
 * not allocated before get the numbers n_alloc, n_alloc + 1, ... in link
 * order (x fastest, then y, then z). depth[] holds the cameras' pixels one
 * camera after another, row-major. Returns the number of vertices added;
 * links is updated in place. */
int64_t orc_grow(const int32_t res[3], const double lo[3], const double hi[3],
                 int32_t *links, int64_t n_alloc, const orc_camera *cams,
                 int32_t n_cams, const float *depth, int32_t depth_is_z,
                 double band) {
  const int64_t nv = (int64_t)res[0] * res[1] * res[2];
  unsigned char *mark = (unsigned char *)calloc((size_t)nv, 1);
  if (!mark) return -1;
  double h[3];
  for (int a = 0; a < 3; ++a) h[a] = (hi[a] - lo[a]) / (double)(res[a] - 1);
  int64_t row = 0;
  for (int c = 0; c < n_cams; ++c) {
    const orc_camera *cam = &cams[c];
    const double *T = cam->T_wc;
    for (int v = 0; v < cam->height; ++v) {
      for (int u = 0; u < cam->width; ++u, ++row) {
        const double z = (double)depth[row];
        if (!(isfinite(z) && z > 0.0)) continue;
        const double dc0 = (u + 0.5 - cam->cx) / cam->fx;
        const double dc1 = (v + 0.5 - cam->cy) / cam->fy;
        const double dc2 = 1.0;
        const double s =
            depth_is_z ? z : z / sqrt(dc0 * dc0 + dc1 * dc1 + dc2 * dc2);
        int64_t i0[3], i1[3];
        int empty = 0;
        for (int a = 0; a < 3; ++a) {
          const double w = T[4 * a + 0] * dc0 + T[4 * a + 1] * dc1 + T[4 * a + 2] * dc2;
          const double X = T[4 * a + 3] + s * w;
          const double gc = (X - lo[a]) / h[a];
          double first = ceil(gc - band), last = floor(gc + band);
          if (first < 0.0) first = 0.0;
          if (last > (double)(res[a] - 1)) last = (double)(res[a] - 1);
          if (first > last) { empty = 1; break; }
          i0[a] = (int64_t)first;
          i1[a] = (int64_t)last;
        }
        if (empty) continue;
        for (int64_t iz = i0[2]; iz <= i1[2]; ++iz)
          for (int64_t iy = i0[1]; iy <= i1[1]; ++iy)
            for (int64_t ix = i0[0]; ix <= i1[0]; ++ix)
              mark[(iz * res[1] + iy) * res[0] + ix] = 1;
      }
    }
  }
  int64_t added = 0;
  for (int64_t i = 0; i < nv; ++i) {
    if (mark[i] && links[i] < 0) {
      links[i] = (int32_t)(n_alloc + added);
      ++added;
    }
  }
  free(mark);
  return added;
}

/* ---------------------------------------------- Levenberg-Marquardt step */
/* Gauss-Newton with Marquardt's damping (the paper optimises the pose with
 * Adam, Sec. 5.4; the plain GN step of Sec. 5.3 can overshoot where the
 * density ramps are steep). One call per Jacobian evaluation at the current
 * pose, with that pose's loss. state[64]: [0] lambda, [1] loss of the last
 * accepted pose, [2] calls made, [3] 1 if this call accepted, [4..15] the
 * accepted pose, [16..51] its H, [52..57] its b; zero it before the first
 * call. A call accepts the current pose when it is the first or its loss is
 * not above the last accepted one (then lambda /= factor, at least 1e-12),
 * else restores the accepted pose (lambda *= factor, at most 1e12). It then
 * solves (H + lambda (diag H + 1e-12 max diag H)) xi = -b with the accepted
 * pose's H, b (lambda grows by factor while that is not positive definite,
 * up to 8 times) and sets pose <- exp(xi^) pose. Returns 0 on an accepted
 * pose, 2 after a rejection, 1 if no damping made the system definite (pose
 * left at the accepted one). */
static int solve_damped(const double H[36], const double b[6], double lam, double xi[6]) {
  double L[6][6] = {{0}}, y[6], dmax = 0.0;
  for (int i = 0; i < 6; ++i) dmax = H[7 * i] > dmax ? H[7 * i] : dmax;
  for (int i = 0; i < 6; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = H[6 * i + j] + (i == j ? lam * (H[7 * i] + 1e-12 * dmax) : 0.0);
      for (int l = 0; l < j; ++l) s -= L[i][l] * L[j][l];
      if (i == j) {
        if (!(s > 0.0)) return 1;
        L[i][i] = sqrt(s);
      } else {
        L[i][j] = s / L[j][j];
      }
    }
  }
  for (int i = 0; i < 6; ++i) {
    double s = -b[i];
    for (int l = 0; l < i; ++l) s -= L[i][l] * y[l];
    y[i] = s / L[i][i];
  }
  for (int i = 5; i >= 0; --i) {
    double s = y[i];
    for (int l = i + 1; l < 6; ++l) s -= L[l][i] * xi[l];
    xi[i] = s / L[i][i];
  }
  return 0;
}

int orc_pose_step_lm(const double H[36], const double b[6], double loss, double state[64],
                     double lambda_init, double factor, double T_wc[12], double xi_out[6]) {
  const int first = state[2] == 0.0;
  const int accept = first || !(loss > state[1]);
  double lam = first ? lambda_init : state[0];
  if (accept) {
    if (!first) lam = lam / factor < 1e-12 ? 1e-12 : lam / factor;
    memcpy(state + 4, T_wc, 12 * sizeof(double));
    state[1] = loss;
    memcpy(state + 16, H, 36 * sizeof(double));
    memcpy(state + 52, b, 6 * sizeof(double));
  } else {
    lam = lam * factor > 1e12 ? 1e12 : lam * factor;
    memcpy(T_wc, state + 4, 12 * sizeof(double));
  }
  double xi[6] = {0, 0, 0, 0, 0, 0};
  int ok = 0;
  for (int tries = 0; tries <= 8; ++tries) {
    if (solve_damped(state + 16, state + 52, lam, xi) == 0) {
      ok = 1;
      break;
    }
    lam *= factor;
  }
  state[0] = lam;
  state[2] += 1.0;
  state[3] = accept;
  if (xi_out) memcpy(xi_out, ok ? xi : (double[6]){0, 0, 0, 0, 0, 0}, 6 * sizeof(double));
  if (!ok) return 1;
  double E[12], Tn[12];
  orc_se3_exp(xi, E);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = j == 3 ? E[4 * i + 3] : 0.0;
      for (int l = 0; l < 3; ++l) s += E[4 * i + l] * T_wc[4 * l + j];
      Tn[4 * i + j] = s;
    }
  memcpy(T_wc, Tn, sizeof(Tn));
  return accept ? 0 : 2;
}
