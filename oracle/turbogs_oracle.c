/*
 * TurboGS double-precision CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load or call this code.  The
 * CUDA library never does, and the two share no source, header, table or
 * constant generator: the spherical-harmonic constants below are computed from
 * their normalisation formula, the random stream from the published SplitMix64
 * finaliser.
 *
 * Every function restates, in plain double-precision C, what one step of the
 * TurboGS training iteration computes (TurboGS, ICML 2026: Sec. 3.1 Eq. 1 for
 * compositing, Sec. 3.3-3.5 for error/age maps, view and pixel sampling
 * (view sampling: Sec. 3.4 Eqs. 5-6), Sec. 3.7 and
 * App. A for the loss and its gradients, Sec. 3.8 for the error
 * back-projection statistics and the difficulty scores of Eq. 13 (no kernel
 * yet), Sec. 3.9 and App. A for the hybrid solver).  The
 * projection follows the 3D Gaussian Splatting model the paper builds on
 * (Sec. 3.1: centre, covariance from scale and rotation, opacity, SH colour;
 * the paper defers the rest to the standard 3DGS pipeline).  No blocking, fusion or reordering
 * beyond what those definitions state: each sampled pixel is rendered on its own
 * from the full Gaussian set, each tile's loss from its own pixel list.
 *
 * Where a floating-point comparison decides an integer the paper leaves the
 * precision open; the oracle then decides in single precision, the precision
 * of the kernels (tile membership of a splat: rect_axis below).  Everything
 * else is double precision.
 *
 * Pins (tests/test_oracle_*.py, run with -m "not gpu"): SH basis against
 * scipy's spherical harmonics; closed-form image of one isotropic Gaussian;
 * transmittance identity; pixel independence; brute-force tile overlap;
 * rotated anisotropic and off-centre projections, SH view direction;
 * sampling counts, brute-force TopK, inclusion probabilities of the weighted
 * draw against exact enumeration of sequential draws (tiles, pixels and
 * views); exact view error sums against fp16 values summed in numpy; camera
 * pose against the look-at construction; NCC invariances and
 * finite differences of the loss; finite differences of the whole
 * project -> render -> loss chain against the analytic backward; Cholesky
 * against LU, Sherman-Morrison and J = 0 for the hybrid step; fp16 rounding
 * against numpy.  Parity status: pinned (no function here is unpinned).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TILE 16
#define ORC_NSH 16

/* ------------------------------------------------------------------------ */
/* small helpers                                                            */
/* ------------------------------------------------------------------------ */

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* C = A (m x k) * B (k x n), row-major */
static void matmul(const double* A, const double* B, double* C, int m, int k, int n) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int l = 0; l < k; ++l) s += A[i * k + l] * B[l * n + j];
      C[i * n + j] = s;
    }
}

static void transpose(const double* A, double* At, int m, int n) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) At[j * m + i] = A[i * n + j];
}

/* Rotation matrix of the unit quaternion q = (w, x, y, z). */
static void quat_to_rot(const double q[4], double R[9]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* ------------------------------------------------------------------------ */
/* fp16 <-> double (IEEE 754 binary16, round to nearest even)               */
/* ------------------------------------------------------------------------ */

double orc_half_to_double(uint16_t h) {
  int s = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
  double v;
  if (e == 0) v = ldexp((double)m, -24);
  else if (e == 31) v = m ? NAN : INFINITY;
  else v = ldexp((double)(1024 + m), e - 25);
  return s ? -v : v;
}

uint16_t orc_double_to_half(double x) {
  uint16_t s = signbit(x) ? 0x8000 : 0;
  double a = fabs(x);
  if (isnan(x)) return 0x7e00;
  if (a < ldexp(1.0, -14)) {                 /* subnormal range: units of 2^-24 */
    double q = rint(a * 16777216.0);         /* exact scaling, RNE */
    return (uint16_t)(s | (uint16_t)q);      /* q == 1024 encodes the smallest normal */
  }
  int E;
  double f = frexp(a, &E);                   /* a = f * 2^E, f in [0.5, 1) */
  int e = E - 1;                             /* a = (2f) * 2^e */
  double m = rint(2.0 * f * 1024.0);         /* in [1024, 2048] */
  if (m >= 2048.0) { m = 1024.0; e += 1; }
  if (e > 15) return (uint16_t)(s | 0x7c00);
  return (uint16_t)(s | (uint16_t)((e + 15) << 10) | (uint16_t)(m - 1024.0));
}

/* ------------------------------------------------------------------------ */
/* real spherical harmonics, degree <= 3                                    */
/* ------------------------------------------------------------------------ */

/* K_l^m = sqrt((2l+1)/(4 pi) * (l-m)!/(l+m)!) */
static double sh_norm(int l, int m) {
  double num = 1.0, den = 1.0;
  for (int k = 2; k <= l - m; ++k) num *= k;
  for (int k = 2; k <= l + m; ++k) den *= k;
  return sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * num / den);
}

/*
 * Real SH Y_{l,m} (m = -l..l, index l*l+l+m) of a unit direction d, with the
 * Condon-Shortley phase in the associated Legendre functions:
 *   m > 0: sqrt2 K_l^m cos(m phi) P_l^m(cos theta)
 *   m = 0: K_l^0 P_l^0(cos theta)
 *   m < 0: sqrt2 K_l^|m| sin(|m| phi) P_l^|m|(cos theta)
 * written out as polynomials of (x, y, z) on the unit sphere, using
 * P_1^1 = -sin, P_2^1 = -3 cos sin, P_2^2 = 3 sin^2, P_3^1 = -3/2 (5cos^2-1) sin,
 * P_3^2 = 15 cos sin^2, P_3^3 = -15 sin^3 and x = sin cos(phi), y = sin sin(phi).
 * grad (optional, [16][3]) receives the gradient of each polynomial.
 */
void orc_sh_basis(const double d[3], double Y[16], double grad[48]) {
  const double r2 = sqrt(2.0);
  double x = d[0], y = d[1], z = d[2];
  double c0 = sh_norm(0, 0);
  double c1 = r2 * sh_norm(1, 1), c10 = sh_norm(1, 0);
  double c22 = r2 * sh_norm(2, 2), c21 = r2 * sh_norm(2, 1), c20 = sh_norm(2, 0);
  double c33 = r2 * sh_norm(3, 3), c32 = r2 * sh_norm(3, 2), c31 = r2 * sh_norm(3, 1), c30 = sh_norm(3, 0);
  /* polynomial coefficients */
  double k1 = -c1, k2 = c10, k3 = -c1;
  double k4 = 6 * c22, k5 = -3 * c21, k6 = 0.5 * c20, k7 = -3 * c21, k8 = 3 * c22;
  double k9 = -15 * c33, k10 = 30 * c32, k11 = -1.5 * c31, k12 = 0.5 * c30, k13 = -1.5 * c31,
         k14 = 15 * c32, k15 = -15 * c33;
  Y[0] = c0;
  Y[1] = k1 * y;
  Y[2] = k2 * z;
  Y[3] = k3 * x;
  Y[4] = k4 * x * y;
  Y[5] = k5 * y * z;
  Y[6] = k6 * (2 * z * z - x * x - y * y);
  Y[7] = k7 * x * z;
  Y[8] = k8 * (x * x - y * y);
  Y[9] = k9 * y * (3 * x * x - y * y);
  Y[10] = k10 * x * y * z;
  Y[11] = k11 * y * (4 * z * z - x * x - y * y);
  Y[12] = k12 * z * (2 * z * z - 3 * x * x - 3 * y * y);
  Y[13] = k13 * x * (4 * z * z - x * x - y * y);
  Y[14] = k14 * z * (x * x - y * y);
  Y[15] = k15 * x * (x * x - 3 * y * y);
  if (!grad) return;
  double* g = grad;
#define G(i, a, b, c) do { g[3 * (i)] = (a); g[3 * (i) + 1] = (b); g[3 * (i) + 2] = (c); } while (0)
  G(0, 0, 0, 0);
  G(1, 0, k1, 0);
  G(2, 0, 0, k2);
  G(3, k3, 0, 0);
  G(4, k4 * y, k4 * x, 0);
  G(5, 0, k5 * z, k5 * y);
  G(6, -2 * k6 * x, -2 * k6 * y, 4 * k6 * z);
  G(7, k7 * z, 0, k7 * x);
  G(8, 2 * k8 * x, -2 * k8 * y, 0);
  G(9, 6 * k9 * x * y, k9 * (3 * x * x - 3 * y * y), 0);
  G(10, k10 * y * z, k10 * x * z, k10 * x * y);
  G(11, -2 * k11 * x * y, k11 * (4 * z * z - x * x - 3 * y * y), 8 * k11 * y * z);
  G(12, -6 * k12 * x * z, -6 * k12 * y * z, k12 * (6 * z * z - 3 * x * x - 3 * y * y));
  G(13, k13 * (4 * z * z - 3 * x * x - y * y), -2 * k13 * x * y, 8 * k13 * x * z);
  G(14, 2 * k14 * x * z, -2 * k14 * y * z, k14 * (x * x - y * y));
  G(15, k15 * (3 * x * x - 3 * y * y), -6 * k15 * x * y, 0);
#undef G
}

/* ------------------------------------------------------------------------ */
/* camera                                                                   */
/* ------------------------------------------------------------------------ */

/* cam = [viewmat (16, row-major world->camera; x right, y down, z forward),
 *        fx, fy, cx, cy, znear] */
typedef struct {
  double W[9], t[3], fx, fy, cx, cy, znear, campos[3];
  int width, height, tiles_x, tiles_y;
} cam_t;

static void cam_load(const double* c, int width, int height, cam_t* o) {
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 3; ++k) o->W[r * 3 + k] = c[r * 4 + k];
    o->t[r] = c[r * 4 + 3];
  }
  o->fx = c[16]; o->fy = c[17]; o->cx = c[18]; o->cy = c[19]; o->znear = c[20];
  o->width = width; o->height = height;
  o->tiles_x = (width + ORC_TILE - 1) / ORC_TILE;
  o->tiles_y = (height + ORC_TILE - 1) / ORC_TILE;
  for (int k = 0; k < 3; ++k)
    o->campos[k] = -(o->W[0 * 3 + k] * o->t[0] + o->W[1 * 3 + k] * o->t[1] + o->W[2 * 3 + k] * o->t[2]);
}

/*
 * Tiles [lo, hi) on one axis covered by the square [c - r, c + r]: tile k
 * (pixels [16k, 16k+16)) is covered when 16k <= c + r and 16(k+1) > c - r.
 * Decided in single precision (see file header).
 */
static void rect_axis(double c, int r, int ntiles, int* lo, int* hi) {
  float cf = (float)c, rf = (float)r;
  float a = floorf((cf - rf) * 0.0625f);
  float b = floorf((cf + rf) * 0.0625f) + 1.0f;
  a = fminf(fmaxf(a, 0.0f), (float)ntiles);
  b = fminf(fmaxf(b, 0.0f), (float)ntiles);
  *lo = (int)a;
  *hi = (int)b;
}

/* distance in pixels of the single-precision rect decision to its switching
 * points, scaled so that 1e-4 is ~100 times the single-precision error of the
 * centre coordinate (diagnostic for parity tests) */
static double rect_margin(double c, int r) {
  double a = (c - r) / 16.0, b = (c + r) / 16.0;
  double da = fabs(a - floor(a + 0.5)), db = fabs(b - floor(b + 0.5));
  double m = (da < db ? da : db) * 16.0;
  return m / (10.0 + 0.1 * (fabs(c) + r));
}

/* ------------------------------------------------------------------------ */
/* projection (3DGS forward model: EWA splatting + SH colour)               */
/* ------------------------------------------------------------------------ */

typedef struct {
  int visible;
  double q[4], qnorm, R[9], s[3], Sigma[9];
  double pc[3];
  int clampx, clampy;
  double J[6], T[6];
  double A, B, C;           /* 2D covariance incl. +0.3 dilation */
  double det, conic[3];
  double lam, radius_f;
  int radius;
  double xy[2];
  double v[3], vlen, dir[3];
  double rgb_pre[3], rgb[3];
  double opac;
  double margin;
} gproj_t;

static double minabs(double a, double b) { return a < b ? a : b; }

/*
 * One Gaussian.  means (3), log_scales (3), quat (4, w x y z, unnormalised),
 * opacity logit, sh [16][3].  tile_rank (nullable): [tiles] >= 0 where a tile is
 * active; a Gaussian covering no active tile is culled.
 */
static void project_one(const double* mu, const double* ls, const double* qr, double ol, const double* sh,
                        int sh_degree, const cam_t* cam, const int32_t* tile_rank, gproj_t* g) {
  memset(g, 0, sizeof(*g));
  g->margin = INFINITY;
  /* camera space */
  for (int r = 0; r < 3; ++r)
    g->pc[r] = cam->W[r * 3 + 0] * mu[0] + cam->W[r * 3 + 1] * mu[1] + cam->W[r * 3 + 2] * mu[2] + cam->t[r];
  double z = g->pc[2];
  g->margin = minabs(g->margin, fabs(z - cam->znear) / cam->znear);
  if (!(z > cam->znear)) return;
  /* 3D covariance Sigma = R S S^T R^T */
  g->qnorm = sqrt(qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]);
  for (int k = 0; k < 4; ++k) g->q[k] = qr[k] / g->qnorm;
  quat_to_rot(g->q, g->R);
  for (int k = 0; k < 3; ++k) g->s[k] = exp(ls[k]);
  double M[9], Mt[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) M[r * 3 + c] = g->R[r * 3 + c] * g->s[c];
  transpose(M, Mt, 3, 3);
  matmul(M, Mt, g->Sigma, 3, 3, 3);
  /* local affine approximation of the perspective map (EWA) */
  double limx = 1.3 * (0.5 * cam->width / cam->fx), limy = 1.3 * (0.5 * cam->height / cam->fy);
  double xz = g->pc[0] / z, yz = g->pc[1] / z;
  g->clampx = (xz < -limx || xz > limx);
  g->clampy = (yz < -limy || yz > limy);
  double txz = clampd(xz, -limx, limx), tyz = clampd(yz, -limy, limy);
  g->J[0] = cam->fx / z; g->J[1] = 0.0; g->J[2] = -cam->fx * txz / z;
  g->J[3] = 0.0; g->J[4] = cam->fy / z; g->J[5] = -cam->fy * tyz / z;
  matmul(g->J, cam->W, g->T, 2, 3, 3);
  double TS[6], Tt[6], S2[4];
  matmul(g->T, g->Sigma, TS, 2, 3, 3);
  transpose(g->T, Tt, 2, 3);
  matmul(TS, Tt, S2, 2, 3, 2);
  g->A = S2[0] + 0.3; g->B = S2[1]; g->C = S2[3] + 0.3;
  g->det = g->A * g->C - g->B * g->B;
  g->margin = minabs(g->margin, fabs(g->det) / (g->A * g->C));
  if (!(g->det > 0.0)) return;
  g->conic[0] = g->C / g->det; g->conic[1] = -g->B / g->det; g->conic[2] = g->A / g->det;
  double mid = 0.5 * (g->A + g->C);
  double disc = mid * mid - g->det;
  g->lam = mid + sqrt(disc > 0.1 ? disc : 0.1);
  g->radius_f = 3.0 * sqrt(g->lam);
  g->radius = (int)ceil(g->radius_f);
  g->margin = minabs(g->margin, fabs(g->radius_f - floor(g->radius_f + 0.5)) / (g->radius_f + 1.0));
  g->xy[0] = cam->fx * g->pc[0] / z + cam->cx;
  g->xy[1] = cam->fy * g->pc[1] / z + cam->cy;
  /* tile rectangle (single-precision decision) and active-tile culling */
  int x0, x1, y0, y1;
  rect_axis(g->xy[0], g->radius, cam->tiles_x, &x0, &x1);
  rect_axis(g->xy[1], g->radius, cam->tiles_y, &y0, &y1);
  g->margin = minabs(g->margin, rect_margin(g->xy[0], g->radius));
  g->margin = minabs(g->margin, rect_margin(g->xy[1], g->radius));
  if ((x1 - x0) * (y1 - y0) == 0) { g->radius = 0; return; }
  if (tile_rank) {
    int any = 0;
    for (int ty = y0; ty < y1 && !any; ++ty)
      for (int tx = x0; tx < x1; ++tx)
        if (tile_rank[ty * cam->tiles_x + tx] >= 0) { any = 1; break; }
    if (!any) { g->radius = 0; return; }
  }
  g->visible = 1;
  /* colour: SH evaluated in the direction from the camera centre */
  for (int k = 0; k < 3; ++k) g->v[k] = mu[k] - cam->campos[k];
  g->vlen = sqrt(g->v[0] * g->v[0] + g->v[1] * g->v[1] + g->v[2] * g->v[2]);
  for (int k = 0; k < 3; ++k) g->dir[k] = g->v[k] / g->vlen;
  double Y[16];
  orc_sh_basis(g->dir, Y, NULL);
  int nb = (sh_degree + 1) * (sh_degree + 1);
  for (int c = 0; c < 3; ++c) {
    double s = 0.5;
    for (int k = 0; k < nb; ++k) s += sh[k * 3 + c] * Y[k];
    g->rgb_pre[c] = s;
    g->rgb[c] = s > 0.0 ? s : 0.0;
    g->margin = minabs(g->margin, fabs(s));
  }
  g->opac = 1.0 / (1.0 + exp(-ol));
}

/*
 * Project N Gaussians.  Outputs (culled Gaussians get radius 0 and zeros):
 * xy [N,2] pixel coordinates of the centre (pixel i covers [i, i+1)),
 * conic [N,3] = (a, b, c) of the inverse 2D covariance [[a, b], [b, c]],
 * opac [N], rgb [N,3], depth [N] = camera-space z, radius [N],
 * margin [N] = smallest relative distance of a discrete decision to its
 * threshold (diagnostic, nullable).
 */
int orc_project(int64_t n, const double* means, const double* log_scales, const double* quats,
                const double* opacity_logits, const double* sh, int sh_degree, const double* cam_in,
                int width, int height, const int32_t* tile_rank, double* xy, double* conic, double* opac,
                double* rgb, double* depth, int32_t* radius, double* margin) {
  cam_t cam;
  cam_load(cam_in, width, height, &cam);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    gproj_t g;
    project_one(means + 3 * i, log_scales + 3 * i, quats + 4 * i, opacity_logits[i], sh + 48 * i, sh_degree,
                &cam, tile_rank, &g);
    int vis = g.visible;
    xy[2 * i] = vis ? g.xy[0] : 0.0;
    xy[2 * i + 1] = vis ? g.xy[1] : 0.0;
    for (int k = 0; k < 3; ++k) {
      conic[3 * i + k] = vis ? g.conic[k] : 0.0;
      rgb[3 * i + k] = vis ? g.rgb[k] : 0.0;
    }
    opac[i] = vis ? g.opac : 0.0;
    depth[i] = vis ? g.pc[2] : 0.0;
    radius[i] = vis ? g.radius : 0;
    if (margin) margin[i] = g.margin;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* tile binning (brute force)                                               */
/* ------------------------------------------------------------------------ */

typedef struct { uint64_t key; int32_t id; } isect_t;

static int cmp_isect(const void* a, const void* b) {
  const isect_t* x = (const isect_t*)a;
  const isect_t* y = (const isect_t*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->id < y->id ? -1 : (x->id > y->id);
}

static uint32_t f32_bits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/*
 * Every (active tile, Gaussian) pair whose rectangle covers the tile, ordered
 * by (tile id, depth, Gaussian id): the per-tile lists K sorted by depth
 * (Sec. 3.1).  Inputs are single precision as the library stores them.
 * keys[i] = tile_id << 32 | float bits of depth (depth > 0 orders as an
 * unsigned integer), vals[i] = Gaussian id, counts [tiles] per tile.
 * Returns the number of pairs (capacity < 0: size query only), or -1 if it
 * exceeds capacity.
 */
int64_t orc_bin_tiles(int64_t n, const float* xy, const int32_t* radius, const float* depth, int width,
                      int height, const int32_t* tile_rank, int64_t capacity, uint64_t* keys, int32_t* vals,
                      int32_t* counts) {
  int tx_n = (width + ORC_TILE - 1) / ORC_TILE, ty_n = (height + ORC_TILE - 1) / ORC_TILE;
  int64_t total = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (radius[i] <= 0) continue;
    int x0, x1, y0, y1;
    rect_axis(xy[2 * i], radius[i], tx_n, &x0, &x1);
    rect_axis(xy[2 * i + 1], radius[i], ty_n, &y0, &y1);
    for (int ty = y0; ty < y1; ++ty)
      for (int tx = x0; tx < x1; ++tx)
        if (!tile_rank || tile_rank[ty * tx_n + tx] >= 0) total++;
  }
  for (int t = 0; t < tx_n * ty_n; ++t) counts[t] = 0;
  if (capacity < 0) return total;          /* size query */
  if (total > capacity) return -1;
  isect_t* all = (isect_t*)malloc(sizeof(isect_t) * (size_t)(total > 0 ? total : 1));
  int64_t k = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (radius[i] <= 0) continue;
    int x0, x1, y0, y1;
    rect_axis(xy[2 * i], radius[i], tx_n, &x0, &x1);
    rect_axis(xy[2 * i + 1], radius[i], ty_n, &y0, &y1);
    for (int ty = y0; ty < y1; ++ty)
      for (int tx = x0; tx < x1; ++tx) {
        int t = ty * tx_n + tx;
        if (tile_rank && tile_rank[t] < 0) continue;
        all[k].key = ((uint64_t)t << 32) | f32_bits(depth[i]);
        all[k].id = (int32_t)i;
        counts[t]++;
        k++;
      }
  }
  qsort(all, (size_t)total, sizeof(isect_t), cmp_isect);
  for (int64_t j = 0; j < total; ++j) { keys[j] = all[j].key; vals[j] = all[j].id; }
  free(all);
  return total;
}

/* ------------------------------------------------------------------------ */
/* counter-based random stream and the weighted draw without replacement    */
/* ------------------------------------------------------------------------ */

/* SplitMix64 output function (Steele, Lea, Flood 2014). */
uint64_t orc_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* hash of (seed, iteration, view, stream, tile, item) */
uint64_t orc_hash(uint64_t seed, uint64_t iter, uint32_t view, uint32_t stream, uint32_t tile, uint32_t item) {
  uint64_t h = orc_mix64(seed + 0x9E3779B97F4A7C15ULL);
  h = orc_mix64(h ^ iter);
  h = orc_mix64(h ^ (((uint64_t)view << 8) | stream));
  h = orc_mix64(h ^ (((uint64_t)tile << 16) | item));
  return h;
}

/*
 * -log2(u / 2^64) in fixed point with 32 fractional bits, for u = h | 1,
 * by the binary-logarithm digit recurrence: normalise the mantissa to [1, 2),
 * square it, and read one fractional bit per squaring (value >= 2).
 * Integer-only, so both implementations agree bit for bit.
 */
uint64_t orc_neglog2_q32(uint64_t h) {
  uint64_t u = h | 1ULL;
  int lz = 0;
  while (!((u << lz) & 0x8000000000000000ULL)) lz++;
  int ip = 63 - lz;
  uint64_t m = u << lz;
  uint64_t frac = 0;
  for (int i = 0; i < 32; ++i) {
    unsigned __int128 sq = (unsigned __int128)m * m;
    uint64_t hi = (uint64_t)(sq >> 64);
    frac <<= 1;
    if (hi & 0x8000000000000000ULL) { frac |= 1; m = hi; }
    else m = hi << 1;
  }
  return ((uint64_t)(64 - ip) << 32) - frac;
}

/* integer weight of an fp16 error value: E * 2^24 exactly (0 for negative,
 * NaN or infinity) */
uint64_t orc_err_weight(uint16_t h) {
  if (h & 0x8000) return 0;
  int e = (h >> 10) & 31, m = h & 1023;
  if (e == 31) return 0;
  if (e == 0) return (uint64_t)m;
  return (uint64_t)(1024 + m) << (e - 1);
}

typedef struct {
  int idx;
  uint64_t w;      /* weight for the error-proportional draw */
  uint64_t L;      /* exponential clock -log2(U), fixed point */
  uint32_t age;
  uint64_t u;      /* uniform key */
  int taken;
} item_t;

/*
 * Order of the error-proportional draw without replacement
 * (Efraimidis-Spirakis: ascending L_i / w_i is the order of successive
 * weighted draws).  The key is L / w in IEEE double precision (both integers
 * are exact in double, the division is correctly rounded, so the key is the
 * same on every machine); items of weight 0 follow every positive weight in
 * uniform random order (key L * 2^900, larger than any L / w with w >= 1).
 * Equal keys go to the lower index.
 */
double orc_hard_key(uint64_t w, uint64_t L) {
  return w ? (double)L / (double)w : ldexp((double)L, 900);
}
static int cmp_hard(const void* a, const void* b) {
  const item_t* x = (const item_t*)a;
  const item_t* y = (const item_t*)b;
  double kx = orc_hard_key(x->w, x->L), ky = orc_hard_key(y->w, y->L);
  if (kx != ky) return kx < ky ? -1 : 1;
  return x->idx - y->idx;
}
static int cmp_age(const void* a, const void* b) {   /* descending age, ties by index */
  const item_t* x = (const item_t*)a;
  const item_t* y = (const item_t*)b;
  if (x->age != y->age) return x->age > y->age ? -1 : 1;
  return x->idx - y->idx;
}
static int cmp_unif(const void* a, const void* b) {  /* ascending top 32 hash bits, then index */
  const item_t* x = (const item_t*)a;
  const item_t* y = (const item_t*)b;
  uint32_t ux = (uint32_t)(x->u >> 32), uy = (uint32_t)(y->u >> 32);
  if (ux != uy) return ux < uy ? -1 : 1;
  return x->idx - y->idx;
}
static int cmp_idx(const void* a, const void* b) {
  return ((const item_t*)a)->idx - ((const item_t*)b)->idx;
}

/* split of n draws: hard = round(r_hard n), stable = round(r_stable n) clamped
 * so hard + stable <= n, rest = n - hard - stable (ratios in 1/1000) */
static void split_counts(int n, int hard_pm, int stable_pm, int* kh, int* ks, int* kr) {
  int h = (hard_pm * n + 500) / 1000;
  if (h > n) h = n;
  int s = (stable_pm * n + 500) / 1000;
  if (s > n - h) s = n - h;
  *kh = h; *ks = s; *kr = n - h - s;
}

/*
 * Choose n of the items: kh by the error-proportional draw without
 * replacement, then ks of the rest with the largest age (TopK), then the
 * remainder uniformly without replacement.  Marks taken = 1 on the chosen.
 */
static void choose(item_t* it, int cnt, int n, int hard_pm, int stable_pm) {
  int kh, ks, kr;
  if (n > cnt) n = cnt;
  split_counts(n, hard_pm, stable_pm, &kh, &ks, &kr);
  item_t* tmp = (item_t*)malloc(sizeof(item_t) * (size_t)(cnt > 0 ? cnt : 1));
  int m = 0;
  for (int i = 0; i < cnt; ++i) tmp[m++] = it[i];
  qsort(tmp, (size_t)m, sizeof(item_t), cmp_hard);
  for (int i = 0; i < kh; ++i) it[tmp[i].idx].taken = 1;
  m = 0;
  for (int i = 0; i < cnt; ++i) if (!it[i].taken) tmp[m++] = it[i];
  qsort(tmp, (size_t)m, sizeof(item_t), cmp_age);
  for (int i = 0; i < ks; ++i) it[tmp[i].idx].taken = 1;
  m = 0;
  for (int i = 0; i < cnt; ++i) if (!it[i].taken) tmp[m++] = it[i];
  qsort(tmp, (size_t)m, sizeof(item_t), cmp_unif);
  for (int i = 0; i < kr; ++i) it[tmp[i].idx].taken = 1;
  free(tmp);
}

/* streams of the random hash */
#define ORC_STREAM_TILE_HARD 1
#define ORC_STREAM_TILE_UNIF 2
#define ORC_STREAM_PIX_HARD 3
#define ORC_STREAM_PIX_UNIF 4

/* exposed for the sampling pins: choose n of cnt items with given weights and
 * ages; hash streams of the pixel level of tile `tile`. out_taken [cnt] */
int orc_choose_items(int cnt, const uint64_t* w, const uint32_t* age, int n, int hard_pm, int stable_pm,
                     uint64_t seed, uint64_t iter, uint32_t view, uint32_t tile, uint8_t* out_taken) {
  item_t* it = (item_t*)malloc(sizeof(item_t) * (size_t)(cnt > 0 ? cnt : 1));
  for (int i = 0; i < cnt; ++i) {
    it[i].idx = i; it[i].w = w[i]; it[i].age = age[i]; it[i].taken = 0;
    it[i].L = orc_neglog2_q32(orc_hash(seed, iter, view, ORC_STREAM_PIX_HARD, tile, (uint32_t)i));
    it[i].u = orc_hash(seed, iter, view, ORC_STREAM_PIX_UNIF, tile, (uint32_t)i);
  }
  choose(it, cnt, n, hard_pm, stable_pm);
  for (int i = 0; i < cnt; ++i) out_taken[i] = (uint8_t)it[i].taken;
  free(it);
  return 0;
}

/*
 * Tile selection and tile-wise pixel sampling (Sec. 3.5).
 * Tile level: n_select tiles, split by tile_hard_pm / tile_stable_pm; a tile's
 * weight is the sum of its pixels' weights, its age the smallest pixel age
 * (iterations since any of its pixels was sampled).
 * Pixel level: in each selected tile N_pix = min(n_pix, valid pixels), split
 * into N_hard = round(r_hard N_pix) drawn proportionally to E without
 * replacement, N_stable = round(r_stable N_pix) of largest age among the
 * rest, and the remainder uniformly.
 * Outputs: active_tiles (ascending), *n_active, tile_rank [tiles] (-1 when not
 * selected), pix_off [n_active + 1], pix_idx (local index ly*16+lx, ascending
 * within each tile).
 */
int orc_select(int width, int height, const uint16_t* err, const uint16_t* age, int n_select, int n_pix,
               int tile_hard_pm, int tile_stable_pm, int pix_hard_pm, int pix_stable_pm, uint64_t seed,
               uint64_t iter, uint32_t view, int32_t* active_tiles, int32_t* n_active, int32_t* tile_rank,
               int32_t* pix_off, uint8_t* pix_idx) {
  int tx_n = (width + ORC_TILE - 1) / ORC_TILE, ty_n = (height + ORC_TILE - 1) / ORC_TILE;
  int T = tx_n * ty_n;
  item_t* tiles = (item_t*)malloc(sizeof(item_t) * (size_t)T);
  for (int t = 0; t < T; ++t) {
    int tx = t % tx_n, ty = t / tx_n;
    uint64_t w = 0;
    uint32_t amin = 0xFFFFFFFFu;
    for (int ly = 0; ly < ORC_TILE; ++ly)
      for (int lx = 0; lx < ORC_TILE; ++lx) {
        int x = tx * ORC_TILE + lx, y = ty * ORC_TILE + ly;
        if (x >= width || y >= height) continue;
        w += orc_err_weight(err[(int64_t)y * width + x]);
        uint32_t a = age[(int64_t)y * width + x];
        if (a < amin) amin = a;
      }
    tiles[t].idx = t; tiles[t].w = w; tiles[t].age = amin; tiles[t].taken = 0;
    tiles[t].L = orc_neglog2_q32(orc_hash(seed, iter, view, ORC_STREAM_TILE_HARD, (uint32_t)t, 0));
    tiles[t].u = orc_hash(seed, iter, view, ORC_STREAM_TILE_UNIF, (uint32_t)t, 0);
  }
  choose(tiles, T, n_select < 0 ? 0 : n_select, tile_hard_pm, tile_stable_pm);
  int A = 0;
  pix_off[0] = 0;
  item_t px[ORC_TILE * ORC_TILE];
  for (int t = 0; t < T; ++t) {
    tile_rank[t] = -1;
    if (!tiles[t].taken) continue;
    tile_rank[t] = A;
    active_tiles[A] = t;
    int tx = t % tx_n, ty = t / tx_n;
    int cnt = 0;
    for (int ly = 0; ly < ORC_TILE; ++ly)
      for (int lx = 0; lx < ORC_TILE; ++lx) {
        int x = tx * ORC_TILE + lx, y = ty * ORC_TILE + ly;
        if (x >= width || y >= height) continue;
        int l = ly * ORC_TILE + lx;
        item_t* p = &px[cnt];
        p->idx = cnt;
        p->w = orc_err_weight(err[(int64_t)y * width + x]);
        p->age = age[(int64_t)y * width + x];
        p->L = orc_neglog2_q32(orc_hash(seed, iter, view, ORC_STREAM_PIX_HARD, (uint32_t)t, (uint32_t)l));
        p->u = orc_hash(seed, iter, view, ORC_STREAM_PIX_UNIF, (uint32_t)t, (uint32_t)l);
        p->taken = l;             /* stash local index; reset below */
        cnt++;
      }
    int local[ORC_TILE * ORC_TILE];
    for (int i = 0; i < cnt; ++i) { local[i] = px[i].taken; px[i].taken = 0; }
    choose(px, cnt, n_pix, pix_hard_pm, pix_stable_pm);
    int o = pix_off[A];
    for (int i = 0; i < cnt; ++i)
      if (px[i].taken) pix_idx[o++] = (uint8_t)local[i];
    pix_off[A + 1] = o;
    A++;
  }
  *n_active = A;
  free(tiles);
  (void)cmp_idx;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* sparse forward rendering (Eq. 1), one pixel at a time                    */
/* ------------------------------------------------------------------------ */

typedef struct { double depth; int32_t id; } cand_t;

static int cmp_cand(const void* a, const void* b) {
  const cand_t* x = (const cand_t*)a;
  const cand_t* y = (const cand_t*)b;
  if (x->depth != y->depth) return x->depth < y->depth ? -1 : 1;
  return x->id - y->id;
}

typedef struct {
  int n_cand;
  cand_t* cand;
  /* per accepted splat k (in order) */
  int n_acc;
  int* acc_id;        /* Gaussian id */
  int* acc_pos;       /* position in the candidate list */
  double *T, *alpha, *G, *dx, *dy;
  int* clamped;       /* alpha hit the 0.99 cap */
  double T_final;
  int n_last;         /* position + 1 of the last accepted splat, 0 if none */
  double margin;
} pixel_trace_t;

static void trace_free(pixel_trace_t* p) {
  free(p->cand); free(p->acc_id); free(p->acc_pos); free(p->T); free(p->alpha); free(p->G);
  free(p->dx); free(p->dy); free(p->clamped);
}

/*
 * Front-to-back compositing of pixel (px, py): the Gaussians whose tile
 * rectangle covers the pixel's tile, ordered by depth then id; alpha_k =
 * min(0.99, o_k exp(power_k)) with power = -(a dx^2 + c dy^2)/2 - b dx dy at
 * the pixel centre, splats with power > 0 or alpha < 1/255 skipped, stop
 * before the splat that would take T below 1e-4.
 */
static void trace_pixel(int64_t n, const double* xy, const double* conic, const double* opac,
                        const double* depth, const int32_t* radius, int tx_n, int ty_n, int px, int py,
                        pixel_trace_t* p) {
  memset(p, 0, sizeof(*p));
  p->margin = INFINITY;
  int ptx = px / ORC_TILE, pty = py / ORC_TILE;
  int cap = 64;
  p->cand = (cand_t*)malloc(sizeof(cand_t) * (size_t)cap);
  for (int64_t i = 0; i < n; ++i) {
    if (radius[i] <= 0) continue;
    int x0, x1, y0, y1;
    rect_axis(xy[2 * i], radius[i], tx_n, &x0, &x1);
    rect_axis(xy[2 * i + 1], radius[i], ty_n, &y0, &y1);
    if (ptx < x0 || ptx >= x1 || pty < y0 || pty >= y1) continue;
    if (p->n_cand == cap) { cap *= 2; p->cand = (cand_t*)realloc(p->cand, sizeof(cand_t) * (size_t)cap); }
    p->cand[p->n_cand].depth = depth[i];
    p->cand[p->n_cand].id = (int32_t)i;
    p->n_cand++;
  }
  qsort(p->cand, (size_t)p->n_cand, sizeof(cand_t), cmp_cand);
  int m = p->n_cand > 0 ? p->n_cand : 1;
  p->acc_id = (int*)malloc(sizeof(int) * m);
  p->acc_pos = (int*)malloc(sizeof(int) * m);
  p->T = (double*)malloc(sizeof(double) * m);
  p->alpha = (double*)malloc(sizeof(double) * m);
  p->G = (double*)malloc(sizeof(double) * m);
  p->dx = (double*)malloc(sizeof(double) * m);
  p->dy = (double*)malloc(sizeof(double) * m);
  p->clamped = (int*)malloc(sizeof(int) * m);
  double cxp = px + 0.5, cyp = py + 0.5;
  double T = 1.0;
  double prev_depth = -INFINITY;   /* depth of the last splat blended */
  for (int k = 0; k < p->n_cand; ++k) {
    int i = p->cand[k].id;
    double dx = cxp - xy[2 * i], dy = cyp - xy[2 * i + 1];
    double a = conic[3 * i], b = conic[3 * i + 1], c = conic[3 * i + 2];
    double power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
    if (power > 0.0) continue;
    double G = exp(power);
    double araw = opac[i] * G;
    double alpha = araw < 0.99 ? araw : 0.99;
    p->margin = minabs(p->margin, fabs(alpha * 255.0 - 1.0));
    p->margin = minabs(p->margin, fabs(araw - 0.99) / 0.99);
    if (alpha < 1.0 / 255.0) continue;
    /* order of two blended splats of almost equal depth is a discrete
       decision too (exact ties are ordered by id on both sides) */
    {
      double d1 = p->cand[k].depth;
      if (d1 > prev_depth) p->margin = minabs(p->margin, (d1 - prev_depth) / (fabs(d1) + 1e-30) * 1e2);
    }
    double Tn = T * (1.0 - alpha);
    p->margin = minabs(p->margin, fabs(Tn - 1e-4) / 1e-4);
    if (Tn < 1e-4) break;
    prev_depth = p->cand[k].depth;
    int j = p->n_acc++;
    p->acc_id[j] = i; p->acc_pos[j] = k;
    p->T[j] = T; p->alpha[j] = alpha; p->G[j] = G; p->dx[j] = dx; p->dy[j] = dy;
    p->clamped[j] = araw >= 0.99;
    T = Tn;
    p->n_last = k + 1;
  }
  p->T_final = T;
}

/*
 * Render the listed pixels (pix_xy [P,2] integer coordinates).  Outputs
 * rgb [P,3] = sum_k T_k alpha_k c_k + T_final bg, T_final [P], n_last [P]
 * (position + 1 in the pixel's depth-ordered list of the last splat blended),
 * n_contrib [P] and margin [P] (diagnostics, nullable).
 */
int orc_render_pixels(int64_t n, const double* xy, const double* conic, const double* opac,
                      const double* rgb, const double* depth, const int32_t* radius, int width, int height,
                      const double* bg, int64_t n_pix, const int32_t* pix_xy, double* out_rgb,
                      double* out_T, int32_t* out_nlast, int32_t* out_ncontrib, double* out_margin) {
  int tx_n = (width + ORC_TILE - 1) / ORC_TILE, ty_n = (height + ORC_TILE - 1) / ORC_TILE;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t s = 0; s < n_pix; ++s) {
    pixel_trace_t p;
    trace_pixel(n, xy, conic, opac, depth, radius, tx_n, ty_n, pix_xy[2 * s], pix_xy[2 * s + 1], &p);
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      for (int j = 0; j < p.n_acc; ++j) acc += p.T[j] * p.alpha[j] * rgb[3 * p.acc_id[j] + c];
      out_rgb[3 * s + c] = acc + p.T_final * bg[c];
    }
    out_T[s] = p.T_final;
    out_nlast[s] = p.n_last;
    if (out_ncontrib) out_ncontrib[s] = p.n_acc;
    if (out_margin) out_margin[s] = p.margin;
    trace_free(&p);
  }
  return 0;
}

/*
 * Adjoint of the compositing for the listed pixels, given dL/dI [P,3].
 * With S_k the colour seen behind splat k (S_n = bg,
 * S_k = alpha_k c_k + (1 - alpha_k) S_{k+1}):
 *   dL/dc_k = T_k alpha_k g,  dL/dalpha_k = T_k (c_k - S_{k+1}) . g,
 * alpha = o G (0 when capped at 0.99), G = exp(power).
 * Accumulates grad2d [N,9] = (d x, d y, d a, d b, d c, d opacity, d r, d g, d b).
 */
int orc_render_backward(int64_t n, const double* xy, const double* conic, const double* opac,
                        const double* rgb, const double* depth, const int32_t* radius, int width, int height,
                        const double* bg, int64_t n_pix, const int32_t* pix_xy, const double* dL_drgb,
                        double* grad2d) {
  int tx_n = (width + ORC_TILE - 1) / ORC_TILE, ty_n = (height + ORC_TILE - 1) / ORC_TILE;
  memset(grad2d, 0, sizeof(double) * 9 * (size_t)n);
  for (int64_t s = 0; s < n_pix; ++s) {
    pixel_trace_t p;
    trace_pixel(n, xy, conic, opac, depth, radius, tx_n, ty_n, pix_xy[2 * s], pix_xy[2 * s + 1], &p);
    const double* g = dL_drgb + 3 * s;
    double S[3] = {bg[0], bg[1], bg[2]};
    for (int j = p.n_acc - 1; j >= 0; --j) {
      int i = p.acc_id[j];
      const double* c = rgb + 3 * i;
      double T = p.T[j], al = p.alpha[j];
      double dalpha = 0.0;
      for (int ch = 0; ch < 3; ++ch) {
        grad2d[9 * i + 6 + ch] += T * al * g[ch];
        dalpha += T * (c[ch] - S[ch]) * g[ch];
      }
      for (int ch = 0; ch < 3; ++ch) S[ch] = al * c[ch] + (1.0 - al) * S[ch];
      if (p.clamped[j]) continue;
      double G = p.G[j], o = opac[i];
      grad2d[9 * i + 5] += dalpha * G;
      double dpow = dalpha * o * G;
      double dx = p.dx[j], dy = p.dy[j];
      double a = conic[3 * i], b = conic[3 * i + 1], cc = conic[3 * i + 2];
      /* power = -(a dx^2 + c dy^2)/2 - b dx dy, dx = px + 0.5 - x */
      grad2d[9 * i + 0] += dpow * (a * dx + b * dy);
      grad2d[9 * i + 1] += dpow * (cc * dy + b * dx);
      grad2d[9 * i + 2] += dpow * (-0.5 * dx * dx);
      grad2d[9 * i + 3] += dpow * (-dx * dy);
      grad2d[9 * i + 4] += dpow * (-0.5 * dy * dy);
    }
    trace_free(&p);
  }
  return 0;
}

/*
 * Error back-projection statistics (Sec. 3.8, Eq. 12) over the
 * listed pixels.  With w = T_k alpha_k the compositing weight of splat k at
 * pixel p (as the forward above composites it), stats [N,3] receives
 * (sum_p e(p) w, sum_p w, sum_p D w), where D = sqrt(a dx^2 + 2 b dx dy +
 * c dy^2) is the conic Mahalanobis distance of the pixel centre from the
 * splat's centre.  err [P]: the per-pixel error e(p).
 */
int orc_error_stats(int64_t n, const double* xy, const double* conic, const double* opac, const double* depth,
                    const int32_t* radius, int width, int height, int64_t n_pix, const int32_t* pix_xy,
                    const double* err, double* stats) {
  int tx_n = (width + ORC_TILE - 1) / ORC_TILE, ty_n = (height + ORC_TILE - 1) / ORC_TILE;
  memset(stats, 0, sizeof(double) * 3 * (size_t)n);
  for (int64_t s = 0; s < n_pix; ++s) {
    pixel_trace_t p;
    trace_pixel(n, xy, conic, opac, depth, radius, tx_n, ty_n, pix_xy[2 * s], pix_xy[2 * s + 1], &p);
    for (int j = 0; j < p.n_acc; ++j) {
      int i = p.acc_id[j];
      double w = p.T[j] * p.alpha[j];
      double dx = p.dx[j], dy = p.dy[j];
      double a = conic[3 * i], b = conic[3 * i + 1], c = conic[3 * i + 2];
      double q = a * dx * dx + 2.0 * b * dx * dy + c * dy * dy;
      double D = sqrt(q > 0.0 ? q : 0.0);
      stats[3 * i] += err[s] * w;
      stats[3 * i + 1] += w;
      stats[3 * i + 2] += D * w;
    }
    trace_free(&p);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* adjoint of the projection                                                */
/* ------------------------------------------------------------------------ */

/*
 * grads [N,59] = (means 3, log_scales 3, quats 4, opacity logit 1,
 * sh 48 in [16][3] order) from grad2d [N,9].  Culled Gaussians get zeros.
 */
int orc_project_backward(int64_t n, const double* means, const double* log_scales, const double* quats,
                         const double* opacity_logits, const double* sh, int sh_degree, const double* cam_in,
                         int width, int height, const int32_t* tile_rank, const double* grad2d,
                         double* grads) {
  cam_t cam;
  cam_load(cam_in, width, height, &cam);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double* out = grads + 59 * i;
    memset(out, 0, sizeof(double) * 59);
    gproj_t g;
    const double* mu = means + 3 * i;
    const double* shi = sh + 48 * i;
    project_one(mu, log_scales + 3 * i, quats + 4 * i, opacity_logits[i], shi, sh_degree, &cam, tile_rank, &g);
    if (!g.visible) continue;
    const double* d2 = grad2d + 9 * i;
    double dmu[3] = {0, 0, 0};
    /* opacity */
    out[10] = d2[5] * g.opac * (1.0 - g.opac);
    /* colour through SH (clamp at 0 passes no gradient) */
    double Y[16], dY[48];
    orc_sh_basis(g.dir, Y, dY);
    int nb = (sh_degree + 1) * (sh_degree + 1);
    double ddir[3] = {0, 0, 0};
    for (int c = 0; c < 3; ++c) {
      double dc = g.rgb_pre[c] >= 0.0 ? d2[6 + c] : 0.0;
      for (int k = 0; k < nb; ++k) {
        out[11 + 3 * k + c] = dc * Y[k];
        for (int a = 0; a < 3; ++a) ddir[a] += dc * shi[3 * k + c] * dY[3 * k + a];
      }
    }
    double dot = ddir[0] * g.dir[0] + ddir[1] * g.dir[1] + ddir[2] * g.dir[2];
    for (int a = 0; a < 3; ++a) dmu[a] += (ddir[a] - g.dir[a] * dot) / g.vlen;
    /* pixel centre u = fx x/z + cx, v = fy y/z + cy */
    double z = g.pc[2];
    double dpc[3];
    dpc[0] = d2[0] * cam.fx / z;
    dpc[1] = d2[1] * cam.fy / z;
    dpc[2] = -d2[0] * cam.fx * g.pc[0] / (z * z) - d2[1] * cam.fy * g.pc[1] / (z * z);
    /* conic Q = Sigma2^-1: dSigma2 = -Q dQ Q, dQ symmetric with off-diagonal db/2 */
    double Q[4] = {g.conic[0], g.conic[1], g.conic[1], g.conic[2]};
    double dQ[4] = {d2[2], 0.5 * d2[3], 0.5 * d2[3], d2[4]};
    double tmp[4], dS2[4];
    matmul(Q, dQ, tmp, 2, 2, 2);
    matmul(tmp, Q, dS2, 2, 2, 2);
    for (int k = 0; k < 4; ++k) dS2[k] = -dS2[k];
    /* Sigma2 = T Sigma T^T + 0.3 I, T = J W */
    double Tt[6], tmp3[6], dSigma[9], dT[6], dS2T[6], dS2TS[6];
    transpose(g.T, Tt, 2, 3);
    matmul(Tt, dS2, tmp3, 3, 2, 2);        /* T^T dS2     (3x2) */
    matmul(tmp3, g.T, dSigma, 3, 2, 3);    /* T^T dS2 T   (3x3) */
    matmul(dS2, g.T, dS2T, 2, 2, 3);       /* dS2 T       (2x3) */
    matmul(dS2T, g.Sigma, dS2TS, 2, 3, 3); /* dS2 T Sigma (2x3) */
    for (int k = 0; k < 6; ++k) dT[k] = 2.0 * dS2TS[k];
    double Wt[9], dJ[6];
    transpose(cam.W, Wt, 3, 3);
    matmul(dT, Wt, dJ, 2, 3, 3);
    /* J = [[fx/z, 0, -fx tx/z], [0, fy/z, -fy ty/z]], tx = clamp(x/z) */
    dpc[2] += dJ[0] * (-cam.fx / (z * z)) + dJ[4] * (-cam.fy / (z * z));
    if (!g.clampx) {
      dpc[0] += dJ[2] * (-cam.fx / (z * z));
      dpc[2] += dJ[2] * (2.0 * cam.fx * g.pc[0] / (z * z * z));
    } else {
      double lim = 1.3 * (0.5 * cam.width / cam.fx) * (g.pc[0] > 0 ? 1.0 : -1.0);
      dpc[2] += dJ[2] * (cam.fx * lim / (z * z));
    }
    if (!g.clampy) {
      dpc[1] += dJ[5] * (-cam.fy / (z * z));
      dpc[2] += dJ[5] * (2.0 * cam.fy * g.pc[1] / (z * z * z));
    } else {
      double lim = 1.3 * (0.5 * cam.height / cam.fy) * (g.pc[1] > 0 ? 1.0 : -1.0);
      dpc[2] += dJ[5] * (cam.fy * lim / (z * z));
    }
    /* pc = W mu + t */
    for (int a = 0; a < 3; ++a)
      dmu[a] += cam.W[0 * 3 + a] * dpc[0] + cam.W[1 * 3 + a] * dpc[1] + cam.W[2 * 3 + a] * dpc[2];
    out[0] = dmu[0]; out[1] = dmu[1]; out[2] = dmu[2];
    /* Sigma = M M^T, M = R diag(s) */
    double M[9], dM[9];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) M[r * 3 + c] = g.R[r * 3 + c] * g.s[c];
    matmul(dSigma, M, dM, 3, 3, 3);
    for (int k = 0; k < 9; ++k) dM[k] *= 2.0;
    double dR[9];
    for (int c = 0; c < 3; ++c) {
      double ds = 0.0;
      for (int r = 0; r < 3; ++r) ds += g.R[r * 3 + c] * dM[r * 3 + c];
      out[3 + c] = ds * g.s[c];
      for (int r = 0; r < 3; ++r) dR[r * 3 + c] = dM[r * 3 + c] * g.s[c];
    }
    /* rotation of the unit quaternion, then its normalisation */
    double w = g.q[0], x = g.q[1], y = g.q[2], zq = g.q[3];
    double dq[4];
    dq[0] = dR[1] * (-2 * zq) + dR[2] * (2 * y) + dR[3] * (2 * zq) + dR[5] * (-2 * x) + dR[6] * (-2 * y) + dR[7] * (2 * x);
    dq[1] = dR[1] * (2 * y) + dR[2] * (2 * zq) + dR[3] * (2 * y) + dR[4] * (-4 * x) + dR[5] * (-2 * w) + dR[6] * (2 * zq) + dR[7] * (2 * w) + dR[8] * (-4 * x);
    dq[2] = dR[0] * (-4 * y) + dR[1] * (2 * x) + dR[2] * (2 * w) + dR[3] * (2 * x) + dR[5] * (2 * zq) + dR[6] * (-2 * w) + dR[7] * (2 * zq) + dR[8] * (-4 * y);
    dq[3] = dR[0] * (-4 * zq) + dR[1] * (-2 * w) + dR[2] * (2 * x) + dR[3] * (2 * w) + dR[4] * (-4 * zq) + dR[5] * (2 * y) + dR[6] * (2 * x) + dR[7] * (2 * y);
    double qd = dq[0] * g.q[0] + dq[1] * g.q[1] + dq[2] * g.q[2] + dq[3] * g.q[3];
    for (int k = 0; k < 4; ++k) out[6 + k] = (dq[k] - g.q[k] * qd) / g.qnorm;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* sparse loss: Charbonnier L1 + tile-level sparse NCC (Sec. 3.7, App. A)   */
/* ------------------------------------------------------------------------ */

/*
 * For each active tile tau with its n sampled pixels (prediction x, target y,
 * per colour channel):
 *   l1(p) = sum_c sqrt((x - y)^2 + eps_c^2)
 *   NCC_c = cov_c / sqrt(var_x,c var_y,c + eps_n), population moments over the
 *           tile's sampled pixels; S-NCC_tau = 1 - mean_c NCC_c
 *   lambda_tau = clip(mean_p |grad l1(p)|_1 / (mean_p g_ncc(p) + 1e-8), 0, 1),
 *     g_ncc(p) = sum_c |n dNCC_c/dx_p,c| (per-pixel scale, no 1/n)
 *   L = (1/|P|) sum_p l1(p) + (1/A) sum_tau lambda_tau S-NCC_tau, lambda held fixed
 * Outputs dL/dI [P,3], lambda [A], e [P] = sum_c |x - y|, *loss; updates the
 * fp16 error map by E <- (1 - beta) E + beta e at sampled pixels and the age map
 * by +1 (saturating) everywhere, 0 at sampled pixels (Eqs. 3-4).
 * lambda_in (nullable) replaces the computed lambda (for finite differences).
 */
int orc_loss(int width, int height, int n_active, const int32_t* active_tiles, const int32_t* pix_off,
             const uint8_t* pix_idx, const double* rgb, const double* target, const double* lambda_in,
             double eps_c, double eps_n, double beta, uint16_t* err_map, uint16_t* age_map, double* dL_drgb,
             double* lambda_out, double* err_pix, double* loss_out) {
  int tx_n = (width + ORC_TILE - 1) / ORC_TILE;
  int64_t P = pix_off[n_active];
  double loss = 0.0;
  for (int j = 0; j < n_active; ++j) {
    int t = active_tiles[j];
    int tx = t % tx_n, ty = t / tx_n;
    int64_t s0 = pix_off[j], s1 = pix_off[j + 1];
    int nn = (int)(s1 - s0);
    if (nn <= 0) { lambda_out[j] = 0.0; continue; }
    double mx[3] = {0, 0, 0}, my[3] = {0, 0, 0};
    for (int64_t s = s0; s < s1; ++s) {
      int l = pix_idx[s];
      int x = tx * ORC_TILE + (l % ORC_TILE), y = ty * ORC_TILE + (l / ORC_TILE);
      for (int c = 0; c < 3; ++c) {
        mx[c] += rgb[3 * s + c];
        my[c] += target[((int64_t)y * width + x) * 3 + c];
      }
    }
    for (int c = 0; c < 3; ++c) { mx[c] /= nn; my[c] /= nn; }
    double vx[3] = {0, 0, 0}, vy[3] = {0, 0, 0}, cv[3] = {0, 0, 0};
    for (int64_t s = s0; s < s1; ++s) {
      int l = pix_idx[s];
      int x = tx * ORC_TILE + (l % ORC_TILE), y = ty * ORC_TILE + (l / ORC_TILE);
      for (int c = 0; c < 3; ++c) {
        double dx = rgb[3 * s + c] - mx[c], dy = target[((int64_t)y * width + x) * 3 + c] - my[c];
        vx[c] += dx * dx; vy[c] += dy * dy; cv[c] += dx * dy;
      }
    }
    double D[3], ncc[3];
    for (int c = 0; c < 3; ++c) {
      vx[c] /= nn; vy[c] /= nn; cv[c] /= nn;
      D[c] = sqrt(vx[c] * vy[c] + eps_n);
      ncc[c] = cv[c] / D[c];
    }
    /* per-pixel gradients of both terms */
    double sum_g1 = 0.0, sum_gn = 0.0;
    for (int64_t s = s0; s < s1; ++s) {
      int l = pix_idx[s];
      int x = tx * ORC_TILE + (l % ORC_TILE), y = ty * ORC_TILE + (l / ORC_TILE);
      for (int c = 0; c < 3; ++c) {
        double xv = rgb[3 * s + c], yv = target[((int64_t)y * width + x) * 3 + c];
        double d = xv - yv;
        sum_g1 += fabs(d / sqrt(d * d + eps_c * eps_c));
        /* n dNCC_c/dx = ((y - my) - NCC var_y (x - mx) / D) / D */
        double gn = ((yv - my[c]) - ncc[c] * vy[c] * (xv - mx[c]) / D[c]) / D[c];
        sum_gn += fabs(gn);
      }
    }
    double lam = (sum_g1 / nn) / (sum_gn / nn + 1e-8);
    lam = clampd(lam, 0.0, 1.0);
    if (lambda_in) lam = lambda_in[j];
    lambda_out[j] = lam;
    double sncc = 1.0 - (ncc[0] + ncc[1] + ncc[2]) / 3.0;
    loss += lam * sncc / n_active;
    for (int64_t s = s0; s < s1; ++s) {
      int l = pix_idx[s];
      int x = tx * ORC_TILE + (l % ORC_TILE), y = ty * ORC_TILE + (l / ORC_TILE);
      double e = 0.0;
      for (int c = 0; c < 3; ++c) {
        double xv = rgb[3 * s + c], yv = target[((int64_t)y * width + x) * 3 + c];
        double d = xv - yv;
        double r = sqrt(d * d + eps_c * eps_c);
        loss += r / (double)P;
        e += fabs(d);
        double dncc = ((yv - my[c]) - ncc[c] * vy[c] * (xv - mx[c]) / D[c]) / (D[c] * nn);
        dL_drgb[3 * s + c] = d / r / (double)P - lam / (3.0 * n_active) * dncc;
      }
      err_pix[s] = e;
    }
  }
  *loss_out = loss;
  /* age map: +1 everywhere (saturating), then 0 at sampled pixels */
  if (age_map) {
    for (int64_t k = 0; k < (int64_t)width * height; ++k)
      if (age_map[k] < 65535) age_map[k]++;
  }
  for (int j = 0; j < n_active; ++j) {
    int t = active_tiles[j];
    int tx = t % tx_n, ty = t / tx_n;
    for (int64_t s = pix_off[j]; s < pix_off[j + 1]; ++s) {
      int l = pix_idx[s];
      int64_t k = (int64_t)(ty * ORC_TILE + l / ORC_TILE) * width + tx * ORC_TILE + (l % ORC_TILE);
      if (err_map) {
        double old = orc_half_to_double(err_map[k]);
        err_map[k] = orc_double_to_half((1.0 - beta) * old + beta * err_pix[s]);
      }
      if (age_map) age_map[k] = 0;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* sparse loss with the SSIM structure term (Sec. 4, Table 4: S-SSIM)       */
/* ------------------------------------------------------------------------ */

/*
 * The ablation of Table 4 that replaces sparse NCC by sparse SSIM.  The paper
 * names the variant only; this is its reading: the structure term of each
 * active tile is SSIM (Wang et al. 2004, dynamic range 1: C1 = 0.01^2,
 * C2 = 0.03^2) computed per colour channel from population moments over the
 * tile's sampled pixels, as the sparse NCC is:
 *   SSIM_c = (2 mx my + C1)(2 cov + C2) / ((mx^2 + my^2 + C1)(var_x + var_y + C2))
 *   S-SSIM_tau = 1 - mean_c SSIM_c
 *   lambda_tau = clip(mean_p |grad l1(p)|_1 / (mean_p g_s(p) + 1e-8), 0, 1),
 *     g_s(p) = sum_c |n dSSIM_c/dx_p,c| (per-pixel scale, no 1/n, as for NCC)
 *   L = (1/|P|) sum_p l1(p) + (1/A) sum_tau lambda_tau S-SSIM_tau, lambda fixed.
 * With a1 = 2 mx my + C1, a2 = 2 cov + C2, b1 = mx^2 + my^2 + C1,
 * b2 = var_x + var_y + C2 and SSIM = a1 a2 / (b1 b2), the derivative for one
 * pixel's channel value x (dx = x - mx, dy = y - my) is
 *   n dSSIM/dx = 2 ((my a2 + a1 dy) / (b1 b2) - SSIM (mx / b1 + dx / b2)).
 * Everything else (Charbonnier L1, e, the error and age map updates, the
 * arguments and outputs) is as orc_loss.
 */
int orc_loss_ssim(int width, int height, int n_active, const int32_t* active_tiles, const int32_t* pix_off,
                  const uint8_t* pix_idx, const double* rgb, const double* target, const double* lambda_in,
                  double eps_c, double beta, uint16_t* err_map, uint16_t* age_map, double* dL_drgb,
                  double* lambda_out, double* err_pix, double* loss_out) {
  const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
  int tx_n = (width + ORC_TILE - 1) / ORC_TILE;
  int64_t P = pix_off[n_active];
  double loss = 0.0;
  for (int j = 0; j < n_active; ++j) {
    int t = active_tiles[j];
    int tx = t % tx_n, ty = t / tx_n;
    int64_t s0 = pix_off[j], s1 = pix_off[j + 1];
    int nn = (int)(s1 - s0);
    if (nn <= 0) { lambda_out[j] = 0.0; continue; }
    double mx[3] = {0, 0, 0}, my[3] = {0, 0, 0};
    for (int64_t s = s0; s < s1; ++s) {
      int l = pix_idx[s];
      int x = tx * ORC_TILE + (l % ORC_TILE), y = ty * ORC_TILE + (l / ORC_TILE);
      for (int c = 0; c < 3; ++c) {
        mx[c] += rgb[3 * s + c];
        my[c] += target[((int64_t)y * width + x) * 3 + c];
      }
    }
    for (int c = 0; c < 3; ++c) { mx[c] /= nn; my[c] /= nn; }
    double vx[3] = {0, 0, 0}, vy[3] = {0, 0, 0}, cv[3] = {0, 0, 0};
    for (int64_t s = s0; s < s1; ++s) {
      int l = pix_idx[s];
      int x = tx * ORC_TILE + (l % ORC_TILE), y = ty * ORC_TILE + (l / ORC_TILE);
      for (int c = 0; c < 3; ++c) {
        double dx = rgb[3 * s + c] - mx[c], dy = target[((int64_t)y * width + x) * 3 + c] - my[c];
        vx[c] += dx * dx; vy[c] += dy * dy; cv[c] += dx * dy;
      }
    }
    double a1[3], a2[3], b1[3], b2[3], ss[3];
    for (int c = 0; c < 3; ++c) {
      vx[c] /= nn; vy[c] /= nn; cv[c] /= nn;
      a1[c] = 2.0 * mx[c] * my[c] + C1;
      a2[c] = 2.0 * cv[c] + C2;
      b1[c] = mx[c] * mx[c] + my[c] * my[c] + C1;
      b2[c] = vx[c] + vy[c] + C2;
      ss[c] = a1[c] * a2[c] / (b1[c] * b2[c]);
    }
    double sum_g1 = 0.0, sum_gs = 0.0;
    for (int64_t s = s0; s < s1; ++s) {
      int l = pix_idx[s];
      int x = tx * ORC_TILE + (l % ORC_TILE), y = ty * ORC_TILE + (l / ORC_TILE);
      for (int c = 0; c < 3; ++c) {
        double xv = rgb[3 * s + c], yv = target[((int64_t)y * width + x) * 3 + c];
        double d = xv - yv;
        sum_g1 += fabs(d / sqrt(d * d + eps_c * eps_c));
        double gsn = 2.0 * ((my[c] * a2[c] + a1[c] * (yv - my[c])) / (b1[c] * b2[c]) -
                            ss[c] * (mx[c] / b1[c] + (xv - mx[c]) / b2[c]));
        sum_gs += fabs(gsn);
      }
    }
    double lam = (sum_g1 / nn) / (sum_gs / nn + 1e-8);
    lam = clampd(lam, 0.0, 1.0);
    if (lambda_in) lam = lambda_in[j];
    lambda_out[j] = lam;
    loss += lam * (1.0 - (ss[0] + ss[1] + ss[2]) / 3.0) / n_active;
    for (int64_t s = s0; s < s1; ++s) {
      int l = pix_idx[s];
      int x = tx * ORC_TILE + (l % ORC_TILE), y = ty * ORC_TILE + (l / ORC_TILE);
      double e = 0.0;
      for (int c = 0; c < 3; ++c) {
        double xv = rgb[3 * s + c], yv = target[((int64_t)y * width + x) * 3 + c];
        double d = xv - yv;
        double r = sqrt(d * d + eps_c * eps_c);
        loss += r / (double)P;
        e += fabs(d);
        double dss = 2.0 * ((my[c] * a2[c] + a1[c] * (yv - my[c])) / (b1[c] * b2[c]) -
                            ss[c] * (mx[c] / b1[c] + (xv - mx[c]) / b2[c])) / nn;
        dL_drgb[3 * s + c] = d / r / (double)P - lam / (3.0 * n_active) * dss;
      }
      err_pix[s] = e;
    }
  }
  *loss_out = loss;
  if (age_map) {
    for (int64_t k = 0; k < (int64_t)width * height; ++k)
      if (age_map[k] < 65535) age_map[k]++;
  }
  for (int j = 0; j < n_active; ++j) {
    int t = active_tiles[j];
    int tx = t % tx_n, ty = t / tx_n;
    for (int64_t s = pix_off[j]; s < pix_off[j + 1]; ++s) {
      int l = pix_idx[s];
      int64_t k = (int64_t)(ty * ORC_TILE + l / ORC_TILE) * width + tx * ORC_TILE + (l % ORC_TILE);
      if (err_map) {
        double old = orc_half_to_double(err_map[k]);
        err_map[k] = orc_double_to_half((1.0 - beta) * old + beta * err_pix[s]);
      }
      if (age_map) age_map[k] = 0;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* hybrid solver: moment-damped LM blocks + Adam (Sec. 3.9, App. A)         */
/* ------------------------------------------------------------------------ */

/* Cholesky factorisation A = L L^T (row-major d x d) and solve A x = b: the
 * block solve of the LM step (Sec. 3.9, Eq. 14). */
static int cholesky_solve(const double* A, const double* b, double* x, int d) {
  double L[196];
  memset(L, 0, sizeof(L));
  for (int i = 0; i < d; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = A[i * d + j];
      for (int k = 0; k < j; ++k) s -= L[i * d + k] * L[j * d + k];
      if (i == j) {
        if (!(s > 0.0)) return -1;
        L[i * d + i] = sqrt(s);
      } else L[i * d + j] = s / L[j * d + j];
    }
  double y[14];
  for (int i = 0; i < d; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[i * d + k] * y[k];
    y[i] = s / L[i * d + i];
  }
  for (int i = d - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < d; ++k) s -= L[k * d + i] * x[k];
    x[i] = s / L[i * d + i];
  }
  return 0;
}

int orc_cholesky_solve(const double* A, const double* b, double* x, int d) {
  return d > 14 ? -2 : cholesky_solve(A, b, x, d);
}

/*
 * One step for the Gaussians with touched[i] != 0.  Packed parameter rows of
 * 59: (means 3, log_scales 3, quats 4, opacity logit 1, sh 48 with the DC
 * colour at 11..13).  cfg = [lr_means, lr_scales, lr_quats, lr_opacity,
 * lr_sh_dc, lr_sh_rest, beta1, beta2, eps_adam, eps_lm].
 * m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2 for all 59.
 * mode 0: Adam with bias correction on all 59.
 * mode 1: geometry block (0..9) and appearance block (11,12,13,10) solve
 *         (diag(sum_k J_k^2) + diag(sqrt(v) + eps_lm)) D = -m;
 * mode 2: the same with J^T J in full, solved by Cholesky.
 * J rows: rows [K, N, 14] (geometry 10 then appearance 4 in the block order
 * above), or, when rows is NULL, the single row g.  theta += lr * D; the 45
 * higher SH coefficients always take the Adam step -lr m_hat / (sqrt(v_hat) + eps).
 */
int orc_hybrid_step(int64_t n, double* params, const double* grads, double* m, double* v,
                    const uint8_t* touched, const double* rows, int k_rows, int step, int mode,
                    const double* cfg) {
  double b1 = cfg[6], b2 = cfg[7], eps = cfg[8], eps_lm = cfg[9];
  double bc1 = 1.0 - pow(b1, step), bc2 = 1.0 - pow(b2, step);
  static const int geo[10] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9};
  static const int app[4] = {11, 12, 13, 10};
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    if (touched && !touched[i]) continue;
    double* p = params + 59 * i;
    const double* g = grads + 59 * i;
    double* mi = m + 59 * i;
    double* vi = v + 59 * i;
    for (int k = 0; k < 59; ++k) {
      mi[k] = b1 * mi[k] + (1.0 - b1) * g[k];
      vi[k] = b2 * vi[k] + (1.0 - b2) * g[k] * g[k];
    }
    double lr[59];
    for (int k = 0; k < 59; ++k) {
      int grp = k < 3 ? 0 : k < 6 ? 1 : k < 10 ? 2 : k == 10 ? 3 : k < 14 ? 4 : 5;
      lr[k] = cfg[grp];
    }
    if (mode == 0) {
      for (int k = 0; k < 59; ++k) p[k] -= lr[k] * (mi[k] / bc1) / (sqrt(vi[k] / bc2) + eps);
      continue;
    }
    for (int blk = 0; blk < 2; ++blk) {
      const int* ix = blk == 0 ? geo : app;
      int d = blk == 0 ? 10 : 4;
      int off = blk == 0 ? 0 : 10;
      double A[100], rhs[10], D[10];
      memset(A, 0, sizeof(A));
      int K = rows ? k_rows : 1;
      for (int r = 0; r < K; ++r) {
        double J[10];
        for (int a = 0; a < d; ++a)
          J[a] = rows ? rows[((int64_t)r * n + i) * 14 + off + a] : g[ix[a]];
        for (int a = 0; a < d; ++a)
          for (int b = 0; b < d; ++b)
            if (mode == 2 || a == b) A[a * d + b] += J[a] * J[b];
      }
      for (int a = 0; a < d; ++a) {
        A[a * d + a] += sqrt(vi[ix[a]]) + eps_lm;
        rhs[a] = -mi[ix[a]];
      }
      cholesky_solve(A, rhs, D, d);
      for (int a = 0; a < d; ++a) p[ix[a]] += lr[ix[a]] * D[a];
    }
    for (int k = 14; k < 59; ++k) p[k] -= lr[k] * (mi[k] / bc1) / (sqrt(vi[k] / bc2) + eps);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* tile-error predictor: 3-layer MLP 16 -> 128 -> 128 -> 1, ReLU            */
/* (not in the paper; a learned stand-in for refreshing stale error maps)   */
/* ------------------------------------------------------------------------ */

/* IEEE binary32 -> bfloat16 with round to nearest even, returned as a
 * double (bfloat16 is the upper half of a binary32). */
double orc_round_bf16(double x) {
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (double)f;  /* inf / nan */
  uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  u &= 0xffff0000u;
  memcpy(&f, &u, 4);
  return (double)f;
}

#define MLP_IN 16
#define MLP_H 128

/*
 * Forward of rows x [R,16] (features, zero padded).  Weights W1 [128,16],
 * W2 [128,128], W3 [128] (out x in, row-major) and biases b1, b2, b3 [1].
 * bf16 = 1 rounds the input, the weights and the hidden activations to
 * bfloat16 where the kernels do (products summed exactly in double here,
 * in fp32 there); bf16 = 0 is the plain double-precision network.
 * Outputs y [R]; h1, h2 [R,128] post-ReLU activations (nullable).
 */
int orc_mlp_forward(int64_t R, const double* x, const double* W1, const double* b1, const double* W2,
                    const double* b2, const double* W3, const double* b3, int bf16, double* y, double* h1o,
                    double* h2o) {
#pragma omp parallel for schedule(static) if (R > 64)
  for (int64_t r = 0; r < R; ++r) {
    double xin[MLP_IN], h1[MLP_H], h2[MLP_H];
    for (int k = 0; k < MLP_IN; ++k) xin[k] = bf16 ? orc_round_bf16(x[r * MLP_IN + k]) : x[r * MLP_IN + k];
    for (int j = 0; j < MLP_H; ++j) {
      double s = b1[j];
      for (int k = 0; k < MLP_IN; ++k) s += (bf16 ? orc_round_bf16(W1[j * MLP_IN + k]) : W1[j * MLP_IN + k]) * xin[k];
      s = s > 0.0 ? s : 0.0;
      h1[j] = bf16 ? orc_round_bf16(s) : s;
    }
    for (int j = 0; j < MLP_H; ++j) {
      double s = b2[j];
      for (int k = 0; k < MLP_H; ++k) s += (bf16 ? orc_round_bf16(W2[j * MLP_H + k]) : W2[j * MLP_H + k]) * h1[k];
      s = s > 0.0 ? s : 0.0;
      h2[j] = bf16 ? orc_round_bf16(s) : s;
    }
    double s = b3[0];
    for (int k = 0; k < MLP_H; ++k) s += (bf16 ? orc_round_bf16(W3[k]) : W3[k]) * h2[k];
    y[r] = s;
    if (h1o) for (int j = 0; j < MLP_H; ++j) h1o[r * MLP_H + j] = h1[j];
    if (h2o) for (int j = 0; j < MLP_H; ++j) h2o[r * MLP_H + j] = h2[j];
  }
  return 0;
}

/*
 * Loss L = (1/R) sum_r (y_r - t_r)^2 / 2 and its gradient with respect to
 * every weight and bias, by the chain rule through the forward above.
 * With bf16 = 1 the backward rounds the hidden adjoints to bfloat16 before
 * they meet a bfloat16 operand, as the kernels do.  Gradients are written
 * (not accumulated) into dW1 [128,16], db1, dW2 [128,128], db2, dW3 [128], db3.
 */
int orc_mlp_backward(int64_t R, const double* x, const double* t, const double* W1, const double* b1,
                     const double* W2, const double* b2, const double* W3, const double* b3, int bf16,
                     double* loss, double* dW1, double* db1, double* dW2, double* db2, double* dW3, double* db3) {
  memset(dW1, 0, sizeof(double) * MLP_H * MLP_IN);
  memset(db1, 0, sizeof(double) * MLP_H);
  memset(dW2, 0, sizeof(double) * MLP_H * MLP_H);
  memset(db2, 0, sizeof(double) * MLP_H);
  memset(dW3, 0, sizeof(double) * MLP_H);
  db3[0] = 0.0;
  double L = 0.0;
  double* h1 = (double*)malloc(sizeof(double) * MLP_H);
  double* h2 = (double*)malloc(sizeof(double) * MLP_H);
  for (int64_t r = 0; r < R; ++r) {
    double xin[MLP_IN], y;
    for (int k = 0; k < MLP_IN; ++k) xin[k] = bf16 ? orc_round_bf16(x[r * MLP_IN + k]) : x[r * MLP_IN + k];
    orc_mlp_forward(1, x + r * MLP_IN, W1, b1, W2, b2, W3, b3, bf16, &y, h1, h2);
    double e = y - t[r];
    L += 0.5 * e * e / (double)R;
    double dy = e / (double)R;
    db3[0] += dy;
    double dh2[MLP_H], dh1[MLP_H];
    for (int k = 0; k < MLP_H; ++k) {
      dW3[k] += dy * h2[k];
      double w3 = bf16 ? orc_round_bf16(W3[k]) : W3[k];
      double d = h2[k] > 0.0 ? dy * w3 : 0.0;   /* ReLU gate */
      dh2[k] = bf16 ? orc_round_bf16(d) : d;
    }
    for (int j = 0; j < MLP_H; ++j) {
      db2[j] += dh2[j];
      for (int k = 0; k < MLP_H; ++k) dW2[j * MLP_H + k] += dh2[j] * h1[k];
    }
    for (int k = 0; k < MLP_H; ++k) {
      double s = 0.0;
      for (int j = 0; j < MLP_H; ++j) s += dh2[j] * (bf16 ? orc_round_bf16(W2[j * MLP_H + k]) : W2[j * MLP_H + k]);
      double d = h1[k] > 0.0 ? s : 0.0;
      dh1[k] = bf16 ? orc_round_bf16(d) : d;
    }
    for (int j = 0; j < MLP_H; ++j) {
      db1[j] += dh1[j];
      for (int k = 0; k < MLP_IN; ++k) dW1[j * MLP_IN + k] += dh1[j] * xin[k];
    }
  }
  free(h1);
  free(h2);
  *loss = L;
  return 0;
}

/* ------------------------------------------------------------------------
 * Tile memory, features and error-map refresh of the tile-error predictor
 * (not in the paper; it refreshes a stale view's error map by rendering it,
 * Sec. 3.3).  Written from their definitions.
 * ---------------------------------------------------------------------- */

/* For each active rank j < n_active: tile t = active_tiles[j] records
 * (list length, mean T_final, mean err_pix over its sampled pixels, 1) and
 * the iteration; target[j] = log(1 + mean err_pix), less the same of the
 * tile's previous observation when residual and there was one. */
void orc_tile_observe(int n_active, const int32_t* active_tiles, const int32_t* pix_off, const int32_t* ranges,
                      const double* T_final, const double* err_pix, int64_t iter, double* mem, int64_t* mem_iter,
                      double* target, int residual) {
  for (int j = 0; j < n_active; ++j) {
    int p0 = pix_off[j], p1 = pix_off[j + 1], n = p1 - p0 > 0 ? p1 - p0 : 1;
    double st = 0.0, se = 0.0;
    for (int p = p0; p < p1; ++p) {
      st += T_final[p];
      se += err_pix[p];
    }
    int t = active_tiles[j];
    double prev = (residual && mem[4 * t + 3] > 0.0) ? log1p(mem[4 * t + 2]) : 0.0;
    mem[4 * t + 0] = (double)(ranges[2 * j + 1] - ranges[2 * j]);
    mem[4 * t + 1] = st / n;
    mem[4 * t + 2] = se / n;
    mem[4 * t + 3] = 1.0;
    mem_iter[t] = iter;
    if (target) target[j] = log1p(se / n) - prev;
  }
}

/* Features of tile t: the angle between the optical axis and the ray through
 * the tile centre (u, v) from the pinhole (fx, fy, cx, cy) enters as its
 * cosine. */
void orc_tile_features(int n_rows, const int32_t* rows, const double* mem, const int64_t* mem_iter, int width,
                       double fx, double fy, double cx, double cy, double view_cos, int64_t iter, double* x) {
  int tx = (width + 15) / 16;
  for (int r = 0; r < n_rows; ++r) {
    int t = rows ? rows[r] : r;
    double* f = x + 16 * (size_t)r;
    for (int k = 0; k < 16; ++k) f[k] = 0.0;
    int seen = mem[4 * t + 3] > 0.0;
    double age = seen ? (double)(iter - mem_iter[t] > 0 ? iter - mem_iter[t] : 0) : 1e6;
    double u = ((t % tx) * 16 + 8 - cx) / fx, v = ((t / tx) * 16 + 8 - cy) / fy;
    f[0] = log1p(mem[4 * t + 0]);
    f[1] = seen ? mem[4 * t + 1] : 1.0;
    f[2] = log1p(mem[4 * t + 2]);
    f[3] = view_cos;
    f[4] = log1p(age);
    f[5] = cos(atan(sqrt(u * u + v * v)));
    f[6] = seen ? 1.0 : 0.0;
  }
}

/* Each tile's fp16 error values scaled so their mean is exp(p) - 1,
 * p = pred (+ the tile's feature 2 from base, when predictions are residuals),
 * clamped at 0 below; a tile of mean 0 takes the prediction
 * everywhere.  Values are rounded to fp16 (nearest even). */
void orc_tile_refresh(const double* pred, const double* base, uint16_t* err, int width, int height) {
  int tx = (width + 15) / 16, ty = (height + 15) / 16;
  for (int t = 0; t < tx * ty; ++t) {
    int x0 = (t % tx) * 16, y0 = (t / tx) * 16;
    double s = 0.0;
    int n = 0;
    for (int y = y0; y < y0 + 16 && y < height; ++y)
      for (int x = x0; x < x0 + 16 && x < width; ++x) {
        s += orc_half_to_double(err[(size_t)y * width + x]);
        ++n;
      }
    double mean = s / (n > 0 ? n : 1);
    double p = pred[t] + (base ? base[16 * (size_t)t + 2] : 0.0);
    double want = expm1(p > 0.0 ? p : 0.0);
    for (int y = y0; y < y0 + 16 && y < height; ++y)
      for (int x = x0; x < x0 + 16 && x < width; ++x) {
        size_t k = (size_t)y * width + x;
        double e = orc_half_to_double(err[k]);
        err[k] = orc_double_to_half(mean > 0.0 ? e * (want / mean) : want);
      }
  }
}

/* ------------------------------------------------------------------------ */
/* geometry-aware view sampling (Sec. 3.4, Eqs. 5-6; Alg. 1 step 2)         */
/* ------------------------------------------------------------------------ */

/* Eq. 5 before the division: the sum of E_v over the view's W H pixels, as
 * the exact integer sum of E * 2^24 (the weight of the tile draw, so
 * negative, NaN and infinite values count as 0).  The mean view error is
 * sums[v] / 2^24 / (W H). */
void orc_view_error_sums(const uint16_t* maps, int n_views, int64_t view_stride, int width, int height,
                         uint64_t* sums) {
  int64_t n = (int64_t)width * height;
  for (int v = 0; v < n_views; ++v) {
    uint64_t s = 0;
    for (int64_t p = 0; p < n; ++p) s += orc_err_weight(maps[(int64_t)v * view_stride + p]);
    sums[v] = s;
  }
}

/* log2(x) * 2^32 for x >= 1, by the digit recurrence of orc_neglog2_q32:
 * the integer part is the position of the leading bit, each squaring of the
 * mantissa normalised to [1, 2) gives one fractional bit.  It turns the view
 * draw's exponential clocks into logarithms, so that the weights of Sec. 3.4
 * Eq. 6 enter the keys as sums. */
uint64_t orc_log2_q32(uint64_t x) {
  int ip = 63;
  while (!(x >> ip)) ip--;
  uint64_t m = x << (63 - ip);
  uint64_t frac = 0;
  for (int i = 0; i < 32; ++i) {
    unsigned __int128 sq = (unsigned __int128)m * m;
    uint64_t hi = (uint64_t)(sq >> 64);
    frac <<= 1;
    if (hi >> 63) { frac |= 1; m = hi; }
    else m = hi << 1;
  }
  return ((uint64_t)ip << 32) | frac;
}

/* Camera centre c = -R^T t and unit viewing direction (the camera's forward
 * axis, the third row of R) of a row-major world-to-camera matrix whose
 * camera looks along +z: the c_u and d_u of Sec. 3.4 Eq. 6. */
void orc_view_pose(const float* viewmat, double* c, double* d) {
  const float* M = viewmat;
  for (int j = 0; j < 3; ++j) {
    double s = (double)M[j] * (double)M[3];
    s = s + (double)M[4 + j] * (double)M[7];
    s = s + (double)M[8 + j] * (double)M[11];
    c[j] = -s;
  }
  double f0 = M[8], f1 = M[9], f2 = M[10];
  double n = sqrt((f0 * f0 + f1 * f1) + f2 * f2);
  d[0] = f0 / n;
  d[1] = f1 / n;
  d[2] = f2 / n;
}

typedef struct {
  int idx;
  double key;
} vkey_t;

static int cmp_vkey(const void* a, const void* b) {
  const vkey_t* x = (const vkey_t*)a;
  const vkey_t* y = (const vkey_t*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->idx - y->idx;
}

#define ORC_STREAM_VIEW 5

/*
 * K views for iteration `iter`, drawn from the view stack (stack[v] = 1 while
 * view v is on it; updated in place):
 *   - when fewer than K views are on the stack, all views go back on it;
 *   - the anchor v* is the stack view with the largest mean error (Eq. 5;
 *     equal means: the lower index);
 *   - the remaining K - 1 are drawn without replacement from the other stack
 *     views, each draw with probability proportional to
 *     pi(u) = exp(-lambda_d |c_u - c_v*| - lambda_theta (1 - <d_u, d_v*>))
 *     (Eq. 6).  Successive weighted draws are realised as the Efraimidis-
 *     Spirakis order: with the exponential clock L_u = -log2 U_u of the
 *     view's hash (stream 5), the draws are the K - 1 smallest L_u / pi(u),
 *     compared through their base-2 logarithms
 *       log2 L_u + log2(e) (lambda_d |c_u - c_v*| + lambda_theta (1 - <d_u, d_v*>)),
 *     log2 L_u from the digit recurrence above (equal keys: the lower index);
 *   - the K views leave the stack.
 * views [K]: the anchor, then the draws in ascending view order.
 */
void orc_sample_views(const uint64_t* sums, const float* viewmats, int n_views, int k, double lambda_d,
                      double lambda_theta, uint64_t seed, uint64_t iter, uint8_t* stack, int32_t* views) {
  int on_stack = 0;
  for (int v = 0; v < n_views; ++v) on_stack += stack[v] != 0;
  if (on_stack < k)
    for (int v = 0; v < n_views; ++v) stack[v] = 1;
  int anchor = -1;
  for (int v = 0; v < n_views; ++v)
    if (stack[v] && (anchor < 0 || sums[v] > sums[anchor])) anchor = v;
  double ca[3], da[3];
  orc_view_pose(viewmats + 16 * (size_t)anchor, ca, da);
  vkey_t* cand = (vkey_t*)malloc(sizeof(vkey_t) * (size_t)n_views);
  int m = 0;
  for (int u = 0; u < n_views; ++u) {
    if (!stack[u] || u == anchor) continue;
    double c[3], d[3];
    orc_view_pose(viewmats + 16 * (size_t)u, c, d);
    double dx = c[0] - ca[0], dy = c[1] - ca[1], dz = c[2] - ca[2];
    double dist = sqrt((dx * dx + dy * dy) + dz * dz);
    double cosv = (d[0] * da[0] + d[1] * da[1]) + d[2] * da[2];
    double s = lambda_d * dist + lambda_theta * (1.0 - cosv);
    uint64_t L = orc_neglog2_q32(orc_hash(seed, iter, 0, ORC_STREAM_VIEW, (uint32_t)u, 0));
    double lg = (double)(int64_t)(orc_log2_q32(L) - (32ULL << 32)) * 2.3283064365386963e-10; /* 2^-32 */
    cand[m].idx = u;
    cand[m].key = (lg + s * 1.4426950408889634) + 0.0; /* log2(e) */
    m++;
  }
  qsort(cand, (size_t)m, sizeof(vkey_t), cmp_vkey);
  uint8_t* drawn = (uint8_t*)calloc((size_t)n_views, 1);
  for (int i = 0; i < k - 1; ++i) drawn[cand[i].idx] = 1;
  views[0] = anchor;
  int o = 1;
  for (int u = 0; u < n_views; ++u)
    if (drawn[u]) views[o++] = u;
  for (int u = 0; u < n_views; ++u)
    if (drawn[u] || u == anchor) stack[u] = 0;
  free(drawn);
  free(cand);
}

/* ------------------------------------------------------------------------ */
/* Gaussian difficulty scores of error-driven density control               */
/* ------------------------------------------------------------------------ */

/*
 * Sec. 3.8, Eq. 13, from the statistics of Eq. 12 (rows of `stride` doubles
 * holding E_i, W_i, D_i first, as orc_error_stats writes them):
 *   e_i = E_i / (W_i + eps), d_i = D_i / (W_i + eps),
 *   s_i = e_i + lambda_eff d_i, lambda_eff = lambda_base (1 - rho),
 * with rho the training progress.  Eq. 13 states rho in [0, 1); Alg. 1 computes
 * it as min(1, t / tau_until), which reaches 1 from t = tau_until on.  Taking
 * Alg. 1's formula there (so that lambda_eff = 0 once densification ends) is
 * a reading of the two passages; the caller passes rho.
 * Dividing by the visibility W_i removes the bias towards often-seen
 * Gaussians.  e_out and s_out are [n].
 */
void orc_gaussian_scores(int64_t n, const double* stats, int stride, double lambda_base, double rho, double eps,
                         double* e_out, double* s_out) {
  double lambda_eff = lambda_base * (1.0 - rho);
  for (int64_t i = 0; i < n; ++i) {
    const double* r = stats + (int64_t)stride * i;
    double e = r[0] / (r[1] + eps);
    double d = r[2] / (r[1] + eps);
    e_out[i] = e;
    s_out[i] = e + lambda_eff * d;
  }
}

/* ------------------------------------------------------------------------ */
/* error-driven densification and pruning (Sec. 3.8; Alg. 1 step 11)        */
/* ------------------------------------------------------------------------ */

/*
 * The screen-space gradient statistic that selects densification candidates
 * (Alg. 1 step 11 passes the screen-space gradients; Table 6's tau_grad):
 * for every Gaussian with a non-zero compositing adjoint in a view,
 * accum[i] += (|(dL/dx, dL/dy)|, 1), from grad2d rows [N,12] of that view.
 * Single precision, as the library's kernel (sqrtf of x^2 + y^2, one add).
 */
void orc_accumulate_screen_grad(int64_t n, const float* grad2d, float* accum) {
  for (int64_t i = 0; i < n; ++i) {
    const float* g = grad2d + 12 * i;
    int any = 0;
    for (int k = 0; k < 9; ++k) any |= g[k] != 0.0f;
    if (!any) continue;
    float xx = g[0] * g[0];
    float yy = g[1] * g[1];
    accum[2 * i] = accum[2 * i] + sqrtf(xx + yy);
    accum[2 * i + 1] = accum[2 * i + 1] + 1.0f;
  }
}

typedef struct {
  float s;
  int64_t i;
} dens_t;

static int cmp_dens(const void* a, const void* b) {  /* descending score, ties by index */
  const dens_t* x = (const dens_t*)a;
  const dens_t* y = (const dens_t*)b;
  if (x->s != y->s) return x->s > y->s ? -1 : 1;
  return x->i < y->i ? -1 : (x->i > y->i);
}

/*
 * One step of error-driven density control (Sec. 3.8, Eq. 13; Alg. 1 step
 * 11; Table 6).  The paper fixes the scores and says that percentile
 * thresholds of them drive densification and pruning; the procedure is this
 * reading of it.  Every decision is taken in single precision, in the order
 * written here (the kernel takes the same decisions):
 *   e_i = E_i / (W_i + eps), d_i = D_i / (W_i + eps), s_i = e_i + lam_eff d_i
 *   (Eq. 13; lam_eff = lambda_base (1 - rho) is computed by the caller);
 *   g_i = G_i / max(1, c_i), the mean screen-space gradient norm (accum);
 *   candidate: W_i > 0 and g_i >= tau_grad, and not pruned;
 *   densified: the floor(n_cand topk_pm / 1000) candidates with the largest
 *   s_i (ties: lower index);
 *   a densified Gaussian whose largest log-scale is at most log_split is
 *   cloned (kept, plus an identical copy after it), otherwise split: two
 *   children at mu +- sigma_k R e_k (k the axis of the largest scale, ties to
 *   the lower axis; one standard deviation along it), log-scales lowered by
 *   ln 1.6, the rest copied;
 *   pruned: opacity logit < logit_prune; with final = 1 (the final pruning of
 *   Table 6) also every Gaussian outside the floor(n final_pm / 1000) with the
 *   largest W_i (ties: lower index), and nothing is densified.
 * params: packed rows [N,59] float (means 3, log-scales 3, quaternion 4,
 * opacity logit 1, SH 48); stats [N,4] (E, W, D, -); accum [N,2].
 * Output in input order, each surviving Gaussian in place (a clone's copy and
 * a split's second child right after it): out [cap,59] double, src [cap] the
 * input index, kind [cap] 0 kept, 1 clone copy, 2 split child +, 3 split
 * child -.  Returns the output count (cap must hold it).
 */
int64_t orc_density_control(int64_t n, const float* params, const float* stats, const float* accum, float lam_eff,
                            float eps, float tau_grad, float log_split, float logit_prune, int topk_pm, int final,
                            int final_pm, int64_t cap, double* out, int64_t* src, int32_t* kind) {
  uint8_t* prune = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  uint8_t* dens = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  dens_t* list = (dens_t*)malloc(sizeof(dens_t) * (size_t)(n > 0 ? n : 1));
  int64_t nc = 0;
  for (int64_t i = 0; i < n; ++i) {
    const float* p = params + 59 * i;
    prune[i] = p[10] < logit_prune;
    const float* r = stats + 4 * i;
    float W = r[1];
    float e = r[0] / (W + eps);
    float d = r[2] / (W + eps);
    float s = e + lam_eff * d;
    float c = accum[2 * i + 1];
    float g = accum[2 * i] / (c > 1.0f ? c : 1.0f);
    if (!final && !prune[i] && W > 0.0f && g >= tau_grad) {
      list[nc].s = s;
      list[nc].i = i;
      ++nc;
    }
  }
  if (!final) {
    qsort(list, (size_t)nc, sizeof(dens_t), cmp_dens);
    int64_t k = nc * topk_pm / 1000;
    for (int64_t q = 0; q < k; ++q) dens[list[q].i] = 1;
  } else {
    for (int64_t i = 0; i < n; ++i) {
      list[i].s = stats[4 * i + 1];
      list[i].i = i;
    }
    qsort(list, (size_t)n, sizeof(dens_t), cmp_dens);
    int64_t keep = n * final_pm / 1000;
    for (int64_t q = keep; q < n; ++q) prune[list[q].i] = 1;
  }
  int64_t m = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (prune[i]) continue;
    const float* p = params + 59 * i;
    int ax = 0;
    for (int a = 1; a < 3; ++a)
      if (p[3 + a] > p[3 + ax]) ax = a;
    int split = dens[i] && p[3 + ax] > log_split;
    int copies = dens[i] ? 2 : 1;
    if (m + copies > cap) { m += copies; continue; }
    for (int q = 0; q < copies; ++q) {
      double* o = out + 59 * (m + q);
      for (int k = 0; k < 59; ++k) o[k] = p[k];
      src[m + q] = i;
      kind[m + q] = dens[i] ? (split ? 2 + q : q) : 0;
    }
    if (split) {
      double qn[4], R[9];
      double nq = sqrt((double)p[6] * p[6] + (double)p[7] * p[7] + (double)p[8] * p[8] + (double)p[9] * p[9]);
      for (int k = 0; k < 4; ++k) qn[k] = p[6 + k] / nq;
      quat_to_rot(qn, R);
      double sig = exp((double)p[3 + ax]);
      for (int q = 0; q < 2; ++q) {
        double* o = out + 59 * (m + q);
        double sgn = q == 0 ? 1.0 : -1.0;
        for (int a = 0; a < 3; ++a) o[a] = p[a] + sgn * sig * R[3 * a + ax];
        for (int a = 0; a < 3; ++a) o[3 + a] = p[3 + a] - log(1.6);
      }
    }
    m += copies;
  }
  free(prune);
  free(dens);
  free(list);
  return m;
}
