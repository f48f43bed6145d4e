/*
 * gs_oracle.c -- plain FP64 CPU oracle of the differentiable tile rasterizer.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file's library.  It shares no code, header or
 * constant table with the CUDA path.
 *
 * What it computes (the paper trains 3D Gaussian Splatting primitives on
 * isosurface point clouds against orbit views, Section III; the rasterizer's
 * mathematics is the 3D-GS / EWA splatting formulation the paper builds on,
 * Section I.  The constants 0.99 (alpha clamp), 1/255 (alpha skip) and 1e-4
 * (transmittance stop) fix the compositing rule):
 *
 *  project   t = W mu + tau; drop if t_z <= znear.  Sigma = R(q/|q|) S S^T R^T,
 *            S = diag(exp(s)).  J at t with the image-plane slopes t_x/t_z,
 *            t_y/t_z clamped to +-1.3 * (W/(2 fx)), +-1.3 * (H/(2 fy)).
 *            Sigma' = J W3 Sigma W3^T J^T + 0.3 I.  conic = Sigma'^-1 =
 *            (A, B, C) with power = -1/2 (A dx^2 + C dy^2) - B dx dy.
 *            lambda = m + sqrt(max(0.1, m^2 - det)), m = trace/2,
 *            r = ceil(3 sqrt(lambda)).  mu2D = (fx t_x/t_z + cx, fy t_y/t_z + cy).
 *            Tile rect x in [clamp(floor((mu_x - r)/16)), clamp(floor((mu_x + r + 15)/16)))
 *            and likewise in y.  sigma(o) = 1/(1+exp(-o)).
 *            rgb_c = max(0, sum_k sh_kc Y_k(d) + 0.5), d = (mu - campos)/|.|,
 *            Y_k the real orthonormal spherical harmonics (no Condon-Shortley
 *            phase: Y_1 = sqrt(3/4pi) (y, z, x)).
 *  render    pixel p (integer coordinates) of tile tau composites, in order of
 *            increasing depth t_z (ties: increasing Gaussian index), exactly the
 *            Gaussians whose rect contains tau (depth: the FP32 value of t_z
 *            in a fixed evaluation order, see depth32): alpha = min(0.99, sigma e^power);
 *            skip if power > 0 or alpha < 1/255; T' = T (1 - alpha); stop
 *            (excluding this Gaussian) if T' < 1e-4; C += rgb alpha T; T = T'.
 *            Output C + T bg.
 *  gradient  exact derivative of the above where it is differentiable: zero
 *            through a clamped alpha, the slope clamp and the SH clamp.  The
 *            per-pixel part uses dC/dalpha_i = T_i rgb_i - (S_i + T_final bg)/(1-alpha_i)
 *            with S_i the colour composited behind i (explicit suffix sums);
 *            the projection part is differentiated by the complex-step method
 *            (one complex evaluation of the projection per parameter).
 *  adam, l1  textbook Adam with bias correction; mean absolute error.  The
 *            visible-only variant leaves Gaussians that touch no tile in any
 *            view of the batch (and their moments) unchanged.
 *
 * Decisions taken by comparing floating-point numbers (the skip / clamp /
 * stop thresholds, the radius ceil, the rect floors, depth order) are
 * reported as "marginal" when the FP64 value lies within a small relative
 * distance of the threshold, so that tests can leave out the few pixels where
 * an FP32 implementation may legitimately decide the other way.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define TILE 16
#define ALPHA_CLAMP 0.99
#define ALPHA_SKIP (1.0 / 255.0)
#define T_STOP 1e-4
#define DILATION 0.3
#define GUARD 1.3
#define CSTEP 1e-30

/* margins for "marginal" decisions */
#define D_ALPHA 1e-4   /* relative, on alpha vs 1/255 and sigma*G vs 0.99 */
#define D_T 1e-3       /* relative, on T' vs 1e-4 */
#define D_EXT 1e-5     /* relative, 3 sqrt(lambda) vs an integer */
#define D_PX 2e-3      /* pixels, rect edges */
#define D_POWER 1e-6   /* relative, power vs 0 */

/* camera record: 26 doubles */
enum { C_VIEW = 0, C_FX = 16, C_FY, C_CX, C_CY, C_W, C_H, C_ZNEAR, C_BG, C_LEN = C_BG + 3 };

/* parameter planes */
enum { P_MEAN = 0, P_LSCALE = 3, P_QUAT = 6, P_OPAC = 10, P_SH = 11 };

/* Gaussian-level flags */
enum {
  G_VISIBLE = 1,
  G_MARG_ZNEAR = 2,    /* depth within margin of znear (visibility may flip) */
  G_MARG_RECT = 4,     /* radius or rect edge within margin */
  G_MARG_GUARD = 8,    /* slope clamp boundary (derivative jump) */
  G_MARG_SHCLAMP = 16, /* rgb clamp boundary (derivative jump) */
  G_HAS_Q = 32,        /* 2D quantities computed (in front of znear) */
};

/* per-pixel flags */
enum { PX_MARGINAL = 1 };

/* ---------------------------------------------------------------- SH basis */

/* Real orthonormal spherical harmonics Y_{l,m}, k = l*l + l + m, of a unit
 * direction (x, y, z); the unit-sphere forms of the Cartesian polynomials. */
static void sh_basis(int deg, cplx x, cplx y, cplx z, cplx* Y) {
  const double pi = M_PI;
  Y[0] = 0.5 * sqrt(1.0 / pi);
  if (deg < 1) return;
  const double c1 = sqrt(3.0 / (4.0 * pi));
  Y[1] = c1 * y;
  Y[2] = c1 * z;
  Y[3] = c1 * x;
  if (deg < 2) return;
  Y[4] = 0.5 * sqrt(15.0 / pi) * x * y;
  Y[5] = 0.5 * sqrt(15.0 / pi) * y * z;
  Y[6] = 0.25 * sqrt(5.0 / pi) * (3.0 * z * z - 1.0);
  Y[7] = 0.5 * sqrt(15.0 / pi) * x * z;
  Y[8] = 0.25 * sqrt(15.0 / pi) * (x * x - y * y);
  if (deg < 3) return;
  Y[9] = 0.25 * sqrt(35.0 / (2.0 * pi)) * y * (3.0 * x * x - y * y);
  Y[10] = 0.5 * sqrt(105.0 / pi) * x * y * z;
  Y[11] = 0.25 * sqrt(21.0 / (2.0 * pi)) * y * (5.0 * z * z - 1.0);
  Y[12] = 0.25 * sqrt(7.0 / pi) * z * (5.0 * z * z - 3.0);
  Y[13] = 0.25 * sqrt(21.0 / (2.0 * pi)) * x * (5.0 * z * z - 1.0);
  Y[14] = 0.25 * sqrt(105.0 / pi) * z * (x * x - y * y);
  Y[15] = 0.25 * sqrt(35.0 / (2.0 * pi)) * x * (x * x - 3.0 * y * y);
}

void or_sh_basis(int deg, const double* dirs, long n, double* out) {
  int K = (deg + 1) * (deg + 1);
  for (long i = 0; i < n; i++) {
    cplx Y[16];
    sh_basis(deg, dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], Y);
    for (int k = 0; k < K; k++) out[i * K + k] = creal(Y[k]);
  }
}

/* ---------------------------------------------------------------- projection */

typedef struct {
  int flags;
  int r;
  int rect[4]; /* x0, x1, y0, y1 (half-open, tile units) */
  int rect_in[4], rect_out[4]; /* bounds on the rect under small perturbations */
  double depth;
  double ext;  /* 3 sqrt(lambda) */
  cplx q[9];   /* mu_x, mu_y, A, B, C, sigma, r, g, b */
  double raw_rgb[3];
} proj_t;

static long imin_l(long a, long b) { return a < b ? a : b; }
static long imax_l(long a, long b) { return a > b ? a : b; }

static int near_multiple(double v, double period, double margin) {
  double k = floor(v / period + 0.5);
  return fabs(v - k * period) <= margin;
}

static float depth32(const double* V, double mx, double my, double mz) {
  volatile float a = (float)V[8] * (float)mx;
  volatile float b = (float)V[9] * (float)my;
  volatile float c = (float)V[10] * (float)mz;
  volatile float ab = a + b;
  volatile float abc = ab + c;
  volatile float d = abc + (float)V[11];
  return d;
}

/* Rect of tiles touched by the square of half-size r around (px, py); the
 * square is widened by `grow` pixels on every side (negative: shrunk). */
static void tile_rect(double px, double py, int r, double grow, int W, int H, int* rect) {
  const long gw = (W + TILE - 1) / TILE, gh = (H + TILE - 1) / TILE;
  rect[0] = (int)imin_l(gw, imax_l(0, (long)floor((px - r - grow) / TILE)));
  rect[1] = (int)imin_l(gw, imax_l(0, (long)floor((px + r + grow + TILE - 1) / TILE)));
  rect[2] = (int)imin_l(gh, imax_l(0, (long)floor((py - r - grow) / TILE)));
  rect[3] = (int)imin_l(gh, imax_l(0, (long)floor((py + r + grow + TILE - 1) / TILE)));
  if (rect[1] < rect[0]) rect[1] = rect[0];
  if (rect[3] < rect[2]) rect[3] = rect[2];
}

/* Project one Gaussian; pv holds its P parameters (complex for the
 * complex-step derivative; real parts carry the values). */
static void project_one(const cplx* pv, int deg, const double* cam, proj_t* o) {
  memset(o, 0, sizeof(*o));
  const double* V = cam + C_VIEW;
  const double fx = cam[C_FX], fy = cam[C_FY], cx = cam[C_CX], cy = cam[C_CY];
  const int W = (int)cam[C_W], H = (int)cam[C_H];
  const double znear = cam[C_ZNEAR];

  cplx m[3] = {pv[P_MEAN], pv[P_MEAN + 1], pv[P_MEAN + 2]};
  cplx t[3];
  for (int i = 0; i < 3; i++) t[i] = V[4 * i] * m[0] + V[4 * i + 1] * m[1] + V[4 * i + 2] * m[2] + V[4 * i + 3];
  /* The depth that orders and culls is the FP32 value of t_z evaluated as
   * ((V20 mx + V21 my) + V22 mz) + V23, each operation rounded to FP32 (no
   * fused multiply-add): order and culling are discrete decisions, so both
   * implementations take them on this same FP32 number. */
  o->depth = (double)depth32(V, creal(m[0]), creal(m[1]), creal(m[2]));
  if (!(o->depth > (double)(float)znear)) return;

  /* Sigma = R S S^T R^T */
  cplx s[3] = {cexp(pv[P_LSCALE]), cexp(pv[P_LSCALE + 1]), cexp(pv[P_LSCALE + 2])};
  cplx qw = pv[P_QUAT], qx = pv[P_QUAT + 1], qy = pv[P_QUAT + 2], qz = pv[P_QUAT + 3];
  cplx qn = csqrt(qw * qw + qx * qx + qy * qy + qz * qz);
  qw /= qn; qx /= qn; qy /= qn; qz /= qn;
  cplx R[3][3] = {
      {1.0 - 2.0 * (qy * qy + qz * qz), 2.0 * (qx * qy - qw * qz), 2.0 * (qx * qz + qw * qy)},
      {2.0 * (qx * qy + qw * qz), 1.0 - 2.0 * (qx * qx + qz * qz), 2.0 * (qy * qz - qw * qx)},
      {2.0 * (qx * qz - qw * qy), 2.0 * (qy * qz + qw * qx), 1.0 - 2.0 * (qx * qx + qy * qy)}};
  cplx M[3][3];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) M[i][j] = R[i][j] * s[j];
  cplx S3[3][3];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) S3[i][j] = M[i][0] * M[j][0] + M[i][1] * M[j][1] + M[i][2] * M[j][2];

  /* J with clamped slopes */
  const double limx = GUARD * (double)W / (2.0 * fx);
  const double limy = GUARD * (double)H / (2.0 * fy);
  cplx ux = t[0] / t[2], uy = t[1] / t[2];
  if (fabs(fabs(creal(ux)) - limx) <= 1e-6 * limx || fabs(fabs(creal(uy)) - limy) <= 1e-6 * limy)
    o->flags |= G_MARG_GUARD;
  if (creal(ux) > limx) ux = limx;
  if (creal(ux) < -limx) ux = -limx;
  if (creal(uy) > limy) uy = limy;
  if (creal(uy) < -limy) uy = -limy;
  cplx J[2][3] = {{fx / t[2], 0.0, -fx * ux / t[2]}, {0.0, fy / t[2], -fy * uy / t[2]}};
  cplx T[2][3];
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 3; j++) T[i][j] = J[i][0] * V[j] + J[i][1] * V[4 + j] + J[i][2] * V[8 + j];
  cplx TS[2][3];
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 3; j++) TS[i][j] = T[i][0] * S3[0][j] + T[i][1] * S3[1][j] + T[i][2] * S3[2][j];
  cplx c00 = TS[0][0] * T[0][0] + TS[0][1] * T[0][1] + TS[0][2] * T[0][2] + DILATION;
  cplx c01 = TS[0][0] * T[1][0] + TS[0][1] * T[1][1] + TS[0][2] * T[1][2];
  cplx c11 = TS[1][0] * T[1][0] + TS[1][1] * T[1][1] + TS[1][2] * T[1][2] + DILATION;
  cplx det = c00 * c11 - c01 * c01;
  if (creal(det) == 0.0) return;

  /* extent (no derivative) */
  double mid = 0.5 * (creal(c00) + creal(c11));
  double lam = mid + sqrt(fmax(0.1, mid * mid - creal(det)));
  double ext = 3.0 * sqrt(lam);
  int r = (int)ceil(ext);
  o->ext = ext;
  o->r = r;

  cplx mux = fx * t[0] / t[2] + cx;
  cplx muy = fy * t[1] / t[2] + cy;
  o->q[0] = mux;
  o->q[1] = muy;
  o->q[2] = c11 / det;
  o->q[3] = -c01 / det;
  o->q[4] = c00 / det;
  o->q[5] = 1.0 / (1.0 + cexp(-pv[P_OPAC]));

  /* colour */
  cplx cp[3];
  for (int i = 0; i < 3; i++) cp[i] = -(V[i] * V[3] + V[4 + i] * V[7] + V[8 + i] * V[11]);
  cplx d[3] = {m[0] - cp[0], m[1] - cp[1], m[2] - cp[2]};
  cplx dn = csqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  cplx Y[16];
  sh_basis(deg, d[0] / dn, d[1] / dn, d[2] / dn, Y);
  const int K = (deg + 1) * (deg + 1);
  for (int c = 0; c < 3; c++) {
    cplx acc = 0.5;
    for (int k = 0; k < K; k++) acc += pv[P_SH + 3 * k + c] * Y[k];
    o->raw_rgb[c] = creal(acc);
    if (fabs(creal(acc)) <= 1e-6) o->flags |= G_MARG_SHCLAMP;
    o->q[6 + c] = creal(acc) < 0.0 ? 0.0 : acc;
  }
  o->flags |= G_HAS_Q;

  /* tile rect; the rect an FP32 evaluation could give lies between the
   * "inner" and "outer" rects computed with the margins below */
  tile_rect(creal(mux), creal(muy), r, 0.0, W, H, o->rect);
  int r_lo = r, r_hi = r;
  if (near_multiple(ext, 1.0, D_EXT * ext + 1e-9)) {
    r_lo = (int)floor(ext + 0.5);
    r_hi = r_lo + 1;
  }
  tile_rect(creal(mux), creal(muy), r_lo, -D_PX, W, H, o->rect_in);
  tile_rect(creal(mux), creal(muy), r_hi, D_PX, W, H, o->rect_out);
  for (int k = 0; k < 4; k++)
    if (o->rect_in[k] != o->rect_out[k]) o->flags |= G_MARG_RECT;
  if (r <= 0) return;
  if ((o->rect[1] - o->rect[0]) * (o->rect[3] - o->rect[2]) == 0) return;
  o->flags |= G_VISIBLE;
}

static void load_params(const double* params, long stride, long g, int P, cplx* pv) {
  for (int p = 0; p < P; p++) pv[p] = params[(long)p * stride + g];
}

static int n_planes(int deg) { return P_SH + 3 * (deg + 1) * (deg + 1); }

static proj_t* project_all(const double* params, long n, long stride, int deg, const double* cam) {
  proj_t* pr = (proj_t*)malloc(sizeof(proj_t) * (size_t)(n > 0 ? n : 1));
  const int P = n_planes(deg);
#pragma omp parallel for schedule(static)
  for (long g = 0; g < n; g++) {
    cplx pv[64];
    load_params(params, stride, g, P, pv);
    project_one(pv, deg, cam, &pr[g]);
  }
  return pr;
}

/* Projection outputs per Gaussian:
 * fout[g*16 + ...] = mu_x, mu_y, depth, A, B, C, sigma, r, g, b, ext, raw_r, raw_g, raw_b, 0, 0
 * iout[g*8 + ...]  = flags, radius, x0, x1, y0, y1, tiles, 0 */
void or_project(const double* params, long n, long stride, int deg, const double* cam, double* fout,
                int* iout) {
  proj_t* pr = project_all(params, n, stride, deg, cam);
  for (long g = 0; g < n; g++) {
    const proj_t* o = &pr[g];
    double* f = fout + g * 16;
    for (int k = 0; k < 16; k++) f[k] = 0.0;
    f[0] = creal(o->q[0]); f[1] = creal(o->q[1]); f[2] = o->depth;
    for (int k = 2; k < 9; k++) f[k + 1] = creal(o->q[k]);
    f[10] = o->ext;
    f[11] = o->raw_rgb[0]; f[12] = o->raw_rgb[1]; f[13] = o->raw_rgb[2];
    int* ii = iout + g * 8;
    ii[0] = o->flags; ii[1] = o->r;
    ii[2] = o->rect[0]; ii[3] = o->rect[1]; ii[4] = o->rect[2]; ii[5] = o->rect[3];
    ii[6] = (o->flags & G_VISIBLE) ? (o->rect[1] - o->rect[0]) * (o->rect[3] - o->rect[2]) : 0;
    ii[7] = 0;
  }
  free(pr);
}

/* ---------------------------------------------------------------- tile lists */

typedef struct {
  long ntiles, gw, gh;
  long* start;  /* [ntiles + 1] */
  long* ids;    /* Gaussian ids, per tile sorted by (depth, id) */
  long* astart; /* [ntiles + 1]: Gaussians whose membership of the tile is marginal */
  long* aids;
  int all_marginal; /* a Gaussian sits at znear: every pixel is marginal */
} tiles_t;

static const proj_t* g_sort_proj;
static int cmp_depth_id(const void* a, const void* b) {
  long ia = *(const long*)a, ib = *(const long*)b;
  double da = g_sort_proj[ia].depth, db = g_sort_proj[ib].depth;
  if (da < db) return -1;
  if (da > db) return 1;
  return (ia > ib) - (ia < ib);
}

static int in_rect(const int* r, long tx, long ty) {
  return tx >= r[0] && tx < r[1] && ty >= r[2] && ty < r[3];
}

/* Per-tile lists: members (rect contains the tile), sorted by (depth, id);
 * and marginal members (outer rect contains the tile, inner rect does not).
 * Only tiles with want[tile] != 0 (all, if want == NULL). */
static void build_tiles(const proj_t* pr, long n, int W, int H, const uint8_t* want, tiles_t* tl) {
  tl->gw = (W + TILE - 1) / TILE;
  tl->gh = (H + TILE - 1) / TILE;
  tl->ntiles = tl->gw * tl->gh;
  tl->all_marginal = 0;
  long* cnt = (long*)calloc((size_t)tl->ntiles + 1, sizeof(long));
  long* acnt = (long*)calloc((size_t)tl->ntiles + 1, sizeof(long));
  for (int pass = 0; pass < 2; pass++) {
    long *fill = NULL, *afill = NULL;
    if (pass == 1) {
      fill = (long*)malloc(sizeof(long) * (size_t)tl->ntiles);
      afill = (long*)malloc(sizeof(long) * (size_t)tl->ntiles);
      for (long t = 0; t < tl->ntiles; t++) {
        fill[t] = cnt[t];
        afill[t] = acnt[t];
      }
    }
    for (long g = 0; g < n; g++) {
      const proj_t* o = &pr[g];
      if (o->flags & G_MARG_ZNEAR) tl->all_marginal = 1;
      if (o->flags & G_VISIBLE)
        for (long ty = o->rect[2]; ty < o->rect[3]; ty++)
          for (long tx = o->rect[0]; tx < o->rect[1]; tx++) {
            long t = ty * tl->gw + tx;
            if (want && !want[t]) continue;
            if (pass == 0) cnt[t + 1]++;
            else tl->ids[fill[t]++] = g;
          }
      if ((o->flags & G_HAS_Q) && (o->flags & G_MARG_RECT))
        for (long ty = o->rect_out[2]; ty < o->rect_out[3]; ty++)
          for (long tx = o->rect_out[0]; tx < o->rect_out[1]; tx++) {
            long t = ty * tl->gw + tx;
            if ((want && !want[t]) || in_rect(o->rect_in, tx, ty)) continue;
            if (pass == 0) acnt[t + 1]++;
            else tl->aids[afill[t]++] = g;
          }
    }
    if (pass == 0) {
      for (long t = 0; t < tl->ntiles; t++) {
        cnt[t + 1] += cnt[t];
        acnt[t + 1] += acnt[t];
      }
      long total = cnt[tl->ntiles], atotal = acnt[tl->ntiles];
      tl->ids = (long*)malloc(sizeof(long) * (size_t)(total > 0 ? total : 1));
      tl->aids = (long*)malloc(sizeof(long) * (size_t)(atotal > 0 ? atotal : 1));
    } else {
      free(fill);
      free(afill);
    }
  }
  tl->start = cnt;
  tl->astart = acnt;
  g_sort_proj = pr;
  for (long t = 0; t < tl->ntiles; t++) {
    long a = tl->start[t], b = tl->start[t + 1];
    if (b - a > 1) qsort(tl->ids + a, (size_t)(b - a), sizeof(long), cmp_depth_id);
  }
}

static void free_tiles(tiles_t* tl) {
  free(tl->start);
  free(tl->ids);
  free(tl->astart);
  free(tl->aids);
}

/* ---------------------------------------------------------------- composite */

typedef struct {
  long id;     /* Gaussian id */
  double a;    /* alpha */
  double T;    /* transmittance in front of it */
  double G;    /* exp(power) */
  double dx, dy;
  int clamped; /* sigma G > 0.99 */
} contrib_t;

static int near_rel(double v, double thr, double rel) { return fabs(v - thr) <= rel * thr; }

/* alpha of Gaussian o at pixel (px, py) before the skip test; sets *pw */
static double alpha_at(const proj_t* o, double px, double py, double* pw, double* G_out, double* dx_out,
                       double* dy_out, int* clamped) {
  double dx = creal(o->q[0]) - px, dy = creal(o->q[1]) - py;
  double A = creal(o->q[2]), B = creal(o->q[3]), Cc = creal(o->q[4]);
  double power = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy;
  double G = exp(power);
  double sg = creal(o->q[5]) * G;
  *pw = power;
  if (G_out) *G_out = G;
  if (dx_out) *dx_out = dx;
  if (dy_out) *dy_out = dy;
  if (clamped) *clamped = sg > ALPHA_CLAMP;
  return sg < ALPHA_CLAMP ? sg : ALPHA_CLAMP;
}

/* could Gaussian o contribute at the pixel under a small perturbation? */
static int may_contribute(const proj_t* o, double px, double py) {
  double pw;
  double a = alpha_at(o, px, py, &pw, NULL, NULL, NULL, NULL);
  return a >= ALPHA_SKIP * (1.0 - D_ALPHA);
}

/* Composite one pixel; fills contributors (if cb != NULL, capacity cap) and
 * returns their count.  *marg is set when a decision was within its margin. */
static long composite_pixel(const proj_t* pr, const tiles_t* tl, long tile, double px, double py,
                            const double* bg, double* rgb_out, double* T_out, int* marg,
                            contrib_t* cb, long cap) {
  double T = 1.0, C[3] = {0.0, 0.0, 0.0};
  long nc = 0;
  int mg = tl->all_marginal;
  for (long i = tl->start[tile]; i < tl->start[tile + 1]; i++) {
    const proj_t* o = &pr[tl->ids[i]];
    double power, G, dx, dy;
    int clamped;
    double a = alpha_at(o, px, py, &power, &G, &dx, &dy, &clamped);
    double A = creal(o->q[2]), B = creal(o->q[3]), Cc = creal(o->q[4]);
    double scale = 0.5 * (fabs(A) * dx * dx + fabs(Cc) * dy * dy) + fabs(B * dx * dy);
    if (scale > 0.0 && fabs(power) <= D_POWER * scale) mg = 1;
    if (power > 0.0) continue;
    if (near_rel(creal(o->q[5]) * G, ALPHA_CLAMP, D_ALPHA)) mg = 1;
    if (near_rel(a, ALPHA_SKIP, D_ALPHA)) mg = 1;
    if (a < ALPHA_SKIP) continue;
    double Tn = T * (1.0 - a);
    if (near_rel(Tn, T_STOP, D_T)) mg = 1;
    if (Tn < T_STOP) break;
    for (int c = 0; c < 3; c++) C[c] += creal(o->q[6 + c]) * a * T;
    if (cb && nc < cap) {
      cb[nc].id = tl->ids[i];
      cb[nc].a = a;
      cb[nc].T = T;
      cb[nc].G = G;
      cb[nc].dx = dx;
      cb[nc].dy = dy;
      cb[nc].clamped = clamped;
    }
    nc++;
    T = Tn;
  }
  /* Gaussians whose membership of this tile is itself marginal */
  for (long i = tl->astart[tile]; i < tl->astart[tile + 1] && !mg; i++)
    if (may_contribute(&pr[tl->aids[i]], px, py)) mg = 1;
  for (int c = 0; c < 3; c++) rgb_out[c] = C[c] + T * bg[c];
  *T_out = T;
  *marg = mg;
  return nc;
}

/* Full render of one view.  img [3][H][W], tfinal [H][W], marg [H][W] (uint8).
 * tile_want: optional [ntiles] mask of tiles to render (others left as bg, T=1).
 * Returns the number of (pixel, Gaussian) contributions. */
long or_render(const double* params, long n, long stride, int deg, const double* cam,
               const uint8_t* tile_want, double* img, double* tfinal, uint8_t* marg) {
  const int W = (int)cam[C_W], H = (int)cam[C_H];
  proj_t* pr = project_all(params, n, stride, deg, cam);
  tiles_t tl;
  build_tiles(pr, n, W, H, tile_want, &tl);
  const double* bg = cam + C_BG;
  long pairs = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : pairs)
  for (long t = 0; t < tl.ntiles; t++) {
    long tx = t % tl.gw, ty = t / tl.gw;
    for (int j = 0; j < TILE; j++)
      for (int i = 0; i < TILE; i++) {
        long x = tx * TILE + i, y = ty * TILE + j;
        if (x >= W || y >= H) continue;
        long pix = y * W + x;
        double rgb[3], T;
        int mg = 0;
        if (tile_want && !tile_want[t]) {
          for (int c = 0; c < 3; c++) rgb[c] = bg[c];
          T = 1.0;
        } else {
          pairs += composite_pixel(pr, &tl, t, (double)x, (double)y, bg, rgb, &T, &mg, NULL, 0);
        }
        for (int c = 0; c < 3; c++) img[(long)c * W * H + pix] = rgb[c];
        tfinal[pix] = T;
        marg[pix] = (uint8_t)(mg ? PX_MARGINAL : 0);
      }
  }
  free_tiles(&tl);
  free(pr);
  return pairs;
}

/* Render a list of pixels (spot checks on large images); only the tiles that
 * hold a requested pixel are built. */
void or_render_pixels(const double* params, long n, long stride, int deg, const double* cam, long npix,
                      const int* xs, const int* ys, double* rgb_out, double* t_out, uint8_t* marg) {
  const int W = (int)cam[C_W], H = (int)cam[C_H];
  const long gw = (W + TILE - 1) / TILE, gh = (H + TILE - 1) / TILE;
  uint8_t* want = (uint8_t*)calloc((size_t)(gw * gh), 1);
  for (long i = 0; i < npix; i++) want[(ys[i] / TILE) * gw + xs[i] / TILE] = 1;
  proj_t* pr = project_all(params, n, stride, deg, cam);
  tiles_t tl;
  build_tiles(pr, n, W, H, want, &tl);
#pragma omp parallel for schedule(dynamic, 1)
  for (long i = 0; i < npix; i++) {
    long t = (ys[i] / TILE) * gw + xs[i] / TILE;
    int mg = 0;
    composite_pixel(pr, &tl, t, (double)xs[i], (double)ys[i], cam + C_BG, rgb_out + 3 * i, &t_out[i],
                    &mg, NULL, 0);
    marg[i] = (uint8_t)(mg ? PX_MARGINAL : 0);
  }
  free_tiles(&tl);
  free(pr);
  free(want);
}

/* ---------------------------------------------------------------- gradient */

/* dL/d(2D quantities) of one view.  dimg [3][H][W]; g2d [n][9] accumulated
 * (mu_x, mu_y, A, B, C, sigma, r, g, b).  Tiles whose dimg is all zero are
 * skipped. */
static void grad_2d(const proj_t* pr, long n, const double* cam, const double* dimg, double* g2d) {
  const int W = (int)cam[C_W], H = (int)cam[C_H];
  const long gw = (W + TILE - 1) / TILE, gh = (H + TILE - 1) / TILE;
  uint8_t* want = (uint8_t*)calloc((size_t)(gw * gh), 1);
  for (long y = 0; y < H; y++)
    for (long x = 0; x < W; x++) {
      long pix = y * W + x;
      if (dimg[pix] != 0.0 || dimg[(long)W * H + pix] != 0.0 || dimg[2L * W * H + pix] != 0.0)
        want[(y / TILE) * gw + x / TILE] = 1;
    }
  tiles_t tl;
  build_tiles(pr, n, W, H, want, &tl);
  const double* bg = cam + C_BG;
#pragma omp parallel
  {
    long cap = 1024;
    contrib_t* cb = (contrib_t*)malloc(sizeof(contrib_t) * (size_t)cap);
#pragma omp for schedule(dynamic, 1)
    for (long t = 0; t < tl.ntiles; t++) {
      if (!want[t]) continue;
      long len = tl.start[t + 1] - tl.start[t];
      if (len > cap) {
        cap = len;
        cb = (contrib_t*)realloc(cb, sizeof(contrib_t) * (size_t)cap);
      }
      long tx = t % gw, ty = t / gw;
      for (int j = 0; j < TILE; j++)
        for (int i = 0; i < TILE; i++) {
          long x = tx * TILE + i, y = ty * TILE + j;
          if (x >= W || y >= H) continue;
          long pix = y * W + x;
          double dC[3] = {dimg[pix], dimg[(long)W * H + pix], dimg[2L * W * H + pix]};
          if (dC[0] == 0.0 && dC[1] == 0.0 && dC[2] == 0.0) continue;
          double rgb[3], Tf;
          int mg;
          long nc = composite_pixel(pr, &tl, t, (double)x, (double)y, bg, rgb, &Tf, &mg, cb, cap);
          /* S = colour composited behind contributor i (suffix sum) */
          double S[3] = {0.0, 0.0, 0.0};
          for (long k = nc - 1; k >= 0; k--) {
            const contrib_t* c = &cb[k];
            const proj_t* o = &pr[c->id];
            double col[3] = {creal(o->q[6]), creal(o->q[7]), creal(o->q[8])};
            double dL_da = 0.0;
            for (int ch = 0; ch < 3; ch++)
              dL_da += dC[ch] * (c->T * col[ch] - (S[ch] + Tf * bg[ch]) / (1.0 - c->a));
            double gq[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            for (int ch = 0; ch < 3; ch++) gq[6 + ch] = dC[ch] * c->a * c->T;
            if (!c->clamped) {
              double A = creal(o->q[2]), B = creal(o->q[3]), Cc = creal(o->q[4]);
              double sig = creal(o->q[5]);
              gq[5] = dL_da * c->G;
              double dL_dpow = dL_da * sig * c->G;
              gq[0] = dL_dpow * (-(A * c->dx + B * c->dy));
              gq[1] = dL_dpow * (-(Cc * c->dy + B * c->dx));
              gq[2] = dL_dpow * (-0.5 * c->dx * c->dx);
              gq[3] = dL_dpow * (-c->dx * c->dy);
              gq[4] = dL_dpow * (-0.5 * c->dy * c->dy);
            }
            for (int q = 0; q < 9; q++) {
#pragma omp atomic
              g2d[c->id * 9 + q] += gq[q];
            }
            for (int ch = 0; ch < 3; ch++) S[ch] += col[ch] * c->a * c->T;
          }
        }
    }
    free(cb);
  }
  free_tiles(&tl);
  free(want);
}

/* Chain rule from 2D gradients to parameters by complex step. */
static void grad_params(const double* params, long n, long stride, int deg, const double* cam,
                        const proj_t* pr, const double* g2d, double* grad) {
  const int P = n_planes(deg);
#pragma omp parallel for schedule(dynamic, 64)
  for (long g = 0; g < n; g++) {
    const double* gg = g2d + g * 9;
    int any = 0;
    for (int q = 0; q < 9; q++) any |= gg[q] != 0.0;
    if (!any || !(pr[g].flags & G_VISIBLE)) continue;
    cplx pv[64];
    load_params(params, stride, g, P, pv);
    for (int p = 0; p < P; p++) {
      cplx keep = pv[p];
      pv[p] = creal(keep) + I * CSTEP;
      proj_t o;
      project_one(pv, deg, cam, &o);
      double acc = 0.0;
      for (int q = 0; q < 9; q++) acc += gg[q] * cimag(o.q[q]) / CSTEP;
      grad[(long)p * stride + g] += acc;
      pv[p] = keep;
    }
  }
}

/* Gradient of sum(dimg * image) over B views.  cams: B camera records,
 * dimg: per view [3][H_v][W_v] concatenated; grad [P][stride] (accumulated);
 * g2d_out (optional): [B][n][9]. */
void or_render_grad(const double* params, long n, long stride, int deg, const double* cams, int B,
                    const double* dimg, double* grad, double* g2d_out) {
  long off = 0;
  for (int v = 0; v < B; v++) {
    const double* cam = cams + (long)v * C_LEN;
    const int W = (int)cam[C_W], H = (int)cam[C_H];
    proj_t* pr = project_all(params, n, stride, deg, cam);
    double* g2d = (double*)calloc((size_t)(n > 0 ? n : 1) * 9, sizeof(double));
    grad_2d(pr, n, cam, dimg + off, g2d);
    grad_params(params, n, stride, deg, cam, pr, g2d, grad);
    if (g2d_out) memcpy(g2d_out + (long)v * n * 9, g2d, sizeof(double) * (size_t)n * 9);
    free(g2d);
    free(pr);
    off += 3L * W * H;
  }
}

/* Jacobian of the 9 projected quantities with respect to the P parameters of
 * Gaussian g (complex step); jac [9][P]. Returns the Gaussian's flags. */
int or_project_jacobian(const double* params, long n, long stride, int deg, const double* cam, long g,
                        double* jac) {
  const int P = n_planes(deg);
  cplx pv[64];
  (void)n;
  load_params(params, stride, g, P, pv);
  proj_t o;
  project_one(pv, deg, cam, &o);
  int flags = o.flags;
  for (int p = 0; p < P; p++) {
    cplx keep = pv[p];
    pv[p] = creal(keep) + I * CSTEP;
    project_one(pv, deg, cam, &o);
    for (int q = 0; q < 9; q++) jac[q * P + p] = cimag(o.q[q]) / CSTEP;
    pv[p] = keep;
  }
  return flags;
}

/* Gaussian flags for one view (visibility and derivative-discontinuity marks). */
void or_gaussian_flags(const double* params, long n, long stride, int deg, const double* cam, int* flags) {
  proj_t* pr = project_all(params, n, stride, deg, cam);
  for (long g = 0; g < n; g++) flags[g] = pr[g].flags;
  free(pr);
}

/* ---------------------------------------------------------------- loss, Adam */

/* L1: loss = mean |x - y|; grad = sign(x - y) / count (sign(0) = 0). */
double or_l1(const double* x, const double* y, long count, double* grad) {
  double s = 0.0;
  for (long i = 0; i < count; i++) {
    double d = x[i] - y[i];
    s += fabs(d);
    if (grad) grad[i] = (d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0)) / (double)count;
  }
  return s / (double)count;
}

/* Adam with bias correction on P planes of length n (row stride `stride`);
 * lr[P] per plane; step is 1-based. */
void or_adam(double* p, const double* g, double* m, double* v, int P, long n, long stride,
             const double* lr, double b1, double b2, double eps, long step) {
  double bc1 = 1.0 - pow(b1, (double)step), bc2 = 1.0 - pow(b2, (double)step);
  for (int pl = 0; pl < P; pl++)
    for (long i = 0; i < n; i++) {
      long k = (long)pl * stride + i;
      m[k] = b1 * m[k] + (1.0 - b1) * g[k];
      v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k];
      double mh = m[k] / bc1, vh = v[k] / bc2;
      p[k] -= lr[pl] * mh / (sqrt(vh) + eps);
    }
}

/* Visible-only Adam: the sparse variant of the same update, in which a
 * Gaussian that touches no tile in any view of the batch (visible[i] == 0)
 * keeps its parameters and both moments unchanged, and every other Gaussian
 * takes the Adam step above, bias-corrected by the global step count. */
void or_adam_visible(double* p, const double* g, double* m, double* v, int P, long n, long stride,
                     const double* lr, double b1, double b2, double eps, long step, const uint8_t* visible) {
  double bc1 = 1.0 - pow(b1, (double)step), bc2 = 1.0 - pow(b2, (double)step);
  for (int pl = 0; pl < P; pl++)
    for (long i = 0; i < n; i++) {
      if (!visible[i]) continue;
      long k = (long)pl * stride + i;
      m[k] = b1 * m[k] + (1.0 - b1) * g[k];
      v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k];
      double mh = m[k] / bc1, vh = v[k] / bc2;
      p[k] -= lr[pl] * mh / (sqrt(vh) + eps);
    }
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
