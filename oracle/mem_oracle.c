/* Plain CPU oracle of MEM's map-update path (arXiv 2309.16818).
 *
 * TEST INFRASTRUCTURE ONLY (see mem_oracle.h). Built with
 *   gcc -O2 -ffp-contract=off -fno-fast-math
 * so that every binary32 decision below is exactly the written sequence of
 * correctly rounded operations, and sums are plain binary64 loops in input
 * order. Nothing is blocked, fused or reordered beyond the definitions.
 */
#include "mem_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* storage formats                                                          */

static float bf16_bits_to_float(uint16_t b) {
  uint32_t u = (uint32_t)b << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

/* binary32 -> bfloat16, round to nearest, ties to even (NaN kept quiet). */
static float round_bf16(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu)) return f;
  u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
  memcpy(&f, &u, 4);
  return f;
}

static double store_round(const orc_cfg *c, int fmt, double x) {
  if (!c->round_store) return x;
  float f = (float)x;
  if (fmt == ORC_BF16) return (double)round_bf16(f);
  if (fmt == ORC_F16) return (double)(float)(_Float16)f;
  return (double)f;
}

static double load_val(const orc_src *s, int64_t row, int k) {
  if (s->topk > 0) { /* class k of a row of top-k (class id, probability) pairs */
    const float *r = (const float *)s->data + row * 2 * (int64_t)s->topk;
    float v = 0.0f;
    for (int j = 0; j < s->topk; ++j) {
      float id = r[2 * j];
      if (id >= 0.0f && id < (float)s->channels && id == floorf(id) && (int)id == k) v += r[2 * j + 1];
    }
    return (double)v;
  }
  int64_t off = row * (int64_t)s->channels + k;
  switch (s->dtype) {
    case ORC_F32: return (double)((const float *)s->data)[off];
    case ORC_BF16: return (double)bf16_bits_to_float(((const uint16_t *)s->data)[off]);
    case ORC_F16: return (double)(float)((const _Float16 *)s->data)[off];
    case ORC_U8: return (double)((const uint8_t *)s->data)[off];
  }
  return NAN;
}

static int stored_values(const orc_cfg *c, int l) {
  return c->rule[l] == ORC_CLASSMAX ? 2 : c->channels[l];
}

/* ------------------------------------------------------------------------ */
/* map state                                                                */

void orc_init_state(const orc_cfg *c, orc_state *s) {
  int64_t W2 = (int64_t)c->W * c->W;
  for (int64_t j = 0; j < W2; ++j) {
    s->h[j] = 0.0;
    s->var[j] = 0.0;
    s->valid[j] = 0;
    s->n_acc[j] = 0;
    s->n_rej[j] = 0;
  }
  for (int l = 0; l < c->n_layers; ++l) {
    int S = stored_values(c, l);
    for (int64_t j = 0; j < W2; ++j) {
      s->obs[l][j] = 0;
      for (int k = 0; k < S; ++k) {
        double v = 0.0;
        if (c->rule[l] == ORC_DIRICHLET) v = store_round(c, c->store[l], c->alpha0[l]);
        if (c->rule[l] == ORC_CLASSMAX && k == 0) v = -1.0;
        s->layer[l][j * S + k] = v;
      }
      if (c->rule[l] == ORC_GAUSS)
        for (int k = 0; k < c->channels[l]; ++k) s->lvar[l][j * c->channels[l] + k] = INFINITY;
    }
  }
}

/* Sensor pose relative to the map centre, cast to binary32: the rotation is
 * unchanged, the translation loses the map origin's xy. */
void orc_pose_rel(const double T[16], const double origin[2], float Rt[12]) {
  for (int r = 0; r < 3; ++r)
    for (int k = 0; k < 3; ++k) Rt[r * 3 + k] = (float)T[r * 4 + k];
  Rt[9] = (float)(T[3] - origin[0]);
  Rt[10] = (float)(T[7] - origin[1]);
  Rt[11] = (float)T[11];
}

/* Transform, filter and associate one point (Sec. III-B: a point belongs to
 * the cell under its horizontal coordinates). Returns 1 if kept.
 *   p = R p_s + t                          (fmaf chain, fixed order)
 *   range = sqrt(xs^2 + ys^2 + zs^2)       (fmaf chain)
 *   cell x index = floor(x / res) + W/2    (kept iff inside [0, W))
 *   measurement variance = (sigma0 + sigma1 range)^2 */
int orc_point_cell(const orc_cfg *c, const float Rt[12], const float p[3], int32_t *cell,
                   float *z, float *vm) {
  float xs = p[0], ys = p[1], zs = p[2];
  if (!isfinite(xs) || !isfinite(ys) || !isfinite(zs)) return 0;
  float r2 = fmaf(xs, xs, fmaf(ys, ys, zs * zs));
  float rs = sqrtf(r2);
  if (!(rs >= c->range_min && rs <= c->range_max)) return 0;
  float x = fmaf(Rt[0], xs, fmaf(Rt[1], ys, fmaf(Rt[2], zs, Rt[9])));
  float y = fmaf(Rt[3], xs, fmaf(Rt[4], ys, fmaf(Rt[5], zs, Rt[10])));
  float zz = fmaf(Rt[6], xs, fmaf(Rt[7], ys, fmaf(Rt[8], zs, Rt[11])));
  float res = (float)c->res;
  float qx = floorf(x / res);
  float qy = floorf(y / res);
  float half = (float)(c->W / 2);
  if (!(qx >= -half && qx < half && qy >= -half && qy < half)) return 0;
  int32_t ix = (int32_t)qx + c->W / 2;
  int32_t iy = (int32_t)qy + c->W / 2;
  float sm = fmaf(c->sigma1, rs, c->sigma0);
  *cell = iy * c->W + ix;
  *z = zz;
  *vm = sm * sm;
  return 1;
}

/* ------------------------------------------------------------------------ */
/* per-cell fusion rules (Sec. III-C)                                       */

typedef struct {
  double *sum; /* [W2 * C] */
  double *mx;  /* [W2 * C] */
} src_acc;

/* Apply the rule of layer l to cell j from N observations with per-channel
 * sums S and maxima M (for images N = 1 and S = M = the pixel). */
static void apply_rule(const orc_cfg *c, orc_state *s, int l, int64_t j, double N, const double *S,
                       const double *M) {
  int C = c->channels[l];
  int fmt = c->store[l];
  double *th = s->layer[l];
  switch (c->rule[l]) {
    case ORC_LATEST: /* Eq. (1): cell-wise average of this update's observations */
      for (int k = 0; k < C; ++k) th[j * C + k] = store_round(c, fmt, S[k] / N);
      break;
    case ORC_EXPAVG: /* Eq. (2): theta_t = w a_t + (1 - w) theta_{t-1}; a first
                        observation initialises theta_t = a_t */
      for (int k = 0; k < C; ++k) {
        double a = S[k] / N;
        double t = s->obs[l][j] ? c->w[l] * a + (1.0 - c->w[l]) * th[j * C + k] : a;
        th[j * C + k] = store_round(c, fmt, t);
      }
      break;
    case ORC_GAUSS: /* Eqs. (6)-(7): conjugate Gaussian update with known variance
                       sigma_f^2; a never-observed cell has an infinitely wide prior */
      for (int k = 0; k < C; ++k) {
        double sf2 = c->var_meas[l];
        double mu_ml = S[k] / N;
        double mu, s2;
        if (s->obs[l][j]) {
          double s02 = s->lvar[l][j * C + k];
          double mu0 = th[j * C + k];
          double den = N * s02 + sf2;
          mu = sf2 / den * mu0 + N * s02 / den * mu_ml;
          s2 = sf2 * s02 / den;
        } else {
          mu = mu_ml;
          s2 = sf2 / N;
        }
        th[j * C + k] = store_round(c, fmt, mu);
        s->lvar[l][j * C + k] = store_round(c, ORC_F32, s2);
      }
      break;
    case ORC_DIRICHLET: /* Eq. (12): alpha_t = alpha_{t-1} + sum_i m_i */
      for (int k = 0; k < C; ++k) th[j * C + k] = store_round(c, fmt, th[j * C + k] + S[k]);
      break;
    case ORC_CLASSMAX: { /* highest class probability seen in this update; the
                            smallest class index wins a tie */
      double best = -INFINITY;
      int id = -1;
      for (int k = 0; k < C; ++k)
        if (M[k] > best) {
          best = M[k];
          id = k;
        }
      th[j * 2 + 0] = (double)id;
      th[j * 2 + 1] = store_round(c, fmt, best);
      break;
    }
  }
  s->obs[l][j] = 1;
}

/* ------------------------------------------------------------------------ */
/* point-cloud update                                                       */

static _Thread_local double g_last_drift;
static _Thread_local int64_t g_last_drift_points, g_last_cleared;

void orc_last_fuse_info(double *drift, int64_t *drift_points, int64_t *cleared) {
  if (drift) *drift = g_last_drift;
  if (drift_points) *drift_points = g_last_drift_points;
  if (cleared) *cleared = g_last_cleared;
}

/* The map cell of a position relative to the map centre, clamped into the map
 * (the sensor or camera cell of a visibility walk). */
static void clamped_cell(const orc_cfg *c, float px, float py, int32_t *cx, int32_t *cy) {
  float res = (float)c->res;
  float half = (float)(c->W / 2);
  float qx = floorf(px / res), qy = floorf(py / res);
  if (!(qx >= -half)) qx = -half;
  if (!(qx <= half - 1.0f)) qx = half - 1.0f;
  if (!(qy >= -half)) qy = -half;
  if (!(qy <= half - 1.0f)) qy = half - 1.0f;
  *cx = (int32_t)qx + c->W / 2;
  *cy = (int32_t)qy + c->W / 2;
}

int64_t orc_fuse_points(const orc_cfg *c, orc_state *s, int64_t n, const float *xyz, int32_t n_src,
                        const orc_src *src, const double T[16], uint8_t *near_gate,
                        int32_t *cell_out) {
  int64_t W2 = (int64_t)c->W * c->W;
  float Rt[12];
  orc_pose_rel(T, s->origin, Rt);
  double *Sw = calloc((size_t)W2, sizeof(double));
  double *Swz = calloc((size_t)W2, sizeof(double));
  uint32_t *na = calloc((size_t)W2, sizeof(uint32_t));
  uint32_t *nr = calloc((size_t)W2, sizeof(uint32_t));
  uint32_t *np = calloc((size_t)W2, sizeof(uint32_t));
  src_acc acc[ORC_MAX_LAYERS];
  for (int q = 0; q < n_src; ++q) {
    int64_t m = W2 * src[q].channels;
    acc[q].sum = calloc((size_t)m, sizeof(double));
    acc[q].mx = malloc((size_t)m * sizeof(double));
    for (int64_t k = 0; k < m; ++k) acc[q].mx[k] = -INFINITY;
  }
  float lam2 = c->gate_lambda * c->gate_lambda;
  int64_t kept = 0;

  /* z error count and drift compensation (Table I rows "point trsf. & z err. cnt" and "drift
     compensation"; the paper defers both to its predecessor, this is the reading stated in the
     design notes): e = z - h for every kept point whose cell is valid before this call and
     that the outlier gate accepts; if at least drift_min_points such points exist, every
     valid height moves by drift_alpha * mean(e), so the map follows the new cloud before the
     height update gates against it */
  double drift = 0.0;
  int64_t drift_n = 0;
  if (c->drift_alpha != 0.0) {
    double esum = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      int32_t j;
      float z, vm;
      if (!orc_point_cell(c, Rt, &xyz[3 * i], &j, &z, &vm)) continue;
      if (!s->valid[j]) continue;
      float d = z - (float)s->h[j];
      if (d * d > lam2 * ((float)s->var[j] + vm)) continue;
      esum += (double)d;
      ++drift_n;
    }
    if (drift_n > 0 && drift_n >= c->drift_min_points) {
      drift = (double)(float)(c->drift_alpha * (esum / (double)drift_n));
      for (int64_t j = 0; j < W2; ++j)
        if (s->valid[j]) s->h[j] = store_round(c, ORC_F32, s->h[j] + drift);
    }
  }
  g_last_drift = drift;
  g_last_drift_points = drift_n;
  g_last_cleared = 0;

  /* what the ray-cast clean-up needs: the state the gate sees, and every accepted point */
  double *h_gate = NULL;
  uint8_t *valid_gate = NULL;
  int32_t *acc_cell = NULL;
  float *acc_z = NULL;
  int64_t n_accpt = 0;
  if (c->ray_cleanup) {
    h_gate = malloc((size_t)W2 * sizeof(double));
    valid_gate = malloc((size_t)W2);
    memcpy(h_gate, s->h, (size_t)W2 * sizeof(double));
    memcpy(valid_gate, s->valid, (size_t)W2);
    acc_cell = malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    acc_z = malloc((size_t)(n > 0 ? n : 1) * sizeof(float));
  }

  /* association and accumulation, in input order */
  for (int64_t i = 0; i < n; ++i) {
    int32_t j;
    float z, vm;
    if (near_gate) near_gate[i] = 0;
    if (!orc_point_cell(c, Rt, &xyz[3 * i], &j, &z, &vm)) {
      if (cell_out) cell_out[i] = -1;
      continue;
    }
    if (cell_out) cell_out[i] = j;
    ++kept;
    ++np[j];
    /* outlier gate against the state before this update:
       reject iff (z - h)^2 > lambda^2 (sigma_h^2 + sigma_m^2) */
    int rej = 0;
    if (s->valid[j]) {
      float hj = (float)s->h[j];
      float vj = (float)s->var[j];
      float d = z - hj;
      float lhs = d * d;
      float rhs = lam2 * (vj + vm);
      rej = lhs > rhs;
      if (near_gate) near_gate[i] = fabs((double)lhs - (double)rhs) <= 1e-3 * (double)rhs;
    }
    if (rej) {
      ++nr[j];
    } else {
      ++na[j];
      Sw[j] += 1.0 / (double)vm;
      Swz[j] += (double)z / (double)vm;
      if (c->ray_cleanup) {
        acc_cell[n_accpt] = j;
        acc_z[n_accpt] = z;
        ++n_accpt;
      }
    }
    for (int q = 0; q < n_src; ++q) {
      int C = src[q].channels;
      for (int k = 0; k < C; ++k) {
        double v = load_val(&src[q], i, k);
        acc[q].sum[(int64_t)j * C + k] += v;
        if (v > acc[q].mx[(int64_t)j * C + k]) acc[q].mx[(int64_t)j * C + k] = v;
      }
    }
  }

  /* per-cell updates */
  for (int64_t j = 0; j < W2; ++j) {
    if (np[j] == 0) continue;
    /* height: scalar Kalman update in information form */
    if (na[j] > 0) {
      if (s->valid[j]) {
        double P = 1.0 / s->var[j] + Sw[j];
        s->h[j] = store_round(c, ORC_F32, (s->h[j] / s->var[j] + Swz[j]) / P);
        s->var[j] = store_round(c, ORC_F32, 1.0 / P);
      } else {
        s->h[j] = store_round(c, ORC_F32, Swz[j] / Sw[j]);
        s->var[j] = store_round(c, ORC_F32, 1.0 / Sw[j]);
        s->valid[j] = 1;
      }
    }
    if (nr[j] > 0 && c->outlier_var != 0.0f)
      s->var[j] = store_round(c, ORC_F32, s->var[j] + (double)c->outlier_var * nr[j]);
    s->n_acc[j] += na[j];
    s->n_rej[j] += nr[j];
    /* multi-modal layers, in source order then binding order */
    for (int q = 0; q < n_src; ++q) {
      int C = src[q].channels;
      for (int b = 0; b < src[q].n_layers; ++b)
        apply_rule(c, s, src[q].layers[b], j, (double)np[j], &acc[q].sum[j * C], &acc[q].mx[j * C]);
    }
  }
  /* ray-cast clean-up (the "ray cast" of Table I's "height update & ray cast"; reading stated
     in the design notes): every accepted point casts the ray from the sensor to itself over the
     integer Bresenham line of cells from the sensor's cell (clamped into the map) to its own
     cell, both ends excluded. An intermediate cell q that was valid for the gate is passed
     below when its height exceeds the ray height there by more than ray_margin:
       ray = z_s + t_q (z - z_s),  t_q = ((q - s).(e - s)) / |e - s|^2.
     A passed-below cell that accepted no point of this call is stale and becomes invalid. */
  if (c->ray_cleanup) {
    int32_t sx, sy;
    clamped_cell(c, Rt[9], Rt[10], &sx, &sy);
    float zs = Rt[11];
    uint8_t *mark = calloc((size_t)W2, 1);
    int32_t *line = malloc((size_t)(4 * c->W + 8) * sizeof(int32_t));
    for (int64_t a = 0; a < n_accpt; ++a) {
      int32_t ex = acc_cell[a] % c->W, ey = acc_cell[a] / c->W;
      int32_t dxs = ex - sx, dys = ey - sy;
      int32_t den = dxs * dxs + dys * dys;
      int32_t nl = orc_bresenham(sx, sy, ex, ey, line, 2 * c->W + 4);
      for (int32_t m = 1; m + 1 < nl; ++m) {
        int32_t qx = line[2 * m], qy = line[2 * m + 1];
        int64_t q = (int64_t)qy * c->W + qx;
        if (!valid_gate[q]) continue;
        int32_t num = (qx - sx) * dxs + (qy - sy) * dys;
        float tq = (float)num / (float)den;
        float ray = fmaf(tq, acc_z[a] - zs, zs);
        if ((float)h_gate[q] - ray > c->ray_margin) mark[q] = 1;
      }
    }
    for (int64_t q = 0; q < W2; ++q)
      if (mark[q] && na[q] == 0 && s->valid[q]) {
        s->valid[q] = 0;
        ++g_last_cleared;
      }
    free(mark);
    free(line);
    free(h_gate);
    free(valid_gate);
    free(acc_cell);
    free(acc_z);
  }

  if (c->time_var != 0.0f)
    for (int64_t j = 0; j < W2; ++j)
      if (s->valid[j]) s->var[j] = store_round(c, ORC_F32, s->var[j] + (double)c->time_var);

  for (int q = 0; q < n_src; ++q) {
    free(acc[q].sum);
    free(acc[q].mx);
  }
  free(Sw);
  free(Swz);
  free(na);
  free(nr);
  free(np);
  return kept;
}

/* ------------------------------------------------------------------------ */
/* robot-centric re-centring: integer-cell shift of every layer             */

void orc_move(const orc_cfg *c, orc_state *s, const double robot_xy[2]) {
  int W = c->W;
  int64_t W2 = (int64_t)W * W;
  long sx = lround((robot_xy[0] - s->origin[0]) / c->res);
  long sy = lround((robot_xy[1] - s->origin[1]) / c->res);
  if (sx == 0 && sy == 0) return;
  orc_state old = *s;
  /* copies of the old state */
  double *h = malloc((size_t)W2 * sizeof(double)), *v = malloc((size_t)W2 * sizeof(double));
  uint8_t *va = malloc((size_t)W2);
  uint32_t *a = malloc((size_t)W2 * 4), *r = malloc((size_t)W2 * 4);
  memcpy(h, s->h, (size_t)W2 * 8);
  memcpy(v, s->var, (size_t)W2 * 8);
  memcpy(va, s->valid, (size_t)W2);
  memcpy(a, s->n_acc, (size_t)W2 * 4);
  memcpy(r, s->n_rej, (size_t)W2 * 4);
  double *L[ORC_MAX_LAYERS], *LV[ORC_MAX_LAYERS];
  uint8_t *O[ORC_MAX_LAYERS];
  for (int l = 0; l < c->n_layers; ++l) {
    int S = stored_values(c, l);
    L[l] = malloc((size_t)(W2 * S) * 8);
    memcpy(L[l], s->layer[l], (size_t)(W2 * S) * 8);
    O[l] = malloc((size_t)W2);
    memcpy(O[l], s->obs[l], (size_t)W2);
    LV[l] = NULL;
    if (c->rule[l] == ORC_GAUSS) {
      LV[l] = malloc((size_t)(W2 * c->channels[l]) * 8);
      memcpy(LV[l], s->lvar[l], (size_t)(W2 * c->channels[l]) * 8);
    }
  }
  (void)old;
  orc_init_state(c, s);
  /* new cell (ix, iy) holds old cell (ix + sx, iy + sy) */
  for (int iy = 0; iy < W; ++iy) {
    long oy = iy + sy;
    if (oy < 0 || oy >= W) continue;
    for (int ix = 0; ix < W; ++ix) {
      long ox = ix + sx;
      if (ox < 0 || ox >= W) continue;
      int64_t jn = (int64_t)iy * W + ix, jo = (int64_t)oy * W + ox;
      s->h[jn] = h[jo];
      s->var[jn] = v[jo];
      s->valid[jn] = va[jo];
      s->n_acc[jn] = a[jo];
      s->n_rej[jn] = r[jo];
      for (int l = 0; l < c->n_layers; ++l) {
        int S = stored_values(c, l);
        for (int k = 0; k < S; ++k) s->layer[l][jn * S + k] = L[l][jo * S + k];
        s->obs[l][jn] = O[l][jo];
        if (LV[l])
          for (int k = 0; k < c->channels[l]; ++k)
            s->lvar[l][jn * c->channels[l] + k] = LV[l][jo * c->channels[l] + k];
      }
    }
  }
  s->origin[0] = old.origin[0] + (double)sx * c->res;
  s->origin[1] = old.origin[1] + (double)sy * c->res;
  free(h);
  free(v);
  free(va);
  free(a);
  free(r);
  for (int l = 0; l < c->n_layers; ++l) {
    free(L[l]);
    free(O[l]);
    free(LV[l]);
  }
}

/* ------------------------------------------------------------------------ */
/* image association (Sec. III-B): pinhole projection of cells and a        */
/* Bresenham walk over the height grid for the visibility check             */

/* All-octant integer Bresenham line from (sx, sy) to (ex, ey), both ends
 * included; writes up to `cap` (x, y) pairs and returns the cell count. */
int32_t orc_bresenham(int32_t sx, int32_t sy, int32_t ex, int32_t ey, int32_t *xy, int32_t cap) {
  int32_t dx = abs(ex - sx), dy = -abs(ey - sy);
  int32_t stx = sx < ex ? 1 : -1, sty = sy < ey ? 1 : -1;
  int32_t err = dx + dy, x = sx, y = sy, n = 0;
  for (;;) {
    if (n < cap) {
      xy[2 * n] = x;
      xy[2 * n + 1] = y;
    }
    ++n;
    if (x == ex && y == ey) break;
    int32_t e2 = 2 * err;
    if (e2 >= dy) {
      err += dy;
      x += stx;
    }
    if (e2 <= dx) {
      err += dx;
      y += sty;
    }
  }
  return n;
}

int64_t orc_fuse_image(const orc_cfg *c, orc_state *s, int32_t H, int32_t Wi, int32_t n_src,
                       const orc_src *src, const double K[4], const double T[16], uint8_t *vis,
                       int32_t *pix) {
  int W = c->W;
  int64_t W2 = (int64_t)W * W;
  /* map -> camera transform: R_cm = R_mc^T, t_cm = -R_mc^T (t_mc - o) */
  double d[3] = {T[3] - s->origin[0], T[7] - s->origin[1], T[11]};
  float R[9], t[3];
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 3; ++k) R[r * 3 + k] = (float)T[k * 4 + r];
    t[r] = (float)(-(T[0 * 4 + r] * d[0] + T[1 * 4 + r] * d[1] + T[2 * 4 + r] * d[2]));
  }
  float fx = (float)K[0], fy = (float)K[1], cx = (float)K[2], cy = (float)K[3];
  float res = (float)c->res;
  /* camera cell (clamped to the map) and camera height */
  float hc = (float)d[2];
  int32_t sx, sy;
  clamped_cell(c, (float)d[0], (float)d[1], &sx, &sy);
  /* decide every cell against the heights before this image */
  double *h0 = malloc((size_t)W2 * sizeof(double));
  for (int64_t j = 0; j < W2; ++j) h0[j] = s->h[j];
  int32_t *line = malloc((size_t)(4 * W + 8) * sizeof(int32_t));
  double *S = malloc(sizeof(double) * 4096);
  int64_t n_vis = 0;
  for (int32_t iy = 0; iy < W; ++iy)
    for (int32_t ix = 0; ix < W; ++ix) {
      int64_t j = (int64_t)iy * W + ix;
      if (vis) vis[j] = 0;
      if (pix) pix[j] = -1;
      if (!s->valid[j]) continue;
      float xc = ((float)(ix - W / 2) + 0.5f) * res;
      float yc = ((float)(iy - W / 2) + 0.5f) * res;
      float hz = (float)h0[j];
      float Xc = fmaf(R[0], xc, fmaf(R[1], yc, fmaf(R[2], hz, t[0])));
      float Yc = fmaf(R[3], xc, fmaf(R[4], yc, fmaf(R[5], hz, t[1])));
      float Zc = fmaf(R[6], xc, fmaf(R[7], yc, fmaf(R[8], hz, t[2])));
      if (!(Zc > c->z_near)) continue;
      float u = fmaf(fx, Xc / Zc, cx);
      float v = fmaf(fy, Yc / Zc, cy);
      float fu = floorf(u + 0.5f), fv = floorf(v + 0.5f);
      if (!(fu >= 0.0f && fu < (float)Wi && fv >= 0.0f && fv < (float)H)) continue;
      /* visible iff every valid intermediate cell lies strictly below the ray
         from the camera to the cell */
      int32_t dxs = ix - sx, dys = iy - sy;
      int32_t den = dxs * dxs + dys * dys;
      int32_t n = orc_bresenham(sx, sy, ix, iy, line, 2 * W + 4);
      int visible = 1;
      for (int32_t m = 1; m + 1 < n; ++m) {
        int32_t qxi = line[2 * m], qyi = line[2 * m + 1];
        int64_t q = (int64_t)qyi * W + qxi;
        if (!s->valid[q]) continue;
        int32_t num = (qxi - sx) * dxs + (qyi - sy) * dys;
        float tq = (float)num / (float)den;
        float ray = fmaf(tq, hz - hc, hc);
        if ((float)h0[q] >= ray) {
          visible = 0;
          break;
        }
      }
      if (!visible) continue;
      int32_t px = (int32_t)fu, py = (int32_t)fv;
      int64_t p = (int64_t)py * Wi + px;
      if (vis) vis[j] = 1;
      if (pix) pix[j] = (int32_t)p;
      ++n_vis;
      for (int qs = 0; qs < n_src; ++qs) {
        int C = src[qs].channels;
        for (int k = 0; k < C; ++k) S[k] = load_val(&src[qs], p, k);
        for (int b = 0; b < src[qs].n_layers; ++b)
          apply_rule(c, s, src[qs].layers[b], j, 1.0, S, S);
      }
    }
  free(h0);
  free(line);
  free(S);
  return n_vis;
}

/* ------------------------------------------------------------------------ */
/* harmonic (diffusion) fill of unknown cells                               */

/* Unknown cells solve the discrete Laplace equation: each equals the mean of
 * its in-grid 4-neighbours (zero-flux border); known cells are fixed.
 * Gauss-Seidel sweeps in row-major order until the largest residual is below
 * tol. Returns the sweep count. */
int32_t orc_harmonic_fill(int32_t H, int32_t W, double *h, const uint8_t *known, double tol,
                          int32_t max_sweeps, double *residual) {
  int32_t it;
  double r = INFINITY;
  for (it = 0; it < max_sweeps && r > tol; ++it) {
    for (int32_t y = 0; y < H; ++y)
      for (int32_t x = 0; x < W; ++x) {
        int64_t j = (int64_t)y * W + x;
        if (known[j]) continue;
        double s = 0.0;
        int m = 0;
        if (x > 0) s += h[j - 1], ++m;
        if (x + 1 < W) s += h[j + 1], ++m;
        if (y > 0) s += h[j - W], ++m;
        if (y + 1 < H) s += h[j + W], ++m;
        h[j] = s / m;
      }
    r = 0.0;
    for (int32_t y = 0; y < H; ++y)
      for (int32_t x = 0; x < W; ++x) {
        int64_t j = (int64_t)y * W + x;
        if (known[j]) continue;
        double s = 0.0;
        int m = 0;
        if (x > 0) s += h[j - 1], ++m;
        if (x + 1 < W) s += h[j + 1], ++m;
        if (y > 0) s += h[j - W], ++m;
        if (y + 1 < H) s += h[j + W], ++m;
        double e = fabs(s / m - h[j]);
        if (e > r) r = e;
      }
  }
  if (residual) *residual = r;
  return it;
}

/* ------------------------------------------------------------------------ */
/* surface normals of the elevation layer                                   */

/* Slope along one axis at a cell from its two neighbours (a = lower index,
 * b = higher index) in binary32: central difference over 2 res when both are
 * valid, one-sided over res with the cell itself when one is. Returns 0 when
 * neither neighbour is valid. */
static int axis_slope(float hm, int va, float ha, int vb, float hb, float res, float *g) {
  if (va && vb) {
    *g = (hb - ha) / (2.0f * res);
    return 1;
  }
  if (vb) {
    *g = (hb - hm) / res;
    return 1;
  }
  if (va) {
    *g = (hm - ha) / res;
    return 1;
  }
  return 0;
}

void orc_normals(const orc_cfg *c, const orc_state *s, float *out, uint8_t *ok) {
  int W = c->W;
  float res = (float)c->res;
  for (int32_t iy = 0; iy < W; ++iy)
    for (int32_t ix = 0; ix < W; ++ix) {
      int64_t j = (int64_t)iy * W + ix;
      out[3 * j] = out[3 * j + 1] = out[3 * j + 2] = 0.0f;
      ok[j] = 0;
      if (!s->valid[j]) continue;
      float hm = (float)s->h[j];
      int vl = ix > 0 && s->valid[j - 1], vr = ix + 1 < W && s->valid[j + 1];
      int vd = iy > 0 && s->valid[j - W], vu = iy + 1 < W && s->valid[j + W];
      float gx, gy;
      if (!axis_slope(hm, vl, vl ? (float)s->h[j - 1] : 0.0f, vr, vr ? (float)s->h[j + 1] : 0.0f, res, &gx)) continue;
      if (!axis_slope(hm, vd, vd ? (float)s->h[j - W] : 0.0f, vu, vu ? (float)s->h[j + W] : 0.0f, res, &gy)) continue;
      float n2 = fmaf(gx, gx, fmaf(gy, gy, 1.0f));
      float inv = 1.0f / sqrtf(n2);
      out[3 * j] = -gx * inv;
      out[3 * j + 1] = -gy * inv;
      out[3 * j + 2] = inv;
      ok[j] = 1;
    }
}
