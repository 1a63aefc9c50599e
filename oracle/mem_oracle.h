/* Plain CPU oracle of MEM's map-update path (arXiv 2309.16818).
 *
 * TEST INFRASTRUCTURE ONLY: this code exists to check the CUDA library. Only
 * the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load it. It shares no code, header, table or helper with the CUDA path.
 *
 * Conventions (the paper is silent on them; the readings are listed in the
 * design notes):
 *   - maps are W x W cells (W even) of side res; cell (ix, iy) covers
 *     x in [(ix - W/2) res, (ix - W/2 + 1) res) relative to the map centre o;
 *     cell index j = iy * W + ix;
 *   - every per-point / per-cell DECISION (cell index, gate, frustum, pixel,
 *     occlusion) is a fixed sequence of IEEE binary32 operations with
 *     explicit fmaf; every SUM is accumulated in binary64;
 *   - state is kept in binary64 arrays; with round_store set, each stored
 *     value is rounded to its storage precision after each update (binary32
 *     for geometric layers, the layer's own format for multi-modal layers),
 *     which is what a map held in device memory keeps between scans.
 */
#ifndef MEM_ORACLE_H
#define MEM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_LAYERS 16
#define ORC_MAX_SRC_LAYERS 8

enum { ORC_LATEST = 0, ORC_EXPAVG = 1, ORC_GAUSS = 2, ORC_DIRICHLET = 3, ORC_CLASSMAX = 4 };
enum { ORC_F32 = 0, ORC_BF16 = 1, ORC_F16 = 2, ORC_U8 = 3 };

typedef struct {
  int32_t W;
  int32_t n_layers;
  double res;
  float sigma0, sigma1;       /* measurement std  s = sigma0 + sigma1 * range          */
  float gate_lambda;          /* Mahalanobis gate on the height update                 */
  float outlier_var;          /* variance added per rejected point                     */
  float time_var;             /* variance added to every valid cell per scan           */
  float range_min, range_max; /* sensor-range filter                                   */
  float z_near;               /* camera near plane                                     */
  int32_t round_store;        /* 1: round stored values to their storage precision     */
  int32_t channels[ORC_MAX_LAYERS]; /* K or d of the layer                             */
  int32_t rule[ORC_MAX_LAYERS];
  int32_t store[ORC_MAX_LAYERS];    /* ORC_F32 / ORC_BF16 / ORC_F16                    */
  double w[ORC_MAX_LAYERS];         /* exponential-averaging weight                    */
  double var_meas[ORC_MAX_LAYERS];  /* Gaussian rule: known observation variance       */
  double alpha0[ORC_MAX_LAYERS];    /* Dirichlet rule: prior concentration per class   */
  /* drift compensation (Table I "drift compensation"): 0 = off; else the valid heights move
     by drift_alpha times the mean height error of the gate-accepted points in valid cells,
     when at least drift_min_points such points exist */
  double drift_alpha;
  int32_t drift_min_points;
  /* ray-cast clean-up (Table I "height update & ray cast"): 1 = on; a valid cell that a
     gate-accepted point's sensor ray passes more than ray_margin below, and that accepts no
     point of the call, becomes invalid */
  int32_t ray_cleanup;
  float ray_margin;
} orc_cfg;

/* Map state; every array is owned by the caller (W*W cells, or W*W*S values
 * for a layer of S stored values per cell). */
typedef struct {
  double *h, *var;
  uint8_t *valid;
  uint32_t *n_acc, *n_rej;
  double *layer[ORC_MAX_LAYERS]; /* LATEST/EXPAVG/GAUSS: C values; DIRICHLET: alpha (K);
                                    CLASSMAX: 2 values (class id, confidence)            */
  double *lvar[ORC_MAX_LAYERS];  /* GAUSS: per-cell, per-dimension variance (C values)  */
  uint8_t *obs[ORC_MAX_LAYERS];  /* 1 once the layer of that cell has been observed     */
  double origin[2];              /* world xy of the map centre                          */
} orc_state;

/* One input source: a row of `channels` values per point (or per pixel, HWC)
 * fused into each of `layers`. With topk > 0 (class probabilities given as the
 * top k classes, Sec. III-C) a row is instead topk pairs (class id, probability)
 * of float32 (dtype ORC_F32), and `channels` is the class count K: the point
 * stands for the K-vector that holds each listed probability at its class (ids
 * that are not whole numbers in [0, K) are ignored; a repeated id adds up, in
 * float32, in row order) and zero elsewhere. */
typedef struct {
  const void *data;
  int32_t dtype;
  int32_t channels;
  int32_t n_layers;
  int32_t layers[ORC_MAX_SRC_LAYERS];
  int32_t topk;
} orc_src;

void orc_init_state(const orc_cfg *c, orc_state *s);
void orc_pose_rel(const double T[16], const double origin[2], float Rt[12]);
int orc_point_cell(const orc_cfg *c, const float Rt[12], const float p[3], int32_t *cell,
                   float *z, float *vm);
int64_t orc_fuse_points(const orc_cfg *c, orc_state *s, int64_t n, const float *xyz, int32_t n_src,
                        const orc_src *src, const double T[16], uint8_t *near_gate,
                        int32_t *cell_out);
/* Diagnostics of the last orc_fuse_points call on this thread: drift shift applied (m),
   number of points that entered the mean error, cells cleared by the ray cast. */
void orc_last_fuse_info(double *drift, int64_t *drift_points, int64_t *cleared);
void orc_move(const orc_cfg *c, orc_state *s, const double robot_xy[2]);
int32_t orc_bresenham(int32_t sx, int32_t sy, int32_t ex, int32_t ey, int32_t *xy, int32_t cap);
int64_t orc_fuse_image(const orc_cfg *c, orc_state *s, int32_t H, int32_t Wi, int32_t n_src,
                       const orc_src *src, const double K[4], const double T[16], uint8_t *vis,
                       int32_t *pix);
/* Surface normals of the elevation layer (Table I "normal calculation"; the reading is in
   the design notes): out[j] = (-gx, -gy, 1) / |(-gx, -gy, 1)|, with slopes from central
   differences of the valid logical neighbours (one-sided where one is missing);
   ok[j] = 0 where the cell is invalid or has no valid neighbour along x or along y. */
void orc_normals(const orc_cfg *c, const orc_state *s, float *out, uint8_t *ok);
int32_t orc_harmonic_fill(int32_t H, int32_t W, double *h, const uint8_t *known, double tol,
                          int32_t max_sweeps, double *residual);

#ifdef __cplusplus
}
#endif
#endif
