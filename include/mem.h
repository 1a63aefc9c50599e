/* mem.h — C ABI of the GB300 multi-modal elevation-mapping library.
 *
 * Implements the data-parallel map update of "MEM: Multi-Modal Elevation
 * Mapping for Robotics and Learning" (arXiv 2309.16818):
 *   - Sec. III-B (Data association): points -> cells by their horizontal
 *     coordinates; cells -> pixels by pinhole projection with a Bresenham
 *     visibility check against the height map;
 *   - the height update the paper inherits from its predecessor (per-cell
 *     Kalman update with an outlier gate, Table I rows "point trsf. & z err.
 *     cnt" and "height update");
 *   - Sec. III-C (Fusion algorithms): Latest (Eq. 1), Exponential averaging
 *     (Eq. 2), Gaussian Bayesian inference (Eqs. 3-7), Dirichlet Bayesian
 *     inference (Eqs. 8-12), and a class-max layer (the most probable
 *     class of a cell, which Sec. V-B uses to colour the semantic map).
 *
 * Memory and streams
 *   - The library owns every map's device memory (allocated in
 *     mem_create_map, freed in mem_destroy_map).
 *   - Every other pointer argument is caller-owned DEVICE memory unless the
 *     argument says "host"; it must stay valid until the work queued on
 *     `stream` has finished. The library never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). All calls are asynchronous on that stream. Calls on one map
 *     must be ordered (issue them on one stream, or order them yourself).
 *   - Layouts: points are float32 xyz rows [N][3] in the SENSOR frame; a
 *     point source is [N][C] rows; an image source is HWC [H][Wi][C]; poses
 *     are row-major 4x4 float64 (host) mapping sensor (or optical camera:
 *     x right, y down, z forward) coordinates to world coordinates.
 *
 * Errors
 *   - Argument errors are detected on the host before anything is queued;
 *     they change no state and return MEM_ERR_ARG.
 *   - CUDA launch errors return MEM_ERR_CUDA.
 *   - Device-side failures (a bounded wait that ran out) set an error word in
 *     the map; mem_check() synchronises and reports it as MEM_ERR_TIMEOUT.
 *   - mem_last_error() returns a thread-local message for the last failure.
 */
#ifndef MEM_H
#define MEM_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MEM_MAX_LAYERS 16
#define MEM_MAX_SOURCES 8
#define MEM_MAX_SOURCE_LAYERS 8

typedef struct mem_map mem_map; /* opaque */

typedef enum {
  MEM_OK = 0,
  MEM_ERR_ARG = 1,
  MEM_ERR_CUDA = 2,
  MEM_ERR_OOM = 3,
  MEM_ERR_TIMEOUT = 4,
  MEM_ERR_STATE = 5
} mem_status;

/* Per-layer fusion rule (Sec. III-C). For a point cloud, the N_j points of
 * cell j in one call are one observation set; for an image, N_j = 1.
 *   LATEST    theta = mean of the observations (Eq. 1)
 *   EXPAVG    theta = w * mean + (1 - w) * theta_prev (Eq. 2); the first
 *             observation of a cell sets theta = mean
 *   GAUSS     mu, sigma^2 of the conjugate Gaussian update with known
 *             observation variance var_meas (Eqs. 6-7); the first observation
 *             has an infinitely wide prior (mu = mean, sigma^2 = var_meas / N)
 *   DIRICHLET alpha += sum of the observations (Eq. 12), alpha starts at
 *             alpha0; the class probabilities are alpha / sum(alpha) (Eq. 11)
 *   CLASSMAX  (class id, confidence) of the largest class probability seen in
 *             this call, smallest class index on ties; replaces the cell */
typedef enum {
  MEM_RULE_LATEST = 0,
  MEM_RULE_EXPAVG = 1,
  MEM_RULE_GAUSS = 2,
  MEM_RULE_DIRICHLET = 3,
  MEM_RULE_CLASSMAX = 4
} mem_rule;

typedef enum { MEM_F32 = 0, MEM_BF16 = 1, MEM_F16 = 2, MEM_U8 = 3 } mem_dtype;

/* A multi-modal layer (Sec. III-A: a layer that holds data of any modality).
 * channels = K classes or d feature dimensions of the observations.
 * dtype    = storage of the layer values (MEM_F32, MEM_BF16 or MEM_F16);
 *            accumulation is float32 whatever the storage. CLASSMAX and
 *            DIRICHLET layers must be MEM_F32. */
typedef struct {
  int32_t channels;
  int32_t dtype;
  int32_t rule;
  float w;        /* EXPAVG weight of the new observation                 */
  float var_meas; /* GAUSS known observation variance sigma_f^2           */
  float alpha0;   /* DIRICHLET prior concentration per class              */
} mem_layer_desc;

/* Map configuration. W even, 2 <= W <= 16384; n_maps >= 1 maps of the same
 * shape live in one object (the batched path). Height model: measurement
 * std s = sigma0 + sigma1 * range; a point is an outlier of a valid cell
 * when (z - h)^2 > gate_lambda^2 (sigma_h^2 + s^2). */
typedef struct {
  int32_t W;
  int32_t n_maps;
  double res;      /* cell side (m); cells use float32(res), moves use res */
  int32_t n_layers;
  mem_layer_desc layers[MEM_MAX_LAYERS];
  float sigma0, sigma1;
  float gate_lambda;
  float outlier_var; /* added to sigma_h^2 per rejected point              */
  float time_var;    /* added to sigma_h^2 of every valid cell per call    */
  float range_min, range_max;
  float z_near;      /* camera near plane (m)                              */
  int64_t max_points; /* initial point capacity of the per-call scratch    */
  /* Drift compensation (Table I "drift compensation"; the step is defined in
   * the predecessor paper, this is the library's reading): 0 = off. Else,
   * before the height update, the mean height error z - h of the points
   * whose cell is valid and whose outlier gate accepts them (against the
   * state before the call) is taken per map; when at least drift_min_points
   * points enter it, every valid height of that map moves by
   * float32(drift_alpha * mean), so the map follows the new cloud and the
   * height update gates against the moved map. */
  double drift_alpha;
  int32_t drift_min_points;
  /* Ray-cast clean-up (the "ray cast" of Table I's "height update & ray
   * cast"; the library's reading of the predecessor's step): 1 = on. Every
   * point its cell's gate accepts casts the ray from the sensor (the pose's
   * translation; its cell clamped into the map) to the point along the
   * Bresenham line of cells, both ends excluded; an intermediate cell that
   * was valid and whose height exceeds the ray height there by more than
   * ray_margin (m) is passed below, and if it accepted no point of the call
   * it becomes invalid (stale obstacle removed). Runs after the height
   * update, before the time variance. */
  int32_t ray_cleanup;
  float ray_margin;
} mem_map_config;

/* One input source: a row of `channels` values per point (point clouds) or
 * per pixel (images), fused into each listed layer in order.
 * Top-k class input (Sec. III-C: class probabilities may be given as the top
 * k classes, which saves memory when there are many classes): with topk > 0
 * a row is instead topk pairs (class id, probability), 2 * topk float32
 * values (dtype MEM_F32), and `channels` is the class count K of the layers
 * the source feeds. The row stands for the K-vector holding each listed
 * probability at its class and zero elsewhere; ids that are not whole numbers
 * in [0, K) are ignored, a repeated id adds up (float32, in row order). */
#define MEM_MAX_TOPK 16
typedef struct {
  const void *data; /* device; [N][channels] or [H][Wi][channels]            */
  int32_t dtype;    /* mem_dtype of the rows                                 */
  int32_t channels;
  int32_t n_layers;
  int32_t layers[MEM_MAX_SOURCE_LAYERS];
  int32_t topk;     /* 0: dense rows; 1..MEM_MAX_TOPK: rows of topk pairs    */
} mem_source;

/* Geometric layer ids for mem_get_layer / mem_set_layer (part ignored). */
#define MEM_LAYER_HEIGHT (-1)   /* float32 elevation h                    */
#define MEM_LAYER_VARIANCE (-2) /* float32 elevation variance sigma_h^2   */
#define MEM_LAYER_VALID (-3)    /* uint8 1 once a height was fused        */
#define MEM_LAYER_NACC (-4)     /* uint32 accepted points, cumulative     */
#define MEM_LAYER_NREJ (-5)     /* uint32 rejected (outlier) points       */

/* Parts of a multi-modal layer. */
#define MEM_PART_VALUE 0    /* storage dtype, S values per cell (S = channels;
                               CLASSMAX: 2 = {class id as float, confidence}) */
#define MEM_PART_THETA 1    /* DIRICHLET: float32 alpha / sum(alpha), K per cell */
#define MEM_PART_VAR 2      /* GAUSS: float32 sigma^2, one per cell            */
#define MEM_PART_OBSERVED 3 /* uint8, 1 once the layer of the cell was fused   */

/* Create `cfg->n_maps` maps centred on the world origin, every cell empty.
 * The map is the 2.5D grid of Sec. III-A: pure geometric layers (elevation,
 * its variance, validity, the accepted / rejected point counts of the
 * predecessor's height update) plus the configured multi-modal layers, which hold
 * information of any modality, each bound to one fusion rule of Sec. III-C. Layout in HBM: planar arrays of n_maps * W * W cells.
 * Allocates synchronously on the current device (no stream); the library owns
 * the memory until mem_destroy_map. Returns MEM_ERR_ARG for an invalid config
 * (nothing allocated), MEM_ERR_OOM if device memory runs out. */
mem_status mem_create_map(const mem_map_config *cfg, mem_map **out);
mem_status mem_destroy_map(mem_map *m);

/* Robot-centric re-centring (Sec. I and III-A: the map is centred on the
 * robot and moves with it): shift map `map_index` by whole cells so its centre
 * is the cell centre nearest to robot_xy (host, float64 world metres); the
 * shift is round((robot - origin) / res) per axis; cells that enter are reset
 * to every layer's initial state. O(entering cells) on the device (ring-buffer
 * offsets). Errors: MEM_ERR_ARG (bad index, non-finite or huge move; state
 * unchanged), MEM_ERR_CUDA. */
mem_status mem_move_map(mem_map *m, int32_t map_index, const double robot_xy[2], void *stream);

/* Fuse one point cloud into a single-map object (n_maps == 1): Sec. III-B
 * (a point is associated to the cell under its horizontal coordinates, and
 * updates the elevation following the predecessor paper -- Table I rows
 * "point trsf. & z err. cnt" and "height update") and Sec. III-C (each
 * source's channels are fused into its layers by the layer's rule, Eqs. 1-12;
 * the N_j points of a cell in one call are one observation set).
 *   n        number of points (0 allowed), n < 2^30
 *   xyz      device float32 [n][3], sensor frame; non-finite rows are dropped
 *   sources  host array of n_sources (<= MEM_MAX_SOURCES) descriptors whose
 *            `data` are device [n][channels] rows
 *   T_map_sensor host float64 4x4 sensor -> world
 * A layer may be listed by at most one source of a call (else MEM_ERR_ARG).
 * Steps: transform + range filter + cell key; stable radix sort of the keys;
 * per-cell height update with outlier gate; per-layer fusion rules. */
mem_status mem_fuse_pointcloud(mem_map *m, int64_t n, const float *xyz, int32_t n_sources,
                               const mem_source *sources, const double T_map_sensor[16],
                               void *stream);

/* Same as mem_fuse_pointcloud with HOST buffers: xyz and every source's
 * `data` are host memory (page-locked, e.g. cudaHostAlloc, for the upload to
 * run asynchronously; pageable memory works but the host waits for its copy).
 * The library copies them into one of two device staging buffers it owns,
 * used in turn, on a copy stream of its own; the kernels wait for that copy
 * on `stream`. The host buffers must stay unchanged until the call's work on
 * `stream` has completed. Consecutive calls overlap one call's upload with
 * the previous call's kernels. Errors as mem_fuse_pointcloud. */
mem_status mem_fuse_pointcloud_host(mem_map *m, int64_t n, const float *xyz, int32_t n_sources,
                                    const mem_source *sources, const double T_map_sensor[16],
                                    void *stream);

/* Fuse n_maps independent clouds into the n_maps maps of one object in one
 * pass: the same per-map update as mem_fuse_pointcloud (Sec. III-B, III-C),
 * for many maps at once (independent robots or simulated environments; the
 * paper fuses one map). offsets: host int64 [n_maps + 1] CSR offsets into xyz
 * and the source rows (device, as for mem_fuse_pointcloud); T_map_sensor:
 * host float64 [n_maps][16]. Results equal n_maps separate single-map fuses.
 * Errors as mem_fuse_pointcloud; offsets must start at 0 and not decrease. */
mem_status mem_fuse_pointcloud_batch(mem_map *m, const int64_t *offsets, const float *xyz,
                                     int32_t n_sources, const mem_source *sources,
                                     const double *T_map_sensor, void *stream);

/* Fuse one camera image (Sec. III-B, Fig. 2): every valid cell of map
 * `map_index` is projected at its height into the pinhole camera
 * K = {fx, fy, cx, cy} (host) with pose T_map_cam (host, optical frame ->
 * world); it is visible iff in front of z_near, inside the image, and every
 * valid cell on the Bresenham line from the camera's cell lies strictly
 * below the ray. Visible cells fuse their pixel (one observation).
 * vis_out (uint8 [W*W]) and pix_out (int32 [W*W], py*Wi+px or -1) are
 * optional device outputs in logical cell order (row iy, column ix). The map
 * allocates a list of W*W cells (12 bytes each) on the first call, which
 * synchronises the stream. */
mem_status mem_fuse_image(mem_map *m, int32_t map_index, int32_t H, int32_t Wi, int32_t n_sources,
                          const mem_source *sources, const double K[4], const double T_map_cam[16],
                          uint8_t *vis_out, int32_t *pix_out, void *stream);

/* Copy one layer (part) of map `map_index` into device memory `dst`, in
 * logical cell order (cell j = iy * W + ix, values per cell contiguous): the
 * map's layers as the plugins of Sec. III-D and external consumers read them.
 * MEM_PART_THETA of a DIRICHLET layer is the posterior mean alpha / sum(alpha)
 * (Eq. 11). An unobserved cell reads as its layer's initial state. dst is
 * caller-owned, sized W*W*values*element size; asynchronous on `stream`.
 * Errors: MEM_ERR_ARG for a bad index, layer or part (nothing queued). */
mem_status mem_get_layer(mem_map *m, int32_t map_index, int32_t layer, int32_t part, void *dst,
                         void *stream);
/* Inverse of mem_get_layer (MEM_PART_THETA not settable): checkpoint restore
 * and test fixtures. */
mem_status mem_set_layer(mem_map *m, int32_t map_index, int32_t layer, int32_t part,
                         const void *src, void *stream);
/* World xy of the centre of map `map_index` (host output). */
mem_status mem_get_origin(const mem_map *m, int32_t map_index, double out_xy[2]);
/* Synchronise `stream` and report (then clear) the map's device error word.
 * While the word is set, the point path's kernels of this map return without
 * work (the map state is left as it was), so a failed call changes nothing. */
mem_status mem_check(mem_map *m, void *stream);

/* Fault injection for tests (no GPU fault, trap or hang): with
 * MEM_FAULT_SORT_WAIT, every wait of the radix sort's look-back treats its
 * predecessor as not ready, so the bounded wait runs out (a few seconds),
 * the error word is set and the rest of the call does nothing; mem_check then
 * returns MEM_ERR_TIMEOUT. MEM_FAULT_NONE restores normal operation.
 * Synchronises the device. */
typedef enum { MEM_FAULT_NONE = 0, MEM_FAULT_SORT_WAIT = 1 } mem_fault;
mem_status mem_inject_fault(mem_map *m, int32_t kind);

/* Schedule of the point path (results equal within float32 summation order;
 * each schedule is deterministic): radix_bits in [8, 10] is the digit width
 * of the key sort (at most 4 passes); blocks_per_sm in [1, 32] sizes the
 * persistent grids; fuse_kernel 0 sums a call's per-cell quantities in
 * registers, one point per lane (when its summed columns, 4 height sums plus
 * every source's channels and arg-max pair, number at most 32), 1 always in
 * shared-memory column walks over 128-point tiles. Synchronises the device. */
mem_status mem_set_tuning(mem_map *m, int32_t radix_bits, int32_t blocks_per_sm, int32_t fuse_kernel);
/* out = {radix_bits, blocks_per_sm, radix passes, fuse_kernel} (host). */
mem_status mem_get_tuning(const mem_map *m, int32_t out[4]);

/* Autotuner: times every schedule candidate (fuse_kernel in {0, 1},
 * radix_bits in {8, 9, 10}, blocks_per_sm in {2, 4, 8}) on this batched call (arguments as for
 * mem_fuse_pointcloud_batch), `reps` timed runs each from the same saved map
 * state, keeps the fastest and restores the state, so the map is unchanged.
 * Allocates a temporary copy of the map state. ms_out (host, optional) gets
 * the mean time of each candidate tried; *n_out (host, optional) its capacity
 * on entry and the number of candidates tried on return. Synchronises. */
mem_status mem_autotune_batch(mem_map *m, const int64_t *offsets, const float *xyz, int32_t n_sources,
                              const mem_source *sources, const double *T_map_sensor, int32_t reps,
                              void *stream, float *ms_out, int32_t *n_out);

/* Per-kernel timing: with profiling on, every launch group of this map is
 * bracketed by CUDA events on its stream (graph replay is then disabled).
 * mem_get_profile waits for the recorded events and returns, per slot, the
 * summed milliseconds and the number of launches since the previous read:
 * 0 transform+key, 1 digit scan, 2 radix passes, 3 segments, 4 short-cell
 * fuse, 5 long-cell fuse, 6 time variance, 7 image fuse, 8 move, 9 drift
 * compensation, 10 ray-cast clean-up. */
#define MEM_PROFILE_SLOTS 16
mem_status mem_set_profiling(mem_map *m, int32_t on);
mem_status mem_get_profile(mem_map *m, double ms[MEM_PROFILE_SLOTS], int64_t calls[MEM_PROFILE_SLOTS]);
/* Synchronise `stream`; out = {cells whose points cross a tile of 128
 * sorted points, touched cells, kept points, radix passes} of the last point
 * fuse (host output). */
mem_status mem_get_stats(mem_map *m, void *stream, int64_t out[4]);
/* Synchronise `stream`; out (host) = {drift shift applied to map map_index
 * by the last point fuse (m, 0 when off or too few points), points that
 * entered its mean error, cells of all maps invalidated by the last call's
 * ray-cast clean-up}. Table I rows "drift compensation" and "height update &
 * ray cast"; see mem_map_config. MEM_ERR_ARG for a bad index. */
mem_status mem_get_drift(mem_map *m, int32_t map_index, void *stream, double out[3]);

/* Post-processing plugins (Sec. III-D: plugins read the map layers already on
 * the GPU and produce new layers).
 *
 * Surface normals of the elevation layer of map `map_index` (Table I "normal
 * calculation"; the reading is this library's): per valid cell the slopes gx,
 * gy from central differences of its valid logical neighbours over 2 res, or
 * one-sided differences with the cell itself over res where one neighbour is
 * invalid or outside the map; normal = (-gx, -gy, 1) / |(-gx, -gy, 1)|.
 *   normals  device float32 [W*W][3] (out; 0 where there is no normal)
 *   ok       device uint8 [W*W] (out, optional): 1 where the cell is valid and
 *            has a valid neighbour along x and along y
 * Logical cell order (iy * W + ix). Asynchronous on `stream`. */
mem_status mem_compute_normals(mem_map *m, int32_t map_index, float *normals, uint8_t *ok, void *stream);

/* PCA layer of a feature layer (the plugin of Sec. III-D's figure that turns
 * feature layers into a PCA layer; the reading is this library's): over the
 * cells of map `map_index` where `layer` is observed, the mean m and the
 * covariance (1/n) sum (f - m)(f - m)^T of its values, the n_comp
 * eigenvectors of largest eigenvalue (each signed so that its
 * largest-magnitude component is positive), and every observed cell's
 * projections (f - m) . v_k (0 elsewhere).
 *   layer    any multi-modal layer but CLASSMAX, 1..128 channels
 *   n_comp   1..min(8, channels)
 *   proj     device float32 [W*W][n_comp] (out, logical cell order)
 *   info     device float32 (out, optional): n_comp eigenvalues, then the
 *            n_comp vectors [n_comp][channels], then the mean [channels]
 * Float32 sums per block added in float64; eigenvectors by Jacobi sweeps in
 * float32. The map owns a scratch buffer for it (allocated on the first call,
 * which synchronises the stream). MEM_ERR_ARG for bad indices or sizes. */
mem_status mem_pca_layer(mem_map *m, int32_t map_index, int32_t layer, int32_t n_comp, float *proj, float *info,
                         void *stream);

/* Diffusion (harmonic) inpainting of a batch of map crops, the fallback of the
 * learned inpainting and the reference it is judged against: each unknown
 * cell (known == 0) becomes the mean of its in-crop 4-neighbours (zero-flux
 * border) -- the discrete Laplace equation with the known cells as boundary
 * values; known cells are copied. Solved in float32 by red-black successive
 * over-relaxation from the mean of the crop's known cells, until the largest
 * update of a sweep is below tol or after max_iters sweeps. A crop whose rows
 * fit the shared memory of a thread-block cluster of up to 8 CTAs is solved
 * there (rows split over the cluster, the rows next to a CTA's band read from
 * the neighbouring CTAs' shared memory); larger crops in global memory.
 *   h_in, h_out  device float32 [n_crops][H][W] (may not alias)
 *   known        device uint8 [n_crops][H][W]
 *   iters_out    device int32 [n_crops] sweeps used (optional)
 * A group of unknown cells with no known cell around it keeps the mean. */
mem_status mem_inpaint_diffusion(int32_t n_crops, int32_t H, int32_t W, const float *h_in,
                                 const uint8_t *known, float *h_out, float tol, int32_t max_iters,
                                 int32_t *iters_out, void *stream);

/* Inputs of the inpainting network for a batch of map crops (Sec. III-D:
 * a plugin reads map layers and produces a new one; the normalisation is this
 * library's): per crop the mean m of the heights of its known cells (float64
 * sums, rounded once to float32; 0 for a crop without known cells), then per
 * cell the three input channels
 *   x3[.., 0] = fill - m, x3[.., 1] = hidden, x3[.., 2] = known ? 0.1 ln(1e-4) : 0
 * (observed cells carry a variance of 1e-4 m^2, the log-variance channel is
 * scaled by 0.1) and hidden = 1 - known.
 *   h_in, fill   device float32 [n_crops][H][W] (heights; the diffusion fill)
 *   known        device uint8 [n_crops][H][W] (1 = observed)
 *   x3           device float32 [n_crops][H][W][3] (out)
 *   hidden       device uint8 [n_crops][H][W] (out)
 *   mean_out     device float32 [n_crops] (out, optional)
 * MEM_ERR_ARG for NULL pointers or a bad shape (nothing queued). */
mem_status mem_unet_prepare(int32_t n_crops, int32_t H, int32_t W, const float *h_in, const uint8_t *known,
                            const float *fill, float *x3, uint8_t *hidden, float *mean_out, void *stream);

/* Learned inpainting (Sec. III-D: post-processing plugins may run neural
 * networks on map layers to produce a new layer; the network layout is this
 * library's): a U-Net over crops of map layers predicting a residual that is
 * added to the diffusion fill. Four levels of widths[0..3] channels, two 3x3
 * convolutions + ReLU per level, 2x2 max-pooling, nearest upsampling with
 * skip concatenation [upsampled, skip], a final 1x1 convolution. BF16
 * tensor-core kernels (tcgen05, accumulator in tensor memory) with float32
 * accumulation; float32 master weights.
 * Parameters (flat float32, in this order): for each 3x3 convolution
 * e1a e1b e2a e2b e3a e3b e4a e4b d3a d3b d2a d2b d1a d1b its weights
 * [3][3][C_in][C_out] then bias [C_out]; then the 1x1 weights [widths[0]] and
 * bias [1]. Crops are NHWC: x3 = float32 [n][H][W][cin] inputs, fill /
 * target / pred = float32 [n][H][W], hidden = uint8 [n][H][W] (1 = cell whose
 * value the loss scores); H and W multiples of 8. All pointers device. */
typedef struct mem_unet mem_unet;
mem_status mem_unet_create(int32_t cin, const int32_t widths[4], mem_unet **out);
mem_status mem_unet_destroy(mem_unet *u);
mem_status mem_unet_param_count(const mem_unet *u, int64_t *n);
mem_status mem_unet_set_params(mem_unet *u, const float *src, void *stream);
mem_status mem_unet_get_params(const mem_unet *u, float *dst, void *stream);
/* pred = fill + residual(x3) */
mem_status mem_unet_forward(mem_unet *u, int32_t n, int32_t H, int32_t W, const float *x3,
                            const float *fill, float *pred, void *stream);
/* loss = sum over hidden cells of (pred - target)^2 / n_hidden (device
 * float32, optional) and its gradient for every parameter into grads (flat,
 * optional) */
mem_status mem_unet_gradients(mem_unet *u, int32_t n, int32_t H, int32_t W, const float *x3,
                              const float *fill, const float *target, const uint8_t *hidden,
                              int64_t n_hidden, float *grads, float *loss, void *stream);
/* one Adam step (beta 0.9, 0.999) with learning rate lr on that loss */
mem_status mem_unet_train_step(mem_unet *u, int32_t n, int32_t H, int32_t W, const float *x3,
                               const float *fill, const float *target, const uint8_t *hidden,
                               int64_t n_hidden, float lr, float *loss, void *stream);
/* Synchronises the stream and reports a device-side failure of this net's
 * kernels (a bounded wait inside a convolution that ran out) as
 * MEM_ERR_TIMEOUT, clearing the error word; MEM_OK otherwise. */
mem_status mem_unet_check(mem_unet *u, void *stream);

/* Allocation-free height fuse. The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc -- code that runs inside
 * another framework's memory pool, real-time loops that forbid allocation
 * after start-up, hosts whose device allocator is owned by someone else.
 * It fuses one point cloud into caller-owned height layers (the height update
 * with outlier gate and the time-dependent variance growth of
 * mem_fuse_pointcloud, no multi-modal layers) and allocates nothing: no
 * cudaMalloc, cudaFree, pinned memory or allocating library routine. Its sort
 * and segment scratch is one file-scope device array sized for
 * MEM_NOALLOC_MAX_POINTS points (about 22 MB, held by every GPU that loads
 * the library until the process exits); the call's parameters reach the
 * device as kernel arguments.
 *   cfg       host; n_maps must be 1, n_layers 0, drift_alpha 0 and
 *             ray_cleanup 0; max_points is ignored
 *   origin_xy host; world xy of the map centre (cell W/2 lower corner)
 *   n         points, 0 <= n <= MEM_NOALLOC_MAX_POINTS (larger: MEM_ERR_ARG)
 *   xyz       device float32 [n][3], sensor frame
 *   h, var    device float32 [W*W] elevation and variance (cell iy*W + ix)
 *   valid     device uint32 [W*W], 1 once the cell holds a height, else 0
 *   n_acc, n_rej device uint32 [W*W] cumulative accepted / rejected points
 * The caller initialises the layers (all zero = empty map). The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) and
 * sets kernel attributes; make that first call before any stream capture.
 * Every call shares the one array and overwrites it: calls that overlap on
 * the GPU (other streams, other threads) race and must be serialised by the
 * caller. A call whose bounded device wait runs out leaves the layers as they
 * were and returns MEM_OK (the failure happens after the call returned); the
 * next call starts afresh, and mem_noalloc_check reports the failure. */
#define MEM_NOALLOC_MAX_POINTS (1 << 18)
mem_status mem_fuse_pointcloud_noalloc(const mem_map_config *cfg, const double origin_xy[2],
                                       int64_t n, const float *xyz, const double T_map_sensor[16],
                                       float *h, float *var, uint32_t *valid, uint32_t *n_acc,
                                       uint32_t *n_rej, void *stream);
/* Companion of mem_fuse_pointcloud_noalloc (no paper counterpart, allocates
 * nothing): synchronises `stream`, then returns MEM_ERR_TIMEOUT (and clears
 * the record) if an allocation-free fuse on the current device timed out in a
 * bounded device wait since the previous check, MEM_OK otherwise. */
mem_status mem_noalloc_check(void *stream);
/* Thread-local description of the last error. */
const char *mem_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
