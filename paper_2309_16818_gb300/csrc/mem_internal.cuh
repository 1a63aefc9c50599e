// Internal device-side structures and helpers of the mapping library.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mem.h"

namespace memk {

typedef uint32_t u32;
typedef uint64_t u64;

constexpr int kMaxLayers = MEM_MAX_LAYERS;
constexpr int kMaxSources = MEM_MAX_SOURCES;
constexpr int kMaxSrcLayers = MEM_MAX_SOURCE_LAYERS;
constexpr u32 kFlagValid = 1u;               // bit 0: height valid
constexpr u32 kSpinLimit = 1u << 22;         // bounded waits (x ~100 ns each)
constexpr int kDevErrTimeout = 1;
constexpr int kSortThreads = 512;            // threads of a radix-sort CTA (two per SM)
constexpr int kSortItems = 6;                // keys per thread
constexpr int kSortTile = kSortThreads * kSortItems;  // keys per radix tile (look-back unit)
constexpr int kFuseTile = 128;               // sorted points per tile of the fuse kernels
constexpr int kSlotHdr = 16;                 // words of a fuse slot before its channel sums
// fuse slot header: sum w, sum w z, accepted, rejected (floats), then (bits)
// cell key, points in the piece, used/begin/end bits, pre-call flags,
// height, variance, accepted and rejected counts
enum { kSlotKey = 4, kSlotN, kSlotBits, kSlotFl, kSlotH0, kSlotV0, kSlotNacc, kSlotNrej };
static_assert(kSlotHdr % 4 == 0 && kSlotKey % 4 == 0 && kSlotH0 % 4 == 0, "16-byte aligned header groups");

// words of the fuse scratch for `cap` points: two slots of `acc` words per
// tile (`acc` a multiple of 4, so every slot is 16-byte aligned)
__host__ __device__ constexpr int64_t fuse_scratch_words(int64_t cap, int acc) {
  return 2 * (cap / kFuseTile + 2) * (int64_t)acc;
}
// Per-layer static description (device copy of mem_layer_desc + derived).
struct LayerDev {
  int C;        // channels of the observations
  int S;        // stored values per cell
  int dtype;    // storage
  int rule;
  float w, one_minus_w, var_meas, alpha0;
  void* data;   // [cells][S]
  float* gvar;  // GAUSS: [cells]
};

// Everything about a map object that does not change between calls.
struct MapDev {
  int W, n_maps;
  u32 W2;        // W*W
  u32 sentinel;  // n_maps * W2: key of dropped points
  float res;
  float sigma0, sigma1, lam2, outlier_var, time_var, range_min, range_max, z_near;
  int n_layers;
  const LayerDev* L;  // [n_layers] in device memory (indexed at run time by the kernels)
  float* h;
  float* var;
  u32* flags;  // bit0 valid, bit (1 + l) layer l observed
  u32* n_acc;
  u32* n_rej;
  // scratch of the point path
  u32 *keys0, *keys1, *vals0, *vals1;
  u32* hist;        // [passes][radix] digit counts, then exclusive offsets
  u32* lookback;    // [passes][tiles][radix]
  u32* counters;    // [0..3] tile counters per pass, [4] crossing cells, [5] touched cells,
                    // [6] kept points, [7] [9] tile counters of the fuse kernels, [8] slots,
                    // [10] cells invalidated by the ray-cast clean-up
  float* partial;   // fuse scratch: tile slot bases, tile run counts, slots of acc words
  int64_t partial_cap;  // floats
  int* err;         // [0] device error word (bounded wait ran out), [1] fault injection for tests
  int64_t cap;      // point capacity of the scratch
  int64_t cap_tiles;
  // drift compensation (drift_alpha != 0) and ray-cast clean-up (ray_on)
  double drift_alpha;
  int drift_min;
  int ray_on;
  float ray_margin;
  float* perr;      // [cap] per point: z - h if it enters the mean height error, else NaN
  int drift_R;      // blocks per map of the drift reduction
  double* dpart;    // [n_maps][drift_R][2] partial sums and counts of the errors
  float* drift_out; // [n_maps][2] shift applied, points in the mean (as float bits of a u32)
  u64* zacc;        // [n_maps * W2] (call id << 32) | ~ordered(lowest accepted z of the call)
};

// Per-map, per-call parameters.
struct MapCall {
  float R[9];  // rotation (point path: sensor -> map; image path: map -> camera)
  float t[3];  // translation relative to the map centre
  int ring_x, ring_y;
  float cam_x, cam_y, cam_h;  // image path: camera position relative to the map centre
  float pad;
};

struct SrcDev {
  const void* data;
  int dtype, C, n_layers;
  int layers[kMaxSrcLayers];
  int vec_ok;        // data is 16-byte aligned: rows may be read with vector loads
  int has_classmax;  // a CLASSMAX layer is bound: track the arg-max
  int acc_off;       // offset of this source's sums (then maxima) in a partial record
  int topk;          // > 0: rows are topk (class id, probability) float32 pairs over C classes
  int unused;
};

constexpr int kFuseQ = 32;  // stage columns of the fuse kernel per round

// Up to four consecutive channels of one source that the fuse kernel stages
// together.
struct __align__(16) ChunkDesc {
  const void* data;
  int C, ch0;       // row length, first channel
  int col, n;       // first stage column, channels
  int dtype, vec;   // storage, 16-byte aligned rows
  int am;           // arg-max value column of the source (-1: none); bit 30: last chunk
  int src;
  int topk;         // > 0: the source's rows are topk (class id, probability) pairs
  int unused;
};

// Stage layout of the fuse kernel, built on the host for a call whose
// columns fit one round (one_round != 0); otherwise the kernel builds the
// column part round by round. The rule-layer lists hold for every call.
struct FuseTables {
  int ncol;  // columns of the call: 4 height sums, then per source C channels (+ arg-max pair)
  int one_round, n_ck, n_pair;
  int col_src[kFuseQ];  // per column: source (-1: height sums)
  int col_ch[kFuseQ];   // channel, -1 / -2 for a source's arg-max value / channel, or height sum
  ChunkDesc ck[kFuseQ];
  int pair_col[kMaxSources];  // arg-max value columns
  int qc0[kMaxSources], qch0[kMaxSources], qn[kMaxSources];  // per source: first column, channel, count
  int rlay[kMaxSources][kMaxSrcLayers];  // per source: its layers other than class max
  int nrlay[kMaxSources];
  int any_gauss;
};

// Per-call job of the point path, resident in device memory so the whole
// kernel sequence can be replayed from a CUDA graph.
struct PointJob {
  int64_t n;
  u32 call_id;  // increases by one per point-path call of a map object (never 0)
  const float* xyz;
  const int64_t* offsets;  // [n_maps + 1] or nullptr for one map
  const MapCall* maps;     // [n_maps]
  int n_maps;
  int n_src;
  int acc;  // words per fuse slot: kSlotHdr, then per source C sums (+ max value, class)
  SrcDev src[kMaxSources];
  FuseTables ft;
};

// ---------------------------------------------------------------------------
// numeric helpers: fixed IEEE sequences (never contracted by the compiler)

struct PointEval {
  float z, vm;
  int ix, iy;  // logical cell
  bool keep;
};

// Transform, filter and associate one sensor-frame point:
//   p = R p_s + t (fmaf chain), range = sqrt(xs^2 + ys^2 + zs^2),
//   cell = floor(x / res) + W/2, variance = (sigma0 + sigma1 range)^2.
__device__ __forceinline__ PointEval eval_point(const MapDev& md, const MapCall& mc, float xs,
                                                float ys, float zs) {
  PointEval e;
  e.keep = false;
  e.ix = e.iy = 0;
  e.z = e.vm = 0.f;
  if (!(isfinite(xs) && isfinite(ys) && isfinite(zs))) return e;
  float r2 = __fmaf_rn(xs, xs, __fmaf_rn(ys, ys, __fmul_rn(zs, zs)));
  float rs = __fsqrt_rn(r2);
  if (!(rs >= md.range_min && rs <= md.range_max)) return e;
  float x = __fmaf_rn(mc.R[0], xs, __fmaf_rn(mc.R[1], ys, __fmaf_rn(mc.R[2], zs, mc.t[0])));
  float y = __fmaf_rn(mc.R[3], xs, __fmaf_rn(mc.R[4], ys, __fmaf_rn(mc.R[5], zs, mc.t[1])));
  float z = __fmaf_rn(mc.R[6], xs, __fmaf_rn(mc.R[7], ys, __fmaf_rn(mc.R[8], zs, mc.t[2])));
  float qx = floorf(__fdiv_rn(x, md.res));
  float qy = floorf(__fdiv_rn(y, md.res));
  float half = (float)(md.W / 2);
  if (!(qx >= -half && qx < half && qy >= -half && qy < half)) return e;
  float sm = __fmaf_rn(md.sigma1, rs, md.sigma0);
  e.ix = (int)qx + md.W / 2;
  e.iy = (int)qy + md.W / 2;
  e.z = z;
  e.vm = __fmul_rn(sm, sm);
  e.keep = true;
  return e;
}

__device__ __forceinline__ u32 phys_cell(const MapDev& md, const MapCall& mc, int ix, int iy) {
  int px = ix + mc.ring_x;
  if (px >= md.W) px -= md.W;
  int py = iy + mc.ring_y;
  if (py >= md.W) py -= md.W;
  return (u32)py * (u32)md.W + (u32)px;
}

// Outlier gate of the height update: reject iff (z - h)^2 > lambda^2 (var_h + vm).
__device__ __forceinline__ bool gate_reject(float z, float h, float var_h, float vm, float lam2) {
  float d = __fsub_rn(z, h);
  float lhs = __fmul_rn(d, d);
  float rhs = __fmul_rn(lam2, __fadd_rn(var_h, vm));
  return lhs > rhs;
}

// ---------------------------------------------------------------------------
// loads / stores of source rows and layer values

__device__ __forceinline__ float ld_any(const void* base, int dtype, int64_t off) {
  switch (dtype) {
    case MEM_F32: return __ldg((const float*)base + off);
    case MEM_BF16: return __bfloat162float(((const __nv_bfloat16*)base)[off]);
    case MEM_F16: return __half2float(((const __half*)base)[off]);
    default: return (float)__ldg((const unsigned char*)base + off);
  }
}

// Class c of a row of top-k (class id, probability) pairs over C classes: the
// sum, in row order, of the probabilities listed for c (ids that are not whole
// numbers in [0, C) are ignored).
__device__ __forceinline__ float topk_val(const float* __restrict__ r, int k, int C, int c) {
  float v = 0.f;
  for (int j = 0; j < k; ++j) {
    const float id = __ldg(r + 2 * j);
    if (id >= 0.f && id < (float)C && id == floorf(id) && (int)id == c) v = __fadd_rn(v, __ldg(r + 2 * j + 1));
  }
  return v;
}

// channel c of row `row` of a source (dense or top-k rows)
__device__ __forceinline__ float src_val(const SrcDev& s, int64_t row, int c) {
  if (s.topk) return topk_val((const float*)s.data + row * 2 * s.topk, s.topk, s.C, c);
  return ld_any(s.data, s.dtype, row * s.C + c);
}

// Four consecutive channels c0..c0+3 of row `row` (channels >= C read as 0).
__device__ __forceinline__ void ld_src4(const SrcDev& s, int64_t row, int c0, float v[4]) {
  const int64_t off = row * s.C + c0;
  const int nc = min(4, s.C - c0);
  if (s.vec_ok && nc == 4 && (off & 3) == 0) {
    if (s.dtype == MEM_F32) {
      float4 q = __ldg((const float4*)((const float*)s.data + off));
      v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
      return;
    }
    if (s.dtype == MEM_BF16) {
      uint2 q = __ldg((const uint2*)((const __nv_bfloat16*)s.data + off));
      __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162*>(&q.x);
      __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&q.y);
      float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
      v[0] = fa.x; v[1] = fa.y; v[2] = fb.x; v[3] = fb.y;
      return;
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = k < nc ? ld_any(s.data, s.dtype, off + k) : 0.f;
}

__device__ __forceinline__ float ld_layer(const LayerDev& L, int64_t off) {
  switch (L.dtype) {
    case MEM_BF16: return __bfloat162float(((const __nv_bfloat16*)L.data)[off]);
    case MEM_F16: return __half2float(((const __half*)L.data)[off]);
    default: return ((const float*)L.data)[off];
  }
}

__device__ __forceinline__ void st_layer(const LayerDev& L, int64_t off, float v) {
  switch (L.dtype) {
    case MEM_BF16: ((__nv_bfloat16*)L.data)[off] = __float2bfloat16_rn(v); break;
    case MEM_F16: ((__half*)L.data)[off] = __float2half_rn(v); break;
    default: ((float*)L.data)[off] = v;
  }
}

// Per-(cell, layer) coefficients of a fusion rule for N observations, computed
// once per cell so that each channel costs one multiply-add:
//   LATEST    theta = S a                       (a = 1/N, Eq. 1)
//   EXPAVG    theta = w (S a) + (1 - w) theta   (first observation: S a, Eq. 2)
//   GAUSS     mu = a mu0 + b S with a = sf2/(N s02 + sf2), b = s02/(N s02 + sf2),
//             var = sf2 s02/(N s02 + sf2)        (first observation: mu = S/N,
//             var = sf2/N; Eqs. 6-7)
//   DIRICHLET alpha = alpha + S                 (Eq. 12)
struct RuleCoef {
  float a, b, var_new;
  bool obs;
};

__device__ __forceinline__ RuleCoef rule_coef(const LayerDev& L, float N, float rN, bool obs, float s02) {
  RuleCoef r;
  r.obs = obs;
  r.a = rN;
  r.b = 0.f;
  r.var_new = 0.f;
  if (L.rule == MEM_RULE_GAUSS) {
    if (obs) {
      const float rden = __frcp_rn(__fmaf_rn(N, s02, L.var_meas));
      r.a = L.var_meas * rden;
      r.b = s02 * rden;
      r.var_new = L.var_meas * s02 * rden;
    } else {
      r.var_new = L.var_meas * rN;
    }
  }
  return r;
}

// New value of one channel from its old value and the channel's sum S over
// the cell's observations (not CLASSMAX, which needs the whole row).
__device__ __forceinline__ float rule_value(const LayerDev& L, float old, float S, const RuleCoef& r) {
  switch (L.rule) {
    case MEM_RULE_LATEST: return S * r.a;
    case MEM_RULE_EXPAVG: {
      const float a = S * r.a;
      return r.obs ? fmaf(L.w, a, L.one_minus_w * old) : a;
    }
    case MEM_RULE_GAUSS: return r.obs ? fmaf(r.a, old, r.b * S) : S * r.a;
    case MEM_RULE_DIRICHLET: return (r.obs ? old : L.alpha0) + S;  // unobserved cell: prior alpha0
    default: return old;
  }
}

// the stored value is only read for an observed cell: an unobserved cell
// holds its layer's initial value whatever is in memory (lazy reset)
__device__ __forceinline__ bool needs_old(const LayerDev& L, const RuleCoef& r) {
  return r.obs && L.rule != MEM_RULE_LATEST;
}

__device__ __forceinline__ void apply_rule(const LayerDev& L, int64_t off, float S, const RuleCoef& r) {
  st_layer(L, off, rule_value(L, needs_old(L, r) ? ld_layer(L, off) : 0.f, S, r));
}

// initial value of stored value k of a layer (what an unobserved cell holds)
__device__ __forceinline__ float layer_init(const LayerDev& L, int k) {
  if (L.rule == MEM_RULE_DIRICHLET) return L.alpha0;
  if (L.rule == MEM_RULE_CLASSMAX && k == 0) return -1.f;
  return 0.f;
}

// float -> u32 with the same order (negative values reversed), and back
__host__ __device__ __forceinline__ u32 ordered_bits(u32 u) { return (u & 0x80000000u) ? ~u : (u | 0x80000000u); }
__host__ __device__ __forceinline__ u32 unordered_bits(u32 o) { return (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o; }

// the cell of a map-frame position, clamped into the map (the sensor's cell of
// a clean-up ray, the camera's cell of a visibility walk)
__device__ __forceinline__ void clamped_cell(const MapDev& md, float px, float py, int& cx, int& cy) {
  const float half = (float)(md.W / 2);
  float qx = floorf(__fdiv_rn(px, md.res)), qy = floorf(__fdiv_rn(py, md.res));
  if (!(qx >= -half)) qx = -half;
  if (!(qx <= half - 1.0f)) qx = half - 1.0f;
  if (!(qy >= -half)) qy = -half;
  if (!(qy <= half - 1.0f)) qy = half - 1.0f;
  cx = (int)qx + md.W / 2;
  cy = (int)qy + md.W / 2;
}

// relaxed device-scope loads/stores for the radix-sort look-back
__device__ __forceinline__ u32 ld_relaxed(const u32* p) {
  u32 v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(u32* p, u32 v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}


}  // namespace memk

// host-side launchers (defined in the .cu files)
namespace memh {
struct Map;
cudaError_t launch_point_fuse(Map* m, const memk::PointJob* d_job, cudaStream_t st);
cudaError_t launch_image_fuse(Map* m, int map_index, const memk::MapCall& mc, int H, int Wi,
                              int n_src, const memk::SrcDev* src, const float K[4],
                              uint8_t* vis, int32_t* pix, cudaStream_t st);
cudaError_t launch_clear_entering(Map* m, int map_index, int sx, int sy, int ring_x, int ring_y,
                                  cudaStream_t st);
cudaError_t launch_layer_copy(Map* m, int map_index, int layer, int part, void* buf, bool to_map,
                              cudaStream_t st);
cudaError_t launch_init_state(Map* m, cudaStream_t st);
}  // namespace memh
