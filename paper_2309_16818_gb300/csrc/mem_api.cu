// C ABI of the mapping library: map objects, argument checking, pose
// composition on the host (float64), and the move / layer-copy kernels.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>

#include "mem_host.h"

struct mem_map {
  memh::Map m;
};

namespace {
thread_local std::string g_err;

mem_status fail(mem_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

mem_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? MEM_ERR_OOM : MEM_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define CK(call, what)                           \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

size_t dtype_size(int dt) {
  switch (dt) {
    case MEM_F32: return 4;
    case MEM_BF16:
    case MEM_F16: return 2;
    case MEM_U8: return 1;
  }
  return 0;
}
}  // namespace

namespace memh {
mem_status api_fail(mem_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}
mem_status api_cuda_fail(cudaError_t e, const char* what) { return cuda_fail(e, what); }
Map* map_of(mem_map* mm) { return &mm->m; }
}  // namespace memh

// ---------------------------------------------------------------------------
// device kernels: reset of cells, layer copies

namespace memk {

// A cell is reset by clearing its flags (height invalid, no layer observed)
// and its counters: every kernel treats the stored values of an unobserved
// layer (and the height of an invalid cell) as the layer's initial value.
__device__ __forceinline__ void reset_cell(const MapDev& md, int64_t g) {
  md.flags[g] = 0u;
  md.n_acc[g] = 0u;
  md.n_rej[g] = 0u;
}

// Reset every cell of every map (map < 0), or the cells of `map` that entered
// with the shift (sx, sy): new logical (ix, iy) had no old cell
// (ix + sx, iy + sy) inside the map.
__global__ void k_reset(MapDev md, int map, int sx, int sy, int rx, int ry) {
  if (map < 0) {
    const int64_t total = (int64_t)md.n_maps * md.W2;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total;
         c += (int64_t)gridDim.x * blockDim.x)
      reset_cell(md, c);
    return;
  }
  // only the entering strips: |sx| columns and |sy| rows (corners twice)
  const u32 W = (u32)md.W;
  const u32 ax = (u32)min(abs(sx), md.W), ay = (u32)min(abs(sy), md.W);
  const u32 total = (ax + ay) * W;
  for (u32 u = blockIdx.x * blockDim.x + threadIdx.x; u < total; u += gridDim.x * blockDim.x) {
    int ix, iy;
    if (u < ax * W) {
      const u32 col = u / W;
      iy = (int)(u - col * W);
      ix = sx > 0 ? (int)(W - 1 - col) : (int)col;
    } else {
      const u32 v = u - ax * W, row = v / W;
      ix = (int)(v - row * W);
      iy = sy > 0 ? (int)(W - 1 - row) : (int)row;
    }
    int px = ix + rx;
    if (px >= md.W) px -= md.W;
    int py = iy + ry;
    if (py >= md.W) py -= md.W;
    reset_cell(md, (int64_t)map * md.W2 + (int64_t)py * md.W + px);
  }
}

// Copy one layer part between the map (physical order) and a buffer
// (logical order). to_map = 1 writes the map.
__global__ void k_layer_copy(MapDev md, int map, int rx, int ry, int layer, int part, void* buf,
                             int to_map) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < md.W2;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(j % md.W), iy = (int)(j / md.W);
    int px = ix + rx;
    if (px >= md.W) px -= md.W;
    int py = iy + ry;
    if (py >= md.W) py -= md.W;
    const int64_t g = (int64_t)map * md.W2 + (int64_t)py * md.W + px;
    if (layer < 0) {
      switch (layer) {
        case MEM_LAYER_HEIGHT:
          if (to_map) md.h[g] = ((const float*)buf)[j];
          else ((float*)buf)[j] = (md.flags[g] & kFlagValid) ? md.h[g] : 0.f;
          break;
        case MEM_LAYER_VARIANCE:
          if (to_map) md.var[g] = ((const float*)buf)[j];
          else ((float*)buf)[j] = (md.flags[g] & kFlagValid) ? md.var[g] : 0.f;
          break;
        case MEM_LAYER_VALID:
          if (to_map) md.flags[g] = (md.flags[g] & ~kFlagValid) | (((const uint8_t*)buf)[j] ? 1u : 0u);
          else ((uint8_t*)buf)[j] = (uint8_t)(md.flags[g] & kFlagValid);
          break;
        case MEM_LAYER_NACC:
          if (to_map) md.n_acc[g] = ((const u32*)buf)[j];
          else ((u32*)buf)[j] = md.n_acc[g];
          break;
        case MEM_LAYER_NREJ:
          if (to_map) md.n_rej[g] = ((const u32*)buf)[j];
          else ((u32*)buf)[j] = md.n_rej[g];
          break;
      }
      continue;
    }
    const LayerDev& L = md.L[layer];
    const bool obs = md.flags[g] & (2u << layer);
    if (!to_map && !obs) {  // an unobserved cell reads as the layer's initial state
      if (part == MEM_PART_VALUE) {
        if (L.dtype == MEM_F32)
          for (int k = 0; k < L.S; ++k) ((float*)buf)[j * L.S + k] = layer_init(L, k);
        else if (L.dtype == MEM_BF16)
          for (int k = 0; k < L.S; ++k) ((__nv_bfloat16*)buf)[j * L.S + k] = __float2bfloat16_rn(layer_init(L, k));
        else
          for (int k = 0; k < L.S; ++k) ((__half*)buf)[j * L.S + k] = __float2half_rn(layer_init(L, k));
      } else if (part == MEM_PART_THETA) {
        for (int k = 0; k < L.S; ++k) ((float*)buf)[j * L.S + k] = __frcp_rn((float)L.S);
      } else if (part == MEM_PART_VAR) {
        ((float*)buf)[j] = 0.f;
      } else {
        ((uint8_t*)buf)[j] = 0;
      }
      continue;
    }
    switch (part) {
      case MEM_PART_VALUE: {
        if (L.dtype == MEM_F32) {
          float* a = (float*)L.data + g * L.S;
          float* b = (float*)buf + j * L.S;
          for (int k = 0; k < L.S; ++k) {
            if (to_map) a[k] = b[k];
            else b[k] = a[k];
          }
        } else {
          uint16_t* a = (uint16_t*)L.data + g * L.S;
          uint16_t* b = (uint16_t*)buf + j * L.S;
          for (int k = 0; k < L.S; ++k) {
            if (to_map) a[k] = b[k];
            else b[k] = a[k];
          }
        }
        break;
      }
      case MEM_PART_THETA: {
        float s = 0.f;
        for (int k = 0; k < L.S; ++k) s = __fadd_rn(s, ld_layer(L, g * L.S + k));
        for (int k = 0; k < L.S; ++k) ((float*)buf)[j * L.S + k] = __fdiv_rn(ld_layer(L, g * L.S + k), s);
        break;
      }
      case MEM_PART_VAR:
        if (to_map) L.gvar[g] = ((const float*)buf)[j];
        else ((float*)buf)[j] = L.gvar[g];
        break;
      case MEM_PART_OBSERVED: {
        const u32 bit = 2u << layer;
        if (to_map) md.flags[g] = (md.flags[g] & ~bit) | (((const uint8_t*)buf)[j] ? bit : 0u);
        else ((uint8_t*)buf)[j] = (md.flags[g] & bit) ? 1 : 0;
        break;
      }
    }
  }
}

}  // namespace memk

// ---------------------------------------------------------------------------
// host helpers

namespace memh {
using namespace memk;

static cudaError_t dalloc(Map* m, void** p, size_t bytes, bool scratch) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e == cudaSuccess) (scratch ? m->scratch_allocs : m->allocs).push_back(*p);
  return e;
}

void free_scratch(Map* m) {
  for (void* p : m->scratch_allocs) cudaFree(p);
  m->scratch_allocs.clear();
  if (m->graph) {
    cudaGraphExecDestroy(m->graph);
    m->graph = nullptr;
  }
}

cudaError_t alloc_scratch(Map* m, int64_t cap) {
  MapDev& md = m->md;
  cap = cap < kSortTile ? kSortTile : cap;
  const int64_t tiles = (cap + kSortTile - 1) / kSortTile;
  cudaError_t e;
  void* p;
#define A(field, type, count)                                               \
  e = dalloc(m, &p, sizeof(type) * (size_t)(count), true);                  \
  if (e != cudaSuccess) return e;                                           \
  md.field = (type*)p;
  A(keys0, u32, cap + 4);
  A(keys1, u32, cap + 4);
  A(vals0, u32, cap + 4);
  A(vals1, u32, cap + 4);
  A(lookback, u32, 4 * tiles * 1024);
  if (md.drift_alpha != 0.0) {
    A(perr, float, cap + 4);
  }
#undef A
  md.cap = cap;
  md.cap_tiles = tiles;
  md.partial = nullptr;
  md.partial_cap = 0;
  return cudaSuccess;
}

// fuse scratch: tile tables and one slot of acc words per run piece
static cudaError_t ensure_partial(Map* m, int acc) {
  MapDev& md = m->md;
  const int64_t need = fuse_scratch_words(md.cap, acc);
  if (need <= md.partial_cap) return cudaSuccess;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return e;
  if (md.partial) {
    for (auto it = m->scratch_allocs.begin(); it != m->scratch_allocs.end(); ++it)
      if (*it == md.partial) {
        m->scratch_allocs.erase(it);
        break;
      }
    cudaFree(md.partial);
    md.partial = nullptr;
    md.partial_cap = 0;
  }
  void* p;
  e = dalloc(m, &p, sizeof(float) * (size_t)need, true);
  if (e != cudaSuccess) return e;
  md.partial = (float*)p;
  md.partial_cap = need;
  if (m->graph) {  // the graph captured the old buffer
    cudaGraphExecDestroy(m->graph);
    m->graph = nullptr;
  }
  return cudaSuccess;
}

cudaError_t launch_clear_entering(Map* m, int map_index, int sx, int sy, int ring_x, int ring_y,
                                  cudaStream_t st) {
  ProfScope ps(m, kProfMove, st);
  // one thread per entering cell (the strips: |sx| columns and |sy| rows), at most 4 blocks per SM
  const int64_t W = m->md.W;
  const int64_t cells = (std::min<int64_t>(std::abs(sx), W) + std::min<int64_t>(std::abs(sy), W)) * W;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((int64_t)m->n_sm * 4, (cells + 255) / 256));
  k_reset<<<(unsigned)blocks, 256, 0, st>>>(m->md, map_index, sx, sy, ring_x, ring_y);
  return cudaGetLastError();
}

cudaError_t launch_init_state(Map* m, cudaStream_t st) {
  k_reset<<<m->n_sm * 4, 256, 0, st>>>(m->md, -1, 0, 0, 0, 0);
  return cudaGetLastError();
}

cudaError_t launch_layer_copy(Map* m, int map_index, int layer, int part, void* buf, bool to_map,
                              cudaStream_t st) {
  k_layer_copy<<<m->n_sm * 4, 256, 0, st>>>(m->md, map_index, m->ring[2 * map_index],
                                             m->ring[2 * map_index + 1], layer, part, buf, to_map);
  return cudaGetLastError();
}

// Sensor pose relative to the map centre, cast to float32 (rotation as is,
// translation minus the map origin's xy).
static void pose_rel(const double T[16], const double o[2], MapCall& mc) {
  for (int r = 0; r < 3; ++r)
    for (int k = 0; k < 3; ++k) mc.R[r * 3 + k] = (float)T[r * 4 + k];
  mc.t[0] = (float)(T[3] - o[0]);
  mc.t[1] = (float)(T[7] - o[1]);
  mc.t[2] = (float)T[11];
}

// Map -> camera transform: R_cm = R_mc^T, t_cm = -R_mc^T (t_mc - o).
static void camera_rel(const double T[16], const double o[2], MapCall& mc) {
  const double d[3] = {T[3] - o[0], T[7] - o[1], T[11]};
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 3; ++k) mc.R[r * 3 + k] = (float)T[k * 4 + r];
    mc.t[r] = (float)(-(T[0 * 4 + r] * d[0] + T[1 * 4 + r] * d[1] + T[2 * 4 + r] * d[2]));
  }
  mc.cam_x = (float)d[0];
  mc.cam_y = (float)d[1];
  mc.cam_h = (float)d[2];
}

// Stage a job block in a pinned slot and queue its copy to the device.
static mem_status stage_job(Map* m, const void* host, size_t bytes, cudaStream_t st) {
  if (bytes > m->job_bytes) return fail(MEM_ERR_STATE, "job block too large (%zu bytes)", bytes);
  const int s = m->job_slot;
  m->job_slot = (s + 1) % kJobSlots;
  CK(cudaEventSynchronize(m->job_ev[s]), "cudaEventSynchronize");
  memcpy(m->h_job[s], host, bytes);
  CK(cudaMemcpyAsync(m->d_job, m->h_job[s], bytes, cudaMemcpyHostToDevice, st), "job upload");
  CK(cudaEventRecord(m->job_ev[s], st), "cudaEventRecord");
  return MEM_OK;
}

}  // namespace memh

// ---------------------------------------------------------------------------
// C ABI

using namespace memh;
using memk::LayerDev;
using memk::MapCall;
using memk::PointJob;
using memk::SrcDev;

extern "C" const char* mem_last_error(void) { return g_err.c_str(); }

static mem_status check_cfg(const mem_map_config* c) {
  if (!c) return fail(MEM_ERR_ARG, "config is NULL");
  if (c->W < 2 || c->W > 16384 || (c->W & 1)) return fail(MEM_ERR_ARG, "W must be even in [2, 16384]");
  if (c->n_maps < 1) return fail(MEM_ERR_ARG, "n_maps must be >= 1");
  if ((uint64_t)c->n_maps * (uint64_t)c->W * (uint64_t)c->W >= (1ull << 32) - 1)
    return fail(MEM_ERR_ARG, "n_maps * W * W must be < 2^32 - 1");
  if (!(c->res > 0.0) || !isfinite(c->res)) return fail(MEM_ERR_ARG, "res must be > 0");
  if (c->n_layers < 0 || c->n_layers > MEM_MAX_LAYERS) return fail(MEM_ERR_ARG, "n_layers out of range");
  if (!(c->range_min <= c->range_max)) return fail(MEM_ERR_ARG, "range_min > range_max");
  if (!(c->sigma0 >= 0.f) || !(c->sigma1 >= 0.f) || !(c->sigma0 + c->sigma1 > 0.f))
    return fail(MEM_ERR_ARG, "sigma0, sigma1 must be >= 0 and not both 0");
  for (int l = 0; l < c->n_layers; ++l) {
    const mem_layer_desc& L = c->layers[l];
    if (L.channels < 1 || L.channels > 4096) return fail(MEM_ERR_ARG, "layer %d: channels in [1, 4096]", l);
    if (L.rule < 0 || L.rule > MEM_RULE_CLASSMAX) return fail(MEM_ERR_ARG, "layer %d: bad rule", l);
    if (L.dtype != MEM_F32 && L.dtype != MEM_BF16 && L.dtype != MEM_F16)
      return fail(MEM_ERR_ARG, "layer %d: storage must be F32, BF16 or F16", l);
    if ((L.rule == MEM_RULE_CLASSMAX || L.rule == MEM_RULE_DIRICHLET) && L.dtype != MEM_F32)
      return fail(MEM_ERR_ARG, "layer %d: CLASSMAX / DIRICHLET layers are F32", l);
    if (L.rule == MEM_RULE_EXPAVG && !(L.w > 0.f && L.w <= 1.f)) return fail(MEM_ERR_ARG, "layer %d: w in (0, 1]", l);
    if (L.rule == MEM_RULE_GAUSS && !(L.var_meas > 0.f)) return fail(MEM_ERR_ARG, "layer %d: var_meas > 0", l);
    if (L.rule == MEM_RULE_DIRICHLET && !(L.alpha0 > 0.f)) return fail(MEM_ERR_ARG, "layer %d: alpha0 > 0", l);
  }
  if (!isfinite(c->drift_alpha)) return fail(MEM_ERR_ARG, "drift_alpha must be finite");
  if (c->drift_min_points < 0) return fail(MEM_ERR_ARG, "drift_min_points must be >= 0");
  if (c->ray_cleanup != 0 && c->ray_cleanup != 1) return fail(MEM_ERR_ARG, "ray_cleanup must be 0 or 1");
  if (c->ray_cleanup && !(c->ray_margin >= 0.f && isfinite(c->ray_margin)))
    return fail(MEM_ERR_ARG, "ray_margin must be finite and >= 0");
  return MEM_OK;
}

extern "C" mem_status mem_create_map(const mem_map_config* cfg, mem_map** out) {
  if (!out) return fail(MEM_ERR_ARG, "out is NULL");
  *out = nullptr;
  mem_status s = check_cfg(cfg);
  if (s != MEM_OK) return s;
  mem_map* mm = new (std::nothrow) mem_map();
  if (!mm) return fail(MEM_ERR_OOM, "host allocation failed");
  Map* m = &mm->m;
  m->cfg = *cfg;
  cudaGetDevice(&m->device);
  cudaDeviceGetAttribute(&m->n_sm, cudaDevAttrMultiProcessorCount, m->device);
  MapDev& md = m->md;
  memset(&md, 0, sizeof(md));
  md.W = cfg->W;
  md.n_maps = cfg->n_maps;
  md.W2 = (uint32_t)cfg->W * (uint32_t)cfg->W;
  md.sentinel = (uint32_t)cfg->n_maps * md.W2;
  md.res = (float)cfg->res;
  md.sigma0 = cfg->sigma0;
  md.sigma1 = cfg->sigma1;
  md.lam2 = cfg->gate_lambda * cfg->gate_lambda;
  md.outlier_var = cfg->outlier_var;
  md.time_var = cfg->time_var;
  md.range_min = cfg->range_min;
  md.range_max = cfg->range_max;
  md.z_near = cfg->z_near;
  md.n_layers = cfg->n_layers;
  md.drift_alpha = cfg->drift_alpha;
  md.drift_min = cfg->drift_min_points;
  md.ray_on = cfg->ray_cleanup;
  md.ray_margin = cfg->ray_margin;
  const int64_t cells = (int64_t)cfg->n_maps * md.W2;
  cudaError_t e = cudaSuccess;
  void* p = nullptr;
  auto bail = [&](cudaError_t err, const char* what) {
    mem_status st = cuda_fail(err, what);
    mem_destroy_map(mm);
    return st;
  };
#define ALLOC(ptr, type, count, what)                                  \
  e = dalloc(m, &p, sizeof(type) * (size_t)(count), false);            \
  if (e != cudaSuccess) return bail(e, what);                          \
  ptr = (type*)p;
  ALLOC(md.h, float, cells, "alloc h");
  ALLOC(md.var, float, cells, "alloc var");
  ALLOC(md.flags, uint32_t, cells, "alloc flags");
  ALLOC(md.n_acc, uint32_t, cells, "alloc n_acc");
  ALLOC(md.n_rej, uint32_t, cells, "alloc n_rej");
  for (int l = 0; l < cfg->n_layers; ++l) {
    const mem_layer_desc& D = cfg->layers[l];
    LayerDev& L = m->Lh[l];
    L.C = D.channels;
    L.S = D.rule == MEM_RULE_CLASSMAX ? 2 : D.channels;
    L.dtype = D.dtype;
    L.rule = D.rule;
    L.w = D.w;
    L.one_minus_w = 1.0f - D.w;
    L.var_meas = D.var_meas;
    L.alpha0 = D.alpha0;
    e = dalloc(m, &p, dtype_size(D.dtype) * (size_t)cells * L.S, false);
    if (e != cudaSuccess) return bail(e, "alloc layer");
    L.data = p;
    L.gvar = nullptr;
    if (D.rule == MEM_RULE_GAUSS) {
      ALLOC(L.gvar, float, cells, "alloc gauss variance");
    }
  }
  {
    LayerDev* dl = nullptr;
    ALLOC(dl, LayerDev, cfg->n_layers > 0 ? cfg->n_layers : 1, "alloc layer table");
    if (cfg->n_layers > 0 &&
        (e = cudaMemcpy(dl, m->Lh, sizeof(LayerDev) * cfg->n_layers, cudaMemcpyHostToDevice)) != cudaSuccess)
      return bail(e, "upload layer table");
    md.L = dl;
  }
  ALLOC(md.hist, uint32_t, 4 * 1024 + 16, "alloc hist");
  md.counters = md.hist + 4 * 1024;
  ALLOC(md.err, int, 2, "alloc err");  // [0] error word, [1] fault injection
  // drift reduction: about four blocks per SM over all maps, at least one per map
  md.drift_R = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (4LL * m->n_sm + cfg->n_maps - 1) / cfg->n_maps));
  ALLOC(md.dpart, double, (int64_t)cfg->n_maps * md.drift_R * 2, "alloc drift partials");
  ALLOC(md.drift_out, float, 2 * (int64_t)cfg->n_maps, "alloc drift record");
  if (md.ray_on) {
    ALLOC(md.zacc, memk::u64, cells, "alloc clean-up stamps");
    if ((e = cudaMemset(md.zacc, 0, sizeof(memk::u64) * (size_t)cells)) != cudaSuccess) return bail(e, "memset");
  }
  if ((e = cudaMemset(md.drift_out, 0, sizeof(float) * 2 * (size_t)cfg->n_maps)) != cudaSuccess)
    return bail(e, "memset");
#undef ALLOC
  e = alloc_scratch(m, cfg->max_points > 0 ? cfg->max_points : (1 << 20));
  if (e != cudaSuccess) return bail(e, "alloc scratch");
  // job block: header + per-map calls + offsets
  m->job_bytes = sizeof(PointJob) + sizeof(MapCall) * cfg->n_maps + sizeof(int64_t) * (cfg->n_maps + 1) + 64;
  e = dalloc(m, &p, m->job_bytes, false);
  if (e != cudaSuccess) return bail(e, "alloc job");
  m->d_job = (char*)p;
  for (int s2 = 0; s2 < kJobSlots; ++s2) {
    e = cudaMallocHost(&p, m->job_bytes);
    if (e != cudaSuccess) return bail(e, "pinned job slot");
    m->h_job[s2] = (char*)p;
    e = cudaEventCreateWithFlags(&m->job_ev[s2], cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(e, "event");
  }
  m->origin.assign(2 * cfg->n_maps, 0.0);
  m->ring.assign(2 * cfg->n_maps, 0);
  if ((e = prepare_kernels()) != cudaSuccess) return bail(e, "kernel attributes");
  m->key_bits = key_bits_for(m);
  m->tune.radix_bits = m->key_bits <= 16 ? 8 : 9;
  m->passes = (m->key_bits + m->tune.radix_bits - 1) / m->tune.radix_bits;
  if ((e = cudaMemset(md.err, 0, 2 * sizeof(int))) != cudaSuccess) return bail(e, "memset");
  if ((e = launch_init_state(m, 0)) != cudaSuccess) return bail(e, "init");
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bail(e, "init sync");
  *out = mm;
  return MEM_OK;
}

extern "C" mem_status mem_destroy_map(mem_map* mm) {
  if (!mm) return MEM_OK;
  Map* m = &mm->m;
  cudaDeviceSynchronize();
  free_scratch(m);
  for (void* p : m->allocs) cudaFree(p);
  for (int s = 0; s < kJobSlots; ++s) {
    if (m->h_job[s]) cudaFreeHost(m->h_job[s]);
    if (m->job_ev[s]) cudaEventDestroy(m->job_ev[s]);
  }
  for (int k = 0; k < 2; ++k) {
    if (m->stage_buf[k]) cudaFree(m->stage_buf[k]);
    if (m->stage_copied[k]) cudaEventDestroy(m->stage_copied[k]);
    if (m->stage_done[k]) cudaEventDestroy(m->stage_done[k]);
  }
  if (m->copy_stream) cudaStreamDestroy(m->copy_stream);
  if (m->pca_buf) cudaFree(m->pca_buf);
  if (m->img_buf) cudaFree(m->img_buf);
  for (cudaEvent_t e : m->prof_pool) cudaEventDestroy(e);
  delete mm;
  return MEM_OK;
}

extern "C" mem_status mem_set_tuning(mem_map* mm, int32_t radix_bits, int32_t blocks_per_sm, int32_t fuse_kernel) {
  if (!mm) return fail(MEM_ERR_ARG, "map is NULL");
  if (radix_bits < 8 || radix_bits > 10) return fail(MEM_ERR_ARG, "radix_bits in [8, 10]");
  if (blocks_per_sm < 1 || blocks_per_sm > 32) return fail(MEM_ERR_ARG, "blocks_per_sm in [1, 32]");
  if (fuse_kernel < 0 || fuse_kernel > 1) return fail(MEM_ERR_ARG, "fuse_kernel is 0 or 1");
  Map* m = &mm->m;
  if ((m->key_bits + radix_bits - 1) / radix_bits > 4) return fail(MEM_ERR_ARG, "too many radix passes");
  cudaDeviceSynchronize();
  m->tune.radix_bits = radix_bits;
  m->tune.blocks_per_sm = blocks_per_sm;
  m->tune.fuse_kernel = fuse_kernel;
  m->passes = (m->key_bits + radix_bits - 1) / radix_bits;
  if (m->passes > 4) return fail(MEM_ERR_ARG, "too many radix passes");
  if (m->graph) {
    cudaGraphExecDestroy(m->graph);
    m->graph = nullptr;
  }
  return MEM_OK;
}

extern "C" mem_status mem_get_tuning(const mem_map* mm, int32_t out[4]) {
  if (!mm || !out) return fail(MEM_ERR_ARG, "NULL argument");
  out[0] = mm->m.tune.radix_bits;
  out[1] = mm->m.tune.blocks_per_sm;
  out[2] = mm->m.passes;
  out[3] = mm->m.tune.fuse_kernel;
  return MEM_OK;
}

extern "C" mem_status mem_move_map(mem_map* mm, int32_t map_index, const double robot_xy[2], void* stream) {
  if (!mm || !robot_xy) return fail(MEM_ERR_ARG, "NULL argument");
  Map* m = &mm->m;
  if (map_index < 0 || map_index >= m->cfg.n_maps) return fail(MEM_ERR_ARG, "map_index out of range");
  if (!isfinite(robot_xy[0]) || !isfinite(robot_xy[1])) return fail(MEM_ERR_ARG, "robot_xy not finite");
  double* o = &m->origin[2 * map_index];
  const double fx = (robot_xy[0] - o[0]) / m->cfg.res, fy = (robot_xy[1] - o[1]) / m->cfg.res;
  if (fabs(fx) > 1e9 || fabs(fy) > 1e9) return fail(MEM_ERR_ARG, "move too large");
  const long sx = lround(fx), sy = lround(fy);
  if (sx == 0 && sy == 0) return MEM_OK;
  const int W = m->cfg.W;
  int* r = &m->ring[2 * map_index];
  const int rx = (int)(((r[0] + sx) % W + W) % W), ry = (int)(((r[1] + sy) % W + W) % W);
  const int csx = (int)(sx > W ? W : (sx < -W ? -W : sx));
  const int csy = (int)(sy > W ? W : (sy < -W ? -W : sy));
  cudaError_t e = launch_clear_entering(m, map_index, csx, csy, rx, ry, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "move");
  r[0] = rx;
  r[1] = ry;
  o[0] = o[0] + (double)sx * m->cfg.res;
  o[1] = o[1] + (double)sy * m->cfg.res;
  return MEM_OK;
}

static mem_status check_sources(const Map* m, int32_t n_sources, const mem_source* sources,
                                 SrcDev* out, bool image) {
  if (n_sources < 0 || n_sources > MEM_MAX_SOURCES) return fail(MEM_ERR_ARG, "n_sources out of range");
  if (n_sources > 0 && !sources) return fail(MEM_ERR_ARG, "sources is NULL");
  for (int q = 0; q < n_sources; ++q) {
    const mem_source& s = sources[q];
    if (!s.data) return fail(MEM_ERR_ARG, "source %d: data is NULL", q);
    if (dtype_size(s.dtype) == 0) return fail(MEM_ERR_ARG, "source %d: bad dtype", q);
    if (s.topk < 0 || s.topk > MEM_MAX_TOPK) return fail(MEM_ERR_ARG, "source %d: topk in [0, %d]", q, MEM_MAX_TOPK);
    if (s.topk && s.dtype != MEM_F32) return fail(MEM_ERR_ARG, "source %d: top-k rows are float32 pairs", q);
    if (s.channels < 1 || s.channels > 4096) return fail(MEM_ERR_ARG, "source %d: channels", q);
    if (s.n_layers < 0 || s.n_layers > MEM_MAX_SOURCE_LAYERS) return fail(MEM_ERR_ARG, "source %d: n_layers", q);
    for (int b = 0; b < s.n_layers; ++b) {
      const int l = s.layers[b];
      if (l < 0 || l >= m->cfg.n_layers) return fail(MEM_ERR_ARG, "source %d: layer %d out of range", q, l);
      if (m->cfg.layers[l].channels != s.channels)
        return fail(MEM_ERR_ARG, "source %d: %d channels but layer %d has %d", q, s.channels, l,
                    m->cfg.layers[l].channels);
      for (int b2 = 0; b2 < b; ++b2)
        if (s.layers[b2] == l) return fail(MEM_ERR_ARG, "source %d: layer %d listed twice", q, l);
      for (int q2 = 0; q2 < q && !image; ++q2)
        for (int b2 = 0; b2 < sources[q2].n_layers; ++b2)
          if (sources[q2].layers[b2] == l)
            return fail(MEM_ERR_ARG, "layer %d is bound to sources %d and %d", l, q2, q);
    }
    out[q].data = s.data;
    out[q].dtype = s.dtype;
    out[q].C = s.channels;
    out[q].n_layers = s.n_layers;
    out[q].topk = s.topk;
    out[q].unused = 0;
    out[q].vec_ok = !s.topk && ((uintptr_t)s.data & 15) == 0;
    out[q].has_classmax = 0;
    for (int b = 0; b < s.n_layers; ++b)
      if (m->cfg.layers[s.layers[b]].rule == MEM_RULE_CLASSMAX) out[q].has_classmax = 1;
    for (int b = 0; b < MEM_MAX_SOURCE_LAYERS; ++b) out[q].layers[b] = b < s.n_layers ? s.layers[b] : 0;
  }
  return MEM_OK;
}

void memh::build_fuse_tables(PointJob& job, int acc_raw, const mem_map_config& cfg) {
  memk::FuseTables& f = job.ft;
  memset(&f, 0, sizeof(f));
  const int n_src = job.n_src;
  for (int q = 0; q < n_src; ++q) {
    int nl = 0;
    for (int b = 0; b < job.src[q].n_layers; ++b) {
      const int l = job.src[q].layers[b];
      const int rule = cfg.layers[l].rule;
      if (rule != MEM_RULE_CLASSMAX) f.rlay[q][nl++] = l;
      if (rule == MEM_RULE_GAUSS) f.any_gauss = 1;
    }
    f.nrlay[q] = nl;
  }
  const int G = acc_raw - (kSlotHdr - 4);
  f.ncol = G;
  f.one_round = G <= memk::kFuseQ;
  if (!f.one_round) return;
  // columns: height sums, then each source's channels and arg-max pair
  for (int c = 0; c < G; ++c) {
    f.col_src[c] = -1;
    f.col_ch[c] = c;
    if (c < 4) continue;
    const int o = c + (kSlotHdr - 4);
    int q = 0;
    for (int k = 1; k < n_src; ++k)
      if (job.src[k].acc_off <= o) q = k;
    const int ch = o - job.src[q].acc_off;
    f.col_src[c] = q;
    f.col_ch[c] = ch < job.src[q].C ? ch : (ch == job.src[q].C ? -1 : -2);
  }
  // staging chunks: runs of up to four consecutive channels of one source,
  // aligned to four channels
  int n = 0;
  for (int c = 0; c < G; ++c) {
    const int q = f.col_src[c], ch = f.col_ch[c];
    if (q < 0 || ch < 0) continue;
    const bool extend = n > 0 && f.ck[n - 1].n < 4 && (ch & 3) != 0 && f.col_src[c - 1] == q &&
                        f.col_ch[c - 1] == ch - 1 && f.ck[n - 1].col + f.ck[n - 1].n == c;
    if (extend) {
      ++f.ck[n - 1].n;
      continue;
    }
    memk::ChunkDesc& d = f.ck[n++];
    d.data = job.src[q].data;
    d.C = job.src[q].C;
    d.ch0 = ch;
    d.col = c;
    d.n = 1;
    d.dtype = job.src[q].dtype;
    d.vec = job.src[q].vec_ok;
    d.src = q;
    d.topk = job.src[q].topk;
  }
  f.n_ck = n;
  for (int k = 0; k < n; ++k) {
    const int q = f.ck[k].src;
    const int av = f.ck[k].col - f.ck[k].ch0 + job.src[q].C;  // arg-max value column
    const bool last = k + 1 == n || f.ck[k + 1].src != q;
    f.ck[k].am = job.src[q].has_classmax ? (av | (last ? (1 << 30) : 0)) : -1;
  }
  for (int q = 0; q < n_src; ++q) {
    f.qc0[q] = job.src[q].acc_off - (kSlotHdr - 4);
    f.qch0[q] = 0;
    f.qn[q] = job.src[q].C;
    if (job.src[q].has_classmax) f.pair_col[f.n_pair++] = f.qc0[q] + job.src[q].C;
  }
}

static mem_status ensure_capacity(Map* m, int64_t n) {
  if (n <= m->md.cap) return MEM_OK;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "sync before scratch growth");
  free_scratch(m);
  e = alloc_scratch(m, n + n / 4);
  if (e != cudaSuccess) return cuda_fail(e, "scratch growth");
  return MEM_OK;
}

// Builds and uploads the job block, then queues the kernel sequence
// (replayed from a CUDA graph when `graph` is set and the stream allows it).
// The job block is uploaded on `job_st` (default: `st`); with `ready` set, the
// kernels on `st` wait for an event recorded on `job_st` after that upload.
static mem_status run_points(Map* m, int nm, const int64_t* offsets, int64_t n, const float* xyz,
                             const SrcDev* src, int n_src, const double* T, bool graph, cudaStream_t st,
                             cudaStream_t job_st = nullptr, cudaEvent_t ready = nullptr) {
  mem_status s = ensure_capacity(m, n);
  if (s != MEM_OK) return s;
  std::string buf(m->job_bytes, '\0');
  char* h = &buf[0];
  PointJob* job = (PointJob*)h;
  MapCall* mcs = (MapCall*)(h + sizeof(PointJob));
  int64_t* offs = (int64_t*)(h + sizeof(PointJob) + sizeof(MapCall) * nm);
  job->n = n;
  if (++m->call_id == 0) m->call_id = 1;  // 0 marks "never stamped"
  job->call_id = m->call_id;
  job->xyz = xyz;
  job->n_maps = nm;
  job->n_src = n_src;
  int acc = kSlotHdr;  // slot header
  for (int q = 0; q < n_src; ++q) {
    job->src[q] = src[q];
    job->src[q].acc_off = acc;
    acc += src[q].C + 2 * src[q].has_classmax;  // channel sums, then (max value, class)
  }
  build_fuse_tables(*job, acc, m->cfg);
  m->fuse_variant = job->ft.one_round ? 2 : 0;
  for (int q = 0; q < n_src; ++q) m->fuse_variant |= src[q].topk ? 1 : 0;
  if (m->graph && m->graph_variant != m->fuse_variant) {  // the graph launches another kernel variant
    cudaGraphExecDestroy(m->graph);
    m->graph = nullptr;
  }
  acc = (acc + 3) / 4 * 4;  // slots start on 16-byte boundaries (vector loads of their headers)
  job->acc = acc;
  {
    cudaError_t e = ensure_partial(m, acc);
    if (e != cudaSuccess) return cuda_fail(e, "partial-record buffer");
  }
  if (((uintptr_t)m->md.partial & 15) != 0) return fail(MEM_ERR_STATE, "fuse scratch not 16-byte aligned");
  job->maps = (const MapCall*)(m->d_job + sizeof(PointJob));
  job->offsets = nm > 1 ? (const int64_t*)(m->d_job + sizeof(PointJob) + sizeof(MapCall) * nm) : nullptr;
  for (int b = 0; b < nm; ++b) {
    memset(&mcs[b], 0, sizeof(MapCall));
    pose_rel(T + 16 * b, &m->origin[2 * b], mcs[b]);
    mcs[b].ring_x = m->ring[2 * b];
    mcs[b].ring_y = m->ring[2 * b + 1];
  }
  size_t bytes = sizeof(PointJob) + sizeof(MapCall) * nm;
  if (nm > 1) {
    for (int b = 0; b <= nm; ++b) offs[b] = offsets[b];
    bytes += sizeof(int64_t) * (nm + 1);
  }
  s = stage_job(m, h, bytes, ready ? job_st : st);
  if (s != MEM_OK) return s;
  if (ready) {
    CK(cudaEventRecord(ready, job_st), "job upload record");
    CK(cudaStreamWaitEvent(st, ready, 0), "job upload wait");
  }
  if (n == 0) {  // no points: only the time-dependent variance growth of the valid cells
    // (the call's statistics and drift record read as zero)
    CK(cudaMemsetAsync(m->md.counters, 0, sizeof(uint32_t) * 16, st), "clear counters");
    CK(cudaMemsetAsync(m->md.drift_out, 0, sizeof(float) * 2 * (size_t)nm, st), "clear drift record");
    CK(launch_time_update(m, st), "time update launch");
    return MEM_OK;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (graph && st) cudaStreamIsCapturing(st, &cap);
  if (graph && st && cap == cudaStreamCaptureStatusNone && m->use_graph && !m->prof_on) {
    if (!m->graph) {
      cudaGraph_t gph;
      CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
      cudaError_t e = launch_point_fuse(m, (const PointJob*)m->d_job, st);
      cudaError_t e2 = cudaStreamEndCapture(st, &gph);
      if (e != cudaSuccess) return cuda_fail(e, "capture launch");
      if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
      e = cudaGraphInstantiate(&m->graph, gph, 0);
      cudaGraphDestroy(gph);
      if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
      m->graph_variant = m->fuse_variant;
    }
    CK(cudaGraphLaunch(m->graph, st), "graph launch");
    return MEM_OK;
  }
  CK(launch_point_fuse(m, (const PointJob*)m->d_job, st), "point fuse launch");
  return MEM_OK;
}

static bool finite16(const double* T) {
  for (int k = 0; k < 16; ++k)
    if (!isfinite(T[k])) return false;
  return true;
}

extern "C" mem_status mem_fuse_pointcloud(mem_map* mm, int64_t n, const float* xyz, int32_t n_sources,
                                          const mem_source* sources, const double T_map_sensor[16],
                                          void* stream) {
  if (!mm || !T_map_sensor) return fail(MEM_ERR_ARG, "NULL argument");
  Map* m = &mm->m;
  if (m->cfg.n_maps != 1) return fail(MEM_ERR_ARG, "map object holds %d maps: use mem_fuse_pointcloud_batch", m->cfg.n_maps);
  if (n < 0 || n >= (1ll << 30)) return fail(MEM_ERR_ARG, "n out of range [0, 2^30)");
  if (n > 0 && !xyz) return fail(MEM_ERR_ARG, "xyz is NULL");
  if (!finite16(T_map_sensor)) return fail(MEM_ERR_ARG, "pose not finite");
  SrcDev src[MEM_MAX_SOURCES];
  mem_status s = check_sources(m, n_sources, sources, src, false);
  if (s != MEM_OK) return s;
  return run_points(m, 1, nullptr, n, xyz, src, n_sources, T_map_sensor, true, (cudaStream_t)stream);
}

// Host-buffer variant of mem_fuse_pointcloud: the call's inputs are copied
// into one of two device staging buffers (used in turn) on the map's copy
// stream; the kernels wait for that copy on the caller's stream, and the
// next call's copy waits only for the kernels that last read the same
// buffer, so uploads overlap the previous call's fuse.
extern "C" mem_status mem_fuse_pointcloud_host(mem_map* mm, int64_t n, const float* xyz, int32_t n_sources,
                                               const mem_source* sources, const double T_map_sensor[16],
                                               void* stream) {
  if (!mm || !T_map_sensor) return fail(MEM_ERR_ARG, "NULL argument");
  Map* m = &mm->m;
  if (m->cfg.n_maps != 1) return fail(MEM_ERR_ARG, "map object holds %d maps: use mem_fuse_pointcloud_batch", m->cfg.n_maps);
  if (n < 0 || n >= (1ll << 30)) return fail(MEM_ERR_ARG, "n out of range [0, 2^30)");
  if (n > 0 && !xyz) return fail(MEM_ERR_ARG, "xyz is NULL");
  if (!finite16(T_map_sensor)) return fail(MEM_ERR_ARG, "pose not finite");
  SrcDev src[MEM_MAX_SOURCES];
  mem_status s = check_sources(m, n_sources, sources, src, false);
  if (s != MEM_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  // layout of the staging buffer: xyz, then every source's rows, 256-byte aligned
  size_t off[MEM_MAX_SOURCES + 1], bytes = 0;
  auto take = [&](size_t b) {
    const size_t o = bytes;
    bytes += (b + 255) & ~(size_t)255;
    return o;
  };
  // bytes of a source's rows: C values, or 2 * topk float32 for top-k rows
  auto row_bytes = [&](int q) {
    return src[q].topk ? (size_t)(2 * src[q].topk) * 4 : (size_t)src[q].C * dtype_size(src[q].dtype);
  };
  off[0] = take((size_t)n * 12);
  for (int q = 0; q < n_sources; ++q) off[q + 1] = take((size_t)n * row_bytes(q));
  if (!m->copy_stream) {
    CK(cudaStreamCreateWithFlags(&m->copy_stream, cudaStreamNonBlocking), "copy stream");
    for (int k = 0; k < 2; ++k) {
      CK(cudaEventCreateWithFlags(&m->stage_copied[k], cudaEventDisableTiming), "staging event");
      CK(cudaEventCreateWithFlags(&m->stage_done[k], cudaEventDisableTiming), "staging event");
    }
  }
  const int k = m->stage_slot;
  m->stage_slot ^= 1;
  if (bytes > m->stage_cap[k]) {  // grow (waits for every use of the old buffer)
    CK(cudaEventSynchronize(m->stage_done[k]), "staging sync");
    if (m->stage_buf[k]) cudaFree(m->stage_buf[k]);
    m->stage_buf[k] = nullptr;
    m->stage_cap[k] = 0;
    CK(cudaMalloc(&m->stage_buf[k], bytes + bytes / 4), "staging buffer");
    m->stage_cap[k] = bytes + bytes / 4;
  }
  char* d = (char*)m->stage_buf[k];
  CK(cudaStreamWaitEvent(m->copy_stream, m->stage_done[k], 0), "staging wait");
  if (n > 0) {
    CK(cudaMemcpyAsync(d + off[0], xyz, (size_t)n * 12, cudaMemcpyHostToDevice, m->copy_stream), "upload xyz");
    for (int q = 0; q < n_sources; ++q) {
      CK(cudaMemcpyAsync(d + off[q + 1], sources[q].data, (size_t)n * row_bytes(q), cudaMemcpyHostToDevice,
                         m->copy_stream),
         "upload source");
      src[q].data = d + off[q + 1];
      src[q].vec_ok = !src[q].topk;  // 256-byte aligned
    }
  }
  // the job block follows the inputs on the copy stream; the kernels wait for both
  s = run_points(m, 1, nullptr, n, (const float*)(d + off[0]), src, n_sources, T_map_sensor, true, st,
                 m->copy_stream, m->stage_copied[k]);
  if (s != MEM_OK) return s;
  CK(cudaEventRecord(m->stage_done[k], st), "staging record");
  return MEM_OK;
}

extern "C" mem_status mem_fuse_pointcloud_batch(mem_map* mm, const int64_t* offsets, const float* xyz,
                                                int32_t n_sources, const mem_source* sources,
                                                const double* T_map_sensor, void* stream) {
  if (!mm || !offsets || !T_map_sensor) return fail(MEM_ERR_ARG, "NULL argument");
  Map* m = &mm->m;
  const int nm = m->cfg.n_maps;
  if (offsets[0] != 0) return fail(MEM_ERR_ARG, "offsets[0] must be 0");
  for (int b = 0; b < nm; ++b)
    if (offsets[b + 1] < offsets[b]) return fail(MEM_ERR_ARG, "offsets must be non-decreasing");
  const int64_t n = offsets[nm];
  if (n >= (1ll << 30)) return fail(MEM_ERR_ARG, "total points must be < 2^30");
  if (n > 0 && !xyz) return fail(MEM_ERR_ARG, "xyz is NULL");
  for (int b = 0; b < nm; ++b)
    if (!finite16(T_map_sensor + 16 * b)) return fail(MEM_ERR_ARG, "pose %d not finite", b);
  SrcDev src[MEM_MAX_SOURCES];
  mem_status s = check_sources(m, n_sources, sources, src, false);
  if (s != MEM_OK) return s;
  return run_points(m, nm, offsets, n, xyz, src, n_sources, T_map_sensor, true, (cudaStream_t)stream);
}

extern "C" mem_status mem_fuse_image(mem_map* mm, int32_t map_index, int32_t H, int32_t Wi,
                                     int32_t n_sources, const mem_source* sources, const double K[4],
                                     const double T_map_cam[16], uint8_t* vis_out, int32_t* pix_out,
                                     void* stream) {
  if (!mm || !K || !T_map_cam) return fail(MEM_ERR_ARG, "NULL argument");
  Map* m = &mm->m;
  if (map_index < 0 || map_index >= m->cfg.n_maps) return fail(MEM_ERR_ARG, "map_index out of range");
  if (H < 1 || Wi < 1 || (int64_t)H * Wi >= (1ll << 31)) return fail(MEM_ERR_ARG, "bad image size");
  if (!finite16(T_map_cam)) return fail(MEM_ERR_ARG, "pose not finite");
  for (int k = 0; k < 4; ++k)
    if (!isfinite(K[k])) return fail(MEM_ERR_ARG, "intrinsics not finite");
  SrcDev src[MEM_MAX_SOURCES];
  mem_status s = check_sources(m, n_sources, sources, src, true);
  if (s != MEM_OK) return s;
  MapCall mc;
  memset(&mc, 0, sizeof(mc));
  camera_rel(T_map_cam, &m->origin[2 * map_index], mc);
  mc.ring_x = m->ring[2 * map_index];
  mc.ring_y = m->ring[2 * map_index + 1];
  const float Kf[4] = {(float)K[0], (float)K[1], (float)K[2], (float)K[3]};
  cudaError_t e = launch_image_fuse(m, map_index, mc, H, Wi, n_sources, src, Kf, vis_out, pix_out,
                                    (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "image fuse launch");
  return MEM_OK;
}

static mem_status check_layer(const Map* m, int32_t map_index, int32_t layer, int32_t part, bool set) {
  if (map_index < 0 || map_index >= m->cfg.n_maps) return fail(MEM_ERR_ARG, "map_index out of range");
  if (layer < MEM_LAYER_NREJ || layer >= m->cfg.n_layers) return fail(MEM_ERR_ARG, "layer out of range");
  if (layer >= 0) {
    const int rule = m->cfg.layers[layer].rule;
    if (part < MEM_PART_VALUE || part > MEM_PART_OBSERVED) return fail(MEM_ERR_ARG, "bad part");
    if (part == MEM_PART_THETA && (rule != MEM_RULE_DIRICHLET || set))
      return fail(MEM_ERR_ARG, "THETA is a read-only part of DIRICHLET layers");
    if (part == MEM_PART_VAR && rule != MEM_RULE_GAUSS) return fail(MEM_ERR_ARG, "VAR is a part of GAUSS layers");
  }
  return MEM_OK;
}

extern "C" mem_status mem_get_layer(mem_map* mm, int32_t map_index, int32_t layer, int32_t part, void* dst,
                                    void* stream) {
  if (!mm || !dst) return fail(MEM_ERR_ARG, "NULL argument");
  Map* m = &mm->m;
  mem_status s = check_layer(m, map_index, layer, part, false);
  if (s != MEM_OK) return s;
  CK(launch_layer_copy(m, map_index, layer, part, dst, false, (cudaStream_t)stream), "get layer");
  return MEM_OK;
}

extern "C" mem_status mem_set_layer(mem_map* mm, int32_t map_index, int32_t layer, int32_t part,
                                    const void* src, void* stream) {
  if (!mm || !src) return fail(MEM_ERR_ARG, "NULL argument");
  Map* m = &mm->m;
  mem_status s = check_layer(m, map_index, layer, part, true);
  if (s != MEM_OK) return s;
  CK(launch_layer_copy(m, map_index, layer, part, (void*)src, true, (cudaStream_t)stream), "set layer");
  return MEM_OK;
}

extern "C" mem_status mem_get_origin(const mem_map* mm, int32_t map_index, double out_xy[2]) {
  if (!mm || !out_xy) return fail(MEM_ERR_ARG, "NULL argument");
  if (map_index < 0 || map_index >= mm->m.cfg.n_maps) return fail(MEM_ERR_ARG, "map_index out of range");
  out_xy[0] = mm->m.origin[2 * map_index];
  out_xy[1] = mm->m.origin[2 * map_index + 1];
  return MEM_OK;
}

// Autotuner of the point path's schedule: every candidate (fuse kernel x radix
// digit width x persistent-grid size) runs the given batched call `reps` times from the same
// saved map state; the fastest is kept and the state is restored.
extern "C" mem_status mem_autotune_batch(mem_map* mm, const int64_t* offsets, const float* xyz,
                                         int32_t n_sources, const mem_source* sources,
                                         const double* T_map_sensor, int32_t reps, void* stream,
                                         float* ms_out, int32_t* n_out) {
  if (!mm || !offsets || !T_map_sensor) return fail(MEM_ERR_ARG, "NULL argument");
  if (reps < 1 || reps > 1000) return fail(MEM_ERR_ARG, "reps in [1, 1000]");
  Map* m = &mm->m;
  cudaStream_t st = (cudaStream_t)stream;
  // every state array of the map, saved once
  std::vector<std::pair<void*, size_t>> arrays;
  const size_t cells = (size_t)m->cfg.n_maps * m->md.W2;
  arrays.push_back({m->md.h, cells * 4});
  arrays.push_back({m->md.var, cells * 4});
  arrays.push_back({m->md.flags, cells * 4});
  arrays.push_back({m->md.n_acc, cells * 4});
  arrays.push_back({m->md.n_rej, cells * 4});
  for (int l = 0; l < m->cfg.n_layers; ++l) {
    arrays.push_back({m->Lh[l].data, cells * m->Lh[l].S * dtype_size(m->Lh[l].dtype)});
    if (m->Lh[l].gvar) arrays.push_back({m->Lh[l].gvar, cells * 4});
  }
  size_t total = 0;
  for (auto& a : arrays) total += (a.second + 255) & ~(size_t)255;
  char* backup = nullptr;
  CK(cudaMalloc(&backup, total), "autotune backup");
  auto copy_all = [&](bool save) -> cudaError_t {
    size_t o = 0;
    for (auto& a : arrays) {
      cudaError_t e = save ? cudaMemcpyAsync(backup + o, a.first, a.second, cudaMemcpyDeviceToDevice, st)
                           : cudaMemcpyAsync(a.first, backup + o, a.second, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
      o += (a.second + 255) & ~(size_t)255;
    }
    return cudaSuccess;
  };
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const Tuning saved = m->tune;
  const int saved_passes = m->passes;
  float best = 1e30f;
  Tuning best_t = saved;
  int count = 0;
  mem_status s = MEM_OK;
  cudaError_t ce = copy_all(true);
  const int bits_opts[3] = {8, 9, 10}, bps_opts[3] = {2, 4, 8};
  for (int ki = 0; ki < 6 && ce == cudaSuccess && s == MEM_OK; ++ki) {
    const int bi = ki % 3, fk = ki / 3;  // both fuse kernels (they differ only where the columns fit one round)
    const int passes = (m->key_bits + bits_opts[bi] - 1) / bits_opts[bi];
    if (passes > 4) continue;
    for (int pi = 0; pi < 3 && ce == cudaSuccess && s == MEM_OK; ++pi) {
      cudaStreamSynchronize(st);
      m->tune.radix_bits = bits_opts[bi];
      m->tune.blocks_per_sm = bps_opts[pi];
      m->tune.fuse_kernel = fk;
      m->passes = passes;
      if (m->graph) {
        cudaGraphExecDestroy(m->graph);
        m->graph = nullptr;
      }
      float acc_ms = 0.f;
      for (int r = 0; r <= reps && s == MEM_OK; ++r) {  // r = 0 warms up (and captures the graph)
        if ((ce = copy_all(false)) != cudaSuccess) break;
        cudaEventRecord(e0, st);
        s = mem_fuse_pointcloud_batch(mm, offsets, xyz, n_sources, sources, T_map_sensor, stream);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (r > 0) acc_ms += t;
      }
      if (s != MEM_OK || ce != cudaSuccess) break;
      const float ms = acc_ms / reps;
      if (ms_out && n_out && count < *n_out) ms_out[count] = ms;
      ++count;
      if (ms < best) {
        best = ms;
        best_t = m->tune;
      }
    }
  }
  cudaStreamSynchronize(st);
  m->tune = (s == MEM_OK && ce == cudaSuccess) ? best_t : saved;
  m->passes = (s == MEM_OK && ce == cudaSuccess) ? (m->key_bits + m->tune.radix_bits - 1) / m->tune.radix_bits
                                                 : saved_passes;
  if (m->graph) {
    cudaGraphExecDestroy(m->graph);
    m->graph = nullptr;
  }
  cudaError_t ce2 = copy_all(false);
  cudaStreamSynchronize(st);
  cudaFree(backup);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (n_out) *n_out = count;
  if (s != MEM_OK) return s;
  if (ce != cudaSuccess) return cuda_fail(ce, "autotune state copy");
  if (ce2 != cudaSuccess) return cuda_fail(ce2, "autotune state restore");
  return MEM_OK;
}

extern "C" mem_status mem_set_profiling(mem_map* mm, int32_t on) {
  if (!mm) return fail(MEM_ERR_ARG, "NULL argument");
  mm->m.prof_on = on != 0;
  return MEM_OK;
}

extern "C" mem_status mem_get_profile(mem_map* mm, double ms[MEM_PROFILE_SLOTS],
                                      int64_t calls[MEM_PROFILE_SLOTS]) {
  if (!mm || !ms || !calls) return fail(MEM_ERR_ARG, "NULL argument");
  Map* m = &mm->m;
  for (auto& p : m->prof_pending) {
    CK(cudaEventSynchronize(p.b), "profile event");
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, p.a, p.b), "profile elapsed");
    m->prof_ms[p.slot] += t;
    m->prof_calls[p.slot] += 1;
  }
  m->prof_pending.clear();
  m->prof_next = 0;  // every pooled event is free again
  for (int k = 0; k < MEM_PROFILE_SLOTS; ++k) {
    ms[k] = k < 16 ? m->prof_ms[k] : 0.0;
    calls[k] = k < 16 ? m->prof_calls[k] : 0;
    if (k < 16) {
      m->prof_ms[k] = 0.0;
      m->prof_calls[k] = 0;
    }
  }
  return MEM_OK;
}

extern "C" mem_status mem_get_stats(mem_map* mm, void* stream, int64_t out[4]) {
  if (!mm || !out) return fail(MEM_ERR_ARG, "NULL argument");
  Map* m = &mm->m;
  CK(cudaStreamSynchronize((cudaStream_t)stream), "stream synchronize");
  uint32_t c[8];
  CK(cudaMemcpy(c, m->md.counters, sizeof(c), cudaMemcpyDeviceToHost), "read counters");
  out[0] = c[4];
  out[1] = c[5];
  out[2] = c[6];
  out[3] = m->passes;
  return MEM_OK;
}

extern "C" mem_status mem_get_drift(mem_map* mm, int32_t map_index, void* stream, double out[3]) {
  if (!mm || !out) return fail(MEM_ERR_ARG, "NULL argument");
  Map* m = &mm->m;
  if (map_index < 0 || map_index >= m->cfg.n_maps) return fail(MEM_ERR_ARG, "map_index out of range");
  CK(cudaStreamSynchronize((cudaStream_t)stream), "stream synchronize");
  float d[2];
  uint32_t c[16];
  CK(cudaMemcpy(d, m->md.drift_out + 2 * map_index, sizeof(d), cudaMemcpyDeviceToHost), "read drift record");
  CK(cudaMemcpy(c, m->md.counters, sizeof(c), cudaMemcpyDeviceToHost), "read counters");
  uint32_t cnt;
  memcpy(&cnt, &d[1], 4);
  out[0] = d[0];
  out[1] = (double)cnt;
  out[2] = (double)c[10];
  return MEM_OK;
}

extern "C" mem_status mem_inject_fault(mem_map* mm, int32_t kind) {
  if (!mm) return fail(MEM_ERR_ARG, "NULL argument");
  if (kind != MEM_FAULT_NONE && kind != MEM_FAULT_SORT_WAIT) return fail(MEM_ERR_ARG, "unknown fault kind %d", kind);
  Map* m = &mm->m;
  CK(cudaDeviceSynchronize(), "synchronize");
  const int v = kind;
  CK(cudaMemcpy(m->md.err + 1, &v, sizeof(int), cudaMemcpyHostToDevice), "write fault word");
  return MEM_OK;
}

extern "C" mem_status mem_check(mem_map* mm, void* stream) {
  if (!mm) return fail(MEM_ERR_ARG, "NULL argument");
  Map* m = &mm->m;
  CK(cudaStreamSynchronize((cudaStream_t)stream), "stream synchronize");
  int err = 0;
  CK(cudaMemcpy(&err, m->md.err, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
  if (err) {
    CK(cudaMemset(m->md.err, 0, sizeof(int)), "clear error word");
    return fail(MEM_ERR_TIMEOUT, "a bounded device wait ran out (error word %d)", err);
  }
  return MEM_OK;
}
