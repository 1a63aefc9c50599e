// Point-cloud path of the map update (Sec. III-B association + height update +
// Sec. III-C fusion rules), as one fixed kernel sequence:
//
//   k_points_key    transform, range filter and cell key of every point
//                   (+ digit histograms of every radix pass)
//   k_digit_scan    exclusive offsets of each digit
//   k_onesweep      stable LSD radix-sort pass with decoupled look-back,
//                   one per digit (keys = map * W*W + physical cell)
//   k_fuse_window / per cell: outlier gate + Kalman height update, then every
//   k_fuse_span     multi-modal layer's rule, as a reduce-by-key over 32-point
//                   windows (no float atomics, fixed summation order, so the
//                   results are run-to-run identical)
//
// Every kernel reads its per-call parameters from the device-resident job, so
// the sequence replays unchanged from a CUDA graph.
#include "mem_host.h"

namespace memk {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kTile = kSortThreads * kSortItems;  // keys per radix tile
constexpr u32 kLbA = 1u << 30;                    // aggregate published
constexpr u32 kLbP = 2u << 30;                    // inclusive prefix published
constexpr u32 kLbFlags = 3u << 30;
constexpr u32 kLbVal = (1u << 30) - 1;

__device__ __forceinline__ int find_map(const int64_t* __restrict__ off, int nm, int64_t i) {
  int lo = 0, hi = nm;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// 1. transform + key + histograms

template <int RB>
__global__ void __launch_bounds__(256) k_points_key(MapDev md, const PointJob* __restrict__ job,
                                                    int passes) {
  constexpr int RADIX = 1 << RB;
  extern __shared__ u32 shist[];  // [passes][RADIX], then the kept-point count
  for (int i = threadIdx.x; i <= passes * RADIX; i += blockDim.x) shist[i] = 0;
  __syncthreads();
  const int64_t n = job->n;
  const int nm = job->n_maps;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  // clear this call's look-back words (the sort passes run after this kernel)
  {
    const int64_t words = ((n + kTile - 1) / kTile) * RADIX;
    for (int p = 0; p < passes; ++p) {
      u32* lbp = md.lookback + (size_t)p * md.cap_tiles * RADIX;
      for (int64_t w = gtid; w < words; w += gstride) lbp[w] = 0;
    }
  }
  const float* __restrict__ xyz = job->xyz;
  const bool vec = ((uintptr_t)xyz & 15) == 0;
  const int64_t n4 = (n + 3) >> 2;
  MapCall mc = job->maps[0];
  int cur_b = 0;
  u32 kept = 0;
  for (int64_t q = gtid; q < n4; q += gstride) {
    const int64_t i0 = q * 4;
    float p[12];
    if (vec && i0 + 4 <= n) {
      const float4* v4 = reinterpret_cast<const float4*>(xyz + i0 * 3);
      float4 a = __ldg(v4), b = __ldg(v4 + 1), c = __ldg(v4 + 2);
      p[0] = a.x; p[1] = a.y; p[2] = a.z; p[3] = a.w;
      p[4] = b.x; p[5] = b.y; p[6] = b.z; p[7] = b.w;
      p[8] = c.x; p[9] = c.y; p[10] = c.z; p[11] = c.w;
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) p[k] = (i0 + k / 3 < n) ? __ldg(xyz + i0 * 3 + k) : 0.f;
    }
    u32 keys[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t i = i0 + k;
      keys[k] = md.sentinel;
      if (i >= n) continue;
      int b = 0;
      if (nm > 1) {
        b = find_map(job->offsets, nm, i);
        if (b != cur_b) {
          mc = job->maps[b];
          cur_b = b;
        }
      }
      PointEval e = eval_point(md, mc, p[3 * k], p[3 * k + 1], p[3 * k + 2]);
      const u32 key = e.keep ? (u32)b * md.W2 + phys_cell(md, mc, e.ix, e.iy) : md.sentinel;
      keys[k] = key;
      kept += e.keep ? 1u : 0u;
      for (int ps = 0; ps < passes; ++ps)
        atomicAdd(&shist[ps * RADIX + ((key >> (ps * RB)) & (RADIX - 1))], 1u);
    }
    if (i0 + 4 <= n) {
      *reinterpret_cast<uint4*>(md.keys0 + i0) = make_uint4(keys[0], keys[1], keys[2], keys[3]);
    } else {
      for (int k = 0; k < 4; ++k)
        if (i0 + k < n) md.keys0[i0 + k] = keys[k];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
  if ((threadIdx.x & 31) == 0 && kept) atomicAdd(&shist[passes * RADIX], kept);
  __syncthreads();
  for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x)
    if (shist[i]) atomicAdd(&md.hist[i], shist[i]);
  if (threadIdx.x == 0 && shist[passes * RADIX]) atomicAdd(&md.counters[6], shist[passes * RADIX]);
}

// 2. digit counts -> exclusive digit offsets, for every pass (one block of 1024)
__global__ void __launch_bounds__(1024) k_digit_scan(MapDev md, int passes, int radix) {
  __shared__ u32 wsum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int p = 0; p < passes; ++p) {
    u32* h = md.hist + p * radix;
    u32 x = threadIdx.x < radix ? h[threadIdx.x] : 0u;
    u32 inc = x;
    for (int o = 1; o < 32; o <<= 1) {
      u32 y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    u32 base = 0;
    for (int w = 0; w < warp; ++w) base += wsum[w];
    __syncthreads();
    if (threadIdx.x < radix) h[threadIdx.x] = base + inc - x;
    __syncthreads();
  }
}

// 3. one stable radix pass (onesweep: tiles taken in order from a counter,
//    global digit prefixes by decoupled look-back with bounded waits)
template <int RB>
__global__ void __launch_bounds__(kSortThreads) k_onesweep(MapDev md, const PointJob* __restrict__ job,
                                                           int pass) {
  constexpr int RADIX = 1 << RB;
  constexpr int WARPS = kSortThreads / 32;
  constexpr int RPT = RADIX / kSortThreads;
  extern __shared__ __align__(16) u32 sm[];
  u32* whist = sm;                       // [WARPS][RADIX]
  u32* skeys = whist + WARPS * RADIX;    // [kTile]
  u32* svals = skeys + kTile;            // [kTile]
  u32* scnt = svals + kTile;             // [RADIX]
  int* sstart = (int*)(scnt + RADIX);    // [RADIX]
  int* sgbase = sstart + RADIX;          // [RADIX]
  __shared__ int s_tile;
  __shared__ u32 s_wsum[WARPS];

  const int64_t n = job->n;
  const int n_tiles = (int)((n + kTile - 1) / kTile);
  const int shift = pass * RB;
  const u32* __restrict__ kin = (pass & 1) ? md.keys1 : md.keys0;
  u32* __restrict__ kout = (pass & 1) ? md.keys0 : md.keys1;
  const u32* __restrict__ vin = (pass & 1) ? md.vals1 : md.vals0;
  u32* __restrict__ vout = (pass & 1) ? md.vals0 : md.vals1;
  const u32* gdig = md.hist + pass * RADIX;
  u32* lb = md.lookback + (size_t)pass * md.cap_tiles * RADIX;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 lt = (1u << lane) - 1u;

  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&md.counters[pass], 1);
    for (int d = threadIdx.x; d < WARPS * RADIX; d += kSortThreads) whist[d] = 0;
    __syncthreads();
    const int tile = s_tile;
    if (tile >= n_tiles) break;
    const int64_t base = (int64_t)tile * kTile;
    const int64_t wbase = base + warp * (kSortItems * 32);
    u32 key[kSortItems], val[kSortItems], rnk[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      const int64_t idx = wbase + j * 32 + lane;
      const bool ok = idx < n;
      key[j] = ok ? kin[idx] : 0xffffffffu;
      val[j] = ok ? (pass == 0 ? (u32)idx : vin[idx]) : 0u;
    }
    // ranks within the warp, in (item, lane) order = input order
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      const bool ok = wbase + j * 32 + lane < n;
      const u32 d = ok ? (key[j] >> shift) & (RADIX - 1) : (u32)RADIX;
      const u32 peers = __match_any_sync(0xffffffffu, d);
      const int leader = __ffs(peers) - 1;
      u32 b = 0;
      if (ok && lane == leader) {
        b = whist[warp * RADIX + d];
        whist[warp * RADIX + d] = b + __popc(peers);
      }
      b = __shfl_sync(0xffffffffu, b, leader);
      rnk[j] = b + __popc(peers & lt);
      __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps per digit; tile count per digit
    for (int d = threadIdx.x; d < RADIX; d += kSortThreads) {
      u32 run = 0;
#pragma unroll
      for (int w = 0; w < WARPS; ++w) {
        u32 t = whist[w * RADIX + d];
        whist[w * RADIX + d] = run;
        run += t;
      }
      scnt[d] = run;
    }
    __syncthreads();
    // exclusive prefix over digits inside the tile
    {
      u32 loc[RPT];
      u32 tsum = 0;
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        loc[r] = scnt[threadIdx.x * RPT + r];
        tsum += loc[r];
      }
      u32 inc = tsum;
      for (int o = 1; o < 32; o <<= 1) {
        u32 y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      if (lane == 31) s_wsum[warp] = inc;
      __syncthreads();
      u32 run = inc - tsum;
      for (int w = 0; w < warp; ++w) run += s_wsum[w];
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        sstart[threadIdx.x * RPT + r] = (int)run;
        run += loc[r];
      }
    }
    // publish this tile's counts, then look back for the exclusive prefix
    for (int d = threadIdx.x; d < RADIX; d += kSortThreads) {
      const u32 c = scnt[d];
      u32* me = lb + (size_t)tile * RADIX + d;
      u32 excl = 0;
      if (tile == 0) {
        st_relaxed(me, kLbP | c);
      } else {
        st_relaxed(me, kLbA | c);
        // walk back 8 predecessors per round: add aggregates until an
        // inclusive prefix is found; wait (bounded) where one is not ready
        int k = tile - 1;
        u32 spins = 0;
        for (;;) {
          u32 v[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) v[j] = (k - j >= 0) ? ld_relaxed(lb + (size_t)(k - j) * RADIX + d) : kLbP;
          int adv = 8;
          bool fin = false, wait = false;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            if (!fin && !wait) {
              const u32 f = v[j] & kLbFlags;
              if (f == 0) {
                wait = true;
                adv = j;
              } else {
                excl += v[j] & kLbVal;
                if (f == kLbP) fin = true;
              }
            }
          }
          if (fin) break;
          k -= adv;
          if (wait) {
            if (++spins > kSpinLimit) {
              atomicExch(md.err, kDevErrTimeout);
              break;
            }
            __nanosleep(32);
          }
        }
        st_relaxed(me, kLbP | ((excl + c) & kLbVal));
      }
      sgbase[d] = (int)(gdig[d] + excl) - sstart[d];
    }
    __syncthreads();
    // stage the tile in digit order, then write runs of equal digits
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
      if (wbase + j * 32 + lane < n) {
        const u32 d = (key[j] >> shift) & (RADIX - 1);
        const int pos = sstart[d] + (int)whist[warp * RADIX + d] + (int)rnk[j];
        skeys[pos] = key[j];
        svals[pos] = val[j];
      }
    }
    __syncthreads();
    const int tile_n = (int)min((int64_t)kTile, n - base);
    for (int i = threadIdx.x; i < tile_n; i += kSortThreads) {
      const u32 k = skeys[i];
      const int64_t dst = (int64_t)sgbase[(k >> shift) & (RADIX - 1)] + i;
      if (dst >= 0 && dst < n) {  // always true unless a look-back wait gave up
        kout[dst] = k;
        vout[dst] = svals[i];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// 4. per-cell fusion, as a reduce-by-key over the sorted points
//
// k_fuse_window: one warp per window of 32 consecutive sorted points, one
//   lane per point. Every lane issues its loads at once (point, source rows,
//   its cell's prior state), then the per-cell sums and maxima are formed by
//   segmented scans across the lanes. A cell whose points all lie in the
//   window is finished right there by the lane holding its last point. A cell
//   that crosses a window boundary leaves one partial record per window it
//   touches: slot 1 of the window where it starts, slot 0 of every later
//   window (flagged on the window where it ends).
// k_fuse_span: one warp per window whose slot 1 holds a crossing cell adds
//   the cell's records in window order and applies the rules (lane c owns
//   channel c).
// The float32 summation order only depends on the sorted order, which is
// deterministic: results are identical from run to run.

// record header (floats): sum w, sum w z, accepted (bits), rejected (bits),
// flag (bits), cell key (bits), 2 unused
constexpr int kRecHdr = 8;
constexpr u32 kRecStart = 1u;  // slot 1: a crossing cell starts in this window
constexpr u32 kRecMore = 1u;   // slot 0: the cell continues past this window
constexpr u32 kRecLast = 2u;   // slot 0: the cell ends in this window

// map-frame z and measurement variance of a point already known to be kept
// (the same operation sequence as eval_point, so the same bits)
__device__ __forceinline__ void eval_zvm(const MapDev& md, const MapCall& mc, float xs, float ys,
                                         float zs, float& z, float& vm) {
  float r2 = __fmaf_rn(xs, xs, __fmaf_rn(ys, ys, __fmul_rn(zs, zs)));
  float rs = __fsqrt_rn(r2);
  z = __fmaf_rn(mc.R[6], xs, __fmaf_rn(mc.R[7], ys, __fmaf_rn(mc.R[8], zs, mc.t[2])));
  float sm = __fmaf_rn(md.sigma1, rs, md.sigma0);
  vm = __fmul_rn(sm, sm);
}

struct HeightAcc {
  float sw, swz;
  u32 na, nr;
};

// Kalman height update in information form (float32) + cumulative counts.
__device__ __forceinline__ void height_update(const MapDev& md, int64_t g, u32& fl, float h0, float v0,
                                              const HeightAcc& a) {
  float h = h0, v = v0;
  if (a.na > 0) {
    if (fl & kFlagValid) {
      const float P = __frcp_rn(v0) + a.sw;
      h = (h0 * __frcp_rn(v0) + a.swz) * __frcp_rn(P);
      v = __frcp_rn(P);
    } else {
      h = a.swz * __frcp_rn(a.sw);
      v = __frcp_rn(a.sw);
      fl |= kFlagValid;
    }
  }
  if (a.nr > 0 && md.outlier_var != 0.f) v = fmaf(md.outlier_var, (float)a.nr, v);
  md.h[g] = h;
  md.var[g] = v;
  md.n_acc[g] += a.na;
  md.n_rej[g] += a.nr;
}

// coefficients of layer l for one cell
__device__ __forceinline__ RuleCoef layer_coef(const MapDev& md, int l, int64_t g, u32 fl, float N, float rN) {
  const LayerDev& L = md.L[l];
  const bool obs = fl & (2u << l);
  const float s02 = (L.rule == MEM_RULE_GAUSS && obs) ? L.gvar[g] : 0.f;
  return rule_coef(L, N, rN, obs, s02);
}

// class-max and Gaussian-variance writes after all channels of a source
__device__ __forceinline__ void finish_source(const MapDev& md, const SrcDev& src, int64_t g, u32& fl,
                                              float N, float rN, float best, int bid) {
  for (int b = 0; b < src.n_layers; ++b) {
    const int l = src.layers[b];
    const LayerDev& L = md.L[l];
    if (L.rule == MEM_RULE_CLASSMAX) {
      float* d = (float*)L.data + g * 2;
      d[0] = (float)bid;
      d[1] = best;
    } else if (L.rule == MEM_RULE_GAUSS) {
      L.gvar[g] = layer_coef(md, l, g, fl, N, rN).var_new;
    }
  }
  for (int b = 0; b < src.n_layers; ++b) fl |= 2u << src.layers[b];
}

// old values of four channels of a layer (vector access when possible)
__device__ __forceinline__ void ld_old4(const LayerDev& L, int64_t off, int nc, float o[4]) {
  if (nc == 4 && (off & 3) == 0 && L.dtype == MEM_F32) {
    const float4 q = *reinterpret_cast<const float4*>((const float*)L.data + off);
    o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
    return;
  }
  if (nc == 4 && (off & 3) == 0 && L.dtype == MEM_BF16) {
    const uint2 q = *reinterpret_cast<const uint2*>((const __nv_bfloat16*)L.data + off);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.y));
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    return;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) o[k] = k < nc ? ld_layer(L, off + k) : 0.f;
}

__device__ __forceinline__ void st_new4(const LayerDev& L, int64_t off, int nc, const float n[4]) {
  if (nc == 4 && (off & 3) == 0 && L.dtype == MEM_F32) {
    *reinterpret_cast<float4*>((float*)L.data + off) = make_float4(n[0], n[1], n[2], n[3]);
    return;
  }
  if (nc == 4 && (off & 3) == 0 && L.dtype == MEM_BF16) {
    __nv_bfloat162 a = __floats2bfloat162_rn(n[0], n[1]), b = __floats2bfloat162_rn(n[2], n[3]);
    uint2 q;
    q.x = *reinterpret_cast<u32*>(&a);
    q.y = *reinterpret_cast<u32*>(&b);
    *reinterpret_cast<uint2*>((__nv_bfloat16*)L.data + off) = q;
    return;
  }
  for (int k = 0; k < nc; ++k) st_layer(L, off + k, n[k]);
}

// segmented inclusive scans over the lanes of a warp: `use[s]` says whether
// the lane 2^s positions down belongs to the same run
__device__ __forceinline__ float seg_sum(float v, const bool use[5]) {
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const float y = __shfl_up_sync(0xffffffffu, v, 1 << s);
    if (use[s]) v += y;
  }
  return v;
}
__device__ __forceinline__ u32 seg_sum_u(u32 v, const bool use[5]) {
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const u32 y = __shfl_up_sync(0xffffffffu, v, 1 << s);
    if (use[s]) v += y;
  }
  return v;
}
__device__ __forceinline__ float seg_max(float v, const bool use[5]) {
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const float y = __shfl_up_sync(0xffffffffu, v, 1 << s);
    if (use[s]) v = fmaxf(v, y);
  }
  return v;
}

constexpr int kPre = 4;   // layers per source whose coefficients stay in registers
constexpr int kBlk = 16;  // channels per block in the window kernel

// typed access to four consecutive stored values
template <int DT>
__device__ __forceinline__ void ld4t(const void* base, int64_t off, float o[4]) {
  if (DT == MEM_F32) {
    const float4 q = *reinterpret_cast<const float4*>((const float*)base + off);
    o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
  } else if (DT == MEM_BF16) {
    const uint2 q = *reinterpret_cast<const uint2*>((const __nv_bfloat16*)base + off);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.y));
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  } else {
    const uint2 q = *reinterpret_cast<const uint2*>((const __half*)base + off);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&q.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  }
}
template <int DT>
__device__ __forceinline__ void st4t(void* base, int64_t off, const float n[4]) {
  if (DT == MEM_F32) {
    *reinterpret_cast<float4*>((float*)base + off) = make_float4(n[0], n[1], n[2], n[3]);
  } else if (DT == MEM_BF16) {
    __nv_bfloat162 a = __floats2bfloat162_rn(n[0], n[1]), b = __floats2bfloat162_rn(n[2], n[3]);
    uint2 q;
    q.x = *reinterpret_cast<u32*>(&a);
    q.y = *reinterpret_cast<u32*>(&b);
    *reinterpret_cast<uint2*>((__nv_bfloat16*)base + off) = q;
  } else {
    __half2 a = __floats2half2_rn(n[0], n[1]), b = __floats2half2_rn(n[2], n[3]);
    uint2 q;
    q.x = *reinterpret_cast<u32*>(&a);
    q.y = *reinterpret_cast<u32*>(&b);
    *reinterpret_cast<uint2*>((__half*)base + off) = q;
  }
}
template <int DT>
__device__ __forceinline__ float ld1t(const void* base, int64_t off) {
  if (DT == MEM_F32) return ((const float*)base)[off];
  if (DT == MEM_BF16) return __bfloat162float(((const __nv_bfloat16*)base)[off]);
  return __half2float(((const __half*)base)[off]);
}
template <int DT>
__device__ __forceinline__ void st1t(void* base, int64_t off, float v) {
  if (DT == MEM_F32) ((float*)base)[off] = v;
  else if (DT == MEM_BF16) ((__nv_bfloat16*)base)[off] = __float2bfloat16_rn(v);
  else ((__half*)base)[off] = __float2half_rn(v);
}

template <int RULE>
__device__ __forceinline__ float rule_value_t(const LayerDev& L, float old, float S, const RuleCoef& r) {
  if (RULE == MEM_RULE_LATEST) return S * r.a;
  if (RULE == MEM_RULE_EXPAVG) {
    const float a = S * r.a;
    return r.obs ? fmaf(L.w, a, L.one_minus_w * old) : a;
  }
  if (RULE == MEM_RULE_GAUSS) return r.obs ? fmaf(r.a, old, r.b * S) : S * r.a;
  return (r.obs ? old : L.alpha0) + S;  // DIRICHLET
}

// One layer's rule over a block of nb <= kBlk channels starting at `off`:
// every old value of the block is loaded before any new value is stored.
template <int RULE, int DT>
__device__ __forceinline__ void apply_block_t(const LayerDev& L, int64_t off, const float S[kBlk], int nb,
                                              const RuleCoef& r) {
  const bool need = RULE != MEM_RULE_LATEST && r.obs;
  float o[kBlk];
  const bool vec = (off & 3) == 0;
#pragma unroll
  for (int j = 0; j < kBlk / 4; ++j) {
    o[4 * j] = o[4 * j + 1] = o[4 * j + 2] = o[4 * j + 3] = 0.f;
    if (need && 4 * j < nb) {
      if (vec && 4 * j + 4 <= nb) {
        ld4t<DT>(L.data, off + 4 * j, &o[4 * j]);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (4 * j + k < nb) o[4 * j + k] = ld1t<DT>(L.data, off + 4 * j + k);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kBlk / 4; ++j) {
    if (4 * j < nb) {
      float n[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) n[k] = rule_value_t<RULE>(L, o[4 * j + k], S[4 * j + k], r);
      if (vec && 4 * j + 4 <= nb) {
        st4t<DT>(L.data, off + 4 * j, n);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (4 * j + k < nb) st1t<DT>(L.data, off + 4 * j + k, n[k]);
      }
    }
  }
}

__device__ __forceinline__ void apply_block(const LayerDev& L, int64_t off, const float S[kBlk], int nb,
                                              const RuleCoef& r) {
#define MEM_AB(R, D) \
  case R * 4 + D: apply_block_t<R, D>(L, off, S, nb, r); break;
  switch (L.rule * 4 + L.dtype) {
    MEM_AB(MEM_RULE_LATEST, MEM_F32) MEM_AB(MEM_RULE_LATEST, MEM_BF16) MEM_AB(MEM_RULE_LATEST, MEM_F16)
    MEM_AB(MEM_RULE_EXPAVG, MEM_F32) MEM_AB(MEM_RULE_EXPAVG, MEM_BF16) MEM_AB(MEM_RULE_EXPAVG, MEM_F16)
    MEM_AB(MEM_RULE_GAUSS, MEM_F32) MEM_AB(MEM_RULE_GAUSS, MEM_BF16) MEM_AB(MEM_RULE_GAUSS, MEM_F16)
    MEM_AB(MEM_RULE_DIRICHLET, MEM_F32)
    default: break;
  }
#undef MEM_AB
}

__global__ void __launch_bounds__(256) k_fuse_window(MapDev md, const PointJob* __restrict__ job,
                                                     int sorted1) {
  const u32* __restrict__ sk = sorted1 ? md.keys1 : md.keys0;
  const u32* __restrict__ sv = sorted1 ? md.vals1 : md.vals0;
  const int64_t n_kept = *(volatile u32*)&md.counters[6];
  const float* __restrict__ xyz = job->xyz;
  const int n_src = job->n_src;
  const int acc = job->acc;
  float* __restrict__ part = md.partial;
  const int lane = threadIdx.x & 31;
  const u32 lt = (1u << lane) - 1u;
  const int64_t n_win = (n_kept + 31) >> 5;
  const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n_win; w += wstride) {
    const int64_t p = w * 32 + lane;
    const bool active = p < n_kept;
    const u32 key = active ? sk[p] : 0xffffffffu;
    const u32 idx = active ? sv[p] : 0u;
    // neighbours (lane 0 / lane 31 look across the window edge)
    u32 prev = __shfl_up_sync(0xffffffffu, key, 1);
    u32 next = __shfl_down_sync(0xffffffffu, key, 1);
    if (lane == 0) prev = p > 0 ? sk[p - 1] : 0xfffffffeu;
    if (lane == 31) next = (p + 1 < n_kept) ? sk[p + 1] : 0xfffffffeu;
    const bool ghead = active && prev != key;                 // first point of its cell
    const bool gend = active && next != key;                  // last point of its cell
    const bool lhead = active && (lane == 0 || prev != key);  // first point of the run in this window
    const bool lend = active && (lane == 31 || next != key);  // last point of the run in this window
    const u32 heads = __ballot_sync(0xffffffffu, lhead);
    const int rs = 31 - __clz(heads & (lt | (1u << lane)));  // run start lane
    bool use[5];
#pragma unroll
    for (int s = 0; s < 5; ++s) use[s] = lane - (1 << s) >= rs;
    const int run_ghead = __shfl_sync(0xffffffffu, (int)ghead, rs & 31);  // all lanes take part
    const int lane0_ghead = __shfl_sync(0xffffffffu, (int)ghead, 0);
    const bool complete = lend && gend && run_ghead != 0;
    const bool partial = lend && !complete;
    const bool from_before = rs == 0 && lane0_ghead == 0;  // run entered from the previous window
    // this lane's cell
    const u32 b = md.n_maps > 1 ? key / md.W2 : 0u;
    const MapCall& mc = job->maps[active ? b : 0u];
    const int64_t g = active ? key : 0;
    u32 fl = active ? md.flags[g] : 0u;
    const float h0 = active ? md.h[g] : 0.f, v0 = active ? md.var[g] : 0.f;
    // height contribution of this point
    HeightAcc a = {0.f, 0.f, 0u, 0u};
    if (active) {
      float z, vm;
      eval_zvm(md, mc, __ldg(xyz + 3 * (int64_t)idx), __ldg(xyz + 3 * (int64_t)idx + 1),
               __ldg(xyz + 3 * (int64_t)idx + 2), z, vm);
      if ((fl & kFlagValid) && gate_reject(z, h0, v0, vm, md.lam2)) {
        a.nr = 1;
      } else {
        a.na = 1;
        a.sw = __frcp_rn(vm);
        a.swz = z * a.sw;
      }
    }
    a.sw = seg_sum(a.sw, use);
    a.swz = seg_sum(a.swz, use);
    a.na = seg_sum_u(a.na, use);
    a.nr = seg_sum_u(a.nr, use);
    float* rec = part + ((w * 2 + (from_before ? 0 : 1)) * (int64_t)acc);
    if (complete) height_update(md, g, fl, h0, v0, a);
    if (partial) {
      rec[0] = a.sw;
      rec[1] = a.swz;
      rec[2] = __uint_as_float(a.na);
      rec[3] = __uint_as_float(a.nr);
      rec[4] = __uint_as_float(from_before ? (gend ? kRecLast : kRecMore) : kRecStart);
      rec[5] = __uint_as_float(key);
    }
    // slot 1 of every window says whether a crossing cell starts here
    if (lane == 31) {
      const bool starts = partial && !from_before;
      if (!starts) part[(w * 2 + 1) * (int64_t)acc + 4] = __uint_as_float(0u);
    }
    const float N = (float)(lane - rs + 1), rN = __frcp_rn(N);
    for (int q = 0; q < n_src; ++q) {
      const SrcDev& src = job->src[q];
      // this point's largest class probability (smallest class on ties)
      float pbest = -INFINITY;
      int pbid = 0x7fffffff;
      RuleCoef co[kPre];
#pragma unroll
      for (int bb = 0; bb < kPre; ++bb) {
        co[bb].a = co[bb].b = co[bb].var_new = 0.f;
        co[bb].obs = false;
        if (complete && bb < src.n_layers) co[bb] = layer_coef(md, src.layers[bb], g, fl, N, rN);
      }
      // channels in blocks of 16: loads, per-point arg-max, segmented sums,
      // then each bound layer applies its rule to the whole block (rule and
      // storage type resolved once per layer and block)
      for (int cb = 0; cb < src.C; cb += kBlk) {
        const int nb = min(kBlk, src.C - cb);
        float v[kBlk];
#pragma unroll
        for (int j = 0; j < kBlk / 4; ++j) {
          v[4 * j] = v[4 * j + 1] = v[4 * j + 2] = v[4 * j + 3] = 0.f;
          if (active && 4 * j < nb) ld_src4(src, idx, cb + 4 * j, &v[4 * j]);
        }
        if (src.has_classmax && active) {
#pragma unroll
          for (int k = 0; k < kBlk; ++k)
            if (k < nb && v[k] > pbest) {
              pbest = v[k];
              pbid = cb + k;
            }
        }
        float S[kBlk];
#pragma unroll
        for (int k = 0; k < kBlk; ++k) S[k] = (k < nb) ? seg_sum(v[k], use) : 0.f;
        if (complete) {
          for (int bb = 0; bb < src.n_layers; ++bb) {
            const LayerDev& L = md.L[src.layers[bb]];
            if (L.rule == MEM_RULE_CLASSMAX) continue;
            RuleCoef r;
#pragma unroll
            for (int u = 0; u < kPre; ++u)
              if (u == bb) r = co[u];
            if (bb >= kPre) r = layer_coef(md, src.layers[bb], g, fl, N, rN);
            apply_block(L, g * L.S + cb, S, nb, r);
          }
        }
        if (partial) {
          float* r = rec + src.acc_off + cb;
#pragma unroll
          for (int k = 0; k < kBlk; ++k)
            if (k < nb) r[k] = S[k];
        }
      }
      // class max of the run: one segmented scan of (value, class) pairs
      float best = -INFINITY;
      int bid = -1;
      if (src.has_classmax) {
#pragma unroll
        for (int s = 0; s < 5; ++s) {
          const float ov = __shfl_up_sync(0xffffffffu, pbest, 1 << s);
          const int oi = __shfl_up_sync(0xffffffffu, pbid, 1 << s);
          if (use[s] && (ov > pbest || (ov == pbest && oi < pbid))) {
            pbest = ov;
            pbid = oi;
          }
        }
        best = pbest;
        bid = pbest == -INFINITY ? -1 : pbid;
        if (partial) {
          rec[src.acc_off + src.C] = best;
          rec[src.acc_off + src.C + 1] = __int_as_float(bid);
        }
      }
      if (complete) finish_source(md, src, g, fl, N, rN, best, bid);
    }
    if (complete) md.flags[g] = fl;
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ u32 warp_sum_u(u32 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// record of piece j (0 = the starting window w0) of a crossing cell
__device__ __forceinline__ const float* span_rec(const float* part, int64_t w0, int64_t j, int acc) {
  return part + ((w0 + j) * 2 + (j == 0 ? 1 : 0)) * (int64_t)acc;
}

__global__ void __launch_bounds__(256) k_fuse_span(MapDev md, const PointJob* __restrict__ job) {
  const int64_t n_kept = *(volatile u32*)&md.counters[6];
  const int64_t n_win = (n_kept + 31) >> 5;
  const int n_src = job->n_src;
  const int acc = job->acc;
  const float* __restrict__ part = md.partial;
  const int lane = threadIdx.x & 31;
  const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w0 < n_win; w0 += wstride) {
    const float* r0 = part + (w0 * 2 + 1) * (int64_t)acc;
    if (__float_as_uint(r0[4]) != kRecStart) continue;  // warp-uniform
    // number of pieces: walk the slot-0 flags of the following windows, 32 at a time
    int64_t np = 0;
    for (int64_t j0 = 1;; j0 += 32) {
      const int64_t j = j0 + lane;
      const u32 f = (w0 + j < n_win) ? __float_as_uint(span_rec(part, w0, j, acc)[4]) : kRecLast;
      const u32 last = __ballot_sync(0xffffffffu, f == kRecLast);
      if (last) {
        np = j0 + (__ffs(last) - 1) + 1;
        break;
      }
    }
    const u32 key = __float_as_uint(r0[5]);
    const int64_t g = key;
    u32 fl = md.flags[g];
    const float h0 = md.h[g], v0 = md.var[g];
    // height: lanes over pieces, then a fixed-order tree
    HeightAcc a = {0.f, 0.f, 0u, 0u};
    for (int64_t j = lane; j < np; j += 32) {
      const float* r = span_rec(part, w0, j, acc);
      a.sw += r[0];
      a.swz += r[1];
      a.na += __float_as_uint(r[2]);
      a.nr += __float_as_uint(r[3]);
    }
    a.sw = warp_sum(a.sw);
    a.swz = warp_sum(a.swz);
    a.na = warp_sum_u(a.na);
    a.nr = warp_sum_u(a.nr);
    const float N = (float)(a.na + a.nr), rN = __frcp_rn(N);
    if (lane == 0) height_update(md, g, fl, h0, v0, a);
    fl = __shfl_sync(0xffffffffu, fl, 0);
    for (int q = 0; q < n_src; ++q) {
      const SrcDev& src = job->src[q];
      float best = -INFINITY;
      int bid = -1;
      for (int cb = 0; cb < src.C; cb += 32) {
        const int c = cb + lane;
        const bool on = c < src.C;
        float s = 0.f;
        if (on) {
          int64_t j = 0;
          for (; j + 8 <= np; j += 8) {
            float x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = (span_rec(part, w0, j + u, acc) + src.acc_off)[c];
#pragma unroll
            for (int u = 0; u < 8; ++u) s += x[u];
          }
          for (; j < np; ++j) s += (span_rec(part, w0, j, acc) + src.acc_off)[c];
          for (int bb = 0; bb < src.n_layers; ++bb) {
            const LayerDev& L = md.L[src.layers[bb]];
            if (L.rule != MEM_RULE_CLASSMAX)
              apply_rule(L, g * L.S + c, s, layer_coef(md, src.layers[bb], g, fl, N, rN));
          }
        }
      }
      if (src.has_classmax) {
        // (value, class) of every piece: largest value, smallest class on ties
        float bv = -INFINITY;
        int bi = 0x7fffffff;
        for (int64_t j = lane; j < np; j += 32) {
          const float* r = span_rec(part, w0, j, acc) + src.acc_off + src.C;
          const float ov = r[0];
          const int oi = __float_as_int(r[1]);
          if (ov > bv || (ov == bv && oi < bi)) {
            bv = ov;
            bi = oi;
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ov > bv || (ov == bv && oi < bi)) {
            bv = ov;
            bi = oi;
          }
        }
        best = bv;
        bid = bv == -INFINITY ? -1 : bi;
      }
      if (lane == 0) finish_source(md, src, g, fl, N, rN, best, bid);
      fl = __shfl_sync(0xffffffffu, fl, 0);
    }
    if (lane == 0) md.flags[g] = fl;
  }
}

// time-dependent variance growth of every valid cell
__global__ void k_time_update(MapDev md, int64_t cells) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < cells;
       g += (int64_t)gridDim.x * blockDim.x)
    if (md.flags[g] & kFlagValid) md.var[g] = __fadd_rn(md.var[g], md.time_var);
}

}  // namespace memk

// ---------------------------------------------------------------------------
// host launcher

namespace memh {
using namespace memk;

template <int RB>
static size_t sort_smem() {
  constexpr int RADIX = 1 << RB;
  return sizeof(u32) * ((kSortThreads / 32) * RADIX + 2 * kTile + 3 * RADIX);
}

template <int RB>
static cudaError_t set_attrs() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_onesweep<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sort_smem<RB>());
  if (e == cudaSuccess) done = true;
  return e;
}

template <int RB>
static cudaError_t launch_rb(Map* m, const PointJob* d_job, cudaStream_t st) {
  const MapDev& md = m->md;
  cudaError_t e = set_attrs<RB>();
  if (e != cudaSuccess) return e;
  const int P = m->passes;
  const int sms = m->n_sm;
  const int bps = m->tune.blocks_per_sm;
  // digit histograms + counters are one contiguous block
  e = cudaMemsetAsync(md.hist, 0, sizeof(u32) * (4 * 1024 + 16), st);
  if (e != cudaSuccess) return e;
  {
    ProfScope ps(m, kProfKey, st);
    k_points_key<RB><<<sms * bps, 256, sizeof(u32) * (P * (1 << RB) + 1), st>>>(md, d_job, P);
  }
  {
    ProfScope ps(m, kProfDigits, st);
    k_digit_scan<<<1, 1024, 0, st>>>(md, P, 1 << RB);
  }
  {
    ProfScope ps(m, kProfSort, st);
    for (int p = 0; p < P; ++p) k_onesweep<RB><<<sms * 2, kSortThreads, sort_smem<RB>(), st>>>(md, d_job, p);
  }
  {
    ProfScope ps(m, kProfFuseWindow, st);
    k_fuse_window<<<sms * bps, 256, 0, st>>>(md, d_job, P & 1);
  }
  {
    ProfScope ps(m, kProfFuseSpan, st);
    k_fuse_span<<<sms * bps, 256, 0, st>>>(md, d_job);
  }
  if (md.time_var != 0.f) {
    ProfScope ps(m, kProfTime, st);
    const int64_t cells = (int64_t)md.n_maps * md.W2;
    k_time_update<<<sms * bps, 256, 0, st>>>(md, cells);
  }
  return cudaGetLastError();
}

cudaError_t prepare_kernels() {
  cudaError_t e = set_attrs<8>();
  if (e == cudaSuccess) e = set_attrs<9>();
  if (e == cudaSuccess) e = set_attrs<10>();
  return e;
}

cudaError_t launch_point_fuse(Map* m, const PointJob* d_job, cudaStream_t st) {
  switch (m->tune.radix_bits) {
    case 8: return launch_rb<8>(m, d_job, st);
    case 9: return launch_rb<9>(m, d_job, st);
    case 10: return launch_rb<10>(m, d_job, st);
  }
  return cudaErrorInvalidValue;
}

int key_bits_for(const Map* m) {
  const uint64_t top = (uint64_t)m->md.sentinel;  // largest key
  int b = 1;
  while (b < 32 && (top >> b) != 0) ++b;
  return b;
}

}  // namespace memh
