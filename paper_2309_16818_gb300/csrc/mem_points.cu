// Point-cloud path of the map update (Sec. III-B association + height update +
// Sec. III-C fusion rules), as one fixed kernel sequence:
//
//   k_points_key    transform, range filter and cell key of every point
//                   (+ digit histograms of every radix pass)
//   k_digit_scan    exclusive offsets of each digit
//   k_onesweep      stable LSD radix-sort pass with decoupled look-back,
//                   one per digit (keys = map * W*W + physical cell)
//   k_segments      runs of equal keys = the points of one cell, split into
//                   short runs (one thread each) and long runs (one warp each)
//   k_fuse_small /  per cell: outlier gate + Kalman height update, then every
//   k_fuse_large    multi-modal layer's rule; no float atomics, fixed
//                   summation order, so results are run-to-run identical
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
  extern __shared__ u32 shist[];  // [passes][RADIX]
  for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x) shist[i] = 0;
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
  __syncthreads();
  for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x)
    if (shist[i]) atomicAdd(&md.hist[i], shist[i]);
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
        int k = tile - 1;
        u32 spins = 0;
        for (;;) {
          const u32 v = ld_relaxed(lb + (size_t)k * RADIX + d);
          if ((v & kLbFlags) == 0) {
            if (++spins > kSpinLimit) {
              atomicExch(md.err, kDevErrTimeout);
              break;
            }
            __nanosleep(100);
            continue;
          }
          excl += v & kLbVal;
          if ((v & kLbP) || k == 0) break;
          --k;
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
// 4. segments: runs of equal keys in the sorted order

__device__ __forceinline__ void warp_append(bool pred, uint2 v, uint2* list, u32* counter) {
  const u32 m = __ballot_sync(0xffffffffu, pred);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  u32 b = 0;
  if (lane == leader) b = atomicAdd(counter, (u32)__popc(m));
  b = __shfl_sync(0xffffffffu, b, leader);
  if (pred) list[b + __popc(m & ((1u << lane) - 1u))] = v;
}

__global__ void __launch_bounds__(256) k_segments(MapDev md, const PointJob* __restrict__ job,
                                                  int sorted1, int small_max) {
  const u32* __restrict__ sk = sorted1 ? md.keys1 : md.keys0;
  const int64_t n = job->n;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t i = base + lane;
    bool head = false;
    int64_t e = 0;
    if (i < n) {
      const u32 k = sk[i];
      if (k != md.sentinel && (i == 0 || sk[i - 1] != k)) {
        head = true;
        int64_t lo = i, hi = n, step = 1;
        for (;;) {  // gallop to bracket the end of the run
          const int64_t p = i + step;
          if (p >= n) break;
          if (sk[p] != k) {
            hi = p;
            break;
          }
          lo = p;
          step <<= 1;
        }
        while (hi - lo > 1) {
          const int64_t mid = (lo + hi) >> 1;
          if (sk[mid] == k) lo = mid;
          else hi = mid;
        }
        e = hi;
      }
    }
    const bool small = head && (e - i) <= small_max;
    const uint2 v = make_uint2((u32)i, (u32)e);
    warp_append(small, v, md.seg_small, &md.counters[4]);
    warp_append(head && !small, v, md.seg_large, &md.counters[5]);
    // kept points (statistics)
    u32 kept = head ? (u32)(e - i) : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
    if (lane == 0 && kept) atomicAdd(&md.counters[6], kept);
  }
}

// ---------------------------------------------------------------------------
// 5. per-cell fusion

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
      const float P = __fadd_rn(__frcp_rn(v0), a.sw);
      h = __fdiv_rn(__fadd_rn(__fdiv_rn(h0, v0), a.swz), P);
      v = __frcp_rn(P);
    } else {
      h = __fdiv_rn(a.swz, a.sw);
      v = __frcp_rn(a.sw);
      fl |= kFlagValid;
    }
  }
  if (a.nr > 0 && md.outlier_var != 0.f) v = __fmaf_rn(md.outlier_var, (float)a.nr, v);
  md.h[g] = h;
  md.var[g] = v;
  md.n_acc[g] += a.na;
  md.n_rej[g] += a.nr;
}

// rules of every layer bound to source q, for channels c0..c0+3, after the
// sums S / maxima M of the cell's N points are known
__device__ __forceinline__ void apply_chunk(const MapDev& md, const SrcDev& src, int64_t g, u32 fl,
                                            int c0, float N, const float S[4], const float gv[kMaxSrcLayers]) {
  const int nc = min(4, src.C - c0);
  for (int b = 0; b < src.n_layers; ++b) {
    const int l = src.layers[b];
    const LayerDev& L = md.L[l];
    if (L.rule == MEM_RULE_CLASSMAX) continue;
    const bool obs = fl & (2u << l);
    for (int k = 0; k < nc; ++k) apply_rule_ch(L, g, c0 + k, N, S[k], obs, gv[b]);
  }
}

__device__ __forceinline__ void finish_source(const MapDev& md, const SrcDev& src, int64_t g, u32& fl,
                                              float N, float best, int bid, const float gv[kMaxSrcLayers]) {
  for (int b = 0; b < src.n_layers; ++b) {
    const int l = src.layers[b];
    const LayerDev& L = md.L[l];
    const bool obs = fl & (2u << l);
    if (L.rule == MEM_RULE_CLASSMAX) {
      float* d = (float*)L.data + g * 2;
      d[0] = (float)bid;
      d[1] = best;
    } else if (L.rule == MEM_RULE_GAUSS) {
      L.gvar[g] = gauss_new_var(L, N, obs, gv[b]);
    }
  }
  for (int b = 0; b < src.n_layers; ++b) fl |= 2u << src.layers[b];
}

__device__ __forceinline__ void load_gv(const MapDev& md, const SrcDev& src, int64_t g, u32 fl,
                                        float gv[kMaxSrcLayers]) {
  for (int b = 0; b < kMaxSrcLayers; ++b) {
    gv[b] = 0.f;
    if (b < src.n_layers) {
      const int l = src.layers[b];
      if (md.L[l].rule == MEM_RULE_GAUSS && (fl & (2u << l))) gv[b] = md.L[l].gvar[g];
    }
  }
}

// one thread per short segment
__global__ void __launch_bounds__(256) k_fuse_small(MapDev md, const PointJob* __restrict__ job,
                                                    int sorted1) {
  const u32* __restrict__ sk = sorted1 ? md.keys1 : md.keys0;
  const u32* __restrict__ sv = sorted1 ? md.vals1 : md.vals0;
  const u32 ns = *(volatile u32*)&md.counters[4];
  const float* __restrict__ xyz = job->xyz;
  const int n_src = job->n_src;
  for (u32 t = blockIdx.x * blockDim.x + threadIdx.x; t < ns; t += gridDim.x * blockDim.x) {
    const uint2 se = md.seg_small[t];
    const u32 key = sk[se.x];
    const u32 b = md.n_maps > 1 ? key / md.W2 : 0u;
    const MapCall& mc = job->maps[b];
    const int64_t g = key;
    u32 fl = md.flags[g];
    const bool valid = fl & kFlagValid;
    const float h0 = md.h[g], v0 = md.var[g];
    HeightAcc a = {0.f, 0.f, 0u, 0u};
    for (u32 p = se.x; p < se.y; ++p) {
      const int64_t i = sv[p];
      float z, vm;
      eval_zvm(md, mc, __ldg(xyz + 3 * i), __ldg(xyz + 3 * i + 1), __ldg(xyz + 3 * i + 2), z, vm);
      if (valid && gate_reject(z, h0, v0, vm, md.lam2)) {
        ++a.nr;
      } else {
        ++a.na;
        const float w = __frcp_rn(vm);
        a.sw = __fadd_rn(a.sw, w);
        a.swz = __fmaf_rn(z, w, a.swz);
      }
    }
    height_update(md, g, fl, h0, v0, a);
    const float N = (float)(se.y - se.x);
    for (int q = 0; q < n_src; ++q) {
      const SrcDev& src = job->src[q];
      float gv[kMaxSrcLayers];
      load_gv(md, src, g, fl, gv);
      float best = -INFINITY;
      int bid = -1;
      for (int c0 = 0; c0 < src.C; c0 += 4) {
        float S[4] = {0.f, 0.f, 0.f, 0.f}, M[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
        for (u32 p = se.x; p < se.y; ++p) {
          float v[4];
          ld_src4(src, sv[p], c0, v);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            S[k] = __fadd_rn(S[k], v[k]);
            M[k] = v[k] > M[k] ? v[k] : M[k];
          }
        }
        const int nc = min(4, src.C - c0);
        for (int k = 0; k < nc; ++k)
          if (M[k] > best) {
            best = M[k];
            bid = c0 + k;
          }
        apply_chunk(md, src, g, fl, c0, N, S, gv);
      }
      finish_source(md, src, g, fl, N, best, bid, gv);
    }
    md.flags[g] = fl;
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ u32 warp_sum_u(u32 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// one warp per long segment (lanes stride over the points)
__global__ void __launch_bounds__(256) k_fuse_large(MapDev md, const PointJob* __restrict__ job,
                                                    int sorted1) {
  const u32* __restrict__ sk = sorted1 ? md.keys1 : md.keys0;
  const u32* __restrict__ sv = sorted1 ? md.vals1 : md.vals0;
  const u32 nl = *(volatile u32*)&md.counters[5];
  const float* __restrict__ xyz = job->xyz;
  const int n_src = job->n_src;
  const int lane = threadIdx.x & 31;
  const u32 wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u32 nw = (gridDim.x * blockDim.x) >> 5;
  for (u32 t = wid; t < nl; t += nw) {
    const uint2 se = md.seg_large[t];
    const u32 key = sk[se.x];
    const u32 b = md.n_maps > 1 ? key / md.W2 : 0u;
    const MapCall& mc = job->maps[b];
    const int64_t g = key;
    u32 fl = md.flags[g];
    const bool valid = fl & kFlagValid;
    const float h0 = md.h[g], v0 = md.var[g];
    HeightAcc a = {0.f, 0.f, 0u, 0u};
    for (u32 p = se.x + lane; p < se.y; p += 32) {
      const int64_t i = sv[p];
      float z, vm;
      eval_zvm(md, mc, __ldg(xyz + 3 * i), __ldg(xyz + 3 * i + 1), __ldg(xyz + 3 * i + 2), z, vm);
      if (valid && gate_reject(z, h0, v0, vm, md.lam2)) {
        ++a.nr;
      } else {
        ++a.na;
        const float w = __frcp_rn(vm);
        a.sw = __fadd_rn(a.sw, w);
        a.swz = __fmaf_rn(z, w, a.swz);
      }
    }
    a.sw = warp_sum(a.sw);
    a.swz = warp_sum(a.swz);
    a.na = warp_sum_u(a.na);
    a.nr = warp_sum_u(a.nr);
    if (lane == 0) height_update(md, g, fl, h0, v0, a);
    fl = __shfl_sync(0xffffffffu, fl, 0);
    const float N = (float)(se.y - se.x);
    for (int q = 0; q < n_src; ++q) {
      const SrcDev& src = job->src[q];
      float gv[kMaxSrcLayers];
      load_gv(md, src, g, fl, gv);
      float best = -INFINITY;
      int bid = -1;
      for (int c0 = 0; c0 < src.C; c0 += 4) {
        float S[4] = {0.f, 0.f, 0.f, 0.f}, M[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
        for (u32 p = se.x + lane; p < se.y; p += 32) {
          float v[4];
          ld_src4(src, sv[p], c0, v);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            S[k] = __fadd_rn(S[k], v[k]);
            M[k] = v[k] > M[k] ? v[k] : M[k];
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          S[k] = warp_sum(S[k]);
          M[k] = warp_max(M[k]);
        }
        const int nc = min(4, src.C - c0);
        for (int k = 0; k < nc; ++k)
          if (M[k] > best) {
            best = M[k];
            bid = c0 + k;
          }
        if (lane == 0) apply_chunk(md, src, g, fl, c0, N, S, gv);
      }
      if (lane == 0) finish_source(md, src, g, fl, N, best, bid, gv);
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
    k_points_key<RB><<<sms * bps, 256, sizeof(u32) * P * (1 << RB), st>>>(md, d_job, P);
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
    ProfScope ps(m, kProfSegments, st);
    k_segments<<<sms * bps, 256, 0, st>>>(md, d_job, P & 1, m->tune.small_max);
  }
  {
    ProfScope ps(m, kProfFuseSmall, st);
    k_fuse_small<<<sms * bps, 256, 0, st>>>(md, d_job, P & 1);
  }
  {
    ProfScope ps(m, kProfFuseLarge, st);
    k_fuse_large<<<sms * bps, 256, 0, st>>>(md, d_job, P & 1);
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
