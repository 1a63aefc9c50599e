// Point-cloud path of the map update (Sec. III-B association + height update +
// Sec. III-C fusion rules), as one fixed kernel sequence:
//
//   k_points_key    transform, range filter and cell key of every point
//                   (+ digit histograms of every radix pass)
//   k_onesweep      stable LSD radix-sort pass with decoupled look-back,
//                   one per digit (keys = map * W*W + physical cell); each
//                   CTA first scans the digit counts into global offsets
//   k_fuse_tiles    per tile of sorted points: outlier gate, sums of every
//                   cell's quantities (a reduce-by-key in a fixed order), then
//                   for the cells inside the tile the Kalman height update and
//                   every multi-modal layer's rule
//   k_fuse_cross    the same for the cells whose points cross tiles (no float
//                   atomics, fixed summation order: run-to-run identical)
//
// Every kernel reads its per-call parameters from the device-resident job, so
// the sequence replays unchanged from a CUDA graph.
#include "mem_host.h"

namespace memk {

constexpr int kTile = kSortTile;  // keys per radix tile
constexpr u32 kLbA = 1u << 30;                    // aggregate published
constexpr u32 kLbP = 2u << 30;                    // inclusive prefix published
constexpr u32 kLbFlags = 3u << 30;
constexpr u32 kLbVal = (1u << 30) - 1;
constexpr int kLookBack = 16;                     // predecessors read per look-back round

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
  if (*(volatile int*)md.err) return;  // a device error is pending: the point path does nothing
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
  u32 kept = 0, dropped = 0;
  const int lane = threadIdx.x & 31;
  const bool drift = md.drift_alpha != 0.0;
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
    float pe[4];  // drift compensation: z - h of a point that enters the mean height error, else NaN
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t i = i0 + k;
      keys[k] = md.sentinel;
      pe[k] = __int_as_float(0x7fc00000);
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
      if (drift && e.keep && (md.flags[key] & kFlagValid)) {
        // the z error count: a point of a valid cell that the gate accepts (pre-call state)
        const float h = md.h[key];
        if (!gate_reject(e.z, h, md.var[key], e.vm, md.lam2)) pe[k] = __fsub_rn(e.z, h);
      }
      kept += e.keep ? 1u : 0u;
      dropped += e.keep ? 0u : 1u;
    }
    // kept points' digits; dropped points (the sentinel key) are counted once per thread
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (i0 + k < n && keys[k] != md.sentinel)
        for (int ps = 0; ps < passes; ++ps) atomicAdd(&shist[ps * RADIX + ((keys[k] >> (ps * RB)) & (RADIX - 1))], 1u);
    if (i0 + 4 <= n) {
      *reinterpret_cast<uint4*>(md.keys0 + i0) = make_uint4(keys[0], keys[1], keys[2], keys[3]);
      if (drift) *reinterpret_cast<float4*>(md.perr + i0) = make_float4(pe[0], pe[1], pe[2], pe[3]);
    } else {
      for (int k = 0; k < 4; ++k)
        if (i0 + k < n) {
          md.keys0[i0 + k] = keys[k];
          if (drift) md.perr[i0 + k] = pe[k];
        }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    kept += __shfl_xor_sync(0xffffffffu, kept, o);
    dropped += __shfl_xor_sync(0xffffffffu, dropped, o);
  }
  if (lane == 0 && kept) atomicAdd(&shist[passes * RADIX], kept);
  if (lane == 0 && dropped)
    for (int ps = 0; ps < passes; ++ps) atomicAdd(&shist[ps * RADIX + ((md.sentinel >> (ps * RB)) & (RADIX - 1))], dropped);
  __syncthreads();
  for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x)
    if (shist[i]) atomicAdd(&md.hist[i], shist[i]);
  if (threadIdx.x == 0 && shist[passes * RADIX]) atomicAdd(&md.counters[6], shist[passes * RADIX]);
}

// 2. drift compensation: per map, the mean of the height errors of the points
//    that enter it (fixed assignment of points to threads and a fixed reduction
//    tree, in float64), then every valid height of the map moves by
//    float32(alpha * mean) when enough points entered it

__global__ void __launch_bounds__(256) k_drift_reduce(MapDev md, const PointJob* __restrict__ job) {
  if (*(volatile int*)md.err) return;  // a device error is pending: the point path does nothing
  const int b = blockIdx.y, r = blockIdx.x;
  int64_t o0 = 0, o1 = job->n;
  if (job->offsets) {
    o0 = job->offsets[b];
    o1 = job->offsets[b + 1];
  }
  const int64_t len = o1 - o0;
  const int R = md.drift_R;
  const int64_t c0 = o0 + len * r / R, c1 = o0 + len * (r + 1) / R;
  double sum = 0.0, cnt = 0.0;
  for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
    const float e = md.perr[i];
    if (!isnan(e)) {
      sum += (double)e;
      cnt += 1.0;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  __shared__ double ws[8][2];
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    ws[warp][0] = sum;
    ws[warp][1] = cnt;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0, Cn = 0.0;
    for (int w = 0; w < 8; ++w) {
      S += ws[w][0];
      Cn += ws[w][1];
    }
    md.dpart[((int64_t)b * R + r) * 2] = S;
    md.dpart[((int64_t)b * R + r) * 2 + 1] = Cn;
  }
}

__global__ void __launch_bounds__(256) k_drift_apply(MapDev md) {
  if (*(volatile int*)md.err) return;  // a device error is pending: the point path does nothing
  const int b = blockIdx.y;
  __shared__ float s_shift;
  if (threadIdx.x < 32) {  // the map's partials: lanes over a fixed stride, then a fixed tree
    const int R = md.drift_R;
    double S = 0.0, Cn = 0.0;
    for (int r = threadIdx.x; r < R; r += 32) {
      S += md.dpart[((int64_t)b * R + r) * 2];
      Cn += md.dpart[((int64_t)b * R + r) * 2 + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      S += __shfl_xor_sync(0xffffffffu, S, o);
      Cn += __shfl_xor_sync(0xffffffffu, Cn, o);
    }
    if (threadIdx.x == 0) {
      float shift = 0.f;
      if (Cn > 0.0 && Cn >= (double)md.drift_min) shift = (float)(md.drift_alpha * (S / Cn));
      s_shift = shift;
      if (blockIdx.x == 0) {
        md.drift_out[2 * b] = shift;
        md.drift_out[2 * b + 1] = __uint_as_float((u32)Cn);
      }
    }
  }
  __syncthreads();
  const float shift = s_shift;
  if (shift == 0.f) return;
  const int64_t base = (int64_t)b * md.W2;
  for (u32 j = blockIdx.x * blockDim.x + threadIdx.x; j < md.W2; j += gridDim.x * blockDim.x)
    if (md.flags[base + j] & kFlagValid) md.h[base + j] = __fadd_rn(md.h[base + j], shift);
}

// 3. one stable radix pass (onesweep: tiles taken in order from a counter,
//    global digit prefixes by decoupled look-back with bounded waits)
template <int RB>
__global__ void __launch_bounds__(kSortThreads, 2) k_onesweep(MapDev md, const PointJob* __restrict__ job,
                                                           int pass) {
  constexpr int RADIX = 1 << RB;
  constexpr int WARPS = kSortThreads / 32;
  constexpr int RPT = (RADIX + kSortThreads - 1) / kSortThreads;  // digits per thread (threads past RADIX: none)
  extern __shared__ __align__(16) u32 sm[];
  u32* whist = sm;                       // [WARPS][RADIX]
  u32* skeys = whist + WARPS * RADIX;    // [kTile]
  u32* svals = skeys + kTile;            // [kTile]
  u32* scnt = svals + kTile;             // [RADIX]
  int* sstart = (int*)(scnt + RADIX);    // [RADIX]
  int* sgbase = sstart + RADIX;          // [RADIX]
  u32* sgdig = (u32*)(sgbase + RADIX);   // [RADIX] exclusive offsets of the digits over all keys
  __shared__ int s_tile;
  __shared__ u32 s_wsum[WARPS];
  __shared__ volatile int s_fail;  // a look-back wait of this tile ran out: no scatter

  // a device error is pending (the word can be set by other blocks of this pass meanwhile, so the
  // block decides once, through shared memory): the point path does nothing
  if (threadIdx.x == 0) s_fail = *(volatile int*)md.err;
  __syncthreads();
  if (s_fail) return;
  const bool inject = *(volatile int*)(md.err + 1) != 0;  // fault injection (tests): waits run out
  const int64_t n = job->n;
  const int n_tiles = (int)((n + kTile - 1) / kTile);
  const int shift = pass * RB;
  const u32* __restrict__ kin = (pass & 1) ? md.keys1 : md.keys0;
  u32* __restrict__ kout = (pass & 1) ? md.keys0 : md.keys1;
  const u32* __restrict__ vin = (pass & 1) ? md.vals1 : md.vals0;
  u32* __restrict__ vout = (pass & 1) ? md.vals0 : md.vals1;
  u32* lb = md.lookback + (size_t)pass * md.cap_tiles * RADIX;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 lt = (1u << lane) - 1u;
  // exclusive offsets of this pass's digits from the key kernel's counts
  {
    u32 loc[RPT];
    u32 tsum = 0;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      loc[r] = threadIdx.x * RPT + r < RADIX ? md.hist[pass * RADIX + threadIdx.x * RPT + r] : 0u;
      tsum += loc[r];
    }
    u32 inc = tsum;
    for (int o = 1; o < 32; o <<= 1) {
      const u32 y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) s_wsum[warp] = inc;
    __syncthreads();
    u32 run = inc - tsum;
    for (int w = 0; w < warp; ++w) run += s_wsum[w];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      if (threadIdx.x * RPT + r < RADIX) sgdig[threadIdx.x * RPT + r] = run;
      run += loc[r];
    }
    __syncthreads();
  }

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
        loc[r] = threadIdx.x * RPT + r < RADIX ? scnt[threadIdx.x * RPT + r] : 0u;
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
        if (threadIdx.x * RPT + r < RADIX) sstart[threadIdx.x * RPT + r] = (int)run;
        run += loc[r];
      }
    }
    __syncthreads();  // sstart is read below by the thread owning each digit
    // publish this tile's counts, then look back for the exclusive prefix
    for (int d = threadIdx.x; d < RADIX; d += kSortThreads) {
      const u32 c = scnt[d];
      u32* me = lb + (size_t)tile * RADIX + d;
      u32 excl = 0;
      if (tile == 0) {
        st_relaxed(me, kLbP | c);
      } else {
        st_relaxed(me, kLbA | c);
        // walk back kLookBack predecessors per round: add aggregates until
        // an inclusive prefix is found; wait (bounded) where one is not ready
        int k = tile - 1;
        u32 spins = 0;
        bool timed_out = false;
        for (;;) {
          u32 v[kLookBack];
#pragma unroll
          for (int j = 0; j < kLookBack; ++j)
            v[j] = (k - j >= 0) ? ld_relaxed(lb + (size_t)(k - j) * RADIX + d) : kLbP;
          int adv = kLookBack;
          bool fin = false, wait = false;
#pragma unroll
          for (int j = 0; j < kLookBack; ++j) {
            if (!fin && !wait) {
              const u32 f = inject ? 0u : (v[j] & kLbFlags);
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
            if (++spins > kSpinLimit || s_fail) {
              atomicExch(md.err, kDevErrTimeout);
              s_fail = 1;
              timed_out = true;
              break;
            }
            __nanosleep(32);
          }
        }
        // a tile whose wait ran out keeps its aggregate flag: successors still reach a correct prefix
        if (!timed_out) st_relaxed(me, kLbP | ((excl + c) & kLbVal));
      }
      sgbase[d] = (int)(sgdig[d] + excl) - sstart[d];
    }
    __syncthreads();
    if (s_fail) break;  // the prefixes are unknown: write nothing (the error word is set)
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
// 4. per-cell fusion, as a reduce-by-key over tiles of sorted points
//
// The sorted points are cut into tiles of kFuseTile; the points of one cell
// form one run of the sorted order, and a run may cross tile boundaries.
//
// k_fuse_tiles: one CTA per tile (persistent, tiles taken from a counter).
//   Every quantity summed per cell is a column of a stage in shared memory
//   with one row per point: the four height sums (after the outlier gate
//   against the pre-call state), then every source's channels, then, for a
//   source bound to a class-max layer, the point's largest channel value and
//   its channel. Up to kQ columns are staged at once (a round); a thread
//   walks one column over a fixed segment of the tile's points in point
//   order, and the pieces of a run that crosses segments are added in
//   segment order. A run whose points all lie in the tile is then fused
//   right there (Kalman height update, every layer's rule, class max,
//   flags); the layers' rows of the tile's cells were prefetched into L2 when
//   the tile started. A run that crosses the tile's first or last boundary
//   leaves its piece's sums in one of the tile's two slots.
// k_fuse_cross: one warp per run that crosses tile boundaries (the tile
//   where it begins): adds its pieces in tile order, then fuses it.
// The float32 summation order depends only on the sorted order, which is
// deterministic: results are identical from run to run.

constexpr int kFT = kFuseTile;  // threads of a fuse CTA = sorted points per tile
constexpr int kQ = 32;          // stage columns per round
constexpr int kQS = kQ + 1;     // row stride of the stage (odd: conflict-free columns)
constexpr int kSegMax = 32;     // segments of a tile per walk
constexpr int kStageU = 6;      // staging chunks in flight per thread
constexpr int kStageV = 5;      // float4 row loads in flight per thread (warp fuse kernel)
constexpr int kApplyU = 4;      // rule tasks in flight per thread
constexpr int kCrossU = 8;      // slot pieces in flight per lane (runs crossing tiles)
constexpr u32 kBitHead = 1u;    // slot bits: the run begins in the tile
constexpr u32 kBitEnd = 2u;     //            the run ends in the tile
constexpr u32 kBitUsed = 4u;    //            the slot holds a piece of this call
constexpr int kChArgV = -1;     // column of a source's arg-max value
constexpr int kChArgI = -2;     // column of a source's arg-max channel

// fuse scratch: two slots per tile, [0] the piece of a run carried in that
// ends in the tile, [1] the piece of a run that continues past the tile
__device__ __forceinline__ float* fz_slot(const MapDev& md, int acc, int tile, int k) {
  return md.partial + (int64_t)(2 * tile + k) * acc;  // 16-byte aligned (acc % 4 == 0)
}

// slot offset of global column gc (height sums first, then the header)
__device__ __forceinline__ int slot_off(int gc) { return gc < 4 ? gc : gc + (kSlotHdr - 4); }

// typed access to one stored value
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


struct SumSmem {
  u32 key[kFT + 2];  // key[i + 1]: point i; key[0]: the point before the tile; key[np + 1]: after it
  u32 idx[kFT];
  int pinf[kFT];     // point: run << 1 | 1 if it is the last point of its run in the tile
  int rstart[kFT + 1];
  u32 fl[kFT];       // per run: pre-call flags, height, variance (the gate's state)
  float h0[kFT], v0[kFT];
  float stage[kFT * kQS];
  float2 hp[kFT], tp[kFT];  // segment pieces of runs that cross segment boundaries
  int col_src[kQ];          // per column of the round: source (-1: height sums)
  int col_ch[kQ];           // channel, kChArgV / kChArgI, or height sum 0..3
  ChunkDesc ck[kQ];
  int n_ck;
  SrcDev src[kMaxSources];
  MapCall mc0;
  u32 rkey[kFT];     // per run: cell, pre-call accepted / rejected counts, 1 / points
  u32 na0[kFT], nr0[kFT];
  float rN[kFT];
  u32 cmw[kFT / 32][2];     // per warp: arg-max of its last run's points (value, channel)
  int cmr[kFT / 32];        //           and that run
  int qc0[kMaxSources], qch0[kMaxSources], qn[kMaxSources];  // per source: first column,
                                                             // first channel, channels in the round
  int pair_col[kMaxSources];  // arg-max value columns of the round
  int n_pair;
  LayerDev L[kMaxLayers];
  int rlay[kMaxSources][kMaxSrcLayers];  // per source: its layers other than class max
  int nrlay[kMaxSources];
  u32 wcnt[kFT / 32];
  u32 endbits[kFT / 32];  // bit i: point i is the last point of its run in the tile
  int fallback;           // an arg-max pair of the round needs channels of an earlier round
};

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

__device__ __forceinline__ float2 cm_comb(float2 a, float2 b) {  // larger value, smaller channel on ties
  return (b.x > a.x || (b.x == a.x && __float_as_int(b.y) < __float_as_int(a.y))) ? b : a;
}

// source and channel of global column gc >= 4
__device__ __forceinline__ void col_ident(const SrcDev* src, int n_src, int gc, int& q, int& ch) {
  const int o = slot_off(gc);
  q = 0;
  for (int k = 1; k < n_src; ++k)
    if (src[k].acc_off <= o) q = k;
  const int c = o - src[q].acc_off;
  ch = c < src[q].C ? c : (c == src[q].C ? kChArgV : kChArgI);
}

// end of the round that starts at column r0 (an arg-max pair never splits)
__device__ __forceinline__ int round_end(const SrcDev* src, int n_src, int r0, int G) {
  int re = min(r0 + kQ, G);
  if (re < G && re - 1 >= 4) {
    int q, ch;
    col_ident(src, n_src, re - 1, q, ch);
    if (ch == kChArgV) --re;
  }
  return re;
}

// Column table of the round [r0, r0 + nr), then (thread 0) its staging chunks.
__device__ __forceinline__ void build_columns(SumSmem& s, int n_src, int r0, int nr) {
  if (threadIdx.x < nr) {
    int q = -1, ch = r0 + threadIdx.x;
    if (r0 + threadIdx.x >= 4) col_ident(s.src, n_src, r0 + threadIdx.x, q, ch);
    s.col_src[threadIdx.x] = q;
    s.col_ch[threadIdx.x] = ch;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int n = 0;
    for (int c = 0; c < nr; ++c) {
      const int q = s.col_src[c], ch = s.col_ch[c];
      if (q < 0 || ch < 0) continue;
      const bool extend = n > 0 && s.ck[n - 1].n < 4 && (ch & 3) != 0 && s.col_src[c - 1] == q &&
                          s.col_ch[c - 1] == ch - 1 && s.ck[n - 1].col + s.ck[n - 1].n == c;
      if (extend) {
        ++s.ck[n - 1].n;
      } else {
        ChunkDesc& d = s.ck[n++];
        d.data = s.src[q].data;
        d.C = s.src[q].C;
        d.ch0 = ch;
        d.col = c;
        d.n = 1;
        d.dtype = s.src[q].dtype;
        d.vec = s.src[q].vec_ok;
        d.src = q;
        d.topk = s.src[q].topk;
      }
    }
    s.n_ck = n;
    for (int q = 0; q < n_src; ++q) {
      s.qn[q] = 0;
      for (int c = 0; c < nr; ++c)
        if (s.col_src[c] == q && s.col_ch[c] >= 0) {
          if (s.qn[q] == 0) {
            s.qc0[q] = c;
            s.qch0[q] = s.col_ch[c];
          }
          ++s.qn[q];
        }
    }
    s.fallback = 0;
    s.n_pair = 0;
    for (int c = 0; c < nr; ++c)
      if (s.col_ch[c] == kChArgV) {
        s.pair_col[s.n_pair++] = c;
        if (slot_off(r0) > s.src[s.col_src[c]].acc_off) s.fallback = 1;
      }
    // a source whose channels and arg-max pair are all in the round gets its
    // per-point arg-max while it is staged
    for (int k = 0; k < n; ++k) {
      const int q = s.ck[k].src;
      const int first = s.ck[k].col - s.ck[k].ch0;  // column of channel 0
      const int av = first + s.src[q].C;            // arg-max value column
      const bool ok = s.src[q].has_classmax && first >= 0 && av + 1 < nr;
      const bool last = k + 1 == n || s.ck[k + 1].src != q;
      s.ck[k].am = ok ? (av | (last ? (1 << 30) : 0)) : -1;
    }
  }
}

// four consecutive channels of a row (fewer at the end of the row)
template <bool TOPK>
__device__ __forceinline__ void ld_chunk(const ChunkDesc& d, int64_t row, float v[4]) {
  if (TOPK && d.topk) {  // expand the row's (class id, probability) pairs into the chunk's channels
    const float* __restrict__ r = (const float*)d.data + row * 2 * d.topk;
#pragma unroll
    for (int w = 0; w < 4; ++w) v[w] = 0.f;
    for (int j = 0; j < d.topk; ++j) {
      const float id = __ldg(r + 2 * j);
      if (id >= 0.f && id < (float)d.C && id == floorf(id)) {
        const int c = (int)id - d.ch0;
#pragma unroll
        for (int w = 0; w < 4; ++w)
          if (c == w && w < d.n) v[w] = __fadd_rn(v[w], __ldg(r + 2 * j + 1));
      }
    }
    return;
  }
  const int64_t off = row * d.C + d.ch0;
  if (d.n == 4 && d.vec && (off & 3) == 0) {
    if (d.dtype == MEM_F32) {
      const float4 q = __ldg((const float4*)((const float*)d.data + off));
      v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
      return;
    }
    if (d.dtype == MEM_BF16 || d.dtype == MEM_F16) {
      const uint2 q = __ldg((const uint2*)((const uint16_t*)d.data + off));
      if (d.dtype == MEM_BF16) {
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.x));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.y));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
      } else {
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&q.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
      }
      return;
    }
  }
#pragma unroll
  for (int w = 0; w < 4; ++w) v[w] = w < d.n ? ld_any(d.data, d.dtype, off + w) : 0.f;
}


// (i, j) enumeration of the i-major task list k = i * n + j, k = t, t + kFT, ...
// without divisions after the first
struct TaskWalk {
  int i, j, di, dj, n;
  __device__ __forceinline__ TaskWalk(int t, int n_) : n(n_) {
    i = t / n;
    j = t - i * n;
    di = kFT / n;
    dj = kFT - di * n;
  }
  __device__ __forceinline__ void next() {
    i += di;
    j += dj;
    if (j >= n) {
      j -= n;
      ++i;
    }
  }
};

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Kalman height update in information form (float32) + cumulative counts.
__device__ __forceinline__ void height_update(const MapDev& md, u32 g, u32& fl, float h0, float v0, float sw,
                                              float swz, u32 na, u32 nr, u32 na0, u32 nr0) {
  float h = h0, v = v0;
  if (na > 0) {
    if (fl & kFlagValid) {
      const float P = __frcp_rn(v0) + sw;
      h = (h0 * __frcp_rn(v0) + swz) * __frcp_rn(P);
      v = __frcp_rn(P);
    } else {
      h = swz * __frcp_rn(sw);
      v = __frcp_rn(sw);
      fl |= kFlagValid;
    }
  }
  if (nr > 0 && md.outlier_var != 0.f) v = fmaf(md.outlier_var, (float)nr, v);
  md.h[g] = h;
  md.var[g] = v;
  md.n_acc[g] = na0 + na;
  md.n_rej[g] = nr0 + nr;
}

// class max of a source into its class-max layers
__device__ __forceinline__ void write_classmax(const LayerDev* Ls, const SrcDev& src, u32 g, float best, int bid) {
  for (int b = 0; b < src.n_layers; ++b) {
    const LayerDev& L = Ls[src.layers[b]];
    if (L.rule == MEM_RULE_CLASSMAX) {
      float* d = (float*)L.data + (int64_t)g * 2;
      d[0] = (float)bid;
      d[1] = best;
    }
  }
}

// Gaussian variances of a source's layers (after every rule read them)
__device__ __forceinline__ void write_gauss_var(const LayerDev* Ls, const SrcDev& src, u32 g, u32 fl, float N,
                                                float rN) {
  for (int b = 0; b < src.n_layers; ++b) {
    const int l = src.layers[b];
    const LayerDev& L = Ls[l];
    if (L.rule != MEM_RULE_GAUSS) continue;
    const bool obs = fl & (2u << l);
    L.gvar[g] = rule_coef(L, N, rN, obs, obs ? L.gvar[g] : 0.f).var_new;
  }
}

// four consecutive stored values (16-byte aligned for F32, 8-byte for 16-bit types)
template <int DT>
__device__ __forceinline__ void ld4t(const void* base, int64_t off, float o[4]) {
  if (DT == MEM_F32) {
    const float4 q = *reinterpret_cast<const float4*>((const float*)base + off);
    o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
  } else {
    const uint2 q = *reinterpret_cast<const uint2*>((const uint16_t*)base + off);
    float2 a, b;
    if (DT == MEM_BF16) {
      a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.x));
      b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.y));
    } else {
      a = __half22float2(*reinterpret_cast<const __half2*>(&q.x));
      b = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
    }
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  }
}
template <int DT>
__device__ __forceinline__ void st4t(void* base, int64_t off, const float n[4]) {
  if (DT == MEM_F32) {
    *reinterpret_cast<float4*>((float*)base + off) = make_float4(n[0], n[1], n[2], n[3]);
  } else {
    uint2 q;
    if (DT == MEM_BF16) {
      __nv_bfloat162 a = __floats2bfloat162_rn(n[0], n[1]), b = __floats2bfloat162_rn(n[2], n[3]);
      q.x = *reinterpret_cast<u32*>(&a);
      q.y = *reinterpret_cast<u32*>(&b);
    } else {
      __half2 a = __floats2half2_rn(n[0], n[1]), b = __floats2half2_rn(n[2], n[3]);
      q.x = *reinterpret_cast<u32*>(&a);
      q.y = *reinterpret_cast<u32*>(&b);
    }
    *reinterpret_cast<uint2*>((uint16_t*)base + off) = q;
  }
}

// One rule layer over the runs fused in the tile: tasks (run, group of W
// channels of the round), kRuleU per thread in flight (old values and
// Gaussian prior variances first, then the new values). The layer's source
// channels ch0 .. ch0 + nch - 1 are the stage columns c0 ..; W = 4 needs
// ch0, nch and the layer's row length to be multiples of 4 (aligned rows).
template <int RULE, int DT, int W>
__device__ __forceinline__ void tile_rule_t(const SumSmem& s, const LayerDev& Ls, int l, int c0, int ch0, int nch,
                                            int r_lo, int r_hi) {
  constexpr int kRuleU = W == 4 ? 2 : 4;
  const LayerDev L = Ls;  // in registers: the stores below cannot alias it
  const int nq = nch / W;
  const int ntask = (r_hi - r_lo) * nq;
  TaskWalk tw(threadIdx.x, nq);
  for (int k0 = threadIdx.x; k0 < ntask; k0 += kRuleU * kFT) {
    float old[kRuleU][W], s02[kRuleU];
    TaskWalk tw0 = tw;
#pragma unroll
    for (int u = 0; u < kRuleU; ++u) {
      s02[u] = 0.f;
#pragma unroll
      for (int w = 0; w < W; ++w) old[u][w] = 0.f;
      if (k0 + u * kFT < ntask) {
        const int r = r_lo + tw.i;
        const u32 g = s.rkey[r];
        if (s.fl[r] & (2u << l)) {
          const int64_t off = (int64_t)g * L.S + ch0 + tw.j * W;
          if (RULE != MEM_RULE_LATEST) {
            if (W == 4) ld4t<DT>(L.data, off, old[u]);
            else old[u][0] = ld1t<DT>(L.data, off);
          }
          if (RULE == MEM_RULE_GAUSS) s02[u] = L.gvar[g];
        }
      }
      tw.next();
    }
#pragma unroll
    for (int u = 0; u < kRuleU; ++u) {
      if (k0 + u * kFT < ntask) {
        const int r = r_lo + tw0.i;
        const RuleCoef co = rule_coef(L, (float)(s.rstart[r + 1] - s.rstart[r]), s.rN[r],
                                      (s.fl[r] & (2u << l)) != 0, s02[u]);
        const float* S = s.stage + s.rstart[r] * kQS + c0 + tw0.j * W;
        float nv[W];
#pragma unroll
        for (int w = 0; w < W; ++w) nv[w] = rule_value_t<RULE>(L, old[u][w], S[w], co);
        const int64_t off = (int64_t)s.rkey[r] * L.S + ch0 + tw0.j * W;
        if (W == 4) st4t<DT>(L.data, off, nv);
        else st1t<DT>(L.data, off, nv[0]);
      }
      tw0.next();
    }
  }
}

__device__ __forceinline__ void tile_rule(const SumSmem& s, const LayerDev& L, int l, int c0, int ch0, int nch,
                                          int r_lo, int r_hi) {
  const bool v4 = (L.S & 3) == 0 && (ch0 & 3) == 0 && (nch & 3) == 0;
#define MEM_TR(R, D)                                                                  \
  case R * 4 + D:                                                                     \
    if (v4) tile_rule_t<R, D, 4>(s, L, l, c0, ch0, nch, r_lo, r_hi);                  \
    else tile_rule_t<R, D, 1>(s, L, l, c0, ch0, nch, r_lo, r_hi);                     \
    break;
  switch (L.rule * 4 + L.dtype) {
    MEM_TR(MEM_RULE_LATEST, MEM_F32) MEM_TR(MEM_RULE_LATEST, MEM_BF16) MEM_TR(MEM_RULE_LATEST, MEM_F16)
    MEM_TR(MEM_RULE_EXPAVG, MEM_F32) MEM_TR(MEM_RULE_EXPAVG, MEM_BF16) MEM_TR(MEM_RULE_EXPAVG, MEM_F16)
    MEM_TR(MEM_RULE_GAUSS, MEM_F32) MEM_TR(MEM_RULE_GAUSS, MEM_BF16) MEM_TR(MEM_RULE_GAUSS, MEM_F16)
    MEM_TR(MEM_RULE_DIRICHLET, MEM_F32)
    default: break;
  }
#undef MEM_TR
}

// TOPK: some source of the call has top-k rows; RAY: the map runs the ray-cast
// clean-up (both known on the host, so the common call carries neither branch)
template <bool TOPK, bool RAY>
__global__ void __launch_bounds__(kFT, 7) k_fuse_tiles(MapDev md, const PointJob* __restrict__ job,
                                                       int sorted1) {
  extern __shared__ __align__(16) unsigned char fz_raw[];
  SumSmem& s = *reinterpret_cast<SumSmem*>(fz_raw);
  if (*(volatile int*)md.err) return;  // a device error is pending: the point path does nothing
  const u32* __restrict__ sk = sorted1 ? md.keys1 : md.keys0;
  const u32* __restrict__ sv = sorted1 ? md.vals1 : md.vals0;
  const int64_t n_kept = *(volatile u32*)&md.counters[6];
  const int n_tiles = (int)((n_kept + kFT - 1) / kFT);
  const int n_src = job->n_src;
  const int acc = job->acc;
  const FuseTables* __restrict__ ft = &job->ft;
  const int G = ft->ncol;  // columns of the call
  const bool one_round = ft->one_round;
  const bool any_gauss = ft->any_gauss;  // Gaussian variances are written after every rule read them
  const float* __restrict__ xyz = job->xyz;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const u64 call_hi = RAY ? (u64)job->call_id << 32 : 0ull;
  // the call's tables (built on the host) into shared memory
  if (t < n_src) s.src[t] = job->src[t];
  if (t < md.n_layers) s.L[t] = md.L[t];
  if (t == 0) s.mc0 = job->maps[0];
  if (t < kMaxSources) {
    s.nrlay[t] = ft->nrlay[t];
    for (int b = 0; b < kMaxSrcLayers; ++b) s.rlay[t][b] = ft->rlay[t][b];
    s.qc0[t] = ft->qc0[t];
    s.qch0[t] = ft->qch0[t];
    s.qn[t] = ft->qn[t];
    s.pair_col[t] = ft->pair_col[t];
  }
  if (one_round) {
    for (int i = t; i < kQ; i += kFT) {
      s.col_src[i] = ft->col_src[i];
      s.col_ch[i] = ft->col_ch[i];
      s.ck[i] = ft->ck[i];
    }
    if (t == 0) {
      s.n_ck = ft->n_ck;
      s.n_pair = ft->n_pair;
      s.fallback = 0;
    }
  }
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    __syncthreads();  // the previous tile is done with the shared arrays
    const int64_t p0 = (int64_t)tile * kFT;
    const int np = (int)min((int64_t)kFT, n_kept - p0);
    // A. keys, point indices, runs
    if (t < np) {
      s.key[t + 1] = sk[p0 + t];
      s.idx[t] = sv[p0 + t];
    }
    if (t == 0) s.key[0] = p0 > 0 ? sk[p0 - 1] : 0xfffffffeu;
    if (t == 32) s.key[np + 1] = (p0 + np < n_kept) ? sk[p0 + np] : 0xfffffffeu;
    __syncthreads();
    const bool hd = t < np && (t == 0 || s.key[t] != s.key[t + 1]);
    const bool ed = t < np && (t == np - 1 || s.key[t + 1] != s.key[t + 2]);
    const u32 bal = __ballot_sync(0xffffffffu, hd);
    const u32 ebal = __ballot_sync(0xffffffffu, ed);
    if (lane == 0) {
      s.wcnt[warp] = __popc(bal);
      s.endbits[warp] = ebal;
    }
    __syncthreads();
    int nruns = 0, rbase = 0;
#pragma unroll
    for (int w = 0; w < kFT / 32; ++w) {
      const int cw = (int)s.wcnt[w];
      rbase += w < warp ? cw : 0;
      nruns += cw;
    }
    const int myrun = rbase + __popc(bal & ((2u << lane) - 1u)) - 1;
    if (t < np) s.pinf[t] = (myrun << 1) | (ed ? 1 : 0);
    if (hd) {
      s.rstart[myrun] = t;
      s.rkey[myrun] = s.key[t + 1];
    }
    if (t == 0) s.rstart[nruns] = np;
    const int rl = nruns - 1;
    const bool gh0 = s.key[0] != s.key[1];        // run 0 begins in this tile
    const bool geL = s.key[np] != s.key[np + 1];  // the last run ends in this tile
    const int r_lo = gh0 ? 0 : 1, r_hi = geL ? nruns : rl;  // runs fused here
    // pieces carried to slots: a first run begun earlier that ends here ([0]);
    // a last run that continues past the tile ([1], also when it is the only run)
    float* cin = (!gh0 && (nruns > 1 || geL)) ? fz_slot(md, acc, tile, 0) : nullptr;
    float* cout = !geL ? fz_slot(md, acc, tile, 1) : nullptr;
    __syncthreads();
    // B. pre-call state of every run's cell; slot headers of the carried
    //    pieces; the rule layers' rows of the cells into L2; coordinates
    if (t < nruns) {
      const u32 g = s.rkey[t];
      const u32 fl = md.flags[g];
      const float h0 = md.h[g], v0 = md.var[g];
      const u32 na = md.n_acc[g], nr = md.n_rej[g];
      s.fl[t] = fl;
      s.h0[t] = h0;
      s.v0[t] = v0;
      s.na0[t] = na;
      s.nr0[t] = nr;
      s.rN[t] = __frcp_rn((float)(s.rstart[t + 1] - s.rstart[t]));
      float* hdr = (t == 0 && cin) ? cin : (t == rl && cout) ? cout : nullptr;
      if (hdr) {
        const u32 bits = kBitUsed | (t > 0 || gh0 ? kBitHead : 0u) | (t < rl || geL ? kBitEnd : 0u);
        hdr[kSlotKey] = __uint_as_float(g);
        hdr[kSlotN] = __uint_as_float((u32)(s.rstart[t + 1] - s.rstart[t]));
        hdr[kSlotBits] = __uint_as_float(bits);
        hdr[kSlotFl] = __uint_as_float(fl);
        hdr[kSlotH0] = h0;
        hdr[kSlotV0] = v0;
        hdr[kSlotNacc] = __uint_as_float(na);
        hdr[kSlotNrej] = __uint_as_float(nr);
      }
      for (int q = 0; q < n_src; ++q)
        for (int j = 0; j < s.nrlay[q]; ++j) {
          const LayerDev& L = s.L[s.rlay[q][j]];
          if (L.rule == MEM_RULE_LATEST) continue;
          const int bytes = L.S * (L.dtype == MEM_F32 ? 4 : 2);
          const char* row = (const char*)L.data + (int64_t)g * bytes;
          for (int o = 0; o < bytes; o += 128) prefetch_l2(row + o);
          prefetch_l2(row + bytes - 1);
        }
    }
    if (t == 0 && !cin) fz_slot(md, acc, tile, 0)[kSlotBits] = 0.f;  // unused this call
    if (t == 0 && !cout) fz_slot(md, acc, tile, 1)[kSlotBits] = 0.f;
    float xs = 0.f, ys = 0.f, zs = 0.f;
    if (t < np) {
      const int64_t id = s.idx[t];
      xs = __ldg(xyz + 3 * id);
      ys = __ldg(xyz + 3 * id + 1);
      zs = __ldg(xyz + 3 * id + 2);
    }
    // C. rounds of at most kQ columns
    for (int r0 = 0; r0 < G;) {
      const int re = one_round ? G : round_end(s.src, n_src, r0, G);
      const int nr = re - r0;
      if (!one_round) {
        __syncthreads();  // the previous round is done with the column tables
        build_columns(s, n_src, r0, nr);
        __syncthreads();
      }
      // stage the source channels of the round: thread = point, kStageU
      // chunks in flight before their stores; a source bound to a class-max
      // layer gets the point's arg-max on the way
      if (t < np) {
        const int nck = s.n_ck;
        const int64_t row_i = s.idx[t];
        float* srow = s.stage + t * kQS;
        float pb = -INFINITY;
        int pi = 0x7fffffff;
        for (int j0 = 0; j0 < nck; j0 += kStageU) {
          float v[kStageU][4];
#pragma unroll
          for (int u = 0; u < kStageU; ++u)
            if (j0 + u < nck) ld_chunk<TOPK>(s.ck[j0 + u], row_i, v[u]);
#pragma unroll
          for (int u = 0; u < kStageU; ++u) {
            if (j0 + u < nck) {
              const ChunkDesc& d = s.ck[j0 + u];
              const int am = d.am;
#pragma unroll
              for (int w = 0; w < 4; ++w)
                if (w < d.n) {
                  srow[d.col + w] = v[u][w];
                  if (am >= 0 && v[u][w] > pb) {
                    pb = v[u][w];
                    pi = d.ch0 + w;
                  }
                }
              if (am >= 0 && (am >> 30)) {
                srow[am & 0xffff] = pb;
                srow[(am & 0xffff) + 1] = __int_as_float(pi);
                pb = -INFINITY;
                pi = 0x7fffffff;
              }
            }
          }
        }
      }
      __syncthreads();
      u64 zk = 0;  // ray-cast clean-up: (call id, lowest z) key of an accepted point
      if (r0 == 0 && t < np) {
        // outlier gate against the pre-call state: height sums of the point
        const int r = s.pinf[t] >> 1;
        const MapCall* mc = md.n_maps > 1 ? job->maps + s.key[t + 1] / md.W2 : &s.mc0;
        float z, vm;
        eval_zvm(md, *mc, xs, ys, zs, z, vm);
        const bool rej = (s.fl[r] & kFlagValid) && gate_reject(z, s.h0[r], s.v0[r], vm, md.lam2);
        const float w = __frcp_rn(vm);
        float* row = s.stage + t * kQS;
        row[0] = rej ? 0.f : w;
        row[1] = rej ? 0.f : z * w;
        row[2] = rej ? 0.f : 1.f;
        row[3] = rej ? 1.f : 0.f;
        if (RAY && !rej) zk = call_hi | (u64)(~ordered_bits(__float_as_uint(z)));
      }
      if (RAY && r0 == 0) {
        // the lowest accepted z of every cell: a segmented max of the keys over each warp's
        // points (runs are contiguous), one atomic per run piece of the warp
        const int run = t < np ? s.pinf[t] >> 1 : -1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const u64 ok = __shfl_up_sync(0xffffffffu, zk, o);
          const int orun = __shfl_up_sync(0xffffffffu, run, o);
          if (lane >= o && orun == run && ok > zk) zk = ok;
        }
        const int nrun = __shfl_down_sync(0xffffffffu, run, 1);
        if (t < np && zk != 0 && (lane == 31 || t == np - 1 || nrun != run))
          atomicMax((unsigned long long*)(md.zacc + s.key[t + 1]), (unsigned long long)zk);
      }
      // per-point arg-max of a source whose channels began in an earlier round
      for (int c = 0; c < nr && s.fallback; ++c) {
        if (s.col_ch[c] != kChArgV) continue;  // uniform
        const SrcDev& src = s.src[s.col_src[c]];
        if (t < np && slot_off(r0) > src.acc_off) {
          float pb = -INFINITY;
          int pi = 0x7fffffff;
          for (int k = 0; k < src.C; ++k) {
            const float v = src_val(src, (int64_t)s.idx[t], k);
            if (v > pb) {
              pb = v;
              pi = k;
            }
          }
          s.stage[t * kQS + c] = pb;
          s.stage[t * kQS + c + 1] = __int_as_float(pi);
        }
      }
      __syncthreads();
      // class max per run of every arg-max pair of the round: segmented max of
      // (value, channel) over each warp's points (runs are contiguous), then
      // the run's last point adds the tails of earlier warps the run covers;
      // the run's result goes to its first row
      for (int pc = 0; pc < s.n_pair; ++pc) {
        const int c = s.pair_col[pc];
        const int run = t < np ? s.pinf[t] >> 1 : -1 - warp;
        float2 m = t < np ? make_float2(s.stage[t * kQS + c], s.stage[t * kQS + c + 1])
                          : make_float2(-INFINITY, __int_as_float(0x7fffffff));
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const float ov = __shfl_up_sync(0xffffffffu, m.x, o);
          const float oi = __shfl_up_sync(0xffffffffu, m.y, o);
          const int orun = __shfl_up_sync(0xffffffffu, run, o);
          if (lane >= o && orun == run) m = cm_comb(make_float2(ov, oi), m);
        }
        if (lane == 31) {
          s.cmw[warp][0] = __float_as_uint(m.x);
          s.cmw[warp][1] = __float_as_uint(m.y);
          s.cmr[warp] = run;
        }
        __syncthreads();
        if (t < np && (s.pinf[t] & 1)) {
          for (int w = warp - 1; w >= 0 && s.cmr[w] == run; --w)
            m = cm_comb(make_float2(__uint_as_float(s.cmw[w][0]), __uint_as_float(s.cmw[w][1])), m);
          float* row = s.stage + s.rstart[run] * kQS + c;
          row[0] = m.x;
          row[1] = m.y;
        }
        __syncthreads();
      }
      // walk: thread (segment, column) over the segment's points in order
      // (height sums and source channels; the arg-max pairs are done)
      {
        const int nseg = max(1, min(min(kFT / nr, kSegMax), np));
        const int len = (np + nseg - 1) / nseg;
        const int sg = t / nr, c = t - sg * nr;
        const int i0 = sg * len, i1 = min(i0 + len, np);
        const bool on = sg < nseg && i0 < i1 && (s.col_src[c] < 0 || s.col_ch[c] >= 0);
        const bool cont0 = on && i0 > 0 && !((s.endbits[(i0 - 1) >> 5] >> ((i0 - 1) & 31)) & 1u);
        if (on) {
          // run ends of the segment as a bit mask; values eight at a time
          const int n = i1 - i0;
          const int wb = i0 >> 5, ob = i0 & 31;
          u64 e64 = s.endbits[wb];
          if (wb + 1 < kFT / 32) e64 |= (u64)s.endbits[wb + 1] << 32;
          const u32 em = (u32)(e64 >> ob);
          bool cont = cont0;
          float a = 0.f;
          int start = i0;  // first point of the open run in this segment
          for (int j0 = 0; j0 < n; j0 += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = j0 + u < n ? s.stage[(i0 + j0 + u) * kQS + c] : 0.f;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              if (j0 + u < n) {
                a += v[u];
                if ((em >> (j0 + u)) & 1u) {
                  if (cont) s.hp[sg * nr + c].x = a;
                  else s.stage[start * kQS + c] = a;
                  cont = false;
                  a = 0.f;
                  start = i0 + j0 + u + 1;
                }
              }
            }
          }
          if (!((em >> (n - 1)) & 1u)) s.tp[sg * nr + c].x = a;
        }
        __syncthreads();
        // runs that cross segments: finished by the segment holding their last point
        if (cont0) {
          const int r = s.pinf[i0] >> 1;
          if (s.rstart[r + 1] <= i1) {
            const int s0 = s.rstart[r] / len;
            float a = s.tp[s0 * nr + c].x;
            for (int k = s0 + 1; k < sg; ++k) a += s.tp[k * nr + c].x;
            s.stage[s.rstart[r] * kQS + c] = a + s.hp[sg * nr + c].x;
          }
        }
        __syncthreads();
      }
      // D. sums of the carried pieces to their slots (nr <= 32: warp 0)
      if (t < nr) {
        if (cin) cin[slot_off(r0 + t)] = s.stage[s.rstart[0] * kQS + t];
        if (cout) cout[slot_off(r0 + t)] = s.stage[s.rstart[rl] * kQS + t];
      }
      // E. rules of the runs fused here, layer by layer
      for (int q = 0; q < n_src; ++q)
        if (s.qn[q] > 0)
          for (int j = 0; j < s.nrlay[q]; ++j) {
            const int l = s.rlay[q][j];
            tile_rule(s, s.L[l], l, s.qc0[q], s.qch0[q], s.qn[q], r_lo, r_hi);
          }
      // F. per run fused here: height update (first round), class max of the
      //    arg-max pairs of the round (the valid bit joins the flags kept in
      //    shared memory; rules only read the observed bits)
      if (t >= r_lo && t < r_hi) {
        const float* row = s.stage + s.rstart[t] * kQS;
        const u32 g = s.rkey[t];
        if (r0 == 0) {
          u32 fl = s.fl[t];
          height_update(md, g, fl, s.h0[t], s.v0[t], row[0], row[1], (u32)row[2], (u32)row[3], s.na0[t], s.nr0[t]);
          s.fl[t] = fl;
        }
        for (int q = 0; q < n_src; ++q) {
          const int av = s.src[q].acc_off - (kSlotHdr - 4) + s.src[q].C - r0;  // arg-max value column in the round
          if (s.src[q].has_classmax && av >= 0 && av + 1 < nr) {
            const float best = row[av];
            write_classmax(s.L, s.src[q], g, best, best == -INFINITY ? -1 : __float_as_int(row[av + 1]));
          }
        }
      }
      r0 = re;
      __syncthreads();  // the next round overwrites the stage
    }
    // G. Gaussian variances and flags of the runs fused here
    if (t >= r_lo && t < r_hi) {
      const u32 g = s.rkey[t];
      u32 fl = s.fl[t];
      const float N = (float)(s.rstart[t + 1] - s.rstart[t]);
      for (int q = 0; q < n_src; ++q) {
        if (any_gauss) write_gauss_var(s.L, s.src[q], g, fl, N, __frcp_rn(N));
        for (int b = 0; b < s.src[q].n_layers; ++b) fl |= 2u << s.src[q].layers[b];
      }
      md.flags[g] = fl;
    }
    if (t == 0) {
      const u32 heads = (u32)(nruns - (gh0 ? 0 : 1));
      if (heads) atomicAdd(&md.counters[5], heads);
    }
  }
}

// The fusion of one run that crosses tile boundaries, by one warp: it begins in
// tile h (header and first piece in that tile's slot [1]) and ends in tile
// `last` (its piece in slot [0]); the tiles between are covered entirely (their
// slots [1]). Lanes take columns: each adds its column over the pieces in tile
// order and loads the old values of the column's layers together, then stores
// the new values; lane 0 updates the height and flags.
__device__ __forceinline__ void cross_run(const MapDev& md, const LayerDev* sL, const SrcDev* ssrc,
                                          const int (*srlay)[kMaxSrcLayers], const int* snrlay, int n_src,
                                          int G, int acc, int h, int last, int lane) {
  const float* head = fz_slot(md, acc, h, 1);
  const u32 hw = lane < kSlotHdr ? __float_as_uint(__ldcg(head + lane)) : 0u;
  const int np = last - h + 1;      // pieces
  const u32 g = __shfl_sync(0xffffffffu, hw, kSlotKey);
  const u32 fl0 = __shfl_sync(0xffffffffu, hw, kSlotFl);
  // points of the run over its pieces
  u32 n = 0;
  for (int p = lane; p < np; p += 32)
    n += __float_as_uint(__ldcg(fz_slot(md, acc, h + p, h + p == last ? 0 : 1) + kSlotN));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  const float N = (float)n, rN = __frcp_rn(N);
  float hsum[4] = {0.f, 0.f, 0.f, 0.f};
  for (int c0 = 0; c0 < G; c0 += 32) {
    const int gc = c0 + lane;
    int q = -1, ch = gc;
    if (gc < G && gc >= 4) col_ident(ssrc, n_src, gc, q, ch);
    float S = 0.f;
    float2 m = make_float2(-INFINITY, __int_as_float(0x7fffffff));
    float old[kApplyU], s02[kApplyU];
#pragma unroll
    for (int j = 0; j < kApplyU; ++j) old[j] = s02[j] = 0.f;
    if (gc < G) {
      // the column's old layer values first (independent of the sums), then the pieces,
      // kCrossU loads in flight, added in tile order
      if (q >= 0 && ch >= 0) {
#pragma unroll
        for (int j = 0; j < kApplyU; ++j) {
          if (j < snrlay[q]) {
            const int l = srlay[q][j];
            const LayerDev& L = sL[l];
            if (fl0 & (2u << l)) {
              if (L.rule != MEM_RULE_LATEST) old[j] = ld_layer(L, (int64_t)g * L.S + ch);
              if (L.rule == MEM_RULE_GAUSS) s02[j] = L.gvar[g];
            }
          }
        }
      }
      for (int p0 = 0; p0 < np; p0 += kCrossU) {
        float v[kCrossU], w[kCrossU];
#pragma unroll
        for (int u = 0; u < kCrossU; ++u) {
          v[u] = 0.f;
          w[u] = __int_as_float(0x7fffffff);
          if (p0 + u < np) {
            const float* sl = fz_slot(md, acc, h + p0 + u, h + p0 + u == last ? 0 : 1) + slot_off(gc);
            v[u] = __ldcg(sl);
            if (ch == kChArgV) w[u] = __ldcg(sl + 1);
          }
        }
#pragma unroll
        for (int u = 0; u < kCrossU; ++u) {
          if (p0 + u < np) {
            S += v[u];
            if (ch == kChArgV) m = cm_comb(m, make_float2(v[u], w[u]));
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float hv = __shfl_sync(0xffffffffu, S, k);
      if (c0 == 0) hsum[k] = hv;
    }
    if (q >= 0 && ch >= 0) {
#pragma unroll
      for (int j = 0; j < kApplyU; ++j) {
        if (j < snrlay[q]) {
          const int l = srlay[q][j];
          const LayerDev& L = sL[l];
          const bool obs = fl0 & (2u << l);
          st_layer(L, (int64_t)g * L.S + ch, rule_value(L, old[j], S, rule_coef(L, N, rN, obs, s02[j])));
        }
      }
      for (int j = kApplyU; j < snrlay[q]; ++j) {  // more layers than kept in flight
        const int l = srlay[q][j];
        const LayerDev& L = sL[l];
        const bool obs = fl0 & (2u << l);
        const float s2 = (L.rule == MEM_RULE_GAUSS && obs) ? L.gvar[g] : 0.f;
        apply_rule(L, (int64_t)g * L.S + ch, S, rule_coef(L, N, rN, obs, s2));
      }
    }
    if (q >= 0 && ch == kChArgV) write_classmax(sL, ssrc[q], g, m.x, m.x == -INFINITY ? -1 : __float_as_int(m.y));
  }
  const float h0 = __uint_as_float(__shfl_sync(0xffffffffu, hw, kSlotH0));
  const float v0 = __uint_as_float(__shfl_sync(0xffffffffu, hw, kSlotV0));
  const u32 nacc0 = __shfl_sync(0xffffffffu, hw, kSlotNacc), nrej0 = __shfl_sync(0xffffffffu, hw, kSlotNrej);
  __syncwarp();  // every rule read its Gaussian prior variance
  if (lane == 0) {
    u32 fl = fl0;
    height_update(md, g, fl, h0, v0, hsum[0], hsum[1], (u32)hsum[2], (u32)hsum[3], nacc0, nrej0);
    for (int q = 0; q < n_src; ++q) {
      write_gauss_var(sL, ssrc[q], g, fl0, N, rN);
      for (int b = 0; b < ssrc[q].n_layers; ++b) fl |= 2u << ssrc[q].layers[b];
    }
    md.flags[g] = fl;
  }
}

// ---------------------------------------------------------------------------
// 4b. the same fusion for calls whose columns fit one round (at most kQ), with
//     the per-cell sums taken in registers. A warp holds 32 consecutive points
//     of the tile, one per lane: each lane stages its point's channels in its
//     own shared-memory row and adds the height sums after the gate; then every
//     column is summed over the pieces of runs in the warp by a segmented
//     inclusive scan of shuffles (the piece's sum lands on its last lane; an
//     arg-max pair takes the segmented maximum instead). The lane where a run
//     ends adds the pieces of the earlier warps of the tile that the run covers
//     (in warp order) and fuses the run itself: every layer's rule over its
//     cell's rows, class max, Kalman height update, Gaussian variances, flags.
//     Runs that cross the tile's boundaries leave their sums and header in the
//     tile's two slots exactly as k_fuse_tiles does, for k_fuse_cross.

struct WarpSmem {
  float stage[kFT * kQS];  // one row per point of the tile
  SrcDev src[kMaxSources];
  LayerDev L[kMaxLayers];
  ChunkDesc ck[kQ];
  MapCall mc0;
  int rlay[kMaxSources][kMaxSrcLayers];  // per source: its layers other than class max
  int nrlay[kMaxSources];
  int qc0[kMaxSources], qch0[kMaxSources], qn[kMaxSources];
  int pair_col[kMaxSources];
  int n_ck, n_pair;
  u32 whd[kFT / 32];  // per warp: the lanes where a run begins
};

// One rule layer over the channels of a run, by the lane that fuses it: old
// values (and the Gaussian prior variance) first, kRuleU vectors in flight.
template <int RULE, int DT, int W>
__device__ __forceinline__ void lane_rule_t(const LayerDev& L, int l, const float* S, int ch0, int nch, u32 g,
                                            u32 fl, float N, float rN) {
  constexpr int kRuleU = 5;
  const bool obs = (fl & (2u << l)) != 0;
  const float s02 = (RULE == MEM_RULE_GAUSS && obs) ? L.gvar[g] : 0.f;
  const RuleCoef co = rule_coef(L, N, rN, obs, s02);
  const int64_t base = (int64_t)g * L.S + ch0;
  for (int k0 = 0; k0 < nch; k0 += kRuleU * W) {
    float old[kRuleU][W];
#pragma unroll
    for (int u = 0; u < kRuleU; ++u) {
      const int k = k0 + u * W;
#pragma unroll
      for (int w = 0; w < W; ++w) old[u][w] = 0.f;
      if (RULE != MEM_RULE_LATEST && obs && k < nch) {
        if (W == 4) ld4t<DT>(L.data, base + k, old[u]);
        else old[u][0] = ld1t<DT>(L.data, base + k);
      }
    }
#pragma unroll
    for (int u = 0; u < kRuleU; ++u) {
      const int k = k0 + u * W;
      if (k < nch) {
        float nv[W];
#pragma unroll
        for (int w = 0; w < W; ++w) nv[w] = rule_value_t<RULE>(L, old[u][w], S[k + w], co);
        if (W == 4) st4t<DT>(L.data, base + k, nv);
        else st1t<DT>(L.data, base + k, nv[0]);
      }
    }
  }
}

__device__ __forceinline__ void lane_rule(const LayerDev& L, int l, const float* S, int ch0, int nch, u32 g, u32 fl,
                                          float N, float rN) {
  const bool v4 = (L.S & 3) == 0 && (ch0 & 3) == 0 && (nch & 3) == 0;
#define MEM_LR(R, D)                                                \
  case R * 4 + D:                                                   \
    if (v4) lane_rule_t<R, D, 4>(L, l, S, ch0, nch, g, fl, N, rN);  \
    else lane_rule_t<R, D, 1>(L, l, S, ch0, nch, g, fl, N, rN);     \
    break;
  switch (L.rule * 4 + L.dtype) {
    MEM_LR(MEM_RULE_LATEST, MEM_F32) MEM_LR(MEM_RULE_LATEST, MEM_BF16) MEM_LR(MEM_RULE_LATEST, MEM_F16)
    MEM_LR(MEM_RULE_EXPAVG, MEM_F32) MEM_LR(MEM_RULE_EXPAVG, MEM_BF16) MEM_LR(MEM_RULE_EXPAVG, MEM_F16)
    MEM_LR(MEM_RULE_GAUSS, MEM_F32) MEM_LR(MEM_RULE_GAUSS, MEM_BF16) MEM_LR(MEM_RULE_GAUSS, MEM_F16)
    MEM_LR(MEM_RULE_DIRICHLET, MEM_F32)
    default: break;
  }
#undef MEM_LR
}

// four (one) source values of any storage type, from their bits
__device__ __forceinline__ float4 ld4_any(const void* base, int dtype, int64_t off) {
  if (dtype == MEM_F32) return __ldg(reinterpret_cast<const float4*>((const float*)base + off));
  if (dtype == MEM_U8) {
    const u32 b = __ldg(reinterpret_cast<const u32*>((const unsigned char*)base + off));
    return make_float4((float)(b & 0xffu), (float)((b >> 8) & 0xffu), (float)((b >> 16) & 0xffu), (float)(b >> 24));
  }
  const uint2 q = __ldg(reinterpret_cast<const uint2*>((const uint16_t*)base + off));
  if (dtype == MEM_BF16)
    return make_float4(__uint_as_float(q.x << 16), __uint_as_float(q.x & 0xffff0000u), __uint_as_float(q.y << 16),
                       __uint_as_float(q.y & 0xffff0000u));
  return make_float4(__half2float(__ushort_as_half((unsigned short)(q.x & 0xffffu))),
                     __half2float(__ushort_as_half((unsigned short)(q.x >> 16))),
                     __half2float(__ushort_as_half((unsigned short)(q.y & 0xffffu))),
                     __half2float(__ushort_as_half((unsigned short)(q.y >> 16))));
}
__device__ __forceinline__ float ld1_any(const void* base, int dtype, int64_t off) {
  if (dtype == MEM_F32) return __ldg((const float*)base + off);
  if (dtype == MEM_U8) return (float)__ldg((const unsigned char*)base + off);
  const unsigned short b = __ldg((const unsigned short*)base + off);
  return dtype == MEM_BF16 ? __uint_as_float((u32)b << 16) : __half2float(__ushort_as_half(b));
}

// One source's channels of a point into its stage row (columns col0 .. col0 +
// C - 1), then, for a source bound to a class-max layer, the point's largest
// channel value and its channel (the smaller channel on ties) in the next two
// columns. Rows of C % 4 == 0 channels of 16-byte aligned data are read four
// channels at a time.
__device__ __forceinline__ void stage_src(float* srow, const void* data, int dtype, int64_t id, int C, int col0,
                                          bool vec, bool cm) {
  float pb = -INFINITY;
  int pi = 0x7fffffff;
  const int64_t base = id * C;
  if (vec && (C & 3) == 0) {
    for (int k0 = 0; k0 < C; k0 += 4 * kStageV) {
      float4 v[kStageV];
#pragma unroll
      for (int u = 0; u < kStageV; ++u)
        if (k0 + 4 * u < C) v[u] = ld4_any(data, dtype, base + k0 + 4 * u);
#pragma unroll
      for (int u = 0; u < kStageV; ++u)
        if (k0 + 4 * u < C)
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            const float e = w == 0 ? v[u].x : w == 1 ? v[u].y : w == 2 ? v[u].z : v[u].w;
            srow[col0 + k0 + 4 * u + w] = e;
            if (cm && e > pb) {
              pb = e;
              pi = k0 + 4 * u + w;
            }
          }
    }
  } else {
    for (int k0 = 0; k0 < C; k0 += 8) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (k0 + u < C) v[u] = ld1_any(data, dtype, base + k0 + u);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (k0 + u < C) {
          srow[col0 + k0 + u] = v[u];
          if (cm && v[u] > pb) {
            pb = v[u];
            pi = k0 + u;
          }
        }
    }
  }
  if (cm) {
    srow[col0 + C] = pb;
    srow[col0 + C + 1] = __int_as_float(pi);
  }
}

// The chunks of the top-k sources (rows of (class id, probability) pairs
// expanded into channels), with their arg-max.
__device__ __noinline__ void stage_topk_chunks(const ChunkDesc* ck, int nck, const SrcDev* src, float* srow,
                                               int64_t id) {
  float pb = -INFINITY;
  int pi = 0x7fffffff;
  for (int k = 0; k < nck; ++k) {
    const ChunkDesc& d = ck[k];
    if (!src[d.src].topk) continue;
    float v[4];
    ld_chunk<true>(d, id, v);
    for (int w = 0; w < d.n; ++w) {
      srow[d.col + w] = v[w];
      if (d.am >= 0 && v[w] > pb) {
        pb = v[w];
        pi = d.ch0 + w;
      }
    }
    if (d.am >= 0 && (d.am >> 30)) {
      srow[d.am & 0xffff] = pb;
      srow[(d.am & 0xffff) + 1] = __int_as_float(pi);
      pb = -INFINITY;
      pi = 0x7fffffff;
    }
  }
}

template <bool TOPK, bool RAY>
__global__ void __launch_bounds__(kFT, 6) k_fuse_warps(MapDev md, const PointJob* __restrict__ job, int sorted1) {
  extern __shared__ __align__(16) unsigned char fw_raw[];
  WarpSmem& s = *reinterpret_cast<WarpSmem*>(fw_raw);
  if (*(volatile int*)md.err) return;  // a device error is pending: the point path does nothing
  const u32* __restrict__ sk = sorted1 ? md.keys1 : md.keys0;
  const u32* __restrict__ sv = sorted1 ? md.vals1 : md.vals0;
  const int64_t n_kept = *(volatile u32*)&md.counters[6];
  const int n_tiles = (int)((n_kept + kFT - 1) / kFT);
  const int n_src = job->n_src;
  const int acc = job->acc;
  const FuseTables* __restrict__ ft = &job->ft;
  const int G = ft->ncol;  // columns of the call (at most kQ)
  const bool any_gauss = ft->any_gauss;
  const float* __restrict__ xyz = job->xyz;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const u64 call_hi = RAY ? (u64)job->call_id << 32 : 0ull;
  // the call's tables (built on the host) into shared memory
  if (t < n_src) s.src[t] = job->src[t];
  if (t < md.n_layers) s.L[t] = md.L[t];
  if (t < kQ) s.ck[t] = ft->ck[t];
  if (t < kMaxSources) {
    s.nrlay[t] = ft->nrlay[t];
    for (int b = 0; b < kMaxSrcLayers; ++b) s.rlay[t][b] = ft->rlay[t][b];
    s.qc0[t] = ft->qc0[t];
    s.qch0[t] = ft->qch0[t];
    s.qn[t] = ft->qn[t];
    s.pair_col[t] = ft->pair_col[t];
  }
  if (t == 0) {
    s.mc0 = job->maps[0];
    s.n_ck = ft->n_ck;
    s.n_pair = ft->n_pair;
  }
  // columns of the arg-max pairs (value, channel): maxima, not sums
  u32 am_val = 0;
  for (int k = 0; k < ft->n_pair; ++k) am_val |= 1u << ft->pair_col[k];
  const u32 am_any = am_val | (am_val << 1);
  const u32 le = 0xffffffffu >> (31 - lane);  // lanes up to this one
  u32 heads = 0;  // runs that begin at this thread's points
  float* srow = s.stage + t * kQS;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    __syncthreads();  // tables in place; the previous tile is done with the stage
    const int64_t p0 = (int64_t)tile * kFT;
    const int np = (int)min((int64_t)kFT, n_kept - p0);
    const int64_t p = p0 + t;
    const bool on = t < np;
    // A. key, neighbours' keys, runs and pieces
    u32 key = 0xfffffffeu, kprev = 0xfffffffeu, knext = 0xfffffffeu, id = 0;
    if (on) {
      key = sk[p];
      id = sv[p];
      if (p > 0) kprev = sk[p - 1];
      if (p + 1 < n_kept) knext = sk[p + 1];
    }
    const bool hd = on && key != kprev;  // a run begins here
    const bool ed = on && key != knext;  // a run ends here
    const bool tl = t == np - 1;         // the tile's last point
    const u32 hb = __ballot_sync(0xffffffffu, hd);
    if (lane == 0) s.whd[warp] = hb;
    heads += hd ? 1u : 0u;
    const int hl = 31 - __clz((hb | 1u) & le);  // first lane of this lane's piece (run within the warp)
    // pre-call state of the cell (the gate's), coordinates
    u32 fl = 0;
    float h0 = 0.f, v0 = 0.f, xs = 0.f, ys = 0.f, zs = 0.f;
    u32 na0 = 0, nr0 = 0;  // pre-call counts of the cell, for the lane that ends the run's piece
    if (on && (ed || tl)) {
      na0 = md.n_acc[key];
      nr0 = md.n_rej[key];
    }
    if (on) {
      fl = md.flags[key];
      h0 = md.h[key];
      v0 = md.var[key];
      xs = __ldg(xyz + 3 * (int64_t)id);
      ys = __ldg(xyz + 3 * (int64_t)id + 1);
      zs = __ldg(xyz + 3 * (int64_t)id + 2);
    }
    if (ed) {  // rule layers' rows of a cell this lane may fuse, into L2
      for (int q = 0; q < n_src; ++q)
        for (int j = 0; j < s.nrlay[q]; ++j) {
          const LayerDev& L = s.L[s.rlay[q][j]];
          if (L.rule == MEM_RULE_LATEST) continue;
          const int bytes = L.S * (L.dtype == MEM_F32 ? 4 : 2);
          const char* row = (const char*)L.data + (int64_t)key * bytes;
          for (int o = 0; o < bytes; o += 128) prefetch_l2(row + o);
          prefetch_l2(row + bytes - 1);
        }
    }
    // B. the point's channels into its row, with the arg-max of a class-max
    //    source on the way (top-k sources by the chunk table)
    if (on) {
      for (int q = 0; q < n_src; ++q) {
        const SrcDev& S = s.src[q];
        if (TOPK && S.topk) continue;
        stage_src(srow, S.data, S.dtype, id, S.C, s.qc0[q], S.vec_ok, S.has_classmax);
      }
      if (TOPK) stage_topk_chunks(s.ck, s.n_ck, s.src, srow, id);
    }
    // C. outlier gate against the pre-call state: the point's height sums
    u64 zk = 0;  // ray-cast clean-up: (call id, lowest z) key of an accepted point
    if (on) {
      const MapCall* mc = md.n_maps > 1 ? job->maps + key / md.W2 : &s.mc0;
      float z, vm;
      eval_zvm(md, *mc, xs, ys, zs, z, vm);
      const bool rej = (fl & kFlagValid) && gate_reject(z, h0, v0, vm, md.lam2);
      const float w = __frcp_rn(vm);
      srow[0] = rej ? 0.f : w;
      srow[1] = rej ? 0.f : z * w;
      srow[2] = rej ? 0.f : 1.f;
      srow[3] = rej ? 1.f : 0.f;
      if (RAY && !rej) zk = call_hi | (u64)(~ordered_bits(__float_as_uint(z)));
    }
    // D. sums over the pieces of runs in the warp: lane c walks column c down
    //    the warp's rows in point order and leaves each piece's sum in the
    //    piece's last row; the arg-max pairs take a segmented maximum by
    //    shuffles (the piece's last lane ends with the piece's pair)
    __syncwarp();  // every lane's row is staged
    const u32 pm = __ballot_sync(0xffffffffu, on && (ed || lane == 31 || tl));  // last lanes of pieces
    {
      const bool keep = lane < G && !((am_any >> lane) & 1u);
      float* col = s.stage + warp * 32 * kQS + lane;
      const int nv = min(32, np - warp * 32);  // points of this warp (warp-uniform)
      float a = 0.f;
      for (int i0 = 0; i0 < nv; i0 += 8) {
        float x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = col[(i0 + u) * kQS];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (i0 + u < nv) {
            a += x[u];
            if ((pm >> (i0 + u)) & 1u) {
              if (keep) col[(i0 + u) * kQS] = a;
              a = 0.f;
            }
          }
        }
      }
    }
    if (s.n_pair) {
      bool take[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) take[k] = lane - (1 << k) >= hl;
      for (int k = 0; k < s.n_pair; ++k) {
        const int c = s.pair_col[k];
        float2 m = make_float2(srow[c], srow[c + 1]);
#pragma unroll
        for (int b = 0; b < 5; ++b) {
          const float ov = __shfl_up_sync(0xffffffffu, m.x, 1 << b);
          const float oi = __shfl_up_sync(0xffffffffu, m.y, 1 << b);
          if (take[b]) m = cm_comb(make_float2(ov, oi), m);
        }
        srow[c] = m.x;
        srow[c + 1] = m.y;
      }
    }
    if (RAY) {  // the lowest accepted z of every cell: segmented maximum of the keys, one atomic per piece
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const u64 o = __shfl_up_sync(0xffffffffu, zk, 1 << k);
        if (lane - (1 << k) >= hl && o > zk) zk = o;
      }
      if (on && zk != 0 && ((pm >> lane) & 1u)) atomicMax((unsigned long long*)(md.zacc + key), (unsigned long long)zk);
    }
    if (t == 0) {  // both slots unused unless a piece below writes one
      fz_slot(md, acc, tile, 0)[kSlotBits] = 0.f;
      fz_slot(md, acc, tile, 1)[kSlotBits] = 0.f;
    }
    __syncthreads();  // every warp's last row (the piece continuing into the next warp) is complete
    // E. the lane where a run ends, or where the tile ends inside a run: the
    //    run's sums over the tile, then the run is fused here or its piece
    //    goes to a slot
    if (on && (ed || tl)) {
      int ht = -1;  // tile index of the run's first point (-1: the run began in an earlier tile)
      int w1 = warp;
      if ((hb >> hl) & 1u) {
        ht = warp * 32 + hl;
      } else {
        w1 = 0;
        for (int w = warp - 1; w >= 0; --w) {
          const u32 b = s.whd[w];
          if (b) {
            ht = w * 32 + 31 - __clz(b);
            w1 = w;
            break;
          }
        }
      }
      if (w1 < warp) {  // the pieces of earlier warps, in warp order, then this lane's piece
        for (int c = 0; c < G; ++c) {
          if ((am_val >> c) & 1u) {
            float2 m = make_float2(s.stage[(w1 * 32 + 31) * kQS + c], s.stage[(w1 * 32 + 31) * kQS + c + 1]);
            for (int w = w1 + 1; w < warp; ++w)
              m = cm_comb(m, make_float2(s.stage[(w * 32 + 31) * kQS + c], s.stage[(w * 32 + 31) * kQS + c + 1]));
            m = cm_comb(m, make_float2(srow[c], srow[c + 1]));
            srow[c] = m.x;
            srow[c + 1] = m.y;
            ++c;
          } else {
            float a = s.stage[(w1 * 32 + 31) * kQS + c];
            for (int w = w1 + 1; w < warp; ++w) a += s.stage[(w * 32 + 31) * kQS + c];
            srow[c] = a + srow[c];
          }
        }
      }
      const u32 nt = (u32)(t - max(ht, 0) + 1);  // points of the run in the tile
      const u32 g = key;
      if (ht >= 0 && ed) {
        // the whole run lies in the tile: every layer's rule, class max, height, flags
        const float N = (float)nt, rN = __frcp_rn(N);
        for (int q = 0; q < n_src; ++q)
          if (s.qn[q] > 0)
            for (int j = 0; j < s.nrlay[q]; ++j) {
              const int l = s.rlay[q][j];
              lane_rule(s.L[l], l, srow + s.qc0[q], s.qch0[q], s.qn[q], g, fl, N, rN);
            }
        for (int q = 0; q < n_src; ++q)
          if (s.src[q].has_classmax) {
            const int av = s.qc0[q] + s.src[q].C;  // arg-max value column
            const float best = srow[av];
            write_classmax(s.L, s.src[q], g, best, best == -INFINITY ? -1 : __float_as_int(srow[av + 1]));
          }
        u32 f = fl;
        height_update(md, g, f, h0, v0, srow[0], srow[1], (u32)srow[2], (u32)srow[3], na0, nr0);
        for (int q = 0; q < n_src; ++q) {
          if (any_gauss) write_gauss_var(s.L, s.src[q], g, f, N, rN);
          for (int b = 0; b < s.src[q].n_layers; ++b) f |= 2u << s.src[q].layers[b];
        }
        md.flags[g] = f;
      } else {
        // [0]: a run begun in an earlier tile that ends here; [1]: a run that continues past the tile
        float* hdr = fz_slot(md, acc, tile, ed ? 0 : 1);
        const u32 bits = kBitUsed | (ht >= 0 ? kBitHead : 0u) | (ed ? kBitEnd : 0u);
        hdr[kSlotKey] = __uint_as_float(g);
        hdr[kSlotN] = __uint_as_float(nt);
        hdr[kSlotBits] = __uint_as_float(bits);
        hdr[kSlotFl] = __uint_as_float(fl);
        hdr[kSlotH0] = h0;
        hdr[kSlotV0] = v0;
        hdr[kSlotNacc] = __uint_as_float(na0);
        hdr[kSlotNrej] = __uint_as_float(nr0);
        for (int c = 0; c < G; ++c) hdr[slot_off(c)] = srow[c];
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) heads += __shfl_xor_sync(0xffffffffu, heads, o);
  if (lane == 0 && heads) atomicAdd(&md.counters[5], heads);
}

// ---------------------------------------------------------------------------

// One warp per run that crosses tile boundaries, started from the tile where
// it begins: the pieces are that tile's slot [1], the slots [1] of the tiles
// it covers entirely, and slot [0] of the tile where it ends. Lanes first
// read the header words and 32 following tiles' slot bits at once (the end
// is the first following slot [0] in use), then take columns: each adds its
// column over the pieces in tile order and loads the old values of the
// column's layers together, then stores the new values.
__global__ void __launch_bounds__(128) k_fuse_cross(MapDev md, const PointJob* __restrict__ job) {
  if (*(volatile int*)md.err) return;  // a device error is pending: the point path does nothing
  __shared__ LayerDev sL[kMaxLayers];
  __shared__ SrcDev ssrc[kMaxSources];
  __shared__ int srlay[kMaxSources][kMaxSrcLayers], snrlay[kMaxSources];
  const int64_t n_kept = *(volatile u32*)&md.counters[6];
  const int n_tiles = (int)((n_kept + kFT - 1) / kFT);
  const int n_src = job->n_src;
  const int acc = job->acc;
  const int G = job->ft.ncol;
  const int t = threadIdx.x;
  if (t < md.n_layers) sL[t] = md.L[t];
  if (t < n_src) ssrc[t] = job->src[t];
  if (t < kMaxSources) {
    snrlay[t] = job->ft.nrlay[t];
    for (int b = 0; b < kMaxSrcLayers; ++b) srlay[t][b] = job->ft.rlay[t][b];
  }
  __syncthreads();
  const int lane = t & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  u32 crossing = 0;
  for (int h = (blockIdx.x * blockDim.x + t) >> 5; h < n_tiles; h += nwarps) {
    const float* head = fz_slot(md, acc, h, 1);
    const u32 hw = lane < kSlotHdr ? __float_as_uint(__ldcg(head + lane)) : 0u;
    const int t1 = h + 1 + lane;
    const u32 b0 = t1 < n_tiles ? __float_as_uint(__ldcg(fz_slot(md, acc, t1, 0) + kSlotBits)) : kBitUsed;
    const u32 hb = __shfl_sync(0xffffffffu, hw, kSlotBits);
    if ((hb & (kBitUsed | kBitHead)) != (kBitUsed | kBitHead)) continue;  // warp-uniform
    ++crossing;
    // the tile where the run ends
    u32 em = __ballot_sync(0xffffffffu, (b0 & kBitUsed) != 0u);
    int last = em ? h + __ffs(em) : -1;
    for (int t0 = h + 33; last < 0 && t0 < n_tiles; t0 += 32) {  // runs longer than 32 tiles
      const int tt = t0 + lane;
      em = __ballot_sync(0xffffffffu,
                         tt < n_tiles && (__float_as_uint(__ldcg(fz_slot(md, acc, tt, 0) + kSlotBits)) & kBitUsed));
      if (em) last = t0 + __ffs(em) - 1;
    }
    if (last < 0) last = n_tiles - 1;  // not reached for a consistent slot table
    cross_run(md, sL, ssrc, srlay, snrlay, n_src, G, acc, h, last, lane);
  }
  if (lane == 0 && crossing) atomicAdd(&md.counters[4], crossing);
}

// 5. ray-cast clean-up: every cell that accepted points in this call walks the
//    Bresenham line from the sensor's cell to itself (both ends excluded) with
//    the ray of its lowest accepted point, and invalidates every intermediate
//    cell that is valid, accepted no point of the call and stands more than
//    ray_margin above the ray. The lowest point's ray passes below every cell
//    any other point of the cell passes below (the ray height grows with the
//    point's z under round-to-nearest, t >= 0), so one walk per cell decides
//    exactly what one walk per accepted point decides. The heights read here
//    belong to cells without accepted points, which this call did not change;
//    invalidation is idempotent, so the result does not depend on the order.
//
//    A block takes a 16 x 16 tile of cells and first lists its walking cells in
//    shared memory, so the walks run on consecutive threads; each walk advances
//    four cells at a time with their loads issued together. The ray height is
//    first estimated with a reciprocal of |e - s|^2 (relative error below
//    2^-22 in t); only where that estimate lies within a bound of the margin is
//    the exact sequence (correctly rounded division, fma, subtraction) taken,
//    so every decision equals the exact one.
__device__ __forceinline__ void bres_step(int& x, int& y, int& err, int dx, int dy, int stx, int sty) {
  const int e2 = 2 * err;
  if (e2 >= dy) {
    err += dy;
    x += stx;
  }
  if (e2 <= dx) {
    err += dx;
    y += sty;
  }
}

__global__ void __launch_bounds__(256) k_raycast(MapDev md, const PointJob* __restrict__ job) {
  if (*(volatile int*)md.err) return;  // a device error is pending: the point path does nothing
  const int W = md.W;
  const int b = blockIdx.z;
  const int tid = threadIdx.y * 16 + threadIdx.x;
  __shared__ MapCall smc;
  __shared__ int s_n;
  __shared__ u32 s_cell[256];
  __shared__ float s_z[256];
  if (tid == 0) {
    smc = job->maps[b];
    s_n = 0;
  }
  __syncthreads();
  const u32 call = job->call_id;
  const u32 base = (u32)b * md.W2;
  const u32* __restrict__ stamp = reinterpret_cast<const u32*>(md.zacc);  // [2g + 1]: call id of cell g
  {
    const int ix = blockIdx.x * 16 + threadIdx.x, iy = blockIdx.y * 16 + threadIdx.y;
    if (ix < W && iy < W) {
      const u64 v = __ldg((const unsigned long long*)(md.zacc + base + phys_cell(md, smc, ix, iy)));
      if ((u32)(v >> 32) == call) {
        const int k = atomicAdd(&s_n, 1);
        s_cell[k] = ((u32)iy << 16) | (u32)ix;
        s_z[k] = __uint_as_float(unordered_bits(~(u32)v));
      }
    }
  }
  __syncthreads();
  if (tid >= s_n) return;
  const int ix = (int)(s_cell[tid] & 0xffffu), iy = (int)(s_cell[tid] >> 16);
  const float z = s_z[tid];
  int sx, sy;
  clamped_cell(md, smc.t[0], smc.t[1], sx, sy);
  const float zs = smc.t[2];
  const float dz = __fsub_rn(z, zs);
  const float margin = md.ray_margin;
  const int dx = abs(ix - sx), dy = -abs(iy - sy);
  const int stx = sx < ix ? 1 : -1, sty = sy < iy ? 1 : -1;
  const int dxs = ix - sx, dys = iy - sy;
  const float den = (float)(dxs * dxs + dys * dys);
  const float rden = __frcp_rn(den);
  // bound on |estimate - exact| of (h - ray - margin), far above the estimate's error
  const float tol = 4e-6f * (fabsf(dz) + fabsf(zs) + margin + 1.f);
  int err = dx + dy, x = sx, y = sy;
  bool done = (x == ix && y == iy);
  u32 cleared = 0;
  while (!done) {
    int qx[4], qy[4];
    bool act[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      act[u] = false;
      qx[u] = qy[u] = 0;
      if (!done) {
        bres_step(x, y, err, dx, dy, stx, sty);
        if (x == ix && y == iy) {
          done = true;
        } else {
          qx[u] = x;
          qy[u] = y;
          act[u] = true;
        }
      }
    }
    u32 q[4], fl[4], st[4];
    float hq[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      q[u] = base + phys_cell(md, smc, qx[u], qy[u]);
      fl[u] = act[u] ? md.flags[q[u]] : 0u;
      st[u] = act[u] ? __ldg(stamp + 2 * (size_t)q[u] + 1) : call;
      hq[u] = act[u] ? __ldg(md.h + q[u]) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (!act[u] || !(fl[u] & kFlagValid) || st[u] == call) continue;
      const int num = (qx[u] - sx) * dxs + (qy[u] - sy) * dys;
      const float ra = __fmaf_rn(__fmul_rn((float)num, rden), dz, zs);
      const float est = hq[u] - ra - margin;
      bool clear = est > 0.f;
      if (fabsf(est) <= tol + 4e-6f * fabsf(hq[u])) {  // near the margin: the exact sequence
        const float tq = __fdiv_rn((float)num, den);
        clear = __fsub_rn(hq[u], __fmaf_rn(tq, dz, zs)) > margin;
      }
      if (clear) cleared += (atomicAnd(md.flags + q[u], ~kFlagValid) & kFlagValid) ? 1u : 0u;
    }
  }
  if (cleared) atomicAdd(&md.counters[10], cleared);
}

// time-dependent variance growth of every valid cell
__global__ void k_time_update(MapDev md, int64_t cells) {
  if (*(volatile int*)md.err) return;  // a device error is pending: the point path does nothing
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < cells;
       g += (int64_t)gridDim.x * blockDim.x)
    if (md.flags[g] & kFlagValid) md.var[g] = __fadd_rn(md.var[g], md.time_var);
}

}  // namespace memk

// ---------------------------------------------------------------------------
// host launcher

namespace memh {
using namespace memk;

// Kernel attributes are per device: the current device's index selects the
// entry of these tables (set by prepare_kernels with that device current).
constexpr int kMaxDevices = 128;
// resident CTAs per SM of the tile and warp fuse kernels (their persistent grids)
static int g_sums_ctas_per_sm[kMaxDevices] = {};
static int g_warps_ctas_per_sm[kMaxDevices] = {};

static int current_device() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) d = 0;
  return d;
}

template <int RB>
static size_t sort_smem() {
  constexpr int RADIX = 1 << RB;
  return sizeof(u32) * ((kSortThreads / 32) * RADIX + 2 * kTile + 4 * RADIX);
}

template <int RB>
static cudaError_t set_attrs() {
  static bool done[kMaxDevices] = {};
  const int dev = current_device();
  if (done[dev]) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_onesweep<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sort_smem<RB>());
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

cudaError_t launch_time_update(Map* m, cudaStream_t st) {
  const MapDev& md = m->md;
  if (md.time_var == 0.f) return cudaSuccess;
  ProfScope ps(m, kProfTime, st);
  const int64_t cells = (int64_t)md.n_maps * md.W2;
  k_time_update<<<m->n_sm * m->tune.blocks_per_sm, 256, 0, st>>>(md, cells);
  return cudaGetLastError();
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
  if (md.drift_alpha != 0.0) {
    ProfScope ps(m, kProfDrift, st);
    k_drift_reduce<<<dim3(md.drift_R, md.n_maps), 256, 0, st>>>(md, d_job);
    const u32 per_map = (md.W2 + 256 * 8 - 1) / (256 * 8);
    k_drift_apply<<<dim3(per_map, md.n_maps), 256, 0, st>>>(md);
  }
  {
    ProfScope ps(m, kProfSort, st);
    for (int p = 0; p < P; ++p) k_onesweep<RB><<<sms * 2, kSortThreads, sort_smem<RB>(), st>>>(md, d_job, p);
  }
  {
    ProfScope ps(m, kProfFuseTiles, st);
    const bool topk = m->fuse_variant & 1;
    if ((m->fuse_variant & 2) && m->tune.fuse_kernel == 0) {  // the columns fit one round: warp kernel
      const int cps = g_warps_ctas_per_sm[current_device()];
      const dim3 grid(sms * (cps > 0 ? cps : 1));
      const size_t sm = sizeof(WarpSmem);
      if (topk)
        md.ray_on ? k_fuse_warps<true, true><<<grid, kFT, sm, st>>>(md, d_job, P & 1)
                  : k_fuse_warps<true, false><<<grid, kFT, sm, st>>>(md, d_job, P & 1);
      else
        md.ray_on ? k_fuse_warps<false, true><<<grid, kFT, sm, st>>>(md, d_job, P & 1)
                  : k_fuse_warps<false, false><<<grid, kFT, sm, st>>>(md, d_job, P & 1);
    } else {
      const int cps = g_sums_ctas_per_sm[current_device()];
      const dim3 grid(sms * (cps > 0 ? cps : 1));
      if (topk)
        md.ray_on ? k_fuse_tiles<true, true><<<grid, kFT, sizeof(SumSmem), st>>>(md, d_job, P & 1)
                  : k_fuse_tiles<true, false><<<grid, kFT, sizeof(SumSmem), st>>>(md, d_job, P & 1);
      else
        md.ray_on ? k_fuse_tiles<false, true><<<grid, kFT, sizeof(SumSmem), st>>>(md, d_job, P & 1)
                  : k_fuse_tiles<false, false><<<grid, kFT, sizeof(SumSmem), st>>>(md, d_job, P & 1);
    }
  }
  {
    ProfScope ps(m, kProfFuseCross, st);
    k_fuse_cross<<<sms * 8, 128, 0, st>>>(md, d_job);
  }
  if (md.ray_on) {
    ProfScope ps(m, kProfRay, st);
    k_raycast<<<dim3((md.W + 15) / 16, (md.W + 15) / 16, md.n_maps), dim3(16, 16), 0, st>>>(md, d_job);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_time_update(m, st);
}

cudaError_t prepare_kernels() {
  const int dev = current_device();
  cudaError_t e = cudaSuccess;
  for (auto f : {k_fuse_tiles<false, false>, k_fuse_tiles<false, true>, k_fuse_tiles<true, false>,
                 k_fuse_tiles<true, true>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SumSmem));
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_sums_ctas_per_sm[dev], k_fuse_tiles<false, false>, kFT,
                                                      sizeof(SumSmem));
  if (g_sums_ctas_per_sm[dev] < 1) g_sums_ctas_per_sm[dev] = 1;
  for (auto f : {k_fuse_warps<false, false>, k_fuse_warps<false, true>, k_fuse_warps<true, false>,
                 k_fuse_warps<true, true>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(WarpSmem));
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_warps_ctas_per_sm[dev], k_fuse_warps<false, false>, kFT,
                                                      sizeof(WarpSmem));
  if (g_warps_ctas_per_sm[dev] < 1) g_warps_ctas_per_sm[dev] = 1;
  if (e == cudaSuccess) e = set_attrs<8>();
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
