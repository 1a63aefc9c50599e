// Post-processing plugins that read map layers already on the GPU and produce
// new layers (Sec. III-D): surface normals of the elevation layer (Table I
// "normal calculation") and the PCA layer of a feature layer (the plugin of
// the post-processing figure that turns feature layers into a PCA layer).
//
// Normals: one thread per logical cell; slopes from central differences of
// the valid neighbours (one-sided where one is missing), as fixed float32
// sequences, so the result does not depend on the launch.
//
// PCA: per map, over the cells where the layer is observed,
//   1. mean: blocks take fixed cell ranges, threads take channels; the block
//      sums (float32) are added in block order in float64;
//   2. covariance of (f - mean): blocks take fixed cell ranges and stage 32
//      centred rows at a time in shared memory; each thread accumulates a
//      T x T tile of the C x C matrix with float32 FMAs; the partial matrices
//      are added in block order in float64;
//   3. eigenvectors: one block runs cyclic Jacobi sweeps (round-robin pairs,
//      C/2 disjoint rotations at a time) in float32 shared memory until the
//      off-diagonal mass is at the float32 rounding level of the matrix
//      (at most 20 sweeps), then sorts the
//      eigenvalues and signs each kept vector so that its largest-magnitude
//      component is positive;
//   4. projection of every observed cell on the kept vectors.
#include <math.h>

#include <vector>

#include "mem_host.h"

namespace memk {

// ---------------------------------------------------------------------------
// normals

__device__ __forceinline__ bool axis_slope(float hm, bool va, float ha, bool vb, float hb, float res, float& g) {
  if (va && vb) {
    g = __fdiv_rn(__fsub_rn(hb, ha), __fmul_rn(2.0f, res));
    return true;
  }
  if (vb) {
    g = __fdiv_rn(__fsub_rn(hb, hm), res);
    return true;
  }
  if (va) {
    g = __fdiv_rn(__fsub_rn(hm, ha), res);
    return true;
  }
  return false;
}

__global__ void __launch_bounds__(256) k_normals(MapDev md, int map, int rx, int ry, float* __restrict__ out,
                                                 uint8_t* __restrict__ ok) {
  const int W = md.W;
  const int ix = blockIdx.x * 16 + threadIdx.x, iy = blockIdx.y * 16 + threadIdx.y;
  if (ix >= W || iy >= W) return;
  const u32 base = (u32)map * md.W2;
  auto g_of = [&](int x, int y) {
    int px = x + rx;
    if (px >= W) px -= W;
    int py = y + ry;
    if (py >= W) py -= W;
    return base + (u32)py * (u32)W + (u32)px;
  };
  const int64_t j = (int64_t)iy * W + ix;
  float n0 = 0.f, n1 = 0.f, n2 = 0.f;
  bool good = false;
  const u32 g = g_of(ix, iy);
  if (md.flags[g] & kFlagValid) {
    const float hm = md.h[g];
    const bool vl = ix > 0 && (md.flags[g_of(ix - 1, iy)] & kFlagValid);
    const bool vr = ix + 1 < W && (md.flags[g_of(ix + 1, iy)] & kFlagValid);
    const bool vd = iy > 0 && (md.flags[g_of(ix, iy - 1)] & kFlagValid);
    const bool vu = iy + 1 < W && (md.flags[g_of(ix, iy + 1)] & kFlagValid);
    float gx, gy;
    if (axis_slope(hm, vl, vl ? md.h[g_of(ix - 1, iy)] : 0.f, vr, vr ? md.h[g_of(ix + 1, iy)] : 0.f, md.res, gx) &&
        axis_slope(hm, vd, vd ? md.h[g_of(ix, iy - 1)] : 0.f, vu, vu ? md.h[g_of(ix, iy + 1)] : 0.f, md.res, gy)) {
      const float q = __fmaf_rn(gx, gx, __fmaf_rn(gy, gy, 1.0f));
      const float inv = __fdiv_rn(1.0f, __fsqrt_rn(q));
      n0 = __fmul_rn(-gx, inv);
      n1 = __fmul_rn(-gy, inv);
      n2 = inv;
      good = true;
    }
  }
  out[3 * j] = n0;
  out[3 * j + 1] = n1;
  out[3 * j + 2] = n2;
  if (ok) ok[j] = good ? 1 : 0;
}

// ---------------------------------------------------------------------------
// PCA

constexpr int kPcaMaxC = 128;      // channels of a PCA input layer
constexpr int kPcaRows = 32;       // centred rows staged at a time by the covariance blocks
constexpr int kPcaMaxComp = 8;

struct PcaArgs {
  int map, layer, C, n_comp, blocks;
  const void* data;  // the layer's values [cells][S]
  int S, dtype;
  u32 obs_bit;
  double* mean_part;  // [blocks][C + 1] (sums, then the count)
  float* cov_part;    // [blocks][C][C]
  float* mean;        // [C]
  float* cov;         // [C][C]
  float* vecs;        // [n_comp][C]
  float* vals;        // [n_comp]
  float* proj;        // [W2][n_comp] (logical order)
  float* info;        // optional: [n_comp] values, [n_comp][C] vectors, [C] mean
};

__device__ __forceinline__ float layer_val(const void* data, int dtype, int64_t off) {
  if (dtype == MEM_BF16) return __bfloat162float(((const __nv_bfloat16*)data)[off]);
  if (dtype == MEM_F16) return __half2float(((const __half*)data)[off]);
  return ((const float*)data)[off];
}

// the fixed cell range of block b of `blocks` over W2 cells
__device__ __forceinline__ void block_range(u32 W2, int b, int blocks, u32& c0, u32& c1) {
  c0 = (u32)(((uint64_t)W2 * b) / blocks);
  c1 = (u32)(((uint64_t)W2 * (b + 1)) / blocks);
}

__global__ void __launch_bounds__(256) k_pca_mean(MapDev md, PcaArgs a) {
  // thread t: column c = t % (C + 1) (column C counts the cells), cell lane t / (C + 1);
  // lanes take every lanes-th cell of the block's range, four at a time
  __shared__ float part[256];
  u32 c0, c1;
  block_range(md.W2, blockIdx.x, a.blocks, c0, c1);
  const u32 base = (u32)a.map * md.W2;
  const int cols = a.C + 1, lanes = blockDim.x / cols;
  const int c = threadIdx.x % cols, lane = threadIdx.x / cols;
  float s = 0.f;
  if (lane < lanes) {
    float q[4] = {0.f, 0.f, 0.f, 0.f};
    for (u32 p = c0 + lane; p < c1; p += 4 * lanes) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const u32 pu = p + u * lanes;
        if (pu < c1 && (md.flags[base + pu] & a.obs_bit))
          q[u] += c < a.C ? layer_val(a.data, a.dtype, (int64_t)(base + pu) * a.S + c) : 1.f;
      }
    }
    s = (q[0] + q[1]) + (q[2] + q[3]);
  }
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < cols) {
    float t = 0.f;
    for (int l = 0; l < lanes; ++l) t += part[l * cols + threadIdx.x];
    a.mean_part[(int64_t)blockIdx.x * cols + threadIdx.x] = (double)t;
  }
}

__global__ void k_pca_mean_final(PcaArgs a) {
  for (int c = threadIdx.x; c <= a.C; c += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < a.blocks; ++b) s += a.mean_part[(int64_t)b * (a.C + 1) + c];
    a.mean_part[(int64_t)a.blocks * (a.C + 1) + c] = s;  // totals after the partials
  }
  __syncthreads();
  const double n = a.mean_part[(int64_t)a.blocks * (a.C + 1) + a.C];
  for (int c = threadIdx.x; c < a.C; c += blockDim.x)
    a.mean[c] = n > 0.0 ? (float)(a.mean_part[(int64_t)a.blocks * (a.C + 1) + c] / n) : 0.f;
}

// partial covariance sums of one block's cells: thread (ty, tx) owns rows
// ty*T .. and columns tx*T .. of the C x C matrix (T = ceil(C / 16))
template <int T>
__global__ void __launch_bounds__(256) k_pca_cov(MapDev md, PcaArgs a) {
  __shared__ float xs[kPcaRows][kPcaMaxC + 1];
  u32 c0, c1;
  block_range(md.W2, blockIdx.x, a.blocks, c0, c1);
  const u32 base = (u32)a.map * md.W2;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[T][T];
#pragma unroll
  for (int i = 0; i < T; ++i)
#pragma unroll
    for (int k = 0; k < T; ++k) acc[i][k] = 0.f;
  for (u32 p0 = c0; p0 < c1; p0 += 256) {
    // list the observed cells of the next 256 (in cell order), then stage them 32 at a time
    const u32 p = p0 + threadIdx.x;
    const bool on = p < c1 && (md.flags[base + p] & a.obs_bit);
    __shared__ u32 wcnt[8];
    const u32 bal = __ballot_sync(0xffffffffu, on);
    if ((threadIdx.x & 31) == 0) wcnt[threadIdx.x >> 5] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < 8; ++w) {
      before += w < (int)(threadIdx.x >> 5) ? (int)wcnt[w] : 0;
      total += (int)wcnt[w];
    }
    const int my = before + __popc(bal & ((1u << (threadIdx.x & 31)) - 1u));
    __shared__ u32 list[256];
    if (on) list[my] = p;
    __syncthreads();
    for (int r0 = 0; r0 < total; r0 += kPcaRows) {
      const int nr = min(kPcaRows, total - r0);
      for (int e = threadIdx.x; e < nr * a.C; e += blockDim.x) {
        const int r = e / a.C, c = e - r * a.C;
        xs[r][c] = __fsub_rn(layer_val(a.data, a.dtype, (int64_t)(base + list[r0 + r]) * a.S + c), a.mean[c]);
      }
      __syncthreads();
      for (int r = 0; r < nr; ++r) {
        float xa[T], xb[T];
#pragma unroll
        for (int i = 0; i < T; ++i) {
          const int ra = ty * T + i, cb = tx * T + i;
          xa[i] = ra < a.C ? xs[r][ra] : 0.f;
          xb[i] = cb < a.C ? xs[r][cb] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < T; ++i)
#pragma unroll
          for (int k = 0; k < T; ++k) acc[i][k] = __fmaf_rn(xa[i], xb[k], acc[i][k]);
      }
      __syncthreads();
    }
  }
  float* out = a.cov_part + (int64_t)blockIdx.x * a.C * a.C;
#pragma unroll
  for (int i = 0; i < T; ++i)
#pragma unroll
    for (int k = 0; k < T; ++k) {
      const int ra = ty * T + i, cb = tx * T + k;
      if (ra < a.C && cb < a.C) out[ra * a.C + cb] = acc[i][k];
    }
}

__global__ void k_pca_cov_final(PcaArgs a) {
  const double n = a.mean_part[(int64_t)a.blocks * (a.C + 1) + a.C];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < a.C * a.C; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < a.blocks; ++b) s += (double)a.cov_part[(int64_t)b * a.C * a.C + e];
    a.cov[e] = n > 0.0 ? (float)(s / n) : 0.f;
  }
}

// Cyclic Jacobi with round-robin pairs on the C x C covariance (C padded to an
// even n with a zero row and column), in shared memory; one block of 1024.
__global__ void __launch_bounds__(1024) k_pca_eig(PcaArgs a) {
  extern __shared__ float sm[];
  const int C = a.C, n = (C + 1) & ~1;
  float* A = sm;                 // [n][n + 1]
  float* V = A + n * (n + 1);    // [n][n + 1]
  float* cs = V + n * (n + 1);   // [n / 2][2] rotation cosines and sines
  int* pr = (int*)(cs + n);      // [n] round-robin positions
  __shared__ float s_off, s_tot;
  const int ld = n + 1;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, k = e - i * n;
    A[i * ld + k] = (i < C && k < C) ? a.cov[i * C + k] : 0.f;
    V[i * ld + k] = i == k ? 1.f : 0.f;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) pr[i] = i;
  __syncthreads();
  __shared__ float red[2][32];
  // converged when the off-diagonal mass is at the float32 rounding level of the matrix
  const float conv = (4.f * n * 5.96e-8f) * (4.f * n * 5.96e-8f);
  for (int sweep = 0; sweep < 20; ++sweep) {
    float off = 0.f, tot = 0.f;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e / n, k = e - i * n;
      const float v = A[i * ld + k] * A[i * ld + k];
      tot += v;
      if (i != k) off += v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = off;
      red[1][threadIdx.x >> 5] = tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float o2 = 0.f, t2 = 0.f;
      for (int w = 0; w < 32; ++w) {
        o2 += red[0][w];
        t2 += red[1][w];
      }
      s_off = o2;
      s_tot = t2;
    }
    __syncthreads();
    if (!(s_off > conv * s_tot)) break;
    for (int step = 0; step < n - 1; ++step) {
      // pair m: positions m and n - 1 - m of the round-robin order
      for (int m = threadIdx.x; m < n / 2; m += blockDim.x) {
        int p = pr[m], q = pr[n - 1 - m];
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        const float apq = A[p * ld + q], app = A[p * ld + p], aqq = A[q * ld + q];
        float c = 1.f, s = 0.f;
        if (apq != 0.f) {
          const float tau = (aqq - app) / (2.f * apq);
          const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
          c = 1.f / sqrtf(1.f + t * t);
          s = t * c;
        }
        cs[2 * m] = c;
        cs[2 * m + 1] = s;
      }
      __syncthreads();
      // rows: A <- J^T A (pair m mixes rows p and q)
      for (int e = threadIdx.x; e < (n / 2) * n; e += blockDim.x) {
        const int m = e / n, k = e - m * n;
        int p = pr[m], q = pr[n - 1 - m];
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        const float c = cs[2 * m], s = cs[2 * m + 1];
        const float ap = A[p * ld + k], aq = A[q * ld + k];
        A[p * ld + k] = c * ap - s * aq;
        A[q * ld + k] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int e = threadIdx.x; e < (n / 2) * n; e += blockDim.x) {
        const int m = e / n, k = e - m * n;
        int p = pr[m], q = pr[n - 1 - m];
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        const float c = cs[2 * m], s = cs[2 * m + 1];
        const float ap = A[k * ld + p], aq = A[k * ld + q];
        A[k * ld + p] = c * ap - s * aq;
        A[k * ld + q] = s * ap + c * aq;
        const float vp = V[k * ld + p], vq = V[k * ld + q];
        V[k * ld + p] = c * vp - s * vq;
        V[k * ld + q] = s * vp + c * vq;
      }
      __syncthreads();
      // next round-robin order: position 0 fixed, the others rotate by one
      if (threadIdx.x == 0) {
        const int last = pr[n - 1];
        for (int i = n - 1; i > 1; --i) pr[i] = pr[i - 1];
        pr[1] = last;
      }
      __syncthreads();
    }
  }
  // the n_comp largest eigenvalues (the smaller index first on ties), signed vectors
  if (threadIdx.x == 0) {
    int used[kPcaMaxComp];
    for (int k = 0; k < a.n_comp; ++k) {
      int best = -1;
      for (int i = 0; i < C; ++i) {
        bool taken = false;
        for (int j = 0; j < k; ++j) taken |= used[j] == i;
        if (!taken && (best < 0 || A[i * ld + i] > A[best * ld + best])) best = i;
      }
      used[k] = best;
      int big = 0;
      for (int r = 1; r < C; ++r)
        if (fabsf(V[r * ld + best]) > fabsf(V[big * ld + best])) big = r;
      const float sg = V[big * ld + best] < 0.f ? -1.f : 1.f;
      a.vals[k] = A[best * ld + best];
      for (int r = 0; r < C; ++r) a.vecs[k * C + r] = sg * V[r * ld + best];
    }
  }
  __syncthreads();
  if (a.info) {
    for (int k = threadIdx.x; k < a.n_comp; k += blockDim.x) a.info[k] = a.vals[k];
    for (int e = threadIdx.x; e < a.n_comp * C; e += blockDim.x) a.info[a.n_comp + e] = a.vecs[e];
    for (int c = threadIdx.x; c < C; c += blockDim.x) a.info[a.n_comp + a.n_comp * C + c] = a.mean[c];
  }
}

__global__ void __launch_bounds__(256) k_pca_project(MapDev md, PcaArgs a, int rx, int ry) {
  __shared__ float sv[kPcaMaxComp * kPcaMaxC], sm[kPcaMaxC];
  for (int e = threadIdx.x; e < a.n_comp * a.C; e += blockDim.x) sv[e] = a.vecs[e];
  for (int c = threadIdx.x; c < a.C; c += blockDim.x) sm[c] = a.mean[c];
  __syncthreads();
  const int W = md.W;
  for (u32 j = blockIdx.x * blockDim.x + threadIdx.x; j < md.W2; j += gridDim.x * blockDim.x) {
    const int ix = (int)(j % (u32)W), iy = (int)(j / (u32)W);
    int px = ix + rx;
    if (px >= W) px -= W;
    int py = iy + ry;
    if (py >= W) py -= W;
    const u32 g = (u32)a.map * md.W2 + (u32)py * (u32)W + (u32)px;
    float out[kPcaMaxComp];
#pragma unroll
    for (int k = 0; k < kPcaMaxComp; ++k) out[k] = 0.f;
    if (md.flags[g] & a.obs_bit) {
      for (int c = 0; c < a.C; ++c) {
        const float x = __fsub_rn(layer_val(a.data, a.dtype, (int64_t)g * a.S + c), sm[c]);
#pragma unroll
        for (int k = 0; k < kPcaMaxComp; ++k)
          if (k < a.n_comp) out[k] = __fmaf_rn(x, sv[k * a.C + c], out[k]);
      }
    }
    for (int k = 0; k < a.n_comp; ++k) a.proj[(int64_t)j * a.n_comp + k] = out[k];
  }
}

}  // namespace memk

// ---------------------------------------------------------------------------
// host

namespace memh {
using namespace memk;

cudaError_t launch_normals(Map* m, int map_index, float* out, uint8_t* ok, cudaStream_t st) {
  dim3 blk(16, 16), grd((m->md.W + 15) / 16, (m->md.W + 15) / 16);
  k_normals<<<grd, blk, 0, st>>>(m->md, map_index, m->ring[2 * map_index], m->ring[2 * map_index + 1], out, ok);
  return cudaGetLastError();
}

// scratch of the PCA plugin, owned by the map (grown on demand, outside graphs)
cudaError_t launch_pca(Map* m, int map_index, int layer, int n_comp, float* proj, float* info, cudaStream_t st) {
  const LayerDev& L = m->Lh[layer];
  const int C = L.C;
  const int blocks = m->n_sm * 4;
  const size_t need = sizeof(double) * (size_t)(blocks + 1) * (C + 1) + sizeof(float) * (size_t)blocks * C * C +
                      sizeof(float) * ((size_t)C * C + C + (size_t)kPcaMaxComp * (C + 1)) + 1024;
  if (need > m->pca_cap) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    if (m->pca_buf) cudaFree(m->pca_buf);
    m->pca_buf = nullptr;
    m->pca_cap = 0;
    e = cudaMalloc(&m->pca_buf, need);
    if (e != cudaSuccess) return e;
    m->pca_cap = need;
  }
  char* p = (char*)m->pca_buf;
  PcaArgs a;
  a.map = map_index;
  a.layer = layer;
  a.C = C;
  a.n_comp = n_comp;
  a.blocks = blocks;
  a.data = L.data;
  a.S = L.S;
  a.dtype = L.dtype;
  a.obs_bit = 2u << layer;
  a.mean_part = (double*)p;
  p += sizeof(double) * (size_t)(blocks + 1) * (C + 1);
  a.cov_part = (float*)p;
  p += sizeof(float) * (size_t)blocks * C * C;
  a.cov = (float*)p;
  p += sizeof(float) * (size_t)C * C;
  a.mean = (float*)p;
  p += sizeof(float) * (size_t)C;
  a.vecs = (float*)p;
  p += sizeof(float) * (size_t)kPcaMaxComp * C;
  a.vals = (float*)p;
  a.proj = proj;
  a.info = info;
  k_pca_mean<<<blocks, 256, 0, st>>>(m->md, a);
  k_pca_mean_final<<<1, 256, 0, st>>>(a);
  const int T = (C + 15) / 16;
  if (T <= 1) k_pca_cov<1><<<blocks, 256, 0, st>>>(m->md, a);
  else if (T <= 2) k_pca_cov<2><<<blocks, 256, 0, st>>>(m->md, a);
  else if (T <= 4) k_pca_cov<4><<<blocks, 256, 0, st>>>(m->md, a);
  else k_pca_cov<8><<<blocks, 256, 0, st>>>(m->md, a);
  k_pca_cov_final<<<(C * C + 255) / 256, 256, 0, st>>>(a);
  const int n = (C + 1) & ~1;
  const size_t esm = sizeof(float) * (2 * (size_t)n * (n + 1) + n) + sizeof(int) * n;
  static bool attr[128] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 128 && !attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_pca_eig, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(float) * (2 * 128 * 129 + 128) + sizeof(int) * 128));
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  k_pca_eig<<<1, 1024, esm, st>>>(a);
  k_pca_project<<<m->n_sm * 4, 256, 0, st>>>(m->md, a, m->ring[2 * map_index], m->ring[2 * map_index + 1]);
  return cudaGetLastError();
}

}  // namespace memh

extern "C" mem_status mem_compute_normals(mem_map* mm, int32_t map_index, float* normals, uint8_t* ok,
                                          void* stream) {
  if (!mm || !normals) return memh::api_fail(MEM_ERR_ARG, "NULL argument");
  memh::Map* m = memh::map_of(mm);
  if (map_index < 0 || map_index >= m->cfg.n_maps) return memh::api_fail(MEM_ERR_ARG, "map_index out of range");
  cudaError_t e = memh::launch_normals(m, map_index, normals, ok, (cudaStream_t)stream);
  if (e != cudaSuccess) return memh::api_cuda_fail(e, "normals launch");
  return MEM_OK;
}

extern "C" mem_status mem_pca_layer(mem_map* mm, int32_t map_index, int32_t layer, int32_t n_comp, float* proj,
                                    float* info, void* stream) {
  if (!mm || !proj) return memh::api_fail(MEM_ERR_ARG, "NULL argument");
  memh::Map* m = memh::map_of(mm);
  if (map_index < 0 || map_index >= m->cfg.n_maps) return memh::api_fail(MEM_ERR_ARG, "map_index out of range");
  if (layer < 0 || layer >= m->cfg.n_layers) return memh::api_fail(MEM_ERR_ARG, "layer out of range");
  if (m->cfg.layers[layer].rule == MEM_RULE_CLASSMAX) return memh::api_fail(MEM_ERR_ARG, "a class-max layer has no features");
  const int C = m->cfg.layers[layer].channels;
  if (C < 1 || C > memk::kPcaMaxC) return memh::api_fail(MEM_ERR_ARG, "PCA takes layers of 1..%d channels", memk::kPcaMaxC);
  if (n_comp < 1 || n_comp > memk::kPcaMaxComp || n_comp > C)
    return memh::api_fail(MEM_ERR_ARG, "n_comp in [1, min(%d, channels)]", memk::kPcaMaxComp);
  cudaError_t e = memh::launch_pca(m, map_index, layer, n_comp, proj, info, (cudaStream_t)stream);
  if (e != cudaSuccess) return memh::api_cuda_fail(e, "PCA launch");
  return MEM_OK;
}
