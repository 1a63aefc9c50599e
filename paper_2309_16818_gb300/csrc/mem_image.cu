// Image association and fusion (Sec. III-B, Fig. 2): every valid cell is
// projected at its elevation into a pinhole camera; a cell is visible iff
// every valid cell on the Bresenham line from the camera's cell to it lies
// strictly below the ray from the camera to the cell (equality occludes).
// Visible cells fuse their pixel with the layer rules (one observation).
//
// A 16x16 tile of cells per block: the cells that need a visibility walk are
// listed in shared memory and walked by consecutive threads (neighbouring
// cells, so neighbouring lines read neighbouring heights through L1); each warp
// then fuses its visible cells one at a time with its lanes spread over the
// channels, so pixel rows and layer rows are read and written coalesced.
#include "mem_host.h"

namespace memk {

struct ImgParams {
  float R[9], t[3];  // map-centre frame -> optical camera frame
  float fx, fy, cx, cy;
  float hc;          // camera height
  int sx, sy;        // camera cell (clamped into the map)
  int H, Wi;
  int map_index, ring_x, ring_y;
  int n_src;
  SrcDev src[kMaxSources];
};

__device__ __forceinline__ u32 phys(const MapDev& md, int rx, int ry, int x, int y) {
  int px = x + rx;
  if (px >= md.W) px -= md.W;
  int py = y + ry;
  if (py >= md.W) py -= md.W;
  return (u32)py * (u32)md.W + (u32)px;
}

// Walk the integer Bresenham line from the camera cell (sx, sy) to (ex, ey)
// and test every intermediate cell against the ray height
//   ray = h_cam + t (h_cell - h_cam),  t = ((q - s).(e - s)) / |e - s|^2.
// Four cells per step with their loads issued together; the ray height is
// first estimated with a reciprocal of |e - s|^2 (relative error of t below
// 2^-22), and only where the estimate lies within a bound of the cell's
// height is the exact sequence (correctly rounded division, fma) taken, so
// every decision equals the exact one. Stops at the first occluder.
__device__ __forceinline__ bool walk_visible(const MapDev& md, u32 base, int rx, int ry, int sx, int sy,
                                             int ex, int ey, float hz, float hc) {
  const int dx = abs(ex - sx), dy = -abs(ey - sy);
  const int stx = sx < ex ? 1 : -1, sty = sy < ey ? 1 : -1;
  const int dxs = ex - sx, dys = ey - sy;
  const float den = (float)(dxs * dxs + dys * dys);
  const float rden = __frcp_rn(den);
  const float dh = __fsub_rn(hz, hc);
  const float tol = 4e-6f * (fabsf(dh) + fabsf(hc) + 1.f);
  int err = dx + dy, x = sx, y = sy;
  bool done = (x == ex && y == ey);
  while (!done) {
    int qx[4], qy[4];
    bool act[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      act[u] = false;
      qx[u] = qy[u] = 0;
      if (!done) {
        const int e2 = 2 * err;
        if (e2 >= dy) {
          err += dy;
          x += stx;
        }
        if (e2 <= dx) {
          err += dx;
          y += sty;
        }
        if (x == ex && y == ey) {
          done = true;
        } else {
          qx[u] = x;
          qy[u] = y;
          act[u] = true;
        }
      }
    }
    u32 fl[4];
    float hq[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const u32 q = base + phys(md, rx, ry, qx[u], qy[u]);
      fl[u] = act[u] ? md.flags[q] : 0u;
      hq[u] = act[u] ? __ldg(md.h + q) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (!act[u] || !(fl[u] & kFlagValid)) continue;
      const int num = (qx[u] - sx) * dxs + (qy[u] - sy) * dys;
      const float est = hq[u] - __fmaf_rn(__fmul_rn((float)num, rden), dh, hc);
      bool occ = est > 0.f;
      if (fabsf(est) <= tol + 4e-6f * fabsf(hq[u])) {  // near the ray: the exact sequence
        const float tq = __fdiv_rn((float)num, den);
        occ = hq[u] >= __fmaf_rn(tq, dh, hc);
      }
      if (occ) return false;
    }
  }
  return true;
}

// Fuse pixel p into cell g with the whole warp (lanes over channels).
__device__ __forceinline__ void fuse_pixel_warp(const MapDev& md, const ImgParams& ip, int64_t g,
                                                int64_t p, u32 fl) {
  const int lane = (threadIdx.x + threadIdx.y * blockDim.x) & 31;
  for (int q = 0; q < ip.n_src; ++q) {
    const SrcDev& s = ip.src[q];
    for (int b = 0; b < s.n_layers; ++b) {
      const int l = s.layers[b];
      const LayerDev& L = md.L[l];
      const bool obs = fl & (2u << l);
      if (L.rule == MEM_RULE_CLASSMAX) {
        float best = -INFINITY;
        int bid = 0x7fffffff;
        for (int c = lane; c < s.C; c += 32) {
          const float v = src_val(s, p, c);
          if (v > best) {
            best = v;
            bid = c;
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float ov = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bid, o);
          if (ov > best || (ov == best && oi < bid)) {
            best = ov;
            bid = oi;
          }
        }
        if (lane == 0) {
          float* d = (float*)L.data + g * 2;
          d[0] = best == -INFINITY ? -1.f : (float)bid;
          d[1] = best;
        }
      } else {
        const float s02 = (L.rule == MEM_RULE_GAUSS && obs) ? L.gvar[g] : 0.f;
        const RuleCoef co = rule_coef(L, 1.f, 1.f, obs, s02);
        for (int c = lane; c < s.C; c += 32) apply_rule(L, g * L.S + c, src_val(s, p, c), co);
        if (L.rule == MEM_RULE_GAUSS) {
          __syncwarp();
          if (lane == 0) L.gvar[g] = co.var_new;
        }
      }
      __syncwarp();
    }
    for (int b = 0; b < s.n_layers; ++b) fl |= 2u << s.layers[b];
  }
  if (lane == 0) md.flags[g] = fl;
}

// A block takes a 16 x 16 tile of cells: every thread projects its cell, the
// cells that are valid, in front of the camera and inside the image are listed
// in shared memory, and consecutive threads walk the listed cells' lines (the
// others are done); each warp then fuses its visible cells' pixels.
__global__ void __launch_bounds__(256) k_image(MapDev md, ImgParams ip, uint8_t* __restrict__ vis,
                                               int32_t* __restrict__ pix) {
  const int W = md.W;
  const int tid = threadIdx.y * 16 + threadIdx.x;
  const u32 base = (u32)ip.map_index * md.W2;
  __shared__ int s_n;
  __shared__ u32 s_cell[256];
  __shared__ float s_hz[256];
  __shared__ int32_t s_pix[256];
  if (tid == 0) s_n = 0;
  __syncthreads();
  {
    const int ix = blockIdx.x * 16 + threadIdx.x;
    const int iy = blockIdx.y * 16 + threadIdx.y;
    if (ix < W && iy < W) {
      const u32 g = base + phys(md, ip.ring_x, ip.ring_y, ix, iy);
      bool listed = false;
      if (md.flags[g] & kFlagValid) {
        const float xc = __fmul_rn(__fadd_rn((float)(ix - W / 2), 0.5f), md.res);
        const float yc = __fmul_rn(__fadd_rn((float)(iy - W / 2), 0.5f), md.res);
        const float hz = md.h[g];
        const float Xc = __fmaf_rn(ip.R[0], xc, __fmaf_rn(ip.R[1], yc, __fmaf_rn(ip.R[2], hz, ip.t[0])));
        const float Yc = __fmaf_rn(ip.R[3], xc, __fmaf_rn(ip.R[4], yc, __fmaf_rn(ip.R[5], hz, ip.t[1])));
        const float Zc = __fmaf_rn(ip.R[6], xc, __fmaf_rn(ip.R[7], yc, __fmaf_rn(ip.R[8], hz, ip.t[2])));
        if (Zc > md.z_near) {
          const float u = __fmaf_rn(ip.fx, __fdiv_rn(Xc, Zc), ip.cx);
          const float v = __fmaf_rn(ip.fy, __fdiv_rn(Yc, Zc), ip.cy);
          const float fu = floorf(__fadd_rn(u, 0.5f));
          const float fv = floorf(__fadd_rn(v, 0.5f));
          if (fu >= 0.f && fu < (float)ip.Wi && fv >= 0.f && fv < (float)ip.H) {
            const int k = atomicAdd(&s_n, 1);
            s_cell[k] = ((u32)iy << 16) | (u32)ix;
            s_hz[k] = hz;
            s_pix[k] = (int32_t)((int64_t)fv * ip.Wi + (int64_t)fu);
            listed = true;
          }
        }
      }
      if (!listed) {
        const int64_t j = (int64_t)iy * W + ix;
        if (vis) vis[j] = 0;
        if (pix) pix[j] = -1;
      }
    }
  }
  __syncthreads();
  const int n = s_n;
  __shared__ int s_nv;
  __shared__ u32 s_vg[256];
  __shared__ int32_t s_vp[256];
  if (tid == 0) s_nv = 0;
  __syncthreads();
  if (tid < n) {
    const int ix = (int)(s_cell[tid] & 0xffffu), iy = (int)(s_cell[tid] >> 16);
    const bool visible = walk_visible(md, base, ip.ring_x, ip.ring_y, ip.sx, ip.sy, ix, iy, s_hz[tid], ip.hc);
    const int64_t j = (int64_t)iy * W + ix;
    if (vis) vis[j] = visible ? 1 : 0;
    if (pix) pix[j] = visible ? s_pix[tid] : -1;
    if (visible && ip.n_src > 0) {
      const int k = atomicAdd(&s_nv, 1);
      s_vg[k] = base + phys(md, ip.ring_x, ip.ring_y, ix, iy);
      s_vp[k] = s_pix[tid];
    }
  }
  if (ip.n_src == 0) return;
  __syncthreads();
  // the visible cells dealt out to the block's warps, each fused by a whole warp
  const int warp = tid >> 5, nwarps = (blockDim.x * blockDim.y) >> 5;
  for (int v = warp; v < s_nv; v += nwarps) {
    const u32 gv = s_vg[v];
    fuse_pixel_warp(md, ip, gv, s_vp[v], md.flags[gv]);
  }
}

}  // namespace memk

namespace memh {
using namespace memk;

cudaError_t launch_image_fuse(Map* m, int map_index, const MapCall& mc, int H, int Wi, int n_src,
                              const SrcDev* src, const float K[4], uint8_t* vis, int32_t* pix,
                              cudaStream_t st) {
  const MapDev& md = m->md;
  ImgParams ip;
  for (int k = 0; k < 9; ++k) ip.R[k] = mc.R[k];
  for (int k = 0; k < 3; ++k) ip.t[k] = mc.t[k];
  ip.fx = K[0];
  ip.fy = K[1];
  ip.cx = K[2];
  ip.cy = K[3];
  // camera cell, clamped into the map; camera height
  const float res = md.res;
  const float half = (float)(md.W / 2);
  float qx = floorf(mc.cam_x / res), qy = floorf(mc.cam_y / res);
  if (!(qx >= -half)) qx = -half;
  if (!(qx <= half - 1.0f)) qx = half - 1.0f;
  if (!(qy >= -half)) qy = -half;
  if (!(qy <= half - 1.0f)) qy = half - 1.0f;
  ip.sx = (int)qx + md.W / 2;
  ip.sy = (int)qy + md.W / 2;
  ip.hc = mc.cam_h;
  ip.H = H;
  ip.Wi = Wi;
  ip.map_index = map_index;
  ip.ring_x = mc.ring_x;
  ip.ring_y = mc.ring_y;
  ip.n_src = n_src;
  for (int q = 0; q < n_src; ++q) ip.src[q] = src[q];
  dim3 blk(16, 16), grd((md.W + 15) / 16, (md.W + 15) / 16);
  ProfScope ps(m, kProfImage, st);
  k_image<<<grd, blk, 0, st>>>(md, ip, vis, pix);
  return cudaGetLastError();
}

}  // namespace memh
