// Image association and fusion (Sec. III-B, Fig. 2): every valid cell is
// projected at its elevation into a pinhole camera; a cell is visible iff
// every valid cell on the Bresenham line from the camera's cell to it lies
// strictly below the ray from the camera to the cell (equality occludes).
// Visible cells fuse their pixel with the layer rules (one observation).
//
// One thread per cell walks its own line (16x16 cell tiles, so neighbouring
// threads read neighbouring heights through L1); the warp then fuses the
// visible cells one at a time with its lanes spread over the channels, so
// pixel rows and layer rows are read and written coalesced.
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
__device__ __forceinline__ bool walk_visible(const MapDev& md, u32 base, int rx, int ry, int sx, int sy,
                                             int ex, int ey, float hz, float hc) {
  const int dx = abs(ex - sx), dy = -abs(ey - sy);
  const int stx = sx < ex ? 1 : -1, sty = sy < ey ? 1 : -1;
  const int dxs = ex - sx, dys = ey - sy;
  const float den = (float)(dxs * dxs + dys * dys);
  const float dh = __fsub_rn(hz, hc);
  int err = dx + dy, x = sx, y = sy;
  if (x == ex && y == ey) return true;
  for (;;) {
    const int e2 = 2 * err;
    if (e2 >= dy) {
      err += dy;
      x += stx;
    }
    if (e2 <= dx) {
      err += dx;
      y += sty;
    }
    if (x == ex && y == ey) return true;
    const u32 q = base + phys(md, rx, ry, x, y);
    if (__ldg(md.flags + q) & kFlagValid) {
      const int num = (x - sx) * dxs + (y - sy) * dys;
      const float tq = __fdiv_rn((float)num, den);
      const float ray = __fmaf_rn(tq, dh, hc);
      if (__ldg(md.h + q) >= ray) return false;
    }
  }
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

__global__ void __launch_bounds__(256) k_image(MapDev md, ImgParams ip, uint8_t* __restrict__ vis,
                                               int32_t* __restrict__ pix) {
  const int W = md.W;
  const int ix = blockIdx.x * 16 + threadIdx.x;
  const int iy = blockIdx.y * 16 + threadIdx.y;
  const bool inside = ix < W && iy < W;
  const u32 base = (u32)ip.map_index * md.W2;
  bool visible = false;
  int64_t g = 0, p = -1;
  u32 fl = 0;
  if (inside) {
    g = base + phys(md, ip.ring_x, ip.ring_y, ix, iy);
    fl = md.flags[g];
    if (fl & kFlagValid) {
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
          visible = walk_visible(md, base, ip.ring_x, ip.ring_y, ip.sx, ip.sy, ix, iy, hz, ip.hc);
          if (visible) p = (int64_t)fv * ip.Wi + (int64_t)fu;
        }
      }
    }
    const int64_t j = (int64_t)iy * W + ix;
    if (vis) vis[j] = visible ? 1 : 0;
    if (pix) pix[j] = visible ? (int32_t)p : -1;
  }
  if (ip.n_src == 0) return;
  u32 m = __ballot_sync(0xffffffffu, visible);
  while (m) {
    const int v = __ffs(m) - 1;
    m &= m - 1;
    const int64_t gv = __shfl_sync(0xffffffffu, g, v);
    const int64_t pv = __shfl_sync(0xffffffffu, p, v);
    const u32 flv = __shfl_sync(0xffffffffu, fl, v);
    fuse_pixel_warp(md, ip, gv, pv, flv);
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
