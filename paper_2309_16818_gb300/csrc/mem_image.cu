// Image association and fusion (Sec. III-B, Fig. 2): every valid cell is
// projected at its elevation into a pinhole camera; a cell is visible iff
// every valid cell on the Bresenham line from the camera's cell to it lies
// strictly below the ray from the camera to the cell (equality occludes).
// Visible cells fuse their pixel with the layer rules (one observation).
//
// Three kernels: the cells that need a visibility walk are listed for the whole
// map; consecutive threads walk consecutive listed cells' lines (neighbouring
// cells, so neighbouring lines read neighbouring heights through L1) and list
// the visible cells; every warp of a grid that fills the GPU then fuses visible
// cells one at a time with its lanes spread over the channels, so pixel rows and
// layer rows are read and written coalesced and the cells' chains of dependent
// accesses run side by side.
#include "mem_host.h"

namespace memk {

// the cells an image call lists for a visibility walk, then its visible cells
// (capacity W * W each)
struct ImgList {
  u32* n;         // [0] listed cells, [1] visible cells
  u32* cell;      // listed: y << 16 | x
  float* hz;      // the cell's height
  int32_t* pix;   // its pixel
  u32* vg;        // visible: the cell's state index
  int32_t* vp;    // its pixel
};

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

// 1. Listing: a block takes a 16 x 16 tile of cells, every thread projects
// its cell; the cells that are valid, in front of the camera and inside the
// image are appended to one list for the whole map (a warp's cells together,
// so neighbouring cells stay neighbours in the list); the others are done.
__global__ void __launch_bounds__(256) k_image_list(MapDev md, ImgParams ip, ImgList li, uint8_t* __restrict__ vis,
                                                    int32_t* __restrict__ pix) {
  const int W = md.W;
  const u32 base = (u32)ip.map_index * md.W2;
  const int lane = (threadIdx.y * 16 + threadIdx.x) & 31;
  const int ix = blockIdx.x * 16 + threadIdx.x;
  const int iy = blockIdx.y * 16 + threadIdx.y;
  bool listed = false;
  float hz = 0.f;
  int32_t px = -1;
  if (ix < W && iy < W) {
    const u32 g = base + phys(md, ip.ring_x, ip.ring_y, ix, iy);
    if (md.flags[g] & kFlagValid) {
      const float xc = __fmul_rn(__fadd_rn((float)(ix - W / 2), 0.5f), md.res);
      const float yc = __fmul_rn(__fadd_rn((float)(iy - W / 2), 0.5f), md.res);
      hz = md.h[g];
      const float Xc = __fmaf_rn(ip.R[0], xc, __fmaf_rn(ip.R[1], yc, __fmaf_rn(ip.R[2], hz, ip.t[0])));
      const float Yc = __fmaf_rn(ip.R[3], xc, __fmaf_rn(ip.R[4], yc, __fmaf_rn(ip.R[5], hz, ip.t[1])));
      const float Zc = __fmaf_rn(ip.R[6], xc, __fmaf_rn(ip.R[7], yc, __fmaf_rn(ip.R[8], hz, ip.t[2])));
      if (Zc > md.z_near) {
        const float u = __fmaf_rn(ip.fx, __fdiv_rn(Xc, Zc), ip.cx);
        const float v = __fmaf_rn(ip.fy, __fdiv_rn(Yc, Zc), ip.cy);
        const float fu = floorf(__fadd_rn(u, 0.5f));
        const float fv = floorf(__fadd_rn(v, 0.5f));
        if (fu >= 0.f && fu < (float)ip.Wi && fv >= 0.f && fv < (float)ip.H) {
          listed = true;
          px = (int32_t)((int64_t)fv * ip.Wi + (int64_t)fu);
        }
      }
    }
    if (!listed) {
      const int64_t j = (int64_t)iy * W + ix;
      if (vis) vis[j] = 0;
      if (pix) pix[j] = -1;
    }
  }
  const u32 bal = __ballot_sync(0xffffffffu, listed);
  u32 k0 = 0;
  if (lane == 0 && bal) k0 = atomicAdd(li.n, (u32)__popc(bal));
  k0 = __shfl_sync(0xffffffffu, k0, 0);
  if (listed) {
    const u32 k = k0 + (u32)__popc(bal & ((1u << lane) - 1u));
    li.cell[k] = ((u32)iy << 16) | (u32)ix;
    li.hz[k] = hz;
    li.pix[k] = px;
  }
}

// 2. Visibility over the list: consecutive threads walk consecutive listed
// cells' lines (neighbouring cells, so neighbouring lines read neighbouring
// heights through L1); visible cells are appended to the second list.
__global__ void __launch_bounds__(256) k_image_walk(MapDev md, ImgParams ip, ImgList li, uint8_t* __restrict__ vis,
                                                    int32_t* __restrict__ pix) {
  const int W = md.W;
  const u32 base = (u32)ip.map_index * md.W2;
  const int n = (int)*li.n;
  const int lane = threadIdx.x & 31;
  for (int i0 = blockIdx.x * blockDim.x; i0 < n; i0 += gridDim.x * blockDim.x) {  // uniform per warp
    const int i = i0 + threadIdx.x;
    bool visible = false;
    int32_t px = -1;
    u32 gv = 0;
    if (i < n) {
      const u32 c = li.cell[i];
      const int ix = (int)(c & 0xffffu), iy = (int)(c >> 16);
      px = li.pix[i];
      visible = walk_visible(md, base, ip.ring_x, ip.ring_y, ip.sx, ip.sy, ix, iy, li.hz[i], ip.hc);
      const int64_t j = (int64_t)iy * W + ix;
      if (vis) vis[j] = visible ? 1 : 0;
      if (pix) pix[j] = visible ? px : -1;
      gv = base + phys(md, ip.ring_x, ip.ring_y, ix, iy);
    }
    const u32 bal = __ballot_sync(0xffffffffu, visible);
    u32 k0 = 0;
    if (lane == 0 && bal) k0 = atomicAdd(li.n + 1, (u32)__popc(bal));
    k0 = __shfl_sync(0xffffffffu, k0, 0);
    if (visible) {
      const u32 k = k0 + (u32)__popc(bal & ((1u << lane) - 1u));
      li.vg[k] = gv;
      li.vp[k] = px;
    }
  }
}

// 3. Fusion: every warp of the grid takes visible cells in turn and fuses each
// with its lanes spread over the channels (pixel rows and layer rows read and
// written coalesced). Each cell is fused on its own, so the lists' order does
// not change a result.
__global__ void __launch_bounds__(128) k_image_fuse(MapDev md, ImgParams ip, ImgList li) {
  const int nv = (int)li.n[1];
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < nv; v += nwarps) {
    const u32 gv = li.vg[v];
    fuse_pixel_warp(md, ip, gv, li.vp[v], md.flags[gv]);
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
  // the list (one map's cells at most), allocated on the first call
  const size_t need = sizeof(u32) * (4 + 5 * (size_t)md.W2);
  if (need > m->img_cap) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    if (m->img_buf) cudaFree(m->img_buf);
    m->img_buf = nullptr;
    m->img_cap = 0;
    e = cudaMalloc(&m->img_buf, need);
    if (e != cudaSuccess) return e;
    m->img_cap = need;
  }
  ImgList li;
  li.n = (u32*)m->img_buf;
  li.cell = li.n + 4;
  li.hz = (float*)(li.cell + md.W2);
  li.pix = (int32_t*)(li.hz + md.W2);
  li.vg = (u32*)(li.pix + md.W2);
  li.vp = (int32_t*)(li.vg + md.W2);
  ProfScope ps(m, kProfImage, st);
  cudaError_t e = cudaMemsetAsync(li.n, 0, 2 * sizeof(u32), st);
  if (e != cudaSuccess) return e;
  dim3 blk(16, 16), grd((md.W + 15) / 16, (md.W + 15) / 16);
  k_image_list<<<grd, blk, 0, st>>>(md, ip, li, vis, pix);
  k_image_walk<<<m->n_sm * 8, 128, 0, st>>>(md, ip, li, vis, pix);
  if (n_src > 0) k_image_fuse<<<m->n_sm * 16, 128, 0, st>>>(md, ip, li);
  return cudaGetLastError();
}

}  // namespace memh
