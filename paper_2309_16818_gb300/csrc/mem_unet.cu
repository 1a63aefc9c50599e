// Learned inpainting: a small U-Net trained and run with BF16 tensor-core
// kernels (float32 accumulation, float32 master weights, Adam).
//
// Layout: activations NHWC bf16. A 3x3 convolution is an implicit GEMM
// C[pixels, cout] = A[pixels, 9*cin] B[9*cin, cout]: every block stages the
// input halo of an 8 x 16 output tile (32 channels at a time) and a 32 x BN
// slice of the weights per tap in shared memory with cp.async (zero fill at
// the border), and its eight warps run m16n8k16 BF16 MMAs from ldmatrix
// fragments, all nine taps from one staged halo. The decoder's
// nearest-neighbour upsampling and channel concatenation are folded into
// that gather (two input tensors, the first at half resolution). The data
// gradient is the same kernel with flipped, transposed weights; the weight
// gradient is a GEMM over pixels split across blocks with float32 atomics.
#include <math.h>
#include <string.h>

#include <vector>

#include "mem_host.h"

typedef __nv_bfloat16 bf16;

namespace memk {

// ---------------------------------------------------------------------------
// tensor-core helpers (PTX)

__device__ __forceinline__ u32 smem_u32(const void* p) {
  return (u32)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const int n = valid ? 16 : 0;  // zero fill when not valid
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }

__device__ __forceinline__ void ldsm_x4(u32 r[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(u32 r[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma_bf16(float d[4], const u32 a[4], u32 b0, u32 b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------------------
// 3x3 convolution (forward, and data gradient with flipped weights)

struct ConvArgs {
  const bf16* in0;  // [N, H(/2), W(/2), c0]
  const bf16* in1;  // [N, H, W, c1] or null
  int c0, c1, up0;  // up0: in0 is at half resolution (nearest upsample)
  int cin_pad;      // rows of the weight matrix per tap (multiple of 32, >= c0 + c1)
  const bf16* w;    // [9][cin_pad][cout]
  const float* bias;
  bf16* out;        // [N, H, W, cout]
  int cout, N, H, W, relu;
};

// ---------------------------------------------------------------------------
// 3x3 convolution on halo tiles: a block computes an 8 x 16 tile of output
// pixels for BN output channels. For every 32-channel chunk of the input it
// stages the tile's (8 + 2) x (16 + 2) input halo once (zero outside the
// image; nearest upsampling and channel concatenation folded into the
// gather), then runs the nine taps from it, streaming the weights of one
// (chunk, tap) at a time; halo and weights are double-buffered with
// cp.async. Eight warps: 4 along pixels (32 each) x 2 along channels.

constexpr int kTH = 8, kTW = 16;                  // output tile
constexpr int kHH = kTH + 2, kHW = kTW + 2;       // halo tile
constexpr int kHS = 40;                           // bf16 per halo pixel (32 + 8: conflict-free ldmatrix)

template <int BN>
__global__ void __launch_bounds__(256) k_conv3x3h(ConvArgs a) {
  constexpr int kBpad = BN + 8;
  __shared__ __align__(16) bf16 Hs[2][kHH * kHW * kHS];
  __shared__ __align__(16) bf16 Bs[2][32][kBpad];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;
  const int tx = (a.W + kTW - 1) / kTW, ty = (a.H + kTH - 1) / kTH;
  int b = blockIdx.x;
  const int n = b / (tx * ty);
  b -= n * tx * ty;
  const int y0 = (b / tx) * kTH, x0 = (b % tx) * kTW;
  const int n0 = blockIdx.y * BN;
  const int kchunks = a.cin_pad / 32;
  const int S = kchunks * 9;
  auto stage_halo = [&](int c, int buf) {
    const int cb = c * 32;
    for (int i = tid; i < kHH * kHW * 4; i += 256) {
      const int hp = i >> 2, ck = i & 3;
      const int hy = hp / kHW, hx = hp - hy * kHW;
      const int yy = y0 + hy - 1, xx = x0 + hx - 1;
      const int ci = cb + 8 * ck;
      const bool ok = yy >= 0 && yy < a.H && xx >= 0 && xx < a.W && ci < a.c0 + a.c1;
      const bf16* src = a.in0;
      if (ok) {
        if (ci < a.c0) {
          if (a.up0) src = a.in0 + (((int64_t)n * (a.H >> 1) + (yy >> 1)) * (a.W >> 1) + (xx >> 1)) * a.c0 + ci;
          else src = a.in0 + (((int64_t)n * a.H + yy) * a.W + xx) * a.c0 + ci;
        } else {
          src = a.in1 + (((int64_t)n * a.H + yy) * a.W + xx) * a.c1 + (ci - a.c0);
        }
      }
      cp_async16(&Hs[buf][hp * kHS + 8 * ck], src, ok);
    }
  };
  auto stage_w = [&](int c, int t, int buf) {
    constexpr int CPR = BN / 8;
    for (int i = tid; i < 32 * CPR; i += 256) {
      const int r = i / CPR, cc = i - r * CPR;
      cp_async16(&Bs[buf][r][8 * cc], a.w + ((int64_t)(t * a.cin_pad + c * 32 + r) * a.cout + n0 + 8 * cc), true);
    }
  };
  constexpr int NT = BN / 16;
  float acc[2][NT][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.f;
  stage_halo(0, 0);
  stage_w(0, 0, 0);
  cp_async_commit();
  for (int st = 0; st < S; ++st) {
    const int c = st / 9, t = st - c * 9;
    if (st + 1 < S) {
      const int c1 = (st + 1) / 9, t1 = st + 1 - c1 * 9;
      stage_w(c1, t1, (st + 1) & 1);
      if (t1 == 0) stage_halo(c1, c1 & 1);
      cp_async_commit();
      cp_async_wait1();
    } else {
      cp_async_wait0();
    }
    __syncthreads();
    const bf16* H = Hs[c & 1];
    const int dy = t / 3, dx = t - dy * 3;  // halo offset of the tap
#pragma unroll
    for (int kk = 0; kk < 32; kk += 16) {
      u32 af[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int pp = wm * 32 + mt * 16 + (lane & 15);  // output pixel of this ldmatrix row
        const int hp = ((pp >> 4) + dy) * kHW + (pp & 15) + dx;
        ldsm_x4(af[mt], &H[hp * kHS + kk + (lane >> 4) * 8]);
      }
#pragma unroll
      for (int np = 0; np < NT / 2; ++np) {
        u32 bfr[4];
        ldsm_x4_t(bfr, &Bs[st & 1][kk + (lane & 7) + ((lane >> 3) & 1) * 8][wn * (BN / 2) + np * 16 + (lane >> 4) * 8]);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          mma_bf16(acc[mt][2 * np], af[mt], bfr[0], bfr[1]);
          mma_bf16(acc[mt][2 * np + 1], af[mt], bfr[2], bfr[3]);
        }
      }
    }
    __syncthreads();
  }
  // epilogue: bias, ReLU, bf16 pairs
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int pp = wm * 32 + mt * 16 + (lane >> 2) + 8 * h;
      const int yy = y0 + (pp >> 4), xx = x0 + (pp & 15);
      if (yy >= a.H || xx >= a.W) continue;
      bf16* o = a.out + (((int64_t)n * a.H + yy) * a.W + xx) * a.cout;
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int co = n0 + wn * (BN / 2) + nt * 8 + (lane & 3) * 2;
        float v0 = acc[mt][nt][2 * h], v1 = acc[mt][nt][2 * h + 1];
        if (a.bias) {
          v0 += a.bias[co];
          v1 += a.bias[co + 1];
        }
        if (a.relu) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        *reinterpret_cast<__nv_bfloat162*>(o + co) = __floats2bfloat162_rn(v0, v1);
      }
    }
}

// ---------------------------------------------------------------------------
// weight gradient: dW[t][ci][co] += sum_p A[p, (t, ci)] dY[p, co]

struct WgradArgs {
  const bf16* in0;
  const bf16* in1;
  int c0, c1, up0, cin_pad;
  const bf16* dy;  // [P, cout]
  float* dw;       // [9][cin_pad][cout] float32
  int cout, N, H, W;
  int64_t pix_per_split;
};

template <int BN>
__global__ void __launch_bounds__(128) k_wgrad3x3(WgradArgs a) {
  constexpr int kBpad = BN + 8;
  __shared__ __align__(16) bf16 Xs[2][32][40];      // [pixel][ci]
  __shared__ __align__(16) bf16 Ds[2][32][kBpad];   // [pixel][co]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;  // warp tile: 16 ci x BN/2 co
  const int kchunks = a.cin_pad / 32;
  const int t = blockIdx.y / kchunks, cb = (blockIdx.y - t * kchunks) * 32;
  const int n0 = blockIdx.z * BN;
  const int dy = t / 3 - 1, dx = t % 3 - 1;
  const int64_t P = (int64_t)a.N * a.H * a.W;
  const int64_t p_begin = (int64_t)blockIdx.x * a.pix_per_split;
  const int64_t p_end = min(P, p_begin + a.pix_per_split);
  const int HW = a.H * a.W;
  constexpr int NT = BN / 16;
  float acc[NT][4];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  auto stage = [&](int64_t pb, int buf) {
    // X: 32 pixels x 32 channels = 128 chunks, one per thread
    {
      const int r = tid >> 2, ck = tid & 3;
      const int64_t p = pb + r;
      bool ok = p < p_end;
      const int64_t pp = ok ? p : 0;
      const int n = (int)(pp / HW);
      const int rem = (int)(pp - (int64_t)n * HW);
      const int yy = rem / a.W + dy, xx = rem % a.W + dx;
      const int ci = cb + 8 * ck;
      ok = ok && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W && ci < a.c0 + a.c1;
      const bf16* src = a.in0;
      if (ok) {
        if (ci < a.c0) {
          if (a.up0) {
            const int Hh = a.H >> 1, Wh = a.W >> 1;
            src = a.in0 + (((int64_t)n * Hh + (yy >> 1)) * Wh + (xx >> 1)) * a.c0 + ci;
          } else {
            src = a.in0 + (((int64_t)n * a.H + yy) * a.W + xx) * a.c0 + ci;
          }
        } else {
          src = a.in1 + (((int64_t)n * a.H + yy) * a.W + xx) * a.c1 + (ci - a.c0);
        }
      }
      cp_async16(&Xs[buf][r][8 * ck], src, ok);
    }
    // dY: 32 pixels x BN channels
    constexpr int CPR = BN / 8;
#pragma unroll
    for (int i = 0; i < (32 * CPR) / 128; ++i) {
      const int c = tid + 128 * i;
      const int r = c / CPR, cc = c - r * CPR;
      const int64_t p = pb + r;
      const bool ok = p < p_end;
      cp_async16(&Ds[buf][r][8 * cc], a.dy + (ok ? p : 0) * a.cout + n0 + 8 * cc, ok);
    }
    cp_async_commit();
  };
  if (p_begin < p_end) {
    stage(p_begin, 0);
    int buf = 0;
    for (int64_t pb = p_begin; pb < p_end; pb += 32) {
      if (pb + 32 < p_end) {
        stage(pb + 32, buf ^ 1);
        cp_async_wait1();
      } else {
        cp_async_wait0();
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < 32; kk += 16) {
        // A = X^T: rows ci, columns pixels -> transposed load of the [pixel][ci] tile
        u32 af[4];
        ldsm_x4_t(af, &Xs[buf][kk + (lane & 7) + (lane >> 4) * 8][wm * 16 + ((lane >> 3) & 1) * 8]);
#pragma unroll
        for (int np = 0; np < NT / 2; ++np) {
          u32 bfr[4];
          ldsm_x4_t(bfr, &Ds[buf][kk + (lane & 7) + ((lane >> 3) & 1) * 8][wn * (BN / 2) + np * 16 + (lane >> 4) * 8]);
          mma_bf16(acc[2 * np], af, bfr[0], bfr[1]);
          mma_bf16(acc[2 * np + 1], af, bfr[2], bfr[3]);
        }
      }
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int ci = cb + wm * 16 + (lane >> 2) + 8 * h;
      const int co = n0 + wn * (BN / 2) + nt * 8 + (lane & 3) * 2;
      float* d = a.dw + ((int64_t)(t * a.cin_pad + ci) * a.cout + co);
      atomicAdd(d, acc[nt][2 * h]);
      atomicAdd(d + 1, acc[nt][2 * h + 1]);
    }
}

// ---------------------------------------------------------------------------
// element-wise pieces

// 2x2 max pooling (NHWC)
__global__ void k_maxpool(const bf16* __restrict__ x, bf16* __restrict__ y, int N, int H, int W, int C) {
  const int Ho = H / 2, Wo = W / 2;
  const int64_t total = (int64_t)N * Ho * Wo * C;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    int64_t r = i / C;
    const int xo = (int)(r % Wo);
    r /= Wo;
    const int yo = (int)(r % Ho);
    const int n = (int)(r / Ho);
    const bf16* p = x + (((int64_t)n * H + 2 * yo) * W + 2 * xo) * C + c;
    const float a = __bfloat162float(p[0]), b = __bfloat162float(p[C]);
    const float d = __bfloat162float(p[(int64_t)W * C]), e = __bfloat162float(p[(int64_t)W * C + C]);
    y[i] = __float2bfloat16_rn(fmaxf(fmaxf(a, b), fmaxf(d, e)));
  }
}

// gradient of 2x2 max pooling to the first maximum of each window (row-major),
// added to `acc` (the gradient that reached the same tensor through the skip)
__global__ void k_maxpool_bwd(const bf16* __restrict__ x, const bf16* __restrict__ dy, bf16* __restrict__ acc,
                              int N, int H, int W, int C) {
  const int Ho = H / 2, Wo = W / 2;
  const int64_t total = (int64_t)N * Ho * Wo * C;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    int64_t r = i / C;
    const int xo = (int)(r % Wo);
    r /= Wo;
    const int yo = (int)(r % Ho);
    const int n = (int)(r / Ho);
    const int64_t base = (((int64_t)n * H + 2 * yo) * W + 2 * xo) * C + c;
    const int64_t off[4] = {0, C, (int64_t)W * C, (int64_t)W * C + C};
    int am = 0;
    float best = __bfloat162float(x[base]);
    for (int k = 1; k < 4; ++k) {
      const float v = __bfloat162float(x[base + off[k]]);
      if (v > best) {
        best = v;
        am = k;
      }
    }
    const float g = __bfloat162float(dy[i]);
    for (int k = 0; k < 4; ++k) {
      const float prev = __bfloat162float(acc[base + off[k]]);
      acc[base + off[k]] = __float2bfloat16_rn(prev + (k == am ? g : 0.f));
    }
  }
}

// ReLU gradient in place: dy *= (y > 0)
__global__ void k_relu_bwd(const bf16* __restrict__ y, bf16* __restrict__ dy, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!(__bfloat162float(y[i]) > 0.f)) dy[i] = __float2bfloat16_rn(0.f);
}

// gradient of concat([upsample(low), skip]): low gets the 2x2 sums of the
// first c_up channels, skip the remaining channels
__global__ void k_split_cat_bwd(const bf16* __restrict__ dcat, bf16* __restrict__ dlow,
                                bf16* __restrict__ dskip, int N, int H, int W, int c_up, int c_skip) {
  const int Ho = H / 2, Wo = W / 2;
  const int C = c_up + c_skip;
  const int64_t tl = (int64_t)N * Ho * Wo * c_up;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tl; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % c_up);
    int64_t r = i / c_up;
    const int xo = (int)(r % Wo);
    r /= Wo;
    const int yo = (int)(r % Ho);
    const int n = (int)(r / Ho);
    const int64_t b = (((int64_t)n * H + 2 * yo) * W + 2 * xo) * C + c;
    const float s = __bfloat162float(dcat[b]) + __bfloat162float(dcat[b + C]) +
                    __bfloat162float(dcat[b + (int64_t)W * C]) + __bfloat162float(dcat[b + (int64_t)W * C + C]);
    dlow[i] = __float2bfloat16_rn(s);
  }
  const int64_t ts = (int64_t)N * H * W * c_skip;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ts; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % c_skip);
    const int64_t p = i / c_skip;
    dskip[i] = dcat[p * C + c_up + c];
  }
}

// bias gradient: db[c] += sum over pixels of dy[p][c]
__global__ void k_bias_grad(const bf16* __restrict__ dy, float* __restrict__ db, int64_t P, int C) {
  const int c = threadIdx.x % C, lanes = blockDim.x / C;
  const int sub = threadIdx.x / C;
  if (sub >= lanes) return;
  float s = 0.f;
  for (int64_t p = (int64_t)blockIdx.x * lanes + sub; p < P; p += (int64_t)gridDim.x * lanes)
    s += __bfloat162float(dy[p * C + c]);
  atomicAdd(&db[c], s);
}

// final 1x1 convolution (residual over the diffusion fill), masked-MSE loss and
// its gradients: res = b + d1 . w ; pred = fill + res
__global__ void k_head(const bf16* __restrict__ d1, int C, const float* __restrict__ w, const float* __restrict__ b,
                       const float* __restrict__ fill, float* __restrict__ pred, const float* __restrict__ target,
                       const uint8_t* __restrict__ hidden, float inv_cnt, int64_t P, float* __restrict__ loss,
                       bf16* __restrict__ dd1, float* __restrict__ dw, float* __restrict__ dbias) {
  __shared__ float s_w[256], s_dw[256];
  __shared__ float s_loss, s_db;
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    s_w[c] = w[c];
    s_dw[c] = 0.f;
  }
  if (threadIdx.x == 0) s_loss = s_db = 0.f;
  __syncthreads();
  float l = 0.f, gb = 0.f;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    float r = b[0];
    for (int c = 0; c < C; ++c) r = fmaf(__bfloat162float(d1[p * C + c]), s_w[c], r);
    const float pr = fill[p] + r;
    if (pred) pred[p] = pr;
    if (target) {
      const float diff = hidden[p] ? pr - target[p] : 0.f;
      l += diff * diff;
      const float g = 2.f * diff * inv_cnt;
      gb += g;
      for (int c = 0; c < C; ++c) {
        dd1[p * C + c] = __float2bfloat16_rn(g * s_w[c]);
        atomicAdd(&s_dw[c], g * __bfloat162float(d1[p * C + c]));
      }
    }
  }
  if (target) {
    atomicAdd(&s_loss, l * inv_cnt);
    atomicAdd(&s_db, gb);
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) atomicAdd(&dw[c], s_dw[c]);
    if (threadIdx.x == 0) {
      atomicAdd(loss, s_loss);
      atomicAdd(dbias, s_db);
    }
  }
}

// float32 master weights [3][3][cin][cout] -> bf16 forward copy [9][cin_pad][cout]
// and (optionally) the data-gradient copy [9][cout_pad][cin] with flipped taps
__global__ void k_prep_weights(const float* __restrict__ w, int cin, int cout, int cin_pad, bf16* __restrict__ wf,
                               bf16* __restrict__ wd, int cout_pad, int cin_out) {
  const int64_t nf = 9LL * cin_pad * cout;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    const int co = (int)(i % cout);
    const int64_t r = i / cout;
    const int ci = (int)(r % cin_pad), t = (int)(r / cin_pad);
    wf[i] = __float2bfloat16_rn(ci < cin ? w[((int64_t)t * cin + ci) * cout + co] : 0.f);
  }
  if (!wd) return;
  const int64_t nd = 9LL * cout_pad * cin_out;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nd; i += (int64_t)gridDim.x * blockDim.x) {
    const int ci = (int)(i % cin_out);
    const int64_t r = i / cin_out;
    const int co = (int)(r % cout_pad), t = (int)(r / cout_pad);
    const int tf = 8 - t;
    wd[i] = __float2bfloat16_rn((co < cout && ci < cin) ? w[((int64_t)tf * cin + ci) * cout + co] : 0.f);
  }
}

// Adam on float32 parameters
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// [9][cin_pad][cout] -> [9][cin][cout]
__global__ void k_unpad_rows(const float* __restrict__ src, float* __restrict__ dst, int cin, int cin_pad, int cout) {
  const int64_t n = 9LL * cin * cout;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int co = (int)(i % cout);
    const int64_t r = i / cout;
    const int ci = (int)(r % cin), t = (int)(r / cin);
    dst[i] = src[((int64_t)t * cin_pad + ci) * cout + co];
  }
}

// input packing: 3 float32 channels [P][3] -> bf16 [P][16] (zero padded)
__global__ void k_pack_input(const float* __restrict__ x3, bf16* __restrict__ x16, int64_t P) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P * 16; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i & 15);
    x16[i] = __float2bfloat16_rn(c < 3 ? x3[(i >> 4) * 3 + c] : 0.f);
  }
}

}  // namespace memk

// ---------------------------------------------------------------------------
// host: the network object

namespace {
using namespace memk;

struct ConvLayer {
  int cin, cout;          // cin = c0 + c1 (real channels)
  int c0, c1, up0;        // input composition
  int cin_pad, cout_pad;  // padded to 32
  int level;              // resolution level (0 = full)
  size_t w_off, b_off;    // offsets in the flat float32 parameter vector
  bf16 *wf = nullptr, *wd = nullptr;
};

}  // namespace

struct mem_unet {
  int cin, widths[4];
  std::vector<ConvLayer> L;  // 14 3x3 convolutions
  size_t n_params = 0, head_w = 0, head_b = 0;
  float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
  int64_t adam_t = 0;
  // activations for the current batch size
  int N = 0, H = 0, W = 0;
  std::vector<void*> bufs;
  bf16* x16 = nullptr;
  bf16* act[14] = {};     // conv outputs (post-ReLU)
  bf16* pool[3] = {};     // pooled e1, e2, e3
  bf16* dact[14] = {};    // gradient of each conv output (reused as the pre-ReLU gradient)
  bf16* dcat = nullptr;   // gradient of a concatenated decoder input
  bf16* dpool[3] = {};    // gradient of the pooled tensors
  float* d_loss = nullptr;
  float* g0pad = nullptr;  // weight gradient of the first layer with padded input channels
  int n_sm = 148;
};

namespace {

int pad32(int c) { return (c + 31) / 32 * 32; }

cudaError_t ensure_acts(mem_unet* u, int N, int H, int W) {
  if (u->N >= N && u->H == H && u->W == W && u->x16) return cudaSuccess;
  for (void* p : u->bufs) cudaFree(p);
  u->bufs.clear();
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) return nullptr;
    u->bufs.push_back(p);
    return p;
  };
  const int64_t P = (int64_t)N * H * W;
  u->x16 = (bf16*)alloc(P * 16 * 2);
  int64_t maxcat = 0;
  for (size_t i = 0; i < u->L.size(); ++i) {
    const ConvLayer& c = u->L[i];
    const int64_t Pl = P >> (2 * c.level);
    u->act[i] = (bf16*)alloc(Pl * c.cout * 2);
    u->dact[i] = (bf16*)alloc(Pl * c.cout * 2);
    if (c.c1) maxcat = std::max<int64_t>(maxcat, Pl * c.cin);
    if (!u->act[i] || !u->dact[i]) return cudaErrorMemoryAllocation;
  }
  for (int l = 0; l < 3; ++l) {
    u->pool[l] = (bf16*)alloc((P >> (2 * (l + 1))) * u->widths[l] * 2);
    u->dpool[l] = (bf16*)alloc((P >> (2 * (l + 1))) * u->widths[l] * 2);
  }
  u->dcat = (bf16*)alloc(maxcat * 2);
  u->d_loss = (float*)alloc(4);
  if (!u->x16 || !u->dcat || !u->d_loss) return cudaErrorMemoryAllocation;
  u->N = N;
  u->H = H;
  u->W = W;
  return cudaSuccess;
}

int grid_for(int64_t n, int n_sm) {
  int64_t b = (n + 255) / 256;
  const int64_t cap = (int64_t)n_sm * 16;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

cudaError_t conv(mem_unet* u, const ConvLayer& c, const bf16* in0, const bf16* in1, const bf16* w,
                 const float* bias, bf16* out, int cout, int cin_pad, int c0, int c1, int up0, int N, int H,
                 int W, int relu, cudaStream_t st) {
  ConvArgs a;
  a.in0 = in0;
  a.in1 = in1;
  a.c0 = c0;
  a.c1 = c1;
  a.up0 = up0;
  a.cin_pad = cin_pad;
  a.w = w;
  a.bias = bias;
  a.out = out;
  a.cout = cout;
  a.N = N;
  a.H = H;
  a.W = W;
  a.relu = relu;
  (void)c;
  if (cout % 32 != 0 || cin_pad % 32 != 0) return cudaErrorInvalidValue;
  const unsigned tiles = (unsigned)(N * ((H + kTH - 1) / kTH) * ((W + kTW - 1) / kTW));
  if (cout % 128 == 0) k_conv3x3h<128><<<dim3(tiles, cout / 128), 256, 0, st>>>(a);
  else if (cout % 64 == 0) k_conv3x3h<64><<<dim3(tiles, cout / 64), 256, 0, st>>>(a);
  else k_conv3x3h<32><<<dim3(tiles, cout / 32), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t wgrad(mem_unet* u, const ConvLayer& c, const bf16* in0, const bf16* in1, const bf16* dy,
                  float* dw_pad, int N, int H, int W, cudaStream_t st) {
  WgradArgs a;
  a.in0 = in0;
  a.in1 = in1;
  a.c0 = c.c0;
  a.c1 = c.c1;
  a.up0 = c.up0;
  a.cin_pad = c.cin_pad;
  a.dy = dy;
  a.dw = dw_pad;
  a.cout = c.cout;
  a.N = N;
  a.H = H;
  a.W = W;
  const int64_t P = (int64_t)N * H * W;
  const int blocks_yz = 9 * (c.cin_pad / 32) * (c.cout / (c.cout % 64 == 0 ? 64 : 32));
  int64_t splits = ((int64_t)u->n_sm * 8 + blocks_yz - 1) / blocks_yz;
  if (splits < 1) splits = 1;
  int64_t per = (P + splits - 1) / splits;
  per = (per + 31) / 32 * 32;
  splits = (P + per - 1) / per;
  a.pix_per_split = per;
  if (c.cout % 64 == 0) {
    dim3 g((unsigned)splits, 9 * (c.cin_pad / 32), c.cout / 64);
    k_wgrad3x3<64><<<g, 128, 0, st>>>(a);
  } else {
    dim3 g((unsigned)splits, 9 * (c.cin_pad / 32), c.cout / 32);
    k_wgrad3x3<32><<<g, 128, 0, st>>>(a);
  }
  return cudaGetLastError();
}

// layer inputs in execution order: e1a e1b e2a e2b e3a e3b e4a e4b d3a d3b d2a d2b d1a d1b
const bf16* input0(mem_unet* u, int i) {
  switch (i) {
    case 0: return u->x16;
    case 2: return u->pool[0];
    case 4: return u->pool[1];
    case 6: return u->pool[2];
    case 8: return u->act[7];
    case 10: return u->act[9];
    case 12: return u->act[11];
    default: return u->act[i - 1];
  }
}
const bf16* input1(mem_unet* u, int i) {
  switch (i) {
    case 8: return u->act[5];
    case 10: return u->act[3];
    case 12: return u->act[1];
    default: return nullptr;
  }
}

cudaError_t prep_weights(mem_unet* u, cudaStream_t st) {
  for (size_t i = 0; i < u->L.size(); ++i) {
    ConvLayer& c = u->L[i];
    k_prep_weights<<<grid_for(9LL * c.cin_pad * c.cout, u->n_sm), 256, 0, st>>>(
        u->params + c.w_off, c.cin, c.cout, c.cin_pad, c.wf, i == 0 ? nullptr : c.wd, c.cout_pad, c.cin);
  }
  return cudaGetLastError();
}

cudaError_t forward(mem_unet* u, int N, int H, int W, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < u->L.size() && e == cudaSuccess; ++i) {
    const ConvLayer& c = u->L[i];
    const int l = c.level;
    const int Hl = H >> l, Wl = W >> l;
    const int c0 = i == 0 ? 16 : c.c0;
    e = conv(u, c, input0(u, (int)i), input1(u, (int)i), c.wf, u->params + c.b_off, u->act[i], c.cout, c.cin_pad,
             c0, c.c1, c.up0, N, Hl, Wl, 1, st);
    if (i == 1 || i == 3 || i == 5) {  // pool the end of encoder levels 1..3
      const int lv = (int)i / 2;
      k_maxpool<<<grid_for((int64_t)N * (Hl / 2) * (Wl / 2) * c.cout, u->n_sm), 256, 0, st>>>(
          u->act[i], u->pool[lv], N, Hl, Wl, c.cout);
    }
  }
  return e == cudaSuccess ? cudaGetLastError() : e;
}

cudaError_t backward(mem_unet* u, int N, int H, int W, cudaStream_t st) {
  // u->dact[13] holds d loss / d d1 (post-ReLU); grads zeroed except the head's
  for (int i = 13; i >= 0; --i) {
    const ConvLayer& c = u->L[i];
    const int l = c.level;
    const int Hl = H >> l, Wl = W >> l;
    const int64_t Pl = (int64_t)N * Hl * Wl;
    k_relu_bwd<<<grid_for(Pl * c.cout, u->n_sm), 256, 0, st>>>(u->act[i], u->dact[i], Pl * c.cout);
    const int c0 = i == 0 ? 16 : c.c0;
    ConvLayer cc = c;
    cc.c0 = c0;
    float* dw = i == 0 ? u->g0pad : u->grads + c.w_off;  // only the first layer has padded rows
    if (i == 0) cudaMemsetAsync(u->g0pad, 0, 9ull * c.cin_pad * c.cout * 4, st);
    cudaError_t e = wgrad(u, cc, input0(u, i), input1(u, i), u->dact[i], dw, N, Hl, Wl, st);
    if (e != cudaSuccess) return e;
    if (i == 0)
      k_unpad_rows<<<grid_for(9LL * c.cin * c.cout, u->n_sm), 256, 0, st>>>(u->g0pad, u->grads + c.w_off, c.cin,
                                                                            c.cin_pad, c.cout);
    // bias gradient
    {
      const int lanes = 256 / c.cout;
      k_bias_grad<<<grid_for(Pl / lanes + 1, u->n_sm), lanes * c.cout, 0, st>>>(u->dact[i], u->grads + c.b_off, Pl,
                                                                                 c.cout);
    }
    if (i == 0) break;
    // data gradient into the layer input
    if (c.c1) {  // decoder concat input: d(concat) then split
      e = conv(u, c, u->dact[i], nullptr, c.wd, nullptr, u->dcat, c.cin, c.cout_pad, c.cout, 0, 0, N, Hl, Wl, 0, st);
      if (e != cudaSuccess) return e;
      // low-resolution source gradient -> dact of the producing layer; skip -> dact of the skip layer
      const int lowi = i - 1, skipi = (i == 8) ? 5 : (i == 10 ? 3 : 1);
      k_split_cat_bwd<<<grid_for(Pl * c.cin, u->n_sm), 256, 0, st>>>(u->dcat, u->dact[lowi], u->dact[skipi], N, Hl, Wl,
                                                                      c.c0, c.c1);
    } else if (i == 2 || i == 4 || i == 6) {  // input is a pooled tensor
      const int lv = i / 2 - 1;
      e = conv(u, c, u->dact[i], nullptr, c.wd, nullptr, u->dpool[lv], c.cin, c.cout_pad, c.cout, 0, 0, N, Hl, Wl, 0,
               st);
      if (e != cudaSuccess) return e;
      // route through the pooling and add to the skip gradient already in dact[i - 1]
      const int src = i - 1;
      const ConvLayer& ps = u->L[src];
      k_maxpool_bwd<<<grid_for((int64_t)N * Hl * Wl * ps.cout, u->n_sm), 256, 0, st>>>(
          u->act[src], u->dpool[lv], u->dact[src], N, Hl * 2, Wl * 2, ps.cout);
    } else {
      e = conv(u, c, u->dact[i], nullptr, c.wd, nullptr, u->dact[i - 1], c.cin, c.cout_pad, c.cout, 0, 0, N, Hl, Wl,
               0, st);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

}  // namespace

extern "C" mem_status mem_unet_create(int32_t cin, const int32_t widths[4], mem_unet** out) {
  if (!out || !widths) return memh::api_fail(MEM_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (cin < 1 || cin > 16) return memh::api_fail(MEM_ERR_ARG, "cin in [1, 16]");
  for (int k = 0; k < 4; ++k)
    if (widths[k] < 32 || widths[k] > 256 || widths[k] % 32)
      return memh::api_fail(MEM_ERR_ARG, "widths must be multiples of 32 in [32, 256]");
  mem_unet* u = new mem_unet();
  u->cin = cin;
  for (int k = 0; k < 4; ++k) u->widths[k] = widths[k];
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&u->n_sm, cudaDevAttrMultiProcessorCount, dev);
  const int c1 = widths[0], c2 = widths[1], c3 = widths[2], c4 = widths[3];
  struct Spec {
    int c0, c1, cout, up0, level;
  } specs[14] = {{cin, 0, c1, 0, 0}, {c1, 0, c1, 0, 0}, {c1, 0, c2, 0, 1},      {c2, 0, c2, 0, 1},
                 {c2, 0, c3, 0, 2},  {c3, 0, c3, 0, 2}, {c3, 0, c4, 0, 3},      {c4, 0, c4, 0, 3},
                 {c4, c3, c3, 1, 2}, {c3, 0, c3, 0, 2}, {c3, c2, c2, 1, 1},     {c2, 0, c2, 0, 1},
                 {c2, c1, c1, 1, 0}, {c1, 0, c1, 0, 0}};
  size_t off = 0;
  for (int i = 0; i < 14; ++i) {
    ConvLayer c;
    c.c0 = specs[i].c0;
    c.c1 = specs[i].c1;
    c.cin = c.c0 + c.c1;
    c.cout = specs[i].cout;
    c.up0 = specs[i].up0;
    c.level = specs[i].level;
    c.cin_pad = pad32(i == 0 ? 16 : c.cin);
    c.cout_pad = pad32(c.cout);
    c.w_off = off;
    off += 9 * (size_t)c.cin * c.cout;
    c.b_off = off;
    off += c.cout;
    u->L.push_back(c);
  }
  u->head_w = off;
  off += c1;
  u->head_b = off;
  off += 1;
  u->n_params = off;
  auto fail_oom = [&]() {
    mem_unet_destroy(u);
    return memh::api_fail(MEM_ERR_OOM, "U-Net allocation failed");
  };
  if (cudaMalloc(&u->params, off * 4) != cudaSuccess || cudaMalloc(&u->grads, off * 4) != cudaSuccess ||
      cudaMalloc(&u->adam_m, off * 4) != cudaSuccess || cudaMalloc(&u->adam_v, off * 4) != cudaSuccess ||
      cudaMalloc(&u->g0pad, 9ull * u->L[0].cin_pad * u->L[0].cout * 4) != cudaSuccess)
    return fail_oom();
  cudaMemset(u->params, 0, off * 4);
  cudaMemset(u->adam_m, 0, off * 4);
  cudaMemset(u->adam_v, 0, off * 4);
  for (auto& c : u->L) {
    if (cudaMalloc(&c.wf, 9 * (size_t)c.cin_pad * c.cout * 2) != cudaSuccess ||
        cudaMalloc(&c.wd, 9 * (size_t)c.cout_pad * c.cin * 2) != cudaSuccess)
      return fail_oom();
  }
  *out = u;
  return MEM_OK;
}

extern "C" mem_status mem_unet_destroy(mem_unet* u) {
  if (!u) return MEM_OK;
  cudaDeviceSynchronize();
  for (void* p : u->bufs) cudaFree(p);
  for (auto& c : u->L) {
    cudaFree(c.wf);
    cudaFree(c.wd);
  }
  cudaFree(u->params);
  cudaFree(u->grads);
  cudaFree(u->adam_m);
  cudaFree(u->adam_v);
  cudaFree(u->g0pad);
  delete u;
  return MEM_OK;
}

extern "C" mem_status mem_unet_param_count(const mem_unet* u, int64_t* n) {
  if (!u || !n) return memh::api_fail(MEM_ERR_ARG, "NULL argument");
  *n = (int64_t)u->n_params;
  return MEM_OK;
}

extern "C" mem_status mem_unet_set_params(mem_unet* u, const float* src, void* stream) {
  if (!u || !src) return memh::api_fail(MEM_ERR_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(u->params, src, u->n_params * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = prep_weights(u, st);
  if (e != cudaSuccess) return memh::api_cuda_fail(e, "set params");
  return MEM_OK;
}

extern "C" mem_status mem_unet_get_params(const mem_unet* u, float* dst, void* stream) {
  if (!u || !dst) return memh::api_fail(MEM_ERR_ARG, "NULL argument");
  cudaError_t e = cudaMemcpyAsync(dst, u->params, u->n_params * 4, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
  if (e != cudaSuccess) return memh::api_cuda_fail(e, "get params");
  return MEM_OK;
}

static mem_status check_shape(const mem_unet* u, int32_t n, int32_t H, int32_t W) {
  if (!u) return memh::api_fail(MEM_ERR_ARG, "NULL net");
  if (n < 1 || H < 8 || W < 8 || H % 8 || W % 8) return memh::api_fail(MEM_ERR_ARG, "H, W multiples of 8, n >= 1");
  if ((int64_t)n * H * W > (1LL << 31) / 16) return memh::api_fail(MEM_ERR_ARG, "batch too large");
  return MEM_OK;
}

// Residual prediction: pred = fill + head(U-Net(x)).
extern "C" mem_status mem_unet_forward(mem_unet* u, int32_t n, int32_t H, int32_t W, const float* x3,
                                       const float* fill, float* pred, void* stream) {
  mem_status s = check_shape(u, n, H, W);
  if (s != MEM_OK) return s;
  if (!x3 || !fill || !pred) return memh::api_fail(MEM_ERR_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = ensure_acts(u, n, H, W);
  if (e != cudaSuccess) return memh::api_cuda_fail(e, "U-Net activations");
  const int64_t P = (int64_t)n * H * W;
  k_pack_input<<<grid_for(P * 16, u->n_sm), 256, 0, st>>>(x3, u->x16, P);
  e = forward(u, n, H, W, st);
  if (e != cudaSuccess) return memh::api_cuda_fail(e, "U-Net forward");
  k_head<<<grid_for(P, u->n_sm), 256, 0, st>>>(u->act[13], u->widths[0], u->params + u->head_w,
                                                u->params + u->head_b, fill, pred, nullptr, nullptr, 0.f, P,
                                                nullptr, nullptr, nullptr, nullptr);
  e = cudaGetLastError();
  if (e != cudaSuccess) return memh::api_cuda_fail(e, "U-Net head");
  return MEM_OK;
}

// Loss (masked MSE over hidden cells) and the gradient of every parameter
// (flat float32, the parameter order of mem_unet_set_params) into `grads`.
extern "C" mem_status mem_unet_gradients(mem_unet* u, int32_t n, int32_t H, int32_t W, const float* x3,
                                         const float* fill, const float* target, const uint8_t* hidden,
                                         int64_t n_hidden, float* grads, float* loss, void* stream) {
  mem_status s = check_shape(u, n, H, W);
  if (s != MEM_OK) return s;
  if (!x3 || !fill || !target || !hidden) return memh::api_fail(MEM_ERR_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = ensure_acts(u, n, H, W);
  if (e != cudaSuccess) return memh::api_cuda_fail(e, "U-Net activations");
  const int64_t P = (int64_t)n * H * W;
  k_pack_input<<<grid_for(P * 16, u->n_sm), 256, 0, st>>>(x3, u->x16, P);
  e = forward(u, n, H, W, st);
  if (e != cudaSuccess) return memh::api_cuda_fail(e, "U-Net forward");
  cudaMemsetAsync(u->grads, 0, u->n_params * 4, st);
  cudaMemsetAsync(u->d_loss, 0, 4, st);
  // the skip tensors' gradients are accumulated: start from zero
  for (int i : {1, 3, 5}) {
    const ConvLayer& c = u->L[i];
    cudaMemsetAsync(u->dact[i], 0, (P >> (2 * c.level)) * c.cout * 2, st);
  }
  const float inv = 1.f / (float)(n_hidden > 0 ? n_hidden : 1);
  k_head<<<grid_for(P, u->n_sm), 256, 0, st>>>(u->act[13], u->widths[0], u->params + u->head_w,
                                                u->params + u->head_b, fill, nullptr, target, hidden, inv, P,
                                                u->d_loss, u->dact[13], u->grads + u->head_w, u->grads + u->head_b);
  e = backward(u, n, H, W, st);
  if (e != cudaSuccess) return memh::api_cuda_fail(e, "U-Net backward");
  if (grads) e = cudaMemcpyAsync(grads, u->grads, u->n_params * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, u->d_loss, 4, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return memh::api_cuda_fail(e, "U-Net gradient copy");
  return MEM_OK;
}

// One Adam step on the masked-MSE loss of this batch.
extern "C" mem_status mem_unet_train_step(mem_unet* u, int32_t n, int32_t H, int32_t W, const float* x3,
                                          const float* fill, const float* target, const uint8_t* hidden,
                                          int64_t n_hidden, float lr, float* loss, void* stream) {
  mem_status s = mem_unet_gradients(u, n, H, W, x3, fill, target, hidden, n_hidden, nullptr, loss, stream);
  if (s != MEM_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  u->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f / (1.f - powf(b1, (float)u->adam_t)), c2 = 1.f / (1.f - powf(b2, (float)u->adam_t));
  k_adam<<<grid_for((int64_t)u->n_params, u->n_sm), 256, 0, st>>>(u->params, u->grads, u->adam_m, u->adam_v,
                                                                  (int64_t)u->n_params, lr, b1, b2, 1e-8f, c1, c2);
  cudaError_t e = prep_weights(u, st);
  if (e != cudaSuccess) return memh::api_cuda_fail(e, "U-Net update");
  return MEM_OK;
}
