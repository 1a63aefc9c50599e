// Learned inpainting: a small U-Net trained and run with BF16 tensor-core
// kernels (float32 accumulation, float32 master weights, Adam).
//
// Layout: activations NHWC bf16. A 3x3 convolution is an implicit GEMM
// C[pixels, cout] = A[pixels, 9*cin] B[9*cin, cout] on the tcgen05 tensor
// cores: TMA box loads bring the input halo of a 16 x 16 output tile (16
// channels per pipeline stage, zero outside the image) and one bulk copy the
// stage's packed weights into shared memory; one thread issues the MMAs of all
// nine taps from that one halo (descriptors offset per tap), and the float32
// accumulator lives in tensor memory until the epilogue. The decoder's
// concatenation is a choice of tensor map and its nearest upsampling a
// half-resolution box replicated in shared memory. The data gradient is the
// same kernel with flipped, transposed weights; the weight gradient is a
// tcgen05 GEMM over pixels (both operands MN-major from TMA-loaded planes, one
// TMEM accumulator per tap) split across blocks with float32 atomics.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "mem_host.h"

typedef __nv_bfloat16 bf16;

namespace memk {

// ---------------------------------------------------------------------------
// PTX helpers

__device__ __forceinline__ u32 smem_u32(const void* p) {
  return (u32)__cvta_generic_to_shared(p);
}

// ---------------------------------------------------------------------------
// 5th-generation tensor cores (tcgen05): shared-memory operands, TMEM
// accumulator, mbarrier completion; bounded waits

__device__ __forceinline__ void mbar_init(u32 bar, u32 count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(u32 bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(u32 bar, u32 bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// wait for the phase of the given parity; false (and the error word set) after about 2^31 cycles
__device__ __forceinline__ bool mbar_wait(u32 bar, u32 parity, int* err) {
  const long long t0 = clock64();
  for (;;) {
    u32 ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > (1ll << 31)) {
      atomicExch(err, 1);
      return false;
    }
  }
}
// bulk copy global -> shared, completion counted in bytes on an mbarrier
__device__ __forceinline__ void bulk_g2s(u32 dst, const void* src, u32 bytes, u32 bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// tiled TMA load of a 4-D box (coordinates innermost first) into shared memory; elements
// outside the tensor read as zero
__device__ __forceinline__ void tma_load_4d(u32 dst, const CUtensorMap* map, int c, int x, int y, int n, u32 bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c), "r"(x), "r"(y), "r"(n), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// shared-memory matrix descriptor, no swizzle: K-major core matrices of 8 rows x 16 bytes, `lbo`
// bytes apart along K and `sbo` bytes apart along M (or N); bit 46 is the descriptor version
__device__ __forceinline__ uint64_t sdesc(u32 saddr, u32 lbo, u32 sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// D[tmem] (+)= A[smem] B[smem]^T, BF16 inputs, float32 accumulator
__device__ __forceinline__ void mma_bf16_tc(u32 d_tmem, uint64_t ad, uint64_t bd, u32 idesc, u32 accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive on the mbarrier once every MMA issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(u32 bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 16 consecutive float32 columns of this thread's TMEM lane (complete after tmem_wait_ld)
__device__ __forceinline__ void tmem_ld16_async(u32 taddr, u32 v[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld16(u32 taddr, u32 v[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------------------
// 3x3 convolution (forward, and data gradient with flipped weights)

struct ConvArgs {
  const bf16* in0;  // [N, H(/2), W(/2), c0]
  const bf16* in1;  // [N, H, W, c1] or null
  int c0, c1, up0;  // up0: in0 is at half resolution (nearest upsample)
  int cin_pad;      // input channels of the packed weights (multiple of 16, >= c0 + c1)
  const bf16* w;    // packed [cout / BN][cin_pad / 16][9 taps][2][BN][8] (see conv_bn)
  const float* bias;
  bf16* out;        // [N, H, W, cout]
  int cout, N, H, W, relu;
  int* err;         // set when a bounded wait runs out
  int store;        // write `out` (0: only the fused outputs below are wanted)
  bf16* pool;       // optional 2x2 max pooling of the output, [N, H/2, W/2, cout]
  // optional fused 1x1 head (one column block only): pred = fill + head_b + sum_c head_w[c] out[c]
  const float* head_w;
  const float* head_b;
  const float* fill;
  float* pred;
};

// output channels per block: the largest of 128, 64, 32 that divides cout
__host__ __device__ inline int conv_bn(int cout) { return cout % 128 == 0 ? 128 : (cout % 64 == 0 ? 64 : 32); }

// A work item is a 16 x 16 tile of output pixels for BN output channels,
// computed as an implicit GEMM on the tensor cores: D[256 pixels, BN]
// accumulates in TMEM as two M = 128 halves (16 rows x 8 columns of pixels
// each), K = 9 taps x the input channels. The input is consumed 16 channels
// per pipeline stage: the 18 x 18 halo of the tile arrives in shared memory
// as two planes of 8 channels (16 bytes per pixel) by two TMA box loads,
// which read zero outside the image, so the 8-pixel rows of a tap's A operand
// are eight consecutive 16-byte halo pixels: every tap reads the same halo
// through a descriptor offset by (dy * 18 + dx) pixels, with 288 bytes between
// pixel rows and one plane between the two 8-channel halves of K. The
// decoder's concatenation is a choice of tensor map per stage; its nearest
// upsampling loads the 10 x 10 half-resolution box and the gather warps
// replicate it into the halo planes. The stage's weights (9 taps x 16
// channels x BN, packed in core-matrix order) arrive with one bulk copy.
//
// The kernel is persistent (a block loops over work items) and warp
// specialised: warp 0 owns TMEM and one of its threads issues the 18 MMAs of
// each stage; warps 1..3 fill an NST-slot ring that runs across work items
// (one thread issues the copies); warps 4..7 drain the accumulator (warp w
// reads TMEM lanes 32 (w % 4)..), add bias, apply ReLU, store bf16 and the
// fused outputs. The accumulator is double-buffered in TMEM, so one item's
// epilogue overlaps the next item's MMAs. mbarriers: slot full (96 gather
// arrivals + the copied bytes), slot empty (MMA commit), half-resolution
// staging full (its bytes), accumulator full (MMA commit), accumulator empty
// (128 epilogue arrivals). Every wait is bounded.
constexpr int kTY = 16, kTX = 16;              // output tile
constexpr int kHY = kTY + 2, kHX = kTX + 2;    // input halo
constexpr int kPlaneBytes = kHY * kHX * 16;    // one 8-channel halo plane as loaded (5184)
constexpr int kPlane = 5248;                   // its stride in shared memory (128-byte multiple)
constexpr int kHalfBox = 10;                   // half-resolution box side for upsampled input
constexpr int kStgBytes = kHalfBox * kHalfBox * 16;  // one plane of it (1600)
constexpr int kStg = 1664;                     // its stride in shared memory
constexpr int kConvProd = 96;                  // gathering threads (warps 1..3)
constexpr int kConvEpi = 128;                  // epilogue threads (warps 4..7)

template <int BN, int NST>
struct ConvCfg {
  static constexpr int kWBytes = 9 * 2 * BN * 16;             // weights of one stage
  static constexpr int kSlot = 2 * kPlane + kWBytes + 2 * kStg;  // one pipeline slot
  static constexpr int kSmem = NST * kSlot + 256 + 2048 + 1024;  // + barriers, bias and head, slack
  static constexpr int kCols = 4 * BN;                        // TMEM columns: 2 buffers x 2 halves
  static constexpr int kMaxBlocksPerSm = 512 / kCols;         // TMEM holds 512 columns
};

template <int BN, int NST>
__global__ void __launch_bounds__(256, ConvCfg<BN, NST>::kMaxBlocksPerSm)
    k_conv3x3t(const __grid_constant__ CUtensorMap tm0, const __grid_constant__ CUtensorMap tm1, ConvArgs a) {
  using C = ConvCfg<BN, NST>;
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const u32 sbase = (smem_u32(sm_raw) + 1023u) & ~1023u;  // slots start 1024-byte aligned
  unsigned char* sm = sm_raw + (sbase - smem_u32(sm_raw));
  // barriers: full[NST], empty[NST], stage[NST], acc_full[2], acc_empty[2], done; TMEM address; abort
  unsigned char* tail = sm + NST * C::kSlot;
  const u32 bar0 = sbase + NST * C::kSlot;
  const u32 full0 = bar0, empty0 = bar0 + 8 * NST, stg0 = bar0 + 16 * NST, accf0 = bar0 + 24 * NST;
  const u32 acce0 = accf0 + 16, done_bar = acce0 + 16;
  u32* tmem_slot = reinterpret_cast<u32*>(tail + 24 * NST + 40);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* sbias = reinterpret_cast<float*>(tail + 256);  // [256] bias of every output channel
  float* shead = sbias + 256;                            // [256] 1x1 head weights
  const int tx = (a.W + kTX - 1) / kTX, ty = (a.H + kTY - 1) / kTY;
  const int NB = a.cout / BN;
  const int items = a.N * tx * ty * NB;
  const int S = (a.c0 + a.c1 + 15) / 16, CS = a.cin_pad / 16;  // stages past the real channels are all zero
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(full0 + 8 * s, kConvProd + 1);
      mbar_init(empty0 + 8 * s, 1);
      mbar_init(stg0 + 8 * s, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(accf0 + 8 * i, 1);
      mbar_init(acce0 + 8 * i, kConvEpi);
    }
    mbar_init(done_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < 256; i += 256) {  // output channels <= 256 wherever bias or head is given
    sbias[i] = (a.bias && i < a.cout) ? a.bias[i] : 0.f;
    shead[i] = (a.head_w && i < a.cout) ? a.head_w[i] : 0.f;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(C::kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const u32 tmem = *tmem_slot;
  if (warp == 0) {
    if (lane == 0) {
      // instruction descriptor: f32 accumulator, bf16 A and B, both K-major, N = BN, M = 128
      const u32 idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((u32)(BN >> 3) << 17) | ((u32)(128 >> 4) << 24);
      int g = 0;  // stage counter across work items
      bool run = true;
      for (int w = blockIdx.x, it = 0; w < items && run; w += gridDim.x, ++it) {
        const int ab = it & 1;
        if (it >= 2 && !mbar_wait(acce0 + 8 * ab, ((it >> 1) - 1) & 1, a.err)) {
          run = false;
          break;
        }
        tc_fence_after();
        const u32 acc = tmem + (u32)(ab * 2 * BN);
        for (int s = 0; s < S; ++s, ++g) {
          const int slot = g % NST;
          if (!mbar_wait(full0 + 8 * slot, (g / NST) & 1, a.err)) {
            run = false;
            break;
          }
          tc_fence_after();
          const u32 hb = sbase + slot * C::kSlot, wb = hb + 2 * kPlane;
#pragma unroll
          for (int t = 0; t < 9; ++t) {
            const int dy = t / 3, dx = t % 3;
            const uint64_t bd = sdesc(wb + t * 2 * BN * 16, BN * 16, 128);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const uint64_t ad = sdesc(hb + (dy * kHX + 8 * h + dx) * 16, kPlane, kHX * 16);
              mma_bf16_tc(acc + h * BN, ad, bd, idesc, (s | t) != 0);
            }
          }
          mma_commit(empty0 + 8 * slot);
        }
        if (run) mma_commit(accf0 + 8 * ab);
      }
      if (!run) *abort_flag = 1;
      mma_commit(done_bar);
    }
  } else if (warp < 4) {
    const int pt = tid - 32;
    int g = 0;
    u32 stg_phase = 0;  // bit per slot: parity of the next half-resolution load into it
    bool run = true;
    for (int w = blockIdx.x; w < items && run; w += gridDim.x) {
      const int nb = w % NB;
      int b = w / NB;
      const int n = b / (tx * ty);
      b -= n * tx * ty;
      const int y0 = (b / tx) * kTY, x0 = (b % tx) * kTX;
      for (int s = 0; s < S; ++s, ++g) {
        const int slot = g % NST;
        if ((g >= NST && !mbar_wait(empty0 + 8 * slot, ((g / NST) - 1) & 1, a.err)) || *abort_flag) {
          run = false;
          break;
        }
        const u32 hb = sbase + slot * C::kSlot, wb = hb + 2 * kPlane, sb = wb + C::kWBytes;
        const int cb = s * 16;
        const bool from0 = cb < a.c0, up = from0 && a.up0;
        const CUtensorMap* map = from0 ? &tm0 : &tm1;
        const int c = from0 ? cb : cb - a.c0;
        if (pt == 0) {
          const u32 bytes = C::kWBytes + (up ? 0u : 2u * kPlaneBytes);
          mbar_arrive_tx(full0 + 8 * slot, bytes);
          bulk_g2s(wb, a.w + (int64_t)(nb * CS + s) * (9 * 2 * BN * 8), C::kWBytes, full0 + 8 * slot);
          if (up) {
            mbar_arrive_tx(stg0 + 8 * slot, 2u * kStgBytes);
            tma_load_4d(sb, map, c, (x0 >> 1) - 1, (y0 >> 1) - 1, n, stg0 + 8 * slot);
            tma_load_4d(sb + kStg, map, c + 8, (x0 >> 1) - 1, (y0 >> 1) - 1, n, stg0 + 8 * slot);
          } else {
            tma_load_4d(hb, map, c, x0 - 1, y0 - 1, n, full0 + 8 * slot);
            tma_load_4d(hb + kPlane, map, c + 8, x0 - 1, y0 - 1, n, full0 + 8 * slot);
          }
        }
        if (up) {
          // nearest upsampling: halo pixel (hy, hx) is half-resolution box pixel ((hy + 1) / 2, (hx + 1) / 2)
          if (!mbar_wait(stg0 + 8 * slot, (stg_phase >> slot) & 1, a.err)) {
            *abort_flag = 1;
            run = false;
          }
          stg_phase ^= 1u << slot;
          if (run) {
            for (int i = pt; i < 2 * kHY * kHX; i += kConvProd) {
              const int pl = i >= kHY * kHX, hp = i - pl * kHY * kHX;
              const int hy = hp / kHX, hx = hp - hy * kHX;
              const uint4 v = *reinterpret_cast<const uint4*>(sm + (sb - sbase) + pl * kStg +
                                                              (((hy + 1) >> 1) * kHalfBox + ((hx + 1) >> 1)) * 16);
              *reinterpret_cast<uint4*>(sm + (hb - sbase) + pl * kPlane + hp * 16) = v;
            }
            fence_proxy_async();
          }
        }
        mbar_arrive(full0 + 8 * slot);
        if (!run) break;
      }
    }
  } else {
    const int q = warp & 3;
    const int m = q * 32 + lane;  // accumulator row = pixel (m / 8, 8 h + m % 8) of a tile half
    for (int w = blockIdx.x, it = 0; w < items; w += gridDim.x, ++it) {
      const int ab = it & 1;
      bool ok = mbar_wait(accf0 + 8 * ab, (it >> 1) & 1, a.err);
      ok = __all_sync(0xffffffffu, ok && !*abort_flag);
      if (!ok) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const int nb = w % NB;
      int b = w / NB;
      const int n = b / (tx * ty);
      b -= n * tx * ty;
      const int y0 = (b / tx) * kTY, x0 = (b % tx) * kTX;
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int yy = y0 + (m >> 3), xx = x0 + 8 * h + (m & 7);
        const bool inside = yy < a.H && xx < a.W;
        const int64_t pix = ((int64_t)n * a.H + (inside ? yy : 0)) * a.W + (inside ? xx : 0);
        bf16* o = a.out + pix * a.cout + nb * BN;
        // pooling partners: lanes ^1 (x + 1) and ^8 (y + 1); lane bits 0 and 3 clear = top-left
        // pixel, and H, W are even wherever pooling happens, so a window is wholly inside or outside
        const bool pool_writer = inside && (lane & 9) == 0;
        bf16* po = a.pool ? a.pool + (((int64_t)n * (a.H >> 1) + (yy >> 1)) * (a.W >> 1) + (xx >> 1)) * a.cout +
                                nb * BN
                          : nullptr;
        float hr = a.head_w ? a.head_b[0] : 0.f;
#pragma unroll 1
        for (int c32 = 0; c32 < BN; c32 += 32) {
          u32 v[2][16];
          const u32 ta = tmem + ((u32)(q * 32) << 16) + (u32)(ab * 2 * BN + h * BN + c32);
          tmem_ld16_async(ta, v[0]);
          tmem_ld16_async(ta + 16, v[1]);
          tmem_wait_ld();
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const int c0 = c32 + 16 * k;
            const float* bz = sbias + nb * BN + c0;
            u32 pk[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              float f0 = __uint_as_float(v[k][2 * j]) + bz[2 * j], f1 = __uint_as_float(v[k][2 * j + 1]) + bz[2 * j + 1];
              if (a.relu) {
                f0 = fmaxf(f0, 0.f);
                f1 = fmaxf(f1, 0.f);
              }
              __nv_bfloat162 p2 = __floats2bfloat162_rn(f0, f1);
              pk[j] = *reinterpret_cast<u32*>(&p2);
            }
            if (inside && a.store) {
              uint4* dst = reinterpret_cast<uint4*>(o + c0);
              dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
              dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            }
            if (po) {
              u32 mx[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const u32 o1 = __shfl_xor_sync(0xffffffffu, pk[j], 1);
                const u32 o8 = __shfl_xor_sync(0xffffffffu, pk[j], 8);
                const u32 o9 = __shfl_xor_sync(0xffffffffu, pk[j], 9);
                const float2 a0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&pk[j]));
                const float2 a1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&o1));
                const float2 a8 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&o8));
                const float2 a9 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&o9));
                __nv_bfloat162 r2 = __floats2bfloat162_rn(fmaxf(fmaxf(a0.x, a1.x), fmaxf(a8.x, a9.x)),
                                                          fmaxf(fmaxf(a0.y, a1.y), fmaxf(a8.y, a9.y)));
                mx[j] = *reinterpret_cast<u32*>(&r2);
              }
              if (pool_writer) {
                uint4* dst = reinterpret_cast<uint4*>(po + c0);
                dst[0] = make_uint4(mx[0], mx[1], mx[2], mx[3]);
                dst[1] = make_uint4(mx[4], mx[5], mx[6], mx[7]);
              }
            }
            if (a.head_w) {
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&pk[j]));
                hr = fmaf(f.x, shead[c0 + 2 * j], hr);
                hr = fmaf(f.y, shead[c0 + 2 * j + 1], hr);
              }
            }
          }
        }
        if (a.head_w && inside) a.pred[pix] = a.fill[pix] + hr;
      }
      tc_fence_before();
      mbar_arrive(acce0 + 8 * ab);
    }
  }
  // every MMA this block issued has completed before its TMEM is released
  mbar_wait(done_bar, 0, a.err);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::kCols) : "memory");
  }
}

// ---------------------------------------------------------------------------
// weight gradient: dW[t][ci][co] = sum_p X[p + off(t)][ci] dY[p][co]
//
// On the tensor cores with both operands read MN-major straight from TMA-loaded
// planes: per 16 x 8 tile of output pixels, the 18 x 10 input halo arrives as
// up to 16 planes of 8 channels (the block's 128 input channels = M) and dY as
// NB/8 planes of 8 output channels (N); a K = 16 step is one 16-pixel row, so
// tap (dy, dx) and row py read the halo through a descriptor offset by
// ((py + dy) * 18 + dx) pixels, 128 bytes between the two 8-pixel halves of K
// and one plane between 8-channel groups of M (and N). Each tap of the block's
// tap group accumulates in its own TMEM columns over all tiles of the block's
// pixel range; the epilogue adds the float32 sums to dW with atomics (blocks
// split the pixels). Warp 0: TMEM and the MMA thread; warp 1: one thread
// issues the copies; all four warps drain TMEM at the end. Waits are bounded.

struct WgradArgs {
  int Cx, cin_pad, cout;  // input channels in the tensor (real), rows of dW per tap, dY channels
  float* dw;              // [9][cin_pad][cout] float32, accumulated into
  int N, H, W;
  int tiles;              // 16 x 8 pixel tiles over the batch
  int* err;
};

constexpr int kWgPlane = 2944;          // one 18 x 10 x 8-channel halo plane (2880 bytes), 128-byte stride
constexpr int kWgPlaneBytes = 18 * 10 * 16;
constexpr int kWgDyPlane = 16 * 8 * 16;  // one 16 x 8 x 8-channel dY plane (2048 bytes)

template <int NB, int TAPG, int NST>
struct WgCfg {
  static constexpr int kSlot = 16 * kWgPlane + (NB / 8) * kWgDyPlane;
  static constexpr int kSmem = NST * kSlot + 128 + 1024;  // + barriers, alignment slack
};

template <int NB, int TAPG, int NST>
__global__ void __launch_bounds__(128, 1)
    k_wgrad3x3t(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmy, WgradArgs a) {
  using C = WgCfg<NB, TAPG, NST>;
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const u32 sbase = (smem_u32(sm_raw) + 1023u) & ~1023u;
  unsigned char* tail = sm_raw + (sbase - smem_u32(sm_raw)) + NST * C::kSlot;
  const u32 bar0 = sbase + NST * C::kSlot;
  const u32 full0 = bar0, empty0 = bar0 + 8 * NST, done_bar = bar0 + 16 * NST;
  u32* tmem_slot = reinterpret_cast<u32*>(tail + 16 * NST + 8);
  const int mb = blockIdx.y;                                  // input channels mb*128 ..
  const int nb = blockIdx.z % (a.cout / NB), tg = blockIdx.z / (a.cout / NB);  // output block, tap group
  const int t_first = tg * TAPG, n_taps = min(TAPG, 9 - t_first);
  const int t_begin = (int)((int64_t)blockIdx.x * a.tiles / gridDim.x);
  const int t_end = (int)((int64_t)(blockIdx.x + 1) * a.tiles / gridDim.x);
  const int nt = t_end - t_begin;
  const int planes = min(16, (a.Cx - mb * 128 + 7) / 8);  // halo planes holding real channels (> 0)
  const int tx = (a.W + 15) / 16, ty = (a.H + 7) / 8;
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const u32 tmem = *tmem_slot;
  bool ok = true;
  if (warp == 0 && lane == 0) {
    // f32 accumulator, bf16 A and B, both MN-major, N = NB, M = 128
    const u32 idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((u32)(NB >> 3) << 17) |
                      ((u32)(128 >> 4) << 24);
    for (int it = 0; it < nt; ++it) {
      const int slot = it % NST;
      if (!mbar_wait(full0 + 8 * slot, (it / NST) & 1, a.err)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const u32 hb = sbase + slot * C::kSlot, yb = hb + 16 * kWgPlane;
      for (int tl = 0; tl < n_taps; ++tl) {
        const int t = t_first + tl, dy = t / 3, dx = t % 3;
#pragma unroll
        for (int py = 0; py < 8; ++py) {
          const uint64_t ad = sdesc(hb + ((py + dy) * 18 + dx) * 16, 128, kWgPlane);
          const uint64_t bd = sdesc(yb + py * 16 * 16, 128, kWgDyPlane);
          mma_bf16_tc(tmem + (u32)(tl * NB), ad, bd, idesc, (it | py) != 0);
        }
      }
      mma_commit(empty0 + 8 * slot);
    }
    mma_commit(done_bar);
  } else if (warp == 1 && lane == 0) {
    for (int it = 0; it < nt; ++it) {
      const int slot = it % NST;
      if (it >= NST && !mbar_wait(empty0 + 8 * slot, ((it / NST) - 1) & 1, a.err)) break;
      int b = t_begin + it;
      const int n = b / (tx * ty);
      b -= n * tx * ty;
      const int y0 = (b / tx) * 8, x0 = (b % tx) * 16;
      const u32 hb = sbase + slot * C::kSlot, yb = hb + 16 * kWgPlane;
      mbar_arrive_tx(full0 + 8 * slot, (u32)(planes * kWgPlaneBytes + (NB / 8) * kWgDyPlane));
      for (int pl = 0; pl < planes; ++pl)
        tma_load_4d(hb + pl * kWgPlane, &tmx, mb * 128 + pl * 8, x0 - 1, y0 - 1, n, full0 + 8 * slot);
      for (int j = 0; j < NB / 8; ++j)
        tma_load_4d(yb + j * kWgDyPlane, &tmy, nb * NB + j * 8, x0, y0, n, full0 + 8 * slot);
    }
  }
  // all MMAs of this block done (bounded); then every thread owns TMEM lane tid = input channel
  ok = mbar_wait(done_bar, 0, a.err) && ok;
  tc_fence_after();
  ok = __all_sync(0xffffffffu, ok) && nt > 0;
  const int ci = mb * 128 + tid;
  if (ok) {
    for (int tl = 0; tl < n_taps; ++tl) {
      const int t = t_first + tl;
#pragma unroll 1
      for (int c0 = 0; c0 < NB; c0 += 16) {
        u32 v[16];
        tmem_ld16(tmem + ((u32)(warp * 32) << 16) + (u32)(tl * NB + c0), v);
        if (ci < a.Cx && ci < a.cin_pad) {
          float* d = a.dw + ((int64_t)t * a.cin_pad + ci) * a.cout + nb * NB + c0;
#pragma unroll
          for (int j = 0; j < 16; ++j) atomicAdd(d + j, __uint_as_float(v[j]));
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

// decoder input for the weight gradient: [upsampled in0 (c0), in1 (c1)] at full resolution
__global__ void k_cat_up(const bf16* __restrict__ in0, const bf16* __restrict__ in1, bf16* __restrict__ out, int N,
                         int H, int W, int c0, int c1) {
  const int cin = c0 + c1, chunks = cin / 8;
  const int64_t total = (int64_t)N * H * W * chunks;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int ch = (int)(i % chunks) * 8;
    const int64_t p = i / chunks;
    const int x = (int)(p % W), y = (int)((p / W) % H), n = (int)(p / ((int64_t)W * H));
    const uint4* src = ch < c0 ? reinterpret_cast<const uint4*>(
                                     in0 + (((int64_t)n * (H / 2) + y / 2) * (W / 2) + x / 2) * c0 + ch)
                               : reinterpret_cast<const uint4*>(in1 + p * c1 + (ch - c0));
    *reinterpret_cast<uint4*>(out + p * cin + ch) = *src;
  }
}

// ---------------------------------------------------------------------------
// element-wise pieces

// gradient of 2x2 max pooling to the first maximum of each window (row-major),
// added to `acc` (the gradient that reached the same tensor through the skip)
__global__ void k_maxpool_bwd(const bf16* __restrict__ x, const bf16* __restrict__ dy, bf16* __restrict__ acc,
                              int N, int H, int W, int C) {
  // a thread owns one 8-channel chunk (16-byte accesses) of one 2x2 window
  const int Ho = H / 2, Wo = W / 2, chunks = C / 8;
  const int64_t total = (int64_t)N * Ho * Wo * chunks;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % chunks) * 8;
    int64_t r = i / chunks;
    const int xo = (int)(r % Wo);
    r /= Wo;
    const int yo = (int)(r % Ho);
    const int n = (int)(r / Ho);
    const int64_t base = (((int64_t)n * H + 2 * yo) * W + 2 * xo) * C + c;
    const int64_t off[4] = {0, C, (int64_t)W * C, (int64_t)W * C + C};
    float xv[4][8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint4 v = *reinterpret_cast<const uint4*>(x + base + off[k]);
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 f = __bfloat1622float2(h[j]);
        xv[k][2 * j] = f.x;
        xv[k][2 * j + 1] = f.y;
      }
    }
    int am[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {  // first maximum of the window in row-major order
      am[j] = 0;
      float best = xv[0][j];
#pragma unroll
      for (int k = 1; k < 4; ++k)
        if (xv[k][j] > best) {
          best = xv[k][j];
          am[j] = k;
        }
    }
    const uint4 gv = *reinterpret_cast<const uint4*>(dy + i * 8);
    const __nv_bfloat162* gh = reinterpret_cast<const __nv_bfloat162*>(&gv);
    float g[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 f = __bfloat1622float2(gh[j]);
      g[2 * j] = f.x;
      g[2 * j + 1] = f.y;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      uint4* ap = reinterpret_cast<uint4*>(acc + base + off[k]);
      uint4 v = *ap;
      __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&v);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 f = __bfloat1622float2(h[j]);
        h[j] = __floats2bfloat162_rn(f.x + (am[2 * j] == k ? g[2 * j] : 0.f), f.y + (am[2 * j + 1] == k ? g[2 * j + 1] : 0.f));
      }
      *ap = v;
    }
  }
}

// ReLU gradient in place: dy *= (y > 0), 8 channels (16 bytes) per step
__global__ void k_relu_bwd(const bf16* __restrict__ y, bf16* __restrict__ dy, int64_t n) {
  const int64_t n8 = n / 8;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n8; i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 yv = *reinterpret_cast<const uint4*>(y + i * 8);
    uint4 dv = *reinterpret_cast<const uint4*>(dy + i * 8);
    const __nv_bfloat162* yh = reinterpret_cast<const __nv_bfloat162*>(&yv);
    __nv_bfloat162* dh = reinterpret_cast<__nv_bfloat162*>(&dv);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 f = __bfloat1622float2(yh[j]);
      const float2 d = __bfloat1622float2(dh[j]);
      dh[j] = __floats2bfloat162_rn(f.x > 0.f ? d.x : 0.f, f.y > 0.f ? d.y : 0.f);
    }
    *reinterpret_cast<uint4*>(dy + i * 8) = dv;
  }
}

// gradient of concat([upsample(low), skip]): low gets the 2x2 sums of the
// first c_up channels, skip the remaining channels; 8 channels (16 bytes) per step
__global__ void k_split_cat_bwd(const bf16* __restrict__ dcat, bf16* __restrict__ dlow,
                                bf16* __restrict__ dskip, int N, int H, int W, int c_up, int c_skip) {
  const int Ho = H / 2, Wo = W / 2;
  const int C = c_up + c_skip, cu8 = c_up / 8, cs8 = c_skip / 8;
  const int64_t tl = (int64_t)N * Ho * Wo * cu8;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tl; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % cu8) * 8;
    int64_t r = i / cu8;
    const int xo = (int)(r % Wo);
    r /= Wo;
    const int yo = (int)(r % Ho);
    const int n = (int)(r / Ho);
    const int64_t b = (((int64_t)n * H + 2 * yo) * W + 2 * xo) * C + c;
    const int64_t off[4] = {0, C, (int64_t)W * C, (int64_t)W * C + C};
    float s[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint4 v = *reinterpret_cast<const uint4*>(dcat + b + off[k]);
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 f = __bfloat1622float2(h[j]);
        s[2 * j] = k ? s[2 * j] + f.x : f.x;
        s[2 * j + 1] = k ? s[2 * j + 1] + f.y : f.y;
      }
    }
    uint4 o;
    __nv_bfloat162* oh = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
    for (int j = 0; j < 4; ++j) oh[j] = __floats2bfloat162_rn(s[2 * j], s[2 * j + 1]);
    *reinterpret_cast<uint4*>(dlow + i * 8) = o;
  }
  const int64_t ts = (int64_t)N * H * W * cs8;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ts; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % cs8) * 8;
    const int64_t p = i / cs8;
    *reinterpret_cast<uint4*>(dskip + i * 8) = *reinterpret_cast<const uint4*>(dcat + p * C + c_up + c);
  }
}

// bias gradient: db[c] += sum over pixels of dy[p][c]
// bias gradient db[c] += sum_p dy[p][c]: a thread owns one 8-channel chunk (16-byte loads) over
// a stride of pixels; partial sums meet in shared memory, one atomic per channel per block
__global__ void k_bias_grad(const bf16* __restrict__ dy, float* __restrict__ db, int64_t P, int C) {
  __shared__ float s_db[256];
  for (int c = threadIdx.x; c < C; c += blockDim.x) s_db[c] = 0.f;
  __syncthreads();
  const int chunks = C / 8;  // divides the grid's thread count, so a thread keeps its chunk
  const int64_t items = P * chunks, stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int64_t i = i0; i < items; i += stride) {
    const uint4 v = *reinterpret_cast<const uint4*>(dy + i * 8);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 f = __bfloat1622float2(h[j]);
      acc[2 * j] += f.x;
      acc[2 * j + 1] += f.y;
    }
  }
  if (i0 < items) {
    const int k = (int)(i0 % chunks) * 8;
#pragma unroll
    for (int j = 0; j < 8; ++j) atomicAdd(&s_db[k + j], acc[j]);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) atomicAdd(&db[c], s_db[c]);
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// final 1x1 convolution (residual over the diffusion fill), masked-MSE loss and
// its gradients: res = b + d1 . w ; pred = fill + res. A thread owns a pixel and reads
// its channels 8 at a time; the weight gradient is summed across the warp by shuffles
// (one shared-memory add per warp and channel), skipped where no lane has a hidden cell.
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
  const int lane = threadIdx.x & 31;
  float l = 0.f, gb = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // every lane of a warp runs the same number of iterations (the shuffles need all 32)
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < P; base += stride) {
    const int64_t p = base + threadIdx.x;
    const bool in = p < P;
    float g = 0.f;
    if (in) {
      float r = b[0];
      for (int c = 0; c < C; c += 8) {
        const uint4 v = *reinterpret_cast<const uint4*>(d1 + p * C + c);
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float2 f = __bfloat1622float2(h[j]);
          r = fmaf(f.x, s_w[c + 2 * j], r);
          r = fmaf(f.y, s_w[c + 2 * j + 1], r);
        }
      }
      const float pr = fill[p] + r;
      if (pred) pred[p] = pr;
      if (target) {
        const float diff = hidden[p] ? pr - target[p] : 0.f;
        l += diff * diff;
        g = 2.f * diff * inv_cnt;
        gb += g;
        for (int c = 0; c < C; c += 8) {
          u32 o[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            __nv_bfloat162 q = __floats2bfloat162_rn(g * s_w[c + 2 * j], g * s_w[c + 2 * j + 1]);
            o[j] = *reinterpret_cast<u32*>(&q);
          }
          *reinterpret_cast<uint4*>(dd1 + p * C + c) = make_uint4(o[0], o[1], o[2], o[3]);
        }
      }
    }
    if (target && __any_sync(0xffffffffu, g != 0.f)) {
      for (int c = 0; c < C; c += 8) {
        uint4 v = make_uint4(0, 0, 0, 0);
        if (in) v = *reinterpret_cast<const uint4*>(d1 + p * C + c);
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float2 f = __bfloat1622float2(h[j]);
          const float s0 = warp_sum(g * f.x), s1 = warp_sum(g * f.y);
          if (lane == 0) {
            atomicAdd(&s_dw[c + 2 * j], s0);
            atomicAdd(&s_dw[c + 2 * j + 1], s1);
          }
        }
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

// index of weight (tap t, input channel ci, output channel co) in the packed
// layout the convolution streams: [co / BN][ci / 16][t][(ci / 8) % 2][co % BN][ci % 8]
// (one pipeline stage = one contiguous run of 9 x 16 x BN values)
__device__ __forceinline__ void unpack_index(int64_t i, int BN, int CS, int& t, int& ci, int& co) {
  const int k = (int)(i & 7);
  int64_t r = i >> 3;
  const int col = (int)(r % BN);
  r /= BN;
  const int g = (int)(r & 1);
  r >>= 1;
  t = (int)(r % 9);
  r /= 9;
  const int cs = (int)(r % CS), nb = (int)(r / CS);
  ci = cs * 16 + g * 8 + k;
  co = nb * BN + col;
}

// float32 master weights [3][3][cin][cout] -> packed bf16 forward weights (cin_pad
// input channels) and (optionally) the data-gradient weights: taps flipped, roles of
// input and output channels exchanged (cout_pad input channels, cin_out outputs)
__global__ void k_prep_weights(const float* __restrict__ w, int cin, int cout, int cin_pad, bf16* __restrict__ wf,
                               bf16* __restrict__ wd, int cout_pad, int cin_out) {
  const int64_t nf = 9LL * cin_pad * cout;
  const int bnf = conv_bn(cout), csf = cin_pad / 16;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    int t, ci, co;
    unpack_index(i, bnf, csf, t, ci, co);
    wf[i] = __float2bfloat16_rn(ci < cin ? w[((int64_t)t * cin + ci) * cout + co] : 0.f);
  }
  if (!wd) return;
  const int64_t nd = 9LL * cout_pad * cin_out;
  const int bnd = conv_bn(cin_out), csd = cout_pad / 16;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nd; i += (int64_t)gridDim.x * blockDim.x) {
    int t, k, j;  // k: input channel of the data-gradient conv (= layer output), j: its output (= layer input)
    unpack_index(i, bnd, csd, t, k, j);
    wd[i] = __float2bfloat16_rn((k < cout && j < cin) ? w[((int64_t)(8 - t) * cin + j) * cout + k] : 0.f);
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
  int* d_err = nullptr;    // set by a convolution whose bounded wait ran out
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

template <int BN, int NST>
void launch_conv(int items, const CUtensorMap& tm0, const CUtensorMap& tm1, const ConvArgs& a, int n_sm,
                 cudaStream_t st) {
  using C = ConvCfg<BN, NST>;
  static int per_sm = 0;  // resident blocks per SM: shared memory per SM, capped by TMEM; set up once
  if (!per_sm) {
    cudaFuncSetAttribute(k_conv3x3t<BN, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
    int dev = 0, smem_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const int by_smem = smem_sm / (C::kSmem + 1024);  // 1 KB per block is reserved by the system
    per_sm = by_smem < 1 ? 1 : (by_smem > C::kMaxBlocksPerSm ? C::kMaxBlocksPerSm : by_smem);
  }
  const int grid = items < n_sm * per_sm ? items : n_sm * per_sm;
  k_conv3x3t<BN, NST><<<grid, 256, C::kSmem, st>>>(tm0, tm1, a);
}

// the driver's tensor-map encoder, looked up once through the runtime
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// NHWC bf16 activations [n][h][w][c] as a 4-D tensor (c innermost) read in boxes of
// 8 channels x box x box pixels; false if the encoder is unavailable or refuses
bool activation_map(CUtensorMap* m, const bf16* base, int c, int w, int h, int n, int box) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)c, (cuuint64_t)w, (cuuint64_t)h, (cuuint64_t)n};
  const cuuint64_t strides[3] = {(cuuint64_t)c * 2, (cuuint64_t)c * 2 * w, (cuuint64_t)c * 2 * w * h};
  const cuuint32_t boxd[4] = {8, (cuuint32_t)box, (cuuint32_t)box, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(base), dims, strides, boxd, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// outputs fused into a convolution's epilogue
struct ConvFuse {
  bool store = true;           // write the convolution output itself
  bf16* pool = nullptr;        // 2x2 max pooling of the output
  const float* head_w = nullptr;  // 1x1 head: pred = fill + head_b + head_w . out
  const float* head_b = nullptr;
  const float* fill = nullptr;
  float* pred = nullptr;
};

cudaError_t conv(mem_unet* u, const ConvLayer& c, const bf16* in0, const bf16* in1, const bf16* w,
                 const float* bias, bf16* out, int cout, int cin_pad, int c0, int c1, int up0, int N, int H,
                 int W, int relu, cudaStream_t st, const ConvFuse& fz = ConvFuse()) {
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
  a.err = u->d_err;
  a.store = fz.store ? 1 : 0;
  a.pool = fz.pool;
  a.head_w = fz.head_w;
  a.head_b = fz.head_b;
  a.fill = fz.fill;
  a.pred = fz.pred;
  (void)c;
  // a 16-channel stage comes from one input: c0 and c1 are multiples of 16; TMA boxes start on
  // 16-byte channel offsets and rows of whole 16-byte multiples
  if (cout % 32 != 0 || cin_pad % 16 != 0 || c0 % 16 != 0 || c1 % 16 != 0 || c0 < 16 || c0 + c1 > cin_pad ||
      (c1 && !in1))
    return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(in0) | reinterpret_cast<uintptr_t>(in1) | reinterpret_cast<uintptr_t>(w)) & 15)
    return cudaErrorInvalidValue;
  CUtensorMap tm0, tm1;
  if (!activation_map(&tm0, in0, c0, up0 ? W / 2 : W, up0 ? H / 2 : H, N, up0 ? kHalfBox : kHX))
    return cudaErrorInvalidValue;
  if (c1) {
    if (!activation_map(&tm1, in1, c1, W, H, N, kHX)) return cudaErrorInvalidValue;
  } else {
    tm1 = tm0;
  }
  if ((fz.pool && (H % 2 || W % 2)) || (fz.head_w && conv_bn(cout) != cout)) return cudaErrorInvalidValue;
  if ((bias || fz.head_w) && cout > 256) return cudaErrorInvalidValue;  // staged in 256-entry tables
  const int items = N * ((H + kTY - 1) / kTY) * ((W + kTX - 1) / kTX) * (cout / conv_bn(cout));
  // pipeline depth per column-block width (measured on 256 crops of 256 x 256): 3 slots for 128
  // channels (one block per SM), 2 for 64 and 32 (two and four blocks per SM)
  switch (conv_bn(cout)) {
    case 128: launch_conv<128, 3>(items, tm0, tm1, a, u->n_sm, st); break;
    case 64: launch_conv<64, 2>(items, tm0, tm1, a, u->n_sm, st); break;
    default: launch_conv<32, 2>(items, tm0, tm1, a, u->n_sm, st); break;
  }
  return cudaGetLastError();
}

template <int NB, int TAPG, int NST>
void launch_wgrad(dim3 grid, const CUtensorMap& tmx, const CUtensorMap& tmy, const WgradArgs& a, cudaStream_t st) {
  using C = WgCfg<NB, TAPG, NST>;
  static bool attr = false;  // dynamic shared memory above 48 KB is opted into once
  if (!attr) {
    cudaFuncSetAttribute(k_wgrad3x3t<NB, TAPG, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
    attr = true;
  }
  k_wgrad3x3t<NB, TAPG, NST><<<grid, 128, C::kSmem, st>>>(tmx, tmy, a);
}

// NHWC bf16 tensor [n][h][w][c] as a 4-D tensor map with boxes of 8 channels x bw x bh pixels
bool nhwc_map(CUtensorMap* m, const bf16* base, int c, int w, int h, int n, int bw, int bh) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)c, (cuuint64_t)w, (cuuint64_t)h, (cuuint64_t)n};
  const cuuint64_t strides[3] = {(cuuint64_t)c * 2, (cuuint64_t)c * 2 * w, (cuuint64_t)c * 2 * w * h};
  const cuuint32_t boxd[4] = {8, (cuuint32_t)bw, (cuuint32_t)bh, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(base), dims, strides, boxd, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// dW (float32, [9][cin_pad][cout], accumulated into) of one 3x3 convolution whose input is
// in0 (c0 channels; at half resolution when up0) concatenated with in1 (c1 channels)
cudaError_t wgrad(mem_unet* u, const ConvLayer& c, const bf16* in0, const bf16* in1, const bf16* dy,
                  float* dw_pad, int N, int H, int W, cudaStream_t st) {
  const bf16* X = in0;
  int Cx = c.c0;
  if (c.c1 || c.up0) {  // decoder input: materialise [upsampled, skip] in the concat scratch
    Cx = c.c0 + c.c1;
    k_cat_up<<<grid_for((int64_t)N * H * W * (Cx / 8), u->n_sm), 256, 0, st>>>(in0, in1, u->dcat, N, H, W, c.c0,
                                                                                  c.c1);
    X = u->dcat;
  }
  if (Cx % 8 || c.cout % 32 || c.cin_pad % 8 || Cx > c.cin_pad) return cudaErrorInvalidValue;
  CUtensorMap tmx, tmy;
  if (!nhwc_map(&tmx, X, Cx, W, H, N, 18, 10) || !nhwc_map(&tmy, dy, c.cout, W, H, N, 16, 8))
    return cudaErrorInvalidValue;
  WgradArgs a;
  a.Cx = Cx;
  a.cin_pad = c.cin_pad;
  a.cout = c.cout;
  a.dw = dw_pad;
  a.N = N;
  a.H = H;
  a.W = W;
  a.tiles = N * ((H + 7) / 8) * ((W + 15) / 16);
  a.err = u->d_err;
  // output-channel block and tap group: TMEM holds the tap group's accumulators (<= 512 columns)
  const int NB = c.cout % 128 == 0 ? 128 : (c.cout % 64 == 0 ? 64 : 32);
  const int TAPG = NB == 128 ? 3 : (NB == 64 ? 5 : 9);
  const int mbk = (Cx + 127) / 128, groups = (c.cout / NB) * ((9 + TAPG - 1) / TAPG);
  int splits = (u->n_sm + mbk * groups - 1) / (mbk * groups);  // about one block per SM
  if (splits > a.tiles / 8) splits = a.tiles / 8;  // at least 8 tiles per block: the epilogue's atomics
                                                  // cost about as much as 8 tiles of MMAs
  if (splits < 1) splits = 1;
  const dim3 grid((unsigned)splits, (unsigned)mbk, (unsigned)groups);
  switch (NB) {
    case 128: launch_wgrad<128, 3, 2>(grid, tmx, tmy, a, st); break;
    case 64: launch_wgrad<64, 5, 3>(grid, tmx, tmy, a, st); break;
    default: launch_wgrad<32, 9, 3>(grid, tmx, tmy, a, st); break;
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

// The encoder levels' pooling runs in the epilogue of their second convolution.
// With `pred` (inference), the 1x1 head runs in the epilogue of the last
// convolution when that convolution is a single column block (widths[0] of 32,
// 64 or 128), and its output is not stored; *head_done says whether it did.
cudaError_t forward(mem_unet* u, int N, int H, int W, cudaStream_t st, const float* fill = nullptr,
                    float* pred = nullptr, bool* head_done = nullptr) {
  cudaError_t e = cudaSuccess;
  if (head_done) *head_done = false;
  for (size_t i = 0; i < u->L.size() && e == cudaSuccess; ++i) {
    const ConvLayer& c = u->L[i];
    const int l = c.level;
    const int Hl = H >> l, Wl = W >> l;
    const int c0 = i == 0 ? 16 : c.c0;
    ConvFuse fz;
    if (i == 1 || i == 3 || i == 5) fz.pool = u->pool[i / 2];  // the end of encoder levels 1..3
    if (i == 13 && pred && conv_bn(c.cout) == c.cout) {
      fz.store = false;
      fz.head_w = u->params + u->head_w;
      fz.head_b = u->params + u->head_b;
      fz.fill = fill;
      fz.pred = pred;
      if (head_done) *head_done = true;
    }
    e = conv(u, c, input0(u, (int)i), input1(u, (int)i), c.wf, u->params + c.b_off, u->act[i], c.cout, c.cin_pad,
             c0, c.c1, c.up0, N, Hl, Wl, 1, st, fz);
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
    k_relu_bwd<<<grid_for(Pl * c.cout / 8, u->n_sm), 256, 0, st>>>(u->act[i], u->dact[i], Pl * c.cout);
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
    k_bias_grad<<<u->n_sm * 2, 256, 0, st>>>(u->dact[i], u->grads + c.b_off, Pl, c.cout);
    if (i == 0) break;
    // data gradient into the layer input
    if (c.c1) {  // decoder concat input: d(concat) then split
      e = conv(u, c, u->dact[i], nullptr, c.wd, nullptr, u->dcat, c.cin, c.cout_pad, c.cout, 0, 0, N, Hl, Wl, 0, st);
      if (e != cudaSuccess) return e;
      // low-resolution source gradient -> dact of the producing layer; skip -> dact of the skip layer
      const int lowi = i - 1, skipi = (i == 8) ? 5 : (i == 10 ? 3 : 1);
      k_split_cat_bwd<<<grid_for(Pl * c.cin / 8, u->n_sm), 256, 0, st>>>(u->dcat, u->dact[lowi], u->dact[skipi], N, Hl, Wl,
                                                                      c.c0, c.c1);
    } else if (i == 2 || i == 4 || i == 6) {  // input is a pooled tensor
      const int lv = i / 2 - 1;
      e = conv(u, c, u->dact[i], nullptr, c.wd, nullptr, u->dpool[lv], c.cin, c.cout_pad, c.cout, 0, 0, N, Hl, Wl, 0,
               st);
      if (e != cudaSuccess) return e;
      // route through the pooling and add to the skip gradient already in dact[i - 1]
      const int src = i - 1;
      const ConvLayer& ps = u->L[src];
      k_maxpool_bwd<<<grid_for((int64_t)N * Hl * Wl * ps.cout / 8, u->n_sm), 256, 0, st>>>(
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
      cudaMalloc(&u->g0pad, 9ull * u->L[0].cin_pad * u->L[0].cout * 4) != cudaSuccess ||
      cudaMalloc(&u->d_err, sizeof(int)) != cudaSuccess)
    return fail_oom();
  cudaMemset(u->d_err, 0, sizeof(int));
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
  cudaFree(u->d_err);
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

extern "C" mem_status mem_unet_check(mem_unet* u, void* stream) {
  if (!u) return memh::api_fail(MEM_ERR_ARG, "NULL argument");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return memh::api_cuda_fail(e, "stream synchronize");
  int err = 0;
  e = cudaMemcpy(&err, u->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return memh::api_cuda_fail(e, "read error word");
  if (err) {
    cudaMemset(u->d_err, 0, sizeof(int));
    return memh::api_fail(MEM_ERR_TIMEOUT, "a bounded wait in a U-Net convolution ran out");
  }
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
  bool head_done = false;
  e = forward(u, n, H, W, st, fill, pred, &head_done);
  if (e != cudaSuccess) return memh::api_cuda_fail(e, "U-Net forward");
  if (!head_done)
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
