// Height-only point-cloud fuse into caller-owned buffers that allocates no
// device or pinned memory: the sort and segment scratch of the point path
// lives in one file-scope __device__ array of fixed size instead.
//
// Callers that cannot allocate -- code running inside another framework's
// memory pool, real-time loops that forbid allocation after start-up, or
// hosts whose device allocator is owned by someone else -- can still run the
// map update on buffers they already hold.
#include <math.h>
#include <stddef.h>
#include <string.h>

#include <mutex>

#include "mem_host.h"

namespace {

using memk::u32;

constexpr int64_t kMaxPts = MEM_NOALLOC_MAX_POINTS;
constexpr int64_t kTiles = (kMaxPts + memk::kSortTile - 1) / memk::kSortTile;
constexpr int64_t kAlign = 64;  // u32 words = 256 bytes
constexpr int64_t up(int64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
// word offsets of the sub-arrays
constexpr int64_t kKeys0 = 0;
constexpr int64_t kKeys1 = kKeys0 + up(kMaxPts + 4);
constexpr int64_t kVals0 = kKeys1 + up(kMaxPts + 4);
constexpr int64_t kVals1 = kVals0 + up(kMaxPts + 4);
constexpr int64_t kHist = kVals1 + up(kMaxPts + 4);           // 4*1024 digits + 16 counters
constexpr int64_t kLook = kHist + up(4 * 1024 + 16);           // 4 passes x tiles x 1024
constexpr int64_t kPart = kLook + up(4 * kTiles * 1024);       // fuse tile tables + slots
// error words: [0] a bounded wait of this call ran out (the point kernels then
// return at entry), [1] fault injection (always 0 here), [2] sticky record of
// timeouts since the last mem_noalloc_check
constexpr int64_t kErr = kPart + up(memk::fuse_scratch_words(kMaxPts, memk::kSlotHdr));
constexpr int64_t kJob = kErr + up(1);
struct JobBlock {
  memk::PointJob job;
  memk::MapCall mc;
};
constexpr int64_t kJobWords = up((sizeof(JobBlock) + 3) / 4);
constexpr int64_t kWords = kJob + kJobWords;

// every GPU that loads the library holds this array (about 22 MB) until exit
static __device__ __align__(256) u32 g_noalloc_scratch[kWords];

std::mutex g_mu;
void* g_addr[128] = {};
int g_nsm[128] = {};

// Writes the call's job block into the static array from the kernel's own
// parameters (passed by value, so nothing is read from host memory after the
// launch), and starts the call with a clear error word: a timeout of an
// earlier call is kept in the sticky word [2] instead.
__global__ void k_noalloc_job(JobBlock jb, u32* dst, int* err) {
  const u32* src = reinterpret_cast<const u32*>(&jb);
  constexpr int kw = (int)(sizeof(JobBlock) / 4);
  for (int i = threadIdx.x; i < kw; i += blockDim.x) dst[i] = src[i];
  if (threadIdx.x == 0) {
    if (err[0]) err[2] = err[0];
    err[0] = 0;
    err[1] = 0;
  }
}
static_assert(sizeof(JobBlock) % 4 == 0 && sizeof(JobBlock) <= 4000, "job block fits the kernel parameters");

// the array's device address on the current device (looked up once per device)
mem_status noalloc_base(int* dev_out, void** base, int* n_sm) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return memh::api_cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 128) return memh::api_fail(MEM_ERR_STATE, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return memh::api_cuda_fail(e, "cudaGetSymbolAddress");
    e = memh::prepare_kernels();
    if (e != cudaSuccess) return memh::api_cuda_fail(e, "kernel attributes");
    e = cudaDeviceGetAttribute(&g_nsm[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return memh::api_cuda_fail(e, "device attribute");
    g_addr[dev] = p;
  }
  *dev_out = dev;
  *base = g_addr[dev];
  if (n_sm) *n_sm = g_nsm[dev];
  return MEM_OK;
}

}  // namespace

extern "C" mem_status mem_fuse_pointcloud_noalloc(const mem_map_config* cfg, const double origin_xy[2],
                                                  int64_t n, const float* xyz,
                                                  const double T_map_sensor[16], float* h, float* var,
                                                  uint32_t* valid, uint32_t* n_acc, uint32_t* n_rej,
                                                  void* stream) {
  using namespace memk;
  if (!cfg || !origin_xy || !T_map_sensor || !h || !var || !valid || !n_acc || !n_rej)
    return memh::api_fail(MEM_ERR_ARG, "NULL argument");
  if (cfg->n_maps != 1 || cfg->n_layers != 0)
    return memh::api_fail(MEM_ERR_ARG, "the allocation-free fuse takes one map with no multi-modal layers");
  if (cfg->drift_alpha != 0.0 || cfg->ray_cleanup != 0)
    return memh::api_fail(MEM_ERR_ARG, "the allocation-free fuse runs without drift compensation and ray-cast clean-up");
  if (cfg->W < 2 || cfg->W > 16384 || (cfg->W & 1)) return memh::api_fail(MEM_ERR_ARG, "W must be even in [2, 16384]");
  if (!(cfg->res > 0.0)) return memh::api_fail(MEM_ERR_ARG, "res must be > 0");
  if (!(cfg->range_min <= cfg->range_max)) return memh::api_fail(MEM_ERR_ARG, "range_min > range_max");
  if (n < 0 || n > kMaxPts)
    return memh::api_fail(MEM_ERR_ARG, "n = %lld points exceeds the allocation-free limit of %lld",
                          (long long)n, (long long)kMaxPts);
  if (n > 0 && !xyz) return memh::api_fail(MEM_ERR_ARG, "xyz is NULL");
  for (int k = 0; k < 16; ++k)
    if (!isfinite(T_map_sensor[k])) return memh::api_fail(MEM_ERR_ARG, "pose not finite");

  // set-up, once per device, with that device current
  int dev = 0, n_sm = 0;
  void* base = nullptr;
  mem_status ms = noalloc_base(&dev, &base, &n_sm);
  if (ms != MEM_OK) return ms;
  u32* w = (u32*)base;

  memh::Map m;  // host-side description only; owns nothing
  m.cfg = *cfg;
  m.n_sm = n_sm;
  MapDev& md = m.md;
  memset(&md, 0, sizeof(md));  // drift compensation and clean-up off, their buffers absent
  md.W = cfg->W;
  md.n_maps = 1;
  md.W2 = (u32)cfg->W * (u32)cfg->W;
  md.sentinel = md.W2;
  md.res = (float)cfg->res;
  md.sigma0 = cfg->sigma0;
  md.sigma1 = cfg->sigma1;
  md.lam2 = cfg->gate_lambda * cfg->gate_lambda;
  md.outlier_var = cfg->outlier_var;
  md.time_var = cfg->time_var;
  md.range_min = cfg->range_min;
  md.range_max = cfg->range_max;
  md.z_near = cfg->z_near;
  md.n_layers = 0;
  md.h = h;
  md.var = var;
  md.flags = valid;
  md.n_acc = n_acc;
  md.n_rej = n_rej;
  md.keys0 = w + kKeys0;
  md.keys1 = w + kKeys1;
  md.vals0 = w + kVals0;
  md.vals1 = w + kVals1;
  md.hist = w + kHist;
  md.counters = md.hist + 4 * 1024;
  md.lookback = w + kLook;
  md.partial = (float*)(w + kPart);
  md.partial_cap = memk::fuse_scratch_words(kMaxPts, memk::kSlotHdr);
  md.err = (int*)(w + kErr);
  md.cap = kMaxPts;
  md.cap_tiles = kTiles;
  m.key_bits = memh::key_bits_for(&m);
  m.tune.radix_bits = m.key_bits <= 16 ? 8 : 9;
  m.passes = (m.key_bits + m.tune.radix_bits - 1) / m.tune.radix_bits;

  // the job block, in the same array
  JobBlock hj;
  memset(&hj, 0, sizeof(hj));
  u32* d_job = w + kJob;
  hj.job.n = n;
  hj.job.xyz = xyz;
  hj.job.offsets = nullptr;
  hj.job.maps = (const MapCall*)((char*)d_job + offsetof(JobBlock, mc));
  hj.job.n_maps = 1;
  hj.job.n_src = 0;
  hj.job.acc = memk::kSlotHdr;
  memh::build_fuse_tables(hj.job, memk::kSlotHdr, *cfg);
  m.fuse_variant = hj.job.ft.one_round ? 2 : 0;
  for (int r = 0; r < 3; ++r)
    for (int k = 0; k < 3; ++k) hj.mc.R[r * 3 + k] = (float)T_map_sensor[r * 4 + k];
  hj.mc.t[0] = (float)(T_map_sensor[3] - origin_xy[0]);
  hj.mc.t[1] = (float)(T_map_sensor[7] - origin_xy[1]);
  hj.mc.t[2] = (float)T_map_sensor[11];
  cudaStream_t st = (cudaStream_t)stream;
  k_noalloc_job<<<1, 128, 0, st>>>(hj, d_job, md.err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return memh::api_cuda_fail(e, "allocation-free job launch");
  // no points: only the time-dependent variance growth of the valid cells
  e = n == 0 ? memh::launch_time_update(&m, st) : memh::launch_point_fuse(&m, (const PointJob*)d_job, st);
  if (e != cudaSuccess) return memh::api_cuda_fail(e, "allocation-free fuse launch");
  return MEM_OK;
}

extern "C" mem_status mem_noalloc_check(void* stream) {
  int dev = 0;
  void* base = nullptr;
  mem_status ms = noalloc_base(&dev, &base, nullptr);
  if (ms != MEM_OK) return ms;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return memh::api_cuda_fail(e, "stream synchronize");
  int* err = (int*)((u32*)base + kErr);
  int w[3] = {0, 0, 0};
  e = cudaMemcpy(w, err, sizeof(w), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return memh::api_cuda_fail(e, "read error words");
  if (w[0] || w[2]) {
    e = cudaMemset(err, 0, sizeof(w));
    if (e != cudaSuccess) return memh::api_cuda_fail(e, "clear error words");
    return memh::api_fail(MEM_ERR_TIMEOUT, "an allocation-free fuse timed out in a bounded device wait "
                                           "and left the layers of that call unchanged");
  }
  return MEM_OK;
}
