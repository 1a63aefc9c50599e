// Host-side map object shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "mem_internal.cuh"

namespace memh {

constexpr int kJobSlots = 8;

struct Tuning {
  int radix_bits = 9;   // digit width of the radix sort (8..10)
  int blocks_per_sm = 4;
  int fuse_kernel = 0;   // 0: the warp fuse kernel where a call's columns fit one round; 1: the tile kernel
};

struct Map {
  mem_map_config cfg;
  memk::MapDev md;
  memk::LayerDev Lh[memk::kMaxLayers];  // host copy of the device layer table md.L
  Tuning tune;
  int passes = 1;
  int key_bits = 1;
  uint32_t call_id = 0;  // point-path calls so far (the clean-up's per-cell stamps)
  // fuse kernel variant of the current point-path call: bit 0 a source has top-k rows,
  // bit 1 its columns fit one round (the warp kernel runs instead of the tile kernel)
  int fuse_variant = 0;
  int graph_variant = -1;  // the variant the captured graph launches
  int n_sm = 148;
  int device = 0;
  std::vector<double> origin;  // [n_maps][2] world xy of each map centre
  std::vector<int> ring;       // [n_maps][2] ring-buffer offsets (physical = logical + ring mod W)
  // device job block and pinned staging slots
  char* d_job = nullptr;
  size_t job_bytes = 0;
  char* h_job[kJobSlots] = {};
  cudaEvent_t job_ev[kJobSlots] = {};
  int job_slot = 0;
  // CUDA graph of the batched point path
  cudaGraphExec_t graph = nullptr;
  cudaStream_t graph_stream = nullptr;
  bool use_graph = true;
  // optional per-kernel timing (CUDA events around each launch group)
  bool prof_on = false;
  struct ProfMark {
    int slot;
    cudaEvent_t a, b;
  };
  std::vector<ProfMark> prof_pending;
  std::vector<cudaEvent_t> prof_pool;  // events of the pending marks, reused after each read
  size_t prof_next = 0;
  double prof_ms[16] = {};
  int64_t prof_calls[16] = {};
  // host-buffer fuse: two device staging buffers used in turn, filled on a
  // copy stream of the map's own so that a call's upload overlaps the
  // previous call's kernels
  void* stage_buf[2] = {};
  size_t stage_cap[2] = {};
  cudaEvent_t stage_copied[2] = {}, stage_done[2] = {};
  cudaStream_t copy_stream = nullptr;
  int stage_slot = 0;
  // scratch of the PCA plugin (grown on demand)
  void* pca_buf = nullptr;
  size_t pca_cap = 0;
  void* img_buf = nullptr;  // image fusion: the list of cells to walk
  size_t img_cap = 0;
  // allocations to free
  std::vector<void*> allocs;
  std::vector<void*> scratch_allocs;
};

// profile slots
enum { kProfKey = 0, kProfDigits, kProfSort, kProfUnused3, kProfFuseTiles, kProfFuseCross,
       kProfTime, kProfImage, kProfMove, kProfDrift, kProfRay, kProfSlots };

// Brackets a launch group with events when profiling is on. Events come from a
// pool the map keeps (created on first use, reused after each read of the
// profile), so recording costs no event creation between the launches.
inline cudaEvent_t prof_event(Map* m) {
  if (m->prof_next < m->prof_pool.size()) return m->prof_pool[m->prof_next++];
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  m->prof_pool.push_back(e);
  ++m->prof_next;
  return e;
}

struct ProfScope {
  Map* m;
  int slot;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  ProfScope(Map* m_, int slot_, cudaStream_t st_) : m(m_), slot(slot_), st(st_) {
    if (m->prof_on && (a = prof_event(m)) != nullptr) cudaEventRecord(a, st);
  }
  ~ProfScope() {
    if (!a) return;
    cudaEvent_t b = prof_event(m);
    if (!b) return;
    cudaEventRecord(b, st);
    m->prof_pending.push_back({slot, a, b});
  }
};

cudaError_t alloc_scratch(Map* m, int64_t cap);
void free_scratch(Map* m);
int key_bits_for(const Map* m);
cudaError_t prepare_kernels();
// time-dependent variance growth of every valid cell (no-op when time_var == 0)
cudaError_t launch_time_update(Map* m, cudaStream_t st);
// stage layout and rule-layer lists of a point-path call (job.src, n_src and
// the raw slot length `acc_raw` set), as the fuse kernel reads them
void build_fuse_tables(memk::PointJob& job, int acc_raw, const mem_map_config& cfg);
mem_status api_fail(mem_status s, const char* fmt, ...);
Map* map_of(mem_map* mm);
mem_status api_cuda_fail(cudaError_t e, const char* what);

}  // namespace memh
