// gsc_internal.cuh -- shared declarations of the CUDA library's translation units.
#pragma once

#include <nvtx3/nvToolsExt.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gsc.h"

#define GSC_SH 16
#define GSC_MODES 14

enum { T_PLAN = 0, T_BC1, T_BC7, T_RATE, T_DECODE, T_EVAL, T_TEX, T_EVAL_TEX, T_BATCH, T_RENDER, T_BLEND, T_COUNT };

struct gsc_timer_rec { int id; cudaEvent_t a, b; };

struct gsc_tex_slot {
  cudaArray_t arr;
  cudaTextureObject_t tex;
  int64_t nblk;
};

struct gsc_ctx {
  int device;
  gsc_tex_slot tex[2];        // texture path: [0] BC1, [1] BC7, kept between calls
  uint8_t* tex_lin[2];
  size_t tex_lin_bytes[2];
  int sm_count;
  int timing;                 // record events around kernels
  gsc_timer_rec* recs;        // pending records
  int n_recs, cap_recs;
  double t_ms[T_COUNT];
  int64_t t_launches[T_COUNT];
  int* d_status;        // first device-side error code (0 = none)
  int* d_diag;          // where it happened (kernel-defined)
  void* h_pinned;       // small pinned host buffer for table read-back
  size_t h_pinned_bytes;
};

#define GSC_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return GSC_ERR_CUDA;          \
  } while (0)

static inline int64_t ceil_div64(int64_t a, int64_t b) { return (a + b - 1) / b; }
static inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Host-side count of kernel launches (measurement only).
void gsc_count_launch();
// Streaming multiprocessors of the current device (queried once per device; grids are sized from it).
int gsc_sm_count();
// Event pair around a kernel when the context's timing is on (measurement only).
int gsc_timer_begin(gsc_ctx* c, int id, cudaStream_t st);
void gsc_timer_end(gsc_ctx* c, int rec, cudaStream_t st);
struct GscTimed {
  gsc_ctx* c; int rec; cudaStream_t st;
  GscTimed(gsc_ctx* c_, int id, cudaStream_t st_) : c(c_), rec(gsc_timer_begin(c_, id, st_)), st(st_) {}
  ~GscTimed() { gsc_timer_end(c, rec, st); }
};

// NVTX range over one C-ABI call (header-only NVTX 3: a no-op unless a profiler is attached), so
// timelines show each call with its kernels.
struct GscRange {
  explicit GscRange(const char* name) { nvtxRangePushA(name); }
  ~GscRange() { nvtxRangePop(); }
};

// Records the first device-detected error into the context status word.
__device__ __forceinline__ void gsc_record(int* status, int* diag, int code, int where) {
  if (atomicCAS(status, 0, code) == 0 && diag) *diag = where;
}

// 8-bit quantisation of Sec. V-A: q = clamp(128 + rint(fl(fl(x / s) * 255)), 0, 255).
__device__ __forceinline__ uint32_t gsc_quant1(float x, float s) {
  float t = __fmul_rn(__fdiv_rn(x, s), 255.0f);
  t = fminf(fmaxf(t, -256.0f), 256.0f);  // NaN-free inputs assumed; clamping first keeps rint in range
  int q = 128 + __float2int_rn(t);
  return (uint32_t)min(max(q, 0), 255);
}

// Bump allocator over a caller-provided workspace (256-byte aligned pieces).
struct Carve {
  uint8_t* base;
  size_t off, cap;
  template <class T> T* take(int64_t count) {
    off = align_up(off, 256);
    T* p = reinterpret_cast<T*>(base + off);
    off += sizeof(T) * (size_t)(count > 0 ? count : 1);
    return p;
  }
  bool ok() const { return off <= cap; }
};

// Checked build (GSC_CHECKED): takes and clears the first slot-order check failure recorded by
// the decode kernels on the current device (GSC_ERR_DEVICE and the slot), or 0.
int gsc_check_take(int* where);

// A context on `device`; init_tables = false skips the constant tables (already loaded by an
// earlier context in this process), as the request loop's per-slot contexts do.
gsc_status ctx_new(int device, bool init_tables, gsc_ctx** out);

// ---- launchers implemented by the translation units ------------------------------
// plan.cu
size_t plan_ws_bytes(int64_t n);
gsc_status plan_run(gsc_ctx* ctx, const float* pos, const float* sh, const gsc_plan_params* pp, int32_t* perm,
                    float* scales, void* ws, size_t ws_bytes, cudaStream_t st);
cudaError_t launch_quantise(const float* sh, int64_t n, const float* scales, uint8_t* q, cudaStream_t st);
size_t radix_ws_bytes(int64_t n);
size_t scan_ws_bytes(int64_t n);
// Exclusive scan of n values (uint32 or uint64); *total (device, optional) gets the sum.
template <class T>
cudaError_t scan_exclusive(const T* in, T* out, int64_t n, uint64_t* total, void* ws, cudaStream_t st);
// Stable LSD radix sort of (64-bit key, 32-bit value) pairs on the low key_bits bits.
// Result lands in keys/vals (the input arrays); ws holds the ping-pong buffers.
cudaError_t radix_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t n, int key_bits, void* ws, cudaStream_t st);

// bc1.cu
cudaError_t bc1_init_tables();
// Group kernel: stage layout-D texels from sh/perm/scales and code all 16 blocks of
// each group; blocks [g][k][8]; sse1 / sse0 [g][k] optional (BC1 error, error of 128).
cudaError_t launch_bc1_groups(const float* sh, const int32_t* perm, const float* scales, int64_t n_groups,
                              uint8_t* blocks, uint32_t* sse1, uint32_t* sse0, cudaStream_t st);
cudaError_t launch_bc1_blocks(const uint8_t* tex, int64_t nblk, uint8_t* out, uint64_t* sse, cudaStream_t st);

// bc7.cu
cudaError_t bc7_init_tables();
cudaError_t launch_bc7_groups(const float* sh, const int32_t* perm, const float* scales, int64_t n_groups,
                              uint8_t* blocks, uint32_t* sse7, cudaStream_t st);
cudaError_t launch_bc7_blocks(const uint8_t* tex, int64_t nblk, uint8_t* out, uint64_t* sse, cudaStream_t st);
// Persistent multi-scene encode. Scenes are listed in schedule order; scene i owns tiles
// [tile0, tile0 + n_tiles) of tile_groups groups each (a multiple of 8) over its first
// work_groups groups, coded BC1 (kind 1, optionally with the per-block errors of BC1 and of
// the zero coding that the rate control needs) or BC7 (kind 7, optionally with its errors).
struct BatchSceneDev {
  const float* sh;
  const int32_t* perm;
  const float* scales;
  int64_t n_groups, work_groups;
  int64_t tile0, n_tiles;
  int32_t kind, tile_groups;
  uint8_t* b1;
  uint8_t* b7;
  uint32_t *sse1, *sse7, *sse0;
};
// kind 1 or 7: every listed scene must be of that kind.
cudaError_t launch_batch_encode(int kind, const BatchSceneDev* scenes, int n_scenes, int64_t n_tiles, int schedule,
                                int ctas_per_sm, int sm_count, int* counter, cudaStream_t st);

// rate.cu
size_t rate_ws_bytes(int64_t n_groups);
size_t rate_select_ws_bytes(int64_t n_groups);
gsc_status rate_select(gsc_ctx* ctx, int64_t n, const int32_t* perm, const float* scales, uint32_t target_x4,
                       const uint8_t* b1, const uint8_t* b7, const uint32_t* sse1, const uint32_t* sse7,
                       const uint32_t* sse0, uint8_t* blocks, int32_t* perm_out, gsc_stream_table* table, void* ws,
                       size_t ws_bytes, cudaStream_t st);
gsc_status rate_run(gsc_ctx* ctx, const float* sh, int64_t n, const int32_t* perm, const float* scales,
                    uint32_t target_x4, uint8_t* blocks, int32_t* perm_out, gsc_stream_table* table, void* ws,
                    size_t ws_bytes, uint8_t* bc1_all, uint8_t* bc7_all, cudaStream_t st);

// layout.cu: fixed codings of any layout with j BC7 blocks per group (texels staged in ws)
size_t layout_ws_bytes(int64_t n_groups, int j);
gsc_status layout_encode_run(gsc_ctx* ctx, const float* sh, int64_t n, const int32_t* perm, const float* scales,
                             int layout, int j, uint8_t* blocks, void* ws, size_t ws_bytes, cudaStream_t st);

// decode.cu
cudaError_t decode_init_tables();
// Flattened stream table for kernels (passed by value).
struct DevTable {
  int32_t n_streams;
  int32_t n;
  int32_t n_groups;
  int32_t bands[GSC_MODES], bc7[GSC_MODES];
  int64_t first_group[GSC_MODES], stream_groups[GSC_MODES], byte_offset[GSC_MODES];
  float scales[GSC_SH];
  int32_t layout;  // gsc_layout
};
// Band weights of the rate-distortion objective from the 16 scales (fp64, Sec. IV-B).
void host_weights(const float* scales, uint32_t* w);
gsc_status make_dev_table(const gsc_stream_table* t, DevTable* d);
cudaError_t launch_decode(const DevTable& t, const uint8_t* blocks, const int32_t* perm, uint8_t* texels,
                          cudaStream_t st);
// glist (optional): evaluate only the groups glist[0, n_list) (-1 entries skipped); pos_slot
// (optional): centres in slot order [n_groups * 16][3], read instead of pos[perm[s]]
cudaError_t launch_decode_eval(const DevTable& t, const uint8_t* blocks, const int32_t* perm, const float* dirs,
                               const float* pos, const float* cams, int V, int out_order, float* rgb, int sm_count,
                               cudaStream_t st, const int32_t* glist = nullptr, int64_t n_list = 0,
                               const float* pos_slot = nullptr);
cudaError_t launch_decode_blocks(const uint8_t* blocks, int64_t nblk, int format, uint8_t* rgba, cudaStream_t st);
// centres in slot order: out[s] = pos[perm[s]] (0 for padding slots), s < ns
cudaError_t launch_pos_to_slots(const float* pos, const int32_t* perm, int64_t n, int64_t ns, float* out, int sm_count,
                                cudaStream_t st);
gsc_status decode_tex_run(gsc_ctx* ctx, const DevTable& t, const uint8_t* blocks, const int32_t* perm,
                          uint8_t* texels, cudaStream_t st);
void tex_cache_free(gsc_ctx* ctx);
gsc_status decode_blocks_tex_run(gsc_ctx* ctx, const uint8_t* blocks, int64_t nblk, int format, uint8_t* rgba,
                                 cudaStream_t st);

// Sharded single-scene encode (plan.cu, rate.cu)
cudaError_t shard_bbox(const float* pos, int64_t n, int64_t* bb, int sm_count, cudaStream_t st);
cudaError_t shard_morton(const float* pos, int64_t n, const int64_t* bb, uint64_t* keys, int sm_count, cudaStream_t st);
size_t shard_order_ws_bytes(int64_t n);
cudaError_t shard_order(uint64_t* keys, int64_t n, int32_t* order, void* ws, int sm_count, cudaStream_t st);
size_t shard_select_state_bytes();
cudaError_t shard_select_begin(int64_t n_total, int permille, void* state, cudaStream_t st);
cudaError_t shard_select_hist(const float* sh, int64_t n, int shift, void* state, int64_t* hist, int sm_count,
                              cudaStream_t st);
cudaError_t shard_select_pick(void* state, const int64_t* hist_total, int shift, cudaStream_t st);
cudaError_t shard_select_scales(const void* state, float* scales, cudaStream_t st);
size_t shard_plan_ws_bytes(int64_t n);
gsc_status shard_plan(const float* sh, int64_t n, const float* scales, int64_t group_size, int32_t* perm, void* ws,
                      size_t ws_bytes, int sm_count, cudaStream_t st);
size_t shard_rate_ws_bytes(int64_t ng);
gsc_status shard_rate_begin(gsc_ctx* ctx, const float* sh, int64_t n, const int32_t* perm, const float* scales,
                            uint8_t* b1, uint8_t* b7, void* ws, size_t ws_bytes, int64_t* part, cudaStream_t st);
gsc_status shard_rate_search_begin(int64_t ng, void* ws, int64_t n_total, uint32_t target_x4, const int64_t* min_total,
                                   cudaStream_t st);
gsc_status shard_rate_count(gsc_ctx* ctx, int64_t ng, void* ws, int pass, int64_t* part, cudaStream_t st);
gsc_status shard_rate_narrow(int64_t ng, void* ws, int pass, const int64_t* total, cudaStream_t st);
gsc_status shard_rate_fill(gsc_ctx* ctx, int64_t ng, void* ws, int64_t* part, cudaStream_t st);
gsc_status shard_rate_apply(gsc_ctx* ctx, int64_t ng, void* ws, const int64_t* in, int64_t* part, cudaStream_t st);
gsc_status shard_rate_assemble(gsc_ctx* ctx, int64_t ng, void* ws, const uint8_t* b1, const uint8_t* b7,
                               const int32_t* perm, const int32_t* index_map, const int64_t* counts_all, int n_shards,
                               int shard, int64_t n_total, uint8_t* blocks, int32_t* perm_out, gsc_stream_table* table,
                               cudaStream_t st);
// bc7.cu: the mode-1 search alone, thread per block (warp = 0) or warp per block (1)
cudaError_t launch_bc7_mode1(const uint8_t* tex, int64_t nblk, int warp, uint32_t* sse, int32_t* part, int sm_count,
                             cudaStream_t st);
