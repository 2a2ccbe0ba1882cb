// shard.cu -- C-ABI of the sharded single-scene encode: one scene split over shards (ranks or
// streams), each shard coding whole chunks of the scene's slot order, with every decision taken
// from integer sums over the shards, so the result is the whole-scene call's, byte for byte
// (Sec. V-A: the 16 scales are order statistics of the whole scene; Sec. III-C: the reorder
// works chunk by chunk within the spatial order; Sec. IV-B: one rate budget for the scene).
#include <string.h>

#include "gsc_internal.cuh"

#define SEL_PASSES 4
#define RATE_PASSES 13

static bool al(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }
static bool n_ok(int64_t n) { return n >= 0 && n < (int64_t)0x7FFFFFF0; }

extern "C" size_t gsc_shard_order_ws_bytes(int64_t n_total) { return n_ok(n_total) ? shard_order_ws_bytes(n_total) : 0; }
extern "C" size_t gsc_shard_select_state_bytes(void) { return shard_select_state_bytes(); }
extern "C" size_t gsc_shard_plan_ws_bytes(int64_t n) { return n_ok(n) ? shard_plan_ws_bytes(n) : 0; }
extern "C" size_t gsc_shard_rate_ws_bytes(int64_t n) { return n_ok(n) ? shard_rate_ws_bytes(ceil_div64(n, 16)) : 0; }

extern "C" gsc_status gsc_shard_bounds(int64_t n_total, int32_t n_shards, int64_t group_size, int64_t* bounds) {
  if (!bounds || !n_ok(n_total) || n_shards < 1 || group_size <= 0 || group_size % 16 != 0) return GSC_ERR_INVALID_ARG;
  const int64_t chunks = ceil_div64(n_total, group_size);
  for (int32_t s = 0; s <= n_shards; s++) {
    const int64_t b = (chunks * s / n_shards) * group_size;
    bounds[s] = b < n_total ? b : n_total;
  }
  return GSC_OK;
}

extern "C" gsc_status gsc_shard_bbox(gsc_ctx* c, const float* d_pos, int64_t n, int64_t* d_bb, void* stream) {
  GscRange r_("gsc_shard_bbox");
  if (!c || !n_ok(n) || !d_bb || (n > 0 && !d_pos) || !al(d_pos, 4) || !al(d_bb, 8)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  GSC_CUDA(shard_bbox(d_pos, n, d_bb, c->sm_count, (cudaStream_t)stream));
  return GSC_OK;
}

extern "C" gsc_status gsc_shard_morton(gsc_ctx* c, const float* d_pos, int64_t n, const int64_t* d_bb, uint64_t* d_keys,
                                       void* stream) {
  GscRange r_("gsc_shard_morton");
  if (!c || !n_ok(n) || !d_bb || (n > 0 && (!d_pos || !d_keys)) || !al(d_pos, 4) || !al(d_bb, 8) || !al(d_keys, 8))
    return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  GSC_CUDA(shard_morton(d_pos, n, d_bb, d_keys, c->sm_count, (cudaStream_t)stream));
  return GSC_OK;
}

extern "C" gsc_status gsc_shard_order(gsc_ctx* c, uint64_t* d_keys, int64_t n_total, int32_t* d_order, void* d_ws,
                                      size_t ws_bytes, void* stream) {
  GscRange r_("gsc_shard_order");
  if (!c || !n_ok(n_total) || (n_total > 0 && (!d_keys || !d_order || !d_ws))) return GSC_ERR_INVALID_ARG;
  if (!al(d_keys, 8) || !al(d_order, 4) || !al(d_ws, 256)) return GSC_ERR_INVALID_ARG;
  if (n_total > 0 && ws_bytes < shard_order_ws_bytes(n_total)) return GSC_ERR_OOM;
  GSC_CUDA(cudaSetDevice(c->device));
  GSC_CUDA(shard_order(d_keys, n_total, d_order, d_ws, c->sm_count, (cudaStream_t)stream));
  return GSC_OK;
}

extern "C" gsc_status gsc_shard_select_begin(gsc_ctx* c, int64_t n_total, uint32_t permille, void* d_state,
                                             void* stream) {
  GscRange r_("gsc_shard_select_begin");
  if (!c || !n_ok(n_total) || !d_state || !al(d_state, 256) || permille == 0 || permille > 1000)
    return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  GSC_CUDA(shard_select_begin(n_total, (int)permille, d_state, (cudaStream_t)stream));
  return GSC_OK;
}

extern "C" gsc_status gsc_shard_select_hist(gsc_ctx* c, const float* d_sh, int64_t n, int32_t pass, void* d_state,
                                            int64_t* d_hist, void* stream) {
  GscRange r_("gsc_shard_select_hist");
  if (!c || !n_ok(n) || pass < 0 || pass >= SEL_PASSES || !d_state || !d_hist || (n > 0 && !d_sh))
    return GSC_ERR_INVALID_ARG;
  if (!al(d_sh, 16) || !al(d_state, 256) || !al(d_hist, 8)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  GSC_CUDA(shard_select_hist(d_sh, n, 24 - 8 * pass, d_state, d_hist, c->sm_count, (cudaStream_t)stream));
  return GSC_OK;
}

extern "C" gsc_status gsc_shard_select_pick(gsc_ctx* c, void* d_state, const int64_t* d_hist, int32_t pass,
                                            void* stream) {
  GscRange r_("gsc_shard_select_pick");
  if (!c || pass < 0 || pass >= SEL_PASSES || !d_state || !d_hist || !al(d_state, 256) || !al(d_hist, 8))
    return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  GSC_CUDA(shard_select_pick(d_state, d_hist, 24 - 8 * pass, (cudaStream_t)stream));
  return GSC_OK;
}

extern "C" gsc_status gsc_shard_select_scales(gsc_ctx* c, const void* d_state, float* d_scales, void* stream) {
  GscRange r_("gsc_shard_select_scales");
  if (!c || !d_state || !d_scales || !al(d_state, 256) || !al(d_scales, 4)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  GSC_CUDA(shard_select_scales(d_state, d_scales, (cudaStream_t)stream));
  return GSC_OK;
}

extern "C" gsc_status gsc_shard_plan(gsc_ctx* c, const float* d_sh, int64_t n, const float* d_scales,
                                     int64_t group_size, int32_t* d_perm, void* d_ws, size_t ws_bytes, void* stream) {
  GscRange r_("gsc_shard_plan");
  if (!c || !n_ok(n) || !d_scales || group_size <= 0 || group_size % 16 != 0) return GSC_ERR_INVALID_ARG;
  if (n > 0 && (!d_sh || !d_perm || !d_ws)) return GSC_ERR_INVALID_ARG;
  if (!al(d_sh, 16) || !al(d_perm, 4) || !al(d_ws, 256)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  GscTimed tm(c, T_PLAN, (cudaStream_t)stream);
  return shard_plan(d_sh, n, d_scales, group_size, d_perm, d_ws, ws_bytes, c->sm_count, (cudaStream_t)stream);
}

static bool rate_ws_ok(int64_t n, const void* d_ws) { return n_ok(n) && d_ws && al(d_ws, 256); }

extern "C" gsc_status gsc_shard_rate_begin(gsc_ctx* c, const float* d_sh, int64_t n, const int32_t* d_perm,
                                           const float* d_scales, uint8_t* d_bc1, uint8_t* d_bc7, void* d_ws,
                                           size_t ws_bytes, int64_t* d_part, void* stream) {
  GscRange r_("gsc_shard_rate_begin");
  if (!c || !rate_ws_ok(n, d_ws) || !d_scales || !d_part || !al(d_part, 8)) return GSC_ERR_INVALID_ARG;
  if (n > 0 && (!d_sh || !d_perm || !d_bc1 || !d_bc7)) return GSC_ERR_INVALID_ARG;
  if (!al(d_sh, 16) || !al(d_bc1, 16) || !al(d_bc7, 16) || !al(d_perm, 4)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  return shard_rate_begin(c, d_sh, n, d_perm, d_scales, d_bc1, d_bc7, d_ws, ws_bytes, d_part, (cudaStream_t)stream);
}

extern "C" gsc_status gsc_shard_rate_search_begin(gsc_ctx* c, int64_t n, void* d_ws, int64_t n_total, uint32_t target_x4,
                                                  const int64_t* d_min_total, void* stream) {
  GscRange r_("gsc_shard_rate_search_begin");
  if (!c || !rate_ws_ok(n, d_ws) || !n_ok(n_total) || n > n_total || !d_min_total || !al(d_min_total, 8))
    return GSC_ERR_INVALID_ARG;
  if (target_x4 == 0 || target_x4 > 64) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  return shard_rate_search_begin(ceil_div64(n, 16), d_ws, n_total, target_x4, d_min_total, (cudaStream_t)stream);
}

extern "C" gsc_status gsc_shard_rate_count(gsc_ctx* c, int64_t n, void* d_ws, int32_t pass, int64_t* d_part,
                                           void* stream) {
  GscRange r_("gsc_shard_rate_count");
  if (!c || !rate_ws_ok(n, d_ws) || pass < 0 || pass >= RATE_PASSES || !d_part || !al(d_part, 8))
    return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  return shard_rate_count(c, ceil_div64(n, 16), d_ws, pass, d_part, (cudaStream_t)stream);
}

extern "C" gsc_status gsc_shard_rate_narrow(gsc_ctx* c, int64_t n, void* d_ws, int32_t pass, const int64_t* d_total,
                                            void* stream) {
  GscRange r_("gsc_shard_rate_narrow");
  if (!c || !rate_ws_ok(n, d_ws) || pass < 0 || pass >= RATE_PASSES || !d_total || !al(d_total, 8))
    return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  return shard_rate_narrow(ceil_div64(n, 16), d_ws, pass, d_total, (cudaStream_t)stream);
}

extern "C" gsc_status gsc_shard_rate_fill(gsc_ctx* c, int64_t n, void* d_ws, int64_t* d_part, void* stream) {
  GscRange r_("gsc_shard_rate_fill");
  if (!c || !rate_ws_ok(n, d_ws) || !d_part || !al(d_part, 8)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  return shard_rate_fill(c, ceil_div64(n, 16), d_ws, d_part, (cudaStream_t)stream);
}

extern "C" gsc_status gsc_shard_rate_apply(gsc_ctx* c, int64_t n, void* d_ws, const int64_t* d_in, int64_t* d_part,
                                           void* stream) {
  GscRange r_("gsc_shard_rate_apply");
  if (!c || !rate_ws_ok(n, d_ws) || !d_in || !d_part || !al(d_in, 8) || !al(d_part, 8)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  return shard_rate_apply(c, ceil_div64(n, 16), d_ws, d_in, d_part, (cudaStream_t)stream);
}

extern "C" gsc_status gsc_shard_rate_assemble(gsc_ctx* c, int64_t n, void* d_ws, const uint8_t* d_bc1,
                                              const uint8_t* d_bc7, const int32_t* d_perm, const int32_t* d_index_map,
                                              const float* d_scales, const int64_t* d_parts_all, int32_t n_shards,
                                              int32_t shard, int64_t n_total, uint8_t* d_blocks, int32_t* d_perm_out,
                                              gsc_stream_table* h_table, void* stream) {
  GscRange r_("gsc_shard_rate_assemble");
  if (!c || !rate_ws_ok(n, d_ws) || !d_scales || !d_parts_all || !h_table || !n_ok(n_total) || n > n_total)
    return GSC_ERR_INVALID_ARG;
  if (n_shards < 1 || shard < 0 || shard >= n_shards) return GSC_ERR_INVALID_ARG;
  if (n > 0 && (!d_bc1 || !d_bc7 || !d_perm || !d_blocks || !d_perm_out)) return GSC_ERR_INVALID_ARG;
  if (!al(d_bc1, 16) || !al(d_bc7, 16) || !al(d_blocks, 16) || !al(d_perm, 4) || !al(d_perm_out, 4) ||
      !al(d_index_map, 4) || !al(d_parts_all, 8))
    return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  memset(h_table, 0, sizeof(*h_table));
  GscTimed tm(c, T_RATE, st);
  gsc_status s = shard_rate_assemble(c, ceil_div64(n, 16), d_ws, d_bc1, d_bc7, d_perm, d_index_map, d_parts_all,
                                     n_shards, shard, n_total, d_blocks, d_perm_out, h_table, st);
  if (s != GSC_OK) return s;
  float* hs = reinterpret_cast<float*>(c->h_pinned);
  GSC_CUDA(cudaMemcpyAsync(hs, d_scales, sizeof(float) * GSC_SH, cudaMemcpyDeviceToHost, st));
  GSC_CUDA(cudaStreamSynchronize(st));
  memcpy(h_table->scales, hs, sizeof(float) * GSC_SH);
  return GSC_OK;
}
