// batch.cu -- many scenes of uneven sizes through one persistent encode launch, and the
// decode + SH evaluation of many scenes as one captured CUDA graph. Per scene the bits are
// the single-scene calls' (Sec. III-C plan, Sec. IV-B layout and streams, Sec. III-B codes).
#include <algorithm>
#include <string.h>
#include <vector>

#include "gsc_internal.cuh"

struct gsc_graph {
  int device;
  int kernels;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

// the scales of every scene come back through the context's 64 KB pinned buffer
static const int kMaxScenes = 1024;

static bool batch_args_ok(const gsc_batch_scene* sc, int n) {
  if (!sc || n <= 0 || n > kMaxScenes) return false;
  for (int i = 0; i < n; i++) {
    const gsc_batch_scene& s = sc[i];
    if (s.n < 0 || s.n >= (int64_t)0x7FFFFFF0) return false;
    if (s.group_size < 0 || s.group_size % 16 != 0 || (s.sort != 0 && s.sort != 1)) return false;
    if (s.format != GSC_FMT_BC1 && s.format != GSC_FMT_BC7 && s.format != GSC_FMT_RATE) return false;
    if (s.format == GSC_FMT_RATE && (s.target_bpt_x4 == 0 || s.target_bpt_x4 > 64)) return false;
    if (!s.d_scales) return false;
    if (s.n > 0 && (!s.d_sh || !s.d_perm || !s.d_blocks || !s.d_perm_out || (s.sort && !s.d_pos))) return false;
    if (((uintptr_t)s.d_sh % 16) != 0 || ((uintptr_t)s.d_blocks % 16) != 0) return false;
  }
  return true;
}

static int64_t groups_of(int64_t n) { return ceil_div64(n, 16); }

static const int kPlanLanes = 4;
// The autotuner's proxy: every scene's first 1/8 of the groups. Smaller proxies leave too few
// tiles per CTA and favour launch shapes that lose at full size.
static const int64_t kProxyDiv = 8;

struct BatchLayout {
  size_t plan_ws, select_ws, per_rate, total;
};

static BatchLayout layout(const gsc_batch_scene* sc, int n) {
  BatchLayout L = {0, 0, 0, 0};
  for (int i = 0; i < n; i++) {
    L.plan_ws = std::max(L.plan_ws, plan_ws_bytes(sc[i].n));
    if (sc[i].format == GSC_FMT_RATE) {
      const int64_t ng = groups_of(sc[i].n), nb = ng * 16;
      L.per_rate += align_up(8 * (size_t)nb, 256) + align_up(16 * (size_t)nb, 256) + 3 * align_up(4 * (size_t)nb, 256);
      L.select_ws = std::max(L.select_ws, rate_select_ws_bytes(ng));
    }
  }
  // the device scene list holds up to two entries per scene (a rate scene codes BC1 and BC7)
  L.plan_ws = align_up(L.plan_ws, 256);
  L.total = L.plan_ws * (size_t)std::min(n, kPlanLanes) + align_up(L.select_ws, 256) + L.per_rate +
            align_up(sizeof(BatchSceneDev) * 2 * (size_t)n, 256) + 256 + 4096;
  return L;
}

extern "C" size_t gsc_batch_workspace_bytes(const gsc_batch_scene* scenes, int32_t n_scenes) {
  if (!batch_args_ok(scenes, n_scenes)) return 0;
  return layout(scenes, n_scenes).total;
}

struct BatchBufs {
  void* plan_ws;
  void* select_ws;
  BatchSceneDev* d_list;
  size_t list_cap;
  bool fits;
  int* counter;
  std::vector<uint8_t*> b1, b7;
  std::vector<uint32_t*> s1, s7, s0;
};

static BatchBufs carve(const gsc_batch_scene* sc, int n, void* ws) {
  const BatchLayout L = layout(sc, n);
  Carve c{reinterpret_cast<uint8_t*>(ws), 0, L.total};
  BatchBufs B;
  B.plan_ws = c.take<uint8_t>((int64_t)(L.plan_ws * (size_t)std::min(n, kPlanLanes)));
  B.select_ws = c.take<uint8_t>((int64_t)L.select_ws);
  B.d_list = c.take<BatchSceneDev>(2 * (int64_t)n);
  B.list_cap = 2 * (size_t)n;
  B.counter = c.take<int>(64);
  B.b1.assign(n, nullptr); B.b7.assign(n, nullptr);
  B.s1.assign(n, nullptr); B.s7.assign(n, nullptr); B.s0.assign(n, nullptr);
  for (int i = 0; i < n; i++) {
    if (sc[i].format != GSC_FMT_RATE) continue;
    const int64_t nb = groups_of(sc[i].n) * 16;
    B.b1[i] = c.take<uint8_t>(8 * nb);
    B.b7[i] = c.take<uint8_t>(16 * nb);
    B.s1[i] = c.take<uint32_t>(nb);
    B.s7[i] = c.take<uint32_t>(nb);
    B.s0[i] = c.take<uint32_t>(nb);
  }
  B.fits = c.ok();
  return B;
}

// The plans are short, latency-bound launch sequences with no host synchronisation: run them
// on kPlanLanes streams at once (each with its own workspace), forked from and joined back
// into the caller's stream; scenes go to the lane with the least work so far.
static gsc_status run_plans(gsc_ctx* c, gsc_batch_scene* sc, int n, const BatchBufs& B, cudaStream_t st) {
  const int lanes = std::min(n, kPlanLanes);
  const size_t pws = layout(sc, n).plan_ws;
  cudaStream_t ls[kPlanLanes] = {};
  cudaEvent_t fork = nullptr, join[kPlanLanes] = {};
  gsc_status s = GSC_OK;
  cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  for (int l = 0; l < lanes && e == cudaSuccess; l++) {
    e = cudaStreamCreateWithFlags(&ls[l], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[l], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventRecord(fork, st);
  for (int l = 0; l < lanes && e == cudaSuccess; l++) e = cudaStreamWaitEvent(ls[l], fork, 0);
  if (e == cudaSuccess) {
    std::vector<int> order(n);
    for (int i = 0; i < n; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sc[a].n > sc[b].n; });
    int64_t load[kPlanLanes] = {};
    for (int i : order) {
      int l = 0;
      for (int k = 1; k < lanes; k++) if (load[k] < load[l]) l = k;
      load[l] += sc[i].n + 20000;  // a plan's fixed launch cost counts like ~20k Gaussians
      gsc_plan_params pp;
      pp.n = sc[i].n;
      pp.group_size = sc[i].group_size;
      pp.sort = sc[i].sort;
      pp.quantile_permille = 995;
      s = plan_run(c, sc[i].d_pos, sc[i].d_sh, &pp, sc[i].d_perm, sc[i].d_scales,
                   static_cast<uint8_t*>(B.plan_ws) + (size_t)l * pws, pws, ls[l]);
      if (s != GSC_OK) break;
    }
  }
  for (int l = 0; l < lanes; l++) {
    if (ls[l] && join[l]) {
      if (e == cudaSuccess) e = cudaEventRecord(join[l], ls[l]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, join[l], 0);
    }
  }
  for (int l = 0; l < lanes; l++) {
    if (join[l]) cudaEventDestroy(join[l]);
    if (ls[l]) cudaStreamDestroy(ls[l]);
  }
  if (fork) cudaEventDestroy(fork);
  if (e != cudaSuccess) { cudaGetLastError(); return GSC_ERR_CUDA; }
  return s;
}

// Scene list in schedule order with tile ranges; work_div shrinks every scene's work
// (the autotuner's proxy), 1 = the real batch.
// n_tiles[0] / [1]: tiles of the BC7 and of the BC1 entries.
static std::vector<BatchSceneDev> scene_list(const gsc_batch_scene* sc, int n, const BatchBufs& B,
                                             const gsc_batch_tuning& tune, int64_t work_div, int64_t* n_tiles) {
  std::vector<BatchSceneDev> v;
  for (int i = 0; i < n; i++) {
    const int64_t ng = groups_of(sc[i].n);
    if (ng == 0) continue;
    BatchSceneDev d;
    memset(&d, 0, sizeof(d));
    d.sh = sc[i].d_sh;
    d.perm = sc[i].d_perm;
    d.scales = sc[i].d_scales;
    d.n_groups = ng;
    d.work_groups = work_div > 1 ? std::min(ng, std::max<int64_t>(8, ng / work_div / 8 * 8)) : ng;
    // a rate scene is listed twice: its BC1 coding (with both error terms) and its BC7 coding
    const bool rate = sc[i].format == GSC_FMT_RATE;
    if (sc[i].format == GSC_FMT_BC1 || rate) {
      BatchSceneDev e = d;
      e.kind = 1;
      e.b1 = rate ? B.b1[i] : sc[i].d_blocks;
      if (rate) { e.sse1 = B.s1[i]; e.sse0 = B.s0[i]; }
      e.tile_groups = std::max(8, tune.bc1_tile_groups / 8 * 8);
      e.n_tiles = ceil_div64(e.work_groups, e.tile_groups);
      v.push_back(e);
    }
    if (sc[i].format == GSC_FMT_BC7 || rate) {
      BatchSceneDev e = d;
      e.kind = 7;
      e.b7 = rate ? B.b7[i] : sc[i].d_blocks;
      if (rate) e.sse7 = B.s7[i];
      e.tile_groups = 8;
      e.n_tiles = ceil_div64(e.work_groups, e.tile_groups);
      v.push_back(e);
    }
  }
  // BC7 entries first, then BC1 entries (one launch each); within a kind, schedules other than
  // the plain work queue list the scenes by decreasing size
  std::stable_sort(v.begin(), v.end(), [&](const BatchSceneDev& a, const BatchSceneDev& b) {
    if (a.kind != b.kind) return a.kind > b.kind;
    return tune.schedule != 1 && a.work_groups > b.work_groups;
  });
  int64_t t7 = 0, t1 = 0;
  for (auto& d : v) {
    int64_t& t = d.kind == 7 ? t7 : t1;
    d.tile0 = t;
    t += d.n_tiles;
  }
  n_tiles[0] = t7;
  n_tiles[1] = t1;
  return v;
}

static gsc_status launch_list(gsc_ctx* c, const std::vector<BatchSceneDev>& v, const int64_t* n_tiles,
                              const BatchBufs& B, const gsc_batch_tuning& tune, cudaStream_t st) {
  if (v.empty()) return GSC_OK;
  if (v.size() > B.list_cap) return GSC_ERR_INVALID_ARG;
  if (n_tiles[0] >= (int64_t)0x7F000000 || n_tiles[1] >= (int64_t)0x7F000000) return GSC_ERR_INVALID_ARG;
  int n7 = 0;
  while (n7 < (int)v.size() && v[n7].kind == 7) n7++;
  // a pageable source: the copy is staged before cudaMemcpyAsync returns
  GSC_CUDA(cudaMemcpyAsync(B.d_list, v.data(), sizeof(BatchSceneDev) * v.size(), cudaMemcpyHostToDevice, st));
  GSC_CUDA(launch_batch_encode(7, B.d_list, n7, n_tiles[0], tune.schedule, tune.ctas_per_sm, c->sm_count, B.counter,
                               st));
  GSC_CUDA(launch_batch_encode(1, B.d_list + n7, (int)v.size() - n7, n_tiles[1], tune.schedule, tune.ctas_per_sm,
                               c->sm_count, B.counter + 32, st));
  return GSC_OK;
}

static bool tune_ok(const gsc_batch_tuning* t) {
  return t && t->schedule >= 0 && t->schedule <= 3 && t->ctas_per_sm >= 1 && t->ctas_per_sm <= 32 &&
         t->bc1_tile_groups >= 8 && t->bc1_tile_groups <= 4096;
}

extern "C" gsc_status gsc_batch_encode(gsc_ctx* c, gsc_batch_scene* sc, int32_t n, const gsc_batch_tuning* tune,
                                       void* d_ws, size_t ws_bytes, void* stream) {
  GscRange gsc_range_("gsc_batch_encode");
  if (!c || !batch_args_ok(sc, n) || !tune_ok(tune) || ((uintptr_t)d_ws % 256) != 0) return GSC_ERR_INVALID_ARG;
  if (ws_bytes < layout(sc, n).total) return GSC_ERR_OOM;
  GSC_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  BatchBufs B = carve(sc, n, d_ws);
  if (!B.fits) return GSC_ERR_INVALID_ARG;
  gsc_status s = run_plans(c, sc, n, B, st);
  if (s != GSC_OK) return s;
  int64_t n_tiles[2] = {0, 0};
  std::vector<BatchSceneDev> v = scene_list(sc, n, B, *tune, 1, n_tiles);
  {
    GscTimed tm(c, T_BATCH, st);
    s = launch_list(c, v, n_tiles, B, *tune, st);
    if (s != GSC_OK) return s;
  }
  // forced formats keep the planned order; rate scenes select their streams
  for (int i = 0; i < n; i++) {
    const int64_t ng = groups_of(sc[i].n);
    memset(&sc[i].table, 0, sizeof(gsc_stream_table));
    if (sc[i].format != GSC_FMT_RATE && ng > 0)
      GSC_CUDA(cudaMemcpyAsync(sc[i].d_perm_out, sc[i].d_perm, sizeof(int32_t) * ng * 16, cudaMemcpyDeviceToDevice, st));
  }
  float* hs = reinterpret_cast<float*>(c->h_pinned);
  for (int i = 0; i < n; i++) {
    if (sc[i].format != GSC_FMT_RATE) continue;
    const int64_t ng = groups_of(sc[i].n);
    if (ng == 0) { sc[i].table.n_streams = GSC_MODES; sc[i].table.format = GSC_FMT_RATE; continue; }
    s = rate_select(c, sc[i].n, sc[i].d_perm, sc[i].d_scales, sc[i].target_bpt_x4, B.b1[i], B.b7[i], B.s1[i], B.s7[i],
                    B.s0[i], sc[i].d_blocks, sc[i].d_perm_out, &sc[i].table, B.select_ws, layout(sc, n).select_ws, st);
    if (s != GSC_OK) return s;
  }
  for (int i = 0; i < n; i++)
    GSC_CUDA(cudaMemcpyAsync(hs + 16 * i, sc[i].d_scales, sizeof(float) * 16, cudaMemcpyDeviceToHost, st));
  GSC_CUDA(cudaStreamSynchronize(st));
  for (int i = 0; i < n; i++) {
    gsc_stream_table& t = sc[i].table;
    memcpy(t.scales, hs + 16 * i, sizeof(float) * 16);
    if (sc[i].format == GSC_FMT_RATE) continue;
    const int64_t ng = groups_of(sc[i].n);
    const int bpb = sc[i].format == GSC_FMT_BC7 ? 16 : 8;
    t.n_streams = 1;
    t.format = sc[i].format;
    t.n = sc[i].n;
    t.n_groups = ng;
    t.total_bytes = ng * 16 * bpb;
    t.used_bits = (uint64_t)t.total_bytes * 8;
    host_weights(t.scales, t.weights);
    t.s[0].bands = 16;
    t.s[0].bc7_blocks = sc[i].format == GSC_FMT_BC7 ? 16 : 0;
    t.s[0].first_group = 0;
    t.s[0].n_groups = ng;
    t.s[0].byte_offset = 0;
  }
  return GSC_OK;
}

extern "C" gsc_status gsc_batch_autotune(gsc_ctx* c, gsc_batch_scene* sc, int32_t n, gsc_batch_tuning* out,
                                         double* ms_best, void* d_ws, size_t ws_bytes, void* stream) {
  GscRange gsc_range_("gsc_batch_autotune");
  if (!c || !out || !batch_args_ok(sc, n) || ((uintptr_t)d_ws % 256) != 0) return GSC_ERR_INVALID_ARG;
  if (ws_bytes < layout(sc, n).total) return GSC_ERR_OOM;
  GSC_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  BatchBufs B = carve(sc, n, d_ws);
  if (!B.fits) return GSC_ERR_INVALID_ARG;
  gsc_status s = run_plans(c, sc, n, B, st);
  if (s != GSC_OK) return s;
  cudaEvent_t e0, e1;
  GSC_CUDA(cudaEventCreate(&e0));
  GSC_CUDA(cudaEventCreate(&e1));
  double best = 1e30;
  gsc_batch_tuning bt = {1, 5, 8};
  // candidates: resident grids (1..4 CTAs per SM) with work queues, oversubscribed round-robin
  // grids (8..32 CTAs per SM, the hardware balances), one CTA per tile; BC1 tiles of 8 or 32
  static const gsc_batch_tuning kCand[] = {{1, 5, 8}, {2, 5, 8}, {2, 4, 8}, {2, 5, 32}, {0, 10, 8},
                                           {0, 16, 8}, {0, 32, 8}, {0, 32, 32}, {3, 5, 8}};
  for (const gsc_batch_tuning& t : kCand) {
    int64_t n_tiles[2] = {0, 0};
    std::vector<BatchSceneDev> v = scene_list(sc, n, B, t, kProxyDiv, n_tiles);
    double ms = 1e30;
    for (int rep = 0; rep < 2; rep++) {
      cudaEventRecord(e0, st);
      s = launch_list(c, v, n_tiles, B, t, st);
      if (s != GSC_OK) break;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) { s = GSC_ERR_CUDA; break; }
      float f = 0.f;
      cudaEventElapsedTime(&f, e0, e1);
      if (rep > 0) ms = std::min(ms, (double)f);
    }
    if (s != GSC_OK) break;
    if (ms < best) { best = ms; bt = t; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != GSC_OK) return s;
  *out = bt;
  if (ms_best) *ms_best = best;
  return GSC_OK;
}

extern "C" gsc_status gsc_batch_eval_graph(gsc_ctx* c, const gsc_batch_scene* sc, int32_t n, const float* d_cams,
                                           int32_t V, int32_t out_order, float* const* d_rgb, gsc_graph** out,
                                           void* stream) {
  GscRange gsc_range_("gsc_batch_eval_graph");
  if (!c || !sc || n <= 0 || !out || !d_rgb || !d_cams || V < 1 || V > 64 || out_order < 0 || out_order > 3)
    return GSC_ERR_INVALID_ARG;
  *out = nullptr;
  std::vector<DevTable> T(n);
  for (int i = 0; i < n; i++) {
    gsc_status s = make_dev_table(&sc[i].table, &T[i]);
    if (s != GSC_OK) return s;
    if (((uintptr_t)d_rgb[i] % 16) != 0 || (T[i].n_groups > 0 && (!sc[i].d_pos || !sc[i].d_perm_out)))
      return GSC_ERR_INVALID_ARG;
  }
  GSC_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (!st) return GSC_ERR_INVALID_ARG;  // the legacy stream cannot be captured
  gsc_graph* g = new gsc_graph();
  g->device = c->device;
  g->kernels = 0;
  for (int i = 0; i < n; i++) g->kernels += T[i].n_groups > 0;
  g->graph = nullptr;
  g->exec = nullptr;
  // the graph forks into kPlanLanes branches (scenes by decreasing size, each to the branch
  // with the least work) so that evaluations of small scenes overlap
  const int lanes = std::min(n, kPlanLanes);
  cudaStream_t ls[kPlanLanes] = {};
  cudaEvent_t fork = nullptr, join[kPlanLanes] = {};
  cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  for (int l = 0; l < lanes && e == cudaSuccess; l++) {
    e = cudaStreamCreateWithFlags(&ls[l], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[l], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    e = cudaEventRecord(fork, st);
    for (int l = 0; l < lanes && e == cudaSuccess; l++) e = cudaStreamWaitEvent(ls[l], fork, 0);
    std::vector<int> order(n);
    for (int i = 0; i < n; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sc[a].n > sc[b].n; });
    int64_t load[kPlanLanes] = {};
    for (int i : order) {
      if (e != cudaSuccess) break;
      int l = 0;
      for (int k = 1; k < lanes; k++) if (load[k] < load[l]) l = k;
      load[l] += sc[i].n + 20000;
      e = launch_decode_eval(T[i], sc[i].d_blocks, sc[i].d_perm_out, nullptr, sc[i].d_pos, d_cams, V, out_order,
                             d_rgb[i], c->sm_count, ls[l]);
    }
    for (int l = 0; l < lanes; l++) {
      if (e == cudaSuccess) e = cudaEventRecord(join[l], ls[l]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, join[l], 0);
    }
    cudaError_t e2 = cudaStreamEndCapture(st, &g->graph);
    if (e == cudaSuccess) e = e2;
  }
  for (int l = 0; l < lanes; l++) {
    if (join[l]) cudaEventDestroy(join[l]);
    if (ls[l]) cudaStreamDestroy(ls[l]);
  }
  if (fork) cudaEventDestroy(fork);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (e != cudaSuccess) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    cudaGetLastError();
    return GSC_ERR_CUDA;
  }
  *out = g;
  return GSC_OK;
}

extern "C" gsc_status gsc_graph_launch(gsc_graph* g, void* stream) {
  GscRange gsc_range_("gsc_graph_launch");
  if (!g) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(g->device));
  for (int i = 0; i < g->kernels; i++) gsc_count_launch();
  GSC_CUDA(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
  return GSC_OK;
}

extern "C" gsc_status gsc_graph_destroy(gsc_graph* g) {
  if (!g) return GSC_ERR_INVALID_ARG;
  cudaSetDevice(g->device);
  cudaGraphExecDestroy(g->exec);
  cudaGraphDestroy(g->graph);
  delete g;
  return GSC_OK;
}
