// serve.cu -- the request loop: encode and decode + SH evaluation requests arrive at any time,
// coded scenes stay resident on the device, admission is by slot and HBM budget (serve_sched.h),
// evaluation requests on one scene merge into one launch, and every launch runs on its slot's
// own streams so that work of different requests overlaps on the device. Each request's result
// is the one the single calls give: an encode runs gsc_plan_reorder + gsc_encode, an evaluation
// runs gsc_decode_eval_sh, whose colour for one (Gaussian, view) does not depend on the other
// views of the launch (Sec. II evaluation per view).
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "gsc_internal.cuh"
#include "serve_sched.h"

namespace {

struct SceneRes {
  int64_t n = 0;
  gsc_stream_table table;
  uint8_t* blocks = nullptr;
  int32_t* perm = nullptr;
  float* pos = nullptr;
};

struct Rec {
  gsc_request req;
  int32_t status = GSC_OK;
  int32_t merged = 1;
  int64_t n = 0;
  int64_t t_submit = 0, t_admit = 0, t_done = 0;
  bool done = false;
  int view_off = 0;  // first view in its merged launch
};

struct Slot {
  std::thread th;
  gsc_ctx* ctx = nullptr;
  cudaStream_t lo = nullptr, hi = nullptr;
  float* d_views = nullptr;  // [3][64] staged views of one launch
};

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device memory of one encode: what it holds while running and what the coded scene keeps.
void encode_bytes(int64_t n, int fmt, uint32_t t4, bool host_sh, uint64_t* temp, uint64_t* keep) {
  const int64_t ng = ceil_div64(n, 16), ns = ng * 16;
  gsc_encode_params ep = {fmt, t4, nullptr, nullptr};
  *temp = sched_align(4 * (uint64_t)ns) + 256 + sched_align(gsc_workspace_bytes(n, &ep)) +
          (host_sh ? sched_align(192 * (uint64_t)n) : 0);
  *keep = sched_align((uint64_t)ng * (fmt == GSC_FMT_BC1 ? 128 : 256)) + sched_align(4 * (uint64_t)ns) +
          sched_align(12 * (uint64_t)n);
}

bool params_ok(const gsc_server_params* p) {
  return p && p->hbm_budget_bytes > 0 && p->n_slots >= 1 && p->n_slots <= 16 && p->max_views >= 1 &&
         p->max_views <= 64 && p->hold_us >= 0 && (p->merge == 0 || p->merge == 1) && p->encode_slots >= 0 &&
         p->encode_slots <= p->n_slots;
}

int encode_slots(const gsc_server_params& p) {
  return p.encode_slots > 0 ? p.encode_slots : (p.n_slots > 1 ? p.n_slots - 1 : 1);
}

}  // namespace

struct gsc_server {
  int device = 0;
  gsc_server_params prm;
  cudaMemPool_t pool = nullptr;
  Sched sched;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::map<uint64_t, Rec> recs;
  std::map<std::pair<int, int>, SceneRes> scenes;
  std::vector<Slot> slots;
  uint64_t next_ticket = 1, submitted = 0, done = 0, failed = 0;
  bool stop = false;
  std::chrono::steady_clock::time_point t0;

  explicit gsc_server(const gsc_server_params& p)
      : prm(p), sched(p.hbm_budget_bytes, p.merge != 0, p.max_views, 16, p.hold_us * 1000, encode_slots(p)) {}

  int64_t now() const {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

void free_scene(gsc_server* s, int scene, int version, cudaStream_t st) {
  auto it = s->scenes.find({scene, version});
  if (it == s->scenes.end()) return;
  cudaFreeAsync(it->second.blocks, st);
  cudaFreeAsync(it->second.perm, st);
  cudaFreeAsync(it->second.pos, st);
  s->scenes.erase(it);
}

template <class T>
cudaError_t pool_alloc(gsc_server* s, T** p, uint64_t bytes, cudaStream_t st) {
  void* v = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&v, (size_t)(bytes ? bytes : 256), s->pool, st);
  *p = reinterpret_cast<T*>(v);
  return e;
}

// One encode on the slot's low-priority stream; the coded scene goes to *out.
gsc_status run_encode(gsc_server* s, Slot& w, const gsc_request& r, SceneRes* out) {
  GscRange range("serve_encode");
  cudaStream_t st = w.lo;
  const int64_t n = r.n, ng = ceil_div64(n, 16), ns = ng * 16;
  const bool host_sh = !on_device(r.sh);
  gsc_encode_params ep = {r.format, r.target_bpt_x4, nullptr, nullptr};
  const size_t wsb = gsc_workspace_bytes(n, &ep);
  float *sh = nullptr, *scales = nullptr;
  int32_t* perm = nullptr;
  void* ws = nullptr;
  gsc_status rc = GSC_OK;
  cudaError_t e = cudaSuccess;
  out->n = n;
  e = pool_alloc(s, &out->blocks, (uint64_t)ng * (r.format == GSC_FMT_BC1 ? 128 : 256), st);
  if (e == cudaSuccess) e = pool_alloc(s, &out->perm, 4 * (uint64_t)ns, st);
  if (e == cudaSuccess) e = pool_alloc(s, &out->pos, 12 * (uint64_t)n, st);
  if (e == cudaSuccess) e = pool_alloc(s, &perm, 4 * (uint64_t)ns, st);
  if (e == cudaSuccess) e = pool_alloc(s, &scales, 64, st);
  if (e == cudaSuccess) e = pool_alloc(s, &ws, wsb, st);
  if (e == cudaSuccess && host_sh) e = pool_alloc(s, &sh, 192 * (uint64_t)n, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out->pos, r.pos, 12 * (size_t)n, cudaMemcpyDefault, st);
  if (e == cudaSuccess && host_sh) e = cudaMemcpyAsync(sh, r.sh, 192 * (size_t)n, cudaMemcpyDefault, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    rc = e == cudaErrorMemoryAllocation ? GSC_ERR_OOM : GSC_ERR_CUDA;
  }
  const float* shp = host_sh ? sh : r.sh;
  if (rc == GSC_OK) {
    gsc_plan_params pp = {n, r.group_size, r.sort, 995};
    rc = gsc_plan_reorder(w.ctx, out->pos, shp, &pp, perm, scales, ws, wsb, st);
  }
  if (rc == GSC_OK)
    rc = gsc_encode(w.ctx, shp, n, perm, scales, &ep, out->blocks, out->perm, &out->table, ws, wsb, st);
  cudaFreeAsync(perm, st);
  cudaFreeAsync(scales, st);
  cudaFreeAsync(ws, st);
  if (sh) cudaFreeAsync(sh, st);
  if (rc != GSC_OK) {
    cudaFreeAsync(out->blocks, st);
    cudaFreeAsync(out->perm, st);
    cudaFreeAsync(out->pos, st);
    out->blocks = nullptr;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == GSC_OK) rc = GSC_ERR_CUDA;
  return rc;
}

// A coded scene read back from a checkpoint file into resident memory (with its positions).
gsc_status run_load(gsc_server* s, Slot& w, const gsc_request& r, SceneRes* out) {
  cudaStream_t st = w.lo;
  gsc_stream_table t;
  int32_t has_pos = 0;
  gsc_status rc = gsc_scene_read_info(r.path, &t, &has_pos);
  if (rc != GSC_OK) return rc;
  if (!has_pos || t.n != r.n) return GSC_ERR_INVALID_ARG;
  const int64_t ns = t.n_groups * 16;
  cudaError_t e = pool_alloc(s, &out->blocks, (uint64_t)t.total_bytes, st);
  if (e == cudaSuccess) e = pool_alloc(s, &out->perm, 4 * (uint64_t)ns, st);
  if (e == cudaSuccess) e = pool_alloc(s, &out->pos, 12 * (uint64_t)t.n, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the allocations exist before the copies
  if (e != cudaSuccess) {
    cudaGetLastError();
    rc = e == cudaErrorMemoryAllocation ? GSC_ERR_OOM : GSC_ERR_CUDA;
  } else {
    rc = gsc_scene_read(r.path, &out->table, out->blocks, (size_t)t.total_bytes, out->perm, 4 * (size_t)ns, out->pos,
                        12 * (size_t)t.n);
  }
  out->n = t.n;
  if (rc != GSC_OK) {
    cudaFreeAsync(out->blocks, st);
    cudaFreeAsync(out->perm, st);
    cudaFreeAsync(out->pos, st);
    out->blocks = nullptr;
    cudaStreamSynchronize(st);
  }
  return rc;
}

// One evaluation launch (one or several merged requests) on the slot's high-priority stream.
gsc_status run_eval(gsc_server* s, Slot& w, const SceneRes& sc, std::vector<Rec*>& rs, int V_total,
                    uint64_t stage_bytes) {
  GscRange range("serve_eval");
  cudaStream_t st = s->prm.priority ? w.hi : w.lo;
  const gsc_request& r0 = rs[0]->req;
  const bool cams = r0.cams != nullptr;
  cudaError_t e = cudaSuccess;
  // views: gather every request's [V][3] into one [V_total][3] device array
  int off = 0;
  for (Rec* r : rs) {
    const float* src = cams ? r->req.cams : r->req.dirs;
    r->view_off = off;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(w.d_views + 3 * off, src, 12 * (size_t)r->req.V, cudaMemcpyDefault, st);
    off += r->req.V;
  }
  float* stage = nullptr;
  if (e == cudaSuccess && stage_bytes) e = pool_alloc(s, &stage, stage_bytes, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GSC_ERR_OOM : GSC_ERR_CUDA;
  }
  float* dst = stage ? stage : r0.out;
  gsc_status rc = gsc_decode_eval_sh(w.ctx, &sc.table, sc.blocks, sc.perm, cams ? nullptr : w.d_views, sc.pos,
                                     cams ? w.d_views : nullptr, V_total, r0.out_order, dst, st);
  if (rc == GSC_OK && stage) {
    const int64_t n = sc.n, rows = r0.out_order == GSC_OUT_SLOT_ORDER ? ceil_div64(n, 16) * 16 : n;
    for (Rec* r : rs) {
      const int V = r->req.V;
      if (r0.out_order == GSC_OUT_GAUSS_MAJOR) {
        e = cudaMemcpy2DAsync(r->req.out, (size_t)V * 12, stage + 3 * (int64_t)r->view_off, (size_t)V_total * 12,
                              (size_t)V * 12, (size_t)n, cudaMemcpyDefault, st);
      } else {
        e = cudaMemcpyAsync(r->req.out, stage + 3 * (int64_t)r->view_off * rows, (size_t)V * rows * 12,
                            cudaMemcpyDefault, st);
      }
      if (e != cudaSuccess) { cudaGetLastError(); rc = GSC_ERR_CUDA; break; }
    }
  }
  if (stage) cudaFreeAsync(stage, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == GSC_OK) rc = GSC_ERR_CUDA;
  return rc;
}

void slot_main(gsc_server* s, int k) {
  Slot& w = s->slots[k];
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    SchedLaunch L;
    bool got = false;
    s->cv_work.wait(lk, [&] {
      if (s->stop) return true;
      got = s->sched.pick(s->now(), &L);
      return got;
    });
    if (!got) break;  // stopping with nothing admissible
    const int64_t t_admit = s->now();
    std::vector<Rec*> rs;
    for (uint64_t t : L.tickets) {
      Rec& r = s->recs[t];
      r.t_admit = t_admit;
      r.merged = (int32_t)L.tickets.size();
      r.n = L.n;
      rs.push_back(&r);
    }
    if (L.kind == SLAUNCH_REJECT) {
      for (Rec* r : rs) { r->status = GSC_ERR_INVALID_ARG; r->done = true; r->t_done = s->now(); s->failed++; s->done++; }
      s->cv_done.notify_all();
      continue;
    }
    for (auto& ev : L.evict) free_scene(s, ev.first, ev.second, w.lo);
    gsc_status rc;
    if (L.kind == SLAUNCH_ENCODE) {
      const gsc_request req = rs[0]->req;
      lk.unlock();
      SceneRes res;
      rc = req.kind == GSC_REQ_LOAD ? run_load(s, w, req, &res) : run_encode(s, w, req, &res);
      lk.lock();
      if (rc == GSC_OK) s->scenes[{L.scene, L.version}] = res;
    } else {
      const SceneRes sc = s->scenes[{L.scene, L.version}];  // pinned by the scheduler until completion
      lk.unlock();
      rc = run_eval(s, w, sc, rs, L.V_total, L.temp_bytes);
      lk.lock();
    }
    for (auto& f : s->sched.complete(L, rc == GSC_OK)) free_scene(s, f.first, f.second, w.lo);
    const int64_t t_done = s->now();
    for (Rec* r : rs) {
      r->status = rc;
      r->done = true;
      r->t_done = t_done;
      s->done++;
      if (rc != GSC_OK) s->failed++;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

gsc_status request_ok(const gsc_request* r, const gsc_server_params& p) {
  if (!r || r->scene < 0) return GSC_ERR_INVALID_ARG;
  if (r->kind == GSC_REQ_ENCODE) {
    if (r->n <= 0 || r->n >= (int64_t)0x7FFFFFF0 || !r->pos || !r->sh) return GSC_ERR_INVALID_ARG;
    if (r->format != GSC_FMT_BC1 && r->format != GSC_FMT_BC7 && r->format != GSC_FMT_RATE) return GSC_ERR_INVALID_ARG;
    if (r->format == GSC_FMT_RATE && (r->target_bpt_x4 == 0 || r->target_bpt_x4 > 64)) return GSC_ERR_INVALID_ARG;
    if (r->group_size < 0 || r->group_size % 16 != 0 || (r->sort != 0 && r->sort != 1)) return GSC_ERR_INVALID_ARG;
    if (((uintptr_t)r->sh % 16) != 0) return GSC_ERR_INVALID_ARG;
    return GSC_OK;
  }
  if (r->kind == GSC_REQ_LOAD) {
    if (!r->path || r->n <= 0) return GSC_ERR_INVALID_ARG;
    return GSC_OK;
  }
  if (r->kind == GSC_REQ_EVAL) {
    if (r->n <= 0 || r->V < 1 || r->V > p.max_views || !r->out || (!r->dirs == !r->cams)) return GSC_ERR_INVALID_ARG;
    if (r->out_order < 0 || r->out_order > 2 || ((uintptr_t)r->out % 16) != 0) return GSC_ERR_INVALID_ARG;
    return GSC_OK;
  }
  return GSC_ERR_INVALID_ARG;
}

SchedReq sched_req(const gsc_request& r, uint64_t ticket, int64_t t, bool host_sh, bool out_device) {
  SchedReq q;
  q.ticket = ticket;
  q.kind = r.kind == GSC_REQ_EVAL ? SREQ_EVAL : SREQ_ENCODE;  // a load installs a version like an encode
  q.scene = r.scene;
  q.n = r.n;
  q.V = r.V;
  q.out_order = r.out_order;
  q.view_kind = r.cams ? 1 : 0;
  q.out_device = out_device;
  q.t_submit = t;
  if (r.kind == GSC_REQ_ENCODE) encode_bytes(r.n, r.format, r.target_bpt_x4, host_sh, &q.temp_bytes, &q.keep_bytes);
  return q;
}

// Resident bytes of a checkpoint file's scene (0 when the file cannot serve as one).
uint64_t load_bytes(const gsc_request& r) {
  gsc_stream_table t;
  int32_t has_pos = 0;
  if (gsc_scene_read_info(r.path, &t, &has_pos) != GSC_OK || !has_pos || t.n != r.n) return 0;
  return sched_align((uint64_t)t.total_bytes) + sched_align(4 * (uint64_t)t.n_groups * 16) + sched_align(12 * (uint64_t)t.n);
}

}  // namespace

extern "C" gsc_status gsc_server_create(gsc_ctx* c, const gsc_server_params* p, gsc_server** out) {
  if (!c || !out || !params_ok(p)) return GSC_ERR_INVALID_ARG;
  *out = nullptr;
  GSC_CUDA(cudaSetDevice(c->device));
  gsc_server* s = new gsc_server(*p);
  s->device = c->device;
  s->t0 = std::chrono::steady_clock::now();
  cudaMemPoolProps props;
  memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = c->device;
  cudaError_t e = cudaMemPoolCreate(&s->pool, &props);
  if (e == cudaSuccess) {
    uint64_t keep = UINT64_MAX;  // freed blocks stay in the pool for the next request
    e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  int lo_pri = 0, hi_pri = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&lo_pri, &hi_pri);
  s->slots.resize(p->n_slots);
  gsc_status rc = GSC_OK;
  for (auto& w : s->slots) {
    if (e != cudaSuccess || rc != GSC_OK) break;
    rc = ctx_new(c->device, false, &w.ctx);
    if (rc != GSC_OK) break;
    e = cudaStreamCreateWithPriority(&w.lo, cudaStreamNonBlocking, lo_pri);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&w.hi, cudaStreamNonBlocking, hi_pri);
    if (e == cudaSuccess) e = cudaMalloc(&w.d_views, 3 * 64 * sizeof(float));
  }
  if (e != cudaSuccess || rc != GSC_OK) {
    cudaGetLastError();
    for (auto& w : s->slots) {
      if (w.d_views) cudaFree(w.d_views);
      if (w.lo) cudaStreamDestroy(w.lo);
      if (w.hi) cudaStreamDestroy(w.hi);
      if (w.ctx) gsc_ctx_destroy(w.ctx);
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    return rc != GSC_OK ? rc : GSC_ERR_CUDA;
  }
  for (int k = 0; k < p->n_slots; k++) s->slots[k].th = std::thread(slot_main, s, k);
  *out = s;
  return GSC_OK;
}

extern "C" gsc_status gsc_server_submit(gsc_server* s, const gsc_request* r, uint64_t* ticket) {
  GscRange gsc_range_("gsc_server_submit");
  if (!s || !ticket) return GSC_ERR_INVALID_ARG;
  gsc_status rc = request_ok(r, s->prm);
  if (rc != GSC_OK) return rc;
  const bool host_sh = r->kind == GSC_REQ_ENCODE && !on_device(r->sh);
  const bool out_dev = r->kind == GSC_REQ_EVAL && on_device(r->out);
  SchedReq q0 = sched_req(*r, 0, 0, host_sh, out_dev);
  if (r->kind == GSC_REQ_LOAD) {
    q0.keep_bytes = load_bytes(*r);  // the file is read once here to size the request
    if (q0.keep_bytes == 0) return GSC_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return GSC_ERR_INVALID_ARG;
  const uint64_t t = s->next_ticket++;
  const int64_t now = s->now();
  q0.ticket = t;
  q0.t_submit = now;
  if (!s->sched.submit(q0)) return GSC_ERR_BUDGET;
  Rec& rec = s->recs[t];
  rec.req = *r;
  rec.t_submit = now;
  s->submitted++;
  *ticket = t;
  s->cv_work.notify_one();
  return GSC_OK;
}

extern "C" gsc_status gsc_server_wait(gsc_server* s, uint64_t ticket, int64_t timeout_ms, gsc_request_result* res) {
  GscRange gsc_range_("gsc_server_wait");
  if (!s || !res) return GSC_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->recs.find(ticket);
  if (it == s->recs.end()) return GSC_ERR_INVALID_ARG;
  auto ready = [&] { return s->recs[ticket].done; };
  if (timeout_ms < 0) s->cv_done.wait(lk, ready);
  else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return GSC_ERR_TIMEOUT;
  const Rec& r = s->recs[ticket];
  res->status = r.status;
  res->kind = r.req.kind;
  res->scene = r.req.scene;
  res->merged = r.merged;
  res->n = r.n;
  res->t_submit_ms = r.t_submit * 1e-6;
  res->t_admit_ms = r.t_admit * 1e-6;
  res->t_done_ms = r.t_done * 1e-6;
  s->recs.erase(ticket);
  return GSC_OK;
}

extern "C" gsc_status gsc_server_drain(gsc_server* s, int64_t timeout_ms) {
  if (!s) return GSC_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto idle = [&] { return s->sched.idle(); };
  if (timeout_ms < 0) s->cv_done.wait(lk, idle);
  else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), idle)) return GSC_ERR_TIMEOUT;
  return GSC_OK;
}

extern "C" gsc_status gsc_server_read_scene(gsc_server* s, int32_t scene, gsc_stream_table* table, uint8_t* blocks,
                                            size_t blocks_cap, int32_t* perm, size_t perm_cap) {
  if (!s || !table) return GSC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  const int v = s->sched.current(scene);
  auto it = s->scenes.find({scene, v});
  if (v < 0 || it == s->scenes.end()) return GSC_ERR_INVALID_ARG;
  const SceneRes& r = it->second;
  *table = r.table;
  const size_t nb = (size_t)r.table.total_bytes, np = (size_t)r.table.n_groups * 16 * 4;
  if ((blocks && blocks_cap < nb) || (perm && perm_cap < np)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(s->device));
  if (blocks) GSC_CUDA(cudaMemcpy(blocks, r.blocks, nb, cudaMemcpyDefault));
  if (perm) GSC_CUDA(cudaMemcpy(perm, r.perm, np, cudaMemcpyDefault));
  return GSC_OK;
}

extern "C" gsc_status gsc_server_cancel(gsc_server* s, uint64_t ticket) {
  if (!s) return GSC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->recs.find(ticket);
  if (it == s->recs.end() || it->second.done || !s->sched.cancel(ticket)) return GSC_ERR_INVALID_ARG;
  Rec& r = it->second;
  r.status = GSC_ERR_CANCELLED;
  r.t_admit = r.t_done = s->now();
  r.done = true;
  s->done++;
  s->failed++;
  s->cv_done.notify_all();
  s->cv_work.notify_all();  // a request held back behind it may be admissible now
  return GSC_OK;
}

extern "C" gsc_status gsc_server_save_scene(gsc_server* s, int32_t scene, const char* path) {
  if (!s || !path) return GSC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  const int v = s->sched.current(scene);
  auto it = s->scenes.find({scene, v});
  if (v < 0 || it == s->scenes.end()) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(s->device));
  const SceneRes& r = it->second;
  return gsc_scene_write(path, &r.table, r.blocks, r.perm, r.pos);
}

extern "C" gsc_status gsc_server_evict(gsc_server* s, int32_t scene) {
  if (!s) return GSC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  std::vector<std::pair<int, int>> freed;
  if (!s->sched.evict(scene, &freed)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(s->device));
  for (auto& f : freed) free_scene(s, f.first, f.second, s->slots[0].lo);
  GSC_CUDA(cudaStreamSynchronize(s->slots[0].lo));
  s->cv_work.notify_all();
  return GSC_OK;
}

extern "C" gsc_status gsc_server_get_stats(gsc_server* s, gsc_server_stats* st) {
  if (!s || !st) return GSC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  memset(st, 0, sizeof(*st));
  st->submitted = s->submitted;
  st->done = s->done;
  st->failed = s->failed;
  st->merged = s->sched.merged();
  st->evictions = s->sched.evictions();
  st->resident_bytes = s->sched.resident();
  st->used_bytes = s->sched.used();
  st->peak_bytes = s->sched.peak();
  st->queued = (int32_t)s->sched.queued();
  st->resident_versions = (int32_t)s->scenes.size();
  return GSC_OK;
}

extern "C" gsc_status gsc_server_destroy(gsc_server* s) {
  if (!s) return GSC_ERR_INVALID_ARG;
  gsc_server_drain(s, -1);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& w : s->slots)
    if (w.th.joinable()) w.th.join();
  cudaSetDevice(s->device);
  for (auto& kv : s->scenes) {
    cudaFreeAsync(kv.second.blocks, s->slots[0].lo);
    cudaFreeAsync(kv.second.perm, s->slots[0].lo);
    cudaFreeAsync(kv.second.pos, s->slots[0].lo);
  }
  cudaStreamSynchronize(s->slots[0].lo);
  for (auto& w : s->slots) {
    cudaFree(w.d_views);
    cudaStreamDestroy(w.lo);
    cudaStreamDestroy(w.hi);
    gsc_ctx_destroy(w.ctx);
  }
  cudaMemPoolDestroy(s->pool);
  delete s;
  return GSC_OK;
}

// ---- host-side simulation of the admission policy ----------------------------------------
extern "C" gsc_status gsc_server_simulate(const gsc_server_params* p, const gsc_sim_request* rq, int32_t n,
                                          gsc_sim_result* res, uint64_t* peak_bytes) {
  if (!params_ok(p) || n < 0 || (n > 0 && (!rq || !res))) return GSC_ERR_INVALID_ARG;
  Sched sc(p->hbm_budget_bytes, p->merge != 0, p->max_views, 16, p->hold_us * 1000, encode_slots(*p));
  std::vector<int> order(n);
  for (int i = 0; i < n; i++) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return rq[a].t_arrival_ms < rq[b].t_arrival_ms; });
  for (int i = 0; i < n; i++) {
    memset(&res[i], 0, sizeof(res[i]));
    res[i].status = -1;
  }
  struct Run { int64_t end; SchedLaunch L; };
  std::vector<Run> running;
  int free_slots = p->n_slots;
  size_t next = 0;
  int64_t now = 0;
  auto ns = [](double ms) { return (int64_t)(ms * 1e6); };
  for (;;) {
    // start whatever is admissible
    SchedLaunch L;
    while (free_slots > 0 && sc.pick(now, &L)) {
      double dur = 0.0;
      for (uint64_t t : L.tickets) {
        gsc_sim_result& r = res[t - 1];
        r.t_admit_ms = now * 1e-6;
        r.merged = (int32_t)L.tickets.size();
        r.used_bytes_at_admit = sc.used();
        dur += rq[t - 1].service_ms;
      }
      if (L.kind == SLAUNCH_REJECT) {
        for (uint64_t t : L.tickets) { res[t - 1].status = GSC_ERR_INVALID_ARG; res[t - 1].t_done_ms = now * 1e-6; }
        continue;
      }
      res[L.tickets[0] - 1].evictions = (int32_t)L.evict.size();
      running.push_back({now + ns(dur), L});
      free_slots--;
    }
    // next event: an arrival or the earliest completion
    int64_t t_arr = next < (size_t)n ? ns(rq[order[next]].t_arrival_ms) : INT64_MAX;
    size_t first = running.size();
    for (size_t i = 0; i < running.size(); i++)
      if (first == running.size() || running[i].end < running[first].end) first = i;
    int64_t t_end = first < running.size() ? running[first].end : INT64_MAX;
    if (t_arr == INT64_MAX && t_end == INT64_MAX) break;
    if (t_end <= t_arr) {
      now = t_end;
      Run R = running[first];
      running.erase(running.begin() + (std::ptrdiff_t)first);
      sc.complete(R.L, true);
      for (uint64_t t : R.L.tickets) { res[t - 1].status = GSC_OK; res[t - 1].t_done_ms = now * 1e-6; }
      free_slots++;
    } else {
      now = t_arr;
      const int i = order[next++];
      const gsc_sim_request& q = rq[i];
      SchedReq r;
      r.ticket = (uint64_t)i + 1;
      r.kind = q.kind == GSC_REQ_ENCODE ? SREQ_ENCODE : SREQ_EVAL;
      r.scene = q.scene;
      r.n = q.n;
      r.V = q.V;
      r.out_order = q.out_order;
      r.view_kind = q.cams ? 1 : 0;
      r.out_device = q.out_device != 0;
      r.t_submit = now;
      if (r.kind == SREQ_ENCODE) encode_bytes(q.n, q.format, q.target_bpt_x4, q.host_input != 0, &r.temp_bytes, &r.keep_bytes);
      if (!sc.submit(r)) { res[i].status = GSC_ERR_BUDGET; res[i].t_admit_ms = res[i].t_done_ms = now * 1e-6; }
    }
  }
  if (peak_bytes) *peak_bytes = sc.peak();
  return GSC_OK;
}
