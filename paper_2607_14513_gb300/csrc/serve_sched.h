// serve_sched.h -- admission bookkeeping of the request loop: which queued request runs next
// on a free slot, under an HBM budget, in what order relative to the other requests on the
// same scene, merged with which other evaluation requests, and which idle resident scenes
// give their memory up. Host only: no CUDA calls, so the same code drives the GPU server and
// the host-side simulator.
#pragma once
#include <stdint.h>

#include <algorithm>
#include <deque>
#include <map>
#include <utility>
#include <vector>

enum { SREQ_ENCODE = 0, SREQ_EVAL = 1 };
enum { SLAUNCH_ENCODE = 0, SLAUNCH_EVAL = 1, SLAUNCH_REJECT = 2 };

struct SchedReq {
  uint64_t ticket = 0;
  int kind = SREQ_ENCODE;
  int scene = 0;
  int64_t n = 0;            // encode: Gaussians of the scene
  int V = 0;                // eval: views
  int out_order = 0;        // eval: gsc_out_order
  int view_kind = 0;        // eval: 0 directions, 1 camera centres
  bool out_device = true;   // eval: caller's output is device memory (written in place when alone)
  uint64_t temp_bytes = 0;  // encode: device memory held while it runs
  uint64_t keep_bytes = 0;  // encode: device memory the coded scene keeps afterwards
  int64_t t_submit = 0;     // ns
};

struct SchedLaunch {
  int kind = SLAUNCH_ENCODE;
  int scene = 0;
  int version = 0;          // encode: version it writes; eval: version it reads
  int64_t n = 0;            // Gaussians of that version
  std::vector<uint64_t> tickets;
  int V_total = 0;
  uint64_t temp_bytes = 0;  // released at completion
  uint64_t keep_bytes = 0;  // encode: resident after completion
  std::vector<std::pair<int, int>> evict;  // (scene, version) to free before the launch runs
};

static inline uint64_t sched_align(uint64_t b) { return (b + 255) & ~(uint64_t)255; }

// Output staging of an evaluation launch: views x rows x RGB floats.
static inline uint64_t sched_eval_bytes(int64_t n, int V, int out_order) {
  const int64_t rows = out_order == 1 ? (n + 15) / 16 * 16 : n;  // slot order covers whole groups
  return sched_align((uint64_t)V * (uint64_t)rows * 12u);
}

class Sched {
 public:
  Sched(uint64_t budget, bool merge, int max_views, int max_merge, int64_t hold_ns, int max_encodes)
      : budget_(budget), merge_(merge), max_views_(max_views), max_merge_(max_merge), hold_ns_(hold_ns),
        max_encodes_(max_encodes) {}

  // False when the request could never run within the budget.
  bool submit(const SchedReq& r) {
    if (r.kind == SREQ_ENCODE && r.temp_bytes + r.keep_bytes > budget_) return false;
    q_.push_back(r);
    scenes_[r.scene].queued++;
    return true;
  }

  bool idle() const { return q_.empty() && running_ == 0; }
  size_t queued() const { return q_.size(); }
  uint64_t used() const { return used_; }
  uint64_t peak() const { return peak_; }
  uint64_t resident() const { return resident_; }
  uint64_t evictions() const { return evictions_; }
  uint64_t merged() const { return merged_; }

  // Takes the first admissible queued request (and, for an evaluation, the later ones it
  // merges with) in submission order. Requests on one scene keep their submission order
  // around encodes: an encode waits for every earlier request on its scene to start, an
  // evaluation waits for every earlier encode of its scene to finish. A request older than
  // the hold time that does not fit stops the scan, so that big requests are not starved.
  bool pick(int64_t now, SchedLaunch* out) {
    for (size_t i = 0; i < q_.size(); i++) {
      const SchedReq& r = q_[i];
      Scene& S = scenes_[r.scene];
      if (blocked(i)) continue;
      SchedLaunch L;
      L.scene = r.scene;
      if (r.kind == SREQ_EVAL && !S.encoding && (S.cur < 0 || S.vers[S.cur].n != r.n)) {
        L.kind = SLAUNCH_REJECT;  // nothing resident (and no encode ahead of it), or not the size asked for
        L.tickets.push_back(r.ticket);
        take(i);
        *out = L;
        return true;
      }
      if (r.kind == SREQ_ENCODE) {
        L.kind = SLAUNCH_ENCODE;
        L.n = r.n;
        L.temp_bytes = r.temp_bytes;
        L.keep_bytes = r.keep_bytes;
        L.tickets.push_back(r.ticket);
      } else {
        if (S.encoding) continue;
        L.kind = SLAUNCH_EVAL;
        L.version = S.cur;
        L.n = S.vers[S.cur].n;
        L.tickets.push_back(r.ticket);
        L.V_total = r.V;
        std::vector<size_t> more;
        if (merge_) {
          for (size_t j = i + 1; j < q_.size() && (int)L.tickets.size() < max_merge_; j++) {
            const SchedReq& o = q_[j];
            if (o.scene != r.scene) continue;
            if (o.kind == SREQ_ENCODE) break;  // later evaluations read the next version
            if (o.out_order != r.out_order || o.view_kind != r.view_kind || L.V_total + o.V > max_views_) continue;
            L.tickets.push_back(o.ticket);
            L.V_total += o.V;
            more.push_back(j);
          }
        }
        const bool staged = L.tickets.size() > 1 || !r.out_device;
        L.temp_bytes = staged ? sched_eval_bytes(L.n, L.V_total, r.out_order) : 0;
        if (!fits(L.temp_bytes, r.scene, &L.evict)) {
          if (now - r.t_submit > hold_ns_) return false;
          continue;
        }
        for (size_t k = more.size(); k-- > 0;) take(more[k]);
        take(i);
        apply_evictions(L.evict);
        S.vers[L.version].refs++;
        S.last_use = ++clock_;
        used_ += L.temp_bytes;
        peak_ = std::max(peak_, used_);
        merged_ += L.tickets.size() - 1;
        running_++;
        *out = L;
        return true;
      }
      // encode
      if (encoding_ >= max_encodes_) continue;
      if (!fits(L.temp_bytes + L.keep_bytes, r.scene, &L.evict)) {
        if (now - r.t_submit > hold_ns_) return false;
        continue;
      }
      take(i);
      apply_evictions(L.evict);
      S.encoding = true;
      encoding_++;
      L.version = S.next_version++;
      used_ += L.temp_bytes + L.keep_bytes;
      peak_ = std::max(peak_, used_);
      running_++;
      *out = L;
      return true;
    }
    return false;
  }

  // Bookkeeping at the end of a launch; returns the versions whose memory can be freed now
  // (a replaced version, once no evaluation reads it).
  std::vector<std::pair<int, int>> complete(const SchedLaunch& L, bool ok) {
    std::vector<std::pair<int, int>> freed;
    if (L.kind == SLAUNCH_REJECT) return freed;
    running_--;
    Scene& S = scenes_[L.scene];
    S.last_use = ++clock_;
    used_ -= L.temp_bytes;
    if (L.kind == SLAUNCH_ENCODE) {
      S.encoding = false;
      encoding_--;
      if (!ok) {
        used_ -= L.keep_bytes;
        return freed;
      }
      const int old = S.cur;
      S.vers[L.version] = Ver{L.n, L.keep_bytes, 0, false};
      S.cur = L.version;
      resident_ += L.keep_bytes;
      if (old >= 0) retire(S, L.scene, old, &freed);
    } else {
      Ver& v = S.vers[L.version];
      v.refs--;
      if (v.retired && v.refs == 0) drop(S, L.scene, L.version, &freed);
    }
    return freed;
  }

  // Removes a queued request; false when it is not queued (already admitted, or unknown).
  bool cancel(uint64_t ticket) {
    for (size_t i = 0; i < q_.size(); i++)
      if (q_[i].ticket == ticket) { take(i); return true; }
    return false;
  }

  // Frees a scene's current version when nothing queued or running uses it.
  bool evict(int scene, std::vector<std::pair<int, int>>* freed) {
    auto it = scenes_.find(scene);
    if (it == scenes_.end()) return false;
    Scene& S = it->second;
    if (S.cur < 0 || S.queued > 0 || S.encoding || S.vers[S.cur].refs > 0) return false;
    const int v = S.cur;
    S.cur = -1;
    drop(S, scene, v, freed);
    return true;
  }

  // Current version of a resident scene, or -1.
  int current(int scene) const {
    auto it = scenes_.find(scene);
    return it == scenes_.end() ? -1 : it->second.cur;
  }

 private:
  struct Ver {
    int64_t n;
    uint64_t bytes;
    int refs;
    bool retired;
  };
  struct Scene {
    int cur = -1;
    int next_version = 0;
    uint64_t last_use = 0;
    int queued = 0;
    bool encoding = false;
    std::map<int, Ver> vers;
  };

  bool blocked(size_t i) const {
    const SchedReq& r = q_[i];
    for (size_t j = 0; j < i; j++) {
      const SchedReq& o = q_[j];
      if (o.scene != r.scene) continue;
      if (r.kind == SREQ_ENCODE) return true;      // an earlier request on the scene has not started
      if (o.kind == SREQ_ENCODE) return true;      // an earlier encode has not started
    }
    if (r.kind == SREQ_ENCODE) {
      auto it = scenes_.find(r.scene);
      if (it != scenes_.end() && it->second.encoding) return true;
    }
    return false;
  }

  void take(size_t i) {
    scenes_[q_[i].scene].queued--;
    q_.erase(q_.begin() + (std::ptrdiff_t)i);
  }

  // Whether `need` more bytes fit, evicting idle scenes (least recently used first, never
  // `keep_scene`) if that makes them fit; the evictions are returned, not yet applied.
  bool fits(uint64_t need, int keep_scene, std::vector<std::pair<int, int>>* ev) {
    ev->clear();
    if (used_ + need <= budget_) return true;
    std::vector<std::pair<uint64_t, int>> cand;
    uint64_t avail = 0;
    for (auto& kv : scenes_) {
      const Scene& S = kv.second;
      if (kv.first == keep_scene || S.cur < 0 || S.queued > 0 || S.encoding) continue;
      const Ver& v = S.vers.at(S.cur);
      if (v.refs > 0) continue;
      cand.push_back({S.last_use, kv.first});
      avail += v.bytes;
    }
    if (used_ + need > budget_ + avail) return false;
    std::sort(cand.begin(), cand.end());
    uint64_t have = budget_ - std::min(budget_, used_);
    for (auto& c : cand) {
      if (have >= need) break;
      const Scene& S = scenes_[c.second];
      have += S.vers.at(S.cur).bytes;
      ev->push_back({c.second, S.cur});
    }
    return have >= need;
  }

  void apply_evictions(const std::vector<std::pair<int, int>>& ev) {
    for (auto& e : ev) {
      Scene& S = scenes_[e.first];
      S.cur = -1;
      std::vector<std::pair<int, int>> dummy;
      drop(S, e.first, e.second, &dummy);
      evictions_++;
    }
  }

  void retire(Scene& S, int scene, int v, std::vector<std::pair<int, int>>* freed) {
    Ver& x = S.vers[v];
    if (x.refs == 0) drop(S, scene, v, freed);
    else x.retired = true;
  }

  void drop(Scene& S, int scene, int v, std::vector<std::pair<int, int>>* freed) {
    auto it = S.vers.find(v);
    if (it == S.vers.end()) return;
    used_ -= it->second.bytes;
    resident_ -= it->second.bytes;
    S.vers.erase(it);
    freed->push_back({scene, v});
  }

  std::deque<SchedReq> q_;
  std::map<int, Scene> scenes_;
  uint64_t budget_, used_ = 0, peak_ = 0, resident_ = 0, evictions_ = 0, merged_ = 0, clock_ = 0;
  bool merge_;
  int max_views_, max_merge_;
  int64_t hold_ns_;
  int max_encodes_;
  int running_ = 0, encoding_ = 0;
};
