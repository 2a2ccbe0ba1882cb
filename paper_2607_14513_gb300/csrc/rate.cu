// rate.cu -- rate control over several fixed-rate streams (Sec. IV-B: groups of Gaussians
// are coded with different fixed-rate arrangements and each arrangement is its own
// bitstream, so random access survives; Figs. SetupC/SetupD: high-order coefficients
// that are zero are not stored).
//
// Reading (the paper gives the mechanism, not an allocation rule): 14 group modes
// (b coefficients kept, the first j of them BC7, the rest BC1), rate R = 64 (b + j) bits
// per group; distortion D = sum_k w_k SSE_k with w_k = max(1, rint(65536 s_k^2 / max s^2));
// the smallest integer lambda in [0, 2^62] whose per-group argmin of D 2^16 + lambda R
// (ties to the lower rate) fits the budget; then groups whose choice differs at
// lambda - 1 take it, in group order, until the first that would not fit.
//
// GPU structure: every group's choice as a function of lambda is a step function along
// the lower convex hull of its 14 (R, D) points; it is built once per group. The
// smallest feasible lambda is then found by a 64-way search whose passes only count
// step crossings, entirely on the device. Groups are stably partitioned by mode with
// the radix sort, and blocks are copied into their streams.
#include "gsc_internal.cuh"

__constant__ int c_modeB[GSC_MODES] = {1, 1, 4, 4, 4, 9, 9, 9, 9, 16, 16, 16, 16, 16};
__constant__ int c_modeJ[GSC_MODES] = {0, 1, 0, 1, 4, 0, 1, 4, 9, 0, 1, 4, 9, 16};
static const int h_modeB[GSC_MODES] = {1, 1, 4, 4, 4, 9, 9, 9, 9, 16, 16, 16, 16, 16};
static const int h_modeJ[GSC_MODES] = {0, 1, 0, 1, 4, 0, 1, 4, 9, 0, 1, 4, 9, 16};

#define N_PASSES 13

struct RateState {
  uint64_t lo, hi, budget;
  uint64_t min_total;   // sum of rates at lambda = 2^62 (every group in its cheapest mode)
  uint64_t sum_star;    // sum of rates at lambda*
  uint64_t used;        // bits after the fill step
  int infeasible, done;
  uint64_t cnt[N_PASSES][65];  // per pass: [0] sum at the first candidate, [1..63] decrements
  uint32_t counts[GSC_MODES];
};

struct StreamInfo {
  int64_t first[GSC_MODES], ngroups[GSC_MODES], offset[GSC_MODES];
  int64_t total_bytes;
  uint64_t lambda, used, budget;
  int infeasible;
  uint32_t weights[GSC_SH];
};

__device__ __forceinline__ uint64_t rate_of(int m) { return 64ull * (uint64_t)(c_modeB[m] + c_modeJ[m]); }

__global__ void k_weights(const float* __restrict__ scales, uint32_t* __restrict__ w) {
  if (threadIdx.x != 0) return;
  double mx = 0.0;
  for (int k = 0; k < GSC_SH; k++) { double s = scales[k]; if (s * s > mx) mx = s * s; }
  for (int k = 0; k < GSC_SH; k++) {
    double s = scales[k];
    double v = rint((s * s * 65536.0) / mx);
    w[k] = v < 1.0 ? 1u : (uint32_t)v;
  }
}

// 128-bit cost D * 2^16 + lambda * R as (hi, lo)
__device__ __forceinline__ void cost128(uint64_t d16, uint64_t lambda, uint64_t r, uint64_t& hi, uint64_t& lo) {
  uint64_t plo = lambda * r, phi = __umul64hi(lambda, r);
  lo = plo + d16;
  hi = phi + (lo < plo ? 1 : 0);
}

__device__ __forceinline__ int choose(const uint64_t (&D)[GSC_MODES], uint64_t lambda) {
  int best = 0;
  uint64_t bh, bl;
  cost128(D[0] << 16, lambda, rate_of(0), bh, bl);
#pragma unroll
  for (int m = 1; m < GSC_MODES; m++) {
    uint64_t h, l;
    cost128(D[m] << 16, lambda, rate_of(m), h, l);
    bool less = (h < bh) || (h == bh && l < bl);
    bool tie = (h == bh && l == bl);
    if (less || (tie && rate_of(m) < rate_of(best))) { best = m; bh = h; bl = l; }
  }
  return best;
}

// D table and the step function of each group's choice: steps[g][i] = (lambda_i, mode_i)
// with lambda_0 = 0; the choice at lambda is the mode of the last step with lambda_i <= lambda.
__global__ void k_dtable(const uint32_t* __restrict__ sse1, const uint32_t* __restrict__ sse7,
                         const uint32_t* __restrict__ sse0, const uint32_t* __restrict__ w, int64_t ng,
                         uint64_t* __restrict__ dtab, uint64_t* __restrict__ step_l, uint8_t* __restrict__ step_m,
                         uint8_t* __restrict__ n_steps, RateState* __restrict__ S) {
  __shared__ uint32_t s_w[GSC_SH];
  if (threadIdx.x < GSC_SH) s_w[threadIdx.x] = w[threadIdx.x];
  __syncthreads();
  uint64_t local_min = 0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
    uint64_t e1[GSC_SH], e7[GSC_SH], e0[GSC_SH];
#pragma unroll
    for (int k = 0; k < GSC_SH; k++) {
      e1[k] = (uint64_t)s_w[k] * sse1[g * 16 + k];
      e7[k] = (uint64_t)s_w[k] * sse7[g * 16 + k];
      e0[k] = (uint64_t)s_w[k] * sse0[g * 16 + k];
    }
    uint64_t D[GSC_MODES];
#pragma unroll
    for (int m = 0; m < GSC_MODES; m++) {
      uint64_t d = 0;
#pragma unroll
      for (int k = 0; k < GSC_SH; k++) d += k < c_modeJ[m] ? e7[k] : (k < c_modeB[m] ? e1[k] : e0[k]);
      D[m] = d;
      dtab[g * GSC_MODES + m] = d;
    }
    int m = choose(D, 0);
    int ns = 0;
    step_l[g * GSC_MODES + 0] = 0;
    step_m[g * GSC_MODES + 0] = (uint8_t)m;
    ns = 1;
    for (int it = 0; it < GSC_MODES; it++) {
      uint64_t next = ~0ull;
      for (int q = 0; q < GSC_MODES; q++) {
        if (rate_of(q) >= rate_of(m) || D[q] <= D[m]) continue;
        uint64_t num = (D[q] - D[m]) << 16, den = rate_of(m) - rate_of(q);
        uint64_t t = num / den + (num % den != 0);
        next = min(next, t);
      }
      if (next == ~0ull || ns >= GSC_MODES) break;
      m = choose(D, next);
      step_l[g * GSC_MODES + ns] = next;
      step_m[g * GSC_MODES + ns] = (uint8_t)m;
      ns++;
    }
    n_steps[g] = (uint8_t)ns;
    local_min += rate_of(step_m[g * GSC_MODES + ns - 1]);
  }
  atomicAdd((unsigned long long*)&S->min_total, (unsigned long long)local_min);
}

__global__ void k_search_init(RateState* S, uint64_t budget) {
  if (threadIdx.x == 0) {
    S->budget = budget;
    S->infeasible = S->min_total > budget;
    S->lo = 0;
    S->hi = 1ull << 62;
    S->done = S->infeasible;
  }
}

__device__ __forceinline__ void pass_params(const RateState* S, uint64_t& lo, uint64_t& step) {
  lo = S->lo;
  uint64_t span = S->hi - S->lo;
  step = span / 64 + (span % 64 != 0);
  if (step == 0) step = 1;
}

__global__ void k_search_count(const uint64_t* __restrict__ step_l, const uint8_t* __restrict__ step_m,
                               const uint8_t* __restrict__ n_steps, int64_t ng, RateState* __restrict__ S, int pass) {
  __shared__ unsigned long long acc[65];
  if (S->done) return;
  for (int i = threadIdx.x; i < 65; i += blockDim.x) acc[i] = 0;
  __syncthreads();
  uint64_t lo, step;
  pass_params(S, lo, step);
  uint64_t base = 0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
    const int ns = n_steps[g];
    int a = 0;
    while (a + 1 < ns && step_l[g * GSC_MODES + a + 1] <= lo) a++;
    uint64_t r = rate_of(step_m[g * GSC_MODES + a]);
    base += r;
    for (int b = a + 1; b < ns; b++) {
      const uint64_t lb = step_l[g * GSC_MODES + b];
      const uint64_t idx = (lb - lo) / step + ((lb - lo) % step != 0);  // first candidate >= lb
      const uint64_t r2 = rate_of(step_m[g * GSC_MODES + b]);
      if (idx <= 63) atomicAdd(&acc[idx], (unsigned long long)(r - r2));
      r = r2;
    }
  }
  atomicAdd(&acc[64], (unsigned long long)base);
  __syncthreads();
  for (int i = threadIdx.x; i < 65; i += blockDim.x) {
    const int slot = i == 64 ? 0 : i;  // cnt[0] = base, cnt[i] = decrement at candidate i
    if (acc[i] && !(i == 0)) atomicAdd((unsigned long long*)&S->cnt[pass][slot], acc[i]);
  }
}

__global__ void k_search_narrow(RateState* S, int pass) {
  if (threadIdx.x != 0 || S->done) return;
  uint64_t lo, step;
  pass_params(S, lo, step);
  const uint64_t hi = S->hi, B = S->budget;
  uint64_t f = S->cnt[pass][0];
  int found = -1;
  uint64_t last_bad = 0;
  for (int i = 0; i < 64; i++) {
    const uint64_t c = lo + step * (uint64_t)i;
    if (c > hi) break;
    if (i > 0) f -= S->cnt[pass][i];
    if (f <= B) { found = i; break; }
    last_bad = c;
  }
  if (found == 0) { S->hi = lo; }
  else if (found > 0) { S->lo = lo + step * (uint64_t)(found - 1) + 1; S->hi = lo + step * (uint64_t)found; }
  else { S->lo = last_bad + 1; }
  if (S->lo >= S->hi) { S->lo = S->hi; S->done = 1; }
}

__device__ __forceinline__ int mode_at(const uint64_t* step_l, const uint8_t* step_m, int ns, int64_t g, uint64_t lam) {
  int a = 0;
  while (a + 1 < ns && step_l[g * GSC_MODES + a + 1] <= lam) a++;
  return step_m[g * GSC_MODES + a];
}

__global__ void k_fill_prep(const uint64_t* __restrict__ step_l, const uint8_t* __restrict__ step_m,
                            const uint8_t* __restrict__ n_steps, int64_t ng, RateState* __restrict__ S,
                            uint8_t* __restrict__ mode, uint8_t* __restrict__ alt, uint64_t* __restrict__ delta) {
  const uint64_t lam = S->lo;
  uint64_t sum = 0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
    const int ns = n_steps[g];
    const int m = mode_at(step_l, step_m, ns, g, lam);
    const int m2 = lam > 0 ? mode_at(step_l, step_m, ns, g, lam - 1) : m;
    mode[g] = (uint8_t)m;
    alt[g] = (uint8_t)m2;
    delta[g] = rate_of(m2) - rate_of(m);
    sum += rate_of(m);
  }
  atomicAdd((unsigned long long*)&S->sum_star, (unsigned long long)sum);
}

__global__ void k_fill_apply(int64_t ng, RateState* __restrict__ S, uint8_t* __restrict__ mode,
                             const uint8_t* __restrict__ alt, const uint64_t* __restrict__ delta,
                             const uint64_t* __restrict__ prefix, uint64_t* __restrict__ keys,
                             uint32_t* __restrict__ vals) {
  __shared__ uint32_t cnt[GSC_MODES];
  __shared__ unsigned long long used;
  if (threadIdx.x < GSC_MODES) cnt[threadIdx.x] = 0;
  if (threadIdx.x == 0) used = 0;
  __syncthreads();
  const uint64_t slack = S->budget - S->sum_star;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
    int m = mode[g];
    if (delta[g] > 0 && prefix[g] + delta[g] <= slack) m = alt[g];
    mode[g] = (uint8_t)m;
    keys[g] = (uint64_t)m;
    vals[g] = (uint32_t)g;
    atomicAdd(&cnt[m], 1u);
    atomicAdd(&used, (unsigned long long)rate_of(m));
  }
  __syncthreads();
  if (threadIdx.x < GSC_MODES && cnt[threadIdx.x]) atomicAdd(&S->counts[threadIdx.x], cnt[threadIdx.x]);
  if (threadIdx.x == 0 && used) atomicAdd((unsigned long long*)&S->used, used);
}

__global__ void k_stream_info(const RateState* __restrict__ S, const uint32_t* __restrict__ w,
                              StreamInfo* __restrict__ info) {
  if (threadIdx.x != 0) return;
  int64_t g = 0, off = 0;
  for (int m = 0; m < GSC_MODES; m++) {
    info->first[m] = g;
    info->ngroups[m] = S->counts[m];
    info->offset[m] = off;
    g += S->counts[m];
    off += (int64_t)S->counts[m] * (16 * c_modeJ[m] + 8 * (c_modeB[m] - c_modeJ[m]));
  }
  info->total_bytes = off;
  info->lambda = S->lo;
  info->used = S->used;
  info->budget = S->budget;
  info->infeasible = S->infeasible;
  for (int k = 0; k < GSC_SH; k++) info->weights[k] = w[k];
}

__global__ void k_assemble(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ order, int64_t ng,
                           const StreamInfo* __restrict__ info, const uint2* __restrict__ b1,
                           const uint2* __restrict__ b7, const int32_t* __restrict__ perm, uint8_t* __restrict__ out,
                           int32_t* __restrict__ perm_out) {
  for (int64_t G = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; G < ng; G += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = order[G];
    const int m = (int)keys[G];
    const int J = c_modeJ[m], B = c_modeB[m];
    const int64_t gbytes = 16 * J + 8 * (B - J);
    uint2* dst = reinterpret_cast<uint2*>(out + info->offset[m] + (G - info->first[m]) * gbytes);
    for (int k = 0; k < J; k++) { dst[2 * k] = b7[(g * 16 + k) * 2]; dst[2 * k + 1] = b7[(g * 16 + k) * 2 + 1]; }
    for (int k = J; k < B; k++) dst[2 * J + (k - J)] = b1[g * 16 + k];
#pragma unroll
    for (int t = 0; t < 16; t++) perm_out[G * 16 + t] = perm[g * 16 + t];
  }
}

static int gsz(int64_t n, int threads, int cap) {
  int64_t g = ceil_div64(n > 0 ? n : 1, threads);
  return (int)(g > cap ? cap : g);
}

// Stream selection from the per-block codings and errors of every block: D table,
// lambda search, fill, stable partition, assembly; fills *table (synchronises st).
gsc_status rate_select(gsc_ctx* ctx, int64_t n, const int32_t* perm, const float* scales, uint32_t target_x4,
                       const uint8_t* b1, const uint8_t* b7, const uint32_t* sse1, const uint32_t* sse7,
                       const uint32_t* sse0, uint8_t* blocks, int32_t* perm_out, gsc_stream_table* table, void* ws,
                       size_t ws_bytes, cudaStream_t st) {
  const int64_t ng = ceil_div64(n, 16);
  if (ws_bytes < rate_select_ws_bytes(ng)) return GSC_ERR_OOM;
  Carve c{reinterpret_cast<uint8_t*>(ws), 0, ws_bytes};
  uint64_t* dtab = c.take<uint64_t>(ng * GSC_MODES);
  uint64_t* step_l = c.take<uint64_t>(ng * GSC_MODES);
  uint8_t* step_m = c.take<uint8_t>(ng * GSC_MODES);
  uint8_t* n_steps = c.take<uint8_t>(ng);
  uint8_t* mode = c.take<uint8_t>(ng);
  uint8_t* alt = c.take<uint8_t>(ng);
  uint64_t* delta = c.take<uint64_t>(ng);
  uint64_t* prefix = c.take<uint64_t>(ng);
  uint64_t* keys = c.take<uint64_t>(ng);
  uint32_t* vals = c.take<uint32_t>(ng);
  RateState* S = c.take<RateState>(1);
  StreamInfo* info = c.take<StreamInfo>(1);
  uint32_t* w = c.take<uint32_t>(GSC_SH);
  void* rws = c.take<uint8_t>((int64_t)radix_ws_bytes(ng));
  void* sws = c.take<uint8_t>((int64_t)scan_ws_bytes(ng));
  const uint64_t budget = (uint64_t)target_x4 * 4ull * (uint64_t)n;
  const int cap = ctx->sm_count * 8;
  GscTimed tm_rate(ctx, T_RATE, st);
  GSC_CUDA(cudaMemsetAsync(S, 0, sizeof(RateState), st));
  gsc_count_launch(); k_weights<<<1, 32, 0, st>>>(scales, w);
  gsc_count_launch(); k_dtable<<<gsz(ng, 128, cap), 128, 0, st>>>(sse1, sse7, sse0, w, ng, dtab, step_l, step_m, n_steps, S);
  gsc_count_launch(); k_search_init<<<1, 32, 0, st>>>(S, budget);
  for (int p = 0; p < N_PASSES; p++) {
    gsc_count_launch(); k_search_count<<<gsz(ng, 256, cap), 256, 0, st>>>(step_l, step_m, n_steps, ng, S, p);
    gsc_count_launch(); k_search_narrow<<<1, 32, 0, st>>>(S, p);
  }
  gsc_count_launch(); k_fill_prep<<<gsz(ng, 256, cap), 256, 0, st>>>(step_l, step_m, n_steps, ng, S, mode, alt, delta);
  GSC_CUDA(cudaGetLastError());
  GSC_CUDA(scan_exclusive<uint64_t>(delta, prefix, ng, nullptr, sws, st));
  gsc_count_launch(); k_fill_apply<<<gsz(ng, 256, cap), 256, 0, st>>>(ng, S, mode, alt, delta, prefix, keys, vals);
  gsc_count_launch(); k_stream_info<<<1, 32, 0, st>>>(S, w, info);
  GSC_CUDA(cudaGetLastError());
  GSC_CUDA(radix_sort_pairs(keys, vals, ng, 4, rws, st));
  gsc_count_launch(); k_assemble<<<gsz(ng, 128, cap), 128, 0, st>>>(keys, vals, ng, info, reinterpret_cast<const uint2*>(b1),
                                                 reinterpret_cast<const uint2*>(b7), perm, blocks, perm_out);
  GSC_CUDA(cudaGetLastError());
  gsc_timer_end(ctx, tm_rate.rec, st);
  tm_rate.rec = -1;
  StreamInfo* h = reinterpret_cast<StreamInfo*>(ctx->h_pinned);
  GSC_CUDA(cudaMemcpyAsync(h, info, sizeof(StreamInfo), cudaMemcpyDeviceToHost, st));
  GSC_CUDA(cudaStreamSynchronize(st));
  if (h->infeasible) return GSC_ERR_BUDGET;
  table->n_streams = GSC_MODES;
  table->format = GSC_FMT_RATE;
  table->n = n;
  table->n_groups = ng;
  table->total_bytes = h->total_bytes;
  table->budget_bits = h->budget;
  table->used_bits = h->used;
  table->lambda = h->lambda;
  for (int k = 0; k < GSC_SH; k++) table->weights[k] = h->weights[k];
  for (int m = 0; m < GSC_MODES; m++) {
    table->s[m].bands = h_modeB[m];
    table->s[m].bc7_blocks = h_modeJ[m];
    table->s[m].first_group = h->first[m];
    table->s[m].n_groups = h->ngroups[m];
    table->s[m].byte_offset = h->offset[m];
  }
  return GSC_OK;
}

size_t rate_select_ws_bytes(int64_t ng) {
  size_t b = 0;
  b += align_up(8 * (size_t)ng * GSC_MODES, 256);                             // D
  b += align_up(8 * (size_t)ng * GSC_MODES, 256) + align_up((size_t)ng * GSC_MODES, 256);  // steps
  b += 3 * align_up((size_t)ng, 256);                                         // n_steps, mode, alt
  b += 2 * align_up(8 * (size_t)ng, 256);                                     // delta, prefix
  b += align_up(8 * (size_t)ng, 256) + align_up(4 * (size_t)ng, 256);         // keys, vals
  b += align_up(sizeof(RateState), 256) + align_up(sizeof(StreamInfo), 256) + align_up(64, 256);
  b += radix_ws_bytes(ng) + scan_ws_bytes(ng);
  return b + 8192;
}

gsc_status rate_run(gsc_ctx* ctx, const float* sh, int64_t n, const int32_t* perm, const float* scales,
                    uint32_t target_x4, uint8_t* blocks, int32_t* perm_out, gsc_stream_table* table, void* ws,
                    size_t ws_bytes, uint8_t* bc1_all, uint8_t* bc7_all, cudaStream_t st) {
  const int64_t ng = ceil_div64(n, 16);
  if (ws_bytes < rate_ws_bytes(ng)) return GSC_ERR_OOM;
  Carve c{reinterpret_cast<uint8_t*>(ws), 0, ws_bytes};
  uint8_t* b1 = c.take<uint8_t>(8 * ng * 16);
  uint8_t* b7 = c.take<uint8_t>(16 * ng * 16);
  if (bc1_all) b1 = bc1_all;   // the caller keeps the all-BC1 / all-BC7 codings
  if (bc7_all) b7 = bc7_all;
  uint32_t* sse1 = c.take<uint32_t>(ng * 16);
  uint32_t* sse7 = c.take<uint32_t>(ng * 16);
  uint32_t* sse0 = c.take<uint32_t>(ng * 16);
  const size_t used = align_up(c.off, 256);
  {
    GscTimed tm(ctx, T_BC1, st);
    GSC_CUDA(launch_bc1_groups(sh, perm, scales, ng, b1, sse1, sse0, st));
  }
  {
    GscTimed tm(ctx, T_BC7, st);
    GSC_CUDA(launch_bc7_groups(sh, perm, scales, ng, b7, sse7, st));
  }
  return rate_select(ctx, n, perm, scales, target_x4, b1, b7, sse1, sse7, sse0, blocks, perm_out, table,
                     reinterpret_cast<uint8_t*>(ws) + used, ws_bytes - used, st);
}

size_t rate_ws_bytes(int64_t ng) {
  const int64_t nb = ng * 16;
  return align_up(8 * (size_t)nb, 256) + align_up(16 * (size_t)nb, 256) + 3 * align_up(4 * (size_t)nb, 256) + 1024 +
         rate_select_ws_bytes(ng);
}

// ---- one scene split over shards (Sec. IV-B: one rate budget for the whole scene) -----------
// A shard holds whole groups of the scene's slot order (the whole-scene plan split at chunk
// boundaries). Each phase leaves an integer partial that the caller sums (or gathers) over the
// shards and hands to the next phase; with those sums every shard takes the decisions the
// whole-scene search takes, and writes its groups where the whole-scene call writes them.
#define SHARD_PART 15  // per shard after the fill: groups per mode [14] and bits used

struct ShardInfo {
  int64_t first[GSC_MODES], ngroups[GSC_MODES], offset[GSC_MODES], before[GSC_MODES], local_first[GSC_MODES];
  int64_t total_bytes, ng_total;
  uint64_t lambda, used, budget;
  int infeasible;
  uint32_t weights[GSC_SH];
};

struct ShardRate {
  uint32_t *sse1, *sse7, *sse0;
  uint64_t *dtab, *step_l;
  uint8_t *step_m, *n_steps, *mode, *alt;
  uint64_t *delta, *prefix, *keys, *total;
  uint32_t *vals, *w;
  RateState* S;
  ShardInfo* info;
  void *rws, *sws;
  size_t end;
};

static ShardRate shard_carve(void* ws, int64_t ng) {
  Carve c{reinterpret_cast<uint8_t*>(ws), 0, 0};
  ShardRate r;
  r.sse1 = c.take<uint32_t>(ng * 16);
  r.sse7 = c.take<uint32_t>(ng * 16);
  r.sse0 = c.take<uint32_t>(ng * 16);
  r.dtab = c.take<uint64_t>(ng * GSC_MODES);
  r.step_l = c.take<uint64_t>(ng * GSC_MODES);
  r.step_m = c.take<uint8_t>(ng * GSC_MODES);
  r.n_steps = c.take<uint8_t>(ng);
  r.mode = c.take<uint8_t>(ng);
  r.alt = c.take<uint8_t>(ng);
  r.delta = c.take<uint64_t>(ng);
  r.prefix = c.take<uint64_t>(ng);
  r.keys = c.take<uint64_t>(ng);
  r.total = c.take<uint64_t>(1);
  r.vals = c.take<uint32_t>(ng);
  r.w = c.take<uint32_t>(GSC_SH);
  r.S = c.take<RateState>(1);
  r.info = c.take<ShardInfo>(1);
  r.rws = c.take<uint8_t>((int64_t)radix_ws_bytes(ng));
  r.sws = c.take<uint8_t>((int64_t)scan_ws_bytes(ng));
  r.end = c.off;
  return r;
}

size_t shard_rate_ws_bytes(int64_t ng) { return shard_carve(nullptr, ng).end + 256; }

__global__ void k_shard_put(const RateState* __restrict__ S, int what, int pass, int64_t* __restrict__ part) {
  const int i = threadIdx.x;
  if (what == 0 && i == 0) part[0] = (int64_t)S->min_total;
  if (what == 1 && i < 64) part[i] = (int64_t)S->cnt[pass][i];
  if (what == 2 && i < GSC_MODES) part[i] = (int64_t)S->counts[i];
  if (what == 2 && i == GSC_MODES) part[i] = (int64_t)S->used;
}

__global__ void k_shard_search_init(RateState* S, const int64_t* __restrict__ min_total, uint64_t budget) {
  if (threadIdx.x != 0) return;
  S->min_total = (uint64_t)min_total[0];
  S->budget = budget;
  S->infeasible = S->min_total > budget;
  S->lo = 0;
  S->hi = 1ull << 62;
  S->done = S->infeasible;
}

__global__ void k_shard_set_cnt(RateState* S, int pass, const int64_t* __restrict__ tot) {
  if (threadIdx.x < 64) S->cnt[pass][threadIdx.x] = (uint64_t)tot[threadIdx.x];
}

__global__ void k_shard_fill_part(const RateState* __restrict__ S, const uint64_t* __restrict__ total,
                                  int64_t* __restrict__ part) {
  if (threadIdx.x == 0) { part[0] = (int64_t)S->sum_star; part[1] = (int64_t)total[0]; }
}

__global__ void k_shard_offsets(RateState* S, const int64_t* __restrict__ in, uint64_t* __restrict__ prefix, int64_t ng) {
  if (blockIdx.x == 0 && threadIdx.x == 0) S->sum_star = (uint64_t)in[0];
  const uint64_t before = (uint64_t)in[1];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x)
    prefix[g] += before;
}

__global__ void k_shard_info(const RateState* __restrict__ S, const uint32_t* __restrict__ w,
                             const int64_t* __restrict__ counts_all, int n_shards, int shard, ShardInfo* __restrict__ info) {
  if (threadIdx.x != 0) return;
  int64_t g = 0, off = 0, lf = 0, ngt = 0;
  uint64_t used = 0;
  for (int s = 0; s < n_shards; s++) used += (uint64_t)counts_all[s * SHARD_PART + GSC_MODES];
  for (int m = 0; m < GSC_MODES; m++) {
    int64_t tot = 0, before = 0;
    for (int s = 0; s < n_shards; s++) {
      const int64_t c = counts_all[s * SHARD_PART + m];
      tot += c;
      if (s < shard) before += c;
    }
    info->first[m] = g;
    info->ngroups[m] = tot;
    info->offset[m] = off;
    info->before[m] = before;
    info->local_first[m] = lf;
    lf += counts_all[shard * SHARD_PART + m];
    g += tot;
    off += tot * (16 * c_modeJ[m] + 8 * (c_modeB[m] - c_modeJ[m]));
    ngt += tot;
  }
  info->total_bytes = off;
  info->ng_total = ngt;
  info->lambda = S->lo;
  info->used = used;
  info->budget = S->budget;
  info->infeasible = S->infeasible;
  for (int k = 0; k < GSC_SH; k++) info->weights[k] = w[k];
}

__global__ void k_shard_assemble(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ order, int64_t ng,
                                 const ShardInfo* __restrict__ info, const uint2* __restrict__ b1,
                                 const uint2* __restrict__ b7, const int32_t* __restrict__ perm,
                                 const int32_t* __restrict__ index_map, uint8_t* __restrict__ out,
                                 int32_t* __restrict__ perm_out) {
  for (int64_t G = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; G < ng; G += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = order[G];
    const int m = (int)keys[G];
    const int J = c_modeJ[m], B = c_modeB[m];
    const int64_t gbytes = 16 * J + 8 * (B - J);
    const int64_t in_stream = info->before[m] + (G - info->local_first[m]);
    uint2* dst = reinterpret_cast<uint2*>(out + info->offset[m] + in_stream * gbytes);
    for (int k = 0; k < J; k++) { dst[2 * k] = b7[(g * 16 + k) * 2]; dst[2 * k + 1] = b7[(g * 16 + k) * 2 + 1]; }
    for (int k = J; k < B; k++) dst[2 * J + (k - J)] = b1[g * 16 + k];
    const int64_t gs = info->first[m] + in_stream;
#pragma unroll
    for (int t = 0; t < 16; t++) {
      const int32_t p = perm[g * 16 + t];
      perm_out[gs * 16 + t] = (p >= 0 && index_map) ? index_map[p] : p;
    }
  }
}

gsc_status shard_rate_begin(gsc_ctx* ctx, const float* sh, int64_t n, const int32_t* perm, const float* scales,
                            uint8_t* b1, uint8_t* b7, void* ws, size_t ws_bytes, int64_t* part, cudaStream_t st) {
  const int64_t ng = ceil_div64(n, 16);
  if (ws_bytes < shard_rate_ws_bytes(ng)) return GSC_ERR_OOM;
  ShardRate r = shard_carve(ws, ng);
  const int cap = ctx->sm_count * 8;
  GSC_CUDA(cudaMemsetAsync(r.S, 0, sizeof(RateState), st));
  if (ng > 0) {
    {
      GscTimed tm(ctx, T_BC1, st);
      GSC_CUDA(launch_bc1_groups(sh, perm, scales, ng, b1, r.sse1, r.sse0, st));
    }
    {
      GscTimed tm(ctx, T_BC7, st);
      GSC_CUDA(launch_bc7_groups(sh, perm, scales, ng, b7, r.sse7, st));
    }
  }
  gsc_count_launch(); k_weights<<<1, 32, 0, st>>>(scales, r.w);
  if (ng > 0) {
    gsc_count_launch();
    k_dtable<<<gsz(ng, 128, cap), 128, 0, st>>>(r.sse1, r.sse7, r.sse0, r.w, ng, r.dtab, r.step_l, r.step_m, r.n_steps, r.S);
  }
  gsc_count_launch(); k_shard_put<<<1, 64, 0, st>>>(r.S, 0, 0, part);
  GSC_CUDA(cudaGetLastError());
  return GSC_OK;
}

gsc_status shard_rate_search_begin(int64_t ng, void* ws, int64_t n_total, uint32_t target_x4, const int64_t* min_total,
                                   cudaStream_t st) {
  ShardRate r = shard_carve(ws, ng);
  const uint64_t budget = (uint64_t)target_x4 * 4ull * (uint64_t)n_total;
  gsc_count_launch(); k_shard_search_init<<<1, 32, 0, st>>>(r.S, min_total, budget);
  GSC_CUDA(cudaGetLastError());
  return GSC_OK;
}

gsc_status shard_rate_count(gsc_ctx* ctx, int64_t ng, void* ws, int pass, int64_t* part, cudaStream_t st) {
  ShardRate r = shard_carve(ws, ng);
  if (ng > 0) {
    gsc_count_launch();
    k_search_count<<<gsz(ng, 256, ctx->sm_count * 8), 256, 0, st>>>(r.step_l, r.step_m, r.n_steps, ng, r.S, pass);
  }
  gsc_count_launch(); k_shard_put<<<1, 64, 0, st>>>(r.S, 1, pass, part);
  GSC_CUDA(cudaGetLastError());
  return GSC_OK;
}

gsc_status shard_rate_narrow(int64_t ng, void* ws, int pass, const int64_t* total, cudaStream_t st) {
  ShardRate r = shard_carve(ws, ng);
  gsc_count_launch(); k_shard_set_cnt<<<1, 64, 0, st>>>(r.S, pass, total);
  gsc_count_launch(); k_search_narrow<<<1, 32, 0, st>>>(r.S, pass);
  GSC_CUDA(cudaGetLastError());
  return GSC_OK;
}

gsc_status shard_rate_fill(gsc_ctx* ctx, int64_t ng, void* ws, int64_t* part, cudaStream_t st) {
  ShardRate r = shard_carve(ws, ng);
  GSC_CUDA(cudaMemsetAsync(r.total, 0, sizeof(uint64_t), st));
  if (ng > 0) {
    gsc_count_launch();
    k_fill_prep<<<gsz(ng, 256, ctx->sm_count * 8), 256, 0, st>>>(r.step_l, r.step_m, r.n_steps, ng, r.S, r.mode, r.alt,
                                                                 r.delta);
    GSC_CUDA(cudaGetLastError());
    GSC_CUDA(scan_exclusive<uint64_t>(r.delta, r.prefix, ng, r.total, r.sws, st));
  }
  gsc_count_launch(); k_shard_fill_part<<<1, 32, 0, st>>>(r.S, r.total, part);
  GSC_CUDA(cudaGetLastError());
  return GSC_OK;
}

gsc_status shard_rate_apply(gsc_ctx* ctx, int64_t ng, void* ws, const int64_t* in, int64_t* part, cudaStream_t st) {
  ShardRate r = shard_carve(ws, ng);
  const int cap = ctx->sm_count * 8;
  gsc_count_launch(); k_shard_offsets<<<gsz(ng, 256, cap), 256, 0, st>>>(r.S, in, r.prefix, ng);
  if (ng > 0) {
    gsc_count_launch();
    k_fill_apply<<<gsz(ng, 256, cap), 256, 0, st>>>(ng, r.S, r.mode, r.alt, r.delta, r.prefix, r.keys, r.vals);
  }
  gsc_count_launch(); k_shard_put<<<1, 64, 0, st>>>(r.S, 2, 0, part);
  GSC_CUDA(cudaGetLastError());
  return GSC_OK;
}

gsc_status shard_rate_assemble(gsc_ctx* ctx, int64_t ng, void* ws, const uint8_t* b1, const uint8_t* b7,
                               const int32_t* perm, const int32_t* index_map, const int64_t* counts_all, int n_shards,
                               int shard, int64_t n_total, uint8_t* blocks, int32_t* perm_out, gsc_stream_table* table,
                               cudaStream_t st) {
  ShardRate r = shard_carve(ws, ng);
  gsc_count_launch(); k_shard_info<<<1, 32, 0, st>>>(r.S, r.w, counts_all, n_shards, shard, r.info);
  GSC_CUDA(cudaGetLastError());
  if (ng > 0) {
    GSC_CUDA(radix_sort_pairs(r.keys, r.vals, ng, 4, r.rws, st));
    gsc_count_launch();
    k_shard_assemble<<<gsz(ng, 128, ctx->sm_count * 8), 128, 0, st>>>(
        r.keys, r.vals, ng, r.info, reinterpret_cast<const uint2*>(b1), reinterpret_cast<const uint2*>(b7), perm,
        index_map, blocks, perm_out);
    GSC_CUDA(cudaGetLastError());
  }
  ShardInfo* h = reinterpret_cast<ShardInfo*>(ctx->h_pinned);
  GSC_CUDA(cudaMemcpyAsync(h, r.info, sizeof(ShardInfo), cudaMemcpyDeviceToHost, st));
  GSC_CUDA(cudaStreamSynchronize(st));
  if (h->infeasible) return GSC_ERR_BUDGET;
  table->n_streams = GSC_MODES;
  table->format = GSC_FMT_RATE;
  table->n = n_total;
  table->n_groups = h->ng_total;
  table->total_bytes = h->total_bytes;
  table->budget_bits = h->budget;
  table->used_bits = h->used;
  table->lambda = h->lambda;
  for (int k = 0; k < GSC_SH; k++) table->weights[k] = h->weights[k];
  for (int m = 0; m < GSC_MODES; m++) {
    table->s[m].bands = h_modeB[m];
    table->s[m].bc7_blocks = h_modeJ[m];
    table->s[m].first_group = h->first[m];
    table->s[m].n_groups = h->ngroups[m];
    table->s[m].byte_offset = h->offset[m];
  }
  return GSC_OK;
}
