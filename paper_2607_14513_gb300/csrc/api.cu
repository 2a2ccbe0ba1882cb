// api.cu -- the C ABI declared in include/gsc.h: context, argument checks, orchestration.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "gsc_internal.cuh"
#include "layout.cuh"

#include <atomic>

#define PINNED_BYTES 65536

static std::atomic<unsigned long long> g_launches{0};
void gsc_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
extern "C" uint64_t gsc_launch_count(void) { return g_launches.load(); }

static const char* kTimerNames[T_COUNT] = {"plan", "bc1_encode", "bc7_encode", "rate_select", "decode",
                                           "decode_eval", "decode_tex", "decode_eval_tex", "batch_encode", "render",
                                           "render_blend"};

int gsc_timer_begin(gsc_ctx* c, int id, cudaStream_t st) {
  if (!c || !c->timing) return -1;
  if (c->n_recs == c->cap_recs) {
    int cap = c->cap_recs ? 2 * c->cap_recs : 256;
    gsc_timer_rec* r = (gsc_timer_rec*)realloc(c->recs, sizeof(gsc_timer_rec) * cap);
    if (!r) return -1;
    c->recs = r;
    c->cap_recs = cap;
  }
  gsc_timer_rec& r = c->recs[c->n_recs];
  if (cudaEventCreate(&r.a) != cudaSuccess) return -1;
  if (cudaEventCreate(&r.b) != cudaSuccess) { cudaEventDestroy(r.a); return -1; }
  r.id = id;
  cudaEventRecord(r.a, st);
  return c->n_recs++;
}

void gsc_timer_end(gsc_ctx* c, int rec, cudaStream_t st) {
  if (!c || rec < 0) return;
  cudaEventRecord(c->recs[rec].b, st);
}

static void timer_drain(gsc_ctx* c) {
  for (int i = 0; i < c->n_recs; i++) {
    gsc_timer_rec& r = c->recs[i];
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      c->t_ms[r.id] += ms;
      c->t_launches[r.id] += 1;
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  c->n_recs = 0;
}

extern "C" gsc_status gsc_ctx_set_timing(gsc_ctx* c, int enable) {
  if (!c) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  timer_drain(c);
  for (int i = 0; i < T_COUNT; i++) { c->t_ms[i] = 0.0; c->t_launches[i] = 0; }
  c->timing = enable ? 1 : 0;
  return GSC_OK;
}

extern "C" gsc_status gsc_kernel_time(gsc_ctx* c, const char* name, double* ms, int64_t* launches) {
  if (!c || !name || !ms || !launches) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  timer_drain(c);
  for (int i = 0; i < T_COUNT; i++)
    if (strcmp(name, kTimerNames[i]) == 0) { *ms = c->t_ms[i]; *launches = c->t_launches[i]; return GSC_OK; }
  return GSC_ERR_INVALID_ARG;
}

// Integer throughput probe: 8 independent chains per thread, each step an add of three
// values, a three-input logic op and a multiply-add.
__global__ void k_int_peak(uint32_t* out, int iters, uint32_t seed) {
  uint32_t a[8], b[8];
#pragma unroll
  for (int j = 0; j < 8; j++) { a[j] = seed * (threadIdx.x + 1) + j; b[j] = seed ^ (blockIdx.x * 77 + j); }
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < 8; j++) {
      a[j] = a[j] + b[j] + 0x9E3779B9u;
      b[j] = (b[j] ^ a[j]) | 0x5BD1E995u;
      a[j] = a[j] * b[j] + 0x3C6EF372u;
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < 8; j++) s ^= a[j] + b[j];
  if (s == 0x12345678u) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

extern "C" gsc_status gsc_probe_int_peak(gsc_ctx* c, double* ops_per_s, void* stream) {
  if (!c || !ops_per_s) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int threads = 256, blocks = c->sm_count * 8, iters = 4096;
  uint32_t* d = nullptr;
  GSC_CUDA(cudaMalloc(&d, sizeof(uint32_t) * threads * blocks));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; rep++) {
    cudaEventRecord(e0, st);
    gsc_count_launch(); k_int_peak<<<blocks, threads, 0, st>>>(d, iters, 0x1234567u + rep);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (e != cudaSuccess) return GSC_ERR_CUDA;
  *ops_per_s = (double)threads * blocks * iters * 8.0 * 3.0 / (best * 1e-3);
  return GSC_OK;
}

// Per-instruction throughput probes: 8 independent pairs of chains per thread; each step of a
// pair is two instructions of one kind whose operands change every iteration, so no two of them
// fold into one. Kind 5 is the BC7 search's palette evaluation: a dot product of a texel with a
// palette entry, the scaled key (key - 32 * dot) and a running minimum, over 8 entries per texel.
template <int KIND>
__global__ void k_op_probe(uint32_t* out, int iters, uint32_t seed) {
  uint32_t x[8], y[8];
#pragma unroll
  for (int j = 0; j < 8; j++) { x[j] = seed * (threadIdx.x + 1) + 97u * j; y[j] = (seed ^ (blockIdx.x * 77u)) + 31u * j; }
  for (int i = 0; i < iters; i++) {
    const uint32_t k = (uint32_t)i * 0x01030507u + seed;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      if (KIND == 1) {
        x[j] = x[j] + y[j] + k;
        y[j] = y[j] + x[j] + k;
      } else if (KIND == 2) {
        asm("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[j]) : "r"(y[j]), "r"(k));
        asm("lop3.b32 %0, %0, %1, %2, 0xE8;" : "+r"(y[j]) : "r"(x[j]), "r"(k));
      } else if (KIND == 3) {
        x[j] = x[j] * y[j] + k;
        y[j] = y[j] * x[j] + k;
      } else if (KIND == 4) {
        x[j] = (uint32_t)__dp4a(x[j], y[j], k);
        y[j] = (uint32_t)__dp4a(y[j], x[j], k);
      } else {
        // x[j]: palette entry (fixed), y[j]: running minimum; 8 entries share one texel value k
        const int key = (int)(x[j] & 0xFFFFu) - 32 * (int)__dp4a(k, x[j], 0u);
        y[j] = (uint32_t)min((int)y[j], key);
      }
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < 8; j++) s ^= x[j] + y[j];
  if (s == 0x12345678u) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

extern "C" gsc_status gsc_probe_op_rate(gsc_ctx* c, int32_t kind, double* ops_per_s, void* stream) {
  if (!c || !ops_per_s || kind < 1 || kind > 5) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int threads = 256, blocks = c->sm_count * 8, iters = 4096;
  uint32_t* d = nullptr;
  GSC_CUDA(cudaMalloc(&d, sizeof(uint32_t) * threads * blocks));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; rep++) {
    const uint32_t seed = 0x1234567u + rep;
    cudaEventRecord(e0, st);
    gsc_count_launch();
    switch (kind) {
      case 1: k_op_probe<1><<<blocks, threads, 0, st>>>(d, iters, seed); break;
      case 2: k_op_probe<2><<<blocks, threads, 0, st>>>(d, iters, seed); break;
      case 3: k_op_probe<3><<<blocks, threads, 0, st>>>(d, iters, seed); break;
      case 4: k_op_probe<4><<<blocks, threads, 0, st>>>(d, iters, seed); break;
      default: k_op_probe<5><<<blocks, threads, 0, st>>>(d, iters, seed); break;
    }
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (e != cudaSuccess) return GSC_ERR_CUDA;
  // kinds 1-4: two instructions per chain pair and step; kind 5: three (dot, scaled key, minimum)
  *ops_per_s = (double)threads * blocks * iters * 8.0 * (kind == 5 ? 3.0 : 2.0) / (best * 1e-3);
  return GSC_OK;
}

extern "C" gsc_status gsc_probe_bc7_mode1(gsc_ctx* c, const uint8_t* d_tex, int64_t nblk, int32_t warp_per_block,
                                          uint32_t* d_sse, int32_t* d_part, double* ms, void* stream) {
  if (!c || !ms || nblk < 0 || nblk > ((int64_t)1 << 40) || (warp_per_block != 0 && warp_per_block != 1))
    return GSC_ERR_INVALID_ARG;
  if (nblk > 0 && (!d_tex || !d_sse || !d_part)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  GSC_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return GSC_ERR_CUDA; }
  cudaEventRecord(e0, st);
  cudaError_t e = launch_bc7_mode1(d_tex, nblk, warp_per_block, d_sse, d_part, c->sm_count, st);
  cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return GSC_ERR_CUDA;
  *ms = t;
  return GSC_OK;
}

int gsc_sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return 1; }
  if (dev >= 0 && dev < 64) {
    const int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int sm = 0;
  if (cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sm <= 0) {
    cudaGetLastError();
    sm = 1;
  }
  if (dev >= 0 && dev < 64) cache[dev].store(sm, std::memory_order_relaxed);
  return sm;
}

static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

extern "C" const char* gsc_status_string(gsc_status s) {
  switch (s) {
    case GSC_OK: return "ok";
    case GSC_ERR_INVALID_ARG: return "invalid argument";
    case GSC_ERR_CUDA: return "CUDA runtime error";
    case GSC_ERR_OOM: return "workspace too small";
    case GSC_ERR_BUDGET: return "rate target below the cheapest coding of the scene";
    case GSC_ERR_TIMEOUT: return "device-side wait timed out";
    case GSC_ERR_UNSUPPORTED: return "no usable sm_103 device";
    case GSC_ERR_DEVICE: return "device-side check failed";
    case GSC_ERR_CANCELLED: return "request cancelled";
    default: return "unknown status";
  }
}

extern "C" gsc_status gsc_ctx_create(gsc_ctx** out, int device) { return ctx_new(device, true, out); }

gsc_status ctx_new(int device, bool init_tables, gsc_ctx** out) {
  if (!out) return GSC_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return GSC_ERR_UNSUPPORTED;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return GSC_ERR_UNSUPPORTED;
  if (!(prop.major == 10 && prop.minor == 3)) return GSC_ERR_UNSUPPORTED;  // kernels are built for sm_103a only
  if (cudaSetDevice(device) != cudaSuccess) return GSC_ERR_CUDA;
  gsc_ctx* c = (gsc_ctx*)calloc(1, sizeof(gsc_ctx));
  if (!c) return GSC_ERR_OOM;
  c->device = device;
  c->sm_count = prop.multiProcessorCount;
  c->tex[0].nblk = c->tex[1].nblk = -1;
  cudaError_t e = cudaMalloc(&c->d_status, 2 * sizeof(int));
  if (e == cudaSuccess) { c->d_diag = c->d_status + 1; e = cudaMemset(c->d_status, 0, 2 * sizeof(int)); }
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_pinned, PINNED_BYTES);
  c->h_pinned_bytes = PINNED_BYTES;
  if (init_tables) {
    if (e == cudaSuccess) e = bc1_init_tables();
    if (e == cudaSuccess) e = bc7_init_tables();
    if (e == cudaSuccess) e = decode_init_tables();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    if (c->d_status) cudaFree(c->d_status);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    free(c);
    return GSC_ERR_CUDA;
  }
  *out = c;
  return GSC_OK;
}

extern "C" gsc_status gsc_ctx_destroy(gsc_ctx* c) {
  if (!c) return GSC_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  timer_drain(c);
  free(c->recs);
  cudaDeviceSynchronize();
  tex_cache_free(c);
  if (c->d_status) cudaFree(c->d_status);
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  free(c);
  return GSC_OK;
}

extern "C" gsc_status gsc_ctx_sync(gsc_ctx* c, void* stream) {
  if (!c) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  GSC_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  int st[2] = {0, 0};
  GSC_CUDA(cudaMemcpy(st, c->d_status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st[0] != 0) {
    GSC_CUDA(cudaMemset(c->d_status, 0, sizeof(st)));
    return (gsc_status)st[0];
  }
  int where = 0;
  const int chk = gsc_check_take(&where);  // checked build: a slot entry outside [-1, n)
  if (chk != 0) return (gsc_status)chk;
  return GSC_OK;
}

// BC7 blocks per group of a fixed coding, or -1 if the request is not one
static int fixed_bc7_blocks(const gsc_encode_params* ep) {
  if (ep->format == GSC_FMT_BC1) return 0;
  if (ep->format == GSC_FMT_BC7) return 16;
  if (ep->format == GSC_FMT_MIXED) return ep->bc7_blocks;
  return -1;
}

// fixed codings that stage texels in the workspace: every coding of layouts A and B, and the mix
static bool staged_coding(const gsc_encode_params* ep) {
  return ep->layout != GSC_LAYOUT_D || ep->format == GSC_FMT_MIXED;
}

extern "C" size_t gsc_workspace_bytes(int64_t n, const gsc_encode_params* ep) {
  if (n < 0) return 0;
  size_t b = plan_ws_bytes(n);
  if (ep && ep->format == GSC_FMT_RATE) {
    size_t r = rate_ws_bytes(ceil_div64(n, 16));
    if (r > b) b = r;
  }
  if (ep && staged_coding(ep)) {
    const int j = fixed_bc7_blocks(ep);
    if (j >= 0 && j <= 16) {
      size_t r = layout_ws_bytes(ceil_div64(n, 16), j);
      if (r > b) b = r;
    }
  }
  return b;
}

static bool n_ok(int64_t n) { return n >= 0 && n < (int64_t)0x7FFFFFF0; }

extern "C" gsc_status gsc_plan_reorder(gsc_ctx* c, const float* d_pos, const float* d_sh, const gsc_plan_params* pp,
                                       int32_t* d_perm, float* d_scales, void* d_ws, size_t ws_bytes, void* stream) {
  GscRange gsc_range_("gsc_plan_reorder");
  if (!c || !pp || !n_ok(pp->n)) return GSC_ERR_INVALID_ARG;
  if (pp->group_size < 0 || pp->group_size % 16 != 0) return GSC_ERR_INVALID_ARG;
  if (pp->quantile_permille == 0 || pp->quantile_permille > 1000) return GSC_ERR_INVALID_ARG;
  if (pp->sort != 0 && pp->sort != 1) return GSC_ERR_INVALID_ARG;
  if (!d_scales || (pp->n > 0 && (!d_sh || !d_perm || (pp->sort && !d_pos)))) return GSC_ERR_INVALID_ARG;
  if (!aligned(d_sh, 16) || !aligned(d_ws, 256)) return GSC_ERR_INVALID_ARG;
  if (pp->n > 0 && !d_ws) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  GscTimed tm(c, T_PLAN, (cudaStream_t)stream);
  return plan_run(c, d_pos, d_sh, pp, d_perm, d_scales, d_ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" gsc_status gsc_quantise(gsc_ctx* c, const float* d_sh, int64_t n, const float* d_scales, uint8_t* d_q,
                                   void* stream) {
  GscRange gsc_range_("gsc_quantise");
  if (!c || !n_ok(n) || !d_scales || (n > 0 && (!d_sh || !d_q))) return GSC_ERR_INVALID_ARG;
  if (!aligned(d_sh, 16) || !aligned(d_q, 4)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  GSC_CUDA(launch_quantise(d_sh, n, d_scales, d_q, (cudaStream_t)stream));
  return GSC_OK;
}

void host_weights(const float* scales, uint32_t* w) {
  double mx = 0.0;
  for (int k = 0; k < GSC_SH; k++) { double s = scales[k]; if (s * s > mx) mx = s * s; }
  for (int k = 0; k < GSC_SH; k++) {
    double s = scales[k];
    double v = rint((s * s * 65536.0) / mx);
    w[k] = v < 1.0 ? 1u : (uint32_t)v;
  }
}

extern "C" gsc_status gsc_encode(gsc_ctx* c, const float* d_sh, int64_t n, const int32_t* d_perm,
                                 const float* d_scales, const gsc_encode_params* ep, uint8_t* d_blocks,
                                 int32_t* d_perm_out, gsc_stream_table* h_table, void* d_ws, size_t ws_bytes,
                                 void* stream) {
  GscRange gsc_range_("gsc_encode");
  if (!c || !ep || !h_table || !n_ok(n) || !d_scales) return GSC_ERR_INVALID_ARG;
  if (ep->format != GSC_FMT_BC1 && ep->format != GSC_FMT_BC7 && ep->format != GSC_FMT_RATE &&
      ep->format != GSC_FMT_MIXED)
    return GSC_ERR_INVALID_ARG;
  if (ep->layout != GSC_LAYOUT_D && ep->layout != GSC_LAYOUT_A && ep->layout != GSC_LAYOUT_B) return GSC_ERR_INVALID_ARG;
  if (staged_coding(ep) && (ep->format == GSC_FMT_RATE || !lay_ok(ep->layout, fixed_bc7_blocks(ep))))
    return GSC_ERR_INVALID_ARG;
  if (ep->format == GSC_FMT_RATE && (ep->target_bpt_x4 == 0 || ep->target_bpt_x4 > 64)) return GSC_ERR_INVALID_ARG;
  if (n > 0 && (!d_sh || !d_perm || !d_blocks || !d_perm_out)) return GSC_ERR_INVALID_ARG;
  if (!aligned(d_sh, 16) || !aligned(d_blocks, 16) || !aligned(d_ws, 256)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t ng = ceil_div64(n, 16);
  memset(h_table, 0, sizeof(*h_table));
  float* hs = reinterpret_cast<float*>(c->h_pinned);
  GSC_CUDA(cudaMemcpyAsync(hs, d_scales, sizeof(float) * GSC_SH, cudaMemcpyDeviceToHost, st));
  if (ep->format == GSC_FMT_RATE) {
    if (n > 0 && !d_ws) return GSC_ERR_INVALID_ARG;
    GSC_CUDA(cudaStreamSynchronize(st));
    float scales[GSC_SH];
    memcpy(scales, hs, sizeof(scales));
    gsc_status s = GSC_OK;
    if (n > 0) {
      if (!aligned(ep->d_bc1_blocks, 16) || !aligned(ep->d_bc7_blocks, 16)) return GSC_ERR_INVALID_ARG;
      s = rate_run(c, d_sh, n, d_perm, d_scales, ep->target_bpt_x4, d_blocks, d_perm_out, h_table, d_ws, ws_bytes,
                   ep->d_bc1_blocks, ep->d_bc7_blocks, st);
    } else {
      h_table->n_streams = GSC_MODES;
      h_table->format = GSC_FMT_RATE;
    }
    memcpy(h_table->scales, scales, sizeof(scales));
    return s;
  }
  const int j = fixed_bc7_blocks(ep);
  if (staged_coding(ep)) {
    if (n > 0 && (!d_ws || ws_bytes < layout_ws_bytes(ng, j))) return GSC_ERR_OOM;
    const gsc_status s = layout_encode_run(c, d_sh, n, d_perm, d_scales, ep->layout, j, d_blocks, d_ws, ws_bytes, st);
    if (s != GSC_OK) return s;
  } else if (ep->format == GSC_FMT_BC1) {
    GscTimed tm(c, T_BC1, st);
    GSC_CUDA(launch_bc1_groups(d_sh, d_perm, d_scales, ng, d_blocks, nullptr, nullptr, st));
  } else {
    GscTimed tm(c, T_BC7, st);
    GSC_CUDA(launch_bc7_groups(d_sh, d_perm, d_scales, ng, d_blocks, nullptr, st));
  }
  if (ng > 0 && d_perm_out != d_perm)
    GSC_CUDA(cudaMemcpyAsync(d_perm_out, d_perm, sizeof(int32_t) * ng * 16, cudaMemcpyDeviceToDevice, st));
  GSC_CUDA(cudaStreamSynchronize(st));
  h_table->n_streams = 1;
  h_table->format = ep->format;
  h_table->layout = ep->layout;
  h_table->n = n;
  h_table->n_groups = ng;
  h_table->total_bytes = ng * (16 * j + 8 * (16 - j));
  h_table->used_bits = (uint64_t)h_table->total_bytes * 8;
  memcpy(h_table->scales, hs, sizeof(float) * GSC_SH);
  host_weights(h_table->scales, h_table->weights);
  h_table->s[0].bands = 16;
  h_table->s[0].bc7_blocks = j;
  h_table->s[0].first_group = 0;
  h_table->s[0].n_groups = ng;
  h_table->s[0].byte_offset = 0;
  return GSC_OK;
}

gsc_status make_dev_table(const gsc_stream_table* t, DevTable* d) {
  if (!t || !d) return GSC_ERR_INVALID_ARG;
  if (t->n_streams < 1 || t->n_streams > GSC_MODES || !n_ok(t->n)) return GSC_ERR_INVALID_ARG;
  if (t->n_groups != ceil_div64(t->n, 16)) return GSC_ERR_INVALID_ARG;
  if (t->layout != GSC_LAYOUT_D && t->layout != GSC_LAYOUT_A && t->layout != GSC_LAYOUT_B) return GSC_ERR_INVALID_ARG;
  // layouts A and B: one stream of whole groups (all 16 coefficients) with a valid BC7 count
  if (t->layout != GSC_LAYOUT_D && (t->n_streams != 1 || t->s[0].bands != 16 || !lay_ok(t->layout, t->s[0].bc7_blocks)))
    return GSC_ERR_INVALID_ARG;
  memset(d, 0, sizeof(*d));
  d->layout = t->layout;
  d->n_streams = t->n_streams;
  d->n = (int32_t)t->n;
  d->n_groups = (int32_t)t->n_groups;
  int64_t g = 0, off = 0;
  for (int i = 0; i < t->n_streams; i++) {
    const gsc_stream& s = t->s[i];
    if (s.bands < 0 || s.bands > 16 || s.bc7_blocks < 0 || s.bc7_blocks > s.bands) return GSC_ERR_INVALID_ARG;
    if (s.first_group != g || s.n_groups < 0 || s.byte_offset != off) return GSC_ERR_INVALID_ARG;
    d->bands[i] = s.bands;
    d->bc7[i] = s.bc7_blocks;
    d->first_group[i] = s.first_group;
    d->stream_groups[i] = s.n_groups;
    d->byte_offset[i] = s.byte_offset;
    g += s.n_groups;
    off += s.n_groups * (16 * s.bc7_blocks + 8 * (s.bands - s.bc7_blocks));
  }
  if (g != t->n_groups || off != t->total_bytes) return GSC_ERR_INVALID_ARG;
  for (int k = 0; k < GSC_SH; k++) {
    if (!(t->scales[k] > 0.0f) || isinf(t->scales[k])) return GSC_ERR_INVALID_ARG;
    d->scales[k] = t->scales[k];
  }
  return GSC_OK;
}

extern "C" gsc_status gsc_forced_table(const gsc_stream_table* table, int32_t format, gsc_stream_table* out) {
  if (!table || !out || (format != GSC_FMT_BC1 && format != GSC_FMT_BC7)) return GSC_ERR_INVALID_ARG;
  DevTable T;
  const gsc_status st = make_dev_table(table, &T);
  if (st != GSC_OK) return st;
  const int64_t bpb = format == GSC_FMT_BC7 ? 16 : 8;
  gsc_stream_table t;
  memset(&t, 0, sizeof(t));
  t.n_streams = 1;
  t.format = format;
  t.n = table->n;
  t.n_groups = table->n_groups;
  t.layout = table->layout;
  t.total_bytes = table->n_groups * 16 * bpb;
  t.budget_bits = 0;
  t.used_bits = (uint64_t)t.total_bytes * 8u;
  t.lambda = 0;
  for (int k = 0; k < GSC_SH; k++) { t.scales[k] = table->scales[k]; t.weights[k] = table->weights[k]; }
  t.s[0].bands = 16;
  t.s[0].bc7_blocks = format == GSC_FMT_BC7 ? 16 : 0;
  t.s[0].first_group = 0;
  t.s[0].n_groups = table->n_groups;
  t.s[0].byte_offset = 0;
  *out = t;
  return GSC_OK;
}

extern "C" gsc_status gsc_decode(gsc_ctx* c, const gsc_stream_table* table, const uint8_t* d_blocks,
                                 const int32_t* d_perm, uint8_t* d_texels, void* stream) {
  GscRange gsc_range_("gsc_decode");
  if (!c) return GSC_ERR_INVALID_ARG;
  DevTable T;
  gsc_status s = make_dev_table(table, &T);
  if (s != GSC_OK) return s;
  if (T.n_groups > 0 && (!d_blocks || !d_perm || !d_texels)) return GSC_ERR_INVALID_ARG;
  if (!aligned(d_blocks, 8) || !aligned(d_texels, 16)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  GscTimed tm(c, T_DECODE, (cudaStream_t)stream);
  GSC_CUDA(launch_decode(T, d_blocks, d_perm, d_texels, (cudaStream_t)stream));
  return GSC_OK;
}

extern "C" gsc_status gsc_decode_eval_sh(gsc_ctx* c, const gsc_stream_table* table, const uint8_t* d_blocks,
                                         const int32_t* d_perm, const float* d_dirs, const float* d_pos,
                                         const float* d_cams, int32_t V, int32_t out_order, float* d_rgb,
                                         void* stream) {
  GscRange gsc_range_("gsc_decode_eval_sh");
  if (!c) return GSC_ERR_INVALID_ARG;
  DevTable T;
  gsc_status s = make_dev_table(table, &T);
  if (s != GSC_OK) return s;
  if (V < 1 || V > 64 || out_order < 0 || out_order > 3) return GSC_ERR_INVALID_ARG;
  if ((d_dirs == nullptr) == (d_cams == nullptr)) return GSC_ERR_INVALID_ARG;
  if (d_cams && !d_pos && T.n > 0) return GSC_ERR_INVALID_ARG;
  if (T.n_groups > 0 && (!d_blocks || !d_perm || !d_rgb)) return GSC_ERR_INVALID_ARG;
  if (!aligned(d_blocks, 8) || !aligned(d_rgb, 16)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  GscTimed tm(c, T_EVAL, (cudaStream_t)stream);
  GSC_CUDA(launch_decode_eval(T, d_blocks, d_perm, d_dirs, d_pos, d_cams, V, out_order, d_rgb, c->sm_count,
                              (cudaStream_t)stream));
  return GSC_OK;
}

extern "C" gsc_status gsc_decode_eval_sh_slots(gsc_ctx* c, const gsc_stream_table* table, const uint8_t* d_blocks,
                                               const int32_t* d_perm, const float* d_dirs, const float* d_pos_slot,
                                               const float* d_cams, int32_t V, int32_t out_order, float* d_rgb,
                                               void* stream) {
  GscRange gsc_range_("gsc_decode_eval_sh_slots");
  if (!c) return GSC_ERR_INVALID_ARG;
  DevTable T;
  gsc_status s = make_dev_table(table, &T);
  if (s != GSC_OK) return s;
  if (V < 1 || V > 64 || out_order < 0 || out_order > 3) return GSC_ERR_INVALID_ARG;
  if ((d_dirs == nullptr) == (d_cams == nullptr)) return GSC_ERR_INVALID_ARG;
  if (d_cams && !d_pos_slot && T.n > 0) return GSC_ERR_INVALID_ARG;
  if (T.n_groups > 0 && (!d_blocks || !d_perm || !d_rgb)) return GSC_ERR_INVALID_ARG;
  if (!aligned(d_blocks, 8) || !aligned(d_rgb, 16) || !aligned(d_pos_slot, 4)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  GscTimed tm(c, T_EVAL, (cudaStream_t)stream);
  GSC_CUDA(launch_decode_eval(T, d_blocks, d_perm, d_dirs, nullptr, d_cams, V, out_order, d_rgb, c->sm_count,
                              (cudaStream_t)stream, nullptr, 0, d_cams ? d_pos_slot : nullptr));
  return GSC_OK;
}

extern "C" gsc_status gsc_positions_to_slots(gsc_ctx* c, const float* d_pos, int64_t n, const int32_t* d_perm,
                                             int64_t n_slots, float* d_pos_slot, void* stream) {
  GscRange gsc_range_("gsc_positions_to_slots");
  if (!c || !n_ok(n) || n_slots != ceil_div64(n, 16) * 16) return GSC_ERR_INVALID_ARG;
  if (n_slots > 0 && (!d_pos || !d_perm || !d_pos_slot)) return GSC_ERR_INVALID_ARG;
  if (!aligned(d_pos, 4) || !aligned(d_pos_slot, 4) || !aligned(d_perm, 4)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  GSC_CUDA(launch_pos_to_slots(d_pos, d_perm, n, n_slots, d_pos_slot, c->sm_count, (cudaStream_t)stream));
  return GSC_OK;
}

extern "C" gsc_status gsc_decode_tex(gsc_ctx* c, const gsc_stream_table* table, const uint8_t* d_blocks,
                                     const int32_t* d_perm, uint8_t* d_texels, void* stream) {
  GscRange gsc_range_("gsc_decode_tex");
  if (!c) return GSC_ERR_INVALID_ARG;
  DevTable T;
  gsc_status s = make_dev_table(table, &T);
  if (s != GSC_OK) return s;
  if (T.n_groups > 0 && (!d_blocks || !d_perm || !d_texels)) return GSC_ERR_INVALID_ARG;
  if (!aligned(d_blocks, 8)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  GscTimed tm(c, T_TEX, (cudaStream_t)stream);
  return decode_tex_run(c, T, d_blocks, d_perm, d_texels, (cudaStream_t)stream);
}

static bool fmt_ok(int f) { return f == GSC_FMT_BC1 || f == GSC_FMT_BC7; }

extern "C" gsc_status gsc_encode_blocks(gsc_ctx* c, const uint8_t* d_tex, int64_t nblk, int32_t format,
                                        uint8_t* d_out, uint64_t* d_sse, void* stream) {
  GscRange gsc_range_("gsc_encode_blocks");
  if (!c || nblk < 0 || !fmt_ok(format) || (nblk > 0 && (!d_tex || !d_out))) return GSC_ERR_INVALID_ARG;
  if (!aligned(d_out, format == GSC_FMT_BC7 ? 16 : 8) || !aligned(d_sse, 8)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  if (format == GSC_FMT_BC1) GSC_CUDA(launch_bc1_blocks(d_tex, nblk, d_out, d_sse, (cudaStream_t)stream));
  else GSC_CUDA(launch_bc7_blocks(d_tex, nblk, d_out, d_sse, (cudaStream_t)stream));
  return GSC_OK;
}

extern "C" gsc_status gsc_decode_blocks(gsc_ctx* c, const uint8_t* d_blocks, int64_t nblk, int32_t format,
                                        uint8_t* d_rgba, void* stream) {
  GscRange gsc_range_("gsc_decode_blocks");
  if (!c || nblk < 0 || !fmt_ok(format) || (nblk > 0 && (!d_blocks || !d_rgba))) return GSC_ERR_INVALID_ARG;
  if (!aligned(d_blocks, format == GSC_FMT_BC7 ? 16 : 8) || !aligned(d_rgba, 4)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  GSC_CUDA(launch_decode_blocks(d_blocks, nblk, format, d_rgba, (cudaStream_t)stream));
  return GSC_OK;
}

extern "C" gsc_status gsc_decode_blocks_tex(gsc_ctx* c, const uint8_t* d_blocks, int64_t nblk, int32_t format,
                                            uint8_t* d_rgba, void* stream) {
  GscRange gsc_range_("gsc_decode_blocks_tex");
  if (!c || nblk < 0 || !fmt_ok(format) || (nblk > 0 && (!d_blocks || !d_rgba))) return GSC_ERR_INVALID_ARG;
  if (!aligned(d_blocks, 8) || !aligned(d_rgba, 4)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  return decode_blocks_tex_run(c, d_blocks, nblk, format, d_rgba, (cudaStream_t)stream);
}
