// plan.cu -- per-scene scales, quantisation and the reorder plan (Sec. V-A; Sec. III-C,
// Fig. Bit4Scan), plus the device-wide radix sort and scan the plan and the rate
// control share. No host synchronisation: everything is queued on the caller's stream.
#include <mutex>

#include "gsc_internal.cuh"

// ---- scan (exclusive, 64-bit) -------------------------------------------------------------
#define SCAN_BLOCK 1024
static int64_t scan_blocks(int64_t n) { return ceil_div64(n > 0 ? n : 1, SCAN_BLOCK); }
size_t scan_ws_bytes(int64_t n) {
  int64_t nb = scan_blocks(n);
  return align_up(sizeof(uint64_t) * (size_t)nb, 256) + align_up(sizeof(uint64_t) * (size_t)scan_blocks(nb), 256) + 256;
}

template <class T>
__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t* s_warp, uint64_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    uint64_t y = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      uint64_t z = __shfl_up_sync(0xFFFFFFFFu, y, d);
      if (lane >= d) y += z;
    }
    s_warp[lane] = y;  // inclusive over warps
  }
  __syncthreads();
  uint64_t before = (w > 0 ? s_warp[w - 1] : 0) + x - v;
  if (total) *total = s_warp[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

template <class T>
__global__ void k_scan_reduce(const T* __restrict__ in, int64_t n, uint64_t* __restrict__ sums) {
  __shared__ uint64_t s_warp[32];
  const int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
  uint64_t v = i < n ? (uint64_t)in[i] : 0;
  uint64_t tot;
  block_excl_scan<T>(v, s_warp, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <class T>
__global__ void k_scan_apply(const T* __restrict__ in, int64_t n, const uint64_t* __restrict__ offs,
                             T* __restrict__ out, uint64_t* __restrict__ total) {
  __shared__ uint64_t s_warp[32];
  const int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
  uint64_t v = i < n ? (uint64_t)in[i] : 0;
  uint64_t tot;
  uint64_t ex = block_excl_scan<T>(v, s_warp, &tot) + (offs ? offs[blockIdx.x] : 0);
  if (i < n) out[i] = (T)ex;
  if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = (offs ? offs[blockIdx.x] : 0) + tot;
}

// single-block scan of up to SCAN_BLOCK * k elements held in one array (sequential chunks)
__global__ void k_scan_single(uint64_t* __restrict__ a, int64_t n) {
  __shared__ uint64_t s_warp[32];
  __shared__ uint64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n; base += SCAN_BLOCK) {
    const int64_t i = base + threadIdx.x;
    uint64_t v = i < n ? a[i] : 0;
    uint64_t tot;
    uint64_t ex = block_excl_scan<uint64_t>(v, s_warp, &tot);
    if (i < n) a[i] = ex + carry;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
}

// Exclusive scan of n values of T (uint32 or uint64) into out (may alias in); total (device, optional).
template <class T>
cudaError_t scan_exclusive(const T* in, T* out, int64_t n, uint64_t* total, void* ws, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t nb = scan_blocks(n);
  uint64_t* sums = reinterpret_cast<uint64_t*>(ws);
  gsc_count_launch(); k_scan_reduce<T><<<(int)nb, SCAN_BLOCK, 0, st>>>(in, n, sums);
  gsc_count_launch(); k_scan_single<<<1, SCAN_BLOCK, 0, st>>>(sums, nb);
  gsc_count_launch(); k_scan_apply<T><<<(int)nb, SCAN_BLOCK, 0, st>>>(in, n, sums, out, total);
  return cudaGetLastError();
}
template cudaError_t scan_exclusive<uint32_t>(const uint32_t*, uint32_t*, int64_t, uint64_t*, void*, cudaStream_t);
template cudaError_t scan_exclusive<uint64_t>(const uint64_t*, uint64_t*, int64_t, uint64_t*, void*, cudaStream_t);

// ---- stable LSD radix sort of (u64 key, u32 value) pairs, 8-bit digits ---------------------
#define RS_THREADS 256
#define RS_ITEMS 8
#define RS_TILE (RS_THREADS * RS_ITEMS)

static int64_t rs_tiles(int64_t n) { return ceil_div64(n > 0 ? n : 1, RS_TILE); }

size_t radix_ws_bytes(int64_t n) {
  int64_t nt = rs_tiles(n);
  size_t b = 0;
  b += align_up(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1), 256);   // keys ping-pong
  b += align_up(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1), 256);   // values ping-pong
  b += align_up(sizeof(uint32_t) * 256 * (size_t)nt, 256);          // digit x tile counts
  b += scan_ws_bytes(256 * nt);
  return b + 1024;
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                                                       uint32_t* __restrict__ hist, int64_t n_tiles) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll
  for (int r = 0; r < RS_ITEMS; r++) {
    int64_t i = base + r * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint64_t* __restrict__ kin,
                                                          const uint32_t* __restrict__ vin, int64_t n, int shift,
                                                          const uint32_t* __restrict__ offs, int64_t n_tiles,
                                                          uint64_t* __restrict__ kout, uint32_t* __restrict__ vout) {
  __shared__ uint32_t run[256];
  __shared__ uint16_t wcnt[RS_THREADS / 32][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  run[threadIdx.x] = 0;
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  const uint32_t lt = (1u << lane) - 1u;
  for (int r = 0; r < RS_ITEMS; r++) {
    const int64_t i = base + r * RS_THREADS + threadIdx.x;
    const bool live = i < n;
    uint64_t k = live ? kin[i] : 0;
    uint32_t v = live ? vin[i] : 0;
    const uint32_t d = live ? (uint32_t)((k >> shift) & 255) : 256u;
#pragma unroll
    for (int q = 0; q < 8; q++) wcnt[w][lane * 8 + q] = 0;
    __syncwarp();
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
    const int leader = __ffs(peers) - 1;
    if (live && lane == leader) wcnt[w][d] = (uint16_t)__popc(peers);
    __syncthreads();
    if (live) {
      uint32_t pos = run[d] + __popc(peers & lt);
      for (int ww = 0; ww < w; ww++) pos += wcnt[ww][d];
      const uint32_t dst = offs[(int64_t)d * n_tiles + blockIdx.x] + pos;
      kout[dst] = k;
      vout[dst] = v;
    }
    __syncthreads();
    uint32_t add = 0;
#pragma unroll
    for (int ww = 0; ww < RS_THREADS / 32; ww++) add += wcnt[ww][threadIdx.x];
    run[threadIdx.x] += add;
    __syncthreads();
  }
}

cudaError_t radix_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t n, int key_bits, void* ws, cudaStream_t st) {
  if (n <= 1 || key_bits <= 0) return cudaSuccess;
  const int64_t nt = rs_tiles(n);
  Carve c{reinterpret_cast<uint8_t*>(ws), 0, 0};
  uint64_t* k2 = c.take<uint64_t>(n);
  uint32_t* v2 = c.take<uint32_t>(n);
  uint32_t* hist = c.take<uint32_t>(256 * nt);
  void* sws = c.take<uint8_t>((int64_t)scan_ws_bytes(256 * nt));
  uint64_t* ka = keys;
  uint32_t* va = vals;
  uint64_t* kb = k2;
  uint32_t* vb = v2;
  int passes = (key_bits + 7) / 8;
  for (int p = 0; p < passes; p++) {
    gsc_count_launch(); k_rs_hist<<<(int)nt, RS_THREADS, 0, st>>>(ka, n, 8 * p, hist, nt);
    cudaError_t e = scan_exclusive<uint32_t>(hist, hist, 256 * nt, nullptr, sws, st);
    if (e != cudaSuccess) return e;
    gsc_count_launch(); k_rs_scatter<<<(int)nt, RS_THREADS, 0, st>>>(ka, va, n, 8 * p, hist, nt, kb, vb);
    uint64_t* tk = ka; ka = kb; kb = tk;
    uint32_t* tv = va; va = vb; vb = tv;
  }
  if (ka != keys) {
    cudaError_t e = cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

// ---- scales: exact order statistic by 4 passes of 8-bit radix select -----------------------
struct SelState { uint32_t prefix[GSC_SH]; uint64_t rank[GSC_SH]; };

__global__ void k_sel_init(SelState* s, uint64_t r) {
  if (threadIdx.x < GSC_SH) { s->prefix[threadIdx.x] = 0; s->rank[threadIdx.x] = r; }
}

__global__ void __launch_bounds__(256) k_sel_hist(const float4* __restrict__ sh4, int64_t n4, int shift,
                                                  const uint32_t* __restrict__ prefix, uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[GSC_SH * 256];
  __shared__ uint32_t pre[GSC_SH];
  for (int i = threadIdx.x; i < GSC_SH * 256; i += blockDim.x) h[i] = 0;
  if (threadIdx.x < GSC_SH) pre[threadIdx.x] = prefix[threadIdx.x];
  __syncthreads();
  const int hs = shift + 8;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    float4 f = __ldg(sh4 + i);
    const int j0 = (int)((i * 4) % 48);
    float a[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int k = (j0 + q) / 3;
      const uint32_t u = __float_as_uint(a[q]) & 0x7FFFFFFFu;
      if (hs >= 32 || (u >> hs) == (pre[k] >> hs)) atomicAdd(&h[k * 256 + ((u >> shift) & 255)], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < GSC_SH * 256; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

// The digit of this pass: the first whose cumulative count passes the remaining rank. ZERO clears
// the histogram for the next pass (the whole-scene plan reuses one buffer).
template <class T, bool ZERO>
__global__ void k_sel_pick(SelState* st, T* hist, int shift) {
  const int k = threadIdx.x;
  if (k >= GSC_SH) return;
  uint64_t r = st->rank[k], cum = 0;
  int d = 0;
  for (d = 0; d < 256; d++) {
    uint64_t c = (uint64_t)hist[k * 256 + d];
    if (r < cum + c) break;
    cum += c;
  }
  if (d > 255) d = 255;
  st->prefix[k] |= (uint32_t)d << shift;
  st->rank[k] = r - cum;
  if constexpr (ZERO)
    for (int i = 0; i < 256; i++) hist[k * 256 + i] = 0;
}

__global__ void k_sel_finish(const SelState* st, float* scales) {
  const int k = threadIdx.x;
  if (k >= GSC_SH) return;
  float s = 2.0f * __uint_as_float(st->prefix[k]);
  scales[k] = (s == 0.0f) ? 1.0f : s;
}

__global__ void k_fill_scales_one(float* scales) {
  if (threadIdx.x < GSC_SH) scales[threadIdx.x] = 1.0f;
}

// ---- quantisation kernel (Sec. V-A) ----------------------------------------------------------
__global__ void k_quantise(const float4* __restrict__ sh4, int64_t n4, const float* __restrict__ scales,
                           uchar4* __restrict__ q4) {
  __shared__ float s_scale[GSC_SH];
  if (threadIdx.x < GSC_SH) s_scale[threadIdx.x] = scales[threadIdx.x];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    float4 f = __ldg(sh4 + i);
    const int j0 = (int)((i * 4) % 48);
    uchar4 o;
    o.x = (uint8_t)gsc_quant1(f.x, s_scale[(j0 + 0) / 3]);
    o.y = (uint8_t)gsc_quant1(f.y, s_scale[(j0 + 1) / 3]);
    o.z = (uint8_t)gsc_quant1(f.z, s_scale[(j0 + 2) / 3]);
    o.w = (uint8_t)gsc_quant1(f.w, s_scale[(j0 + 3) / 3]);
    q4[i] = o;
  }
}

static int grid_stride(int64_t n, int threads, int cap = gsc_sm_count() * 8) {
  int64_t g = ceil_div64(n > 0 ? n : 1, threads);
  return (int)(g > cap ? cap : g);
}

cudaError_t launch_quantise(const float* sh, int64_t n, const float* scales, uint8_t* q, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t n4 = n * 12;
  gsc_count_launch(); k_quantise<<<grid_stride(n4, 256), 256, 0, st>>>(reinterpret_cast<const float4*>(sh), n4, scales,
                                                    reinterpret_cast<uchar4*>(q));
  return cudaGetLastError();
}

// ---- bounding box, Morton keys, colour keys --------------------------------------------------
__device__ __forceinline__ uint32_t f2ord(float f) {
  uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o);
}

__global__ void k_bbox_init(uint32_t* bb) {
  if (threadIdx.x < 3) { bb[threadIdx.x] = 0xFFFFFFFFu; bb[3 + threadIdx.x] = 0u; }
}

__global__ void k_bbox(const float* __restrict__ pos, int64_t n, uint32_t* __restrict__ bb) {
  uint32_t lo[3] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu}, hi[3] = {0, 0, 0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
      uint32_t o = f2ord(__ldg(pos + 3 * i + a));
      lo[a] = min(lo[a], o);
      hi[a] = max(hi[a], o);
    }
  }
#pragma unroll
  for (int a = 0; a < 3; a++) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      lo[a] = min(lo[a], __shfl_xor_sync(0xFFFFFFFFu, lo[a], d));
      hi[a] = max(hi[a], __shfl_xor_sync(0xFFFFFFFFu, hi[a], d));
    }
  }
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int a = 0; a < 3; a++) { atomicMin(&bb[a], lo[a]); atomicMax(&bb[3 + a], hi[a]); }
}

__device__ __forceinline__ uint32_t spread3(uint32_t x) {  // 10 bits -> every third bit
  x &= 0x3FFu;
  x = (x | (x << 16)) & 0x030000FFu;
  x = (x | (x << 8)) & 0x0300F00Fu;
  x = (x | (x << 4)) & 0x030C30C3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

__device__ __forceinline__ uint32_t grid10(float p, float lo, float ext) {
  if (ext == 0.0f) return 0;
  float t = __fmul_rn(__fdiv_rn(__fsub_rn(p, lo), ext), 1024.0f);
  uint32_t u = (uint32_t)floorf(t);
  return u > 1023u ? 1023u : u;
}

__global__ void k_morton(const float* __restrict__ pos, int64_t n, const uint32_t* __restrict__ bb,
                         uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  float lo[3], ext[3];
#pragma unroll
  for (int a = 0; a < 3; a++) { lo[a] = ord2f(bb[a]); ext[a] = __fsub_rn(ord2f(bb[3 + a]), lo[a]); }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t x = grid10(__ldg(pos + 3 * i + 0), lo[0], ext[0]);
    uint32_t y = grid10(__ldg(pos + 3 * i + 1), lo[1], ext[1]);
    uint32_t z = grid10(__ldg(pos + 3 * i + 2), lo[2], ext[2]);
    keys[i] = (spread3(x) << 2) | (spread3(y) << 1) | spread3(z);
    vals[i] = (uint32_t)i;
  }
}

__device__ __forceinline__ uint32_t spread8(uint32_t x) {  // 8 bits -> every third bit (24-bit result)
  x &= 0xFFu;
  x = (x | (x << 8)) & 0x00F00Fu;
  x = (x | (x << 4)) & 0x0C30C3u;
  x = (x | (x << 2)) & 0x249249u;
  return x;
}

__global__ void k_colour_keys(const float* __restrict__ sh, const float* __restrict__ scales, int64_t n,
                              int64_t group_size, uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals) {
  const float s0 = scales[0];
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = vals[r];
    const float* dc = sh + (int64_t)i * 48;
    uint32_t q0 = gsc_quant1(__ldg(dc + 0), s0), q1 = gsc_quant1(__ldg(dc + 1), s0), q2 = gsc_quant1(__ldg(dc + 2), s0);
    uint64_t chunk = group_size ? (uint64_t)(r / group_size) : 0;
    keys[r] = (chunk << 24) | (spread8(q0) << 2) | (spread8(q1) << 1) | spread8(q2);
  }
}

__global__ void k_finish_perm(const uint32_t* __restrict__ vals, int64_t n, int64_t ns, int identity,
                              int32_t* __restrict__ perm) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x)
    perm[s] = s < n ? (identity ? (int32_t)s : (int32_t)vals[s]) : -1;
}

size_t plan_ws_bytes(int64_t n) {
  size_t b = 0;
  b += align_up(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1), 256);
  b += align_up(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1), 256);
  b += align_up(sizeof(uint32_t) * GSC_SH * 256, 256);
  b += align_up(sizeof(SelState), 256);
  b += align_up(sizeof(uint32_t) * 8, 256);
  b += radix_ws_bytes(n);
  return b + 4096;
}

static int bits_for(uint64_t v) { int b = 0; while (v) { b++; v >>= 1; } return b; }

gsc_status plan_run(gsc_ctx* ctx, const float* pos, const float* sh, const gsc_plan_params* pp, int32_t* perm,
                    float* scales, void* ws, size_t ws_bytes, cudaStream_t st) {
  const int64_t n = pp->n, ns = ceil_div64(n, 16) * 16;
  if (ws_bytes < plan_ws_bytes(n)) return GSC_ERR_OOM;
  Carve c{reinterpret_cast<uint8_t*>(ws), 0, ws_bytes};
  uint64_t* keys = c.take<uint64_t>(n);
  uint32_t* vals = c.take<uint32_t>(n);
  uint32_t* hist = c.take<uint32_t>(GSC_SH * 256);
  SelState* sel = c.take<SelState>(1);
  uint32_t* bb = c.take<uint32_t>(8);
  void* rws = c.take<uint8_t>((int64_t)radix_ws_bytes(n));
  // scales
  if (n == 0) {
    gsc_count_launch(); k_fill_scales_one<<<1, 32, 0, st>>>(scales);
  } else {
    const uint64_t m = 3ull * (uint64_t)n;
    const uint64_t r = ((uint64_t)pp->quantile_permille * m + 999) / 1000 - 1;
    GSC_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * GSC_SH * 256, st));
    gsc_count_launch(); k_sel_init<<<1, 32, 0, st>>>(sel, r);
    const int64_t n4 = n * 12;
    const int g = grid_stride(n4, 256, ctx->sm_count * 4);
    for (int shift = 24; shift >= 0; shift -= 8) {
      gsc_count_launch(); k_sel_hist<<<g, 256, 0, st>>>(reinterpret_cast<const float4*>(sh), n4, shift, sel->prefix, hist);
      gsc_count_launch(); k_sel_pick<uint32_t, true><<<1, 32, 0, st>>>(sel, hist, shift);
    }
    gsc_count_launch(); k_sel_finish<<<1, 32, 0, st>>>(sel, scales);
  }
  GSC_CUDA(cudaGetLastError());
  if (ns == 0) return GSC_OK;
  if (!pp->sort || n == 0) {
    gsc_count_launch(); k_finish_perm<<<grid_stride(ns, 256), 256, 0, st>>>(vals, n, ns, 1, perm);
    GSC_CUDA(cudaGetLastError());
    return GSC_OK;
  }
  // spatial rank: stable sort by 30-bit Morton code of the bounding-box grid
  gsc_count_launch(); k_bbox_init<<<1, 32, 0, st>>>(bb);
  gsc_count_launch(); k_bbox<<<grid_stride(n, 256, ctx->sm_count * 2), 256, 0, st>>>(pos, n, bb);
  gsc_count_launch(); k_morton<<<grid_stride(n, 256), 256, 0, st>>>(pos, n, bb, keys, vals);
  GSC_CUDA(cudaGetLastError());
  GSC_CUDA(radix_sort_pairs(keys, vals, n, 30, rws, st));
  // slot order: stable sort by (chunk, colour key) of the rank-ordered Gaussians
  gsc_count_launch(); k_colour_keys<<<grid_stride(n, 256), 256, 0, st>>>(sh, scales, n, pp->group_size, keys, vals);
  GSC_CUDA(cudaGetLastError());
  const uint64_t max_chunk = pp->group_size ? (uint64_t)((n - 1) / pp->group_size) : 0;
  GSC_CUDA(radix_sort_pairs(keys, vals, n, 24 + bits_for(max_chunk), rws, st));
  gsc_count_launch(); k_finish_perm<<<grid_stride(ns, 256), 256, 0, st>>>(vals, n, ns, 0, perm);
  GSC_CUDA(cudaGetLastError());
  return GSC_OK;
}

// ---- allocation-free variant of gsc_plan_reorder ------------------------------------------
// Scratch lives in this file-scope device array instead of a caller workspace. Every GPU
// that loads the library holds it (2 MiB) until the process exits. Its device address is
// looked up once per device, with that device current, on the first call there, and kept for
// the life of the process: a cudaDeviceReset of that device invalidates it (the module is loaded
// again, possibly elsewhere), so this entry point must not be used after such a reset.
#define GSC_PLAN_STATIC_BYTES (2u << 20)
#define GSC_MAX_DEVICES 64
static __device__ __align__(256) uint8_t g_plan_scratch[GSC_PLAN_STATIC_BYTES];
static std::mutex g_plan_scratch_mu;
static void* g_plan_scratch_ptr[GSC_MAX_DEVICES];

extern "C" gsc_status gsc_plan_reorder_static(gsc_ctx* c, const float* d_pos, const float* d_sh,
                                              const gsc_plan_params* pp, int32_t* d_perm, float* d_scales,
                                              void* stream) {
  GscRange gsc_range_("gsc_plan_reorder_static");
  if (!c || !pp || pp->n < 0 || pp->n > GSC_PLAN_STATIC_MAX_N) return GSC_ERR_INVALID_ARG;
  if (pp->group_size < 0 || pp->group_size % 16 != 0) return GSC_ERR_INVALID_ARG;
  if (pp->quantile_permille == 0 || pp->quantile_permille > 1000) return GSC_ERR_INVALID_ARG;
  if (pp->sort != 0 && pp->sort != 1) return GSC_ERR_INVALID_ARG;
  if (!d_scales || (pp->n > 0 && (!d_sh || !d_perm || (pp->sort && !d_pos)))) return GSC_ERR_INVALID_ARG;
  if (((uintptr_t)d_sh % 16) != 0) return GSC_ERR_INVALID_ARG;
  if (c->device < 0 || c->device >= GSC_MAX_DEVICES) return GSC_ERR_UNSUPPORTED;
  if (plan_ws_bytes(pp->n) > GSC_PLAN_STATIC_BYTES) return GSC_ERR_OOM;
  GSC_CUDA(cudaSetDevice(c->device));
  void* ws = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_plan_scratch_mu);
    if (!g_plan_scratch_ptr[c->device]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_plan_scratch) != cudaSuccess || !p) return GSC_ERR_CUDA;
      g_plan_scratch_ptr[c->device] = p;
    }
    ws = g_plan_scratch_ptr[c->device];
  }
  GscTimed tm(c, T_PLAN, (cudaStream_t)stream);
  return plan_run(c, d_pos, d_sh, pp, d_perm, d_scales, ws, GSC_PLAN_STATIC_BYTES, (cudaStream_t)stream);
}

// ---- one scene split over shards (Sec. V-A: the scales are order statistics of the whole
// scene; Sec. III-C: the reorder works chunk by chunk once the spatial order is known) --------
// Shards hold contiguous ranges of the input. The exchanges are integer: the bounding box
// (elementwise minimum / maximum of order-preserving float codes), the Morton codes of every
// Gaussian (to fix the spatial ranks), and the selection histograms of each pass (sums). Every
// partial and every merged value is int64, so any reduction library can combine them.

__global__ void k_bbox_widen(int64_t* bb) {  // u32 codes [6] at the front of bb -> int64 [6]
  if (threadIdx.x != 0) return;
  const uint32_t* u = reinterpret_cast<const uint32_t*>(bb);
  uint32_t v[6];
  for (int a = 0; a < 6; a++) v[a] = u[a];
  for (int a = 0; a < 6; a++) bb[a] = (int64_t)v[a];
}

__global__ void k_morton_shard(const float* __restrict__ pos, int64_t n, const int64_t* __restrict__ bb,
                               uint64_t* __restrict__ keys) {
  float lo[3], ext[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    lo[a] = ord2f((uint32_t)bb[a]);
    ext[a] = __fsub_rn(ord2f((uint32_t)bb[3 + a]), lo[a]);
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t x = grid10(__ldg(pos + 3 * i + 0), lo[0], ext[0]);
    uint32_t y = grid10(__ldg(pos + 3 * i + 1), lo[1], ext[1]);
    uint32_t z = grid10(__ldg(pos + 3 * i + 2), lo[2], ext[2]);
    keys[i] = (spread3(x) << 2) | (spread3(y) << 1) | spread3(z);
  }
}

__global__ void k_iota(uint32_t* __restrict__ v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (uint32_t)i;
}

__global__ void k_widen_u32(const uint32_t* __restrict__ in, int64_t* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int64_t)in[i];
}

cudaError_t shard_bbox(const float* pos, int64_t n, int64_t* bb, int sm_count, cudaStream_t st) {
  uint32_t* u = reinterpret_cast<uint32_t*>(bb);
  gsc_count_launch(); k_bbox_init<<<1, 32, 0, st>>>(u);
  if (n > 0) { gsc_count_launch(); k_bbox<<<grid_stride(n, 256, sm_count * 2), 256, 0, st>>>(pos, n, u); }
  gsc_count_launch(); k_bbox_widen<<<1, 32, 0, st>>>(bb);
  return cudaGetLastError();
}

cudaError_t shard_morton(const float* pos, int64_t n, const int64_t* bb, uint64_t* keys, int sm_count, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  gsc_count_launch(); k_morton_shard<<<grid_stride(n, 256, sm_count * 8), 256, 0, st>>>(pos, n, bb, keys);
  return cudaGetLastError();
}

size_t shard_order_ws_bytes(int64_t n) { return radix_ws_bytes(n) + 256; }

cudaError_t shard_order(uint64_t* keys, int64_t n, int32_t* order, void* ws, int sm_count, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  uint32_t* vals = reinterpret_cast<uint32_t*>(order);
  gsc_count_launch(); k_iota<<<grid_stride(n, 256, sm_count * 8), 256, 0, st>>>(vals, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return radix_sort_pairs(keys, vals, n, 30, ws, st);  // stable: equal codes keep the input order
}

size_t shard_select_state_bytes() { return align_up(sizeof(SelState), 256) + sizeof(uint32_t) * GSC_SH * 256; }

cudaError_t shard_select_begin(int64_t n_total, int permille, void* state, cudaStream_t st) {
  SelState* sel = reinterpret_cast<SelState*>(state);
  const uint64_t m = 3ull * (uint64_t)n_total;
  const uint64_t r = n_total > 0 ? ((uint64_t)permille * m + 999) / 1000 - 1 : 0;
  gsc_count_launch(); k_sel_init<<<1, 32, 0, st>>>(sel, r);
  return cudaGetLastError();
}

cudaError_t shard_select_hist(const float* sh, int64_t n, int shift, void* state, int64_t* hist, int sm_count,
                              cudaStream_t st) {
  SelState* sel = reinterpret_cast<SelState*>(state);
  uint32_t* h32 = reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(state) + align_up(sizeof(SelState), 256));
  cudaError_t e = cudaMemsetAsync(h32, 0, sizeof(uint32_t) * GSC_SH * 256, st);
  if (e != cudaSuccess) return e;
  if (n > 0) {
    const int64_t n4 = n * 12;
    gsc_count_launch();
    k_sel_hist<<<grid_stride(n4, 256, sm_count * 4), 256, 0, st>>>(reinterpret_cast<const float4*>(sh), n4, shift,
                                                                    sel->prefix, h32);
  }
  gsc_count_launch(); k_widen_u32<<<16, 256, 0, st>>>(h32, hist, GSC_SH * 256);
  return cudaGetLastError();
}

cudaError_t shard_select_pick(void* state, const int64_t* hist_total, int shift, cudaStream_t st) {
  gsc_count_launch();
  k_sel_pick<const int64_t, false><<<1, 32, 0, st>>>(reinterpret_cast<SelState*>(state), hist_total, shift);
  return cudaGetLastError();
}

cudaError_t shard_select_scales(const void* state, float* scales, cudaStream_t st) {
  gsc_count_launch(); k_sel_finish<<<1, 32, 0, st>>>(reinterpret_cast<const SelState*>(state), scales);
  return cudaGetLastError();
}

size_t shard_plan_ws_bytes(int64_t n) {
  return align_up(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1), 256) +
         align_up(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1), 256) + radix_ws_bytes(n) + 1024;
}

// Slot order of a shard whose Gaussians are given in spatial-rank order and whose first one
// starts a chunk: the stable (chunk, colour key) sort of the whole-scene plan, on this range.
gsc_status shard_plan(const float* sh, int64_t n, const float* scales, int64_t group_size, int32_t* perm, void* ws,
                      size_t ws_bytes, int sm_count, cudaStream_t st) {
  const int64_t ns = ceil_div64(n, 16) * 16;
  if (ws_bytes < shard_plan_ws_bytes(n)) return GSC_ERR_OOM;
  if (ns == 0) return GSC_OK;
  Carve c{reinterpret_cast<uint8_t*>(ws), 0, ws_bytes};
  uint64_t* keys = c.take<uint64_t>(n);
  uint32_t* vals = c.take<uint32_t>(n);
  void* rws = c.take<uint8_t>((int64_t)radix_ws_bytes(n));
  gsc_count_launch(); k_iota<<<grid_stride(n, 256, sm_count * 8), 256, 0, st>>>(vals, n);
  gsc_count_launch(); k_colour_keys<<<grid_stride(n, 256, sm_count * 8), 256, 0, st>>>(sh, scales, n, group_size, keys, vals);
  GSC_CUDA(cudaGetLastError());
  const uint64_t max_chunk = (uint64_t)((n - 1) / group_size);
  GSC_CUDA(radix_sort_pairs(keys, vals, n, 24 + bits_for(max_chunk), rws, st));
  gsc_count_launch(); k_finish_perm<<<grid_stride(ns, 256, sm_count * 8), 256, 0, st>>>(vals, n, ns, 0, perm);
  GSC_CUDA(cudaGetLastError());
  return GSC_OK;
}
