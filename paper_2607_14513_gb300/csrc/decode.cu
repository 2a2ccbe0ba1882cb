// decode.cu -- software BC1/BC7 decoders, fused decode + SH evaluation, and the
// texture-object decode path (Sec. I: random access by block index x block size;
// Sec. II: c(f) = H w(f - p); Sec. III-B: BC1 / BC7 formats).
#include "decode_dev.cuh"
#include "layout.cuh"

cudaError_t decode_init_tables() { return dec_tables_upload(); }

// ---- checked build ------------------------------------------------------------------------
// With GSC_CHECKED every slot entry read from the caller's slot order is checked against
// [-1, n): the first entry outside is recorded (status, slot) and every bad entry is treated as
// an empty slot, so no access uses it. gsc_ctx_sync reports the record as GSC_ERR_DEVICE.
#ifdef GSC_CHECKED
static __device__ int g_check[2];
__device__ __forceinline__ int32_t checked_slot(int32_t o, int64_t n, int64_t s) {
  if (o < -1 || (int64_t)o >= n) {
    if (atomicCAS(&g_check[0], 0, (int)GSC_ERR_DEVICE) == 0) g_check[1] = (int)(s < 0x7FFFFFFF ? s : 0x7FFFFFFF);
    return -1;
  }
  return o;
}
int gsc_check_take(int* where) {
  int h[2] = {0, 0};
  if (cudaMemcpyFromSymbol(h, g_check, sizeof(h)) != cudaSuccess) { cudaGetLastError(); return 0; }
  if (h[0]) {
    const int z[2] = {0, 0};
    cudaMemcpyToSymbol(g_check, z, sizeof(z));
  }
  if (where) *where = h[1];
  return h[0];
}
#else
__device__ __forceinline__ int32_t checked_slot(int32_t o, int64_t, int64_t) { return o; }
int gsc_check_take(int* where) {
  if (where) *where = 0;
  return 0;
}
#endif
extern "C" int32_t gsc_build_checked(void) {
#ifdef GSC_CHECKED
  return 1;
#else
  return 0;
#endif
}

// Texel t of a BC1 block as r | g << 8 | b << 16 | a << 24.
__device__ __forceinline__ uint32_t bc1_texel(uint2 w, int t) {
  const uint32_t c0 = w.x & 0xFFFF, c1 = w.x >> 16;
  const int j = (w.y >> (2 * t)) & 3;
  const int r0 = c0 >> 11, g0 = (c0 >> 5) & 63, b0 = c0 & 31;
  const int r1 = c1 >> 11, g1 = (c1 >> 5) & 63, b1 = c1 & 31;
  int r, g, b, a = 255;
  if (j == 0) { r = dx5(r0); g = dx6(g0); b = dx5(b0); }
  else if (j == 1) { r = dx5(r1); g = dx6(g1); b = dx5(b1); }
  else if (c0 > c1) {
    if (j == 2) { r = d_third5(r0, r1); g = d_third6(g0, g1); b = d_third5(b0, b1); }
    else { r = d_third5(r1, r0); g = d_third6(g1, g0); b = d_third5(b1, b0); }
  } else {
    if (j == 2) { r = d_half5(r0, r1); g = d_half6(g0, g1); b = d_half5(b0, b1); }
    else { r = g = b = a = 0; }
  }
  return (uint32_t)r | ((uint32_t)g << 8) | ((uint32_t)b << 16) | ((uint32_t)a << 24);
}

__device__ __forceinline__ uint32_t getbits(uint64_t lo, uint64_t hi, int off, int n) {
  uint64_t v = off >= 64 ? (hi >> (off - 64)) : (off == 0 ? lo : ((lo >> off) | (hi << (64 - off))));
  return (uint32_t)(v & ((1ull << n) - 1ull));
}
__device__ __forceinline__ int d_expand(int v, int n) { return n >= 8 ? v : ((v << (8 - n)) | (v >> (2 * n - 8))); }
__device__ __forceinline__ int d_interp(int e0, int e1, int w) { return ((64 - w) * e0 + w * e1 + 32) >> 6; }

// Texel t of a BC7 block (two little-endian 64-bit halves) as packed RGBA.
__device__ __forceinline__ uint32_t bc7_texel(uint64_t lo, uint64_t hi, int t) {
  const uint32_t b0 = (uint32_t)(lo & 0xFF);
  if (b0 == 0) return 0u;
  const int mode = __ffs(b0) - 1;
  const DModeInfo M = d_mode_info(mode);
  int pos = mode + 1;
  const int part = (int)getbits(lo, hi, pos, M.pb > 0 ? M.pb : 1) * (M.pb > 0);
  pos += M.pb;
  const int rot = M.rb ? (int)getbits(lo, hi, pos, M.rb) : 0;
  pos += M.rb;
  const int isb = M.isb ? (int)getbits(lo, hi, pos, 1) : 0;
  pos += M.isb;
  const uint32_t pm = M.ns == 1 ? 0u : (M.ns == 2 ? d_part2[part] : d_part3[part]);
  const int s = (pm >> (2 * t)) & 3;
  const int cstart = pos;
  const int astart = cstart + 6 * M.ns * M.cb;
  const int pstart = astart + 2 * M.ns * M.ab;
  const int istart = pstart + (M.epb ? 2 * M.ns : (M.spb ? M.ns : 0));
  int p0 = 0, p1 = 0;
  if (M.epb) { p0 = getbits(lo, hi, pstart + 2 * s, 1); p1 = getbits(lo, hi, pstart + 2 * s + 1, 1); }
  if (M.spb) { p0 = p1 = getbits(lo, hi, pstart + s, 1); }
  const int hp = M.epb | M.spb;
  int e0[4], e1[4];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    int c0 = getbits(lo, hi, cstart + ((c * M.ns + s) * 2 + 0) * M.cb, M.cb);
    int c1 = getbits(lo, hi, cstart + ((c * M.ns + s) * 2 + 1) * M.cb, M.cb);
    e0[c] = d_expand(hp ? (c0 << 1) | p0 : c0, M.cb + hp);
    e1[c] = d_expand(hp ? (c1 << 1) | p1 : c1, M.cb + hp);
  }
  if (M.ab) {
    int a0 = getbits(lo, hi, astart + (2 * s + 0) * M.ab, M.ab);
    int a1 = getbits(lo, hi, astart + (2 * s + 1) * M.ab, M.ab);
    e0[3] = d_expand(M.epb ? (a0 << 1) | p0 : a0, M.ab + M.epb);
    e1[3] = d_expand(M.epb ? (a1 << 1) | p1 : a1, M.ab + M.epb);
  }
  int an1 = 16, an2 = 16;
  if (M.ns == 2) an1 = d_anc2[part];
  if (M.ns == 3) { an1 = d_anc3a[part]; an2 = d_anc3b[part]; }
  const int before = (t > 0) + (t > an1) + (t > an2);
  const int is_anchor = (t == 0) | (t == an1) | (t == an2);
  const int pri = getbits(lo, hi, istart + t * M.ib - before, M.ib - is_anchor);
  int ci = pri, cbits = M.ib, ai = pri, abits = M.ib;
  if (M.ib2) {
    const int sec = getbits(lo, hi, istart + 16 * M.ib - 1 + t * M.ib2 - (t > 0), M.ib2 - (t == 0));
    if (isb) { ci = sec; cbits = M.ib2; } else { ai = sec; abits = M.ib2; }
  }
  const int wc = d_wgt(cbits, ci);
  int px[4];
#pragma unroll
  for (int c = 0; c < 3; c++) px[c] = d_interp(e0[c], e1[c], wc);
  px[3] = M.ab ? d_interp(e0[3], e1[3], d_wgt(abits, ai)) : 255;
  if (rot) { int tmp = px[3]; px[3] = px[rot - 1]; px[rot - 1] = tmp; }
  return (uint32_t)px[0] | ((uint32_t)px[1] << 8) | ((uint32_t)px[2] << 16) | ((uint32_t)px[3] << 24);
}

// ---- stream addressing -------------------------------------------------------------------
struct BlockLoc { int64_t off; int kind; };  // kind: 0 dropped, 1 BC1, 7 BC7

__device__ __forceinline__ int stream_of(const DevTable& T, int64_t g) {
  int si = 0;
#pragma unroll 1
  for (int i = 0; i < T.n_streams; i++)
    if (g >= T.first_group[i] && g < T.first_group[i] + T.stream_groups[i]) si = i;
  return si;
}

// Block k of group g: a group's BC7 blocks come first, then its BC1 blocks, each in block
// order (which blocks are BC7 follows the layout); blocks past the kept coefficients (layout D
// streams only) are dropped.
__device__ __forceinline__ BlockLoc locate(const DevTable& T, int si, int64_t g, int k) {
  const int b = T.bands[si], j = T.bc7[si];
  const int64_t gbytes = 16 * j + 8 * (b - j);
  const int64_t base = T.byte_offset[si] + (g - T.first_group[si]) * gbytes;
  BlockLoc L;
  if (k >= b) { L.off = 0; L.kind = 0; }
  else if (lay_bc7(T.layout, j, k)) { L.off = base + 16 * lay_rank(T.layout, j, k); L.kind = 7; }
  else { L.off = base + 16 * j + 8 * lay_rank(T.layout, j, k); L.kind = 1; }
  return L;
}

// Index in a decoded tile (block k's texel t at 17 k + t) of coefficient c of slot u.
template <int LAYOUT>
__device__ __forceinline__ int tile_at(int u, int c) {
  int k, t;
  lay_inv(LAYOUT, u, c, k, t);
  return 17 * k + t;
}


// ---- warp-cooperative decode: one whole block per lane ----------------------------------
// A warp owns two groups (32 slots, 32 blocks). Phase A: lane l decodes block k = l % 16 of
// group l / 16 completely (the block is parsed once) into a shared tile; phase B: lane l
// owns slot l % 16 of the same group and reads its 16 texels back. The tile index
// gw * 272 + 17 k + t keeps both phases free of bank conflicts.
#define WTILE 544

// The raw words of block k of group g (kind 0: dropped, 1: BC1 in w.x/w.y, 7: BC7), loaded
// ahead of their decode.
struct RawBlock {
  uint4 w;
  int kind;
};

template <int KIND>
__device__ __forceinline__ RawBlock fetch_block(const DevTable& T, const uint8_t* __restrict__ blocks, int64_t g, int k) {
  RawBlock r;
  r.w = make_uint4(0u, 0u, 0u, 0u);
  if (KIND == 7) {
    r.w = __ldg(reinterpret_cast<const uint4*>(blocks) + g * 16 + k);
    r.kind = 7;
  } else if (KIND == 1) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(blocks) + g * 16 + k);
    r.w.x = v.x; r.w.y = v.y;
    r.kind = 1;
  } else {
    const int si = stream_of(T, g);
    const BlockLoc L = locate(T, si, g, k);
    r.kind = L.kind;
    if (L.kind != 0) {
      const uint2* p = reinterpret_cast<const uint2*>(blocks + L.off);
      const uint2 w0 = __ldg(p);
      r.w.x = w0.x; r.w.y = w0.y;
      if (L.kind == 7) { const uint2 w1 = __ldg(p + 1); r.w.z = w1.x; r.w.w = w1.y; }
    }
  }
  return r;
}

template <int KIND>
__device__ __forceinline__ void decode_raw(const RawBlock& r, uint32_t (&tx)[16], const DecTables* S, uint4* ep) {
  if (KIND == 7 || (KIND == 0 && r.kind == 7)) {
    bc7_block(((uint64_t)r.w.y << 32) | r.w.x, ((uint64_t)r.w.w << 32) | r.w.z, tx, S, ep);
  } else if (KIND == 1 || (KIND == 0 && r.kind == 1)) {
    bc1_block(make_uint2(r.w.x, r.w.y), tx);
  } else {
#pragma unroll
    for (int t = 0; t < 16; t++) tx[t] = 0xFF808080u;
  }
}

// Block k of group g of the stream table into 16 packed texels (RGB + A); 128 where dropped.
template <int KIND>
__device__ __forceinline__ void block_texels(const DevTable& T, const uint8_t* __restrict__ blocks, int64_t g, int k,
                                             uint32_t (&tx)[16], const DecTables* S, uint4* ep) {
  if (KIND == 7) {
    const uint4 w = __ldg(reinterpret_cast<const uint4*>(blocks) + g * 16 + k);
    bc7_block(((uint64_t)w.y << 32) | w.x, ((uint64_t)w.w << 32) | w.z, tx, S, ep);
  } else if (KIND == 1) {
    bc1_block(__ldg(reinterpret_cast<const uint2*>(blocks) + g * 16 + k), tx);
  } else {
    const int si = stream_of(T, g);
    const BlockLoc L = locate(T, si, g, k);
    if (L.kind == 7) {
      const uint2* p = reinterpret_cast<const uint2*>(blocks + L.off);
      const uint2 w0 = __ldg(p), w1 = __ldg(p + 1);
      bc7_block(((uint64_t)w0.y << 32) | w0.x, ((uint64_t)w1.y << 32) | w1.x, tx, S, ep);
    } else if (L.kind == 1) {
      bc1_block(__ldg(reinterpret_cast<const uint2*>(blocks + L.off)), tx);
    } else {
#pragma unroll
      for (int t = 0; t < 16; t++) tx[t] = 0xFF808080u;
    }
  }
}



template <int KIND, int LAYOUT>
__global__ void __launch_bounds__(256) k_decode2(DevTable T, const uint8_t* __restrict__ blocks,
                                                 const int32_t* __restrict__ perm, uint8_t* __restrict__ texels) {
  __shared__ DecTables S;
  __shared__ uint32_t tile[8][WTILE];
  __shared__ uint4 s_ep[256][3];
  load_tables(&S);
  __syncthreads();
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, gw = l >> 4, kt = l & 15;
  const int64_t npairs = ((int64_t)T.n_groups + 1) / 2;
  uint32_t* my = tile[w] + gw * 272;
  for (int64_t pr = (int64_t)blockIdx.x * 8 + w; pr < npairs; pr += (int64_t)gridDim.x * 8) {
    const int64_t g = pr * 2 + gw;
    const bool live = g < T.n_groups;
    uint32_t tx[16];
    if (live) block_texels<KIND>(T, blocks, g, kt, tx, &S, s_ep[threadIdx.x]);
#pragma unroll
    for (int t = 0; t < 16; t++) my[17 * kt + t] = live ? tx[t] : 0u;
    __syncwarp();
    const int32_t o = live ? checked_slot(__ldg(perm + g * 16 + kt), T.n, g * 16 + kt) : -1;
    if (o >= 0) {
      uint32_t wv[12];
#pragma unroll
      for (int i = 0; i < 12; i++) wv[i] = 0;
#pragma unroll
      for (int k = 0; k < 16; k++) {
        const uint32_t px = my[tile_at<LAYOUT>(kt, k)];
#pragma unroll
        for (int c = 0; c < 3; c++) {
          const int byte = 3 * k + c;
          wv[byte >> 2] |= ((px >> (8 * c)) & 255u) << (8 * (byte & 3));
        }
      }
      uint4* dst = reinterpret_cast<uint4*>(texels + (int64_t)o * 48);
      dst[0] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
      dst[1] = make_uint4(wv[4], wv[5], wv[6], wv[7]);
      dst[2] = make_uint4(wv[8], wv[9], wv[10], wv[11]);
    }
    __syncwarp();
  }
}

// SH evaluation of one Gaussian for V views and the store in the requested order. x holds the
// dequantised coefficients with the SH constants folded in; both decoders share this code, so
// their colours agree bit for bit when their texels do. Views go in pairs through the
// two-lane multiply-adds (one coefficient against the basis of two views), four views at a
// time (three 16-byte stores of a Gaussian-major row when V is a multiple of 4).
// VF > 0: a launch of exactly VF views into Gaussian-major rows, known at compile time.
// ORD: the output order known at compile time (GSC_OUT_SLOT_ROWS), or read at run time among
// orders 0-2 (-1) or 0-3 (-3).
template <bool CAMS, int VF, int ORD = -1>
__device__ __forceinline__ void eval_store(const float (&xr)[16], const float (&xg)[16], const float (&xb)[16],
                                           int64_t o, int64_t s, float3 p, const float (*s_view)[64], int V_,
                                           int out_order_, int64_t n, int64_t ns, float* __restrict__ rgb) {
  const int V = VF > 0 ? VF : V_;
  const int out_order = VF > 0 ? (int)GSC_OUT_GAUSS_MAJOR : out_order_;
  const float2 np0 = make_float2(-p.x, -p.x), np1 = make_float2(-p.y, -p.y), np2 = make_float2(-p.z, -p.z);
  for (int v0 = 0; v0 < V; v0 += 4) {
    float res[12];
#pragma unroll
    for (int pr = 0; pr < 2; pr++) {
      const int v = v0 + 2 * pr;
      if (v >= V) break;
      const int v1 = v + 1 < V ? v + 1 : v;
      float2 dx = make_float2(s_view[0][v], s_view[0][v1]);
      float2 dy = make_float2(s_view[1][v], s_view[1][v1]);
      float2 dz = make_float2(s_view[2][v], s_view[2][v1]);
      if (CAMS) { dx = __fadd2_rn(dx, np0); dy = __fadd2_rn(dy, np1); dz = __fadd2_rn(dz, np2); }
      const float2 n2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
      float2 r;
      r.x = n2.x > 0.f ? rsqrtf(n2.x) : 0.f;
      r.y = n2.y > 0.f ? rsqrtf(n2.y) : 0.f;
      dx = __fmul2_rn(dx, r); dy = __fmul2_rn(dy, r); dz = __fmul2_rn(dz, r);
      // a camera on the Gaussian: r = 0 already zeroes x and y; the direction is (0, 0, 1)
      if (n2.x <= 0.f) dz.x = 1.f;
      if (n2.y <= 0.f) dz.y = 1.f;
      float2 P[16];
      sh_poly2(dx, dy, dz, P);
      float2 ar = make_float2(xr[0], xr[0]), ag = make_float2(xg[0], xg[0]), ab = make_float2(xb[0], xb[0]);
#pragma unroll
      for (int k = 1; k < 16; k++) {
        ar = __ffma2_rn(make_float2(xr[k], xr[k]), P[k], ar);
        ag = __ffma2_rn(make_float2(xg[k], xg[k]), P[k], ag);
        ab = __ffma2_rn(make_float2(xb[k], xb[k]), P[k], ab);
      }
      res[6 * pr + 0] = ar.x; res[6 * pr + 1] = ag.x; res[6 * pr + 2] = ab.x;
      res[6 * pr + 3] = ar.y; res[6 * pr + 4] = ag.y; res[6 * pr + 5] = ab.y;
    }
    const int nv = V - v0 < 4 ? V - v0 : 4;
    if (ORD == GSC_OUT_SLOT_ROWS) {
      if ((V & 3) == 0) {
        float4* d = reinterpret_cast<float4*>(rgb + (s * V + v0) * 3);
        d[0] = make_float4(res[0], res[1], res[2], res[3]);
        d[1] = make_float4(res[4], res[5], res[6], res[7]);
        d[2] = make_float4(res[8], res[9], res[10], res[11]);
      } else {
        float* d = rgb + (s * V + v0) * 3;
#pragma unroll
        for (int q = 0; q < 12; q++)
          if (q < 3 * nv) d[q] = res[q];
      }
    } else if (out_order == GSC_OUT_GAUSS_MAJOR && (V & 3) == 0) {
      float4* d = reinterpret_cast<float4*>(rgb + (o * V + v0) * 3);
      d[0] = make_float4(res[0], res[1], res[2], res[3]);
      d[1] = make_float4(res[4], res[5], res[6], res[7]);
      d[2] = make_float4(res[8], res[9], res[10], res[11]);
    } else if (out_order == GSC_OUT_GAUSS_MAJOR) {
      float* d = rgb + (o * V + v0) * 3;
#pragma unroll
      for (int q = 0; q < 12; q++)
        if (q < 3 * nv) d[q] = res[q];
    } else if (ORD == -3 && out_order == GSC_OUT_SLOT_ROWS) {
      float* d = rgb + (s * V + v0) * 3;
#pragma unroll
      for (int q = 0; q < 12; q++)
        if (q < 3 * nv) d[q] = res[q];
    } else {
      const int64_t idx = out_order == GSC_OUT_VIEW_MAJOR ? o : s;
      const int64_t stride = out_order == GSC_OUT_VIEW_MAJOR ? n : ns;
#pragma unroll
      for (int q = 0; q < 4; q++)
        if (q < nv) {
          float* d = rgb + ((int64_t)(v0 + q) * stride + idx) * 3;
          d[0] = res[3 * q]; d[1] = res[3 * q + 1]; d[2] = res[3 * q + 2];
        }
    }
  }
}

__device__ __forceinline__ void load_views(float (*s_view)[64], float* s_deq, const float* dirs, const float* cams,
                                           int V, const DevTable& T) {
  for (int i = threadIdx.x; i < V; i += blockDim.x) {
    const float* src = cams ? cams : dirs;
    s_view[0][i] = src[3 * i]; s_view[1][i] = src[3 * i + 1]; s_view[2][i] = src[3 * i + 2];
  }
  if (threadIdx.x < 16) s_deq[threadIdx.x] = __fmul_rn(__fdiv_rn(T.scales[threadIdx.x], 255.0f), c_shc[threadIdx.x]);
}

// CTAs of 4 warps (128 threads x at most 128 registers): one fits where one BC7-search CTA
// retired, so an evaluation launched beside an encode on a higher-priority stream starts early.
#define EVAL_THREADS 128
// No register cap: capping at 5 or 6 resident CTAs per SM spills in the evaluation loop and
// measured slower (3M Gaussians, all-BC7, 8 cameras: 0.205 ms uncapped, 0.225 ms and 0.260 ms).
#ifndef EVAL_MIN_BLOCKS
#define EVAL_MIN_BLOCKS 1
#endif
// LIST: only the groups listed in glist[0, n_list) (-1 entries skipped), e.g. those of the chunks a
// view keeps.
template <int KIND, bool CAMS, int VF, int LAYOUT, bool LIST, int ORD>
__global__ void __launch_bounds__(EVAL_THREADS, EVAL_MIN_BLOCKS) k_eval2(DevTable T, const uint8_t* __restrict__ blocks,
                                               const int32_t* __restrict__ perm, const float* __restrict__ dirs,
                                               const float* __restrict__ pos, const float* __restrict__ cams, int V,
                                               int out_order, float* __restrict__ rgb,
                                               const int32_t* __restrict__ glist, int64_t n_list,
                                               const float* __restrict__ pos_slot) {
  __shared__ DecTables S;
  __shared__ uint32_t tile[EVAL_THREADS / 32][WTILE];
  __shared__ uint4 s_ep[EVAL_THREADS][3];
  __shared__ float s_view[3][64];
  __shared__ __align__(8) float s_deq[16];
  load_tables(&S);
  load_views(s_view, s_deq, dirs, cams, V, T);
  __syncthreads();
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, gw = l >> 4, kt = l & 15, nw = blockDim.x >> 5;
  const int64_t npairs = ((LIST ? n_list : (int64_t)T.n_groups) + 1) / 2;
  const int64_t n = T.n, ns = (int64_t)T.n_groups * 16;
  uint32_t* my = tile[w] + gw * 272;
  const int64_t step = (int64_t)gridDim.x * nw;
  // software pipeline: slot order entries two iterations ahead, blocks and positions one ahead
  auto group_of = [&](int64_t pr) -> int64_t {
    if (!LIST) return pr * 2 + gw;
    const int64_t i = pr * 2 + gw;
    return i < n_list ? (int64_t)__ldg(glist + i) : -1;
  };
  auto valid = [&](int64_t g) { return LIST ? g >= 0 : g < T.n_groups; };
  auto perm_at = [&](int64_t pr) -> int32_t {
    if (pr >= npairs) return -1;
    const int64_t g = group_of(pr);
    return valid(g) ? checked_slot(__ldg(perm + g * 16 + kt), T.n, g * 16 + kt) : -1;
  };
  // centre of slot entry o at tile pair pr: in slot order (pos_slot) or gathered through o
  auto pos_at = [&](int64_t pr_, int32_t o) -> float3 {
    if (!CAMS || o < 0) return make_float3(0.f, 0.f, 0.f);
    if (pos_slot) {
      const int64_t s_ = group_of(pr_) * 16 + kt;
      return make_float3(__ldg(pos_slot + 3 * s_), __ldg(pos_slot + 3 * s_ + 1), __ldg(pos_slot + 3 * s_ + 2));
    }
    return make_float3(__ldg(pos + 3 * (int64_t)o), __ldg(pos + 3 * (int64_t)o + 1), __ldg(pos + 3 * (int64_t)o + 2));
  };
  int64_t pr = (int64_t)blockIdx.x * nw + w;
  RawBlock raw;
  raw.kind = 0;
  raw.w = make_uint4(0u, 0u, 0u, 0u);
  if (pr < npairs && valid(group_of(pr))) raw = fetch_block<KIND>(T, blocks, group_of(pr), kt);
  int32_t o = perm_at(pr), o1 = perm_at(pr + step);
  float3 p = pos_at(pr, o);
  for (; pr < npairs; pr += step) {
    const int64_t g = group_of(pr);
    const bool live = valid(g);
    // loads for the next iterations
    const int64_t prn = pr + step;
    RawBlock rawn;
    rawn.kind = 0;
    rawn.w = make_uint4(0u, 0u, 0u, 0u);
    if (prn < npairs && valid(group_of(prn))) rawn = fetch_block<KIND>(T, blocks, group_of(prn), kt);
    const float3 pn = pos_at(prn, o1);
    const int32_t o2 = perm_at(prn + step);
    {
      uint32_t tx[16];
      decode_raw<KIND>(raw, tx, &S, s_ep[threadIdx.x]);  // past the last group: never read back
#pragma unroll
      for (int t = 0; t < 16; t++) my[17 * kt + t] = tx[t];
    }
    __syncwarp();
    const int64_t s = g * 16 + kt;
    if (o >= 0) {
      // (q - 128) * f_k for two consecutive k at once: 0x4B0000qq is 2^23 + q exactly
      float xr[16], xg[16], xb[16];
      const float2 m = make_float2(-8388736.0f, -8388736.0f);
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const uint32_t p0 = my[tile_at<LAYOUT>(kt, 2 * j)], p1 = my[tile_at<LAYOUT>(kt, 2 * j + 1)];
        const float2 f = *reinterpret_cast<const float2*>(s_deq + 2 * j);
        const float2 r = __fmul2_rn(__fadd2_rn(make_float2(u23(p0, 0), u23(p1, 0)), m), f);
        const float2 gg = __fmul2_rn(__fadd2_rn(make_float2(u23(p0, 1), u23(p1, 1)), m), f);
        const float2 b = __fmul2_rn(__fadd2_rn(make_float2(u23(p0, 2), u23(p1, 2)), m), f);
        xr[2 * j] = r.x; xr[2 * j + 1] = r.y; xg[2 * j] = gg.x; xg[2 * j + 1] = gg.y; xb[2 * j] = b.x; xb[2 * j + 1] = b.y;
      }
      eval_store<CAMS, VF, ORD>(xr, xg, xb, o, s, p, s_view, V, out_order, n, ns, rgb);
    } else if (live && out_order == GSC_OUT_SLOT_ORDER) {
      for (int v = 0; v < V; v++) { float* d = rgb + ((int64_t)v * ns + s) * 3; d[0] = d[1] = d[2] = 0.f; }
    } else if (ORD == GSC_OUT_SLOT_ROWS && live) {
      for (int q = 0; q < 3 * V; q++) rgb[s * V * 3 + q] = 0.f;
    }
    __syncwarp();
    raw = rawn;
    p = pn;
    o = o1;
    o1 = o2;
  }
}

static int kind_of(const DevTable& T) {
  if (T.n_streams == 1 && T.bands[0] == 16 && T.byte_offset[0] == 0) return T.bc7[0] == 16 ? 7 : (T.bc7[0] == 0 ? 1 : 0);
  return 0;
}
// kind for the software decoders: the all-BC7 fast path loads whole 16-byte blocks, so blocks that
// are only 8-byte aligned (the API's minimum) take the stream path's 8-byte loads
static int kind_of(const DevTable& T, const void* blocks) {
  const int k = kind_of(T);
  return (k == 7 && ((uintptr_t)blocks & 15u) != 0) ? 0 : k;
}

// CTAs of `warps` warps, one pair of groups per warp per step; at most 64 warps per SM.
static int eval_grid(int64_t n_groups, int sm_count, int warps = 8) {
  int64_t pairs = (n_groups + 1) / 2;
  int64_t g = ceil_div64(pairs, warps);
  int64_t cap = (int64_t)(sm_count > 0 ? sm_count : gsc_sm_count()) * (64 / warps);
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

cudaError_t launch_decode(const DevTable& T, const uint8_t* blocks, const int32_t* perm, uint8_t* texels,
                          cudaStream_t st) {
  if (T.n_groups == 0) return cudaSuccess;
  const int grid = eval_grid(T.n_groups, gsc_sm_count());
#define DEC_LAUNCH(L)                                                                              \
  do {                                                                                             \
    gsc_count_launch();                                                                            \
    switch (kind_of(T, blocks)) {                                                                  \
      case 7: k_decode2<7, L><<<grid, 256, 0, st>>>(T, blocks, perm, texels); break;               \
      case 1: k_decode2<1, L><<<grid, 256, 0, st>>>(T, blocks, perm, texels); break;               \
      default: k_decode2<0, L><<<grid, 256, 0, st>>>(T, blocks, perm, texels); break;              \
    }                                                                                              \
  } while (0)
  if (T.layout == GSC_LAYOUT_A) DEC_LAUNCH(GSC_LAYOUT_A);
  else if (T.layout == GSC_LAYOUT_B) DEC_LAUNCH(GSC_LAYOUT_B);
  else DEC_LAUNCH(GSC_LAYOUT_D);
#undef DEC_LAUNCH
  return cudaGetLastError();
}

cudaError_t launch_decode_eval(const DevTable& T, const uint8_t* blocks, const int32_t* perm, const float* dirs,
                               const float* pos, const float* cams, int V, int out_order, float* rgb, int sm_count,
                               cudaStream_t st, const int32_t* glist, int64_t n_list, const float* pos_slot) {
  if (T.n_groups == 0 || (glist && n_list == 0)) return cudaSuccess;
  if (glist && out_order == GSC_OUT_SLOT_ROWS) return cudaErrorInvalidValue;  // group lists: orders 0-2
  const int grid = eval_grid(glist ? n_list : T.n_groups, sm_count, EVAL_THREADS / 32);
  const int kind = kind_of(T, blocks);
  // runtime view count only: a compile-time 8-view form raised this kernel to 140 registers (one
  // resident CTA fewer) and measured no faster (the texture kernel does use one)
#define EVAL_LAUNCH(K, C, L)                                                                                     \
  do {                                                                                                           \
    gsc_count_launch();                                                                                          \
    if (glist)                                                                                                   \
      k_eval2<K, C, 0, L, true, -1><<<grid, EVAL_THREADS, 0, st>>>(T, blocks, perm, dirs, pos, cams, V,          \
                                                                   out_order, rgb, glist, n_list, pos_slot);     \
    else if (out_order == GSC_OUT_SLOT_ROWS)                                                                     \
      k_eval2<K, C, 0, L, false, GSC_OUT_SLOT_ROWS><<<grid, EVAL_THREADS, 0, st>>>(                            \
          T, blocks, perm, dirs, pos, cams, V, out_order, rgb, nullptr, 0, pos_slot);                            \
    else                                                                                                         \
      k_eval2<K, C, 0, L, false, -1><<<grid, EVAL_THREADS, 0, st>>>(T, blocks, perm, dirs, pos, cams, V,         \
                                                                    out_order, rgb, nullptr, 0, pos_slot);       \
  } while (0)
#define EVAL_KINDS(C, L)                                                                                         \
  do {                                                                                                           \
    if (kind == 7) EVAL_LAUNCH(7, C, L); else if (kind == 1) EVAL_LAUNCH(1, C, L); else EVAL_LAUNCH(0, C, L);    \
  } while (0)
#define EVAL_LAYOUTS(C)                                                                                          \
  do {                                                                                                           \
    if (T.layout == GSC_LAYOUT_A) EVAL_KINDS(C, GSC_LAYOUT_A);                                                   \
    else if (T.layout == GSC_LAYOUT_B) EVAL_KINDS(C, GSC_LAYOUT_B);                                              \
    else EVAL_KINDS(C, GSC_LAYOUT_D);                                                                            \
  } while (0)
  if (cams) EVAL_LAYOUTS(true);
  else EVAL_LAYOUTS(false);
#undef EVAL_LAYOUTS
#undef EVAL_KINDS
#undef EVAL_LAUNCH
  return cudaGetLastError();
}

// Positions in slot order: out[s] = pos[perm[s]] (zeros for padding slots).
__global__ void k_pos_to_slots(const float* __restrict__ pos, const int32_t* __restrict__ perm, int64_t n, int64_t ns,
                               float* __restrict__ out) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
    int32_t o = perm[s];
    o = checked_slot(o, n, s);
    float x = 0.f, y = 0.f, z = 0.f;
    if (o >= 0) { x = pos[3 * (int64_t)o]; y = pos[3 * (int64_t)o + 1]; z = pos[3 * (int64_t)o + 2]; }
    out[3 * s] = x; out[3 * s + 1] = y; out[3 * s + 2] = z;
  }
}

cudaError_t launch_pos_to_slots(const float* pos, const int32_t* perm, int64_t n, int64_t ns, float* out, int sm_count,
                                cudaStream_t st) {
  if (ns <= 0) return cudaSuccess;
  int64_t grid = (ns + 255) / 256;
  const int64_t cap = (int64_t)(sm_count > 0 ? sm_count : 1) * 8;
  if (grid > cap) grid = cap;
  gsc_count_launch();
  k_pos_to_slots<<<(int)grid, 256, 0, st>>>(pos, perm, n, ns, out);
  return cudaGetLastError();
}

// ---- block-level software decode -------------------------------------------------------------
__global__ void k_decode_blocks(const uint8_t* __restrict__ blocks, int64_t nblk, int format,
                                uint32_t* __restrict__ rgba) {
  const int64_t total = nblk * 16;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i >> 4;
    const int t = (int)(i & 15);
    uint32_t px;
    if (format == GSC_FMT_BC1) {
      px = bc1_texel(__ldg(reinterpret_cast<const uint2*>(blocks) + b), t);
    } else {
      uint4 w = __ldg(reinterpret_cast<const uint4*>(blocks) + b);
      px = bc7_texel(((uint64_t)w.y << 32) | w.x, ((uint64_t)w.w << 32) | w.z, t);
    }
    rgba[i] = px;
  }
}

cudaError_t launch_decode_blocks(const uint8_t* blocks, int64_t nblk, int format, uint8_t* rgba, cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
  int64_t grid = ceil_div64(nblk * 16, 256);
  if (grid > gsc_sm_count() * 16) grid = gsc_sm_count() * 16;
  gsc_count_launch(); k_decode_blocks<<<(int)grid, 256, 0, st>>>(blocks, nblk, format, reinterpret_cast<uint32_t*>(rgba));
  return cudaGetLastError();
}

// ---- texture-object path ----------------------------------------------------------------------
// Blocks of one format are laid out row-major, TEXW blocks per row, in a CUDA array whose
// elements are whole blocks (uint2 for BC1, uint4 for BC7) viewed as a BC1 / BC7 texture.
#define TEXW 16384

struct TexImg {
  cudaArray_t arr = nullptr;
  cudaTextureObject_t tex = 0;
};

static cudaError_t make_tex(const uint8_t* d_lin, int64_t nblk, int bc7, TexImg* out, cudaStream_t st) {
  const int64_t w = nblk < TEXW ? (nblk > 0 ? nblk : 1) : TEXW;
  const int64_t h = nblk > 0 ? ceil_div64(nblk, w) : 1;
  const int bpb = bc7 ? 16 : 8;
  cudaChannelFormatDesc d = bc7 ? cudaCreateChannelDesc(32, 32, 32, 32, cudaChannelFormatKindUnsigned)
                                : cudaCreateChannelDesc(32, 32, 0, 0, cudaChannelFormatKindUnsigned);
  cudaError_t e = cudaMallocArray(&out->arr, &d, (size_t)w, (size_t)h);
  if (e != cudaSuccess) return e;
  if (nblk > 0) {
    const int64_t full_rows = nblk / w, rem = nblk % w;
    if (full_rows > 0) {
      e = cudaMemcpy2DToArrayAsync(out->arr, 0, 0, d_lin, (size_t)(w * bpb), (size_t)(w * bpb),
                                   (size_t)full_rows, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
    }
    if (rem > 0) {
      e = cudaMemcpy2DToArrayAsync(out->arr, 0, (size_t)full_rows, d_lin + full_rows * w * bpb,
                                   (size_t)(rem * bpb), (size_t)(rem * bpb), 1, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
    }
  }
  cudaResourceDesc rd = {};
  rd.resType = cudaResourceTypeArray;
  rd.res.array.array = out->arr;
  cudaTextureDesc td = {};
  td.addressMode[0] = td.addressMode[1] = cudaAddressModeClamp;
  td.filterMode = cudaFilterModePoint;
  td.readMode = cudaReadModeElementType;
  td.normalizedCoords = 0;
  cudaResourceViewDesc vd = {};
  vd.format = bc7 ? cudaResViewFormatUnsignedBlockCompressed7 : cudaResViewFormatUnsignedBlockCompressed1;
  vd.width = (size_t)w * 4;
  vd.height = (size_t)h * 4;
  vd.depth = 0;
  return cudaCreateTextureObject(&out->tex, &rd, &td, &vd);
}

static void free_tex(TexImg* t) {
  if (t->tex) cudaDestroyTextureObject(t->tex);
  if (t->arr) cudaFreeArray(t->arr);
  t->tex = 0;
  t->arr = nullptr;
}

__device__ __forceinline__ uint32_t tex_fetch(cudaTextureObject_t tex, int64_t b, int t) {
  const int x = (int)(b % TEXW) * 4 + (t & 3), y = (int)(b / TEXW) * 4 + (t >> 2);
  float4 f = tex2D<float4>(tex, (float)x + 0.5f, (float)y + 0.5f);
  uint32_t r = (uint32_t)__float2int_rn(f.x * 255.0f), g = (uint32_t)__float2int_rn(f.y * 255.0f);
  uint32_t bb = (uint32_t)__float2int_rn(f.z * 255.0f), a = (uint32_t)__float2int_rn(f.w * 255.0f);
  return r | (g << 8) | (bb << 16) | (a << 24);
}

__global__ void k_tex_blocks(cudaTextureObject_t tex, int64_t nblk, uint32_t* __restrict__ rgba) {
  const int64_t total = nblk * 16;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    rgba[i] = tex_fetch(tex, i >> 4, (int)(i & 15));
}

gsc_status decode_blocks_tex_run(gsc_ctx* ctx, const uint8_t* blocks, int64_t nblk, int format, uint8_t* rgba,
                                 cudaStream_t st) {
  (void)ctx;
  if (nblk <= 0) return GSC_OK;
  TexImg img;
  GSC_CUDA(cudaStreamSynchronize(st));
  cudaError_t e = make_tex(blocks, nblk, format == GSC_FMT_BC7, &img, st);
  if (e == cudaSuccess) {
    int64_t grid = ceil_div64(nblk * 16, 256);
    if (grid > gsc_sm_count() * 16) grid = gsc_sm_count() * 16;
    gsc_count_launch(); k_tex_blocks<<<(int)grid, 256, 0, st>>>(img.tex, nblk, reinterpret_cast<uint32_t*>(rgba));
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  free_tex(&img);
  return e == cudaSuccess ? GSC_OK : GSC_ERR_CUDA;
}

struct TexBases { int64_t b7[GSC_MODES], b1[GSC_MODES]; };

// Gathers every kept block of the streams into one linear buffer per format.
__global__ void k_gather_streams(DevTable T, TexBases B, const uint8_t* __restrict__ blocks,
                                 uint8_t* __restrict__ lin7, uint8_t* __restrict__ lin1) {
  const int64_t total = (int64_t)T.n_groups * 16;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = i >> 4;
    const int k = (int)(i & 15);
    const int si = stream_of(T, g);
    BlockLoc L = locate(T, si, g, k);
    const int j = T.bc7[si], b = T.bands[si];
    const int64_t gi = g - T.first_group[si];
    const int r = lay_rank(T.layout, j, k);
    if (L.kind == 7) {
      const uint2* src = reinterpret_cast<const uint2*>(blocks + L.off);
      uint2* dst = reinterpret_cast<uint2*>(lin7 + (B.b7[si] + gi * j + r) * 16);
      dst[0] = src[0]; dst[1] = src[1];
    } else if (L.kind == 1) {
      *reinterpret_cast<uint2*>(lin1 + (B.b1[si] + gi * (b - j) + r) * 8) = *reinterpret_cast<const uint2*>(blocks + L.off);
    }
  }
}

__global__ void k_tex_streams(DevTable T, TexBases B, cudaTextureObject_t tex7, cudaTextureObject_t tex1,
                              const int32_t* __restrict__ perm, uint8_t* __restrict__ texels) {
  const int64_t total = (int64_t)T.n_groups * 16 * 16;  // (slot, k)
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i >> 4;
    const int k = (int)(i & 15);
    const int32_t o = checked_slot(perm[s], T.n, s);
    if (o < 0) continue;
    const int64_t g = s >> 4;
    int blk, t;
    lay_inv(T.layout, (int)(s & 15), k, blk, t);
    const int si = stream_of(T, g);
    const int j = T.bc7[si], b = T.bands[si];
    const int64_t gi = g - T.first_group[si];
    const int r = lay_rank(T.layout, j, blk);
    uint32_t px;
    if (blk >= b) px = 0x808080u;
    else if (lay_bc7(T.layout, j, blk)) px = tex_fetch(tex7, B.b7[si] + gi * j + r, t);
    else px = tex_fetch(tex1, B.b1[si] + gi * (b - j) + r, t);
    uint8_t* d = texels + (int64_t)o * 48 + 3 * k;
    d[0] = px & 255; d[1] = (px >> 8) & 255; d[2] = (px >> 16) & 255;
  }
}

void tex_cache_free(gsc_ctx* c) {
  for (int f = 0; f < 2; f++) {
    TexImg img;
    img.arr = c->tex[f].arr;
    img.tex = c->tex[f].tex;
    free_tex(&img);
    c->tex[f].arr = nullptr;
    c->tex[f].tex = 0;
    c->tex[f].nblk = -1;
    if (c->tex_lin[f]) cudaFree(c->tex_lin[f]);
    c->tex_lin[f] = nullptr;
    c->tex_lin_bytes[f] = 0;
  }
}

// Staging buffer and texture of one format, reused while the block count is unchanged.
static cudaError_t tex_slot(gsc_ctx* c, int f, int64_t nblk, cudaStream_t st, bool* fresh) {
  const size_t need = (size_t)(nblk > 0 ? nblk : 1) * (f ? 16 : 8);
  *fresh = false;
  if (c->tex_lin_bytes[f] < need) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    if (c->tex_lin[f]) cudaFree(c->tex_lin[f]);
    c->tex_lin[f] = nullptr;
    c->tex_lin_bytes[f] = 0;
    e = cudaMalloc(&c->tex_lin[f], need);
    if (e != cudaSuccess) return e;
    c->tex_lin_bytes[f] = need;
  }
  if (c->tex[f].nblk != nblk || !c->tex[f].arr) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    TexImg old;
    old.arr = c->tex[f].arr;
    old.tex = c->tex[f].tex;
    free_tex(&old);
    c->tex[f].arr = nullptr;
    c->tex[f].tex = 0;
    c->tex[f].nblk = -1;
    *fresh = true;
  }
  return cudaSuccess;
}

gsc_status decode_tex_run(gsc_ctx* ctx, const DevTable& T, const uint8_t* blocks, const int32_t* perm,
                          uint8_t* texels, cudaStream_t st) {
  if (T.n_groups == 0) return GSC_OK;
  TexBases B;
  int64_t n7 = 0, n1 = 0;
  for (int i = 0; i < GSC_MODES; i++) { B.b7[i] = 0; B.b1[i] = 0; }
  for (int i = 0; i < T.n_streams; i++) {
    B.b7[i] = n7; B.b1[i] = n1;
    n7 += T.stream_groups[i] * T.bc7[i];
    n1 += T.stream_groups[i] * (T.bands[i] - T.bc7[i]);
  }
  bool fresh7 = false, fresh1 = false;
  cudaError_t e = tex_slot(ctx, 1, n7, st, &fresh7);
  if (e == cudaSuccess) e = tex_slot(ctx, 0, n1, st, &fresh1);
  if (e != cudaSuccess) return GSC_ERR_CUDA;
  int64_t grid = ceil_div64(T.n_groups * 16, 256);
  if (grid > gsc_sm_count() * 16) grid = gsc_sm_count() * 16;
  gsc_count_launch(); k_gather_streams<<<(int)grid, 256, 0, st>>>(T, B, blocks, ctx->tex_lin[1], ctx->tex_lin[0]);
  e = cudaGetLastError();
  // (re)create the arrays if the sizes changed, then copy the staged blocks in stream order
  for (int f = 1; f >= 0 && e == cudaSuccess; f--) {
    const int64_t nb = f ? n7 : n1;
    const bool fresh = f ? fresh7 : fresh1;
    TexImg img;
    img.arr = ctx->tex[f].arr;
    img.tex = ctx->tex[f].tex;
    if (fresh) {
      e = make_tex(ctx->tex_lin[f], nb, f, &img, st);
      ctx->tex[f].arr = img.arr;
      ctx->tex[f].tex = img.tex;
      ctx->tex[f].nblk = nb;
    } else if (nb > 0) {
      const int64_t w = nb < TEXW ? nb : TEXW, bpb = f ? 16 : 8;
      const int64_t full_rows = nb / w, rem = nb % w;
      if (full_rows > 0)
        e = cudaMemcpy2DToArrayAsync(img.arr, 0, 0, ctx->tex_lin[f], (size_t)(w * bpb), (size_t)(w * bpb),
                                     (size_t)full_rows, cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess && rem > 0)
        e = cudaMemcpy2DToArrayAsync(img.arr, 0, (size_t)full_rows, ctx->tex_lin[f] + full_rows * w * bpb,
                                     (size_t)(rem * bpb), (size_t)(rem * bpb), 1, cudaMemcpyDeviceToDevice, st);
    }
  }
  if (e == cudaSuccess) {
    int64_t g2 = ceil_div64(T.n_groups * 256, 256);
    if (g2 > gsc_sm_count() * 16) g2 = gsc_sm_count() * 16;
    gsc_count_launch(); k_tex_streams<<<(int)g2, 256, 0, st>>>(T, B, ctx->tex[1].tex, ctx->tex[0].tex, perm, texels);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? GSC_OK : GSC_ERR_CUDA;
}

// ---- resident texture scene and texture-decoded fused evaluation ----------------------------
// Sec. I: the GPU's fixed-function texture unit decodes BC blocks; a coded scene kept
// resident as BC1/BC7 texture objects is evaluated without a software block decoder.
struct gsc_tex_scene {
  int device;
  DevTable T;
  TexBases B;
  TexImg img[2];       // [0] BC1, [1] BC7
  float4* pos_slot;    // positions in slot order (x, y, z, 0), or null
};

__global__ void k_pos_slot(const float* __restrict__ pos, const int32_t* __restrict__ perm, int64_t n, int64_t ns,
                           float4* __restrict__ out) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t o = checked_slot(perm[s], n, s);
    out[s] = o >= 0 ? make_float4(pos[3 * (int64_t)o], pos[3 * (int64_t)o + 1], pos[3 * (int64_t)o + 2], 0.f)
                    : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// exact (q - 128) from a UNORM8 sample f = q / 255: f * 255 + 1.5 * 2^23 lands on 1.5 * 2^23 + q
__device__ __forceinline__ float unorm_m128(float f) { return fmaf(f, 255.0f, 12582912.0f) - 12583040.0f; }

template <int KIND, bool CAMS, int VF, int LAYOUT>
__global__ void __launch_bounds__(256) k_eval_tex(DevTable T, TexBases B, cudaTextureObject_t tex7,
                                                  cudaTextureObject_t tex1, const int32_t* __restrict__ perm,
                                                  const float* __restrict__ dirs, const float* __restrict__ pos,
                                                  const float* __restrict__ cams, int V, int out_order,
                                                  float* __restrict__ rgb, const float4* __restrict__ pos_slot) {
  __shared__ float s_view[3][64];
  __shared__ __align__(8) float s_deq[16];
  load_views(s_view, s_deq, dirs, cams, V, T);
  __syncthreads();
  const int64_t n = T.n, ns = (int64_t)T.n_groups * 16;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  // the slot's Gaussian and position are loaded one iteration ahead
  auto pos_of = [&](int64_t s, int32_t o) -> float3 {
    if (!CAMS || o < 0) return make_float3(0.f, 0.f, 0.f);
    if (pos_slot) { const float4 q4 = __ldg(pos_slot + s); return make_float3(q4.x, q4.y, q4.z); }
    return make_float3(__ldg(pos + 3 * (int64_t)o), __ldg(pos + 3 * (int64_t)o + 1), __ldg(pos + 3 * (int64_t)o + 2));
  };
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int32_t o_n = s < ns ? checked_slot(__ldg(perm + s), n, s) : -1;
  float3 p_n = pos_of(s, o_n);
  for (; s < ns; s += step) {
    const int32_t o = o_n;
    const float3 p = p_n;
    if (s + step < ns) {
      o_n = checked_slot(__ldg(perm + s + step), n, s + step);
      p_n = pos_of(s + step, o_n);
    }
    if (o < 0) {
      if (out_order == GSC_OUT_SLOT_ORDER)
        for (int v = 0; v < V; v++) { float* d = rgb + ((int64_t)v * ns + s) * 3; d[0] = d[1] = d[2] = 0.f; }
      else if (out_order == GSC_OUT_SLOT_ROWS)
        for (int q = 0; q < 3 * V; q++) rgb[s * V * 3 + q] = 0.f;
      continue;
    }
    const int64_t g = s >> 4;
    const int u = (int)(s & 15);
    int si = 0, j = 16, b = 16;
    int64_t gi = g;
    if (KIND == 0) { si = stream_of(T, g); j = T.bc7[si]; b = T.bands[si]; gi = g - T.first_group[si]; }
    float xr[16], xg[16], xb[16];
#pragma unroll
    for (int k = 0; k < 16; k++) {
      // coefficient k of slot u sits in block blk, texel t of the group
      int blk, t;
      lay_inv(LAYOUT, u, k, blk, t);
      float4 f;
      if (KIND == 7) f = make_float4(0.f, 0.f, 0.f, 0.f);
      if (KIND == 7 || (KIND == 0 && blk < b && lay_bc7(LAYOUT, j, blk))) {
        const int64_t bi = KIND == 7 ? g * 16 + blk : B.b7[si] + gi * j + lay_rank(LAYOUT, j, blk);
        const int x = (int)(bi % TEXW) * 4 + (t & 3), y = (int)(bi / TEXW) * 4 + (t >> 2);
        f = tex2D<float4>(tex7, (float)x + 0.5f, (float)y + 0.5f);
      } else if (KIND == 1 || (KIND == 0 && blk < b)) {
        const int64_t bi = KIND == 1 ? g * 16 + blk : B.b1[si] + gi * (b - j) + lay_rank(LAYOUT, j, blk);
        const int x = (int)(bi % TEXW) * 4 + (t & 3), y = (int)(bi / TEXW) * 4 + (t >> 2);
        f = tex2D<float4>(tex1, (float)x + 0.5f, (float)y + 0.5f);
      } else {
        f = make_float4(128.f / 255.f, 128.f / 255.f, 128.f / 255.f, 1.f);
      }
      // exact q - 128 from the unorm value, into the pair slot of k
      const float q = s_deq[k];
      xr[k] = __fmul_rn(unorm_m128(f.x), q); xg[k] = __fmul_rn(unorm_m128(f.y), q); xb[k] = __fmul_rn(unorm_m128(f.z), q);
    }
    eval_store<CAMS, VF, -3>(xr, xg, xb, o, s, p, s_view, V, out_order, n, ns, rgb);
  }
}

extern "C" gsc_status gsc_tex_scene_create(gsc_ctx* c, const gsc_stream_table* table, const uint8_t* d_blocks,
                                           const int32_t* d_perm, const float* d_pos, gsc_tex_scene** out,
                                           void* stream) {
  GscRange gsc_range_("gsc_tex_scene_create");
  if (!c || !out) return GSC_ERR_INVALID_ARG;
  *out = nullptr;
  DevTable T;
  gsc_status st = make_dev_table(table, &T);
  if (st != GSC_OK) return st;
  if (T.n_groups > 0 && !d_blocks) return GSC_ERR_INVALID_ARG;
  if (((uintptr_t)d_blocks % 8) != 0) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  gsc_tex_scene* sc = new gsc_tex_scene();
  sc->device = c->device;
  sc->T = T;
  int64_t n7 = 0, n1 = 0;
  for (int i = 0; i < GSC_MODES; i++) { sc->B.b7[i] = 0; sc->B.b1[i] = 0; }
  for (int i = 0; i < T.n_streams; i++) {
    sc->B.b7[i] = n7; sc->B.b1[i] = n1;
    n7 += T.stream_groups[i] * T.bc7[i];
    n1 += T.stream_groups[i] * (T.bands[i] - T.bc7[i]);
  }
  uint8_t *lin7 = nullptr, *lin1 = nullptr;
  cudaError_t e = cudaMalloc(&lin7, (size_t)(n7 > 0 ? n7 : 1) * 16);
  if (e == cudaSuccess) e = cudaMalloc(&lin1, (size_t)(n1 > 0 ? n1 : 1) * 8);
  if (e == cudaSuccess && T.n_groups > 0) {
    int64_t grid = ceil_div64(T.n_groups * 16, 256);
    if (grid > gsc_sm_count() * 16) grid = gsc_sm_count() * 16;
    gsc_count_launch(); k_gather_streams<<<(int)grid, 256, 0, s>>>(T, sc->B, d_blocks, lin7, lin1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = make_tex(lin7, n7, 1, &sc->img[1], s);
  if (e == cudaSuccess) e = make_tex(lin1, n1, 0, &sc->img[0], s);
  sc->pos_slot = nullptr;
  if (e == cudaSuccess && d_pos && d_perm && T.n_groups > 0) {
    const int64_t ns = (int64_t)T.n_groups * 16;
    e = cudaMalloc(&sc->pos_slot, sizeof(float4) * ns);
    if (e == cudaSuccess) {
      int64_t grid = ceil_div64(ns, 256);
      if (grid > gsc_sm_count() * 16) grid = gsc_sm_count() * 16;
      gsc_count_launch(); k_pos_slot<<<(int)grid, 256, 0, s>>>(d_pos, d_perm, (int64_t)T.n, ns, sc->pos_slot);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (lin7) cudaFree(lin7);
  if (lin1) cudaFree(lin1);
  if (e != cudaSuccess) {
    free_tex(&sc->img[0]);
    free_tex(&sc->img[1]);
    if (sc->pos_slot) cudaFree(sc->pos_slot);
    delete sc;
    return GSC_ERR_CUDA;
  }
  *out = sc;
  return GSC_OK;
}

extern "C" gsc_status gsc_tex_scene_destroy(gsc_tex_scene* sc) {
  if (!sc) return GSC_ERR_INVALID_ARG;
  cudaSetDevice(sc->device);
  free_tex(&sc->img[0]);
  free_tex(&sc->img[1]);
  if (sc->pos_slot) cudaFree(sc->pos_slot);
  delete sc;
  return GSC_OK;
}

extern "C" gsc_status gsc_decode_eval_sh_tex(gsc_ctx* c, const gsc_tex_scene* sc, const int32_t* d_perm,
                                             const float* d_dirs, const float* d_pos, const float* d_cams, int32_t V,
                                             int32_t out_order, float* d_rgb, void* stream) {
  GscRange gsc_range_("gsc_decode_eval_sh_tex");
  if (!c || !sc || sc->device != c->device) return GSC_ERR_INVALID_ARG;
  const DevTable& T = sc->T;
  if (V < 1 || V > 64 || out_order < 0 || out_order > 3) return GSC_ERR_INVALID_ARG;
  if ((d_dirs == nullptr) == (d_cams == nullptr)) return GSC_ERR_INVALID_ARG;
  if (d_cams && !d_pos && !sc->pos_slot && T.n > 0) return GSC_ERR_INVALID_ARG;
  if (T.n_groups > 0 && (!d_perm || !d_rgb)) return GSC_ERR_INVALID_ARG;
  if (((uintptr_t)d_rgb % 16) != 0) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  if (T.n_groups == 0) return GSC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  GscTimed tm(c, T_EVAL_TEX, st);
  const int64_t ns = (int64_t)T.n_groups * 16;
  int64_t grid = ceil_div64(ns, 256);
  const int64_t cap = (int64_t)(c->sm_count > 0 ? c->sm_count : gsc_sm_count()) * 8;
  if (grid > cap) grid = cap;
  const int kind = kind_of(T);
  // 8 views into Gaussian-major rows (the camera-pose workload) run a compile-time view count
  const bool v8 = V == 8 && out_order == GSC_OUT_GAUSS_MAJOR;
  // (layouts A and B run the runtime view count)
#define TEX_LAUNCH(K, C, VF, L)                                                                                   \
  k_eval_tex<K, C, VF, L><<<(int)grid, 256, 0, st>>>(T, sc->B, sc->img[1].tex, sc->img[0].tex, d_perm, d_dirs,   \
                                                     d_pos, d_cams, V, out_order, d_rgb, sc->pos_slot)
#define TEX_LAYOUTS(K, C)                                                                                         \
  do {                                                                                                            \
    gsc_count_launch();                                                                                           \
    if (T.layout == GSC_LAYOUT_A) TEX_LAUNCH(K, C, 0, GSC_LAYOUT_A);                                              \
    else if (T.layout == GSC_LAYOUT_B) TEX_LAUNCH(K, C, 0, GSC_LAYOUT_B);                                         \
    else if (v8) TEX_LAUNCH(K, C, 8, GSC_LAYOUT_D);                                                               \
    else TEX_LAUNCH(K, C, 0, GSC_LAYOUT_D);                                                                       \
  } while (0)
  if (d_cams) {
    if (kind == 7) TEX_LAYOUTS(7, true); else if (kind == 1) TEX_LAYOUTS(1, true); else TEX_LAYOUTS(0, true);
  } else {
    if (kind == 7) TEX_LAYOUTS(7, false); else if (kind == 1) TEX_LAYOUTS(1, false); else TEX_LAYOUTS(0, false);
  }
#undef TEX_LAYOUTS
#undef TEX_LAUNCH
  GSC_CUDA(cudaGetLastError());
  return GSC_OK;
}
