// decode.cu -- software BC1/BC7 decoders, fused decode + SH evaluation, and the
// texture-object decode path (Sec. I: random access by block index x block size;
// Sec. II: c(f) = H w(f - p); Sec. III-B: BC1 / BC7 formats).
#include "bc7_tables.h"
#include "gsc_internal.cuh"

__constant__ uint32_t d_part2[64];
__constant__ uint32_t d_part3[64];
__constant__ uint8_t d_anc2[64];
__constant__ uint8_t d_anc3a[64];
__constant__ uint8_t d_anc3b[64];

cudaError_t decode_init_tables() {
  uint32_t p2[64], p3[64];
  for (int p = 0; p < 64; p++) { p2[p] = bc7_pack_part2(p); p3[p] = bc7_pack_part3(p); }
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(d_part2, p2, sizeof(p2))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(d_part3, p3, sizeof(p3))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(d_anc2, kBC7Anchor2, 64)) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(d_anc3a, kBC7Anchor3a, 64)) != cudaSuccess) return e;
  return cudaMemcpyToSymbol(d_anc3b, kBC7Anchor3b, 64);
}

// ---- BC1 -----------------------------------------------------------------------------
__device__ __forceinline__ int dx5(int x) { return (x << 3) | (x >> 2); }
__device__ __forceinline__ int dx6(int x) { return (x << 2) | (x >> 4); }
// interior entries: the GB300 texture unit's rule (5-bit on codes, 6-bit on expansions)
__device__ __forceinline__ int d_third5(int a, int b) { return ((2 * a + b) * 11) >> 2; }
__device__ __forceinline__ int d_third6(int a, int b) { int A = dx6(a), B = dx6(b); return A + (((B - A) * 321 + 512) >> 10); }
__device__ __forceinline__ int d_half5(int a, int b) { return ((a + b) * 33) >> 3; }
__device__ __forceinline__ int d_half6(int a, int b) { int A = dx6(a), B = dx6(b); return A + (((B - A) * 257 + 256) >> 9); }

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

// ---- BC7 -----------------------------------------------------------------------------
struct DModeInfo { int ns, pb, rb, isb, cb, ab, epb, spb, ib, ib2; };
__device__ __forceinline__ DModeInfo d_mode_info(int m) {
  switch (m) {
    case 0: return {3, 4, 0, 0, 4, 0, 1, 0, 3, 0};
    case 1: return {2, 6, 0, 0, 6, 0, 0, 1, 3, 0};
    case 2: return {3, 6, 0, 0, 5, 0, 0, 0, 2, 0};
    case 3: return {2, 6, 0, 0, 7, 0, 1, 0, 2, 0};
    case 4: return {1, 0, 2, 1, 5, 6, 0, 0, 2, 3};
    case 5: return {1, 0, 2, 0, 7, 8, 0, 0, 2, 2};
    case 6: return {1, 0, 0, 0, 7, 7, 1, 0, 4, 0};
    default: return {2, 6, 0, 0, 5, 5, 1, 0, 2, 0};
  }
}

__device__ __forceinline__ uint32_t getbits(uint64_t lo, uint64_t hi, int off, int n) {
  uint64_t v = off >= 64 ? (hi >> (off - 64)) : (off == 0 ? lo : ((lo >> off) | (hi << (64 - off))));
  return (uint32_t)(v & ((1ull << n) - 1ull));
}
__device__ __forceinline__ int d_expand(int v, int n) { return n >= 8 ? v : ((v << (8 - n)) | (v >> (2 * n - 8))); }
__device__ __forceinline__ int d_interp(int e0, int e1, int w) { return ((64 - w) * e0 + w * e1 + 32) >> 6; }
__device__ __forceinline__ int d_wgt(int ib, int j) {
  if (ib == 2) return (0x402B1500u >> (8 * j)) & 255;
  if (ib == 3) return (int)((0x40372E251B120900ull >> (8 * j)) & 255);
  return j < 8 ? (int)((0x1E1A15110D090400ull >> (8 * j)) & 255) : (int)((0x403C37332F2B2622ull >> (8 * (j - 8))) & 255);
}

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

__device__ __forceinline__ BlockLoc locate(const DevTable& T, int si, int64_t g, int k) {
  const int b = T.bands[si], j = T.bc7[si];
  const int64_t gbytes = 16 * j + 8 * (b - j);
  const int64_t base = T.byte_offset[si] + (g - T.first_group[si]) * gbytes;
  BlockLoc L;
  if (k < j) { L.off = base + 16 * k; L.kind = 7; }
  else if (k < b) { L.off = base + 16 * j + 8 * (k - j); L.kind = 1; }
  else { L.off = 0; L.kind = 0; }
  return L;
}

__device__ __forceinline__ uint32_t decode_at(const uint8_t* __restrict__ blocks, const BlockLoc& L, int t) {
  if (L.kind == 0) return 0x80808080u | 0xFF000000u;
  const uint2* p = reinterpret_cast<const uint2*>(blocks + L.off);
  uint2 w0 = __ldg(p);
  if (L.kind == 1) return bc1_texel(w0, t);
  uint2 w1 = __ldg(p + 1);
  return bc7_texel(((uint64_t)w0.y << 32) | w0.x, ((uint64_t)w1.y << 32) | w1.x, t);
}

// ---- decode to texels ----------------------------------------------------------------------
__global__ void k_decode(DevTable T, const uint8_t* __restrict__ blocks, const int32_t* __restrict__ perm,
                         uint8_t* __restrict__ texels) {
  const int64_t ns = (int64_t)T.n_groups * 16;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t o = __ldg(perm + s);
    const int64_t g = s >> 4;
    const int t = (int)(s & 15);
    const int si = stream_of(T, g);
    uint32_t w[12];
#pragma unroll
    for (int i = 0; i < 12; i++) w[i] = 0;
#pragma unroll
    for (int k = 0; k < 16; k++) {
      uint32_t px = decode_at(blocks, locate(T, si, g, k), t) & 0xFFFFFFu;
      // bytes 3k .. 3k+2 of the Gaussian's 48-byte row
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const int byte = 3 * k + c;
        w[byte >> 2] |= ((px >> (8 * c)) & 255u) << (8 * (byte & 3));
      }
    }
    if (o >= 0) {
      uint4* dst = reinterpret_cast<uint4*>(texels + (int64_t)o * 48);
      dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
      dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
      dst[2] = make_uint4(w[8], w[9], w[10], w[11]);
    }
  }
}

cudaError_t launch_decode(const DevTable& T, const uint8_t* blocks, const int32_t* perm, uint8_t* texels,
                          cudaStream_t st) {
  const int64_t ns = (int64_t)T.n_groups * 16;
  if (ns == 0) return cudaSuccess;
  int64_t grid = ceil_div64(ns, 256);
  if (grid > 152 * 16) grid = 152 * 16;
  gsc_count_launch(); k_decode<<<(int)grid, 256, 0, st>>>(T, blocks, perm, texels);
  return cudaGetLastError();
}

// ---- fused decode + SH evaluation ----------------------------------------------------------
// Real SH to degree 3 (k = l*l + l + m, Condon-Shortley phase), constants from the closed
// forms sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) with the sqrt(2) of m != 0 folded in.
#define SH_C0 0.28209479177387814f   /* sqrt(1/(4 pi)) */
#define SH_C1 0.4886025119029199f    /* sqrt(3/(4 pi)) */
#define SH_C2A 1.0925484305920792f   /* sqrt(15/(4 pi)) */
#define SH_C2B 0.31539156525252005f  /* sqrt(5/(16 pi)) */
#define SH_C2C 0.5462742152960396f   /* sqrt(15/(16 pi)) */
#define SH_C3A 0.5900435899266435f   /* sqrt(35/(32 pi)) */
#define SH_C3B 2.890611442640554f    /* sqrt(105/(4 pi)) */
#define SH_C3C 0.4570457994644658f   /* sqrt(21/(32 pi)) */
#define SH_C3D 0.3731763325901154f   /* sqrt(7/(16 pi)) */
#define SH_C3E 1.445305721320277f    /* sqrt(105/(16 pi)) */

__device__ __forceinline__ void sh_basis(float x, float y, float z, float (&Y)[16]) {
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[0] = SH_C0;
  Y[1] = -SH_C1 * y;
  Y[2] = SH_C1 * z;
  Y[3] = -SH_C1 * x;
  Y[4] = SH_C2A * x * y;
  Y[5] = -SH_C2A * y * z;
  Y[6] = SH_C2B * (2.0f * zz - xx - yy);
  Y[7] = -SH_C2A * x * z;
  Y[8] = SH_C2C * (xx - yy);
  Y[9] = -SH_C3A * y * (3.0f * xx - yy);
  Y[10] = SH_C3B * x * y * z;
  Y[11] = -SH_C3C * y * (4.0f * zz - xx - yy);
  Y[12] = SH_C3D * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
  Y[13] = -SH_C3C * x * (4.0f * zz - xx - yy);
  Y[14] = SH_C3E * z * (xx - yy);
  Y[15] = -SH_C3A * x * (xx - 3.0f * yy);
}

__global__ void k_decode_eval(DevTable T, const uint8_t* __restrict__ blocks, const int32_t* __restrict__ perm,
                              const float* __restrict__ dirs, const float* __restrict__ pos,
                              const float* __restrict__ cams, int V, int out_order, float* __restrict__ rgb) {
  __shared__ float s_deq[16];
  if (threadIdx.x < 16) s_deq[threadIdx.x] = __fdiv_rn(T.scales[threadIdx.x], 255.0f);
  __syncthreads();
  const int64_t ns = (int64_t)T.n_groups * 16;
  const int64_t n = T.n;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t o = __ldg(perm + s);
    const int64_t g = s >> 4;
    const int t = (int)(s & 15);
    if (o < 0) {
      if (out_order == GSC_OUT_SLOT_ORDER)
        for (int v = 0; v < V; v++) { float* d = rgb + ((int64_t)v * ns + s) * 3; d[0] = d[1] = d[2] = 0.0f; }
      continue;
    }
    const int si = stream_of(T, g);
    float x[16][3];
#pragma unroll
    for (int k = 0; k < 16; k++) {
      uint32_t px = decode_at(blocks, locate(T, si, g, k), t);
#pragma unroll
      for (int c = 0; c < 3; c++) x[k][c] = (float)((int)((px >> (8 * c)) & 255u) - 128) * s_deq[k];
    }
    float px0 = 0.f, py0 = 0.f, pz0 = 0.f;
    if (cams) { px0 = __ldg(pos + 3 * o); py0 = __ldg(pos + 3 * o + 1); pz0 = __ldg(pos + 3 * o + 2); }
    for (int v = 0; v < V; v++) {
      float dx, dy, dz;
      if (cams) {
        dx = __ldg(cams + 3 * v) - px0; dy = __ldg(cams + 3 * v + 1) - py0; dz = __ldg(cams + 3 * v + 2) - pz0;
      } else {
        dx = __ldg(dirs + 3 * v); dy = __ldg(dirs + 3 * v + 1); dz = __ldg(dirs + 3 * v + 2);
      }
      float n2 = dx * dx + dy * dy + dz * dz;
      if (n2 > 0.0f) { float r = rsqrtf(n2); dx *= r; dy *= r; dz *= r; }
      else { dx = 0.0f; dy = 0.0f; dz = 1.0f; }
      float Y[16];
      sh_basis(dx, dy, dz, Y);
      float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int k = 0; k < 16; k++)
#pragma unroll
        for (int c = 0; c < 3; c++) acc[c] = fmaf(x[k][c], Y[k], acc[c]);
      float* d;
      if (out_order == GSC_OUT_VIEW_MAJOR) d = rgb + ((int64_t)v * n + o) * 3;
      else if (out_order == GSC_OUT_SLOT_ORDER) d = rgb + ((int64_t)v * ns + s) * 3;
      else d = rgb + ((int64_t)o * V + v) * 3;
      d[0] = acc[0]; d[1] = acc[1]; d[2] = acc[2];
    }
  }
}

cudaError_t launch_decode_eval(const DevTable& T, const uint8_t* blocks, const int32_t* perm, const float* dirs,
                               const float* pos, const float* cams, int V, int out_order, float* rgb, int sm_count,
                               cudaStream_t st) {
  const int64_t ns = (int64_t)T.n_groups * 16;
  if (ns == 0) return cudaSuccess;
  int64_t grid = ceil_div64(ns, 256);
  int64_t cap = (int64_t)(sm_count > 0 ? sm_count : 152) * 8;
  if (grid > cap) grid = cap;
  gsc_count_launch(); k_decode_eval<<<(int)grid, 256, 0, st>>>(T, blocks, perm, dirs, pos, cams, V, out_order, rgb);
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
  if (grid > 152 * 16) grid = 152 * 16;
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

static cudaError_t make_tex(const uint8_t* d_lin, int64_t nblk, int bc7, TexImg* out) {
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
      e = cudaMemcpy2DToArray(out->arr, 0, 0, d_lin, (size_t)(w * bpb), (size_t)(w * bpb), (size_t)full_rows,
                              cudaMemcpyDeviceToDevice);
      if (e != cudaSuccess) return e;
    }
    if (rem > 0) {
      e = cudaMemcpy2DToArray(out->arr, 0, (size_t)full_rows, d_lin + full_rows * w * bpb, (size_t)(rem * bpb),
                              (size_t)(rem * bpb), 1, cudaMemcpyDeviceToDevice);
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
  cudaError_t e = make_tex(blocks, nblk, format == GSC_FMT_BC7, &img);
  if (e == cudaSuccess) {
    int64_t grid = ceil_div64(nblk * 16, 256);
    if (grid > 152 * 16) grid = 152 * 16;
    gsc_count_launch(); k_tex_blocks<<<(int)grid, 256, 0, st>>>(img.tex, nblk, reinterpret_cast<uint32_t*>(rgba));
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  free_tex(&img);
  return e == cudaSuccess ? GSC_OK : GSC_ERR_CUDA;
}

// Gathers every kept block of the streams into one linear buffer per format.
__global__ void k_gather_streams(DevTable T, const uint8_t* __restrict__ blocks, const int64_t* __restrict__ base7,
                                 const int64_t* __restrict__ base1, uint8_t* __restrict__ lin7,
                                 uint8_t* __restrict__ lin1) {
  const int64_t total = (int64_t)T.n_groups * 16;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = i >> 4;
    const int k = (int)(i & 15);
    const int si = stream_of(T, g);
    BlockLoc L = locate(T, si, g, k);
    const int j = T.bc7[si], b = T.bands[si];
    const int64_t gi = g - T.first_group[si];
    if (L.kind == 7) {
      const uint2* src = reinterpret_cast<const uint2*>(blocks + L.off);
      uint2* dst = reinterpret_cast<uint2*>(lin7 + (base7[si] + gi * j + k) * 16);
      dst[0] = src[0]; dst[1] = src[1];
    } else if (L.kind == 1) {
      *reinterpret_cast<uint2*>(lin1 + (base1[si] + gi * (b - j) + (k - j)) * 8) =
          *reinterpret_cast<const uint2*>(blocks + L.off);
    }
  }
}

__global__ void k_tex_streams(DevTable T, cudaTextureObject_t tex7, cudaTextureObject_t tex1,
                              const int64_t* __restrict__ base7, const int64_t* __restrict__ base1,
                              const int32_t* __restrict__ perm, uint8_t* __restrict__ texels) {
  const int64_t total = (int64_t)T.n_groups * 16 * 16;  // (slot, k)
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i >> 4;
    const int k = (int)(i & 15);
    const int32_t o = perm[s];
    if (o < 0) continue;
    const int64_t g = s >> 4;
    const int t = (int)(s & 15);
    const int si = stream_of(T, g);
    const int j = T.bc7[si], b = T.bands[si];
    const int64_t gi = g - T.first_group[si];
    uint32_t px;
    if (k < j) px = tex_fetch(tex7, base7[si] + gi * j + k, t);
    else if (k < b) px = tex_fetch(tex1, base1[si] + gi * (b - j) + (k - j), t);
    else px = 0x808080u;
    uint8_t* d = texels + (int64_t)o * 48 + 3 * k;
    d[0] = px & 255; d[1] = (px >> 8) & 255; d[2] = (px >> 16) & 255;
  }
}

gsc_status decode_tex_run(gsc_ctx* ctx, const DevTable& T, const uint8_t* blocks, const int32_t* perm,
                          uint8_t* texels, cudaStream_t st) {
  (void)ctx;
  if (T.n_groups == 0) return GSC_OK;
  int64_t h7[GSC_MODES], h1[GSC_MODES], n7 = 0, n1 = 0;
  for (int i = 0; i < T.n_streams; i++) {
    h7[i] = n7; h1[i] = n1;
    int64_t ng = T.stream_groups[i];
    n7 += ng * T.bc7[i];
    n1 += ng * (T.bands[i] - T.bc7[i]);
  }
  uint8_t *lin7 = nullptr, *lin1 = nullptr;
  int64_t* d_base = nullptr;
  TexImg i7, i1;
  cudaError_t e = cudaMalloc(&d_base, sizeof(int64_t) * 2 * GSC_MODES);
  if (e == cudaSuccess) e = cudaMalloc(&lin7, (size_t)(n7 > 0 ? n7 : 1) * 16);
  if (e == cudaSuccess) e = cudaMalloc(&lin1, (size_t)(n1 > 0 ? n1 : 1) * 8);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_base, h7, sizeof(int64_t) * GSC_MODES, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_base + GSC_MODES, h1, sizeof(int64_t) * GSC_MODES, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    int64_t grid = ceil_div64(T.n_groups * 16, 256);
    if (grid > 152 * 16) grid = 152 * 16;
    gsc_count_launch(); k_gather_streams<<<(int)grid, 256, 0, st>>>(T, blocks, d_base, d_base + GSC_MODES, lin7, lin1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = make_tex(lin7, n7, 1, &i7);
  if (e == cudaSuccess) e = make_tex(lin1, n1, 0, &i1);
  if (e == cudaSuccess) {
    int64_t grid = ceil_div64(T.n_groups * 256, 256);
    if (grid > 152 * 16) grid = 152 * 16;
    gsc_count_launch(); k_tex_streams<<<(int)grid, 256, 0, st>>>(T, i7.tex, i1.tex, d_base, d_base + GSC_MODES, perm, texels);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  free_tex(&i7);
  free_tex(&i1);
  if (lin7) cudaFree(lin7);
  if (lin1) cudaFree(lin1);
  if (d_base) cudaFree(d_base);
  return e == cudaSuccess ? GSC_OK : GSC_ERR_CUDA;
}
