// decode_dev.cuh -- device code shared by the software decoders and the fused evaluations:
// the BC1 interpolation rule, the BC7 mode descriptors, partition and anchor tables, whole-block
// decoders and the SH basis polynomials (Sec. III-B: BC1 / BC7 formats; Sec. II: c(f) = H w(f - p)).
// The constant tables are per translation unit (static); each unit that launches a kernel using
// them uploads its own copy with dec_tables_upload() when a context is created.
#pragma once
#include "bc7_tables.h"
#include "gsc_internal.cuh"

static __constant__ uint32_t d_part2[64];
static __constant__ uint32_t d_part3[64];
static __constant__ uint8_t d_anc2[64];
static __constant__ uint8_t d_anc3a[64];
static __constant__ uint8_t d_anc3b[64];

static cudaError_t dec_tables_upload() {
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

// ---- BC7 -----------------------------------------------------------------------------
struct DModeInfo { int ns, pb, rb, isb, cb, ab, epb, spb, ib, ib2; };
__host__ __device__ constexpr DModeInfo d_mode_info(int m) {
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

__device__ __forceinline__ int d_wgt(int ib, int j) {
  if (ib == 2) return (0x402B1500u >> (8 * j)) & 255;
  if (ib == 3) return (int)((0x40372E251B120900ull >> (8 * j)) & 255);
  return j < 8 ? (int)((0x1E1A15110D090400ull >> (8 * j)) & 255) : (int)((0x403C37332F2B2622ull >> (8 * (j - 8))) & 255);
}

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

struct DecTables {
  uint32_t part2[64], part3[64];
  uint8_t anc2[64], anc3a[64], anc3b[64];
  uint32_t desc[8];
  uint8_t wt[48];
};

__device__ __forceinline__ void load_tables(DecTables* s) {
  for (int i = threadIdx.x; i < 64; i += blockDim.x) {
    s->part2[i] = d_part2[i]; s->part3[i] = d_part3[i];
    s->anc2[i] = d_anc2[i]; s->anc3a[i] = d_anc3a[i]; s->anc3b[i] = d_anc3b[i];
  }
  if (threadIdx.x < 8) {
    const DModeInfo M = d_mode_info(threadIdx.x);
    s->desc[threadIdx.x] = (uint32_t)M.ns | (M.pb << 2) | (M.rb << 5) | (M.isb << 7) | (M.cb << 8) | (M.ab << 11) |
                           (M.epb << 15) | (M.spb << 16) | (M.ib << 17) | (M.ib2 << 20);
  }
  if (threadIdx.x < 48) s->wt[threadIdx.x] = (uint8_t)d_wgt(2 + threadIdx.x / 16, threadIdx.x % 16);
}

// bits [off, off + 64) of the 128-bit block (off <= 127)
__device__ __forceinline__ uint64_t shr128(uint64_t lo, uint64_t hi, int off) {
  return off >= 64 ? (hi >> (off - 64)) : (off == 0 ? lo : ((lo >> off) | (hi << (64 - off))));
}

__device__ __forceinline__ void bc1_block(uint2 w, uint32_t (&tx)[16]) {
  const uint32_t c0 = w.x & 0xFFFF, c1 = w.x >> 16;
  const int r0 = c0 >> 11, g0 = (c0 >> 5) & 63, b0 = c0 & 31;
  const int r1 = c1 >> 11, g1 = (c1 >> 5) & 63, b1 = c1 & 31;
  const uint32_t p0 = dx5(r0) | (dx6(g0) << 8) | (dx5(b0) << 16) | 0xFF000000u;
  const uint32_t p1 = dx5(r1) | (dx6(g1) << 8) | (dx5(b1) << 16) | 0xFF000000u;
  uint32_t p2, p3;
  if (c0 > c1) {
    p2 = d_third5(r0, r1) | (d_third6(g0, g1) << 8) | (d_third5(b0, b1) << 16) | 0xFF000000u;
    p3 = d_third5(r1, r0) | (d_third6(g1, g0) << 8) | (d_third5(b1, b0) << 16) | 0xFF000000u;
  } else {
    p2 = d_half5(r0, r1) | (d_half6(g0, g1) << 8) | (d_half5(b0, b1) << 16) | 0xFF000000u;
    p3 = 0u;
  }
#pragma unroll
  for (int t = 0; t < 16; t++) {
    const uint32_t j = (w.y >> (2 * t)) & 3;
    tx[t] = (j & 2) ? ((j & 1) ? p3 : p2) : ((j & 1) ? p1 : p0);
  }
}

// A zero bit inserted at position p (0..63): the index of an anchor texel is stored one bit
// short (its top bit is 0), so this gives every texel the full index width.
__device__ __forceinline__ uint64_t ins0(uint64_t x, int p) {
  const uint64_t m = (1ull << p) - 1ull;
  return (x & m) | ((x & ~m) << 1);
}

// Whole BC7 block, uniform control flow across modes (fields located from the mode descriptor).
// Texel t comes out as r | g << 8 | b << 16 (the alpha byte is unspecified). The block is
// parsed once: endpoints per subset go to this lane's slot `ep` in shared memory as 16-bit
// lanes scaled by 4 (e0 r|g, e0 b|a, e1 r|g, e1 b|a), so that the interpolation
// ((64 - w) e0 + w e1 + 32) >> 6 of two channels is two multiply-adds whose result bytes 1
// and 3 are the two channels; the index streams are re-spaced to a fixed width per texel.
// A rotation (modes 4 and 5) puts the alpha-index interpolation of the alpha endpoints into
// the rotated channel.
__device__ __forceinline__ void bc7_block(uint64_t lo, uint64_t hi, uint32_t (&tx)[16], const DecTables* S,
                                          uint4* ep) {
  const uint32_t b0 = (uint32_t)(lo & 0xFF);
  const int mode = b0 ? __ffs(b0) - 1 : 0;
  const uint32_t d = S->desc[mode];
  const int ns = d & 3, pb = (d >> 2) & 7, rb = (d >> 5) & 3, isb = (d >> 7) & 1, cb = (d >> 8) & 7;
  const int ab = (d >> 11) & 15, epb = (d >> 15) & 1, spb = (d >> 16) & 1, ib = (d >> 17) & 7, ib2 = (d >> 20) & 3;
  int pos = mode + 1;
  const uint64_t head = shr128(lo, hi, pos);
  const int part = (int)(head & ((1u << pb) - 1u));
  const int rot = (int)((head >> pb) & ((1u << rb) - 1u));
  const int isbv = (int)((head >> (pb + rb)) & (uint64_t)isb);
  pos += pb + rb + isb;
  const uint32_t pm = ns == 2 ? S->part2[part] : (ns == 3 ? S->part3[part] : 0u);
  const int a1 = ns == 2 ? S->anc2[part] : (ns == 3 ? S->anc3a[part] : 16);
  const int a2 = ns == 3 ? S->anc3b[part] : 16;
  const int cstart = pos, astart = cstart + 6 * ns * cb, pstart = astart + 2 * ns * ab;
  const int istart = pstart + (epb ? 2 * ns : (spb ? ns : 0));
  const int hp = epb | spb, nb = cb + hp, na = ab + epb;
  const uint64_t pbits = shr128(lo, hi, pstart);
  // one window per channel: the 2 ns endpoint fields of a channel span at most 30 bits
  const uint32_t fr = (uint32_t)shr128(lo, hi, cstart), fg = (uint32_t)shr128(lo, hi, cstart + 2 * ns * cb);
  const uint32_t fb = (uint32_t)shr128(lo, hi, cstart + 4 * ns * cb), fa = (uint32_t)shr128(lo, hi, astart);
  const uint32_t cm = (1u << cb) - 1u, amk = (1u << ab) - 1u;
  // bit replication to 8 bits, (v << (8 - n)) | (v >> (2n - 8)), exact also for n = 8
  const int cl8 = 8 - nb, cr8 = 2 * nb - 8, al8 = 8 - na, ar8 = 2 * na - 8;
#pragma unroll
  for (int s = 0; s < 3; s++) {
    if (s < ns) {
      const uint32_t p0 = epb ? (uint32_t)((pbits >> (2 * s)) & 1) : (spb ? (uint32_t)((pbits >> s) & 1) : 0u);
      const uint32_t p1 = epb ? (uint32_t)((pbits >> (2 * s + 1)) & 1) : p0;
      const int sh0 = 2 * s * cb, sh1 = sh0 + cb;
      uint32_t v0[3], v1[3];
      const uint32_t f3[3] = {fr, fg, fb};
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const uint32_t c0 = ((f3[c] >> sh0) & cm) << hp | (p0 & hp), c1 = ((f3[c] >> sh1) & cm) << hp | (p1 & hp);
        v0[c] = (c0 << cl8) | (c0 >> cr8);
        v1[c] = (c1 << cl8) | (c1 >> cr8);
      }
      uint32_t a0 = 255u, a1 = 255u;
      if (ab) {
        const uint32_t c0 = ((fa >> (2 * s * ab)) & amk) << epb | (p0 & epb), c1 = ((fa >> ((2 * s + 1) * ab)) & amk) << epb | (p1 & epb);
        a0 = (c0 << al8) | (c0 >> ar8);
        a1 = (c1 << al8) | (c1 >> ar8);
      }
      // (64 - w) E0 + w E1 + bias = (64 E0 + bias) + w (E1 - E0) modulo 2^32, and the true value of
      // each 16-bit lane stays below 2^16, so base + w * diff gives the same 32 bits in one multiply-add
      const uint32_t e0rg = (v0[0] | (v0[1] << 16)) << 2, e0ba = (v0[2] | (a0 << 16)) << 2;
      const uint32_t e1rg = (v1[0] | (v1[1] << 16)) << 2, e1ba = (v1[2] | (a1 << 16)) << 2;
      ep[s] = make_uint4(64u * e0rg + 0x00800080u, e1rg - e0rg, 64u * e0ba + 0x00800080u, e1ba - e0ba);
    }
  }
  // index streams at a fixed width per texel (anchor texels: texel 0, and a1, a2 in the primary)
  uint64_t pa = ins0(shr128(lo, hi, istart), ib - 1);
  const int alo = min(a1, a2), ahi = max(a1, a2);
  if (alo < 16) pa = ins0(pa, alo * ib + ib - 1);
  if (ahi < 16) pa = ins0(pa, ahi * ib + ib - 1);
  uint64_t sa = ib2 ? ins0(shr128(lo, hi, istart + 16 * ib - 1), ib2 - 1) : 0ull;
  const bool swap = ib2 && isbv;  // mode 4 with the index selection bit: colour from the 3-bit stream
  const uint64_t cs = swap ? sa : pa, as = swap ? pa : sa;
  const int cbits = swap ? ib2 : ib, abits = ib2 ? (swap ? ib : ib2) : 0;
  const uint32_t cmask = (1u << cbits) - 1u, amask = (1u << abits) - 1u;
  const uint8_t* wc = S->wt + (cbits - 2) * 16;
  const uint8_t* wa = S->wt + (abits ? abits - 2 : 0) * 16;
  // rotation: the alpha result (byte 3 of `al`, operand byte 7) replaces channel rot - 1
  const uint32_t rsel = rot == 0 ? 0x3210u : (rot == 1 ? 0x3217u : (rot == 2 ? 0x3270u : 0x3710u));
  // the reserved mode (first byte 0) decodes to 0: zero endpoints give exactly that below
  if (!b0) ep[0] = ep[1] = ep[2] = make_uint4(0x00800080u, 0u, 0x00800080u, 0u);
  // both streams as 32-bit halves, advanced by funnel shifts (widths are at most 4 bits)
  uint32_t cl = (uint32_t)cs, ch = (uint32_t)(cs >> 32), al32 = (uint32_t)as, ah = (uint32_t)(as >> 32);
#pragma unroll
  for (int t = 0; t < 16; t++) {
    const uint32_t ci = cl & cmask, ai = al32 & amask;
    cl = __funnelshift_r(cl, ch, cbits);
    ch >>= cbits;
    al32 = __funnelshift_r(al32, ah, abits);
    ah >>= abits;
    const uint4 e = ep[(pm >> (2 * t)) & 3];  // (base rg, diff rg, base ba, diff ba)
    const uint32_t cw = wc[ci], aw = wa[ai];
    const uint32_t rg = cw * e.y + e.x;
    const uint32_t ba = cw * e.w + e.z;
    const uint32_t al = aw * e.w + e.z;
    tx[t] = __byte_perm(__byte_perm(rg, ba, 0x0531u), al, rsel);
  }
}

// 2^23 + q as float for byte c of v (0x4B0000qq)
__device__ __forceinline__ float u23(uint32_t v, int c) {
  return __uint_as_float(__byte_perm(v, 0x4B000000u, 0x7650u | (uint32_t)c));
}

// SH basis polynomials without their constants (the constants, with their signs, are folded
// into the per-coefficient dequantisation factors s_k / 255 * C_k), for two directions at once.
// The directions are unit vectors, so x^2 + y^2 + z^2 = 1 shortens the band-2 and band-3 terms:
// 2zz - xx - yy = 3zz - 1, 4zz - xx - yy = 5zz - 1, 2zz - 3xx - 3yy = 5zz - 3.
__device__ __forceinline__ void sh_poly2(float2 x, float2 y, float2 z, float2 (&P)[16]) {
  const float2 xx = __fmul2_rn(x, x), yy = __fmul2_rn(y, y), zz = __fmul2_rn(z, z);
  const float2 xy = __fmul2_rn(x, y), yz = __fmul2_rn(y, z), xz = __fmul2_rn(x, z);
  const float2 m1 = make_float2(-1.f, -1.f), five = make_float2(5.f, 5.f);
  const float2 xmy = __ffma2_rn(yy, m1, xx);                                        // xx - yy
  const float2 t5 = __ffma2_rn(five, zz, m1);                                        // 5zz - 1
  P[0] = make_float2(1.f, 1.f);
  P[1] = y; P[2] = z; P[3] = x;
  P[4] = xy; P[5] = yz; P[6] = __ffma2_rn(make_float2(3.f, 3.f), zz, m1); P[7] = xz; P[8] = xmy;  // 3zz - 1
  P[9] = __fmul2_rn(y, __ffma2_rn(make_float2(3.f, 3.f), xx, make_float2(-yy.x, -yy.y)));      // y (3xx - yy)
  P[10] = __fmul2_rn(xy, z);
  P[11] = __fmul2_rn(y, t5);
  P[12] = __fmul2_rn(z, __ffma2_rn(five, zz, make_float2(-3.f, -3.f)));                 // z (5zz - 3)
  P[13] = __fmul2_rn(x, t5);
  P[14] = __fmul2_rn(z, xmy);
  P[15] = __fmul2_rn(x, __ffma2_rn(make_float2(-3.f, -3.f), yy, xx));                  // x (xx - 3yy)
}

static __constant__ float c_shc[16] = {SH_C0, -SH_C1, SH_C1, -SH_C1, SH_C2A, -SH_C2A, SH_C2B, -SH_C2A, SH_C2C,
                                -SH_C3A, SH_C3B, -SH_C3C, SH_C3D, -SH_C3C, SH_C3E, -SH_C3A};

