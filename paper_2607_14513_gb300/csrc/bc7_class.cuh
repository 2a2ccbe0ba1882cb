// bc7_class.cuh -- BC7 block decoders specialised per mode at compile time (Sec. III-B; the
// D3D11 / Khronos BC7 format): field positions, widths, subset and index counts are constants,
// so a warp that decodes 32 blocks of one mode runs straight-line code.
#pragma once
#include "decode_dev.cuh"

enum { CL_M4S = 8, CL_RES = 9, CL_BC1 = 10, CL_DROP = 11 };

// ---- class decoders ---------------------------------------------------------------------------
// bits [C, C + 64) of the 128-bit block, C a compile-time constant
template <int C>
__device__ __forceinline__ uint64_t shr128c(uint64_t lo, uint64_t hi) {
  if (C == 0) return lo;
  if (C >= 64) return hi >> (C >= 64 ? C - 64 : 0);
  return (lo >> (C & 63)) | (hi << ((64 - C) & 63));
}

// BC7 index weight for index i of a `bits`-wide index: the 2- and 3-bit tables are byte
// permutes of constants (index 0 weighs 0, so the upper bytes of the permute are 0).
template <int BITS>
__device__ __forceinline__ uint32_t wgt_of(uint32_t i, const DecTables* S) {
  if (BITS == 2) return __byte_perm(0x402B1500u, 0u, i);
  if (BITS == 3) return __byte_perm(0x1B120900u, 0x40372E25u, i);
  return S->wt[32 + i];
}

// A zero bit inserted at position p of a 32-bit stream (ins0 for streams that fit 32 bits).
__device__ __forceinline__ uint32_t ins0_32(uint32_t x, int p) {
  const uint32_t m = (1u << p) - 1u;
  return (x & m) | ((x & ~m) << 1);
}

// 8 two-bit fields (bits 0..15 of x) into the low two bits of 8 nibbles
__device__ __forceinline__ uint32_t spread2to4(uint32_t x) {
  x &= 0xFFFFu;
  x = (x | (x << 8)) & 0x00FF00FFu;
  x = (x | (x << 4)) & 0x0F0F0F0Fu;
  return (x | (x << 2)) & 0x33333333u;
}

// Endpoint pair of one subset as 4x-scaled 16-bit lanes: (lo | hi << 16) << 2 of the 8-bit
// expansions (v << (8 - n)) | (v >> (2n - 8)) of n-bit values lo, hi (n = field bits + p-bit).
template <int N>
__device__ __forceinline__ uint32_t expand_pair4(uint32_t y) {  // y = lo | hi << 16, n-bit lanes
  static_assert(N >= 5 && N <= 8, "BC7 endpoint widths with p-bits are 5..8 bits");
  if (N >= 8) return y << 2;
  constexpr uint32_t lowbits = (1u << (8 - N)) - 1u;  // bits the right shift contributes
  constexpr uint32_t mask = (lowbits | (lowbits << 16)) << 2;
  return (y << (10 - N)) | ((y >> (2 * N - 10)) & mask);
}

// One BC7 block of class CL (mode CL, or mode 4 with the index-selection bit set) into 16
// texels r | g << 8 | b << 16 (alpha byte unspecified). The arithmetic is that of bc7_block in
// decode_dev.cuh: endpoints as 4x-scaled 16-bit lanes so that ((64 - w) e0 + w e1 + 32) >> 6 of
// two channels is one multiply-add, index streams re-spaced to a fixed width per texel.
// Multi-subset modes with 2-bit indices (2, 3, 7) first interpolate every (subset, index) pair
// into a palette in this lane's shared slot `ep` (64 bytes, 64-byte aligned) and then look each
// texel up by a 4-bit key (subset << 2 | index) built for all 16 texels at once.
template <int CL>
__device__ __forceinline__ void bc7_class_block(uint64_t lo, uint64_t hi, uint32_t (&tx)[16], const DecTables* S,
                                                uint4* ep) {
  constexpr int mode = CL == CL_M4S ? 4 : CL;
  constexpr DModeInfo D = d_mode_info(mode);
  constexpr int ns = D.ns, pb = D.pb, rb = D.rb, isb = D.isb, cb = D.cb, ab = D.ab, epb = D.epb, spb = D.spb;
  constexpr int ib = D.ib, ib2 = D.ib2;
  constexpr bool swap = CL == CL_M4S;  // colour indices from the 3-bit stream
  constexpr bool palette = ns > 1 && ib == 2;
  constexpr int hp = epb | spb, nb = cb + hp, na = ab + epb;
  constexpr int pos0 = mode + 1;
  constexpr int cstart = pos0 + pb + rb + isb, astart = cstart + 6 * ns * cb, pstart = astart + 2 * ns * ab;
  constexpr int istart = pstart + (epb ? 2 * ns : (spb ? ns : 0));
  const uint32_t w0 = (uint32_t)lo;
  const int part = pb ? (int)((w0 >> pos0) & ((1u << pb) - 1u)) : 0;
  const int rot = rb ? (int)((w0 >> (pos0 + pb)) & 3u) : 0;
  uint32_t pm = 0u;
  int a1 = 16, a2 = 16;
  if (ns == 2) { pm = S->part2[part]; a1 = S->anc2[part]; }
  if (ns == 3) { pm = S->part3[part]; a1 = S->anc3a[part]; a2 = S->anc3b[part]; }
  const uint32_t pbits = (uint32_t)shr128c<pstart>(lo, hi);
  const uint32_t fr = (uint32_t)shr128c<cstart>(lo, hi), fg = (uint32_t)shr128c<cstart + 2 * ns * cb>(lo, hi);
  const uint32_t fb = (uint32_t)shr128c<cstart + 4 * ns * cb>(lo, hi);
  const uint32_t fa = ab ? (uint32_t)shr128c<astart>(lo, hi) : 0u;
  constexpr uint32_t cm = (1u << cb) - 1u, amk = ab ? (1u << ab) - 1u : 0u;
  uint4 e_one = make_uint4(0u, 0u, 0u, 0u);
  uint32_t* pal = reinterpret_cast<uint32_t*>(ep);
  // lanes 2i and 2i + 1 hold their 16-word palettes in opposite bank halves; XOR-ing the entry
  // index with i spreads equal entries of all 32 lanes over distinct banks
  const int sw = (int)((threadIdx.x >> 1) & 15u);
  // endpoint slots of multi-subset blocks (16 bytes each): slot s at s ^ sw4, the same spread
  const int sw4 = sw & 3;
#pragma unroll
  for (int s = 0; s < ns; s++) {
    const uint32_t p0 = epb ? ((pbits >> (2 * s)) & 1u) : (spb ? ((pbits >> s) & 1u) : 0u);
    const uint32_t p1 = epb ? ((pbits >> (2 * s + 1)) & 1u) : p0;
    const int sh0 = 2 * s * cb, sh1 = sh0 + cb;
    // (r | g << 16) and (b | a << 16) of both endpoints at field width, p-bits appended
    const uint32_t rg0 = ((((fr >> sh0) & cm) | (((fg >> sh0) & cm) << 16)) << hp) | (hp ? p0 * 0x10001u : 0u);
    const uint32_t rg1 = ((((fr >> sh1) & cm) | (((fg >> sh1) & cm) << 16)) << hp) | (hp ? p1 * 0x10001u : 0u);
    const uint32_t b0 = (((fb >> sh0) & cm) << hp) | (hp ? p0 : 0u), b1 = (((fb >> sh1) & cm) << hp) | (hp ? p1 : 0u);
    uint32_t e0rg = expand_pair4<nb>(rg0), e1rg = expand_pair4<nb>(rg1);
    uint32_t e0ba, e1ba;
    if constexpr (ab != 0) {
      const uint32_t a0 = (((fa >> (2 * s * ab)) & amk) << epb) | (epb ? p0 : 0u);
      const uint32_t a1v = (((fa >> ((2 * s + 1) * ab)) & amk) << epb) | (epb ? p1 : 0u);
      // colour and alpha widths differ: expand the two lanes separately
      e0ba = expand_pair4<nb>(b0) | (expand_pair4<(ab ? na : 8)>(a0) << 16);
      e1ba = expand_pair4<nb>(b1) | (expand_pair4<(ab ? na : 8)>(a1v) << 16);
    } else {
      e0ba = expand_pair4<nb>(b0) | (255u << 18);
      e1ba = expand_pair4<nb>(b1) | (255u << 18);
    }
    const uint4 e = make_uint4(64u * e0rg + 0x00800080u, e1rg - e0rg, 64u * e0ba + 0x00800080u, e1ba - e0ba);
    if (ns == 1) {
      e_one = e;
    } else if (palette) {
      // weights 0, 21, 43, 64 of the 2-bit index; entry j at word j ^ sw (bank spread across lanes)
      pal[(4 * s + 0) ^ sw] = __byte_perm(e.x, e.z, 0x0531u);
      pal[(4 * s + 1) ^ sw] = __byte_perm(21u * e.y + e.x, 21u * e.w + e.z, 0x0531u);
      pal[(4 * s + 2) ^ sw] = __byte_perm(43u * e.y + e.x, 43u * e.w + e.z, 0x0531u);
      pal[(4 * s + 3) ^ sw] = __byte_perm(64u * e.y + e.x, 64u * e.w + e.z, 0x0531u);
    } else {
      ep[s ^ sw4] = e;
    }
  }
  if (palette) {
    // primary stream re-spaced to 2 bits per texel (anchors: texel 0, a1, a2), then keys
    uint32_t ps = ins0_32((uint32_t)shr128c<istart>(lo, hi), 1);
    if (ns == 2) ps = ins0_32(ps, 2 * a1 + 1);
    if (ns == 3) {
      const int alo = min(a1, a2), ahi = max(a1, a2);
      ps = ins0_32(ps, 2 * alo + 1);
      ps = ins0_32(ps, 2 * ahi + 1);
    }
    const uint32_t klo = spread2to4(ps) | (spread2to4(pm) << 2);
    const uint32_t khi = spread2to4(ps >> 16) | (spread2to4(pm >> 16) << 2);
    // (key << 2 & 0x3C) ^ (sw << 2 | base) = base | ((key ^ sw) << 2): the slot is 64-byte aligned
    const uint32_t swb = (uint32_t)__cvta_generic_to_shared(pal) | ((uint32_t)sw << 2);
#pragma unroll
    for (int t = 0; t < 16; t++) {
      const uint32_t kw = t < 8 ? klo : khi;
      const int j = t & 7;
      const uint32_t off = ((j == 0 ? (kw << 2) : (kw >> (4 * j - 2))) & 0x3Cu) ^ swb;
      uint32_t v;
      asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(off) : "memory");
      tx[t] = v;
    }
    return;
  }
  // index streams at a fixed width per texel (anchors: texel 0, a1 and a2 in the primary stream)
  uint64_t pa = ins0(shr128c<istart>(lo, hi), ib - 1);
  if (ns == 2) pa = ins0(pa, a1 * ib + ib - 1);
  if (ns == 3) {
    const int alo = min(a1, a2), ahi = max(a1, a2);
    pa = ins0(pa, alo * ib + ib - 1);
    pa = ins0(pa, ahi * ib + ib - 1);
  }
  uint64_t sa = 0ull;
  if (ib2) sa = ins0(shr128c<(ib2 ? istart + 16 * ib - 1 : 0)>(lo, hi), (ib2 ? ib2 : 1) - 1);
  constexpr int cbits = swap ? ib2 : ib, abits = ib2 ? (swap ? ib : ib2) : 2;
  const uint64_t cs = swap ? sa : pa, as = swap ? pa : sa;
  // rotation: the alpha-index interpolation (byte 3 of `al`, operand byte 7) replaces channel rot - 1
  const uint32_t rsel = rot == 0 ? 0x3210u : (rot == 1 ? 0x3217u : (rot == 2 ? 0x3270u : 0x3710u));
#pragma unroll
  for (int t = 0; t < 16; t++) {
    const uint32_t ci = (uint32_t)(cs >> (cbits * t)) & ((1u << cbits) - 1u);
    const uint32_t cw = wgt_of<cbits>(ci, S);
    uint4 e = e_one;
    if (ns > 1) {
      const uint32_t sh = t == 0 ? (pm << 4) : (t == 1 ? (pm << 2) : (pm >> (2 * t - 4)));
      const uint32_t eo = (sh & 0x30u) ^ ((uint32_t)__cvta_generic_to_shared(ep) | ((uint32_t)sw4 << 4));
      asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(e.x), "=r"(e.y), "=r"(e.z), "=r"(e.w) : "r"(eo) : "memory");
    }
    const uint32_t rg = cw * e.y + e.x, ba = cw * e.w + e.z;
    uint32_t px = __byte_perm(rg, ba, 0x0531u);
    if (rb) {
      const uint32_t ai = (uint32_t)(as >> (abits * t)) & ((1u << abits) - 1u);
      const uint32_t al = wgt_of<abits>(ai, S) * e.w + e.z;
      px = __byte_perm(px, al, rsel);
    }
    tx[t] = px;
  }
}

// One BC1 block into 16 texels r | g << 8 | b << 16 | a << 24 (bc1_block's values): the four
// palette entries go to this lane's shared slot `ep` (64 bytes, 64-byte aligned) and every texel
// is looked up by its index.
__device__ __forceinline__ void bc1_class_block(uint2 w, uint32_t (&tx)[16], uint4* ep) {
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
  // entry j at word j ^ sw of the 16-word slot (bank spread across lanes, as in bc7_class_block)
  const int sw = (int)((threadIdx.x >> 1) & 15u);
  uint32_t* pal = reinterpret_cast<uint32_t*>(ep);
  pal[0 ^ sw] = p0; pal[1 ^ sw] = p1; pal[2 ^ sw] = p2; pal[3 ^ sw] = p3;
  const uint32_t swb = (uint32_t)__cvta_generic_to_shared(pal) | ((uint32_t)sw << 2);
#pragma unroll
  for (int t = 0; t < 16; t++) {
    const uint32_t off = ((t == 0 ? (w.y << 2) : (t == 1 ? w.y : (w.y >> (2 * t - 2)))) & 0xCu) ^ swb;
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(off) : "memory");
    tx[t] = v;
  }
}
