// bc1_dev.cuh -- BC1 encoder device code (Sec. III-A with P = 16, Q = 2; Sec. III-B), shared
// by the single-scene kernels (bc1.cu) and the persistent multi-scene kernel (bc7.cu).
#pragma once
#include "gsc_internal.cuh"
#include "stage.cuh"

// Per channel value: best (a, b) code pair for a constant block, packed a | b << 8. Each
// translation unit that includes this header has its own copy, filled at context creation
// from bc1_const_tables().
static __constant__ uint16_t c_const5[256];
static __constant__ uint16_t c_const6[256];
void bc1_const_tables(uint16_t* t5, uint16_t* t6);

__device__ __forceinline__ int ex5(int x) { return (x << 3) | (x >> 2); }
__device__ __forceinline__ int ex6(int x) { return (x << 2) | (x >> 4); }
// Interior entries: measured GB300 texture-unit rule (5-bit on codes, 6-bit on expansions).
__device__ __forceinline__ int third5(int a, int b) { return ((2 * a + b) * 11) >> 2; }
__device__ __forceinline__ int third6(int a, int b) {
  int A = ex6(a), B = ex6(b);
  return A + (((B - A) * 321 + 512) >> 10);
}

struct Bc1Res {
  uint32_t sse;
  uint32_t idx;   // 2 bits per texel
  uint16_t c0, c1;
};

__device__ __forceinline__ Bc1Res bc1_eval(const uint32_t (&tx)[16], uint32_t a, uint32_t b) {
  Bc1Res r;
  r.c0 = (uint16_t)max(a, b);
  r.c1 = (uint16_t)min(a, b);
  r.sse = 0;
  r.idx = 0;
  const int ra = r.c0 >> 11, ga = (r.c0 >> 5) & 63, ba = r.c0 & 31;
  const int rb = r.c1 >> 11, gb = (r.c1 >> 5) & 63, bb = r.c1 & 31;
  const int p0r = ex5(ra), p0g = ex6(ga), p0b = ex5(ba);
  if (r.c0 == r.c1) {
#pragma unroll
    for (int t = 0; t < 16; t++) {
      int dr = tex_r(tx[t]) - p0r, dg = tex_g(tx[t]) - p0g, db = tex_b(tx[t]) - p0b;
      r.sse += dr * dr + dg * dg + db * db;
    }
    return r;
  }
  const int p1r = ex5(rb), p1g = ex6(gb), p1b = ex5(bb);
  const int p2r = third5(ra, rb), p2g = third6(ga, gb), p2b = third5(ba, bb);
  const int p3r = third5(rb, ra), p3g = third6(gb, ga), p3b = third5(bb, ba);
#pragma unroll
  for (int t = 0; t < 16; t++) {
    const int vr = tex_r(tx[t]), vg = tex_g(tx[t]), vb = tex_b(tx[t]);
    int d, best, j = 0;
    d = vr - p0r; best = d * d; d = vg - p0g; best += d * d; d = vb - p0b; best += d * d;
    int e1, e2, e3;
    d = vr - p1r; e1 = d * d; d = vg - p1g; e1 += d * d; d = vb - p1b; e1 += d * d;
    d = vr - p2r; e2 = d * d; d = vg - p2g; e2 += d * d; d = vb - p2b; e2 += d * d;
    d = vr - p3r; e3 = d * d; d = vg - p3g; e3 += d * d; d = vb - p3b; e3 += d * d;
    if (e1 < best) { best = e1; j = 1; }
    if (e2 < best) { best = e2; j = 2; }
    if (e3 < best) { best = e3; j = 3; }
    r.sse += best;
    r.idx |= (uint32_t)j << (2 * t);
  }
  return r;
}

// The error of a candidate pair alone (no indices): sumsq is the block's summed squared texel
// norms, and each texel adds min_j (|p_j|^2 - 2 v.p_j) over the palette (one entry when the two
// endpoints are equal), the same integer as bc1_eval's error.
__device__ __forceinline__ uint32_t bc1_sse(const uint32_t (&tx)[16], int sumsq, uint32_t a, uint32_t b) {
  const uint32_t c0 = max(a, b), c1 = min(a, b);
  const int ra = c0 >> 11, ga = (c0 >> 5) & 63, ba = c0 & 31;
  const int rb = c1 >> 11, gb = (c1 >> 5) & 63, bb = c1 & 31;
  const uint32_t P0 = (uint32_t)ex5(ra) | ((uint32_t)ex6(ga) << 8) | ((uint32_t)ex5(ba) << 16);
  const int k0 = (int)__dp4a(P0, P0, 0u);
  int s = 0;
  if (c0 == c1) {
#pragma unroll
    for (int t = 0; t < 16; t++) s += k0 - 2 * (int)__dp4a(tx[t], P0, 0u);
    return (uint32_t)(sumsq + s);
  }
  const uint32_t P1 = (uint32_t)ex5(rb) | ((uint32_t)ex6(gb) << 8) | ((uint32_t)ex5(bb) << 16);
  const uint32_t P2 = (uint32_t)third5(ra, rb) | ((uint32_t)third6(ga, gb) << 8) | ((uint32_t)third5(ba, bb) << 16);
  const uint32_t P3 = (uint32_t)third5(rb, ra) | ((uint32_t)third6(gb, ga) << 8) | ((uint32_t)third5(bb, ba) << 16);
  const int k1 = (int)__dp4a(P1, P1, 0u), k2 = (int)__dp4a(P2, P2, 0u), k3 = (int)__dp4a(P3, P3, 0u);
#pragma unroll
  for (int t = 0; t < 16; t++) {
    const uint32_t v = tx[t];
    const int e0 = k0 - 2 * (int)__dp4a(v, P0, 0u), e1 = k1 - 2 * (int)__dp4a(v, P1, 0u);
    const int e2 = k2 - 2 * (int)__dp4a(v, P2, 0u), e3 = k3 - 2 * (int)__dp4a(v, P3, 0u);
    s += min(min(e0, e1), min(e2, e3));
  }
  return (uint32_t)(sumsq + s);
}

// bc1_eval from byte dot products: key 4 (|p_j|^2 - 2 v.p_j) + j, whose minimum gives the first
// entry of least error (j = key & 3) and the error above the texel's squared norm (key >> 2).
__device__ __forceinline__ Bc1Res bc1_eval_k(const uint32_t (&tx)[16], int sumsq, uint32_t a, uint32_t b) {
  Bc1Res r;
  r.c0 = (uint16_t)max(a, b);
  r.c1 = (uint16_t)min(a, b);
  r.idx = 0;
  const int ra = r.c0 >> 11, ga = (r.c0 >> 5) & 63, ba = r.c0 & 31;
  const int rb = r.c1 >> 11, gb = (r.c1 >> 5) & 63, bb = r.c1 & 31;
  const uint32_t P0 = (uint32_t)ex5(ra) | ((uint32_t)ex6(ga) << 8) | ((uint32_t)ex5(ba) << 16);
  const int k0 = (int)__dp4a(P0, P0, 0u);
  int s = 0;
  if (r.c0 == r.c1) {
#pragma unroll
    for (int t = 0; t < 16; t++) s += k0 - 2 * (int)__dp4a(tx[t], P0, 0u);
    r.sse = (uint32_t)(sumsq + s);
    return r;
  }
  const uint32_t P1 = (uint32_t)ex5(rb) | ((uint32_t)ex6(gb) << 8) | ((uint32_t)ex5(bb) << 16);
  const uint32_t P2 = (uint32_t)third5(ra, rb) | ((uint32_t)third6(ga, gb) << 8) | ((uint32_t)third5(ba, bb) << 16);
  const uint32_t P3 = (uint32_t)third5(rb, ra) | ((uint32_t)third6(gb, ga) << 8) | ((uint32_t)third5(bb, ba) << 16);
  const int q0 = 4 * k0, q1 = 4 * (int)__dp4a(P1, P1, 0u) + 1;
  const int q2 = 4 * (int)__dp4a(P2, P2, 0u) + 2, q3 = 4 * (int)__dp4a(P3, P3, 0u) + 3;
#pragma unroll
  for (int t = 0; t < 16; t++) {
    const uint32_t v = tx[t];
    const int e0 = q0 - 8 * (int)__dp4a(v, P0, 0u), e1 = q1 - 8 * (int)__dp4a(v, P1, 0u);
    const int e2 = q2 - 8 * (int)__dp4a(v, P2, 0u), e3 = q3 - 8 * (int)__dp4a(v, P3, 0u);
    const int key = min(min(e0, e1), min(e2, e3));
    s += key >> 2;
    r.idx |= (uint32_t)(key & 3) << (2 * t);
  }
  r.sse = (uint32_t)(sumsq + s);
  return r;
}

__device__ __forceinline__ int q5(int v) { return (v * 31 + 127) / 255; }
__device__ __forceinline__ int q6(int v) { return (v * 63 + 127) / 255; }
__device__ __forceinline__ uint32_t pack565(int r, int g, int b) { return (q5(r) << 11) | (q6(g) << 5) | q5(b); }

// Encodes one block; returns the palette choice and writes sse0 (error of texel 128) if asked.
__device__ __forceinline__ Bc1Res bc1_encode(const uint32_t (&tx)[16]) {
  bool constant = true;
#pragma unroll
  for (int t = 1; t < 16; t++) constant &= (tx[t] == tx[0]);
  if (constant) {
    uint32_t pr = c_const5[tex_r(tx[0])], pg = c_const6[tex_g(tx[0])], pb = c_const5[tex_b(tx[0])];
    uint32_t c0 = ((pr & 255) << 11) | ((pg & 255) << 5) | (pb & 255);
    uint32_t c1 = ((pr >> 8) << 11) | ((pg >> 8) << 5) | (pb >> 8);
    return bc1_eval(tx, c0, c1);
  }
  int lo[3] = {255, 255, 255}, hi[3] = {0, 0, 0}, s1[3] = {0, 0, 0};
  int s2rg = 0, s2rb = 0, s2gb = 0;
#pragma unroll
  for (int t = 0; t < 16; t++) {
    int v[3] = {tex_r(tx[t]), tex_g(tx[t]), tex_b(tx[t])};
#pragma unroll
    for (int c = 0; c < 3; c++) { lo[c] = min(lo[c], v[c]); hi[c] = max(hi[c], v[c]); s1[c] += v[c]; }
    s2rg += v[0] * v[1]; s2rb += v[0] * v[2]; s2gb += v[1] * v[2];
  }
  int ref = 0;
  if (hi[1] - lo[1] > hi[ref] - lo[ref]) ref = 1;
  if (hi[2] - lo[2] > hi[ref] - lo[ref]) ref = 2;
  // covariance of the reference channel with each other channel (scaled by 16)
  int cov[3];
  cov[0] = ref == 1 ? 16 * s2rg - s1[1] * s1[0] : (ref == 2 ? 16 * s2rb - s1[2] * s1[0] : 0);
  cov[1] = ref == 0 ? 16 * s2rg - s1[0] * s1[1] : (ref == 2 ? 16 * s2gb - s1[2] * s1[1] : 0);
  cov[2] = ref == 0 ? 16 * s2rb - s1[0] * s1[2] : (ref == 1 ? 16 * s2gb - s1[1] * s1[2] : 0);
  int e0[3], e1[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    bool flip = (c != ref) && cov[c] < 0;
    e0[c] = flip ? lo[c] : hi[c];
    e1[c] = flip ? hi[c] : lo[c];
    int d = (hi[c] - lo[c]) >> 4;
    if (e0[c] >= e1[c]) { e0[c] -= d; e1[c] += d; } else { e0[c] += d; e1[c] -= d; }
  }
  int sumsq = 0;
#pragma unroll
  for (int t = 0; t < 16; t++) sumsq += (int)__dp4a(tx[t] & 0xFFFFFFu, tx[t] & 0xFFFFFFu, 0u);
  Bc1Res best = bc1_eval_k(tx, sumsq, pack565(e0[0], e0[1], e0[2]), pack565(e1[0], e1[1], e1[2]));
  // two least-squares refinements: weights (3,0,2,1)/3 on c0 for indices 0..3
  for (int it = 0; it < 2; it++) {
    if (best.c0 == best.c1) break;
    int saa = 0, sbb = 0, sab = 0, sav[3] = {0, 0, 0}, sbv[3] = {0, 0, 0};
#pragma unroll
    for (int t = 0; t < 16; t++) {
      int j = (best.idx >> (2 * t)) & 3;
      int a = (0x1203 >> (4 * j)) & 15;  // j: 0 -> 3, 1 -> 0, 2 -> 2, 3 -> 1
      int b = 3 - a;
      saa += a * a; sbb += b * b; sab += a * b;
      int v[3] = {tex_r(tx[t]), tex_g(tx[t]), tex_b(tx[t])};
#pragma unroll
      for (int c = 0; c < 3; c++) { sav[c] += a * v[c]; sbv[c] += b * v[c]; }
    }
    int det = saa * sbb - sab * sab;
    if (det == 0) break;
    const RoundDiv255 rd = round_div255_of(det);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      e0[c] = round_div255(rd, 3LL * (sbb * sav[c] - sab * sbv[c]));
      e1[c] = round_div255(rd, 3LL * (saa * sbv[c] - sab * sav[c]));
    }
    Bc1Res r = bc1_eval_k(tx, sumsq, pack565(e0[0], e0[1], e0[2]), pack565(e1[0], e1[1], e1[2]));
    if (r.sse < best.sse) best = r; else break;
  }
  // +-1 neighbourhood, order: endpoint (c0, c1) x channel (R, G, B) x step (+1, -1); one copy of
  // the candidate evaluation in a rolled loop keeps the code small enough for the instruction cache.
  // Candidates are compared by error alone; the chosen pair's indices are computed at the end.
  uint32_t bc0 = best.c0, bc1 = best.c1, bsse = best.sse;
  bool moved = false;
  for (int round = 0; round < 4; round++) {
    uint32_t nsse = 0xFFFFFFFFu, n0 = 0, n1 = 0;
    bool found = false;
#pragma unroll 1
    for (int q = 0; q < 12; q++) {
      const int ep = q / 6, c = (q / 2) % 3, sgn = q & 1;
      const int shift = c == 0 ? 11 : (c == 1 ? 5 : 0), mask = c == 1 ? 63 : 31;
      uint32_t cc0 = bc0, cc1 = bc1;
      uint32_t cur = ep ? cc1 : cc0;
      int v = (int)((cur >> shift) & mask) + (sgn ? -1 : 1);
      if (v < 0 || v > mask) continue;
      cur = (cur & ~((uint32_t)mask << shift)) | ((uint32_t)v << shift);
      if (ep) cc1 = cur; else cc0 = cur;
      const uint32_t e = bc1_sse(tx, sumsq, cc0, cc1);
      if (!found || e < nsse) { nsse = e; n0 = max(cc0, cc1); n1 = min(cc0, cc1); found = true; }
    }
    if (found && nsse < bsse) { bsse = nsse; bc0 = n0; bc1 = n1; moved = true; } else break;
  }
  return moved ? bc1_eval_k(tx, sumsq, bc0, bc1) : best;
}

__device__ __forceinline__ uint2 bc1_bits(const Bc1Res& r) {
  return make_uint2((uint32_t)r.c0 | ((uint32_t)r.c1 << 16), r.idx);
}

__device__ __forceinline__ uint32_t sse_zero(const uint32_t (&tx)[16]) {
  uint32_t s = 0;
#pragma unroll
  for (int t = 0; t < 16; t++) {
    int dr = tex_r(tx[t]) - 128, dg = tex_g(tx[t]) - 128, db = tex_b(tx[t]) - 128;
    s += dr * dr + dg * dg + db * db;
  }
  return s;
}

