/*
 * gsc_oracle.c -- plain, slow, scalar CPU oracle for block texture coding of
 * 3DGS spherical-harmonic colour coefficients (Said & Rauwendaal, "Compression of
 * 3D Gaussian Splatting Data Using GPU-friendly Graphics Texture Coding").
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg may load it. It shares no code, header, table or constant
 * generator with the CUDA library, and it is compiled with -ffp-contract=off so
 * that every float operation rounds exactly once.
 *
 * What follows the paper and what is this codec's own reading:
 *  - Sec. V-A: 16 per-scene scale factors so that 99.5% of the coefficients
 *    normalise into [-0.5, 0.5], then 8-bit quantisation. Reading: one scale per
 *    coefficient index k, pooled over R, G, B and all Gaussians, zero-centred.
 *  - Sec. III-C and Sec. V-A: sort by 24-bit RGB bit interleave of the DC texel,
 *    done independently inside larger spatial groups. Reading: spatial groups are
 *    chunks of G consecutive Gaussians in 30-bit Morton order.
 *  - Sec. IV-B, Fig. SetupD: block k of a group holds coefficient k of 16 Gaussians.
 *    Fig. SetupA / SetupB (Table I's other rows): one Gaussian per block, or four
 *    Gaussians' coefficients 4b..4b+3 in block b of four; texel placement inside a
 *    block (raster order, row = Gaussian in B) is this codec's reading.
 *  - Sec. III-A/B: BTC, BC1, BC7 (D3D11 / Khronos BC7 format definitions). The paper
 *    uses a third-party encoder; the encoder here is the codec's own deterministic
 *    integer search (ties go to the lowest enumeration index).
 *  - Sec. IV-B and the abstract: several fixed-rate bitstreams give a variable rate
 *    with random access. The paper gives the mechanism; the integer Lagrangian
 *    choice between 14 group modes is the codec's own reading.
 *  - Sec. II, colour equation c(f) = H w(f - p): real SH to degree 3, evaluated here
 *    in double precision from the closed form.
 */
#include "gsc_oracle.h"

#include <pthread.h>

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Scales (Sec. V-A): s_k = 2 * a_k, a_k the r-th smallest |x| over the 3N     */
/* values of coefficient k, r = ceil(permille * 3N / 1000) - 1.              */
/* ------------------------------------------------------------------------- */
static int cmp_float(const void* a, const void* b) {
  float x = *(const float*)a, y = *(const float*)b;
  return (x > y) - (x < y);
}

/* Sec. V-A: the per-coefficient scale factors. */
int or_scales(const float* sh, int64_t n, uint32_t permille, float* scales) {
  if (permille == 0 || permille > 1000) return -1;
  if (n <= 0) {
    for (int k = 0; k < OR_SH; k++) scales[k] = 1.0f;
    return 0;
  }
  int64_t m = 3 * n;
  float* v = (float*)malloc(sizeof(float) * (size_t)m);
  if (!v) return -2;
  int64_t r = ((int64_t)permille * m + 999) / 1000 - 1;
  for (int k = 0; k < OR_SH; k++) {
    for (int64_t i = 0; i < n; i++)
      for (int c = 0; c < 3; c++) v[3 * i + c] = fabsf(sh[(i * OR_SH + k) * 3 + c]);
    qsort(v, (size_t)m, sizeof(float), cmp_float);
    float s = 2.0f * v[r];
    scales[k] = (s == 0.0f) ? 1.0f : s;
  }
  free(v);
  return 0;
}

/* Quantise (Sec. V-A): q = clamp(128 + rint(fl(fl(x / s) * 255)), 0, 255), round half to even. */
uint8_t or_quant1(float x, float s) {
  float t = x / s;
  t = t * 255.0f;
  if (t > 256.0f) t = 256.0f;
  if (t < -256.0f) t = -256.0f;
  long r = lrintf(t);
  long q = 128 + r;
  if (q < 0) q = 0;
  if (q > 255) q = 255;
  return (uint8_t)q;
}

/* Sec. V-A: 8-bit quantisation of the scaled coefficients. */
void or_quantise(const float* sh, int64_t n, const float* scales, uint8_t* q) {
  for (int64_t i = 0; i < n; i++)
    for (int k = 0; k < OR_SH; k++)
      for (int c = 0; c < 3; c++) q[(i * OR_SH + k) * 3 + c] = or_quant1(sh[(i * OR_SH + k) * 3 + c], scales[k]);
}

/* ------------------------------------------------------------------------- */
/* Reorder (Sec. III-C, Fig. Bit4Scan; Sec. V-A).                             */
/* ------------------------------------------------------------------------- */
uint32_t or_morton30(uint32_t x, uint32_t y, uint32_t z) {
  uint32_t m = 0;
  for (int i = 0; i < 10; i++) {
    m |= ((x >> i) & 1u) << (3 * i + 2);
    m |= ((y >> i) & 1u) << (3 * i + 1);
    m |= ((z >> i) & 1u) << (3 * i);
  }
  return m;
}

/* 24-bit key: bit i of R at 3i+2, of G at 3i+1, of B at 3i (Fig. Bit4Scan). */
uint32_t or_colour_key(uint32_t r, uint32_t g, uint32_t b) {
  uint32_t k = 0;
  for (int i = 0; i < 8; i++) {
    k |= ((r >> i) & 1u) << (3 * i + 2);
    k |= ((g >> i) & 1u) << (3 * i + 1);
    k |= ((b >> i) & 1u) << (3 * i);
  }
  return k;
}

typedef struct { uint64_t a, b, c; int64_t idx; } key3;
static int cmp_key3(const void* p, const void* q) {
  const key3* x = (const key3*)p; const key3* y = (const key3*)q;
  if (x->a != y->a) return x->a < y->a ? -1 : 1;
  if (x->b != y->b) return x->b < y->b ? -1 : 1;
  if (x->c != y->c) return x->c < y->c ? -1 : 1;
  return 0;
}

static uint32_t grid10(float p, float lo, float ext) {
  if (ext == 0.0f) return 0;
  float t = (p - lo) / ext;
  t = t * 1024.0f;
  float f = floorf(t);
  uint32_t u = (uint32_t)f;
  return u > 1023 ? 1023 : u;
}

/* Sec. III-C, Sec. V-A. perm[s] = original index of slot s; slots padded to a multiple of 16 with -1.
 * sort = 0 keeps the original order; sort = 1 sorts by (chunk, colour key, spatial rank),
 * chunk = spatial rank / group_size (group_size 0 = whole scene). */
int or_plan(const float* pos, const uint8_t* q, int64_t n, int64_t group_size, int sort, int32_t* perm) {
  if (group_size < 0 || group_size % 16 != 0) return -1;
  int64_t ns = (n + 15) / 16 * 16;
  for (int64_t s = 0; s < ns; s++) perm[s] = -1;
  if (n == 0) return 0;
  if (!sort) {
    for (int64_t i = 0; i < n; i++) perm[i] = (int32_t)i;
    return 0;
  }
  float lo[3], hi[3], ext[3];
  for (int a = 0; a < 3; a++) { lo[a] = pos[a]; hi[a] = pos[a]; }
  for (int64_t i = 0; i < n; i++)
    for (int a = 0; a < 3; a++) {
      float p = pos[3 * i + a];
      if (p < lo[a]) lo[a] = p;
      if (p > hi[a]) hi[a] = p;
    }
  for (int a = 0; a < 3; a++) ext[a] = hi[a] - lo[a];
  key3* k = (key3*)malloc(sizeof(key3) * (size_t)n);
  if (!k) return -2;
  /* spatial rank: stable sort by Morton code (original index breaks ties) */
  for (int64_t i = 0; i < n; i++) {
    uint32_t x = grid10(pos[3 * i + 0], lo[0], ext[0]);
    uint32_t y = grid10(pos[3 * i + 1], lo[1], ext[1]);
    uint32_t z = grid10(pos[3 * i + 2], lo[2], ext[2]);
    k[i].a = or_morton30(x, y, z); k[i].b = (uint64_t)i; k[i].c = 0; k[i].idx = i;
  }
  qsort(k, (size_t)n, sizeof(key3), cmp_key3);
  /* colour key inside chunks; the spatial rank breaks ties */
  for (int64_t r = 0; r < n; r++) {
    int64_t i = k[r].idx;
    const uint8_t* dc = &q[(i * OR_SH + 0) * 3];
    k[r].a = group_size ? (uint64_t)(r / group_size) : 0;
    k[r].b = or_colour_key(dc[0], dc[1], dc[2]);
    k[r].c = (uint64_t)r;
  }
  qsort(k, (size_t)n, sizeof(key3), cmp_key3);
  for (int64_t s = 0; s < n; s++) perm[s] = (int32_t)k[s].idx;
  free(k);
  return 0;
}

/* Layout D (Sec. IV-B, Fig. SetupD): block k of group g, texel t (raster order) =
 * coefficient k of the Gaussian in slot 16g + t. A padding slot repeats the last
 * valid slot of its group. */
void or_stage_group(const uint8_t* q, const int32_t* perm, int64_t g, uint8_t* tex) {
  int64_t last = -1;
  for (int t = 0; t < 16; t++) {
    int32_t o = perm[16 * g + t];
    if (o >= 0) last = o;
    for (int k = 0; k < OR_SH; k++)
      for (int c = 0; c < 3; c++) tex[(k * 16 + t) * 3 + c] = (last >= 0) ? q[(last * OR_SH + k) * 3 + c] : 128;
  }
}

/* ------------------------------------------------------------------------- */
/* Block layouts (Sec. IV-B). A group is slots 16g..16g+15 and 16 blocks of     */
/* 4 x 4 texels (texel t in raster order, row t / 4, column t % 4).             */
/*  D, Fig. SetupD: block k, texel t = coefficient k of slot t.                 */
/*  A, Fig. SetupA: one Gaussian per block: block k, texel t = coefficient t of */
/*     slot k.                                                                  */
/*  B, Fig. SetupB: four Gaussians in four blocks: the group is 4 quads of 4    */
/*     slots; block b of quad v (k = 4v + b), row i, column j holds coefficient */
/*     4b + j of slot 4v + i, so block 0 of a quad carries the first four       */
/*     coefficients (bands 0 and 1) of its Gaussians.                           */
/* ------------------------------------------------------------------------- */
void or_layout_map(int layout, int k, int t, int* u, int* c) {
  if (layout == OR_LAYOUT_A) { *u = k; *c = t; }
  else if (layout == OR_LAYOUT_B) {
    int v = k / 4, b = k % 4, i = t / 4, j = t % 4;
    *u = 4 * v + i; *c = 4 * b + j;
  } else { *u = t; *c = k; }
}

/* A fixed coding of a layout gives j of each group's 16 blocks to BC7 and the rest to
 * BC1 (Table I: BC7 on the first block of each quad in layout B, on block 0 in D). D: the
 * first j blocks; A: all or none; B: the first j / 4 blocks of every quad. */
int or_layout_ok(int layout, int j) {
  if (layout == OR_LAYOUT_D) return j >= 0 && j <= 16;
  if (layout == OR_LAYOUT_A) return j == 0 || j == 16;
  if (layout == OR_LAYOUT_B) return j >= 0 && j <= 16 && j % 4 == 0;
  return 0;
}

/* Sec. IV-B, Table I: whether block k of a layout's group is BC7 in a fixed mix. */
int or_layout_bc7(int layout, int j, int k) {
  if (layout == OR_LAYOUT_A) return j == 16;
  if (layout == OR_LAYOUT_B) return (k % 4) < j / 4;
  return k < j;
}

/* Sec. IV-B, Figs. SetupA/B/D.
 * Texels of group g in a layout: tex[k][t][c]. A padding slot repeats the last valid slot
 * before it in its group (128 if there is none), as in layout D. */
void or_stage_layout(const uint8_t* q, const int32_t* perm, int layout, int64_t g, uint8_t* tex) {
  int64_t src[16];
  int64_t last = -1;
  for (int u = 0; u < 16; u++) {
    if (perm[16 * g + u] >= 0) last = perm[16 * g + u];
    src[u] = last;
  }
  for (int k = 0; k < 16; k++)
    for (int t = 0; t < 16; t++) {
      int u, c;
      or_layout_map(layout, k, t, &u, &c);
      for (int ch = 0; ch < 3; ch++)
        tex[(k * 16 + t) * 3 + ch] = src[u] >= 0 ? q[(src[u] * OR_SH + c) * 3 + ch] : 128;
    }
}

/* ------------------------------------------------------------------------- */
/* Integer helpers                                                           */
/* ------------------------------------------------------------------------- */
static int64_t round_div(int64_t num, int64_t den) { /* den > 0, half away from zero */
  if (num >= 0) return (2 * num + den) / (2 * den);
  return -((-2 * num + den) / (2 * den));
}
static int clampi(int64_t v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : (int)v); }
static int sq(int v) { return v * v; }

/* ------------------------------------------------------------------------- */
/* BC1 (Sec. III-A with P = 16, Q = 2 on 4x4 blocks; D3D BC1 format).         */
/* ------------------------------------------------------------------------- */
static int ex5(int x) { return (x << 3) | (x >> 2); }
static int ex6(int x) { return (x << 2) | (x >> 4); }

static int floor_div(int num, int den) { /* den > 0 */
  return num >= 0 ? num / den : -((-num + den - 1) / den);
}

/* Interior palette entries. The BC1 definition leaves their rounding to a
 * tolerance; the reading here is the rule of the GB300 texture unit, measured over
 * every code pair of both bit depths and both modes and reproduced exactly by these
 * closed forms. a, b are channel codes (5 bits for R and B, 6 bits for G).
 * Four-colour mode, the entry two thirds of the way from b to a: */
static int bc1_third(int a, int b, int bits) {
  if (bits == 5) return ((2 * a + b) * 11) >> 2;
  int A = ex6(a), B = ex6(b);
  return A + floor_div((B - A) * 321 + 512, 1024);
}
/* Three-colour mode, the entry between c0's channel a and c1's channel b: */
static int bc1_half(int a, int b, int bits) {
  if (bits == 5) return ((a + b) * 33) >> 3;
  int A = ex6(a), B = ex6(b);
  return A + floor_div((B - A) * 257 + 256, 512);
}

/* Sec. III-A; BC1 format: the four-entry palette of two endpoints. */
void or_bc1_palette(uint16_t c0, uint16_t c1, uint8_t* pal) {
  int a[3] = {c0 >> 11, (c0 >> 5) & 63, c0 & 31};
  int b[3] = {c1 >> 11, (c1 >> 5) & 63, c1 & 31};
  for (int c = 0; c < 3; c++) {
    int bits = (c == 1) ? 6 : 5;
    pal[0 * 4 + c] = (uint8_t)(bits == 6 ? ex6(a[c]) : ex5(a[c]));
    pal[1 * 4 + c] = (uint8_t)(bits == 6 ? ex6(b[c]) : ex5(b[c]));
    if (c0 > c1) {
      pal[2 * 4 + c] = (uint8_t)bc1_third(a[c], b[c], bits);
      pal[3 * 4 + c] = (uint8_t)bc1_third(b[c], a[c], bits);
    } else {
      pal[2 * 4 + c] = (uint8_t)bc1_half(a[c], b[c], bits);
      pal[3 * 4 + c] = 0;
    }
  }
  pal[0 * 4 + 3] = pal[1 * 4 + 3] = pal[2 * 4 + 3] = 255;
  pal[3 * 4 + 3] = (c0 > c1) ? 255 : 0;
}

/* Sec. III-A; BC1 format: a block to its 16 texels. */
void or_bc1_decode(const uint8_t* blk, uint8_t* out) {
  uint16_t c0 = (uint16_t)(blk[0] | (blk[1] << 8));
  uint16_t c1 = (uint16_t)(blk[2] | (blk[3] << 8));
  uint32_t ix = (uint32_t)blk[4] | ((uint32_t)blk[5] << 8) | ((uint32_t)blk[6] << 16) | ((uint32_t)blk[7] << 24);
  uint8_t pal[16];
  or_bc1_palette(c0, c1, pal);
  for (int t = 0; t < 16; t++) {
    int j = (ix >> (2 * t)) & 3;
    for (int c = 0; c < 4; c++) out[t * 4 + c] = pal[j * 4 + c];
  }
}

typedef struct { uint64_t sse; uint16_t c0, c1; int idx[16]; } bc1_sol;

/* Evaluate an endpoint pair: c0 == c1 codes one colour with all indices 0;
 * otherwise the pair is ordered so that c0 > c1 (four-colour mode) and each texel
 * takes the palette entry of least squared error, ties to the lowest index. */
static bc1_sol bc1_eval(const uint8_t* tex, uint16_t a, uint16_t b) {
  bc1_sol r;
  uint8_t pal[16];
  r.c0 = a > b ? a : b;
  r.c1 = a > b ? b : a;
  r.sse = 0;
  or_bc1_palette(r.c0, r.c1, pal);
  int nent = (r.c0 == r.c1) ? 1 : 4;
  for (int t = 0; t < 16; t++) {
    int best = -1, bj = 0;
    for (int j = 0; j < nent; j++) {
      int e = sq(tex[3 * t] - pal[4 * j]) + sq(tex[3 * t + 1] - pal[4 * j + 1]) + sq(tex[3 * t + 2] - pal[4 * j + 2]);
      if (best < 0 || e < best) { best = e; bj = j; }
    }
    r.idx[t] = bj;
    r.sse += (uint64_t)best;
  }
  return r;
}

uint64_t or_bc1_candidate_sse(const uint8_t* tex, uint16_t c0, uint16_t c1) { return bc1_eval(tex, c0, c1).sse; }

static int q5(int v) { return (v * 31 + 127) / 255; }
static int q6(int v) { return (v * 63 + 127) / 255; }
static uint16_t pack565(const int e[3]) { return (uint16_t)((q5(e[0]) << 11) | (q6(e[1]) << 5) | q5(e[2])); }

static void bc1_write(const bc1_sol* s, uint8_t* out) {
  uint32_t ix = 0;
  for (int t = 0; t < 16; t++) ix |= (uint32_t)s->idx[t] << (2 * t);
  out[0] = s->c0 & 255; out[1] = s->c0 >> 8; out[2] = s->c1 & 255; out[3] = s->c1 >> 8;
  out[4] = ix & 255; out[5] = (ix >> 8) & 255; out[6] = (ix >> 16) & 255; out[7] = ix >> 24;
}

/* Sec. III-A/B; BC1 format: the least-error block under the encoder specification. */
uint64_t or_bc1_encode(const uint8_t* tex, uint8_t* out) {
  int constant = 1;
  for (int t = 1; t < 16; t++)
    if (tex[3 * t] != tex[0] || tex[3 * t + 1] != tex[1] || tex[3 * t + 2] != tex[2]) constant = 0;
  bc1_sol best;
  if (constant) {
    /* per channel, the code pair whose two-thirds point is nearest (ties: smallest a, then b) */
    int ca[3], cb[3];
    for (int c = 0; c < 3; c++) {
      int bits = (c == 1) ? 6 : 5, lim = 1 << bits, be = -1;
      for (int a = 0; a < lim; a++)
        for (int b = 0; b < lim; b++) {
          int e = abs(bc1_third(a, b, bits) - tex[c]);
          if (be < 0 || e < be) { be = e; ca[c] = a; cb[c] = b; }
        }
    }
    uint16_t c0 = (uint16_t)((ca[0] << 11) | (ca[1] << 5) | ca[2]);
    uint16_t c1 = (uint16_t)((cb[0] << 11) | (cb[1] << 5) | cb[2]);
    best = bc1_eval(tex, c0, c1);
    bc1_write(&best, out);
    return best.sse;
  }
  /* (ii) bounding-box diagonal oriented by covariance signs, inset by range/16 */
  int lo[3] = {255, 255, 255}, hi[3] = {0, 0, 0};
  int64_t s1[3] = {0, 0, 0}, s2[3][3];
  memset(s2, 0, sizeof(s2));
  for (int t = 0; t < 16; t++)
    for (int c = 0; c < 3; c++) {
      int v = tex[3 * t + c];
      if (v < lo[c]) lo[c] = v;
      if (v > hi[c]) hi[c] = v;
      s1[c] += v;
      for (int d = 0; d < 3; d++) s2[c][d] += v * tex[3 * t + d];
    }
  int ref = 0;
  for (int c = 1; c < 3; c++) if (hi[c] - lo[c] > hi[ref] - lo[ref]) ref = c;
  int e0[3], e1[3];
  for (int c = 0; c < 3; c++) {
    int flip = 0;
    if (c != ref) flip = (16 * s2[ref][c] - s1[ref] * s1[c]) < 0;
    e0[c] = flip ? lo[c] : hi[c];
    e1[c] = flip ? hi[c] : lo[c];
    int d = (hi[c] - lo[c]) >> 4;
    if (e0[c] >= e1[c]) { e0[c] -= d; e1[c] += d; } else { e0[c] += d; e1[c] -= d; }
  }
  best = bc1_eval(tex, pack565(e0), pack565(e1));
  /* (iii) two least-squares refinements on the current indices */
  for (int it = 0; it < 2; it++) {
    static const int A3[4] = {3, 0, 2, 1};
    int64_t saa = 0, sbb = 0, sab = 0, sav[3] = {0, 0, 0}, sbv[3] = {0, 0, 0};
    if (best.c0 == best.c1) break;
    for (int t = 0; t < 16; t++) {
      int a = A3[best.idx[t]], b = 3 - a;
      saa += a * a; sbb += b * b; sab += a * b;
      for (int c = 0; c < 3; c++) { sav[c] += a * tex[3 * t + c]; sbv[c] += b * tex[3 * t + c]; }
    }
    int64_t det = saa * sbb - sab * sab;
    if (det == 0) break;
    for (int c = 0; c < 3; c++) {
      e0[c] = clampi(round_div(3 * (sbb * sav[c] - sab * sbv[c]), det), 0, 255);
      e1[c] = clampi(round_div(3 * (saa * sbv[c] - sab * sav[c]), det), 0, 255);
    }
    bc1_sol r = bc1_eval(tex, pack565(e0), pack565(e1));
    if (r.sse < best.sse) best = r; else break;
  }
  /* (iv) +-1 neighbourhood on the six endpoint channels, at most four rounds */
  for (int round = 0; round < 4; round++) {
    bc1_sol nb; nb.sse = UINT64_MAX; int found = 0;
    for (int ep = 0; ep < 2; ep++)
      for (int c = 0; c < 3; c++)
        for (int sgn = 0; sgn < 2; sgn++) {
          uint16_t cc[2] = {best.c0, best.c1};
          int shift = c == 0 ? 11 : (c == 1 ? 5 : 0), mask = c == 1 ? 63 : 31;
          int v = (cc[ep] >> shift) & mask;
          v += sgn ? -1 : 1;
          if (v < 0 || v > mask) continue;
          cc[ep] = (uint16_t)((cc[ep] & ~(mask << shift)) | (v << shift));
          bc1_sol r = bc1_eval(tex, cc[0], cc[1]);
          if (!found || r.sse < nb.sse) { nb = r; found = 1; }
        }
    if (found && nb.sse < best.sse) best = nb; else break;
  }
  bc1_write(&best, out);
  return best.sse;
}

/* ------------------------------------------------------------------------- */
/* BC7 (D3D11 / Khronos BC7 format definition; Sec. III-B).                   */
/* ------------------------------------------------------------------------- */
typedef struct { int ns, pb, rb, isb, cb, ab, epb, spb, ib, ib2; } bc7_mode;
static const bc7_mode MODE[8] = {
    {3, 4, 0, 0, 4, 0, 1, 0, 3, 0}, {2, 6, 0, 0, 6, 0, 0, 1, 3, 0}, {3, 6, 0, 0, 5, 0, 0, 0, 2, 0},
    {2, 6, 0, 0, 7, 0, 1, 0, 2, 0}, {1, 0, 2, 1, 5, 6, 0, 0, 2, 3}, {1, 0, 2, 0, 7, 8, 0, 0, 2, 2},
    {1, 0, 0, 0, 7, 7, 1, 0, 4, 0}, {2, 6, 0, 0, 5, 5, 1, 0, 2, 0}};

/* Two-subset partitions, one row per partition id, texel 0..15 in raster order. */
static const char* PART2[64] = {
    "0011001100110011", "0001000100010001", "0111011101110111", "0001001100110111",
    "0000000100010011", "0011011101111111", "0001001101111111", "0000000100110111",
    "0000000000010011", "0011011111111111", "0000000101111111", "0000000000010111",
    "0001011111111111", "0000000011111111", "0000111111111111", "0000000000001111",
    "0000100011101111", "0111000100000000", "0000000010001110", "0111001100010000",
    "0011000100000000", "0000100011001110", "0000000010001100", "0111001100110001",
    "0011000100010000", "0000100010001100", "0110011001100110", "0011011001101100",
    "0001011111101000", "0000111111110000", "0111000110001110", "0011100110011100",
    "0101010101010101", "0000111100001111", "0101101001011010", "0011001111001100",
    "0011110000111100", "0101010110101010", "0110100101101001", "0101101010100101",
    "0111001111001110", "0001001111001000", "0011001001001100", "0011101111011100",
    "0110100110010110", "0011110011000011", "0110011010011001", "0000011001100000",
    "0100111001000000", "0010011100100000", "0000001001110010", "0000010011100100",
    "0110110010010011", "0011011011001001", "0110001110011100", "0011100111000110",
    "0110110011001001", "0110001100111001", "0111111010000001", "0001100011100111",
    "0000111100110011", "0011001111110000", "0010001011101110", "0100010001110111"};
/* Three-subset partitions. */
static const char* PART3[64] = {
    "0011001102212222", "0001001122112221", "0000200122112211", "0222002200110111",
    "0000000011221122", "0011001100220022", "0022002211111111", "0011001122112211",
    "0000000011112222", "0000111111112222", "0000111122222222", "0012001200120012",
    "0112011201120112", "0122012201220122", "0011011211221222", "0011200122002220",
    "0001001101121122", "0111001120012200", "0000112211221122", "0022002200221111",
    "0111011102220222", "0001000122212221", "0000001101220122", "0000110022102210",
    "0122012200110000", "0012001211222222", "0110122112210110", "0000011012211221",
    "0022110211020022", "0110011020022222", "0011012201220011", "0000200022112221",
    "0000000211221222", "0222002200120011", "0011001200220222", "0120012001200120",
    "0000111122220000", "0120120120120120", "0120201212010120", "0011220011220011",
    "0011112222000011", "0101010122222222", "0000000021212121", "0022112200221122",
    "0022001100220011", "0220122102201221", "0101222222220101", "0000212121212121",
    "0101010101012222", "0222011102220111", "0002111200021112", "0000211221122112",
    "0222011101110222", "0002111211120002", "0110011001102222", "0000000021122112",
    "0110011022222222", "0022001100110022", "0022112211220022", "0000000000002112",
    "0002000100020001", "0222122202221222", "0101222222222222", "0111201122012220"};
/* Anchor texels: second subset of two-subset partitions; second and third subsets
 * of three-subset partitions (the first subset's anchor is always texel 0). */
static const int ANCH2[64] = {
    15, 15, 15, 15, 15, 15, 15, 15, 15, 15, 15, 15, 15, 15, 15, 15, 15, 2, 8, 2, 2, 8, 8, 15, 2, 8, 2, 2, 8, 8, 2, 2,
    15, 15, 6, 8, 2, 8, 15, 15, 2, 8, 2, 2, 2, 15, 15, 6, 6, 2, 6, 8, 15, 15, 2, 2, 15, 15, 15, 15, 15, 2, 2, 15};
static const int ANCH3A[64] = {
    3, 3, 15, 15, 8, 3, 15, 15, 8, 8, 6, 6, 6, 5, 3, 3, 3, 3, 8, 15, 3, 3, 6, 10, 5, 8, 8, 6, 8, 5, 15, 15,
    8, 15, 3, 5, 6, 10, 8, 15, 15, 3, 15, 5, 15, 15, 15, 15, 3, 15, 5, 5, 5, 8, 5, 10, 5, 10, 8, 13, 15, 12, 3, 3};
static const int ANCH3B[64] = {
    15, 8, 8, 3, 15, 15, 3, 8, 15, 15, 15, 15, 15, 15, 15, 8, 15, 8, 15, 3, 15, 8, 15, 8, 3, 15, 6, 10, 15, 15, 10, 8,
    15, 3, 15, 10, 10, 8, 9, 10, 6, 15, 8, 15, 3, 6, 6, 8, 15, 3, 15, 15, 15, 15, 15, 15, 15, 15, 15, 15, 3, 15, 15, 8};

static const int WT2[4] = {0, 21, 43, 64};
static const int WT3[8] = {0, 9, 18, 27, 37, 46, 55, 64};
static const int WT4[16] = {0, 4, 9, 13, 17, 21, 26, 30, 34, 38, 43, 47, 51, 55, 60, 64};
static const int* wtab(int ib) { return ib == 2 ? WT2 : (ib == 3 ? WT3 : WT4); }
static int interp7(int e0, int e1, int w) { return ((64 - w) * e0 + w * e1 + 32) >> 6; }
static int expand_bits(int v, int n) { return n >= 8 ? v : ((v << (8 - n)) | (v >> (2 * n - 8))); }

/* Sec. III-B; BC7 format: the subset of texel t in partition part. */
int or_bc7_subset(int ns, int part, int t) {
  if (ns == 1) return 0;
  return (ns == 2 ? PART2[part][t] : PART3[part][t]) - '0';
}
/* Sec. III-B; BC7 format: the anchor texel of subset s. */
int or_bc7_anchor(int ns, int part, int s) {
  if (s == 0) return 0;
  if (ns == 2) return ANCH2[part];
  return s == 1 ? ANCH3A[part] : ANCH3B[part];
}
static int is_anchor(int ns, int part, int t) {
  for (int s = 0; s < ns; s++) if (or_bc7_anchor(ns, part, s) == t) return 1;
  return 0;
}

typedef struct { uint8_t b[16]; int pos; } bitw;
static void bw_put(bitw* w, uint32_t v, int n) {
  for (int i = 0; i < n; i++, w->pos++)
    if ((v >> i) & 1u) w->b[w->pos >> 3] |= (uint8_t)(1u << (w->pos & 7));
}
typedef struct { const uint8_t* b; int pos; } bitr;
static uint32_t br_get(bitr* r, int n) {
  uint32_t v = 0;
  for (int i = 0; i < n; i++, r->pos++) v |= (uint32_t)((r->b[r->pos >> 3] >> (r->pos & 7)) & 1u) << i;
  return v;
}

/* Sec. III-B; BC7 format: a block of any mode to its 16 texels. */
void or_bc7_decode(const uint8_t* blk, uint8_t* out) {
  int m = 0;
  while (m < 8 && !((blk[0] >> m) & 1)) m++;
  if (m == 8) { memset(out, 0, 64); return; }
  const bc7_mode* M = &MODE[m];
  bitr r = {blk, m + 1};
  int part = (int)br_get(&r, M->pb), rot = (int)br_get(&r, M->rb), isb = (int)br_get(&r, M->isb);
  int code[3][2][4], p[3][2];
  for (int c = 0; c < 3; c++)
    for (int s = 0; s < M->ns; s++)
      for (int e = 0; e < 2; e++) code[s][e][c] = (int)br_get(&r, M->cb);
  for (int s = 0; s < M->ns; s++)
    for (int e = 0; e < 2; e++) code[s][e][3] = M->ab ? (int)br_get(&r, M->ab) : 0;
  for (int s = 0; s < M->ns; s++)
    for (int e = 0; e < 2; e++) p[s][e] = 0;
  if (M->epb)
    for (int s = 0; s < M->ns; s++)
      for (int e = 0; e < 2; e++) p[s][e] = (int)br_get(&r, 1);
  if (M->spb)
    for (int s = 0; s < M->ns; s++) p[s][0] = p[s][1] = (int)br_get(&r, 1);
  int pri[16], sec[16];
  for (int t = 0; t < 16; t++) pri[t] = (int)br_get(&r, M->ib - is_anchor(M->ns, part, t));
  for (int t = 0; t < 16; t++) sec[t] = M->ib2 ? (int)br_get(&r, M->ib2 - (t == 0)) : 0;
  int hp = M->epb || M->spb;
  int ev[3][2][4];
  for (int s = 0; s < M->ns; s++)
    for (int e = 0; e < 2; e++) {
      for (int c = 0; c < 3; c++) ev[s][e][c] = expand_bits(hp ? (code[s][e][c] << 1) | p[s][e] : code[s][e][c], M->cb + hp);
      ev[s][e][3] = M->ab ? expand_bits(M->epb ? (code[s][e][3] << 1) | p[s][e] : code[s][e][3], M->ab + M->epb) : 255;
    }
  for (int t = 0; t < 16; t++) {
    int s = or_bc7_subset(M->ns, part, t);
    int ci = pri[t], cbits = M->ib, ai = pri[t], abits = M->ib;
    if (M->ib2) {
      if (isb) { ci = sec[t]; cbits = M->ib2; ai = pri[t]; abits = M->ib; }
      else { ci = pri[t]; cbits = M->ib; ai = sec[t]; abits = M->ib2; }
    }
    int px[4];
    for (int c = 0; c < 3; c++) px[c] = interp7(ev[s][0][c], ev[s][1][c], wtab(cbits)[ci]);
    px[3] = M->ab ? interp7(ev[s][0][3], ev[s][1][3], wtab(abits)[ai]) : 255;
    if (rot) { int tmp = px[3]; px[3] = px[rot - 1]; px[rot - 1] = tmp; }
    for (int c = 0; c < 4; c++) out[t * 4 + c] = (uint8_t)px[c];
  }
}

/* --- BC7 encoder: the codec's own exhaustive integer search ---------------- */
/* Candidate order: mode 0 partitions 0..15; modes 1, 2, 3 partitions 0..63;
 * mode 4 rotation 0..3 x index selection 0..1; mode 5 rotation 0..3; mode 6;
 * mode 7 partitions 0..63. */
typedef struct { int mode, part, rot, isb; } bc7_cand;
static int cand_of(int e, bc7_cand* c) {
  c->part = c->rot = c->isb = 0;
  if (e < 16) { c->mode = 0; c->part = e; return 0; }
  e -= 16;
  if (e < 192) { c->mode = 1 + e / 64; c->part = e % 64; return 0; }
  e -= 192;
  if (e < 8) { c->mode = 4; c->rot = e / 2; c->isb = e % 2; return 0; }
  e -= 8;
  if (e < 4) { c->mode = 5; c->rot = e; return 0; }
  e -= 4;
  if (e < 1) { c->mode = 6; return 0; }
  e -= 1;
  if (e < 64) { c->mode = 7; c->part = e; return 0; }
  return -1;
}
int or_bc7_n_candidates(void) { return 16 + 192 + 8 + 4 + 1 + 64; }

/* Nearest endpoint code for an 8-bit target with a given p-bit (ptype 0: none). */
static int ep_value(int code, int p, int bits, int has_p) { return expand_bits(has_p ? (code << 1) | p : code, bits + has_p); }
static int ep_nearest(int e, int p, int bits, int has_p) {
  int best = 0, be = -1;
  for (int code = 0; code < (1 << bits); code++) {
    int d = abs(ep_value(code, p, bits, has_p) - e);
    if (be < 0 || d < be) { be = d; best = code; }
  }
  return best;
}

typedef struct { int code[2][3]; int p[2]; int idx[16]; uint64_t sse; } fit_res;

/* Fit one subset: chans lists the nch channels coded (the others are not scored).
 * ptype: 0 no p-bit, 1 one p-bit per endpoint, 2 one p-bit shared by both endpoints. */
static fit_res fit_subset(const uint8_t* tex, const int* mem, const int* chans, int nch, int ib, int bits, int ptype) {
  fit_res out;
  memset(&out, 0, sizeof(out));
  out.sse = UINT64_MAX;
  const int* W = wtab(ib);
  int F = 1 << ib;
  int n = 0, lo[3], hi[3];
  int64_t s1[3] = {0, 0, 0}, s2[3][3];
  memset(s2, 0, sizeof(s2));
  for (int i = 0; i < nch; i++) { lo[i] = 255; hi[i] = 0; }
  for (int t = 0; t < 16; t++) {
    if (!mem[t]) continue;
    n++;
    for (int i = 0; i < nch; i++) {
      int v = tex[3 * t + chans[i]];
      if (v < lo[i]) lo[i] = v;
      if (v > hi[i]) hi[i] = v;
      s1[i] += v;
      for (int j = 0; j < nch; j++) s2[i][j] += v * tex[3 * t + chans[j]];
    }
  }
  if (n == 0) { out.sse = 0; return out; }
  int ref = 0;
  for (int i = 1; i < nch; i++) if (hi[i] - lo[i] > hi[ref] - lo[ref]) ref = i;
  int e0[3], e1[3];
  for (int i = 0; i < nch; i++) {
    int flip = (i != ref) && ((int64_t)n * s2[ref][i] - s1[ref] * s1[i] < 0);
    e0[i] = flip ? lo[i] : hi[i];
    e1[i] = flip ? hi[i] : lo[i];
  }
  /* initial indices against the unquantised endpoints */
  int idx[16];
  for (int t = 0; t < 16; t++) {
    idx[t] = 0;
    if (!mem[t]) continue;
    int be = -1;
    for (int j = 0; j < F; j++) {
      int e = 0;
      for (int i = 0; i < nch; i++) e += sq(tex[3 * t + chans[i]] - interp7(e0[i], e1[i], W[j]));
      if (be < 0 || e < be) { be = e; idx[t] = j; }
    }
  }
  /* one least-squares refinement */
  int64_t saa = 0, sbb = 0, sab = 0, sav[3] = {0, 0, 0}, sbv[3] = {0, 0, 0};
  for (int t = 0; t < 16; t++) {
    if (!mem[t]) continue;
    int a = 64 - W[idx[t]], b = W[idx[t]];
    saa += a * a; sbb += b * b; sab += a * b;
    for (int i = 0; i < nch; i++) { sav[i] += a * tex[3 * t + chans[i]]; sbv[i] += b * tex[3 * t + chans[i]]; }
  }
  int64_t det = saa * sbb - sab * sab;
  if (det != 0)
    for (int i = 0; i < nch; i++) {
      e0[i] = clampi(round_div(64 * (sbb * sav[i] - sab * sbv[i]), det), 0, 255);
      e1[i] = clampi(round_div(64 * (saa * sbv[i] - sab * sav[i]), det), 0, 255);
    }
  /* p-bit combinations, each quantised to the nearest codes and re-indexed */
  int ncombo = ptype == 0 ? 1 : (ptype == 1 ? 4 : 2);
  int has_p = ptype != 0;
  for (int cmb = 0; cmb < ncombo; cmb++) {
    int p0 = ptype == 1 ? (cmb & 1) : cmb, p1 = ptype == 1 ? (cmb >> 1) : cmb;
    if (ptype == 0) p0 = p1 = 0;
    fit_res r;
    memset(&r, 0, sizeof(r));
    r.p[0] = p0; r.p[1] = p1;
    int v0[3], v1[3];
    for (int i = 0; i < nch; i++) {
      r.code[0][i] = ep_nearest(e0[i], p0, bits, has_p);
      r.code[1][i] = ep_nearest(e1[i], p1, bits, has_p);
      v0[i] = ep_value(r.code[0][i], p0, bits, has_p);
      v1[i] = ep_value(r.code[1][i], p1, bits, has_p);
    }
    r.sse = 0;
    for (int t = 0; t < 16; t++) {
      r.idx[t] = 0;
      if (!mem[t]) continue;
      int be = -1;
      for (int j = 0; j < F; j++) {
        int e = 0;
        for (int i = 0; i < nch; i++) e += sq(tex[3 * t + chans[i]] - interp7(v0[i], v1[i], W[j]));
        if (be < 0 || e < be) { be = e; r.idx[t] = j; }
      }
      r.sse += (uint64_t)be;
    }
    if (r.sse < out.sse) out = r;
  }
  return out;
}

/* Full solution of one candidate; codes are [subset][endpoint][R,G,B,A-slot]. */
typedef struct {
  bc7_cand c; uint64_t sse;
  int code[3][2][4]; int p[3][2]; int cidx[16]; int aidx[16];
} bc7_sol;

static void bc7_solve(const uint8_t* tex, const bc7_cand* cd, bc7_sol* S) {
  const bc7_mode* M = &MODE[cd->mode];
  memset(S, 0, sizeof(*S));
  S->c = *cd;
  if (cd->mode == 4 || cd->mode == 5) {
    int cib = (cd->mode == 4) ? (cd->isb ? 3 : 2) : 2;
    int aib = (cd->mode == 4) ? (cd->isb ? 2 : 3) : 2;
    int mem[16], chans[3], nch = 0;
    for (int t = 0; t < 16; t++) mem[t] = 1;
    for (int c = 0; c < 3; c++) if (c != cd->rot - 1) chans[nch++] = c;
    fit_res fc = fit_subset(tex, mem, chans, nch, cib, M->cb, 0);
    for (int i = 0; i < nch; i++) { S->code[0][0][chans[i]] = fc.code[0][i]; S->code[0][1][chans[i]] = fc.code[1][i]; }
    for (int t = 0; t < 16; t++) S->cidx[t] = fc.idx[t];
    S->sse = fc.sse;
    if (cd->rot == 0) {
      S->code[0][0][3] = S->code[0][1][3] = (1 << M->ab) - 1;
    } else {
      int ch = cd->rot - 1;
      fit_res fa = fit_subset(tex, mem, &ch, 1, aib, M->ab, 0);
      S->code[0][0][3] = fa.code[0][0]; S->code[0][1][3] = fa.code[1][0];
      for (int t = 0; t < 16; t++) S->aidx[t] = fa.idx[t];
      S->sse += fa.sse;
    }
    return;
  }
  int ptype = M->epb ? 1 : (M->spb ? 2 : 0);
  int chans[3] = {0, 1, 2};
  for (int s = 0; s < M->ns; s++) {
    int mem[16];
    for (int t = 0; t < 16; t++) mem[t] = or_bc7_subset(M->ns, cd->part, t) == s;
    fit_res f = fit_subset(tex, mem, chans, 3, M->ib, M->cb, ptype);
    for (int e = 0; e < 2; e++) {
      for (int c = 0; c < 3; c++) S->code[s][e][c] = f.code[e][c];
      S->code[s][e][3] = M->ab ? (1 << M->ab) - 1 : 0;
      S->p[s][e] = f.p[e];
    }
    for (int t = 0; t < 16; t++) if (mem[t]) S->cidx[t] = f.idx[t];
    S->sse += f.sse;
  }
}

/* Anchor fix (lossless): where an anchor texel's index has its top bit set, swap
 * that subset's endpoints (and p-bits) and invert its indices. Then pack. */
static void bc7_pack(bc7_sol* S, uint8_t* out) {
  const bc7_mode* M = &MODE[S->c.mode];
  int part = S->c.part;
  if (M->ib2) {
    int cib = S->c.isb ? M->ib2 : M->ib, aib = S->c.isb ? M->ib : M->ib2;
    if ((S->cidx[0] >> (cib - 1)) & 1) {
      for (int c = 0; c < 3; c++) { int t = S->code[0][0][c]; S->code[0][0][c] = S->code[0][1][c]; S->code[0][1][c] = t; }
      for (int t = 0; t < 16; t++) S->cidx[t] = (1 << cib) - 1 - S->cidx[t];
    }
    if ((S->aidx[0] >> (aib - 1)) & 1) {
      int t = S->code[0][0][3]; S->code[0][0][3] = S->code[0][1][3]; S->code[0][1][3] = t;
      for (int u = 0; u < 16; u++) S->aidx[u] = (1 << aib) - 1 - S->aidx[u];
    }
  } else {
    for (int s = 0; s < M->ns; s++) {
      int a = or_bc7_anchor(M->ns, part, s);
      if (!((S->cidx[a] >> (M->ib - 1)) & 1)) continue;
      for (int c = 0; c < 4; c++) { int t = S->code[s][0][c]; S->code[s][0][c] = S->code[s][1][c]; S->code[s][1][c] = t; }
      if (M->epb) { int t = S->p[s][0]; S->p[s][0] = S->p[s][1]; S->p[s][1] = t; }
      for (int t = 0; t < 16; t++)
        if (or_bc7_subset(M->ns, part, t) == s) S->cidx[t] = (1 << M->ib) - 1 - S->cidx[t];
    }
  }
  bitw w;
  memset(&w, 0, sizeof(w));
  bw_put(&w, 1u << S->c.mode, S->c.mode + 1);
  bw_put(&w, (uint32_t)part, M->pb);
  bw_put(&w, (uint32_t)S->c.rot, M->rb);
  bw_put(&w, (uint32_t)S->c.isb, M->isb);
  for (int c = 0; c < 3; c++)
    for (int s = 0; s < M->ns; s++)
      for (int e = 0; e < 2; e++) bw_put(&w, (uint32_t)S->code[s][e][c], M->cb);
  if (M->ab)
    for (int s = 0; s < M->ns; s++)
      for (int e = 0; e < 2; e++) bw_put(&w, (uint32_t)S->code[s][e][3], M->ab);
  if (M->epb)
    for (int s = 0; s < M->ns; s++)
      for (int e = 0; e < 2; e++) bw_put(&w, (uint32_t)S->p[s][e], 1);
  if (M->spb)
    for (int s = 0; s < M->ns; s++) bw_put(&w, (uint32_t)S->p[s][0], 1);
  if (M->ib2) {
    for (int t = 0; t < 16; t++) bw_put(&w, (uint32_t)(S->c.isb ? S->aidx[t] : S->cidx[t]), M->ib - (t == 0));
    for (int t = 0; t < 16; t++) bw_put(&w, (uint32_t)(S->c.isb ? S->cidx[t] : S->aidx[t]), M->ib2 - (t == 0));
  } else {
    for (int t = 0; t < 16; t++) bw_put(&w, (uint32_t)S->cidx[t], M->ib - is_anchor(M->ns, part, t));
  }
  memcpy(out, w.b, 16);
}

/* Sec. III-B; BC7 format: the error and block of one enumerated candidate. */
uint64_t or_bc7_candidate(const uint8_t* tex, int e, uint8_t* out) {
  bc7_cand c;
  if (cand_of(e, &c)) return UINT64_MAX;
  bc7_sol S;
  bc7_solve(tex, &c, &S);
  if (out) bc7_pack(&S, out);
  return S.sse;
}

/* Constant blocks (Sec. III-A: the error of a block whose texels are all one colour can go to
 * zero; the format reaches every constant colour). Mode 5, rotation 0, every colour index 1: the
 * 2-bit index's weight 21 interpolates two 7-bit endpoint codes, and for every 8-bit value v some
 * pair (a, b) gives ((64 - 21) ex7(a) + 21 ex7(b) + 32) >> 6 = v. Per channel the pair found first
 * with a = 0..127 outer, b = 0..127 inner is taken; alpha codes are all ones, alpha indices 0. */
static void bc7_const_pair(int v, int* a, int* b) {
  for (int i = 0; i < 128; i++)
    for (int j = 0; j < 128; j++)
      if (interp7(expand_bits(i, 7), expand_bits(j, 7), WT2[1]) == v) { *a = i; *b = j; return; }
  *a = *b = 0; /* not reached: every value has a pair */
}

static void bc7_const_block(const uint8_t* rgb, uint8_t* out) {
  bc7_sol S;
  memset(&S, 0, sizeof(S));
  S.c.mode = 5;
  for (int c = 0; c < 3; c++) bc7_const_pair(rgb[c], &S.code[0][0][c], &S.code[0][1][c]);
  S.code[0][0][3] = S.code[0][1][3] = 255;
  for (int t = 0; t < 16; t++) { S.cidx[t] = 1; S.aidx[t] = 0; }
  bc7_pack(&S, out);
}

/* Sec. III-B; BC7 format: a constant block as above (error 0), otherwise the least-error
 * candidate, first on ties. */
uint64_t or_bc7_encode(const uint8_t* tex, uint8_t* out) {
  int constant = 1;
  for (int t = 1; t < 16; t++)
    if (tex[3 * t] != tex[0] || tex[3 * t + 1] != tex[1] || tex[3 * t + 2] != tex[2]) constant = 0;
  if (constant) {
    if (out) bc7_const_block(tex, out);
    return 0;
  }
  int ne = or_bc7_n_candidates(), best_e = 0;
  uint64_t best = UINT64_MAX;
  for (int e = 0; e < ne; e++) {
    uint64_t s = or_bc7_candidate(tex, e, NULL);
    if (s < best) { best = s; best_e = e; }
  }
  return or_bc7_candidate(tex, best_e, out);
}

/* Encode nblk independent blocks of 16 texels; format 1 = BC1 (8 B), 7 = BC7 (16 B). */
void or_encode_blocks(const uint8_t* tex, int64_t nblk, int format, uint8_t* out, uint64_t* sse) {
  for (int64_t b = 0; b < nblk; b++) {
    uint64_t s = (format == 7) ? or_bc7_encode(tex + 48 * b, out + 16 * b) : or_bc1_encode(tex + 48 * b, out + 8 * b);
    if (sse) sse[b] = s;
  }
}

/* ------------------------------------------------------------------------- */
/* Rate control (Sec. IV-B; abstract; Figs. SetupC/SetupD).                   */
/* 14 group modes (b kept coefficients, j leading BC7 blocks), R = 64 (b + j).  */
/* ------------------------------------------------------------------------- */
static const int MODE_B[OR_MODES] = {1, 1, 4, 4, 4, 9, 9, 9, 9, 16, 16, 16, 16, 16};
static const int MODE_J[OR_MODES] = {0, 1, 0, 1, 4, 0, 1, 4, 9, 0, 1, 4, 9, 16};
static uint64_t mode_rate(int m) { return 64u * (uint64_t)(MODE_B[m] + MODE_J[m]); }

/* Sec. IV-B, Table I: the 14 fixed-rate codings of a group (bands kept, BC7 blocks). */
void or_mode_table(int32_t* bands, int32_t* bc7) {
  for (int m = 0; m < OR_MODES; m++) { bands[m] = MODE_B[m]; bc7[m] = MODE_J[m]; }
}

/* Sec. IV-B. w_k = max(1, rint(65536 s_k^2 / max s^2)) in double precision. */
void or_weights(const float* scales, uint32_t* w) {
  double mx = 0.0;
  for (int k = 0; k < OR_SH; k++) { double s = scales[k]; if (s * s > mx) mx = s * s; }
  for (int k = 0; k < OR_SH; k++) {
    double s = scales[k];
    double v = rint((s * s * 65536.0) / mx);
    w[k] = v < 1.0 ? 1u : (uint32_t)v;
  }
}

/* Per group: argmin over modes of D * 2^16 + lambda * R in 128-bit arithmetic;
 * ties go to the lower rate (rates are distinct). Returns sum of rates (bits). */
static uint64_t choose_all(const uint64_t* D, int64_t ng, uint64_t lambda, uint8_t* mode) {
  uint64_t total = 0;
  for (int64_t g = 0; g < ng; g++) {
    int best = -1;
    unsigned __int128 bc = 0;
    for (int m = 0; m < OR_MODES; m++) {
      unsigned __int128 cost = ((unsigned __int128)D[g * OR_MODES + m] << 16) + (unsigned __int128)lambda * mode_rate(m);
      if (best < 0 || cost < bc || (cost == bc && mode_rate(m) < mode_rate(best))) { best = m; bc = cost; }
    }
    if (mode) mode[g] = (uint8_t)best;
    total += mode_rate(best);
  }
  return total;
}

/* Sec. IV-B: every group's coding at one Lagrange multiplier. */
int or_rate_choose(const uint64_t* D, int64_t ng, uint64_t lambda, uint8_t* mode) {
  choose_all(D, ng, lambda, mode);
  return 0;
}

/* Sec. IV-B. Smallest integer lambda in [0, 2^62] whose choice fits the budget, then a fill
 * step: groups whose choice differs at lambda - 1 take that choice, in group order,
 * until the first one that would exceed the budget. */
int or_rate_control(const uint64_t* D, int64_t ng, uint64_t budget, uint8_t* mode, uint64_t* lambda_out) {
  uint64_t lo = 0, hi = (uint64_t)1 << 62;
  if (choose_all(D, ng, hi, NULL) > budget) return -1;
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (choose_all(D, ng, mid, NULL) <= budget) hi = mid; else lo = mid + 1;
  }
  uint64_t used = choose_all(D, ng, lo, mode);
  if (lo > 0) {
    uint8_t* alt = (uint8_t*)malloc((size_t)(ng > 0 ? ng : 1));
    if (!alt) return -2;
    choose_all(D, ng, lo - 1, alt);
    for (int64_t g = 0; g < ng; g++) {
      if (alt[g] == mode[g]) continue;
      uint64_t up = mode_rate(alt[g]) - mode_rate(mode[g]);
      if (used + up > budget) break;
      used += up;
      mode[g] = alt[g];
    }
    free(alt);
  }
  if (lambda_out) *lambda_out = lo;
  return 0;
}

static uint64_t sse_block(const uint8_t* tex, const uint8_t* rgba) {
  uint64_t s = 0;
  for (int t = 0; t < 16; t++)
    for (int c = 0; c < 3; c++) s += (uint64_t)sq(tex[3 * t + c] - rgba[4 * t + c]);
  return s;
}

/* Whole-scene encode of layout D. format 1/7 forces BC1/BC7 in every block
 * (one stream); format 0 runs rate control at target_x4 / 4 bits per texel.
 * blocks must hold n_groups * 256 bytes; dtab (optional) receives D [ng][14]. */
int or_encode(const uint8_t* q, int64_t n, const int32_t* perm, const float* scales, int format,
              uint32_t target_x4, uint8_t* blocks, int32_t* perm_out, or_table* t, uint64_t* dtab) {
  int64_t ng = (n + 15) / 16;
  memset(t, 0, sizeof(*t));
  t->n = n; t->n_groups = ng; t->format = format;
  for (int k = 0; k < OR_SH; k++) t->scales[k] = scales[k];
  or_weights(scales, t->weights);
  uint8_t tex[16 * 16 * 3];
  if (format == 1 || format == 7) {
    int bpb = format == 7 ? 16 : 8;
    for (int64_t g = 0; g < ng; g++) {
      or_stage_group(q, perm, g, tex);
      for (int k = 0; k < OR_SH; k++) {
        uint8_t* dst = blocks + (g * 16 + k) * bpb;
        if (format == 7) or_bc7_encode(tex + 48 * k, dst); else or_bc1_encode(tex + 48 * k, dst);
      }
    }
    for (int64_t s = 0; s < ng * 16; s++) perm_out[s] = perm[s];
    t->n_streams = 1;
    t->s[0].bands = 16; t->s[0].bc7_blocks = format == 7 ? 16 : 0;
    t->s[0].first_group = 0; t->s[0].n_groups = ng; t->s[0].byte_offset = 0;
    t->total_bytes = ng * 16 * bpb;
    t->used_bits = (uint64_t)t->total_bytes * 8;
    return 0;
  }
  if (format != 0 || target_x4 == 0) return -1;
  /* code every block both ways; keep the blocks and the per-block errors */
  uint8_t* b1 = (uint8_t*)malloc((size_t)(ng * 16 * 8 + 1));
  uint8_t* b7 = (uint8_t*)malloc((size_t)(ng * 16 * 16 + 1));
  uint64_t* D = dtab ? dtab : (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(ng * OR_MODES + 1));
  if (!b1 || !b7 || !D) return -2;
  or_code_groups(q, n, perm, scales, b1, b7, D);
  int rc = or_rate_assemble(n, perm, scales, target_x4, b1, b7, D, blocks, perm_out, t);
  free(b1); free(b7);
  if (!dtab) free(D);
  return rc;
}

/* Groups g0..g1-1 of the rate path: both codings of every block, and D[g][m] = sum over the
 * 16 coefficients of w_k times the error of the coding mode m gives coefficient k. */
static void code_group_range(const uint8_t* q, const int32_t* perm, const uint32_t* w, uint8_t* b1, uint8_t* b7,
                             uint64_t* D, int64_t g0, int64_t g1) {
  uint8_t tex[16 * 16 * 3];
  for (int64_t g = g0; g < g1; g++) {
    uint64_t e1[16], e7[16], e0[16];
    uint8_t rgba[64];
    or_stage_group(q, perm, g, tex);
    for (int k = 0; k < OR_SH; k++) {
      const uint8_t* tk = tex + 48 * k;
      or_bc1_encode(tk, b1 + (g * 16 + k) * 8);
      or_bc1_decode(b1 + (g * 16 + k) * 8, rgba);
      e1[k] = sse_block(tk, rgba);
      or_bc7_encode(tk, b7 + (g * 16 + k) * 16);
      or_bc7_decode(b7 + (g * 16 + k) * 16, rgba);
      e7[k] = sse_block(tk, rgba);
      e0[k] = 0;
      for (int u = 0; u < 48; u++) e0[k] += (uint64_t)sq(tk[u] - 128);
    }
    for (int m = 0; m < OR_MODES; m++) {
      uint64_t d = 0;
      for (int k = 0; k < OR_SH; k++) {
        uint64_t e = k < MODE_J[m] ? e7[k] : (k < MODE_B[m] ? e1[k] : e0[k]);
        d += (uint64_t)w[k] * e;
      }
      D[g * OR_MODES + m] = d;
    }
  }
}

struct code_job {
  const uint8_t* q;
  const int32_t* perm;
  const uint32_t* w;
  uint8_t *b1, *b7;
  uint64_t* D;
  int64_t g0, g1;
};

static void* code_job_run(void* arg) {
  struct code_job* j = (struct code_job*)arg;
  code_group_range(j->q, j->perm, j->w, j->b1, j->b7, j->D, j->g0, j->g1);
  return NULL;
}

static int g_threads = 1;

void or_set_threads(int threads) { g_threads = threads < 1 ? 1 : (threads > 256 ? 256 : threads); }

/* Sec. IV-B. Both codings and the D table of every group. Groups are independent and write disjoint
 * memory, so they may be split over threads (or_set_threads) with identical results. */
void or_code_groups(const uint8_t* q, int64_t n, const int32_t* perm, const float* scales, uint8_t* b1, uint8_t* b7,
                    uint64_t* D) {
  int64_t ng = (n + 15) / 16;
  uint32_t w[OR_SH];
  or_weights(scales, w);
  int nt = g_threads;
  if ((int64_t)nt > ng) nt = ng > 0 ? (int)ng : 1;
  if (nt <= 1) {
    code_group_range(q, perm, w, b1, b7, D, 0, ng);
    return;
  }
  pthread_t th[256];
  struct code_job jobs[256];
  int started = 0;
  for (int i = 0; i < nt; i++) {
    jobs[i] = (struct code_job){q, perm, w, b1, b7, D, ng * i / nt, ng * (i + 1) / nt};
    if (pthread_create(&th[i], NULL, code_job_run, &jobs[i]) == 0) started = i + 1;
    else { code_group_range(q, perm, w, b1, b7, D, jobs[i].g0, jobs[i].g1); }
  }
  for (int i = 0; i < started; i++) pthread_join(th[i], NULL);
}

/* Sec. IV-B, Figs. SetupC/D.
 * Rate control at target_x4 / 4 bits per texel over coded groups, then the 14 streams: the
 * stable partition of groups by mode id, each group's kept blocks back to back. */
int or_rate_assemble(int64_t n, const int32_t* perm, const float* scales, uint32_t target_x4, const uint8_t* b1,
                     const uint8_t* b7, const uint64_t* D, uint8_t* blocks, int32_t* perm_out, or_table* t) {
  int64_t ng = (n + 15) / 16;
  memset(t, 0, sizeof(*t));
  t->n = n; t->n_groups = ng; t->format = 0;
  for (int k = 0; k < OR_SH; k++) t->scales[k] = scales[k];
  or_weights(scales, t->weights);
  if (target_x4 == 0) return -1;
  uint8_t* mode = (uint8_t*)malloc((size_t)(ng + 1));
  if (!mode) return -2;
  uint64_t budget = (uint64_t)target_x4 * 4u * (uint64_t)n;
  t->budget_bits = budget;
  int rc = or_rate_control(D, ng, budget, mode, &t->lambda);
  if (rc == 0) {
    /* streams: stable partition of groups by mode id */
    int64_t gpos = 0, off = 0;
    t->n_streams = OR_MODES;
    for (int m = 0; m < OR_MODES; m++) {
      int64_t gbytes = 16 * MODE_J[m] + 8 * (MODE_B[m] - MODE_J[m]);
      t->s[m].bands = MODE_B[m]; t->s[m].bc7_blocks = MODE_J[m];
      t->s[m].first_group = gpos; t->s[m].byte_offset = off;
      for (int64_t g = 0; g < ng; g++) {
        if (mode[g] != m) continue;
        uint8_t* dst = blocks + off;
        for (int k = 0; k < MODE_B[m]; k++) {
          if (k < MODE_J[m]) { memcpy(dst, b7 + (g * 16 + k) * 16, 16); dst += 16; }
          else { memcpy(dst, b1 + (g * 16 + k) * 8, 8); dst += 8; }
        }
        for (int u = 0; u < 16; u++) perm_out[gpos * 16 + u] = perm[g * 16 + u];
        gpos++; off += gbytes;
      }
      t->s[m].n_groups = gpos - t->s[m].first_group;
    }
    t->total_bytes = off;
    t->used_bits = (uint64_t)off * 8;
  }
  free(mode);
  return rc;
}

/* Sec. I, III; Sec. IV-B. Decode every stream back to texels [n][16][3] in original order (inverse
 * permutation); coefficients a stream does not keep decode to 128 (zero). */
int or_decode(const or_table* t, const uint8_t* blocks, const int32_t* perm, uint8_t* texels) {
  uint8_t rgba[16][64];
  const int layout = t->layout;
  for (int si = 0; si < t->n_streams; si++) {
    const or_stream* S = &t->s[si];
    int64_t gbytes = 16 * S->bc7_blocks + 8 * (S->bands - S->bc7_blocks);
    for (int64_t gi = 0; gi < S->n_groups; gi++) {
      int64_t g = S->first_group + gi;
      const uint8_t* src = blocks + S->byte_offset + gi * gbytes;
      /* a group's BC7 blocks come first, then its BC1 blocks, each in block order;
         blocks past the kept coefficients (layout D only) decode to 128 */
      for (int k = 0; k < OR_SH; k++) {
        if (k < S->bands && or_layout_bc7(layout, S->bc7_blocks, k)) { or_bc7_decode(src, rgba[k]); src += 16; }
      }
      for (int k = 0; k < OR_SH; k++) {
        if (k >= S->bands) memset(rgba[k], 128, sizeof(rgba[k]));
        else if (!or_layout_bc7(layout, S->bc7_blocks, k)) { or_bc1_decode(src, rgba[k]); src += 8; }
      }
      for (int k = 0; k < OR_SH; k++)
        for (int tt = 0; tt < 16; tt++) {
          int u, c;
          or_layout_map(layout, k, tt, &u, &c);
          int32_t o = perm[16 * g + u];
          if (o < 0) continue;
          for (int ch = 0; ch < 3; ch++) texels[((int64_t)o * OR_SH + c) * 3 + ch] = rgba[k][4 * tt + ch];
        }
    }
  }
  return 0;
}

/* Fixed coding of a layout (Sec. IV-B, Table I): j = bc7_blocks of each group's blocks in
 * BC7 (which ones: or_layout_bc7), the rest in BC1, one stream; each group's bytes are its
 * BC7 blocks then its BC1 blocks, in block order. The slot order is the caller's. */
int or_encode_layout(const uint8_t* q, int64_t n, const int32_t* perm, const float* scales, int layout,
                     int bc7_blocks, uint8_t* blocks, or_table* t) {
  if (!or_layout_ok(layout, bc7_blocks)) return -1;
  int64_t ng = (n + 15) / 16;
  const int j = bc7_blocks;
  const int64_t gbytes = 16 * j + 8 * (16 - j);
  memset(t, 0, sizeof(*t));
  t->n = n; t->n_groups = ng; t->layout = layout;
  t->format = j == 16 ? 7 : (j == 0 ? 1 : 2);
  for (int k = 0; k < OR_SH; k++) t->scales[k] = scales[k];
  or_weights(scales, t->weights);
  uint8_t tex[16 * 16 * 3];
  for (int64_t g = 0; g < ng; g++) {
    or_stage_layout(q, perm, layout, g, tex);
    uint8_t* dst = blocks + g * gbytes;
    for (int k = 0; k < OR_SH; k++)
      if (or_layout_bc7(layout, j, k)) { or_bc7_encode(tex + 48 * k, dst); dst += 16; }
    for (int k = 0; k < OR_SH; k++)
      if (!or_layout_bc7(layout, j, k)) { or_bc1_encode(tex + 48 * k, dst); dst += 8; }
  }
  t->n_streams = 1;
  t->s[0].bands = 16; t->s[0].bc7_blocks = j;
  t->s[0].first_group = 0; t->s[0].n_groups = ng; t->s[0].byte_offset = 0;
  t->total_bytes = ng * gbytes;
  t->used_bits = (uint64_t)t->total_bytes * 8;
  return 0;
}

/* ------------------------------------------------------------------------- */
/* SH evaluation (Sec. II, c(f) = H w(f - p)).                                */
/* Real SH to degree 3, k = l*l + l + m, with the Condon-Shortley phase inside   */
/* the associated Legendre function:                                          */
/*   m > 0: sqrt(2) K_l^m P_l^m(cos t) cos(m phi); m = 0: K_l^0 P_l(cos t);       */
/*   m < 0: sqrt(2) K_l^|m| P_l^|m|(cos t) sin(|m| phi),                          */
/*   K_l^m = sqrt((2l + 1) / (4 pi) * (l - m)! / (l + m)!).                       */
/* ------------------------------------------------------------------------- */
static double fact(int n) { double f = 1.0; for (int i = 2; i <= n; i++) f *= i; return f; }

static double assoc_legendre(int l, int m, double z) { /* m >= 0, includes (-1)^m */
  double pmm = 1.0, s = sqrt((1.0 - z) * (1.0 + z));
  for (int i = 1; i <= m; i++) pmm *= -(2.0 * i - 1.0) * s;
  if (l == m) return pmm;
  double pm1 = z * (2.0 * m + 1.0) * pmm;
  if (l == m + 1) return pm1;
  double pl = 0.0;
  for (int ll = m + 2; ll <= l; ll++) {
    pl = ((2.0 * ll - 1.0) * z * pm1 - (ll + m - 1.0) * pmm) / (ll - m);
    pmm = pm1; pm1 = pl;
  }
  return pl;
}

/* Sec. II: the real SH basis to degree 3 at a unit direction. */
void or_sh_basis(double x, double y, double z, double* Y) {
  const double PI = 3.14159265358979323846;
  double phi = atan2(y, x);
  for (int l = 0; l <= 3; l++)
    for (int m = -l; m <= l; m++) {
      int am = m < 0 ? -m : m;
      double K = sqrt((2.0 * l + 1.0) / (4.0 * PI) * fact(l - am) / fact(l + am));
      double P = assoc_legendre(l, am, z);
      double v;
      if (m > 0) v = sqrt(2.0) * K * P * cos(am * phi);
      else if (m < 0) v = sqrt(2.0) * K * P * sin(am * phi);
      else v = K * P;
      Y[l * l + l + m] = v;
    }
}

/* Sec. II, c(f) = H w(f - p).
 * out[v][i][c] = sum_k x'_{i,k,c} Y_k(d), x' = (q - 128) / 255 * s_k, with d the unit
 * direction dirs[v] (shared) or (cams[v] - pos[i]) / |cams[v] - pos[i]|; a zero
 * vector takes d = (0, 0, 1). abs_sum receives sum_k |x' Y_k(d)| for tolerances. */
void or_eval_sh(const uint8_t* texels, int64_t n, const float* scales, const float* pos,
                const float* dirs, const float* cams, int V, double* out, double* abs_sum) {
  double Y[16];
  for (int v = 0; v < V; v++)
    for (int64_t i = 0; i < n; i++) {
      double d[3];
      if (dirs) {
        for (int a = 0; a < 3; a++) d[a] = dirs[3 * v + a];
      } else {
        for (int a = 0; a < 3; a++) d[a] = (double)cams[3 * v + a] - (double)pos[3 * i + a];
      }
      double nn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      if (nn == 0.0) { d[0] = 0.0; d[1] = 0.0; d[2] = 1.0; }
      else for (int a = 0; a < 3; a++) d[a] /= nn;
      or_sh_basis(d[0], d[1], d[2], Y);
      for (int c = 0; c < 3; c++) {
        double acc = 0.0, aa = 0.0;
        for (int k = 0; k < OR_SH; k++) {
          double x = ((double)texels[(i * OR_SH + k) * 3 + c] - 128.0) / 255.0 * (double)scales[k];
          acc += x * Y[k];
          aa += fabs(x * Y[k]);
        }
        out[((int64_t)v * n + i) * 3 + c] = acc;
        if (abs_sum) abs_sum[((int64_t)v * n + i) * 3 + c] = aa;
      }
    }
}

/* ------------------------------------------------------------------------- */
/* Splatting renderer (Sec. II: Eq. sigmoid, Eq. covar, Eq. opac, Eq. blend /   */
/* Eq. preblend with the premultiplied H~ of Eq. premult; Fig. GSRend).         */
/* The paper gives the 3-D opacity g(x) of Eq. opac; the screen-space form here */
/* is the EWA splat of the cited method: the Gaussian projected with the       */
/* Jacobian of the pinhole projection at its centre, plus a 0.3 px^2 low-pass,  */
/* and limited to the 16 x 16 pixel tiles that its 3-sigma square touches.      */
/* Every decision (culling, tile rectangle, depth order) is taken in float      */
/* with the fixed operation order below, so that every implementation takes it */
/* the same way; the blending itself is accumulated in double.                 */
/* ------------------------------------------------------------------------- */
void or_camera_centre(const or_camera* cam, float* f) {
  for (int k = 0; k < 3; k++) {
    double v = ((double)cam->R[k] * cam->t[0] + (double)cam->R[3 + k] * cam->t[1]) + (double)cam->R[6 + k] * cam->t[2];
    f[k] = (float)(-v);
  }
}

/* Sec. II, Eq. covar, Fig. GSRend: the screen-space splat of one Gaussian. */
int or_splat_setup(const float* p, const float* s, const float* q, const or_camera* cam, or_splat* o) {
  const float* R = cam->R;
  memset(o, 0, sizeof(*o));
  /* camera coordinates */
  float x = ((R[0] * p[0] + R[1] * p[1]) + R[2] * p[2]) + cam->t[0];
  float y = ((R[3] * p[0] + R[4] * p[1]) + R[5] * p[2]) + cam->t[1];
  float z = ((R[6] * p[0] + R[7] * p[1]) + R[8] * p[2]) + cam->t[2];
  if (!(z > cam->near_z)) return 0;
  /* Eq. covar: Sigma = R(q) D(s) D(s)^T R(q)^T, q = (w, x, y, z) normalised */
  float nq = sqrtf(((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3]);
  if (!(nq > 0.0f)) return 0;
  float qw = q[0] / nq, qx = q[1] / nq, qy = q[2] / nq, qz = q[3] / nq;
  float r[9];
  r[0] = 1.0f - 2.0f * (qy * qy + qz * qz); r[1] = 2.0f * (qx * qy - qw * qz); r[2] = 2.0f * (qx * qz + qw * qy);
  r[3] = 2.0f * (qx * qy + qw * qz); r[4] = 1.0f - 2.0f * (qx * qx + qz * qz); r[5] = 2.0f * (qy * qz - qw * qx);
  r[6] = 2.0f * (qx * qz - qw * qy); r[7] = 2.0f * (qy * qz + qw * qx); r[8] = 1.0f - 2.0f * (qx * qx + qy * qy);
  float m[9];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) m[3 * i + j] = r[3 * i + j] * s[j];
  float S[9];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) S[3 * i + j] = (m[3 * i] * m[3 * j] + m[3 * i + 1] * m[3 * j + 1]) + m[3 * i + 2] * m[3 * j + 2];
  /* Jacobian of (fx x / z + cx, fy y / z + cy) at the centre, times the view rotation */
  float iz = 1.0f / z;
  float J[6] = {cam->fx * iz, 0.0f, -(cam->fx * x) * (iz * iz), 0.0f, cam->fy * iz, -(cam->fy * y) * (iz * iz)};
  float T[6];
  for (int a = 0; a < 2; a++)
    for (int j = 0; j < 3; j++) T[3 * a + j] = (J[3 * a] * R[j] + J[3 * a + 1] * R[3 + j]) + J[3 * a + 2] * R[6 + j];
  float U[6];
  for (int a = 0; a < 2; a++)
    for (int j = 0; j < 3; j++) U[3 * a + j] = (T[3 * a] * S[j] + T[3 * a + 1] * S[3 + j]) + T[3 * a + 2] * S[6 + j];
  float c00 = (U[0] * T[0] + U[1] * T[1]) + U[2] * T[2];
  float c01 = (U[0] * T[3] + U[1] * T[4]) + U[2] * T[5];
  float c11 = (U[3] * T[3] + U[4] * T[4]) + U[5] * T[5];
  float a = c00 + 0.3f, b = c01, c = c11 + 0.3f;
  float det = a * c - b * b;
  if (!(det > 0.0f)) return 0;
  float mid = 0.5f * (a + c);
  float disc = mid * mid - det;
  float lam = mid + sqrtf(disc > 0.1f ? disc : 0.1f);
  float rad = ceilf(3.0f * sqrtf(lam));
  float u = cam->fx * (x / z) + cam->cx, v = cam->fy * (y / z) + cam->cy;
  int tx = (cam->width + 15) / 16, ty = (cam->height + 15) / 16;
  float fx0 = floorf((u - rad) / 16.0f), fx1 = floorf((u + rad) / 16.0f) + 1.0f;
  float fy0 = floorf((v - rad) / 16.0f), fy1 = floorf((v + rad) / 16.0f) + 1.0f;
  int x0 = fx0 < 0.0f ? 0 : (fx0 > (float)tx ? tx : (int)fx0), x1 = fx1 < 0.0f ? 0 : (fx1 > (float)tx ? tx : (int)fx1);
  int y0 = fy0 < 0.0f ? 0 : (fy0 > (float)ty ? ty : (int)fy0), y1 = fy1 < 0.0f ? 0 : (fy1 > (float)ty ? ty : (int)fy1);
  if (x1 <= x0 || y1 <= y0) return 0;
  o->u = u; o->v = v; o->depth = z;
  o->a = a; o->b = b; o->c = c;
  o->x0 = x0; o->y0 = y0; o->x1 = x1; o->y1 = y1;
  o->visible = 1;
  return 1;
}

typedef struct { uint32_t depth_bits; int64_t i; } depth_key;
static int cmp_depth(const void* pa, const void* pb) {
  const depth_key* a = (const depth_key*)pa;
  const depth_key* b = (const depth_key*)pb;
  if (a->depth_bits != b->depth_bits) return a->depth_bits < b->depth_bits ? -1 : 1;
  return a->i < b->i ? -1 : (a->i > b->i ? 1 : 0);
}

/* Eq. preblend, pixel (x, y) with centre (x + 0.5, y + 0.5): a = sum_i g_i c~_i prod_{j<i} (1 - mu_j g_j)
 * over the Gaussians whose tile rectangle holds the pixel's tile, nearest first (camera depth, then
 * index); c~ = H~ w(f - p) is the premultiplied colour (Eq. premult), mu = sigmoid(t) (Eq. sigmoid).
 * tiles: the tile ids (ty * tiles_x + tx) to render, or NULL for all. trans gets the final
 * prod (1 - mu g); abs_sum the sum of |g c~ prod| per channel (for error bounds). */
int or_render(int64_t n, const float* pos, const float* scale, const float* rot, const float* logit,
              const double* colour, const or_camera* cam, const int32_t* tiles, int64_t n_tiles, double* image,
              double* trans, double* abs_sum) {
  const int W = cam->width, H = cam->height, tx = (W + 15) / 16, ty = (H + 15) / 16;
  or_splat* sp = (or_splat*)malloc(sizeof(or_splat) * (size_t)(n > 0 ? n : 1));
  depth_key* list = (depth_key*)malloc(sizeof(depth_key) * (size_t)(n > 0 ? n : 1));
  if (!sp || !list) { free(sp); free(list); return -1; }
  for (int64_t i = 0; i < n; i++) or_splat_setup(pos + 3 * i, scale + 3 * i, rot + 4 * i, cam, &sp[i]);
  int64_t nt = tiles ? n_tiles : (int64_t)tx * ty;
  for (int64_t ti = 0; ti < nt; ti++) {
    int tile = tiles ? tiles[ti] : (int)ti;
    int bx = tile % tx, by = tile / tx;
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++) {
      const or_splat* g = &sp[i];
      if (g->visible && bx >= g->x0 && bx < g->x1 && by >= g->y0 && by < g->y1) {
        uint32_t bits;
        memcpy(&bits, &g->depth, 4);
        list[m].depth_bits = bits; list[m].i = i; m++;
      }
    }
    qsort(list, (size_t)m, sizeof(depth_key), cmp_depth);
    for (int py = by * 16; py < by * 16 + 16 && py < H; py++)
      for (int px = bx * 16; px < bx * 16 + 16 && px < W; px++) {
        double T = 1.0, acc[3] = {0.0, 0.0, 0.0}, ab[3] = {0.0, 0.0, 0.0};
        for (int64_t k = 0; k < m; k++) {
          const int64_t i = list[k].i;
          const or_splat* g = &sp[i];
          double a = g->a, b = g->b, c = g->c;
          double det = a * c - b * b;
          double ca = c / det, cb = -b / det, cc = a / det;
          double dx = (px + 0.5) - (double)g->u, dy = (py + 0.5) - (double)g->v;
          double gv = exp(-0.5 * (ca * dx * dx + cc * dy * dy) - cb * dx * dy);
          double mu = 1.0 / (1.0 + exp(-(double)logit[i]));
          for (int ch = 0; ch < 3; ch++) {
            double term = gv * colour[3 * i + ch] * T;
            acc[ch] += term;
            ab[ch] += fabs(term);
          }
          T *= 1.0 - mu * gv;
        }
        int64_t pix = (int64_t)py * W + px;
        for (int ch = 0; ch < 3; ch++) {
          image[3 * pix + ch] = acc[ch];
          if (abs_sum) abs_sum[3 * pix + ch] = ab[ch];
        }
        if (trans) trans[pix] = T;
      }
  }
  free(sp);
  free(list);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Geometry streams and the chunk hierarchy (Sec. IV-A: position and shape are  */
/* coded apart from appearance, each parameter simply quantised to a fixed     */
/* number of bits and kept in its own fixed-rate bitstream; a hierarchical     */
/* organisation lets a view use only the primitives of the part it sees).      */
/* Readings (the paper gives no bit allocation): slot order (positions move    */
/* with the Gaussians, so no index is stored); chunks of C consecutive slots;  */
/* per chunk the bounding box of its centres and its largest scale; position   */
/* 3 x 16 bits over the chunk box; scale 3 x bfloat16; rotation as the        */
/* "smallest three" of the unit quaternion (2-bit index of the largest         */
/* component, made positive, and three 10-bit codes of 1022 steps over         */
/* [-1/sqrt2, 1/sqrt2]); opacity logit 8 bits over [-8, 8]. 17 bytes per slot.  */
/* ------------------------------------------------------------------------- */
static uint16_t bf16_rne(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
static float bf16_val(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float x;
  memcpy(&x, &u, 4);
  return x;
}
static uint32_t quant_unit(float t, float levels) { /* round(t * levels), t clamped to [0, 1] */
  float c = t < 0.0f ? 0.0f : (t > 1.0f ? 1.0f : t);
  return (uint32_t)rintf(c * levels);
}

int64_t or_chunks(int64_t n_slots, int64_t chunk_slots) { return (n_slots + chunk_slots - 1) / chunk_slots; }

/* Sec. IV-A. chunk[c] = lo[3], hi[3] (bounds of the chunk's centres), largest decoded scale, 0; a chunk of
 * padding slots only is all zero */
void or_chunk_table(const float* pos, const float* scale, const int32_t* perm, int64_t n_slots, int64_t chunk_slots,
                    float* chunk) {
  int64_t nc = or_chunks(n_slots, chunk_slots);
  for (int64_t c = 0; c < nc; c++) {
    float* e = chunk + 8 * c;
    int any = 0;
    for (int a = 0; a < 8; a++) e[a] = 0.0f;
    for (int64_t s = c * chunk_slots; s < (c + 1) * chunk_slots && s < n_slots; s++) {
      int32_t o = perm[s];
      if (o < 0) continue;
      for (int a = 0; a < 3; a++) {
        float p = pos[3 * (int64_t)o + a];
        float sv = bf16_val(bf16_rne(scale[3 * (int64_t)o + a]));
        if (!any || p < e[a]) e[a] = p;
        if (!any || p > e[3 + a]) e[3 + a] = p;
        if ((!any && a == 0) || sv > e[6]) e[6] = sv;
      }
      any = 1;
    }
  }
}

/* Codes of slot s (Gaussian o = perm[s]) into the streams; padding slots get zero codes. */
void or_geometry_encode(const float* pos, const float* scale, const float* rot, const float* logit,
                        const int32_t* perm, int64_t n_slots, int64_t chunk_slots, const float* chunk,
                        uint16_t* qpos, uint16_t* qscale, uint32_t* qrot, uint8_t* qlogit) {
  for (int64_t s = 0; s < n_slots; s++) {
    int32_t o = perm[s];
    if (o < 0) {
      for (int a = 0; a < 3; a++) { qpos[3 * s + a] = 0; qscale[3 * s + a] = 0; }
      qrot[s] = 0; qlogit[s] = 0;
      continue;
    }
    const float* e = chunk + 8 * (s / chunk_slots);
    for (int a = 0; a < 3; a++) {
      float ext = e[3 + a] - e[a];
      float t = ext > 0.0f ? (pos[3 * (int64_t)o + a] - e[a]) / ext : 0.0f;
      qpos[3 * s + a] = (uint16_t)quant_unit(t, 65535.0f);
      qscale[3 * s + a] = bf16_rne(scale[3 * (int64_t)o + a]);
    }
    /* smallest three: normalise, largest |component| first on ties, made non-negative */
    const float* q = rot + 4 * (int64_t)o;
    float nq = sqrtf(((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3]);
    float u[4];
    for (int a = 0; a < 4; a++) u[a] = nq > 0.0f ? q[a] / nq : (a == 0 ? 1.0f : 0.0f);
    int m = 0;
    for (int a = 1; a < 4; a++) if (fabsf(u[a]) > fabsf(u[m])) m = a;
    float sg = u[m] < 0.0f ? -1.0f : 1.0f;
    uint32_t code = (uint32_t)m, sh = 2;
    for (int a = 0; a < 4; a++) {
      if (a == m) continue;
      float c = sg * u[a];                                 /* in [-1/sqrt2, 1/sqrt2] */
      float t = c * 0.70710678f + 0.5f;                    /* [-1/sqrt2, 1/sqrt2] -> [0, 1] */
      code |= quant_unit(t, 1022.0f) << sh;                /* 1022 steps: 0 is code 511 exactly */
      sh += 10;
    }
    qrot[s] = code;
    float lt = (logit[o] + 8.0f) / 16.0f;
    qlogit[s] = (uint8_t)quant_unit(lt, 255.0f);
  }
}

/* Decoded geometry of slot s in float, with the fixed operation order every decoder uses. */
void or_geometry_decode_slot(const uint16_t* qpos, const uint16_t* qscale, const uint32_t* qrot, const uint8_t* qlogit,
                             int64_t s, int64_t chunk_slots, const float* chunk, float* p, float* sc, float* q,
                             float* t) {
  const float* e = chunk + 8 * (s / chunk_slots);
  for (int a = 0; a < 3; a++) {
    float ext = e[3 + a] - e[a];
    p[a] = e[a] + ((float)qpos[3 * s + a] / 65535.0f) * ext;
    sc[a] = bf16_val(qscale[3 * s + a]);
  }
  uint32_t code = qrot[s];
  int m = (int)(code & 3u);
  float ss = 0.0f;
  int sh = 2;
  for (int a = 0; a < 4; a++) {
    if (a == m) continue;
    float c = (((float)((code >> sh) & 1023u) / 1022.0f) - 0.5f) * 1.41421356f;
    q[a] = c;
    ss = ss + c * c;
    sh += 10;
  }
  float r = 1.0f - ss;
  q[m] = sqrtf(r > 0.0f ? r : 0.0f);
  *t = ((float)qlogit[s] / 255.0f) * 16.0f - 8.0f;
}

/* Sec. IV-A, Fig. FileHier.
 * Chunk visibility (a reading of the hierarchy's view test): a chunk is kept unless its box of
 * centres, grown by 6 times its largest scale, lies entirely at camera depth <= near_z / 2, or is
 * entirely in front of the camera and projects entirely beyond one image side by more than
 * 64 pixels. Corners are projected in float with a fixed operation order. */
int or_chunk_visible(const float* e, const or_camera* cam) {
  float g = 6.0f * e[6];
  const float* R = cam->R;
  int behind = 1, front = 1, left = 1, right = 1, top = 1, bottom = 1;
  float W = (float)cam->width, H = (float)cam->height;
  for (int k = 0; k < 8; k++) {
    float c[3];
    for (int a = 0; a < 3; a++) c[a] = ((k >> a) & 1) ? e[3 + a] + g : e[a] - g;
    float x = ((R[0] * c[0] + R[1] * c[1]) + R[2] * c[2]) + cam->t[0];
    float y = ((R[3] * c[0] + R[4] * c[1]) + R[5] * c[2]) + cam->t[1];
    float z = ((R[6] * c[0] + R[7] * c[1]) + R[8] * c[2]) + cam->t[2];
    if (z > 0.5f * cam->near_z) behind = 0;
    if (!(z > 0.5f * cam->near_z)) { front = 0; continue; }
    float u = cam->fx * (x / z) + cam->cx, v = cam->fy * (y / z) + cam->cy;
    if (!(u < -64.0f)) left = 0;
    if (!(u > W + 64.0f)) right = 0;
    if (!(v < -64.0f)) top = 0;
    if (!(v > H + 64.0f)) bottom = 0;
  }
  if (behind) return 0;
  if (front && (left || right || top || bottom)) return 0;
  return 1;
}

/* Every slot's decoded geometry (or_geometry_decode_slot for s = 0 .. n_slots - 1). */
void or_geometry_decode_all(const uint16_t* qpos, const uint16_t* qscale, const uint32_t* qrot, const uint8_t* qlogit,
                            int64_t n_slots, int64_t chunk_slots, const float* chunk, float* p, float* sc, float* q,
                            float* t) {
  for (int64_t s = 0; s < n_slots; s++)
    or_geometry_decode_slot(qpos, qscale, qrot, qlogit, s, chunk_slots, chunk, p + 3 * s, sc + 3 * s, q + 4 * s, t + s);
}
