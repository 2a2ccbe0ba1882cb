// bc7.cu -- BC7 encoder (Sec. III-B; D3D11 / Khronos BC7 format).
//
// One thread per block; the 32 lanes of a warp walk the same candidate enumeration
// on 32 different blocks, so the partition of the current candidate is warp-uniform
// (constant-cache broadcast) and so is almost every branch. Texels sit in registers.
//
// The search is the codec's own deterministic integer encoder. Candidates, in order:
// mode 0 partitions 0..15; modes 1, 2, 3 partitions 0..63; mode 4 rotation 0..3 x
// index selection 0..1; mode 5 rotation 0..3; mode 6; mode 7 partitions 0..63. For
// each subset: bounding-box diagonal oriented by covariance signs, indices against the
// unquantised palette, one least-squares refinement, then every p-bit combination
// quantised to the nearest codes and re-indexed; the best combination (lowest squared
// error, first on ties) scores the subset. The block takes the first candidate of
// least total error; the winner is solved again, anchors are fixed losslessly by
// swapping endpoints and inverting indices, and the fields are packed LSB first.
#include "bc1_dev.cuh"
#include "bc7_tables.h"
#include "gsc_internal.cuh"
#include "stage.cuh"

__constant__ uint32_t c_part2[64];
__constant__ uint32_t c_part3[64];
__constant__ uint8_t c_anc2[64];
__constant__ uint8_t c_anc3a[64];
__constant__ uint8_t c_anc3b[64];
// nearest endpoint code per 8-bit target: code | expanded value << 8, 12 configurations
__device__ uint16_t g_qtab[12][256];
// constant blocks: per 8-bit value the 7-bit code pair a | b << 8 of mode 5 at weight 21
__constant__ uint16_t c_const7[256];
// three-subset member sets: per (partition, subset) the index of its member set among the distinct
// sets in enumeration order, | 0x100 where that set occurs first (its fit is computed there)
#define BC7_SUB3_SETS 140
__constant__ uint16_t c_sub3[64 * 3];
// member texels of each subset of the two- and three-subset partitions: texel indices in
// increasing order, four bits each from bit 0, and the member count in bits 60-63
__constant__ uint64_t c_mem2[64][2];
__constant__ uint64_t c_mem3[64][3];
// prefits shared across modes: a member set of the first 16 three-subset partitions that is also
// a two-subset member set has the same 3-bit prefit in modes 0 and 1, and one of the 64
// three-subset partitions the same 2-bit prefit in modes 2 and 3/7. Per three-subset subset the
// slot its mode 0 (mode 2) fit stores its prefit in, per two-subset subset the slot its mode 1
// (modes 3/7) fit reads it from; -1 where there is none.
#define BC7_PF3_SLOTS 14
#define BC7_PF_SLOTS 40
__constant__ int8_t c_pf3b[64][3];  // 3-bit: mode 0 store slot
__constant__ int8_t c_pf3a[64][3];  // 2-bit: mode 2 store slot
__constant__ int8_t c_pf2b[64][2];  // 3-bit: mode 1 read slot
__constant__ int8_t c_pf2a[64][2];  // 2-bit: modes 3/7 read slot
cudaError_t bc7_kernel_attributes();

static int h_expand(int v, int n) { return n >= 8 ? v : ((v << (8 - n)) | (v >> (2 * n - 8))); }

cudaError_t bc7_init_tables() {
  uint32_t p2[64], p3[64];
  uint8_t a2[64], a3a[64], a3b[64];
  for (int p = 0; p < 64; p++) {
    p2[p] = bc7_pack_part2(p);
    p3[p] = bc7_pack_part3(p);
    a2[p] = kBC7Anchor2[p];
    a3a[p] = kBC7Anchor3a[p];
    a3b[p] = kBC7Anchor3b[p];
  }
  static const int cfg[12][3] = {{4, 1, 0}, {4, 1, 1}, {5, 0, 0}, {5, 1, 0}, {5, 1, 1}, {6, 0, 0},
                                 {6, 1, 0}, {6, 1, 1}, {7, 0, 0}, {7, 1, 0}, {7, 1, 1}, {8, 0, 0}};
  static uint16_t q[12][256];
  for (int c = 0; c < 12; c++) {
    int bits = cfg[c][0], hp = cfg[c][1], pb = cfg[c][2];
    for (int e = 0; e < 256; e++) {
      int best = 0, be = -1, bv = 0;
      for (int code = 0; code < (1 << bits); code++) {
        int v = h_expand(hp ? (code << 1) | pb : code, bits + hp);
        int d = abs(v - e);
        if (be < 0 || d < be) { be = d; best = code; bv = v; }
      }
      q[c][e] = (uint16_t)(best | (bv << 8));
    }
  }
  // Constant blocks: every 8-bit value v is ((64 - 21) ex7(a) + 21 ex7(b) + 32) >> 6 for some 7-bit
  // pair; the first with a outer and b inner is taken.
  uint16_t c7[256];
  for (int v = 0; v < 256; v++) {
    c7[v] = 0;
    bool found = false;
    for (int a = 0; a < 128 && !found; a++)
      for (int b = 0; b < 128 && !found; b++)
        if (((64 - 21) * h_expand(a, 7) + 21 * h_expand(b, 7) + 32) >> 6 == v) { c7[v] = (uint16_t)(a | (b << 8)); found = true; }
  }
  // A subset's fit depends only on its member texels. Partitions enumerated in order, subsets in
  // order: the first subset with a given member set is fitted, later ones reuse its error.
  uint16_t sub3[64 * 3];
  uint32_t sets[64 * 3];
  int n_sets = 0;
  for (int pp = 0; pp < 64; pp++)
    for (int sb = 0; sb < 3; sb++) {
      const uint32_t x = p3[pp] ^ ((uint32_t)sb * 0x55555555u);
      const uint32_t m = ~(x | (x >> 1)) & 0x55555555u;
      int id = -1;
      for (int k = 0; k < n_sets; k++)
        if (sets[k] == m) { id = k; break; }
      if (id < 0) {
        if (n_sets == BC7_SUB3_SETS) return cudaErrorInvalidValue;
        id = n_sets;
        sets[n_sets++] = m;
        sub3[3 * pp + sb] = (uint16_t)(id | 0x100);
      } else {
        sub3[3 * pp + sb] = (uint16_t)id;
      }
    }
  uint64_t mem2[64][2], mem3[64][3];
  for (int pp = 0; pp < 64; pp++)
    for (int ns = 2; ns <= 3; ns++)
      for (int sb = 0; sb < ns; sb++) {
        const uint32_t part = ns == 2 ? p2[pp] : p3[pp];
        uint64_t list = 0;
        int cnt = 0;
        for (int t = 0; t < 16; t++)
          if (((part >> (2 * t)) & 3u) == (uint32_t)sb) list |= (uint64_t)t << (4 * cnt++);
        if (cnt > 15) return cudaErrorInvalidValue;
        list |= (uint64_t)cnt << 60;
        if (ns == 2) mem2[pp][sb] = list; else mem3[pp][sb] = list;
      }
  // shared prefit slots: 3-bit (mode 0 -> mode 1) first, then 2-bit (mode 2 -> modes 3/7), each
  // set stored by its first subset in enumeration order
  int8_t pf3b[64][3], pf3a[64][3], pf2b[64][2], pf2a[64][2];
  memset(pf3b, -1, sizeof(pf3b)); memset(pf3a, -1, sizeof(pf3a));
  memset(pf2b, -1, sizeof(pf2b)); memset(pf2a, -1, sizeof(pf2a));
  {
    auto set_of = [](uint32_t part, int sb) {
      uint32_t m = 0;
      for (int t = 0; t < 16; t++) if (((part >> (2 * t)) & 3u) == (uint32_t)sb) m |= 1u << t;
      return m;
    };
    int slots = 0;
    for (int kind = 0; kind < 2; kind++) {        // 0: 3-bit (modes 0 / 1), 1: 2-bit (modes 2 / 3, 7)
      const int np3 = kind == 0 ? 16 : 64;
      for (int pp = 0; pp < np3; pp++)
        for (int sb = 0; sb < 3; sb++) {
          const uint32_t m = set_of(p3[pp], sb);
          bool first = true;
          for (int q = 0; q < pp * 3 + sb && first; q++) first = set_of(p3[q / 3], q % 3) != m;
          if (!first) continue;
          int found = 0;
          for (int p2i = 0; p2i < 64; p2i++)
            for (int s2 = 0; s2 < 2; s2++)
              if (set_of(p2[p2i], s2) == m) {
                if (!found) {
                  if (slots == BC7_PF_SLOTS) return cudaErrorInvalidValue;
                  (kind == 0 ? pf3b : pf3a)[pp][sb] = (int8_t)slots;
                  found = 1;
                }
                (kind == 0 ? pf2b : pf2a)[p2i][s2] = (int8_t)slots;
              }
          slots += found;
        }
      if (kind == 0 && slots != BC7_PF3_SLOTS) return cudaErrorInvalidValue;
    }
    if (slots != BC7_PF_SLOTS) return cudaErrorInvalidValue;
  }
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_pf3b, pf3b, sizeof(pf3b))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_pf3a, pf3a, sizeof(pf3a))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_pf2b, pf2b, sizeof(pf2b))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_pf2a, pf2a, sizeof(pf2a))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_mem2, mem2, sizeof(mem2))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_mem3, mem3, sizeof(mem3))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_sub3, sub3, sizeof(sub3))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_const7, c7, sizeof(c7))) != cudaSuccess) return e;
  uint16_t t5[256], t6[256];
  bc1_const_tables(t5, t6);
  if ((e = cudaMemcpyToSymbol(c_const5, t5, sizeof(t5))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_const6, t6, sizeof(t6))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_part2, p2, sizeof(p2))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_part3, p3, sizeof(p3))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_anc2, a2, sizeof(a2))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_anc3a, a3a, sizeof(a3a))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_anc3b, a3b, sizeof(a3b))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(g_qtab, q, sizeof(q))) != cudaSuccess) return e;
  return bc7_kernel_attributes();
}

// table ids: (bits, p-bit present, p)
__host__ __device__ constexpr int qid(int bits, int hp, int p) {
  return bits == 4 ? p : bits == 5 ? (hp ? 3 + p : 2) : bits == 6 ? (hp ? 6 + p : 5) : bits == 7 ? (hp ? 9 + p : 8) : 11;
}

enum { PT_NONE = 0, PT_UNIQUE = 1, PT_SHARED = 2 };

template <int IB> __device__ __forceinline__ int wgt(int j) {
  if (IB == 2) return (0x402B1500u >> (8 * j)) & 255;              // 0, 21, 43, 64
  if (IB == 3) return (int)((0x40372E251B120900ull >> (8 * j)) & 255);  // 0 9 18 27 37 46 55 64
  // 0 4 9 13 17 21 26 30 34 38 43 47 51 55 60 64
  return j < 8 ? (int)((0x1E1A15110D090400ull >> (8 * j)) & 255) : (int)((0x403C37332F2B2622ull >> (8 * (j - 8))) & 255);
}
__device__ __forceinline__ int interp64(int e0, int e1, int w) { return ((64 - w) * e0 + w * e1 + 32) >> 6; }
__device__ __forceinline__ int chan(uint32_t v, int c) { return (v >> (8 * c)) & 255; }

struct FitOut {
  int code[2][3];  // per endpoint, per channel R, G, B (unused channels untouched)
  int p[2];
  uint32_t idx_lo, idx_hi;  // 4 bits per texel, texel t at bits 4t of the 64-bit pair
};

// Texels of the thread's block: tex[t * STAGE_STRIDE], packed r | g << 8 | b << 16 (top byte 0).
// Palette search (exact): with pk_j = 16 |p_j|^2 + j, the key pk_j - 32 dot(v, p_j) equals
// 16 (|v - p_j|^2 - |v|^2) + j, so its minimum gives the first index of least error
// (key & 15) and that error minus |v|^2 (key >> 4, an exact floor shift).
__device__ __forceinline__ uint32_t pack_rgb(int r, int g, int b) { return (uint32_t)r | ((uint32_t)g << 8) | ((uint32_t)b << 16); }

// Palette of F entries between endpoints a and b (R, G, B; uncoded channels 0) with BC7 weights,
// and its keys. Two channels share one multiply-add in 16-bit lanes scaled by 4, so byte 1 of
// each lane is ((64 - w) a + w b + 32) >> 6 exactly.
// IDX: keys 16 |entry|^2 + j (the index j in the low bits picks the first of equal errors);
// otherwise |entry|^2 alone (when only the least error matters).
template <int IB, bool IDX = true>
__device__ __forceinline__ void build_pal(const int (&a)[3], const int (&b)[3], uint32_t (&pal)[1 << IB],
                                          int (&pk)[1 << IB]) {
  const uint32_t A = ((uint32_t)a[0] | ((uint32_t)a[1] << 16)) << 2, B = ((uint32_t)b[0] | ((uint32_t)b[1] << 16)) << 2;
  const uint32_t Ab = (uint32_t)a[2] << 2, Bb = (uint32_t)b[2] << 2;
  // (64 - w) A + w B = 64 A + w (B - A): with B - A formed in 32-bit arithmetic a lane may be
  // negative, but each lane's result lies in [0, 2^16), so the packed sum is exact
  const uint32_t rg0 = 64u * A + 0x00800080u, drg = B - A, bb0 = 64u * Ab + 0x80u, dbb = Bb - Ab;
#pragma unroll
  for (int j = 0; j < (1 << IB); j++) {
    const uint32_t w = (uint32_t)wgt<IB>(j);
    const uint32_t rg = rg0 + w * drg, bb = bb0 + w * dbb;
    pal[j] = __byte_perm(rg, bb, 0x7531u);
    pk[j] = IDX ? 16 * (int)__dp4a(pal[j], pal[j], 0u) + j : (int)__dp4a(pal[j], pal[j], 0u);
  }
}

template <int F, int SCALE = 32>
__device__ __forceinline__ int best_key(uint32_t v, const uint32_t (&pal)[F], const int (&pk)[F]) {
  int k[F];
#pragma unroll
  for (int j = 0; j < F; j++) k[j] = pk[j] - SCALE * (int)__dp4a(v, pal[j], 0u);
#pragma unroll
  for (int w = F / 2; w >= 1; w /= 2)
#pragma unroll
    for (int j = 0; j < w; j++) k[j] = min(k[j], k[j + w]);
  return k[0];
}

// The member texels of one subset: indices four bits each from bit 0, increasing, and their
// count (the same for every lane of a warp).
struct Mem {
  uint64_t list;
  int n;
};
__device__ __forceinline__ Mem mem_all() { return {0xFEDCBA9876543210ull, 16}; }
__device__ __forceinline__ Mem mem_of(int ns, int p, int s) {
  if (ns == 1) return mem_all();
  const uint64_t v = ns == 2 ? c_mem2[p][s] : c_mem3[p][s];
  return {v, (int)(v >> 60)};
}

// Stage 1 of a subset fit: bounding-box diagonal oriented by covariance signs, indices
// against the unquantised palette, one least-squares refinement. Returns the member count;
// sumsq gets the members' summed squared norms over the coded channels (the part of every
// palette error that does not depend on the palette).
// `sel` permutes each texel's bytes on load (identity by default); the rotation search uses it
// to move the rotated channel to byte 2, keeping the other two in their order.
template <int IB, int CHMASK>
__device__ __forceinline__ int prefit(const uint32_t* __restrict__ tex, Mem M, int (&e0)[3], int (&e1)[3],
                                      int& sumsq, uint32_t sel = 0x3210u) {
  constexpr int F = 1 << IB;
  constexpr int NCH = ((CHMASK >> 0) & 1) + ((CHMASK >> 1) & 1) + ((CHMASK >> 2) & 1);
  constexpr uint32_t CM = ((CHMASK & 1) ? 0xFFu : 0u) | ((CHMASK & 2) ? 0xFF00u : 0u) | ((CHMASK & 4) ? 0xFF0000u : 0u);
  int ch[3] = {0, 0, 0};
  {
    int k = 0;
#pragma unroll
    for (int c = 0; c < 3; c++) if ((CHMASK >> c) & 1) ch[k++] = c;
  }
  int n = 0, sq2 = 0, lo[NCH], hi[NCH], s1[NCH], s2[3];
#pragma unroll
  for (int i = 0; i < NCH; i++) { lo[i] = 255; hi[i] = 0; s1[i] = 0; }
  s2[0] = s2[1] = s2[2] = 0;  // channel pairs (0,1), (0,2), (1,2) of the coded channels
  // member texels only (the list is the same for every lane); box and sums are order-free, so
  // two texels per step: both shared-memory reads are in flight together
  auto box = [&](uint32_t v) {
    n++;
    sq2 += (int)__dp4a(v & CM, v & CM, 0u);
    int c[NCH];
#pragma unroll
    for (int i = 0; i < NCH; i++) {
      c[i] = (v >> (8 * ch[i])) & 255;
      lo[i] = min(lo[i], c[i]); hi[i] = max(hi[i], c[i]); s1[i] += c[i];
    }
    if (NCH >= 2) s2[0] += c[0] * c[NCH >= 2 ? 1 : 0];
    if (NCH >= 3) { s2[1] += c[0] * c[NCH >= 3 ? 2 : 0]; s2[2] += c[NCH >= 2 ? 1 : 0] * c[NCH >= 3 ? 2 : 0]; }
  };
  {
    uint64_t L = M.list;
    for (int i = 1; i < M.n; i += 2) {
      const int ta = (int)(L & 15), tb = (int)((L >> 4) & 15);
      L >>= 8;
      const uint32_t va = __byte_perm(tex[ta * STAGE_STRIDE], 0u, sel);
      const uint32_t vb = __byte_perm(tex[tb * STAGE_STRIDE], 0u, sel);
      box(va);
      box(vb);
    }
    if (M.n & 1) box(__byte_perm(tex[(int)(L & 15) * STAGE_STRIDE], 0u, sel));
  }
  sumsq = sq2;
  if (n == 0) return 0;
  // reference channel = widest range (first on ties); selects, not indexing, keep the
  // per-channel sums in registers
  int ref = 0, rw = hi[0] - lo[0], s1r = s1[0];
#pragma unroll
  for (int i = 1; i < NCH; i++)
    if (hi[i] - lo[i] > rw) { rw = hi[i] - lo[i]; ref = i; s1r = s1[i]; }
#pragma unroll
  for (int i = 0; i < NCH; i++) {
    // cross sum of channels i and ref: pairs (0,1), (0,2), (1,2) are s2[0], s2[1], s2[2]
    int cross;
    if (i == 0) cross = ref == 1 ? s2[0] : s2[1];
    else if (i == 1) cross = ref == 0 ? s2[0] : s2[2];
    else cross = ref == 0 ? s2[1] : s2[2];
    const bool flip = i != ref && (n * cross - s1r * s1[i]) < 0;
    e0[i] = flip ? lo[i] : hi[i];
    e1[i] = flip ? hi[i] : lo[i];
  }
  // least-squares sums over the member texels with weights a = 64 - w and w: only sums of w,
  // w^2 and w c are accumulated per texel; with n and the channel sums s1 of the box pass,
  // sum a^2 = 4096 n - 128 sum w + sum w^2, sum a w = 64 sum w - sum w^2, sum a c = 64 s1 - sum w c
  int sw = 0, sbb = 0, sbv[NCH];
  {
    uint32_t pal[F];
    int pk[F];
    {
      int a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
#pragma unroll
      for (int i = 0; i < NCH; i++) { a[ch[i]] = e0[i]; b[ch[i]] = e1[i]; }
      build_pal<IB>(a, b, pal, pk);
    }
#pragma unroll
    for (int i = 0; i < NCH; i++) sbv[i] = 0;
    auto accumulate = [&](uint32_t v, int key) {
      const int w = wgt<IB>(key & 15);
      sw += w; sbb += w * w;
#pragma unroll
      for (int i = 0; i < NCH; i++) sbv[i] += w * (int)((v >> (8 * ch[i])) & 255);
    };
    // two member texels per step (independent palette searches; integer sums, order-free)
    uint64_t L = M.list;
    for (int i = 1; i < M.n; i += 2) {
      const int ta = (int)(L & 15), tb = (int)((L >> 4) & 15);
      L >>= 8;
      // uncoded channels: their palette bytes are 0, so the products ignore those texel bytes
      const uint32_t va = __byte_perm(tex[ta * STAGE_STRIDE], 0u, sel);
      const uint32_t vb = __byte_perm(tex[tb * STAGE_STRIDE], 0u, sel);
      const int ka = best_key<F>(va, pal, pk), kb = best_key<F>(vb, pal, pk);
      accumulate(va, ka);
      accumulate(vb, kb);
    }
    if (M.n & 1) {
      const uint32_t va = __byte_perm(tex[(int)(L & 15) * STAGE_STRIDE], 0u, sel);
      accumulate(va, best_key<F>(va, pal, pk));
    }
  }
  const int saa = 4096 * n - 128 * sw + sbb, sab = 64 * sw - sbb;
  int sav[NCH];
#pragma unroll
  for (int i = 0; i < NCH; i++) sav[i] = 64 * s1[i] - sbv[i];
  const long long det = (long long)saa * sbb - (long long)sab * sab;
  if (det != 0) {
    const RoundDiv255 rd = round_div255_of(det);
#pragma unroll
    for (int i = 0; i < NCH; i++) {
      e0[i] = round_div255(rd, 64LL * ((long long)sbb * sav[i] - (long long)sab * sbv[i]));
      e1[i] = round_div255(rd, 64LL * ((long long)saa * sbv[i] - (long long)sab * sav[i]));
    }
  }
  return n;
}

// Stage 2: every p-bit combination quantised to the nearest codes and re-indexed; the best
// combination (first on ties) scores the subset.
template <int IB, int CHMASK, int PT, int BITS, bool OUT>
__device__ __forceinline__ uint32_t quant_eval(const uint32_t* __restrict__ tex, Mem M,
                                               const int (&e0)[3], const int (&e1)[3], int sumsq, FitOut* out,
                                               const uint16_t* __restrict__ sq, uint32_t sel = 0x3210u) {
  constexpr int F = 1 << IB;
  constexpr int NCH = ((CHMASK >> 0) & 1) + ((CHMASK >> 1) & 1) + ((CHMASK >> 2) & 1);
  int ch[3] = {0, 0, 0};
  {
    int k = 0;
#pragma unroll
    for (int c = 0; c < 3; c++) if ((CHMASK >> c) & 1) ch[k++] = c;
  }
  constexpr int NCOMBO = PT == PT_NONE ? 1 : (PT == PT_UNIQUE ? 4 : 2);
  constexpr int HP = PT == PT_NONE ? 0 : 1;
  // search form: the combinations' palettes built in chunks of at most 16 entries in all, and one
  // pass over the member texels per chunk evaluating every palette of it (each texel is loaded
  // once per chunk)
  constexpr int CH = (NCOMBO * F <= 16) ? NCOMBO : (2 * F <= 16 ? 2 : 1);
  if constexpr (!OUT && CH > 1) {
    uint32_t b = 0xFFFFFFFFu;
#pragma unroll
    for (int c0 = 0; c0 < NCOMBO; c0 += CH) {
      uint32_t pal[CH][F];
      int pk[CH][F], sse[CH];
#pragma unroll
      for (int u = 0; u < CH; u++) {
        const int cmb = c0 + u;
        const int p0 = PT == PT_UNIQUE ? (cmb & 1) : cmb;
        const int p1 = PT == PT_UNIQUE ? (cmb >> 1) : cmb;
        const uint16_t* q0 = sq + 256 * qid(BITS, HP, p0);
        const uint16_t* q1 = sq + 256 * qid(BITS, HP, p1);
        int v0[3] = {0, 0, 0}, v1[3] = {0, 0, 0};
#pragma unroll
        for (int i = 0; i < NCH; i++) { v0[ch[i]] = q0[e0[i]] >> 8; v1[ch[i]] = q1[e1[i]] >> 8; }
        build_pal<IB, false>(v0, v1, pal[u], pk[u]);
        sse[u] = sumsq;
      }
      uint64_t L = M.list;
      for (int i = 1; i < M.n; i += 2) {
        const int ta = (int)(L & 15), tb = (int)((L >> 4) & 15);
        L >>= 8;
        const uint32_t va = __byte_perm(tex[ta * STAGE_STRIDE], 0u, sel);
        const uint32_t vb = __byte_perm(tex[tb * STAGE_STRIDE], 0u, sel);
#pragma unroll
        for (int u = 0; u < CH; u++)
          sse[u] += best_key<F, 2>(va, pal[u], pk[u]) + best_key<F, 2>(vb, pal[u], pk[u]);
      }
      if (M.n & 1) {
        const uint32_t va = __byte_perm(tex[(int)(L & 15) * STAGE_STRIDE], 0u, sel);
#pragma unroll
        for (int u = 0; u < CH; u++) sse[u] += best_key<F, 2>(va, pal[u], pk[u]);
      }
#pragma unroll
      for (int u = 0; u < CH; u++) b = min(b, (uint32_t)sse[u]);
    }
    return b;
  }
  uint32_t best_sse = 0xFFFFFFFFu;
#pragma unroll
  for (int cmb = 0; cmb < NCOMBO; cmb++) {
    const int p0 = PT == PT_UNIQUE ? (cmb & 1) : (PT == PT_SHARED ? cmb : 0);
    const int p1 = PT == PT_UNIQUE ? (cmb >> 1) : (PT == PT_SHARED ? cmb : 0);
    const uint16_t* q0 = sq + 256 * qid(BITS, HP, p0);
    const uint16_t* q1 = sq + 256 * qid(BITS, HP, p1);
    int c0[NCH], c1[NCH], v0[3] = {0, 0, 0}, v1[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < NCH; i++) {
      const uint32_t a = q0[e0[i]], b = q1[e1[i]];
      c0[i] = a & 255; c1[i] = b & 255;
      v0[ch[i]] = a >> 8; v1[ch[i]] = b >> 8;
    }
    uint32_t pal[F];
    int pk[F];
    build_pal<IB, OUT>(v0, v1, pal, pk);  // uncoded channels have zero endpoints, so their bytes are 0
    int sse = sumsq;
    uint32_t il = 0, ih = 0;
    if (OUT) {
      uint64_t L = M.list;
      for (int i = 0; i < M.n; i++, L >>= 4) {
        const int t = (int)(L & 15);
        const uint32_t v = __byte_perm(tex[t * STAGE_STRIDE], 0u, sel);
        const int key = best_key<F>(v, pal, pk);
        sse += key >> 4;
        if (t < 8) il |= (uint32_t)(key & 15) << (4 * t); else ih |= (uint32_t)(key & 15) << (4 * (t - 8));
      }
    } else {
      // two member texels per step: their palette searches are independent chains (the error is
      // an integer sum, so the order of the additions does not matter)
      uint64_t L = M.list;
      for (int i = 1; i < M.n; i += 2) {
        const int ta = (int)(L & 15), tb = (int)((L >> 4) & 15);
        L >>= 8;
        const uint32_t va = __byte_perm(tex[ta * STAGE_STRIDE], 0u, sel);
        const uint32_t vb = __byte_perm(tex[tb * STAGE_STRIDE], 0u, sel);
        sse += best_key<F, 2>(va, pal, pk) + best_key<F, 2>(vb, pal, pk);  // |entry|^2 - 2 dot
      }
      if (M.n & 1) {
        const uint32_t va = __byte_perm(tex[(int)(L & 15) * STAGE_STRIDE], 0u, sel);
        sse += best_key<F, 2>(va, pal, pk);
      }
    }
    if ((uint32_t)sse < best_sse) {
      best_sse = (uint32_t)sse;
      if (OUT) {
        out->idx_lo = il; out->idx_hi = ih; out->p[0] = p0; out->p[1] = p1;
#pragma unroll
        for (int i = 0; i < NCH; i++) { out->code[0][ch[i]] = c0[i]; out->code[1][ch[i]] = c1[i]; }
      }
    }
  }
  return best_sse;
}

// Full subset fit = prefit + quant_eval.
template <int IB, int CHMASK, int PT, int BITS, bool OUT>
__device__ __forceinline__ uint32_t fit_subset(const uint32_t* __restrict__ tex, Mem M, FitOut* out,
                                               const uint16_t* __restrict__ sq, uint32_t sel = 0x3210u) {
  if (OUT) { out->idx_lo = 0; out->idx_hi = 0; out->p[0] = out->p[1] = 0;
#pragma unroll
    for (int i = 0; i < 3; i++) out->code[0][i] = out->code[1][i] = 0; }
  int e0[3] = {0, 0, 0}, e1[3] = {0, 0, 0};
  int sumsq = 0;
  if (prefit<IB, CHMASK>(tex, M, e0, e1, sumsq, sel) == 0) return 0;
  return quant_eval<IB, CHMASK, PT, BITS, OUT>(tex, M, e0, e1, sumsq, out, sq, sel);
}

// ---- candidate scoring (search phase) ----------------------------------------------
// Subsets in a rolled loop: one copy of the fit code per mode keeps the search's instruction
// footprint small (warps at different candidates share the instruction cache).
template <int NS, int IB, int PT, int BITS>
__device__ __forceinline__ uint32_t score_part(const uint32_t* tex, int p, const uint16_t* sq) {
  uint32_t s = 0;
#pragma unroll 1
  for (int sub = 0; sub < NS; sub++) s += fit_subset<IB, 7, PT, BITS, false>(tex, mem_of(NS, p, sub), nullptr, sq);
  return s;
}

// Three-subset partitions with the errors of repeated member sets reused (cache: the errors of
// the distinct member sets met so far, indexed as c_sub3; the reuse pattern is the same for
// every lane). Mode 0 meets 36 distinct sets in its 48 subsets, mode 2 140 in 192.
// A prefit kept for a later mode: endpoints and the members' summed squared norms.
struct Prefit {
  int e0[3], e1[3], sumsq;
};

// The fit of a subset whose prefit may be shared: a slot >= 0 with STORE keeps the prefit there,
// without STORE takes it from there.
template <int IB, int PT, int BITS, bool STORE>
__device__ __forceinline__ uint32_t fit_shared(const uint32_t* tex, Mem M, int slot, Prefit* pfc, const uint16_t* sq) {
  if (slot < 0) return fit_subset<IB, 7, PT, BITS, false>(tex, M, nullptr, sq);
  int e0[3] = {0, 0, 0}, e1[3] = {0, 0, 0}, sumsq = 0;
  if (STORE) {
    prefit<IB, 7>(tex, M, e0, e1, sumsq);
    Prefit& f = pfc[slot];
#pragma unroll
    for (int i = 0; i < 3; i++) { f.e0[i] = e0[i]; f.e1[i] = e1[i]; }
    f.sumsq = sumsq;
  } else {
    const Prefit& f = pfc[slot];
#pragma unroll
    for (int i = 0; i < 3; i++) { e0[i] = f.e0[i]; e1[i] = f.e1[i]; }
    sumsq = f.sumsq;
  }
  return quant_eval<IB, 7, PT, BITS, false>(tex, M, e0, e1, sumsq, nullptr, sq);
}

template <int IB, int PT, int BITS>
__device__ __forceinline__ uint32_t score_part3(const uint32_t* tex, int p, const uint16_t* sq, uint32_t* cache,
                                                Prefit* pfc) {
  uint32_t s = 0;
#pragma unroll 1
  for (int sub = 0; sub < 3; sub++) {
    const uint32_t e = c_sub3[3 * p + sub];
    uint32_t r;
    if (e & 0x100u) {
      const int slot = IB == 3 ? c_pf3b[p][sub] : c_pf3a[p][sub];
      r = fit_shared<IB, PT, BITS, true>(tex, mem_of(3, p, sub), slot, pfc, sq);
      cache[e & 0xFFu] = r;
    } else {
      r = cache[e & 0xFFu];
    }
    s += r;
  }
  return s;
}

// modes 4 / 5: colour over the channels other than rot-1, scalar channel rot-1 in the alpha slot
template <int MODE, int ROT, int ISB>
__device__ __forceinline__ uint32_t score_rot(const uint32_t* tex, FitOut* oc, FitOut* oa, const uint16_t* sq) {
  constexpr int CB = MODE == 4 ? 5 : 7, AB = MODE == 4 ? 6 : 8;
  constexpr int CIB = MODE == 4 ? (ISB ? 3 : 2) : 2, AIB = MODE == 4 ? (ISB ? 2 : 3) : 2;
  constexpr int CM = ROT == 0 ? 7 : (7 & ~(1 << (ROT - 1)));
  const bool out = oc != nullptr;
  uint32_t s;
  if (out) s = fit_subset<CIB, CM, PT_NONE, CB, true>(tex, mem_all(), oc, sq);
  else s = fit_subset<CIB, CM, PT_NONE, CB, false>(tex, mem_all(), nullptr, sq);
  if constexpr (ROT != 0) {
    constexpr int AM = 1 << (ROT > 0 ? ROT - 1 : 0);
    if (out) s += fit_subset<AIB, AM, PT_NONE, AB, true>(tex, mem_all(), oa, sq);
    else s += fit_subset<AIB, AM, PT_NONE, AB, false>(tex, mem_all(), nullptr, sq);
  }
  return s;
}

// Rotations 1-3 in the search: the texels' bytes are permuted so that the rotated channel sits in
// byte 2 and the colour channels keep their order in bytes 0-1; the errors equal score_rot's
// (every step of the fit is symmetric in the channel positions, and the order of the colour
// channels, which decides ties, is kept).
__device__ __forceinline__ uint32_t rot_sel(int rot) {
  // byte 2 <- rotated channel; bytes 0-1 <- the other two in order; byte 3 <- 0
  return rot == 1 ? 0x4021u : (rot == 2 ? 0x4120u : 0x4210u);
}

// SYNC: every thread of the CTA calls the search, and a barrier after each mode's candidates
// keeps the CTA's warps in the same part of the (large) search code, so they share the
// instruction cache.
template <bool SYNC>
__device__ __noinline__ int search_best(const uint32_t* tex, uint32_t* best_sse, const uint16_t* sq) {
  uint32_t best = 0xFFFFFFFFu;
  int be = 0;
  // the block takes the least error, ties to the lowest enumeration index
#define CAND(expr, idx)                                      \
  do {                                                       \
    const uint32_t s_ = (expr);                              \
    const int e_ = (idx);                                    \
    if (s_ < best || (s_ == best && e_ < be)) { best = s_; be = e_; } \
  } while (0)
  uint32_t cache[BC7_SUB3_SETS];
  Prefit pfc[BC7_PF_SLOTS];
  for (int p = 0; p < 16; p++) CAND((score_part3<3, PT_UNIQUE, 4>(tex, p, sq, cache, pfc)), p);
  if (SYNC) __syncthreads();
  for (int p = 0; p < 64; p++) {
    uint32_t s1 = 0;
#pragma unroll 1
    for (int sub = 0; sub < 2; sub++)
      s1 += fit_shared<3, PT_SHARED, 6, false>(tex, mem_of(2, p, sub), c_pf2b[p][sub], pfc, sq);
    CAND(s1, 16 + p);
  }
  if (SYNC) __syncthreads();
  for (int p = 0; p < 64; p++) CAND((score_part3<2, PT_NONE, 5>(tex, p, sq, cache, pfc)), 80 + p);
  if (SYNC) __syncthreads();
  // modes 3 and 7: same partitions and 2-bit weights, so one prefit per subset serves both
  for (int p = 0; p < 64; p++) {
    uint32_t s3 = 0, s7 = 0;
#pragma unroll 1
    for (int sub = 0; sub < 2; sub++) {
      int e0[3] = {0, 0, 0}, e1[3] = {0, 0, 0};
      int sumsq = 0;
      const Mem M = mem_of(2, p, sub);
      const int slot = c_pf2a[p][sub];
      if (slot >= 0) {
        const Prefit& f = pfc[slot];
#pragma unroll
        for (int i = 0; i < 3; i++) { e0[i] = f.e0[i]; e1[i] = f.e1[i]; }
        sumsq = f.sumsq;
      } else if (prefit<2, 7>(tex, M, e0, e1, sumsq) == 0) {
        continue;
      }
      s3 += quant_eval<2, 7, PT_UNIQUE, 7, false>(tex, M, e0, e1, sumsq, nullptr, sq);
      s7 += quant_eval<2, 7, PT_UNIQUE, 5, false>(tex, M, e0, e1, sumsq, nullptr, sq);
    }
    CAND(s3, 144 + p);
    CAND(s7, 221 + p);
  }
  if (SYNC) __syncthreads();
  // Modes 4 and 5 over all 16 texels: mode 5's 2-bit colour prefit equals mode 4's (index
  // selection 0) and its 2-bit alpha prefit equals mode 4's (index selection 1), rotation by
  // rotation, so mode 5 takes them from there (the rotated forms permute the texels' bytes: the
  // rotated channel to byte 2, the others in order).
  Prefit pr[2][4];  // [colour, alpha][rotation]
  {
    int e0[3] = {0, 0, 0}, e1[3] = {0, 0, 0}, sumsq = 0;
    prefit<2, 7>(tex, mem_all(), e0, e1, sumsq);
    CAND((quant_eval<2, 7, PT_NONE, 5, false>(tex, mem_all(), e0, e1, sumsq, nullptr, sq)), 208);
    CAND((quant_eval<2, 7, PT_NONE, 7, false>(tex, mem_all(), e0, e1, sumsq, nullptr, sq)), 216);
  }
  CAND((score_rot<4, 0, 1>(tex, nullptr, nullptr, sq)), 209);
#pragma unroll 1
  for (int rot = 1; rot <= 3; rot++) {
    const uint32_t sel = rot_sel(rot);
    Prefit& f = pr[0][rot];
    prefit<2, 3>(tex, mem_all(), f.e0, f.e1, f.sumsq, sel);
    const uint32_t c = quant_eval<2, 3, PT_NONE, 5, false>(tex, mem_all(), f.e0, f.e1, f.sumsq, nullptr, sq, sel);
    CAND((c + fit_subset<3, 4, PT_NONE, 6, false>(tex, mem_all(), nullptr, sq, sel)), 208 + 2 * rot);
  }
  if (SYNC) __syncthreads();
#pragma unroll 1
  for (int rot = 1; rot <= 3; rot++) {
    const uint32_t sel = rot_sel(rot);
    Prefit& f = pr[1][rot];
    prefit<2, 4>(tex, mem_all(), f.e0, f.e1, f.sumsq, sel);
    const uint32_t a = quant_eval<2, 4, PT_NONE, 6, false>(tex, mem_all(), f.e0, f.e1, f.sumsq, nullptr, sq, sel);
    CAND((fit_subset<3, 3, PT_NONE, 5, false>(tex, mem_all(), nullptr, sq, sel) + a), 209 + 2 * rot);
  }
  if (SYNC) __syncthreads();
#pragma unroll 1
  for (int rot = 1; rot <= 3; rot++) {
    const uint32_t sel = rot_sel(rot);
    const Prefit &fc = pr[0][rot], &fa = pr[1][rot];
    CAND((quant_eval<2, 3, PT_NONE, 7, false>(tex, mem_all(), fc.e0, fc.e1, fc.sumsq, nullptr, sq, sel) +
          quant_eval<2, 4, PT_NONE, 8, false>(tex, mem_all(), fa.e0, fa.e1, fa.sumsq, nullptr, sq, sel)),
         216 + rot);
  }
  CAND((score_part<1, 4, PT_UNIQUE, 7>(tex, 0, sq)), 220);
#undef CAND
  *best_sse = best;
  return be;
}

// ---- final solve and packing -----------------------------------------------------------
struct BitW {
  uint32_t w[4];
  int pos;
  __device__ void put(uint32_t v, int n) {
    if (n == 0) return;
    v &= (n >= 32) ? 0xFFFFFFFFu : ((1u << n) - 1u);
    int word = pos >> 5, off = pos & 31;
    w[word] |= v << off;
    if (off + n > 32) w[word + 1] |= v >> (32 - off);
    pos += n;
  }
};

__device__ __forceinline__ int get_idx(const FitOut& f, int t) {
  return t < 8 ? (f.idx_lo >> (4 * t)) & 15 : (f.idx_hi >> (4 * (t - 8))) & 15;
}

struct ModeInfo { int ns, pb, rb, isb, cb, ab, epb, spb, ib, ib2; };
__device__ __forceinline__ ModeInfo mode_info(int m) {
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

__device__ __forceinline__ uint32_t part_of(int ns, int p) { return ns == 1 ? 0u : (ns == 2 ? c_part2[p] : c_part3[p]); }
__device__ __forceinline__ int anchor_of(int ns, int p, int s) {
  return s == 0 ? 0 : (ns == 2 ? c_anc2[p] : (s == 1 ? c_anc3a[p] : c_anc3b[p]));
}

// Solves candidate e into per-subset fits, fixes anchors and packs the 128 bits.
__device__ __noinline__ uint4 solve_pack(const uint32_t* tx, int e, const uint16_t* sq) {
  int mode, part = 0, rot = 0, isb = 0;
  if (e < 16) { mode = 0; part = e; }
  else if (e < 208) { mode = 1 + (e - 16) / 64; part = (e - 16) % 64; }
  else if (e < 216) { mode = 4; rot = (e - 208) / 2; isb = (e - 208) % 2; }
  else if (e < 220) { mode = 5; rot = e - 216; }
  else if (e < 221) { mode = 6; }
  else { mode = 7; part = e - 221; }
  const ModeInfo M = mode_info(mode);
  FitOut f[3], fa;
  const uint32_t pm = part_of(M.ns, part);
  int acode[3][2];
  for (int s = 0; s < 3; s++) acode[s][0] = acode[s][1] = (1 << M.ab) - 1;
  switch (mode) {
    case 0: for (int s = 0; s < 3; s++) fit_subset<3, 7, PT_UNIQUE, 4, true>(tx, mem_of(3, part, s), &f[s], sq); break;
    case 1: for (int s = 0; s < 2; s++) fit_subset<3, 7, PT_SHARED, 6, true>(tx, mem_of(2, part, s), &f[s], sq); break;
    case 2: for (int s = 0; s < 3; s++) fit_subset<2, 7, PT_NONE, 5, true>(tx, mem_of(3, part, s), &f[s], sq); break;
    case 3: for (int s = 0; s < 2; s++) fit_subset<2, 7, PT_UNIQUE, 7, true>(tx, mem_of(2, part, s), &f[s], sq); break;
    case 6: fit_subset<4, 7, PT_UNIQUE, 7, true>(tx, mem_all(), &f[0], sq); break;
    case 7: for (int s = 0; s < 2; s++) fit_subset<2, 7, PT_UNIQUE, 5, true>(tx, mem_of(2, part, s), &f[s], sq); break;
    case 4:
      switch (rot * 2 + isb) {
        case 0: score_rot<4, 0, 0>(tx, &f[0], &fa, sq); break;
        case 1: score_rot<4, 0, 1>(tx, &f[0], &fa, sq); break;
        case 2: score_rot<4, 1, 0>(tx, &f[0], &fa, sq); break;
        case 3: score_rot<4, 1, 1>(tx, &f[0], &fa, sq); break;
        case 4: score_rot<4, 2, 0>(tx, &f[0], &fa, sq); break;
        case 5: score_rot<4, 2, 1>(tx, &f[0], &fa, sq); break;
        case 6: score_rot<4, 3, 0>(tx, &f[0], &fa, sq); break;
        default: score_rot<4, 3, 1>(tx, &f[0], &fa, sq); break;
      }
      break;
    default:
      switch (rot) {
        case 0: score_rot<5, 0, 0>(tx, &f[0], &fa, sq); break;
        case 1: score_rot<5, 1, 0>(tx, &f[0], &fa, sq); break;
        case 2: score_rot<5, 2, 0>(tx, &f[0], &fa, sq); break;
        default: score_rot<5, 3, 0>(tx, &f[0], &fa, sq); break;
      }
      break;
  }
  // gather codes [subset][endpoint][R, G, B] and indices
  int code[3][2][3], pb[3][2];
  int cidx[16], aidx[16];
  for (int t = 0; t < 16; t++) { cidx[t] = 0; aidx[t] = 0; }
  for (int s = 0; s < M.ns; s++) {
    for (int ep = 0; ep < 2; ep++) {
      for (int c = 0; c < 3; c++) code[s][ep][c] = f[s].code[ep][c];
      pb[s][ep] = f[s].p[ep];
    }
  }
  for (int t = 0; t < 16; t++) {
    int s = (pm >> (2 * t)) & 3;
    cidx[t] = get_idx(f[s], t);
  }
  if (mode == 4 || mode == 5) {
    if (rot != 0) {
      acode[0][0] = fa.code[0][rot - 1];
      acode[0][1] = fa.code[1][rot - 1];
      for (int t = 0; t < 16; t++) aidx[t] = get_idx(fa, t);
    }
    const int cib = isb ? M.ib2 : M.ib, aib = isb ? M.ib : M.ib2;
    if ((cidx[0] >> (cib - 1)) & 1) {
      for (int c = 0; c < 3; c++) { int tmp = code[0][0][c]; code[0][0][c] = code[0][1][c]; code[0][1][c] = tmp; }
      for (int t = 0; t < 16; t++) cidx[t] = (1 << cib) - 1 - cidx[t];
    }
    if ((aidx[0] >> (aib - 1)) & 1) {
      int tmp = acode[0][0]; acode[0][0] = acode[0][1]; acode[0][1] = tmp;
      for (int t = 0; t < 16; t++) aidx[t] = (1 << aib) - 1 - aidx[t];
    }
  } else {
    for (int s = 0; s < M.ns; s++) {
      int a = anchor_of(M.ns, part, s);
      if (!((cidx[a] >> (M.ib - 1)) & 1)) continue;
      for (int c = 0; c < 3; c++) { int tmp = code[s][0][c]; code[s][0][c] = code[s][1][c]; code[s][1][c] = tmp; }
      { int tmp = acode[s][0]; acode[s][0] = acode[s][1]; acode[s][1] = tmp; }
      if (M.epb) { int tmp = pb[s][0]; pb[s][0] = pb[s][1]; pb[s][1] = tmp; }
      for (int t = 0; t < 16; t++)
        if ((int)((pm >> (2 * t)) & 3) == s) cidx[t] = (1 << M.ib) - 1 - cidx[t];
    }
  }
  BitW w;
  w.w[0] = w.w[1] = w.w[2] = w.w[3] = 0;
  w.pos = 0;
  w.put(1u << mode, mode + 1);
  w.put(part, M.pb);
  w.put(rot, M.rb);
  w.put(isb, M.isb);
  for (int c = 0; c < 3; c++)
    for (int s = 0; s < M.ns; s++)
      for (int ep = 0; ep < 2; ep++) w.put(code[s][ep][c], M.cb);
  if (M.ab)
    for (int s = 0; s < M.ns; s++)
      for (int ep = 0; ep < 2; ep++) w.put(acode[s][ep], M.ab);
  if (M.epb)
    for (int s = 0; s < M.ns; s++)
      for (int ep = 0; ep < 2; ep++) w.put(pb[s][ep], 1);
  if (M.spb)
    for (int s = 0; s < M.ns; s++) w.put(pb[s][0], 1);
  if (M.ib2) {
    for (int t = 0; t < 16; t++) w.put(isb ? aidx[t] : cidx[t], M.ib - (t == 0));
    for (int t = 0; t < 16; t++) w.put(isb ? cidx[t] : aidx[t], M.ib2 - (t == 0));
  } else {
    int a1 = M.ns >= 2 ? anchor_of(M.ns, part, 1) : -1, a2 = M.ns >= 3 ? anchor_of(M.ns, part, 2) : -1;
    for (int t = 0; t < 16; t++) w.put(cidx[t], M.ib - ((t == 0) || t == a1 || t == a2));
  }
  return make_uint4(w.w[0], w.w[1], w.w[2], w.w[3]);
}

// Constant blocks (Sec. III-A: a block of one colour can be coded without error; the format
// reaches every constant colour): mode 5, rotation 0, every colour index 1 (weight 21), per
// channel the code pair of c_const7, alpha codes all ones and alpha indices 0. Texel t of the
// thread's block is tx[t * STAGE_STRIDE]; returns whether the block is constant.
__device__ __forceinline__ bool const_block(const uint32_t* tx, uint4* out) {
  const uint32_t c = tx[0];
  bool same = true;
#pragma unroll
  for (int t = 1; t < 16; t++) same &= tx[t * STAGE_STRIDE] == c;
  if (!same) return false;
  BitW w;
  w.w[0] = w.w[1] = w.w[2] = w.w[3] = 0;
  w.pos = 0;
  w.put(1u << 5, 6);  // mode 5
  w.put(0u, 2);       // rotation 0
  for (int ch = 0; ch < 3; ch++) {
    const uint32_t ab = c_const7[(c >> (8 * ch)) & 255u];
    w.put(ab & 255u, 7);
    w.put(ab >> 8, 7);
  }
  w.put(255u, 8);
  w.put(255u, 8);
  w.put(1u, 1);  // texel 0's colour index (anchor: one bit)
  for (int t = 1; t < 16; t++) w.put(1u, 2);
  w.put(0u, 1);  // alpha indices 0
  for (int t = 1; t < 16; t++) w.put(0u, 2);
  *out = make_uint4(w.w[0], w.w[1], w.w[2], w.w[3]);
  return true;
}

// One kernel for both sources: staged layout-D groups (sh / perm / scales) or raw
// texels [nblk][16][3] (texin != nullptr), so the search is compiled once. A CTA is BC7_SUBS
// staging units of 128 threads (one block per thread); each thread's texels stay in its unit's
// shared tile (column threadIdx.x % 128) for the whole search. Every thread searches (threads
// past the last block on texels of 128) so that the barriers between the search's modes are
// reached by the whole CTA.
// 5 units (20 warps, at most 102 registers) per CTA and SM: 70.7 ms for 3M blocks against
// 70.8-71.1 ms with 6 units (80 registers); 4 units (128 registers) were 6% slower.
#ifndef BC7_SUBS
#define BC7_SUBS 5
#endif
// the multi-scene BC1 kernel keeps 128-thread CTAs, 5 per SM (and the default CTAs per SM of the
// multi-scene launches)
#define BC7_MIN_BLOCKS 5
#define BC7_THREADS (BC7_SUBS * STAGE_THREADS)
#define BC7_DYN_SMEM (BC7_SUBS * 16 * STAGE_STRIDE * 4)
__global__ void __launch_bounds__(BC7_THREADS, 1) k_bc7(const float* __restrict__ sh, const int32_t* __restrict__ perm,
                                                        const float* __restrict__ scales, int64_t n_groups,
                                                        const uint8_t* __restrict__ texin, int64_t nblk,
                                                        uint4* __restrict__ blocks, uint32_t* __restrict__ sse7,
                                                        uint64_t* __restrict__ sse64) {
  // the units' texel tiles live in dynamic shared memory (more than 48 KB for six units)
  extern __shared__ uint32_t k_bc7_dyn[];
  uint32_t(*tex)[16][STAGE_STRIDE] = reinterpret_cast<uint32_t(*)[16][STAGE_STRIDE]>(k_bc7_dyn);
  __shared__ float s_scale[16];
  __shared__ uint16_t sq[12 * 256];
  for (int i = threadIdx.x; i < 12 * 256; i += blockDim.x) sq[i] = (&g_qtab[0][0])[i];
  if (!texin && threadIdx.x < 16) s_scale[threadIdx.x] = scales[threadIdx.x];
  __syncthreads();
  const int sub = threadIdx.x / STAGE_THREADS, lt = threadIdx.x % STAGE_THREADS;
  const int64_t total = texin ? nblk : n_groups * 16;
  for (int64_t b0 = (int64_t)blockIdx.x * BC7_THREADS; b0 < total; b0 += (int64_t)gridDim.x * BC7_THREADS) {
    const int64_t bs = b0 + sub * STAGE_THREADS;  // first block of this thread's staging unit
    const int64_t blk = bs + lt;
    if (!texin) {
      stage_groups(sh, perm, s_scale, bs / 16, n_groups, tex[sub], lt);
    } else if (blk < total) {
      const uint8_t* p = texin + blk * 48;
#pragma unroll
      for (int t = 0; t < 16; t++)
        tex[sub][t][lt] = (uint32_t)p[3 * t] | ((uint32_t)p[3 * t + 1] << 8) | ((uint32_t)p[3 * t + 2] << 16);
    } else {
#pragma unroll
      for (int t = 0; t < 16; t++) tex[sub][t][lt] = 0x808080u;
    }
    __syncthreads();
    uint32_t best;
    const uint32_t* my = &tex[sub][0][lt];
    const int e = search_best<true>(my, &best, sq);
    if (blk < total) {
      uint4 cb;
      if (const_block(my, &cb)) {
        blocks[blk] = cb;
        best = 0;
      } else {
        blocks[blk] = solve_pack(my, e, sq);
      }
      if (sse7) sse7[blk] = best;
      if (sse64) sse64[blk] = best;
    }
    __syncthreads();
  }
}

// allows the dynamic shared memory of k_bc7 above 48 KB (called once with the tables)
cudaError_t bc7_kernel_attributes() {
  return cudaFuncSetAttribute(k_bc7, cudaFuncAttributeMaxDynamicSharedMemorySize, BC7_DYN_SMEM);
}

static int grid_for7(int64_t work, int per_cta) {
  int64_t g = ceil_div64(work, per_cta);
  if (g > gsc_sm_count() * 32) g = gsc_sm_count() * 32;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_bc7_groups(const float* sh, const int32_t* perm, const float* scales, int64_t n_groups,
                              uint8_t* blocks, uint32_t* sse7, cudaStream_t st) {
  if (n_groups <= 0) return cudaSuccess;
  gsc_count_launch(); k_bc7<<<grid_for7(n_groups, STAGE_GROUPS * BC7_SUBS), BC7_THREADS, BC7_DYN_SMEM, st>>>(
      sh, perm, scales, n_groups, nullptr, 0, reinterpret_cast<uint4*>(blocks), sse7, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_bc7_blocks(const uint8_t* tex, int64_t nblk, uint8_t* out, uint64_t* sse, cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
  gsc_count_launch(); k_bc7<<<grid_for7(nblk, BC7_THREADS), BC7_THREADS, BC7_DYN_SMEM, st>>>(nullptr, nullptr, nullptr, 0, tex, nblk,
                                                                reinterpret_cast<uint4*>(out), nullptr, sse);
  return cudaGetLastError();
}

// ---- persistent multi-scene encode -----------------------------------------------------------
// One launch per coding (KIND 1 = BC1, 7 = BC7) over the tiles of every listed scene. Tiles
// are claimed round robin (schedule 0), from an atomic work queue (1, 2), or one per CTA unit
// (3, a grid of all tiles); a tile finds its scene by binary search over the list. A BC7 CTA is
// BC7_SUBS staging units of 128 threads, each claiming its own tile, that step through their
// tiles 8 groups at a time in lockstep (units past their tile's end search texels of 128), so
// the search's barriers are reached by the whole CTA, as in k_bc7. The bits equal the
// single-scene kernels'.
template <int KIND>
__global__ void __launch_bounds__((KIND == 7 ? BC7_SUBS : 1) * STAGE_THREADS, KIND == 7 ? 1 : BC7_MIN_BLOCKS)
    k_batch(const BatchSceneDev* __restrict__ scenes, int n_scenes, int64_t n_tiles, int schedule,
            int* __restrict__ counter) {
  constexpr int SUBS = KIND == 7 ? BC7_SUBS : 1;
  __shared__ uint32_t tex[SUBS][16][STAGE_STRIDE];
  __shared__ float s_scale[SUBS][16];
  __shared__ uint16_t sq[KIND == 7 ? 12 * 256 : 1];
  __shared__ long long s_tile[SUBS];
  __shared__ int s_iters;
  if (KIND == 7)
    for (int i = threadIdx.x; i < 12 * 256; i += blockDim.x) sq[i] = (&g_qtab[0][0])[i];
  const int sub = threadIdx.x / STAGE_THREADS, lt = threadIdx.x % STAGE_THREADS;
  for (int64_t it = 0;; it++) {
    __syncthreads();
    if (lt == 0)
      s_tile[sub] = (schedule == 0 || schedule == 3) ? (long long)((blockIdx.x + it * gridDim.x) * SUBS + sub)
                                                     : (long long)atomicAdd(counter, 1);
    if (threadIdx.x == 0) s_iters = 0;
    __syncthreads();
    bool any = false;
#pragma unroll
    for (int u = 0; u < SUBS; u++) any |= s_tile[u] < n_tiles;
    if (!any) break;
    const int64_t ti = s_tile[sub];
    const bool has = ti < n_tiles;
    BatchSceneDev S;
    int64_t gbeg = 0, gend = 0;
    if (has) {
      int lo = 0, hi = n_scenes - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (scenes[mid].tile0 <= ti) lo = mid; else hi = mid - 1;
      }
      S = scenes[lo];
      gbeg = (ti - S.tile0) * S.tile_groups;
      gend = min(gbeg + (int64_t)S.tile_groups, S.work_groups);
      if (lt < 16) s_scale[sub][lt] = S.scales[lt];
      if (lt == 0) atomicMax(&s_iters, (int)((gend - gbeg + STAGE_GROUPS - 1) / STAGE_GROUPS));
    }
    __syncthreads();
    const int iters = s_iters;  // the longest tile of the CTA's units, in staging steps
    for (int k = 0; k < iters; k++) {
      const int64_t g0 = gbeg + (int64_t)k * STAGE_GROUPS;
      const bool live = has && g0 < gend;
      if (live) {
        stage_groups(S.sh, S.perm, s_scale[sub], g0, S.n_groups, tex[sub], lt);
      } else {
#pragma unroll
        for (int t = 0; t < 16; t++) tex[sub][t][lt] = 0x808080u;
      }
      __syncthreads();
      const int64_t blk = g0 * 16 + lt;
      const bool write = live && blk < S.n_groups * 16;
      if (KIND == 1) {
        if (write) {
          uint32_t tx[16];
#pragma unroll
          for (int t = 0; t < 16; t++) tx[t] = tex[sub][t][lt];
          const Bc1Res r = bc1_encode(tx);
          reinterpret_cast<uint2*>(S.b1)[blk] = bc1_bits(r);
          if (S.sse1) S.sse1[blk] = r.sse;
          if (S.sse0) S.sse0[blk] = sse_zero(tx);
        }
      } else {
        uint32_t best;
        const uint32_t* my = &tex[sub][0][lt];
        const int e = search_best<true>(my, &best, sq);
        if (write) {
          uint4 cb;
          if (const_block(my, &cb)) best = 0;
          else cb = solve_pack(my, e, sq);
          reinterpret_cast<uint4*>(S.b7)[blk] = cb;
          if (S.sse7) S.sse7[blk] = best;
        }
      }
      __syncthreads();
    }
  }
}

cudaError_t launch_batch_encode(int kind, const BatchSceneDev* scenes, int n_scenes, int64_t n_tiles, int schedule,
                                int ctas_per_sm, int sm_count, int* counter, cudaStream_t st) {
  if (n_tiles <= 0 || n_scenes <= 0) return cudaSuccess;
  // schedule 3: one CTA unit per tile, left to the hardware block scheduler; a BC7 CTA holds
  // BC7_SUBS units
  const int64_t units = kind == 7 ? BC7_SUBS : 1;
  const int64_t cta_tiles = ceil_div64(n_tiles, units);
  int64_t grid = schedule == 3 ? cta_tiles : (int64_t)(sm_count > 0 ? sm_count : gsc_sm_count()) * (ctas_per_sm > 0 ? ctas_per_sm : BC7_MIN_BLOCKS);
  if (grid > cta_tiles) grid = cta_tiles;
  if (grid > 0x7FFFFFFF) grid = 0x7FFFFFFF;
  if (schedule == 1 || schedule == 2) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
  }
  gsc_count_launch();
  if (kind == 7) k_batch<7><<<(int)grid, BC7_THREADS, 0, st>>>(scenes, n_scenes, n_tiles, schedule, counter);
  else k_batch<1><<<(int)grid, STAGE_THREADS, 0, st>>>(scenes, n_scenes, n_tiles, schedule, counter);
  return cudaGetLastError();
}

// ---- one mode family searched two ways (a measurement of the search's thread mapping) --------
// Mode 1 only (64 two-subset partitions, 6-bit endpoints with a shared p-bit, 3-bit indices):
// the least-error partition of each block, ties to the lowest, with its error. Thread per block
// (as k_bc7: every lane of a warp fits the same partition, so the member loops are uniform) or
// warp per block (lane l fits partitions l and l + 32 of the warp's block, then a shuffle
// minimum over (error, partition)); the results are the same.
template <bool WARP>
__global__ void __launch_bounds__(STAGE_THREADS) k_bc7_mode1(const uint8_t* __restrict__ texin, int64_t nblk,
                                                             uint32_t* __restrict__ sse_out,
                                                             int32_t* __restrict__ part_out) {
  __shared__ uint32_t tex[16][STAGE_STRIDE];
  __shared__ uint16_t sq[12 * 256];
  for (int i = threadIdx.x; i < 12 * 256; i += blockDim.x) sq[i] = (&g_qtab[0][0])[i];
  const int lt = threadIdx.x;
  for (int64_t b0 = (int64_t)blockIdx.x * STAGE_THREADS; b0 < nblk; b0 += (int64_t)gridDim.x * STAGE_THREADS) {
    __syncthreads();
    if (WARP) {
      // 128 blocks per step: texel t of block b0 + j at tex[t][j]; warp w then takes blocks
      // b0 + 32 w + i for i < 32 in turn
      for (int i = lt; i < STAGE_THREADS * 16; i += STAGE_THREADS) {
        const int j = i / 16, t = i % 16;
        const int64_t blk = b0 + j;
        const uint8_t* p = texin + blk * 48 + 3 * t;
        tex[t][j] = blk < nblk ? ((uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16)) : 0x808080u;
      }
    } else {
      const int64_t blk = b0 + lt;
      const uint8_t* p = texin + blk * 48;
#pragma unroll
      for (int t = 0; t < 16; t++)
        tex[t][lt] = blk < nblk ? ((uint32_t)p[3 * t] | ((uint32_t)p[3 * t + 1] << 8) | ((uint32_t)p[3 * t + 2] << 16))
                                : 0x808080u;
    }
    __syncthreads();
    if (WARP) {
      const int w = lt >> 5, lane = lt & 31;
#pragma unroll 1
      for (int i = 0; i < 32; i++) {
        const int j = 32 * w + i;
        const uint32_t* my = &tex[0][j];
        const uint32_t sa = score_part<2, 3, PT_SHARED, 6>(my, lane, sq);
        const uint32_t sb = score_part<2, 3, PT_SHARED, 6>(my, lane + 32, sq);
        uint32_t best = sa;
        int bp = lane;
        if (sb < best) { best = sb; bp = lane + 32; }
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) {
          const uint32_t ob = __shfl_xor_sync(0xFFFFFFFFu, best, d);
          const int op = __shfl_xor_sync(0xFFFFFFFFu, bp, d);
          if (ob < best || (ob == best && op < bp)) { best = ob; bp = op; }
        }
        const int64_t blk = b0 + j;
        if (lane == 0 && blk < nblk) { sse_out[blk] = best; part_out[blk] = bp; }
      }
    } else {
      const uint32_t* my = &tex[0][lt];
      uint32_t best = 0xFFFFFFFFu;
      int bp = 0;
#pragma unroll 1
      for (int p = 0; p < 64; p++) {
        const uint32_t s = score_part<2, 3, PT_SHARED, 6>(my, p, sq);
        if (s < best) { best = s; bp = p; }
      }
      const int64_t blk = b0 + lt;
      if (blk < nblk) { sse_out[blk] = best; part_out[blk] = bp; }
    }
  }
}

cudaError_t launch_bc7_mode1(const uint8_t* tex, int64_t nblk, int warp, uint32_t* sse, int32_t* part, int sm_count,
                             cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
  int64_t g = ceil_div64(nblk, STAGE_THREADS);
  const int64_t cap = (int64_t)sm_count * 8;
  if (g > cap) g = cap;
  gsc_count_launch();
  if (warp) k_bc7_mode1<true><<<(int)g, STAGE_THREADS, 0, st>>>(tex, nblk, sse, part);
  else k_bc7_mode1<false><<<(int)g, STAGE_THREADS, 0, st>>>(tex, nblk, sse, part);
  return cudaGetLastError();
}
