// eval.cu -- fused decode + SH evaluation of a coded scene, tiled through shared memory
// (Sec. I: random access by block index x block size; Sec. II: c(f) = H w(f - p);
// Sec. III-B: BC1 / BC7 formats; Sec. IV-B: block layouts and fixed-rate streams).
//
// A persistent CTA works through tiles of E_TG groups (E_T slots, E_T blocks):
//  1. staging: the tile's blocks, slot entries and slot-ordered positions land in shared memory
//     through TMA bulk copies (cp.async.bulk completing on an mbarrier), issued one tile ahead.
//     Rate streams (blocks at per-stream offsets) and inputs that are not 16-byte aligned use
//     per-thread asynchronous copies (cp.async) instead, also one tile ahead.
//  2. classification: every block gets a class -- BC7 mode 0..7 (mode 4 split by its
//     index-selection bit), the reserved BC7 mode, BC1, or a coefficient the stream drops --
//     and joins that class's list (warp-aggregated shared-memory atomics).
//  3. decode: a warp takes 32 blocks of one class at a time and runs that class's decoder, whose
//     field positions, widths and subset count are compile-time constants; the texels go to a
//     Gaussian-major tile (slot row, coefficient column).
//  4. evaluation: every thread evaluates two Gaussians of the tile. The two share each packed
//     FP32x2 operation lane for lane (coefficients, directions, bases, accumulators), so no
//     operand is broadcast, and per (Gaussian, view) the operations are those of the
//     single-Gaussian evaluation in decode.cu, in the same order: the colours are bit-identical.
#include <stddef.h>

#include "decode_dev.cuh"
#include "layout.cuh"

namespace {

constexpr int E_NT = 192;         // threads per CTA
constexpr int E_NW = E_NT / 32;   // warps per CTA
constexpr int E_T = 2 * E_NT;     // slots (and blocks) per tile: two Gaussians per thread
constexpr int E_TG = E_T / 16;    // groups per tile
constexpr int E_ROW = 20;         // tile words per slot row (16 coefficients + 4 to spread banks)
constexpr int E_GRP = 16 * E_ROW + 4;  // tile words per group
constexpr int E_NCLS = 12;
enum { CL_M4S = 8, CL_RES = 9, CL_BC1 = 10, CL_DROP = 11 };
constexpr int E_MAXV = 64;
// a bounded wait for the staged tile: far beyond any copy's latency
constexpr uint32_t E_WAIT_LIMIT = 1u << 22;

struct EStage {
  uint4 blk[E_T];       // BC7 blocks (16 B), or BC1 blocks (8 B, packed from the start: all-BC1 codings)
  int32_t perm[E_T];
  float pos[E_T * 3];   // slot-ordered positions
  uint8_t cls[E_T];     // rate streams: format of each block as located (BC7 / BC1 / dropped)
};

struct ESmem {
  EStage stage[2];
  uint32_t tile[E_TG * E_GRP];
  uint16_t list[E_NCLS][E_T];
  int cnt[2][E_NCLS];
  uint4 ep[E_NT][3];            // per-lane endpoint slots of multi-subset blocks
  float4 cxy[E_MAXV];           // per view (x, x, y, y) of the camera centre or direction
  float2 cz[E_MAXV];            // (z, z)
  float2 deq[16];               // (f_k, f_k), f_k = s_k / 255 * C_k
  DecTables S;
  unsigned long long mbar[2];
};

static_assert(sizeof(EStage) % 16 == 0, "stage sections must stay 16-byte aligned for TMA");
static_assert(offsetof(EStage, perm) % 16 == 0 && offsetof(EStage, pos) % 16 == 0, "TMA destinations");
static_assert(offsetof(ESmem, tile) % 16 == 0 && (E_GRP * 4) % 16 == 0 && (E_ROW * 4) % 16 == 0, "tile rows");
// two CTAs per SM: 228 KB of shared memory, 1 KB reserved per CTA
static_assert(sizeof(ESmem) <= 113 * 1024, "shared memory of two resident CTAs");

struct EArgs {
  DevTable T;
  const uint8_t* blocks;
  const int32_t* perm;
  const float* pos;       // original order [n][3], or null
  const float* pos_slot;  // slot order [n_groups * 16][3], or null
  const float* dirs;
  const float* cams;
  float* rgb;
  int V, out_order, tma;
};

// First error this translation unit's kernels detected (code, where): a slot entry outside
// [-1, n) in the checked build, or a staged tile that never arrived. Taken by gsc_ctx_sync.
__device__ int g_eval_err[2];
__device__ __forceinline__ void eval_record(int code, int where) {
  if (atomicCAS(&g_eval_err[0], 0, code) == 0) g_eval_err[1] = where;
}

// ---- PTX helpers ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
// true once the phase with the given parity has completed
__device__ __forceinline__ bool mbar_try(unsigned long long* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// 1-D TMA bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(b))
      : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

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

// One BC7 block of class CL (mode CL, or mode 4 with the index-selection bit set) into 16
// texels r | g << 8 | b << 16 (alpha byte unspecified). The arithmetic is that of bc7_block in
// decode_dev.cuh: endpoints as 4x-scaled 16-bit lanes so that ((64 - w) e0 + w e1 + 32) >> 6 of
// two channels is one multiply-add, index streams re-spaced to a fixed width per texel.
template <int CL>
__device__ __forceinline__ void bc7_class_block(uint64_t lo, uint64_t hi, uint32_t (&tx)[16], const DecTables* S,
                                                uint4* ep) {
  constexpr int mode = CL == CL_M4S ? 4 : CL;
  constexpr DModeInfo D = d_mode_info(mode);
  constexpr int ns = D.ns, pb = D.pb, rb = D.rb, isb = D.isb, cb = D.cb, ab = D.ab, epb = D.epb, spb = D.spb;
  constexpr int ib = D.ib, ib2 = D.ib2;
  constexpr bool swap = CL == CL_M4S;  // colour indices from the 3-bit stream
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
  constexpr int cl8 = 8 - nb, cr8 = 2 * nb - 8, al8 = ab ? 8 - na : 0, ar8 = ab ? 2 * na - 8 : 0;
  uint4 e_one = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
  for (int s = 0; s < ns; s++) {
    const uint32_t p0 = epb ? ((pbits >> (2 * s)) & 1u) : (spb ? ((pbits >> s) & 1u) : 0u);
    const uint32_t p1 = epb ? ((pbits >> (2 * s + 1)) & 1u) : p0;
    const int sh0 = 2 * s * cb, sh1 = sh0 + cb;
    uint32_t v0[3], v1[3];
    const uint32_t f3[3] = {fr, fg, fb};
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const uint32_t c0 = (((f3[c] >> sh0) & cm) << hp) | (hp ? p0 : 0u);
      const uint32_t c1 = (((f3[c] >> sh1) & cm) << hp) | (hp ? p1 : 0u);
      v0[c] = (c0 << cl8) | (c0 >> cr8);
      v1[c] = (c1 << cl8) | (c1 >> cr8);
    }
    uint32_t aa0 = 255u, aa1 = 255u;
    if (ab) {
      const uint32_t c0 = (((fa >> (2 * s * ab)) & amk) << epb) | (epb ? p0 : 0u);
      const uint32_t c1 = (((fa >> ((2 * s + 1) * ab)) & amk) << epb) | (epb ? p1 : 0u);
      aa0 = (c0 << al8) | (c0 >> ar8);
      aa1 = (c1 << al8) | (c1 >> ar8);
    }
    const uint32_t e0rg = (v0[0] | (v0[1] << 16)) << 2, e0ba = (v0[2] | (aa0 << 16)) << 2;
    const uint32_t e1rg = (v1[0] | (v1[1] << 16)) << 2, e1ba = (v1[2] | (aa1 << 16)) << 2;
    const uint4 e = make_uint4(64u * e0rg + 0x00800080u, e1rg - e0rg, 64u * e0ba + 0x00800080u, e1ba - e0ba);
    if (ns == 1) e_one = e;
    else ep[s] = e;
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
    const uint4 e = ns == 1 ? e_one : ep[(pm >> (2 * t)) & 3u];
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

template <int CL>
__device__ __forceinline__ void class_block(const EStage& sg, int b, int kind, uint32_t (&tx)[16], const DecTables* S,
                                            uint4* ep) {
  if (CL <= CL_M4S) {
    const uint4 w = sg.blk[b];
    bc7_class_block<CL>(((uint64_t)w.y << 32) | w.x, ((uint64_t)w.w << 32) | w.z, tx, S, ep);
  } else if (CL == CL_BC1) {
    const uint2 w = kind == 1 ? reinterpret_cast<const uint2*>(sg.blk)[b] : make_uint2(sg.blk[b].x, sg.blk[b].y);
    bc1_block(w, tx);
  } else {
    const uint32_t v = CL == CL_RES ? 0u : 0x00808080u;
#pragma unroll
    for (int t = 0; t < 16; t++) tx[t] = v;
  }
}

// texels of block b (tile group b / 16, block k = b % 16) into the Gaussian-major tile
template <int LAYOUT>
__device__ __forceinline__ void tile_store(uint32_t* tile, int b, const uint32_t (&tx)[16]) {
  const int gl = b >> 4, k = b & 15;
  uint32_t* g = tile + gl * E_GRP;
  if (LAYOUT == GSC_LAYOUT_D) {  // texel t -> slot t, coefficient k
#pragma unroll
    for (int t = 0; t < 16; t++) g[t * E_ROW + k] = tx[t];
  } else if (LAYOUT == GSC_LAYOUT_A) {  // texel t -> slot k, coefficient t
#pragma unroll
    for (int q = 0; q < 4; q++)
      *reinterpret_cast<uint4*>(g + k * E_ROW + 4 * q) = make_uint4(tx[4 * q], tx[4 * q + 1], tx[4 * q + 2], tx[4 * q + 3]);
  } else {  // B: block 4v + c of a quad, row i, column j -> slot 4v + i, coefficient 4c + j
    const int v = k >> 2, c = k & 3;
#pragma unroll
    for (int i = 0; i < 4; i++)
      *reinterpret_cast<uint4*>(g + (4 * v + i) * E_ROW + 4 * c) =
          make_uint4(tx[4 * i], tx[4 * i + 1], tx[4 * i + 2], tx[4 * i + 3]);
  }
}

template <int CL, int LAYOUT>
__device__ __forceinline__ void decode_task(ESmem& sm, const EStage& sg, int b, int kind) {
  uint32_t tx[16];
  class_block<CL>(sg, b, kind, tx, &sm.S, sm.ep[threadIdx.x]);
  tile_store<LAYOUT>(sm.tile, b, tx);
}

// stream holding group g: the last stream starting at or before g (streams are back to back)
__device__ __forceinline__ int stream_at(const DevTable& T, int64_t g) {
  int si = 0;
#pragma unroll 1
  for (int i = 1; i < T.n_streams; i++) si += (T.first_group[i] <= g) ? 1 : 0;
  return si;
}

// Issues the copies of tile `tile` into stage `sg`. TMA: one thread, completing on `bar`;
// otherwise every thread copies its own blocks (b = threadIdx.x + i * E_NT) and, without TMA,
// a share of the slot entries and positions.
template <int KIND>
__device__ __forceinline__ void stage_issue(const EArgs& a, EStage& sg, unsigned long long* bar, int64_t tile) {
  const DevTable& T = a.T;
  const int64_t g0 = tile * E_TG;
  const int vg = (int)min((int64_t)E_TG, (int64_t)T.n_groups - g0);
  const int64_t s0 = g0 * 16;
  const int vs = vg * 16;
  const bool tma = a.tma != 0;
  if (tma && threadIdx.x == 0) {
    fence_proxy_async();
    uint32_t bytes = (uint32_t)vs * 4u;
    if (a.pos_slot) bytes += (uint32_t)vs * 12u;
    if (KIND == 7) bytes += (uint32_t)vg * 256u;
    if (KIND == 1) bytes += (uint32_t)vg * 128u;
    mbar_expect_tx(bar, bytes);
    bulk_g2s(sg.perm, a.perm + s0, (uint32_t)vs * 4u, bar);
    if (a.pos_slot) bulk_g2s(sg.pos, a.pos_slot + s0 * 3, (uint32_t)vs * 12u, bar);
    if (KIND == 7) bulk_g2s(sg.blk, a.blocks + g0 * 256, (uint32_t)vg * 256u, bar);
    if (KIND == 1) bulk_g2s(sg.blk, a.blocks + g0 * 128, (uint32_t)vg * 128u, bar);
  }
  if (!tma) {
    for (int s = threadIdx.x; s < vs; s += E_NT) {
      cp_async4(&sg.perm[s], a.perm + s0 + s);
      if (a.pos_slot) {
        const float* src = a.pos_slot + (s0 + s) * 3;
        cp_async4(&sg.pos[3 * s], src);
        cp_async4(&sg.pos[3 * s + 1], src + 1);
        cp_async4(&sg.pos[3 * s + 2], src + 2);
      }
    }
  }
  if (KIND == 0 || !tma) {
#pragma unroll
    for (int i = 0; i < 2; i++) {
      const int b = threadIdx.x + i * E_NT;
      if (b >= vs) continue;
      const int64_t g = g0 + (b >> 4);
      const int k = b & 15;
      if (KIND == 7) {
        const uint8_t* src = a.blocks + (g * 16 + k) * 16;
        cp_async8(&sg.blk[b], src);
        cp_async8(reinterpret_cast<uint2*>(&sg.blk[b]) + 1, src + 8);
      } else if (KIND == 1) {
        cp_async8(reinterpret_cast<uint2*>(sg.blk) + b, a.blocks + (g * 16 + k) * 8);
      } else {
        const int si = stream_at(T, g);
        const int nb = T.bands[si], j = T.bc7[si];
        const int64_t base = T.byte_offset[si] + (g - T.first_group[si]) * (int64_t)(16 * j + 8 * (nb - j));
        uint8_t c = 0;  // 0 dropped, 1 BC1, 7 BC7
        if (k < nb) {
          if (lay_bc7(T.layout, j, k)) {
            const uint8_t* src = a.blocks + base + 16 * lay_rank(T.layout, j, k);
            cp_async8(&sg.blk[b], src);
            cp_async8(reinterpret_cast<uint2*>(&sg.blk[b]) + 1, src + 8);
            c = 7;
          } else {
            cp_async8(&sg.blk[b], a.blocks + base + 16 * j + 8 * lay_rank(T.layout, j, k));
            c = 1;
          }
        }
        sg.cls[b] = c;
      }
    }
  }
  cp_async_commit();
}

__device__ __forceinline__ int bc7_class_of(uint32_t w) {
  const uint32_t b0 = w & 0xFFu;
  if (!b0) return CL_RES;
  const int m = __ffs(b0) - 1;
  return (m == 4 && ((w >> 7) & 1u)) ? CL_M4S : m;
}

// class of the block b this thread staged, appended to the class lists
template <int KIND>
__device__ __forceinline__ void classify(ESmem& sm, const EStage& sg, int cur, int b, bool valid) {
  int cl = 0;
  if (valid) {
    if (KIND == 7) cl = bc7_class_of(sg.blk[b].x);
    else if (KIND == 1) cl = CL_BC1;
    else {
      const int c = sg.cls[b];
      cl = c == 7 ? bc7_class_of(sg.blk[b].x) : (c == 1 ? CL_BC1 : CL_DROP);
    }
  }
  const unsigned act = __ballot_sync(0xFFFFFFFFu, valid);
  if (!valid) return;
  const unsigned peers = __match_any_sync(act, cl);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(&sm.cnt[cur][cl], __popc(peers));
  base = __shfl_sync(peers, base, leader);
  const int rank = __popc(peers & ((1u << lane) - 1u));
  sm.list[cl][base + rank] = (uint16_t)b;
}

template <int KIND, int LAYOUT>
__device__ __forceinline__ void decode_tile(ESmem& sm, const EStage& sg, int cur) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // task j of the tile: chunk (j - first task of class cl) of class cl's list, 32 blocks a chunk
  int ntask = 0;
#pragma unroll
  for (int c = 0; c < E_NCLS; c++) ntask += (sm.cnt[cur][c] + 31) >> 5;
  for (int j = warp; j < ntask; j += E_NW) {
    int cl = 0, first = 0, nc = 0;
    bool found = false;
#pragma unroll
    for (int c = 0; c < E_NCLS; c++) {
      const int cc = sm.cnt[cur][c], tasks = (cc + 31) >> 5;
      if (!found) {
        if (j < first + tasks) { found = true; cl = c; nc = cc; }
        else first += tasks;
      }
    }
    const int idx = (j - first) * 32 + lane;
    if (!found || idx >= nc) continue;
    const int b = sm.list[cl][idx];
    if (b >= E_T) continue;  // never: lists hold tile block indices
    if (KIND == 1) {
      decode_task<CL_BC1, LAYOUT>(sm, sg, b, KIND);
      continue;
    }
    switch (cl) {
      case 0: decode_task<0, LAYOUT>(sm, sg, b, KIND); break;
      case 1: decode_task<1, LAYOUT>(sm, sg, b, KIND); break;
      case 2: decode_task<2, LAYOUT>(sm, sg, b, KIND); break;
      case 3: decode_task<3, LAYOUT>(sm, sg, b, KIND); break;
      case 4: decode_task<4, LAYOUT>(sm, sg, b, KIND); break;
      case 5: decode_task<5, LAYOUT>(sm, sg, b, KIND); break;
      case 6: decode_task<6, LAYOUT>(sm, sg, b, KIND); break;
      case 7: decode_task<7, LAYOUT>(sm, sg, b, KIND); break;
      case CL_M4S: decode_task<CL_M4S, LAYOUT>(sm, sg, b, KIND); break;
      case CL_RES: decode_task<CL_RES, LAYOUT>(sm, sg, b, KIND); break;
      case CL_BC1: decode_task<CL_BC1, LAYOUT>(sm, sg, b, KIND); break;
      default: decode_task<CL_DROP, LAYOUT>(sm, sg, b, KIND); break;
    }
  }
}

// Decoded texels of two slots -> dequantised coefficient pairs (slot A in .x, slot B in .y)
// with the SH constants folded in: x = fl(fl(2^23 + q - (2^23 + 128)) * f_k).
__device__ __forceinline__ void dequant_pair(const ESmem& sm, int ra, int rb, float2 (&xr)[16], float2 (&xg)[16],
                                             float2 (&xb)[16]) {
  const float2 m = make_float2(-8388736.0f, -8388736.0f);
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const uint4 ta = *reinterpret_cast<const uint4*>(sm.tile + ra + 4 * q);
    const uint4 tb = *reinterpret_cast<const uint4*>(sm.tile + rb + 4 * q);
    const uint32_t va[4] = {ta.x, ta.y, ta.z, ta.w}, vb[4] = {tb.x, tb.y, tb.z, tb.w};
#pragma unroll
    for (int i = 0; i < 4; i++) {
      const int k = 4 * q + i;
      const float2 f = sm.deq[k];
      xr[k] = __fmul2_rn(__fadd2_rn(make_float2(u23(va[i], 0), u23(vb[i], 0)), m), f);
      xg[k] = __fmul2_rn(__fadd2_rn(make_float2(u23(va[i], 1), u23(vb[i], 1)), m), f);
      xb[k] = __fmul2_rn(__fadd2_rn(make_float2(u23(va[i], 2), u23(vb[i], 2)), m), f);
    }
  }
}

// colour of view v for the two Gaussians (np*: negated positions, A in .x, B in .y)
template <bool CAMS>
__device__ __forceinline__ void eval_view_pair(const ESmem& sm, int v, float2 npx, float2 npy, float2 npz,
                                               const float2 (&xr)[16], const float2 (&xg)[16], const float2 (&xb)[16],
                                               float2& ar, float2& ag, float2& ab) {
  const float4 cxy = sm.cxy[v];
  float2 dx = make_float2(cxy.x, cxy.y), dy = make_float2(cxy.z, cxy.w), dz = sm.cz[v];
  if (CAMS) { dx = __fadd2_rn(dx, npx); dy = __fadd2_rn(dy, npy); dz = __fadd2_rn(dz, npz); }
  const float2 n2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
  float2 r;
  r.x = n2.x > 0.f ? rsqrtf(n2.x) : 0.f;
  r.y = n2.y > 0.f ? rsqrtf(n2.y) : 0.f;
  dx = __fmul2_rn(dx, r); dy = __fmul2_rn(dy, r); dz = __fmul2_rn(dz, r);
  if (n2.x <= 0.f) dz.x = 1.f;
  if (n2.y <= 0.f) dz.y = 1.f;
  float2 P[16];
  sh_poly2(dx, dy, dz, P);
  ar = xr[0]; ag = xg[0]; ab = xb[0];
#pragma unroll
  for (int k = 1; k < 16; k++) {
    ar = __ffma2_rn(xr[k], P[k], ar);
    ag = __ffma2_rn(xg[k], P[k], ag);
    ab = __ffma2_rn(xb[k], P[k], ab);
  }
}

// Checked build: a slot entry outside [-1, n) is recorded and treated as an empty slot.
__device__ __forceinline__ int32_t e_checked(const EArgs& a, int32_t o, int64_t s) {
#ifdef GSC_CHECKED
  if (o < -1 || (int64_t)o >= (int64_t)a.T.n) {
    eval_record((int)GSC_ERR_DEVICE, (int)(s < 0x7FFFFFFF ? s : 0x7FFFFFFF));
    return -1;
  }
#else
  (void)a; (void)s;
#endif
  return o;
}

template <bool CAMS>
__device__ __forceinline__ void eval_tile(const EArgs& a, const ESmem& sm, const EStage& sg, int64_t tile) {
  const DevTable& T = a.T;
  const int64_t g0 = tile * E_TG;
  const int vs = (int)min((int64_t)E_TG, (int64_t)T.n_groups - g0) * 16;
  const int sa = threadIdx.x, sb = threadIdx.x + E_NT;  // tile slots of Gaussians A and B
  if (sa >= vs) return;
  const bool vb = sb < vs;
  const int64_t s0 = g0 * 16;
  const int64_t n = T.n, ns = (int64_t)T.n_groups * 16;
  const int32_t oa = e_checked(a, sg.perm[sa], s0 + sa);
  const int32_t ob = vb ? e_checked(a, sg.perm[sb], s0 + sb) : -1;
  const int V = a.V, order = a.out_order;
  if (oa < 0 && ob < 0) {
    if (order == GSC_OUT_SLOT_ORDER)
      for (int v = 0; v < V; v++) {
        float* d = a.rgb + ((int64_t)v * ns + s0 + sa) * 3;
        d[0] = d[1] = d[2] = 0.f;
        if (vb) { d += (int64_t)E_NT * 3; d[0] = d[1] = d[2] = 0.f; }
      }
    return;
  }
  float2 npx = make_float2(0.f, 0.f), npy = npx, npz = npx;
  if (CAMS) {
    float3 pa = make_float3(0.f, 0.f, 0.f), pb = pa;
    if (a.pos_slot) {
      pa = make_float3(sg.pos[3 * sa], sg.pos[3 * sa + 1], sg.pos[3 * sa + 2]);
      if (vb) pb = make_float3(sg.pos[3 * sb], sg.pos[3 * sb + 1], sg.pos[3 * sb + 2]);
    } else {
      if (oa >= 0) pa = make_float3(__ldg(a.pos + 3 * (int64_t)oa), __ldg(a.pos + 3 * (int64_t)oa + 1), __ldg(a.pos + 3 * (int64_t)oa + 2));
      if (ob >= 0) pb = make_float3(__ldg(a.pos + 3 * (int64_t)ob), __ldg(a.pos + 3 * (int64_t)ob + 1), __ldg(a.pos + 3 * (int64_t)ob + 2));
    }
    npx = make_float2(-pa.x, -pb.x); npy = make_float2(-pa.y, -pb.y); npz = make_float2(-pa.z, -pb.z);
  }
  float2 xr[16], xg[16], xb[16];
  dequant_pair(sm, (sa >> 4) * E_GRP + (sa & 15) * E_ROW, (sb >> 4) * E_GRP + (sb & 15) * E_ROW, xr, xg, xb);
  const bool gm4 = order == GSC_OUT_GAUSS_MAJOR && (V & 3) == 0;
  for (int v0 = 0; v0 < V; v0 += 4) {
    float ra[12], rb[12];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      if (v0 + q < V) {
        float2 cr, cg, cb;
        eval_view_pair<CAMS>(sm, v0 + q, npx, npy, npz, xr, xg, xb, cr, cg, cb);
        ra[3 * q] = cr.x; ra[3 * q + 1] = cg.x; ra[3 * q + 2] = cb.x;
        rb[3 * q] = cr.y; rb[3 * q + 1] = cg.y; rb[3 * q + 2] = cb.y;
      }
    }
    if (gm4) {
      if (oa >= 0) {
        float4* d = reinterpret_cast<float4*>(a.rgb + ((int64_t)oa * V + v0) * 3);
        d[0] = make_float4(ra[0], ra[1], ra[2], ra[3]);
        d[1] = make_float4(ra[4], ra[5], ra[6], ra[7]);
        d[2] = make_float4(ra[8], ra[9], ra[10], ra[11]);
      }
      if (ob >= 0) {
        float4* d = reinterpret_cast<float4*>(a.rgb + ((int64_t)ob * V + v0) * 3);
        d[0] = make_float4(rb[0], rb[1], rb[2], rb[3]);
        d[1] = make_float4(rb[4], rb[5], rb[6], rb[7]);
        d[2] = make_float4(rb[8], rb[9], rb[10], rb[11]);
      }
    } else {
      const int nv = V - v0 < 4 ? V - v0 : 4;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int32_t o = h ? ob : oa;
        const int64_t s = s0 + (h ? sb : sa);
        if (h && !vb) continue;
        const float* r = h ? rb : ra;
        if (o < 0) {
          if (order == GSC_OUT_SLOT_ORDER)
            for (int q = 0; q < nv; q++) {
              float* d = a.rgb + ((int64_t)(v0 + q) * ns + s) * 3;
              d[0] = d[1] = d[2] = 0.f;
            }
          continue;
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
          if (q >= nv) break;
          float* d;
          if (order == GSC_OUT_GAUSS_MAJOR) d = a.rgb + ((int64_t)o * V + v0 + q) * 3;
          else if (order == GSC_OUT_VIEW_MAJOR) d = a.rgb + ((int64_t)(v0 + q) * n + o) * 3;
          else d = a.rgb + ((int64_t)(v0 + q) * ns + s) * 3;
          d[0] = r[3 * q]; d[1] = r[3 * q + 1]; d[2] = r[3 * q + 2];
        }
      }
    }
  }
}

template <int KIND, bool CAMS, int LAYOUT>
__global__ void __launch_bounds__(E_NT, 2) k_eval3(EArgs a) {
  extern __shared__ __align__(128) uint8_t e_raw[];
  ESmem& sm = *reinterpret_cast<ESmem*>(e_raw);
  const DevTable& T = a.T;
  load_tables(&sm.S);
  for (int i = threadIdx.x; i < a.V; i += E_NT) {
    const float* src = a.cams ? a.cams : a.dirs;
    const float x = src[3 * i], y = src[3 * i + 1], z = src[3 * i + 2];
    sm.cxy[i] = make_float4(x, x, y, y);
    sm.cz[i] = make_float2(z, z);
  }
  if (threadIdx.x < 16) {
    const float f = __fmul_rn(__fdiv_rn(T.scales[threadIdx.x], 255.0f), c_shc[threadIdx.x]);
    sm.deq[threadIdx.x] = make_float2(f, f);
  }
  if (threadIdx.x < 2 * E_NCLS) sm.cnt[threadIdx.x / E_NCLS][threadIdx.x % E_NCLS] = 0;
  if (threadIdx.x == 0) {
    mbar_init(&sm.mbar[0], 1);
    mbar_init(&sm.mbar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const int64_t n_tiles = ((int64_t)T.n_groups + E_TG - 1) / E_TG;
  int64_t tile = blockIdx.x;
  if (tile < n_tiles) stage_issue<KIND>(a, sm.stage[0], &sm.mbar[0], tile);
  uint32_t parity = 0u;  // bit st: parity of the next completion of stage st's barrier
  for (int it = 0; tile < n_tiles; tile += gridDim.x, it++) {
    const int st = it & 1, cur = it & 1;
    EStage& sg = sm.stage[st];
    cp_async_wait_all();
    if (a.tma) {
      uint32_t spins = 0;
      while (!mbar_try(&sm.mbar[st], (parity >> st) & 1u)) {
        if (++spins > E_WAIT_LIMIT) {
          if (threadIdx.x == 0) eval_record((int)GSC_ERR_TIMEOUT, (int)blockIdx.x);
          return;
        }
      }
    }
    parity ^= 1u << st;
    const int vs = (int)min((int64_t)E_TG, (int64_t)T.n_groups - tile * E_TG) * 16;
    classify<KIND>(sm, sg, cur, threadIdx.x, (int)threadIdx.x < vs);
    classify<KIND>(sm, sg, cur, threadIdx.x + E_NT, (int)threadIdx.x + E_NT < vs);
    __syncthreads();
    // the other stage was last read by the previous tile's evaluation, finished before the barrier
    const int64_t next = tile + gridDim.x;
    if (next < n_tiles) stage_issue<KIND>(a, sm.stage[st ^ 1], &sm.mbar[st ^ 1], next);
    // counters of the next tile: last read by the previous tile's decode, before this tile's barrier
    if (threadIdx.x < E_NCLS) sm.cnt[cur ^ 1][threadIdx.x] = 0;
    decode_tile<KIND, LAYOUT>(sm, sg, cur);
    __syncthreads();
    eval_tile<CAMS>(a, sm, sg, tile);
  }
  // nothing is left in flight: a tile's copies are issued only when that tile will be processed
}

template <int KIND, bool CAMS, int LAYOUT>
cudaError_t set_attr() {
  return cudaFuncSetAttribute(k_eval3<KIND, CAMS, LAYOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(ESmem));
}

template <bool CAMS, int LAYOUT>
cudaError_t set_attr_kinds() {
  cudaError_t e = set_attr<7, CAMS, LAYOUT>();
  if (e == cudaSuccess) e = set_attr<1, CAMS, LAYOUT>();
  if (e == cudaSuccess) e = set_attr<0, CAMS, LAYOUT>();
  return e;
}

int kind_of3(const DevTable& T) {
  if (T.n_streams == 1 && T.bands[0] == 16 && T.byte_offset[0] == 0) return T.bc7[0] == 16 ? 7 : (T.bc7[0] == 0 ? 1 : 0);
  return 0;
}

}  // namespace

cudaError_t eval3_init() {
  cudaError_t e = cudaSuccess;
  const int layouts[3] = {GSC_LAYOUT_D, GSC_LAYOUT_A, GSC_LAYOUT_B};
  for (int i = 0; i < 3 && e == cudaSuccess; i++) {
    const int L = layouts[i];
    if (L == GSC_LAYOUT_D) { e = set_attr_kinds<true, GSC_LAYOUT_D>(); if (e == cudaSuccess) e = set_attr_kinds<false, GSC_LAYOUT_D>(); }
    if (L == GSC_LAYOUT_A) { e = set_attr_kinds<true, GSC_LAYOUT_A>(); if (e == cudaSuccess) e = set_attr_kinds<false, GSC_LAYOUT_A>(); }
    if (L == GSC_LAYOUT_B) { e = set_attr_kinds<true, GSC_LAYOUT_B>(); if (e == cudaSuccess) e = set_attr_kinds<false, GSC_LAYOUT_B>(); }
  }
  if (e == cudaSuccess) e = dec_tables_upload();
  return e;
}

size_t eval3_smem_bytes() { return sizeof(ESmem); }

int eval3_err_take(int* where) {
  int h[2] = {0, 0};
  if (cudaMemcpyFromSymbol(h, g_eval_err, sizeof(h)) != cudaSuccess) { cudaGetLastError(); return 0; }
  if (h[0]) {
    const int z[2] = {0, 0};
    cudaMemcpyToSymbol(g_eval_err, z, sizeof(z));
  }
  if (where) *where = h[1];
  return h[0];
}

static bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

cudaError_t launch_eval3(const DevTable& T, const uint8_t* blocks, const int32_t* perm, const float* dirs,
                         const float* pos, const float* pos_slot, const float* cams, int V, int out_order, float* rgb,
                         int sm_count, cudaStream_t st) {
  if (T.n_groups == 0) return cudaSuccess;
  EArgs a;
  a.T = T;
  a.blocks = blocks;
  a.perm = perm;
  a.pos = pos;
  a.pos_slot = pos_slot;
  a.dirs = dirs;
  a.cams = cams;
  a.rgb = rgb;
  a.V = V;
  a.out_order = out_order;
  const int kind = kind_of3(T);
  a.tma = (al16(perm) && (!pos_slot || al16(pos_slot)) && (kind == 0 || al16(blocks))) ? 1 : 0;
  const int64_t n_tiles = ((int64_t)T.n_groups + E_TG - 1) / E_TG;
  const int64_t cap = (int64_t)(sm_count > 0 ? sm_count : 1) * 2;
  const int grid = (int)(n_tiles < cap ? n_tiles : cap);
  const size_t smem = sizeof(ESmem);
#define E3_LAUNCH(K, C, L) k_eval3<K, C, L><<<grid, E_NT, smem, st>>>(a)
#define E3_KINDS(C, L)                                                                 \
  do {                                                                                 \
    if (kind == 7) E3_LAUNCH(7, C, L); else if (kind == 1) E3_LAUNCH(1, C, L); else E3_LAUNCH(0, C, L); \
  } while (0)
#define E3_LAYOUTS(C)                                                                  \
  do {                                                                                 \
    if (T.layout == GSC_LAYOUT_A) E3_KINDS(C, GSC_LAYOUT_A);                           \
    else if (T.layout == GSC_LAYOUT_B) E3_KINDS(C, GSC_LAYOUT_B);                      \
    else E3_KINDS(C, GSC_LAYOUT_D);                                                    \
  } while (0)
  gsc_count_launch();
  if (cams) E3_LAYOUTS(true);
  else E3_LAYOUTS(false);
#undef E3_LAYOUTS
#undef E3_KINDS
#undef E3_LAUNCH
  return cudaGetLastError();
}

// Positions in slot order: out[s] = pos[perm[s]] (zeros for padding slots).
__global__ void k_pos_to_slots(const float* __restrict__ pos, const int32_t* __restrict__ perm, int64_t n, int64_t ns,
                               float* __restrict__ out) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
    int32_t o = perm[s];
#ifdef GSC_CHECKED
    if (o < -1 || (int64_t)o >= n) {
      eval_record((int)GSC_ERR_DEVICE, (int)(s < 0x7FFFFFFF ? s : 0x7FFFFFFF));
      o = -1;
    }
#endif
    (void)n;
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
