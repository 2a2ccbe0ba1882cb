// eval.cu -- fused decode + SH evaluation of a coded scene, tiled through shared memory
// (Sec. I: random access by block index x block size; Sec. II: c(f) = H w(f - p);
// Sec. III-B: BC1 / BC7 formats; Sec. IV-B: block layouts and fixed-rate streams).
//
// One persistent CTA per SM, warp-specialised, works through tiles of E_TG groups (E_T slots,
// E_T blocks) held in a ring of E_NS shared-memory slots:
//  - producer warps (E_PW): stage the tile's blocks into the slot (TMA bulk copy completing on an
//    mbarrier, E_NS tiles ahead; per-thread cp.async for rate streams and unaligned blocks),
//    give every block a class -- BC7 mode 0..7 (mode 4 split by its index-selection bit), the
//    reserved BC7 mode, BC1, or a coefficient the stream drops -- and decode the blocks 32 of one
//    class at a time with that class's own decoder (field positions, widths and subset counts are
//    compile-time constants) into a Gaussian-major tile (slot row, coefficient column);
//  - consumer warps (E_CW): evaluate two Gaussians per thread from the decoded tile; the two share
//    each packed FP32x2 operation lane for lane (coefficients, directions, bases, accumulators),
//    so no operand is broadcast, and per (Gaussian, view) the operations are those of the
//    single-Gaussian evaluation in decode.cu, in the same order: the colours are bit-identical.
// Producers and consumers hand slots over through mbarriers (tile full / tile empty), so the
// integer-heavy decode of one tile runs beside the floating-point evaluation of another.
#include <stddef.h>

#include "bc7_class.cuh"
#include "decode_dev.cuh"
#include "layout.cuh"

namespace {

constexpr int E_PW = 8;                  // producer warps (two warpgroups)
constexpr int E_CW = 8;                  // consumer warps (two warpgroups)
// registers per thread: launched with 128, producers give some up and consumers take them
// (E_PT * E_PREG + E_CT * E_CREG must not exceed E_NT * 128)
constexpr int E_PREG = 88, E_CREG = 168;
constexpr int E_PT = 32 * E_PW;          // producer threads
constexpr int E_CT = 32 * E_CW;          // consumer threads
constexpr int E_NT = E_PT + E_CT;        // threads per CTA
constexpr int E_T = 2 * E_CT;            // slots (and blocks) per tile: two Gaussians per consumer thread
constexpr int E_TG = E_T / 16;           // groups per tile
constexpr int E_NS = 3;                  // tiles in flight (ring slots)
constexpr int E_ROW = 20;                // tile words per slot row (16 coefficients + 4 to spread banks)
constexpr int E_GRP = 16 * E_ROW + 4;    // tile words per group
constexpr int E_NCLS = 12;
constexpr int E_MAXV = 64;
// bounded waits on the ring's barriers: far beyond any copy's or tile's latency
constexpr uint32_t E_WAIT_LIMIT = 1u << 22;
constexpr int E_PBAR = 1;                // named barrier of the producer warps

struct ESlot {
  uint4 blk[E_T];                  // BC7 blocks (16 B), or BC1 blocks (8 B, packed from the start: all-BC1 codings)
  int32_t perm[E_T];               // slot entries of the tile
  float pos[E_T * 3];              // slot-ordered centres of the tile (when given in slot order)
  uint8_t cls[E_T];                // rate streams: format of each block as located (BC7 / BC1 / dropped)
  uint32_t tile[E_TG * E_GRP];     // decoded texels, Gaussian-major
};

struct ESmem {
  ESlot slot[E_NS];
  uint16_t list[E_NCLS][E_T];
  int cnt[2][E_NCLS];
  alignas(64) uint4 ep[E_PT][4];   // per-lane endpoint / palette slots (64-byte aligned)
  float4 cxy[E_MAXV];              // per view (x, x, y, y) of the camera centre or direction
  float2 cz[E_MAXV];               // (z, z)
  float2 deq[16];                  // (f_k, f_k), f_k = s_k / 255 * C_k
  float2 deqF[16], deqC[16];       // (f_k 2^133, f_k 2^133) and (-128 f_k, -128 f_k): one-FMA dequantisation
  int ffma_deq;                    // every f_k 2^133 finite: the one-FMA form applies
  DecTables S;
  unsigned long long blk_full[E_NS], tile_full[E_NS], tile_empty[E_NS];
};

static_assert(sizeof(ESlot) % 16 == 0 && offsetof(ESlot, tile) % 16 == 0 && offsetof(ESlot, perm) % 16 == 0 &&
                  offsetof(ESlot, pos) % 16 == 0, "TMA destinations and tile rows");
static_assert((E_GRP * 4) % 16 == 0 && (E_ROW * 4) % 16 == 0, "tile rows");
static_assert(sizeof(ESmem) <= 227 * 1024, "shared memory of one CTA");
static_assert(E_PT * E_PREG + E_CT * E_CREG <= E_NT * 128, "register split within the launch's registers");
static_assert(E_PW % 4 == 0 && E_CW % 4 == 0, "setmaxnreg acts on whole warpgroups");
static_assert(offsetof(ESmem, ep) % 64 == 0, "palette slots are addressed by OR-ing a 6-bit offset");

struct EArgs {
  DevTable T;
  const uint8_t* blocks;
  const int32_t* perm;
  const float* pos;       // original order [n][3], or null
  const float* pos_slot;  // slot order [n_groups * 16][3], or null
  const float* dirs;
  const float* cams;
  float* rgb;
  int V, out_order;
  int tma_blk;   // blocks staged by TMA (16-byte aligned, one format)
  int tma_meta;  // slot entries and slot-ordered centres staged by TMA (16-byte aligned)
};

// First error this translation unit's kernels detected (code, where): a slot entry outside
// [-1, n) in the checked build, or a ring barrier that never completed. Taken by gsc_ctx_sync.
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

template <int CL>
__device__ __forceinline__ void class_block(const ESlot& sg, int b, int kind, uint32_t (&tx)[16], const DecTables* S,
                                            uint4* ep) {
  if (CL <= CL_M4S) {
    const uint4 w = sg.blk[b];
    bc7_class_block<CL>(((uint64_t)w.y << 32) | w.x, ((uint64_t)w.w << 32) | w.z, tx, S, ep);
  } else if (CL == CL_BC1) {
    const uint2 w = kind == 1 ? reinterpret_cast<const uint2*>(sg.blk)[b] : make_uint2(sg.blk[b].x, sg.blk[b].y);
    bc1_class_block(w, tx, ep);
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
__device__ __forceinline__ void decode_task(ESmem& sm, ESlot& sg, int b, int kind) {
  uint32_t tx[16];
  class_block<CL>(sg, b, kind, tx, &sm.S, sm.ep[threadIdx.x]);
  tile_store<LAYOUT>(sg.tile, b, tx);
}

// Decoded texels of two slots -> dequantised coefficient pairs (slot A in .x, slot B in .y)
// with the SH constants folded in, x = fl((q - 128) f_k). Two exact ways to the same bits:
// fl(fl(2^23 + q - (2^23 + 128)) f_k), or, when f_k 2^133 is finite, one fused multiply-add
// fma(q 2^-133, f_k 2^133, -128 f_k): q placed in bits 16..23 of a float is exactly q 2^-133
// (subnormal below q = 128, the smallest normal exponent from there on), the product is exact
// inside the FMA and -128 f_k is exact, so the single rounding gives fl((q - 128) f_k).
__device__ __forceinline__ void dequant_pair(const ESmem& sm, const uint32_t* tile, int ra, int rb, float2 (&xr)[16],
                                             float2 (&xg)[16], float2 (&xb)[16]) {
  const bool one_fma = sm.ffma_deq != 0;
  const float2 m = make_float2(-8388736.0f, -8388736.0f);
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const uint4 ta = *reinterpret_cast<const uint4*>(tile + ra + 4 * q);
    const uint4 tb = *reinterpret_cast<const uint4*>(tile + rb + 4 * q);
    const uint32_t va[4] = {ta.x, ta.y, ta.z, ta.w}, vb[4] = {tb.x, tb.y, tb.z, tb.w};
#pragma unroll
    for (int i = 0; i < 4; i++) {
      const int k = 4 * q + i;
      if (one_fma) {
        const float2 F = sm.deqF[k], C = sm.deqC[k];
#define QF(v, c) __uint_as_float(__byte_perm(v, 0u, 0x4044u | ((c) << 8)))
        xr[k] = __ffma2_rn(make_float2(QF(va[i], 0), QF(vb[i], 0)), F, C);
        xg[k] = __ffma2_rn(make_float2(QF(va[i], 1), QF(vb[i], 1)), F, C);
        xb[k] = __ffma2_rn(make_float2(QF(va[i], 2), QF(vb[i], 2)), F, C);
#undef QF
      } else {
        const float2 f = sm.deq[k];
        xr[k] = __fmul2_rn(__fadd2_rn(make_float2(u23(va[i], 0), u23(vb[i], 0)), m), f);
        xg[k] = __fmul2_rn(__fadd2_rn(make_float2(u23(va[i], 1), u23(vb[i], 1)), m), f);
        xb[k] = __fmul2_rn(__fadd2_rn(make_float2(u23(va[i], 2), u23(vb[i], 2)), m), f);
      }
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


// ---- ring synchronisation ---------------------------------------------------------------------
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
// waits (bounded) for the completion of the barrier phase with the given parity
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, uint32_t parity) {
  uint32_t spins = 0;
  while (!mbar_try(b, parity))
    if (++spins > E_WAIT_LIMIT) return false;
  return true;
}
// barrier of the producer warps that also tells every producer whether all of them passed their
// waits (a timed-out wait makes all producers stop together)
__device__ __forceinline__ bool producers_sync_all(bool ok) {
  uint32_t r;
  asm volatile(
      "{ .reg .pred p, q; setp.ne.u32 p, %1, 0; bar.red.and.pred q, %2, %3, p; selp.u32 %0, 1, 0, q; }"
      : "=r"(r)
      : "r"((uint32_t)ok), "n"(E_PBAR), "n"(E_PT)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void producers_sync() { asm volatile("bar.sync %0, %1;" ::"n"(E_PBAR), "n"(E_PT) : "memory"); }

// stream holding group g: the last stream starting at or before g (streams are back to back)
__device__ __forceinline__ int stream_at(const DevTable& T, int64_t g) {
  int si = 0;
#pragma unroll 1
  for (int i = 1; i < T.n_streams; i++) si += (T.first_group[i] <= g) ? 1 : 0;
  return si;
}

__device__ __forceinline__ int tile_slots(const DevTable& T, int64_t tile) {
  return (int)min((int64_t)E_TG, (int64_t)T.n_groups - tile * E_TG) * 16;
}

// Producers: copies of tile `tile` (if it exists) into slot `sg`: its blocks, slot entries and,
// when centres come in slot order, its centres. TMA: producer thread 0 issues bulk copies
// completing on `bar`; otherwise producer threads copy with cp.async, each its own blocks
// (b = ptid + i * E_PT: the blocks it will classify). Every call commits one cp.async group.
template <int KIND>
__device__ __forceinline__ void stage_tile(const EArgs& a, ESlot& sg, unsigned long long* bar, int64_t tile,
                                           int64_t n_tiles, int ptid) {
  const DevTable& T = a.T;
  if (tile < n_tiles) {
    const int64_t g0 = tile * E_TG, s0 = g0 * 16;
    const int vs = tile_slots(T, tile), vg = vs >> 4;
    const bool tblk = KIND != 0 && a.tma_blk != 0, tmeta = a.tma_meta != 0;
    if ((tblk || tmeta) && ptid == 0) {
      fence_proxy_async();
      const uint32_t bb = tblk ? (uint32_t)vg * (KIND == 7 ? 256u : 128u) : 0u;
      const uint32_t pb = tmeta ? (uint32_t)vs * 4u : 0u, qb = tmeta && a.pos_slot ? (uint32_t)vs * 12u : 0u;
      mbar_expect_tx(bar, bb + pb + qb);
      if (tblk) bulk_g2s(sg.blk, a.blocks + g0 * (KIND == 7 ? 256 : 128), bb, bar);
      if (pb) bulk_g2s(sg.perm, a.perm + s0, pb, bar);
      if (qb) bulk_g2s(sg.pos, a.pos_slot + s0 * 3, qb, bar);
    }
    if (!tmeta) {
      for (int u = ptid; u < vs; u += E_PT) {
        cp_async4(&sg.perm[u], a.perm + s0 + u);
        if (a.pos_slot) {
          const float* src = a.pos_slot + (s0 + u) * 3;
          cp_async4(&sg.pos[3 * u], src);
          cp_async4(&sg.pos[3 * u + 1], src + 1);
          cp_async4(&sg.pos[3 * u + 2], src + 2);
        }
      }
    }
    if (!tblk) {
      for (int b = ptid; b < vs; b += E_PT) {
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
  }
  cp_async_commit();
}

__device__ __forceinline__ int bc7_class_of(uint32_t w) {
  const uint32_t b0 = w & 0xFFu;
  if (!b0) return CL_RES;
  const int m = __ffs(b0) - 1;
  return (m == 4 && ((w >> 7) & 1u)) ? CL_M4S : m;
}

// class of block b of the slot, appended to the class lists (warp-aggregated)
template <int KIND>
__device__ __forceinline__ void classify(ESmem& sm, const ESlot& sg, int cur, int b, bool valid) {
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

// Producer warp `pw` decodes its share of the slot's blocks: classes in order, each class's list
// in chunks of 32, chunk j of the whole sequence going to warp j % E_PW.
template <int KIND, int LAYOUT, int CL>
__device__ __forceinline__ void decode_class(ESmem& sm, ESlot& sg, int cur, int pw, int lane, int& first) {
  const int cc = sm.cnt[cur][CL], tasks = (cc + 31) >> 5;
  if (tasks == 0) return;
  const int r = first % E_PW;
  for (int j = (pw >= r ? pw - r : pw + E_PW - r); j < tasks; j += E_PW) {
    const int idx = j * 32 + lane;
    if (idx < cc) {
      const int b = sm.list[CL][idx];
      if (b < E_T) decode_task<CL, LAYOUT>(sm, sg, b, KIND);
    }
  }
  first += tasks;
}

template <int KIND, int LAYOUT>
__device__ __forceinline__ void decode_slot(ESmem& sm, ESlot& sg, int cur, int pw, int lane) {
  int first = 0;
  if (KIND == 1) {
    decode_class<KIND, LAYOUT, CL_BC1>(sm, sg, cur, pw, lane, first);
    return;
  }
  decode_class<KIND, LAYOUT, 0>(sm, sg, cur, pw, lane, first);
  decode_class<KIND, LAYOUT, 1>(sm, sg, cur, pw, lane, first);
  decode_class<KIND, LAYOUT, 2>(sm, sg, cur, pw, lane, first);
  decode_class<KIND, LAYOUT, 3>(sm, sg, cur, pw, lane, first);
  decode_class<KIND, LAYOUT, 4>(sm, sg, cur, pw, lane, first);
  decode_class<KIND, LAYOUT, 5>(sm, sg, cur, pw, lane, first);
  decode_class<KIND, LAYOUT, 6>(sm, sg, cur, pw, lane, first);
  decode_class<KIND, LAYOUT, 7>(sm, sg, cur, pw, lane, first);
  decode_class<KIND, LAYOUT, CL_M4S>(sm, sg, cur, pw, lane, first);
  decode_class<KIND, LAYOUT, CL_RES>(sm, sg, cur, pw, lane, first);
  if (KIND == 0) {
    decode_class<KIND, LAYOUT, CL_BC1>(sm, sg, cur, pw, lane, first);
    decode_class<KIND, LAYOUT, CL_DROP>(sm, sg, cur, pw, lane, first);
  }
}

template <int KIND, int LAYOUT>
__device__ void producer(ESmem& sm, const EArgs& a, int64_t n_tiles) {
  const int ptid = threadIdx.x, pw = ptid >> 5, lane = ptid & 31;
  const DevTable& T = a.T;
  const bool tma = (KIND != 0 && a.tma_blk != 0) || a.tma_meta != 0;
  // the first E_NS tiles of this CTA
  for (int i = 0; i < E_NS; i++)
    stage_tile<KIND>(a, sm.slot[i], &sm.blk_full[i], (int64_t)blockIdx.x + (int64_t)i * gridDim.x, n_tiles, ptid);
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, it++) {
    const int s = it % E_NS, use = it / E_NS, cur = it & 1;
    ESlot& sg = sm.slot[s];
    const int vs = tile_slots(T, tile);
    // this thread's copies of the tile (the E_NS - 1 newer groups may stay in flight)
    asm volatile("cp.async.wait_group %0;" ::"n"(E_NS - 1) : "memory");
    bool ok = true;
    if (tma) ok = mbar_wait(&sm.blk_full[s], (uint32_t)use & 1u);
    if (!producers_sync_all(ok)) {
      if (ptid == 0) eval_record((int)GSC_ERR_TIMEOUT, (int)blockIdx.x);
      return;
    }
    for (int b = ptid; b < E_PT * ((E_T + E_PT - 1) / E_PT); b += E_PT) classify<KIND>(sm, sg, cur, b, b < vs);
    // counters of the next tile: last read by the previous tile's decode, before this tile's barriers
    if (ptid < E_NCLS) sm.cnt[cur ^ 1][ptid] = 0;
    // the slot's tile is free once the consumers released its previous use
    ok = use == 0 || mbar_wait(&sm.tile_empty[s], (uint32_t)(use - 1) & 1u);
    if (!producers_sync_all(ok)) {
      if (ptid == 0) eval_record((int)GSC_ERR_TIMEOUT, (int)blockIdx.x);
      return;
    }
    decode_slot<KIND, LAYOUT>(sm, sg, cur, pw, lane);
    producers_sync();
    if (ptid == 0) mbar_arrive(&sm.tile_full[s]);
    // the slot's blocks are decoded: stage the tile E_NS ahead into it
    stage_tile<KIND>(a, sg, &sm.blk_full[s], tile + (int64_t)E_NS * gridDim.x, n_tiles, ptid);
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}


// slot entry and centre of tile slot `u`, from the staged slot (centres in original order are
// gathered through the slot entry)
struct ESlotIn {
  int32_t o;
  float px, py, pz;
};

template <bool CAMS>
__device__ __forceinline__ ESlotIn slot_in(const EArgs& a, const ESlot& sg, int64_t tile, int u) {
  ESlotIn r;
  r.o = -1;
  r.px = r.py = r.pz = 0.f;
  if (u >= tile_slots(a.T, tile)) return r;
  r.o = e_checked(a, sg.perm[u], tile * E_T + u);
  if (CAMS) {
    if (a.pos_slot) {
      r.px = sg.pos[3 * u]; r.py = sg.pos[3 * u + 1]; r.pz = sg.pos[3 * u + 2];
    } else if (r.o >= 0) {
      const float* p = a.pos + 3 * (int64_t)r.o;
      r.px = __ldg(p); r.py = __ldg(p + 1); r.pz = __ldg(p + 2);
    }
  }
  return r;
}

// VF > 0: exactly VF views into Gaussian-major rows, known at compile time.
template <bool CAMS, int VF>
__device__ __forceinline__ void eval_slot_pair(const EArgs& a, const ESmem& sm, const uint32_t* tile, int64_t tile_i,
                                               int sa, int sb, const ESlotIn& A, const ESlotIn& B) {
  const DevTable& T = a.T;
  const int vs = tile_slots(T, tile_i);
  if (sa >= vs) return;
  const bool vb = sb < vs;
  const int64_t s0 = tile_i * E_T;
  const int64_t n = T.n, ns = (int64_t)T.n_groups * 16;
  const int32_t oa = A.o, ob = vb ? B.o : -1;
  const int V = VF > 0 ? VF : a.V, order = VF > 0 ? (int)GSC_OUT_GAUSS_MAJOR : a.out_order;
  if (oa < 0 && ob < 0) {
    if (order == GSC_OUT_SLOT_ORDER)
      for (int v = 0; v < V; v++) {
        float* d = a.rgb + ((int64_t)v * ns + s0 + sa) * 3;
        d[0] = d[1] = d[2] = 0.f;
        if (vb) { d += (int64_t)(sb - sa) * 3; d[0] = d[1] = d[2] = 0.f; }
      }
    return;
  }
  const float2 npx = make_float2(-A.px, -B.px), npy = make_float2(-A.py, -B.py), npz = make_float2(-A.pz, -B.pz);
  float2 xr[16], xg[16], xb[16];
  dequant_pair(sm, tile, (sa >> 4) * E_GRP + (sa & 15) * E_ROW, (sb >> 4) * E_GRP + (sb & 15) * E_ROW, xr, xg, xb);
  const bool gm4 = order == GSC_OUT_GAUSS_MAJOR && (V & 3) == 0;
#pragma unroll
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

template <bool CAMS, int VF>
__device__ void consumer(ESmem& sm, const EArgs& a, int64_t n_tiles) {
  const int ctid = threadIdx.x - E_PT, lane = threadIdx.x & 31;
  const int sa = ctid, sb = ctid + E_CT;  // tile slots of this thread's two Gaussians
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, it++) {
    const int s = it % E_NS, use = it / E_NS;
    const bool ok = __all_sync(0xFFFFFFFFu, mbar_wait(&sm.tile_full[s], (uint32_t)use & 1u));
    if (!ok) {
      if (lane == 0) eval_record((int)GSC_ERR_TIMEOUT, (int)blockIdx.x);
      return;
    }
    const ESlot& sg = sm.slot[s];
    const ESlotIn A = slot_in<CAMS>(a, sg, tile, sa), B = slot_in<CAMS>(a, sg, tile, sb);
    eval_slot_pair<CAMS, VF>(a, sm, sg.tile, tile, sa, sb, A, B);
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.tile_empty[s]);
  }
}

template <int KIND, bool CAMS, int LAYOUT, int VF>
__global__ void __launch_bounds__(E_NT, 1) k_eval4(EArgs a) {
  static_assert(E_NT == 512, "128 registers per thread at launch");
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
  bool fma_ok = true;
  if (threadIdx.x < 16) {
    const float f = __fmul_rn(__fdiv_rn(T.scales[threadIdx.x], 255.0f), c_shc[threadIdx.x]);
    sm.deq[threadIdx.x] = make_float2(f, f);
    const float F = __fmul_rn(__fmul_rn(f, 18446744073709551616.0f), 590295810358705651712.0f);  // f 2^64 2^69
    const float C = __fmul_rn(f, -128.0f);
    sm.deqF[threadIdx.x] = make_float2(F, F);
    sm.deqC[threadIdx.x] = make_float2(C, C);
    fma_ok = fabsf(f) < 0.03125f;  // f 2^133 < 2^128
  }
  if (threadIdx.x < 2 * E_NCLS) sm.cnt[threadIdx.x / E_NCLS][threadIdx.x % E_NCLS] = 0;
  if (threadIdx.x < E_NS) {
    mbar_init(&sm.blk_full[threadIdx.x], 1);
    mbar_init(&sm.tile_full[threadIdx.x], 1);
    mbar_init(&sm.tile_empty[threadIdx.x], E_CW);
  }
  if (threadIdx.x == 0) fence_mbar_init();
  const int all_ok = __syncthreads_and(fma_ok);
  if (threadIdx.x == 0) sm.ffma_deq = all_ok;
  __syncthreads();
  const int64_t n_tiles = ((int64_t)T.n_groups + E_TG - 1) / E_TG;
  if (threadIdx.x < E_PT) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(E_PREG));
    producer<KIND, LAYOUT>(sm, a, n_tiles);
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(E_CREG));
    consumer<CAMS, VF>(sm, a, n_tiles);
  }
}

template <int KIND, bool CAMS, int LAYOUT, int VF>
cudaError_t set_attr() {
  return cudaFuncSetAttribute(k_eval4<KIND, CAMS, LAYOUT, VF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(ESmem));
}

template <bool CAMS, int LAYOUT>
cudaError_t set_attr_kinds() {
  cudaError_t e = set_attr<7, CAMS, LAYOUT, 0>();
  if (e == cudaSuccess) e = set_attr<1, CAMS, LAYOUT, 0>();
  if (e == cudaSuccess) e = set_attr<0, CAMS, LAYOUT, 0>();
  if (LAYOUT == GSC_LAYOUT_D) {
    if (e == cudaSuccess) e = set_attr<7, CAMS, LAYOUT, 8>();
    if (e == cudaSuccess) e = set_attr<1, CAMS, LAYOUT, 8>();
    if (e == cudaSuccess) e = set_attr<0, CAMS, LAYOUT, 8>();
  }
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
  a.tma_blk = al16(blocks) ? 1 : 0;  // rate streams always take per-thread copies
  a.tma_meta = (al16(perm) && (!pos_slot || al16(pos_slot))) ? 1 : 0;
  const int64_t n_tiles = ((int64_t)T.n_groups + E_TG - 1) / E_TG;
  const int64_t cap = (int64_t)(sm_count > 0 ? sm_count : 1);
  const int grid = (int)(n_tiles < cap ? n_tiles : cap);
  const size_t smem = sizeof(ESmem);
  // 8 views into Gaussian-major rows (the camera-pose workload): a compile-time view count
  const bool v8 = V == 8 && out_order == GSC_OUT_GAUSS_MAJOR && T.layout == GSC_LAYOUT_D;
#define E3_LAUNCH(K, C, L)                                                              \
  do {                                                                                 \
    if (L == GSC_LAYOUT_D && v8) k_eval4<K, C, GSC_LAYOUT_D, 8><<<grid, E_NT, smem, st>>>(a); \
    else k_eval4<K, C, L, 0><<<grid, E_NT, smem, st>>>(a);                             \
  } while (0)
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

