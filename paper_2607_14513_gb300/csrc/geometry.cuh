// geometry.cuh -- fixed-rate geometry streams and the chunk hierarchy (Sec. IV-A: position and
// shape coded apart from appearance, each parameter quantised to a fixed number of bits in its
// own bitstream; a hierarchy lets a view use only the primitives of the part it sees).
//
// Streams in slot order (positions move with the Gaussians, so no index is stored), 17 bytes per
// slot: position 3 x 16 bits over the box of the slot's chunk (C consecutive slots), scale 3 x
// bfloat16, rotation as the smallest three of the unit quaternion (2-bit index of the largest
// component, made non-negative, then three 10-bit codes of 1022 steps over [-1/sqrt2, 1/sqrt2]),
// opacity logit 8 bits over [-8, 8]. Per chunk: the box of its centres and its largest decoded
// scale. Every quantiser and decoder is a fixed order of correctly rounded float operations, so
// codes and decoded values are the same bits in every implementation.
#pragma once
#include "gsc_internal.cuh"

struct GeomStreams {
  uint16_t* qpos;    // [n_slots][3]
  uint16_t* qscale;  // [n_slots][3]
  uint32_t* qrot;    // [n_slots]
  uint8_t* qlogit;   // [n_slots]
  gsc_chunk* chunk;  // [n_chunks]
};

// Byte offsets of the streams inside one buffer (each 256-byte aligned).
__host__ __device__ inline size_t geom_align(size_t v) { return (v + 255) / 256 * 256; }
inline size_t geom_bytes(int64_t ns, int64_t chunk_slots, size_t* off /*[5] or null*/) {
  const int64_t nc = (ns + chunk_slots - 1) / chunk_slots;
  size_t o[5], b = 0;
  o[0] = b; b = geom_align(b + 6 * (size_t)ns);
  o[1] = b; b = geom_align(b + 6 * (size_t)ns);
  o[2] = b; b = geom_align(b + 4 * (size_t)ns);
  o[3] = b; b = geom_align(b + (size_t)ns);
  o[4] = b; b = geom_align(b + sizeof(gsc_chunk) * (size_t)(nc > 0 ? nc : 1));
  if (off) for (int i = 0; i < 5; i++) off[i] = o[i];
  return b;
}
inline GeomStreams geom_streams(uint8_t* base, int64_t ns, int64_t chunk_slots) {
  size_t o[5];
  geom_bytes(ns, chunk_slots, o);
  GeomStreams g;
  g.qpos = reinterpret_cast<uint16_t*>(base + o[0]);
  g.qscale = reinterpret_cast<uint16_t*>(base + o[1]);
  g.qrot = reinterpret_cast<uint32_t*>(base + o[2]);
  g.qlogit = base + o[3];
  g.chunk = reinterpret_cast<gsc_chunk*>(base + o[4]);
  return g;
}

__device__ __forceinline__ float gm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float ga(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float gs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float gd(float a, float b) { return __fdiv_rn(a, b); }

// bfloat16 with round to nearest even (finite values)
__device__ __forceinline__ uint16_t bf16_rne(float x) {
  uint32_t u = __float_as_uint(x);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
__device__ __forceinline__ float bf16_val(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

// round(t * levels) with t clamped to [0, 1], half to even
__device__ __forceinline__ uint32_t quant_unit(float t, float levels) {
  const float c = t < 0.0f ? 0.0f : (t > 1.0f ? 1.0f : t);
  return (uint32_t)rintf(gm(c, levels));
}

// Decoded geometry of slot s.
__device__ __forceinline__ void geom_decode(const GeomStreams& G, int64_t s, int64_t chunk_slots, float3& p, float3& sc,
                                            float4& q, float& t) {
  const gsc_chunk e = G.chunk[s / chunk_slots];
  const uint16_t* qp = G.qpos + 3 * s;
  const float lo[3] = {e.lo[0], e.lo[1], e.lo[2]}, hi[3] = {e.hi[0], e.hi[1], e.hi[2]};
  float pv[3];
#pragma unroll
  for (int a = 0; a < 3; a++) pv[a] = ga(lo[a], gm(gd((float)qp[a], 65535.0f), gs(hi[a], lo[a])));
  p = make_float3(pv[0], pv[1], pv[2]);
  const uint16_t* qs = G.qscale + 3 * s;
  sc = make_float3(bf16_val(qs[0]), bf16_val(qs[1]), bf16_val(qs[2]));
  const uint32_t code = G.qrot[s];
  const int m = (int)(code & 3u);
  float c3[3], ss = 0.0f;
#pragma unroll
  for (int j = 0; j < 3; j++) {
    c3[j] = gm(gs(gd((float)((code >> (2 + 10 * j)) & 1023u), 1022.0f), 0.5f), 1.41421356f);
    ss = ga(ss, gm(c3[j], c3[j]));
  }
  const float r = gs(1.0f, ss);
  const float qm = __fsqrt_rn(r > 0.0f ? r : 0.0f);
  float qv[4];
#pragma unroll
  for (int a = 0; a < 4; a++) qv[a] = a < m ? c3[a < 3 ? a : 2] : (a == m ? qm : c3[a > 0 ? a - 1 : 0]);
  q = make_float4(qv[0], qv[1], qv[2], qv[3]);
  t = gs(gm(gd((float)G.qlogit[s], 255.0f), 16.0f), 8.0f);
}
