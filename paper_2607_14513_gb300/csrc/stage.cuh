// stage.cuh -- layout-D tile staging shared by the group encoders (Sec. IV-B, Fig. SetupD).
//
// A CTA of 128 threads owns 8 groups = 128 slots = 128 blocks. Thread i loads slot i
// (group i / 16, texel i % 16): the Gaussian perm[slot] (a padding slot repeats the
// group's last valid slot before it; none -> texel 128), its 48 floats as 12
// 16-byte loads, quantises them (Sec. V-A) and scatters coefficient k into block
// (group, k). Texels are packed r | g << 8 | b << 16 in smem tex[t][block]; the row
// stride of 129 words keeps both the scatter and the per-block reads conflict-free.
#pragma once
#include "gsc_internal.cuh"

#define STAGE_GROUPS 8
#define STAGE_THREADS 128
#define STAGE_STRIDE 129

// i: the thread's index inside its 128-thread staging unit (a multiple of 32 apart from
// threadIdx.x, so the warp-level ballots below see the same lanes)
__device__ __forceinline__ void stage_groups(const float* __restrict__ sh, const int32_t* __restrict__ perm,
                                             const float* s_scale, int64_t g0, int64_t n_groups,
                                             uint32_t (*tex)[STAGE_STRIDE], int i) {
  const int lg = i >> 4, t = i & 15;
  const int64_t g = g0 + lg;
  const bool live = g < n_groups;
  int32_t o = live ? __ldg(perm + g * 16 + t) : -1;
  // last valid slot at or before t inside this half-warp's group
  const unsigned half = 0xFFFFu << (threadIdx.x & 16);
  unsigned valid = __ballot_sync(0xFFFFFFFFu, o >= 0) & half;
  unsigned upto = valid & (0xFFFFFFFFu >> (31 - (threadIdx.x & 31)));
  int src_lane = upto ? 31 - __clz(upto) : -1;
  int32_t src = __shfl_sync(0xFFFFFFFFu, o, src_lane < 0 ? (threadIdx.x & 31) : src_lane);
  if (src_lane < 0) src = -1;
  const int col = lg * 16;
  if (src < 0) {
#pragma unroll
    for (int k = 0; k < 16; k++) tex[t][col + k] = 128u | (128u << 8) | (128u << 16);
    return;
  }
  const float4* p = reinterpret_cast<const float4*>(sh + (int64_t)src * 48);
  float v[48];
#pragma unroll
  for (int j = 0; j < 12; j++) {
    float4 f = __ldg(p + j);
    v[4 * j + 0] = f.x; v[4 * j + 1] = f.y; v[4 * j + 2] = f.z; v[4 * j + 3] = f.w;
  }
#pragma unroll
  for (int k = 0; k < 16; k++) {
    float s = s_scale[k];
    uint32_t r = gsc_quant1(v[3 * k + 0], s), gg = gsc_quant1(v[3 * k + 1], s), b = gsc_quant1(v[3 * k + 2], s);
    tex[t][col + k] = r | (gg << 8) | (b << 16);
  }
}

__device__ __forceinline__ int tex_r(uint32_t v) { return v & 255; }
__device__ __forceinline__ int tex_g(uint32_t v) { return (v >> 8) & 255; }
__device__ __forceinline__ int tex_b(uint32_t v) { return (v >> 16) & 255; }

// Exact clamp(round_div(num, den), 0, 255) for den > 0, round_div rounding half away from zero,
// for several numerators over one denominator: a negative numerator clamps to 0; otherwise
// floor((2num + den) / (2den)) is estimated in float with one reciprocal of 2den per
// denominator and corrected exactly in 64-bit integers. The quotient is below 256 and the
// conversions, the reciprocal and the product carry a relative error of a few 2^-24, so the
// estimate's floor is off by at most one and one exact step each way lands on it.
struct RoundDiv255 {
  long long D;  // 2 den
  float rcp;    // 1 / D, rounded
};
__device__ __forceinline__ RoundDiv255 round_div255_of(long long den) {
  RoundDiv255 r;
  r.D = 2 * den;
  r.rcp = __frcp_rn((float)r.D);
  return r;
}
__device__ __forceinline__ int round_div255(const RoundDiv255& r, long long num) {
  if (num < 0) return 0;
  const long long N = 2 * num + r.D / 2;
  if (N >= 256 * r.D) return 255;
  int q = (int)((float)N * r.rcp);
  q = min(max(q, 0), 255);
  if (q > 0 && (long long)q * r.D > N) q--;
  if (q < 255 && (long long)(q + 1) * r.D <= N) q++;
  return q;
}

